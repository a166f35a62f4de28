"""Every arithmetic form of the CUDA path against the FP64 oracle at the benchmark shape, and
uneven batched systems against the oracle.

The oracle (oracle/afqmc.py, binary64) and the library draw the same Philox fields, so the
trajectories differ only by the arithmetic of the contractions.  The reduced forms are held
to the stated horizon tolerances (reading (a) of the reduced-precision target: the same
walkers and fields, no comb, 10 steps, |E_form - E_oracle| per step):

* FP64: 1e-10 relative (binary64 everywhere, sums in another order);
* FP32 and BF16x3: 0.1 mHa.  FP32 contractions round each product to 2^-24 and BF16x3 keeps
  ~16 significant bits per split product (the lo*lo term dropped, fp32 accumulation), so a
  per-walker two-body energy of a few Ha carries errors of order 2^-16 * |E2| ~ 1e-4 Ha at
  worst, and the weighted mean over 64 walkers averages the independent per-walker errors;
* BF16: 1 mHa (8 significant bits per operand).
"""
import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from oracle import afqmc as orc
from synthetic_inputs import config_medium, make_problem

pytestmark = pytest.mark.gpu

HORIZON_TOL = {"fp32": 1e-4, "bf16x3": 1e-4, "bf16": 1e-3}
NW, NSTEPS, SEED = 64, 10, 240616241


@pytest.fixture(scope="module")
def benchmark_shape_reference():
    """The oracle's 10-step trajectory on the benchmark Hamiltonian (N=108, 21+21, naux=432, RHF),
    64 walkers, dt = 0.005, energy every step, QR every 5, no comb."""
    prob = config_medium()
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, 0.005)
    hist, wk = orc.run_phaseless(st, prob.psiT, NW, NSTEPS, SEED, reortho_every=5, comb_every=0, energy_every=1)
    return prob, st, hist, wk


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "bf16"])
def test_every_form_tracks_the_oracle_at_the_benchmark_shape(benchmark_shape_reference, prec):
    prob, st, hist, wk = benchmark_shape_reference
    ctx = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=NW, dt=0.005,
                    seed=SEED, prec=prec)
    e = ctx.run(NSTEPS, energy_every=1, reortho_every=5, comb_every=0)
    psi_g, _, w_g, step = ctx.get_walkers()
    ctx.close()
    assert step == NSTEPS and e.shape == hist.shape == (NSTEPS, 4)
    eg, er = e[:, 0] / e[:, 1], hist[:, 0] / hist[:, 1]
    if prec == "fp64":
        assert np.max(np.abs(eg - er) / np.abs(er)) < 1e-10
        assert np.allclose(e[:, 1], hist[:, 1], rtol=1e-10, atol=0)
        assert np.allclose(w_g, wk.w, rtol=1e-10, atol=0)
        assert np.allclose(psi_g, wk.psi, rtol=0, atol=1e-10)
        return
    d = np.abs(eg - er)
    assert np.max(d) <= HORIZON_TOL[prec], d
    # the weights follow the oracle's to the accuracy of the log-overlap ratios (the common factor
    # exp(dt (E_T - E_c)) differs between the forms by the form's own E_var, so compare ratios)
    r = (w_g / wk.w) / np.mean(w_g / wk.w)
    assert np.max(np.abs(r - 1.0)) < (1e-4 if prec != "bf16" else 1e-2)


def _batch_problems():
    """Three uneven restricted systems, n = N/6 per spin, naux = 4N (the batched workload's recipe), the
    largest with N = 210."""
    out = []
    for i, n in enumerate((30, 90, 210)):
        nocc = n // 6
        out.append(make_problem(n, nocc, nocc, 4 * n, 0.4 * n, 240617000 + i, orthogonalise=False,
                                scf_iterations=0, name=f"batch_N{n}"))
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_uneven_batch_tracks_the_oracle(prec):
    """One graph launch per step over three uneven systems (N = 30, 90, 210; BF16x3: one launch per
    stage over all three, N = 210 in the large propagation form): each system's mixed energy over 6
    steps (QR every 5, no comb) against the oracle's trajectory on the same fields."""
    from paper_2406_16238_b300._lib import Batch
    probs = _batch_problems()
    nw, nsteps = 8, 6
    seeds = [71, 72, 73]
    ctxs = [pkg.Afqmc(p.h1e, p.chol, p.ecore, p.nalpha, p.nbeta, p.psiT, nwalkers=nw, dt=0.005, seed=s, prec=prec)
            for p, s in zip(probs, seeds)]
    b = Batch(ctxs, mode="graphs" if prec == "fp32" else "grouped")   # tensor-core forms: grouped launches
    assert b.mode() == ("graphs" if prec == "fp32" else "grouped")
    e = b.run(nsteps, energy_every=1, reortho_every=5, comb_every=0)
    b.close()
    for c in ctxs:
        c.close()
    assert e.shape == (3, nsteps, 4)
    for i, (p, s) in enumerate(zip(probs, seeds)):
        st = orc.build_setup(p.h1e, p.chol, p.ecore, p.nalpha, p.nbeta, p.psiT, 0.005)
        hist, _ = orc.run_phaseless(st, p.psiT, nw, nsteps, s, reortho_every=5, comb_every=0, energy_every=1)
        d = np.abs(e[i, :, 0] / e[i, :, 1] - hist[:, 0] / hist[:, 1])
        assert np.max(d) <= HORIZON_TOL[prec], (p.name, d)
