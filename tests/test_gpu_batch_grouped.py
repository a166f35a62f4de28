"""GPU tests of the grouped batch: every stage of the step as one launch over the work of all
systems (persistent tcgen05 exchange and VHS kernels over a (system, spin block, tile) work list,
the propagation over every walker, the per-walker kernels over every walker).

The grouped form runs the arithmetic of the systems' own steps except for the exchange, which it
always takes in the streamed form (also for the force bias of steps without an energy measurement),
so it is compared with the per-system graphs to the rounding of that contraction, and with the
oracle in tests/test_gpu_forms_vs_oracle.py."""
import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from paper_2406_16238_b300._lib import Batch
from synthetic_inputs import make_problem

pytestmark = pytest.mark.gpu


def _systems():
    """Four uneven systems: RHF and UHF, two in the N <= 128 propagation form (operand widths 8 and
    16 columns), two in the large form (N > 128, packed L^T)."""
    return [make_problem(40, 6, 6, 120, 10.0, 501, orthogonalise=False, scf_iterations=0),
            make_problem(70, 9, 7, 210, 15.0, 502, unrestricted=True, orthogonalise=False, scf_iterations=0),
            make_problem(136, 12, 12, 300, 30.0, 503, orthogonalise=False, scf_iterations=0),
            make_problem(150, 14, 11, 320, 30.0, 504, unrestricted=True, orthogonalise=False, scf_iterations=0)]


def _contexts(probs, prec, nw=16):
    return [pkg.Afqmc(p.h1e, p.chol, p.ecore, p.nalpha, p.nbeta, p.psiT, nwalkers=nw, dt=0.005, seed=900 + i,
                      prec=prec) for i, p in enumerate(probs)]


def _run(probs, prec, mode, nsteps=11, groups=0, zero=None, branches=0, et_out=None):
    ctxs = _contexts(probs, prec)
    if et_out is not None:   # E_T follows the running estimate
        for c in ctxs:
            c.set_etrial_update(True)
    if zero is not None:   # walkers of weight zero are frozen (skipped by every grouped kernel)
        for c in ctxs:
            psi, _, w, step = c.get_walkers()
            w = w.copy()
            w[zero] = 0.0
            c.set_walkers(psi, w, step)
    b = Batch(ctxs, mode=mode, exch_groups=groups, branches=branches)
    assert b.mode() == mode
    e = b.run(nsteps, energy_every=1, reortho_every=3, comb_every=5)
    walkers = [c.get_walkers() for c in ctxs]
    if et_out is not None:
        et_out.extend(c.e_trial for c in ctxs)
    b.close()
    for c in ctxs:
        c.close()
    return e, walkers


@pytest.fixture(scope="module")
def systems():
    return _systems()


@pytest.mark.parametrize("prec,tol,branches", [("bf16x3", 2e-5, 2), ("bf16x3", 2e-5, 1), ("bf16", 2e-4, 0)])
def test_grouped_launches_agree_with_per_system_graphs(systems, prec, tol, branches):
    """11 steps with energy every step, QR every 3 and comb every 5 (so the steps after a comb
    rebuild the bf16 Theta operands): mixed energies, weights and step counters; one branch of
    grouped launches, or two side by side."""
    eg, wg = _run(systems, prec, "grouped", branches=branches)
    er, wr = _run(systems, prec, "graphs")
    assert eg.shape == er.shape == (4, 11, 4)
    assert np.all(np.isfinite(eg))
    d = np.abs(eg[:, :, 0] / eg[:, :, 1] - er[:, :, 0] / er[:, :, 1])
    assert np.max(d) < tol, d
    for (pg, _, w_g, sg), (pr, _, w_r, sr) in zip(wg, wr):
        assert sg == sr == 11
        assert np.allclose(w_g, w_r, rtol=50 * tol, atol=0)


def test_grouped_exchange_warpgroup_counts_agree(systems):
    """One, two and four epilogue warpgroups per exchange tile give the same trajectory to rounding."""
    out = [_run(systems, "bf16x3", "grouped", nsteps=4, groups=g)[0] for g in (1, 2, 4)]
    for e in out[1:]:
        assert np.max(np.abs(e[:, :, 0] / e[:, :, 1] - out[0][:, :, 0] / out[0][:, :, 1])) < 1e-5


def test_grouped_skips_frozen_walkers(systems):
    """Walkers of weight zero stay as they are, and the others follow the per-system graphs."""
    zero = [1, 5, 6, 15]
    eg, wg = _run(systems, "bf16x3", "grouped", nsteps=4, zero=zero)
    er, wr = _run(systems, "bf16x3", "graphs", nsteps=4, zero=zero)
    assert np.max(np.abs(eg[:, :, 0] / eg[:, :, 1] - er[:, :, 0] / er[:, :, 1])) < 2e-5
    for (psi_g, _, w_g, _), (psi_r, _, w_r, _) in zip(wg, wr):
        assert np.all(w_g[zero] == 0.0) and np.all(w_r[zero] == 0.0)
        assert np.array_equal(psi_g[zero], psi_r[zero])


def test_grouped_form_needs_one_tensor_core_form():
    probs = _systems()[:2]
    ctxs = [pkg.Afqmc(probs[0].h1e, probs[0].chol, probs[0].ecore, probs[0].nalpha, probs[0].nbeta, probs[0].psiT,
                      nwalkers=8, prec="fp32"),
            pkg.Afqmc(probs[1].h1e, probs[1].chol, probs[1].ecore, probs[1].nalpha, probs[1].nbeta, probs[1].psiT,
                      nwalkers=8, prec="bf16x3")]
    b = Batch(ctxs)
    assert b.mode() == "graphs"   # auto falls back to the per-system graphs
    b.set_mode("grouped")
    with pytest.raises(pkg.AfqmcError, match="tensor-core form"):
        b.run(1)
    b.close()
    for c in ctxs:
        c.close()


def test_grouped_steps_without_energy_and_uneven_cadence(systems):
    """Energy every third step, QR every 4, comb every 6: the grouped steps without an energy
    measurement form the force bias with the grouped exchange (the per-system graphs with a CUDA-core
    product), so the two agree to rounding; the step counters and measurement counts match."""
    def run(mode):
        ctxs = _contexts(systems[:3], "bf16x3")
        b = Batch(ctxs, mode=mode)
        e = b.run(13, energy_every=3, reortho_every=4, comb_every=6)
        steps = [c.get_walkers()[3] for c in ctxs]
        b.close()
        for c in ctxs:
            c.close()
        return e, steps
    eg, sg = run("grouped")
    er, sr = run("graphs")
    assert eg.shape == er.shape == (3, 5, 4) and sg == sr == [13, 13, 13]
    assert np.max(np.abs(eg[:, :, 0] / eg[:, :, 1] - er[:, :, 0] / er[:, :, 1])) < 2e-5


def test_complex_and_free_projection_contexts_batch_as_graphs():
    from synthetic_inputs import make_complex_problem
    pc = make_complex_problem(10, 3, 2, 6, 3.0, 72, unrestricted=True)
    pr = _systems()[0]
    ctxs = [pkg.Afqmc(pc.h1e, pc.chol, pc.ecore, pc.nalpha, pc.nbeta, pc.psiT, nwalkers=8, prec="bf16x3"),
            pkg.Afqmc(pr.h1e, pr.chol, pr.ecore, pr.nalpha, pr.nbeta, pr.psiT, nwalkers=8, prec="bf16x3")]
    b = Batch(ctxs)
    assert b.mode() == "graphs"   # a complex Hamiltonian: the per-system graphs
    e = b.run(3, energy_every=1, reortho_every=5, comb_every=0)
    assert np.all(np.isfinite(e))
    b.close()
    for c in ctxs:
        c.close()
    c1, c2 = [pkg.Afqmc(pr.h1e, pr.chol, pr.ecore, pr.nalpha, pr.nbeta, pr.psiT, nwalkers=8, prec="bf16x3")
              for _ in range(2)]
    c2.set_free_projection(True)
    b = Batch([c1, c2])
    assert b.mode() == "graphs"   # free projection: the per-system graphs
    e = b.run(2, energy_every=1, reortho_every=5, comb_every=0)
    assert np.all(np.isfinite(e))
    b.close()
    for c in (c1, c2):
        c.close()


def test_grouped_trial_energy_update(systems):
    """E_T following the running estimate in grouped launches agrees with the per-system graphs
    (each system's own sums and comb), and moves off E_var."""
    etg, etr = [], []
    eg, wg = _run(systems, "bf16x3", "grouped", et_out=etg)
    er, wr = _run(systems, "bf16x3", "graphs", et_out=etr)
    assert np.max(np.abs(eg[:, :, 0] / eg[:, :, 1] - er[:, :, 0] / er[:, :, 1])) < 2e-5
    for (_, _, w_g, _), (_, _, w_r, _) in zip(wg, wr):
        assert np.allclose(w_g, w_r, rtol=1e-3, atol=0)
    for a, b, e in zip(etg, etr, er):
        assert abs(a - b) < 2e-5
        mix = np.sum(e[:10, 0]) / np.sum(e[:10, 1])   # the last comb, after step 10 (comb every 5)
        assert abs(b - mix) < 1e-9 * abs(mix)
