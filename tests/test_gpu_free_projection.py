"""GPU free projection (Section "Free projection AFQMC") against the FP64 oracle and exact diagonalisation.

Free projection keeps the mean-field subtraction, draws unshifted fields (xbar = 0) and carries
complex weights w e^{i phi} = prod (O'/O) e^{c_mf} e^{dt (E_T - E_c)}; there is no phaseless
projection and no comb.  The estimator is Re(sum w e^{i phi} E_L / sum w e^{i phi}).
"""
import math

import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from oracle import afqmc as orc
from oracle import fci
from synthetic_inputs import config_medium, config_small, make_problem, random_walkers, tiny_problem

pytestmark = pytest.mark.gpu


def _ctx(prob, nw, prec="fp64", seed=5, dt=0.005, **kw):
    return pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, dt=dt,
                     seed=seed, prec=prec, **kw)


def _restricted(prob):
    return prob.nalpha == prob.nbeta and np.array_equal(prob.psiT[:, :prob.nalpha], prob.psiT[:, prob.nalpha:])


def _random_state(prob, nw, seed, spread=0.2):
    rng = np.random.default_rng(seed)
    if _restricted(prob):
        half = random_walkers(rng, prob.norb, prob.nalpha, nw, spread, prob.psiT[:, :prob.nalpha])
        psi = np.concatenate([half, half], axis=2)
    else:
        psi = random_walkers(rng, prob.norb, prob.nalpha + prob.nbeta, nw, spread, prob.psiT)
    return psi, rng.uniform(0.5, 1.5, nw)


def _complex_sums(st, psi, wc):
    num, den = 0.0 + 0.0j, 0.0 + 0.0j
    for i in range(psi.shape[0]):
        _, th_a, th_b = orc.overlap_theta(st, psi[i])
        e = orc.local_energy(st, th_a, th_b)[0]
        num += wc[i] * e
        den += wc[i]
    return np.array([num.real, num.imag, den.real, den.imag])


PROBLEMS = {
    "rhf_N8": lambda: config_small(),
    "uhf_N13_3_2": lambda: make_problem(13, 3, 2, 17, 5.0, 31, unrestricted=True),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_free_projection_trajectory_matches_oracle(name):
    """12 free-projection steps with QR every 5 (FP64): walkers, complex weights and the complex
    estimator sums against the oracle's free-projection step on identical Philox fields."""
    prob = PROBLEMS[name]()
    nw, seed, dt, step0 = 8, 4242, 0.01, 17
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, dt)
    ctx = _ctx(prob, nw, seed=seed, dt=dt)
    psi, w = _random_state(prob, nw, seed=2)
    ctx.set_walkers(psi, w, step0)
    ctx.set_free_projection(True)
    logo = np.array([orc.overlap_theta(st, p)[0] for p in psi])
    wc = w.astype(complex)
    psi_o = psi.copy()
    for s in range(12):
        ctx.propagate(1)
        x_g, xbar_g = ctx.get_fields()
        x = orc.free_projection_step(st, psi_o, logo, wc, seed, step0 + s, e_trial=st.evar)
        assert np.array_equal(x_g.view(np.uint64), x.view(np.uint64))
        assert np.all(xbar_g == 0)
        if (s + 1) % 5 == 0:
            ctx.reortho()
            orc.reorthogonalise(st, orc.Walkers(psi_o, logo, np.abs(wc), step0 + s + 1))
    psi_g, logo_g, w_g, step = ctx.get_walkers()
    ph_g = ctx.weight_phases()
    assert step == step0 + 12
    assert np.allclose(psi_g, psi_o, rtol=0, atol=1e-10)
    assert np.allclose(logo_g.real, logo.real, rtol=1e-10, atol=1e-10)
    assert np.all(np.abs(np.angle(np.exp(1j * (logo_g.imag - logo.imag)))) < 1e-9)
    wc_g = w_g * np.exp(1j * ph_g)
    assert np.allclose(wc_g, wc, rtol=1e-10, atol=0)
    assert np.all(np.abs(ph_g) <= math.pi)
    assert np.max(np.abs(np.angle(wc))) > 1e-3     # the phases are genuinely non-trivial
    sums = ctx.local_energy()
    ref = _complex_sums(st, psi_o, wc)
    assert np.allclose(sums, ref, rtol=1e-10, atol=1e-10 * np.max(np.abs(ref)))


def test_free_projection_rules():
    """No comb in free projection; phases reset when switching; back to phaseless sums afterwards."""
    prob = config_small()
    ctx = _ctx(prob, 16, seed=3)
    ctx.set_free_projection(True)
    ctx.propagate(3)
    assert np.any(ctx.weight_phases() != 0)
    with pytest.raises(pkg.AfqmcError):
        ctx.popcontrol()
    with pytest.raises(pkg.AfqmcError):
        ctx.run(10, energy_every=1, reortho_every=5, comb_every=10)
    ctx.set_free_projection(False)
    assert np.all(ctx.weight_phases() == 0)
    sums = ctx.local_energy()
    _, _, w, _ = ctx.get_walkers()
    assert sums[1] == pytest.approx(np.sum(w), rel=1e-14)     # EDenom again
    e = ctx.run(10, energy_every=1, reortho_every=5, comb_every=10)   # phaseless with comb
    assert np.all(np.isfinite(e))


@pytest.mark.parametrize("prec,nw", [("fp64", 16), ("fp32", 16), ("bf16x3", 24)])
def test_free_projection_graph_replay_is_bit_identical(prec, nw):
    """afqmc_run in free projection (energy every 2nd step, QR every 5) with and without graphs."""
    prob = PROBLEMS["uhf_N13_3_2"]()
    out = {}
    for graphs in (False, True):
        ctx = _ctx(prob, nw, prec=prec, seed=77)
        ctx.set_graphs(graphs)
        ctx.set_free_projection(True)
        e = ctx.run(17, energy_every=2, reortho_every=5, comb_every=0)
        psi, _, w, _ = ctx.get_walkers()
        out[graphs] = (e, psi, w, ctx.weight_phases())
        ctx.close()
    for a, b in zip(out[False], out[True]):
        assert np.array_equal(a, b)
    e = out[True][0]
    assert e.shape == (9, 4) and np.all(np.isfinite(e))


def test_free_projection_reduced_precision_within_tolerance():
    """BF16x3 free projection against the FP64 form on identical fields: 10 steps, N=108, 64 walkers,
    |Re(num/den)| within the 0.1 mHa horizon tolerance of the phaseless forms."""
    prob = config_medium()
    e = {}
    for p in ("fp64", "bf16x3"):
        ctx = _ctx(prob, 64, prec=p, seed=9)
        ctx.set_free_projection(True)
        s = ctx.run(10, energy_every=1, reortho_every=5, comb_every=0)
        e[p] = ((s[:, 0] + 1j * s[:, 1]) / (s[:, 2] + 1j * s[:, 3])).real
        ctx.close()
    assert np.max(np.abs(e["bf16x3"] - e["fp64"])) <= 1e-4, e


def test_free_projection_converges_to_exact_diagonalisation():
    """4 orbitals, 2+2 electrons, naux=6, dt=0.025, 120 steps (tau = 3): the GPU free-projection
    estimator over 4096 walkers (16 groups) reaches E_FCI within its error plus a Trotter allowance,
    starting from a trial that is not exact."""
    prob = tiny_problem(4, 2, 2, naux=6, seed=7)
    sec = fci.Sector(4, 2, 2)
    e_fci = float(np.linalg.eigvalsh(sec.hamiltonian(prob.h1e, fci.eri_from_cholesky(prob.chol), prob.ecore))[0])
    nw, ngroups = 4096, 16
    ctx = _ctx(prob, nw, seed=20240616, dt=0.025)
    evar = ctx.info()["e_var"]
    assert evar - e_fci > 1e-3
    ctx.set_free_projection(True)
    ctx.run(120, energy_every=0, reortho_every=5, comb_every=0)
    _, eloc = ctx.local_energy(per_walker=True)
    _, _, w, _ = ctx.get_walkers()
    wc = w * np.exp(1j * ctx.weight_phases())
    g = np.arange(nw) % ngroups
    est = np.array([(np.sum(wc[g == k] * eloc[g == k, 0]) / np.sum(wc[g == k])).real for k in range(ngroups)])
    mean, err = est.mean(), est.std(ddof=1) / math.sqrt(ngroups)
    assert abs(mean - e_fci) < 4 * err + 2e-3, (mean, err, e_fci, evar)
    assert abs(mean - e_fci) < 0.5 * (evar - e_fci) + 4 * err, (mean, err, e_fci, evar)
