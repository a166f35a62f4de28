"""Pins for the FP64 oracle against things other than itself (CPU only).

Every quantity the oracle computes is checked here against an exact many-body
reference built by brute force in Fock space (oracle.fci, which applies
creation / annihilation operators to bit strings and never uses the
single-determinant formulas), against closed forms, published test vectors, or
invariants of the method.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import afqmc as orc
from oracle import fci, philox
from synthetic_inputs import random_walkers, tiny_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Philox and the normal transform ------------------------------------------------------

def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(t, 16) for t in row]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_series_log_and_trig_accuracy():
    u = np.concatenate([np.geomspace(2.0 ** -52, 1.0, 20001), np.linspace(1e-3, 1.0, 20001)])
    ref = np.log(u)
    err = np.abs(philox.series_log(u) - ref)
    assert np.all(err <= 2.5e-16 * np.maximum(np.abs(ref), 1.0) + 1e-300)
    t = np.linspace(0.0, 1.0, 40001, endpoint=False)
    c, s = philox.series_sincos_turn(t)
    assert np.max(np.abs(c - np.cos(2 * np.pi * t))) < 2e-15
    assert np.max(np.abs(s - np.sin(2 * np.pi * t))) < 2e-15
    # exact special points of the quarter-turn reduction
    c, s = philox.series_sincos_turn(np.array([0.0, 0.25, 0.5, 0.75]))
    assert np.array_equal(c, [1.0, 0.0, -1.0, 0.0]) or np.allclose(c, [1, 0, -1, 0], atol=1e-16)


def test_normals_distribution():
    x = philox.normals(2024, 17, 4000, 250)
    assert x.shape == (4000, 250)
    m, v = x.mean(), x.var()
    n = x.size
    assert abs(m) < 5 / math.sqrt(n)
    assert abs(v - 1) < 5 * math.sqrt(2 / n)
    assert abs((x ** 4).mean() - 3) < 0.05
    # Kolmogorov-Smirnov against N(0,1)
    from scipy import stats
    assert stats.kstest(x.ravel()[:200000], "norm").pvalue > 1e-3
    # distinct steps / walkers / streams give distinct draws; same counters reproduce
    assert np.array_equal(x, philox.normals(2024, 17, 4000, 250))
    assert not np.allclose(x[:10], philox.normals(2024, 18, 10, 250))
    odd = philox.normals(2024, 17, 3, 7)
    assert np.array_equal(odd, x[:3, :7])


def test_uniform52_bounds():
    u = philox.uniform52(np.array([0, 0xFFFFFFFF], dtype=np.uint64), np.array([0, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] == 2.0 ** -53 and u[1] == 1.0 - 2.0 ** -53


# --- Fock-space references ----------------------------------------------------------------

def _fci_case(nalpha=2, nbeta=2, unrestricted=False, naux=6, seed=7):
    prob = tiny_problem(4, nalpha, nbeta, naux=naux, seed=seed, unrestricted=unrestricted)
    sec = fci.Sector(4, nalpha, nbeta)
    eri = fci.eri_from_cholesky(prob.chol)
    hfci = sec.hamiltonian(prob.h1e, eri, prob.ecore)
    return prob, sec, hfci


CASES = [dict(), dict(unrestricted=True, seed=11), dict(nalpha=2, nbeta=1, unrestricted=True, seed=5),
         dict(nalpha=3, nbeta=1, unrestricted=True, seed=3)]


def test_hamiltonian_cholesky_form_matches_eri_form():
    """Eqs. 2-6: sum h a+a + 1/2 g a+a+aa  ==  v0 - 1/2 sum v_g^2 (+E0) as Fock-space matrices."""
    prob, sec, hfci = _fci_case()
    n = prob.norb
    v0 = prob.h1e - 0.5 * np.einsum("gpr,grq->pq", prob.chol, prob.chol)
    h2 = sec.one_body(v0) + prob.ecore * np.eye(sec.dim)
    for g in range(prob.naux):
        vg = 1j * sec.one_body(prob.chol[g])
        h2 = h2 - 0.5 * vg @ vg
    assert np.allclose(hfci, h2, atol=1e-12)
    assert np.allclose(hfci, hfci.conj().T, atol=1e-12)


@pytest.mark.parametrize("case", CASES)
def test_overlap_greens_function_force_bias_energy_vs_fci(case):
    prob, sec, hfci = _fci_case(**case)
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, 0.01)
    rng = np.random.default_rng(3)
    ct = sec.determinant_vector(prob.psiT)
    # E_var = <T|H|T>/<T|T>
    assert abs(st.evar - (ct.conj() @ hfci @ ct).real / (ct.conj() @ ct).real) < 1e-12
    vbar_fci = np.array([(ct.conj() @ (1j * sec.one_body(prob.chol[g])) @ ct) / (ct.conj() @ ct)
                         for g in range(prob.naux)])
    assert np.allclose(1j * st.lbar, vbar_fci, atol=1e-12)
    for psi in random_walkers(rng, 4, prob.nalpha + prob.nbeta, 4, spread=0.6, psiT=prob.psiT):
        cpsi = sec.determinant_vector(psi)
        ovl = ct.conj() @ cpsi
        logo, th_a, th_b = orc.overlap_theta(st, psi)
        assert abs(np.exp(logo) - ovl) < 1e-12 * abs(ovl)
        # Green's function <a+_p a_q> per spin
        for spin, (phi, th) in enumerate(((st.phi_a, th_a), (st.phi_b, th_b))):
            if th.shape[1] == 0:
                continue
            g = orc.greens_function(phi, th)
            gref = np.array([[ct.conj() @ sec.one_body_spin(p, q, spin) @ cpsi for q in range(4)]
                             for p in range(4)]) / ovl
            assert np.allclose(g, gref, atol=1e-11)
            assert np.allclose(g @ g, g, atol=1e-11)                    # idempotent
            assert abs(np.trace(g) - th.shape[1]) < 1e-11               # Tr G = n_sigma
        # force bias <L_g> and the shift of Eq. 12 (uncapped)
        vb = orc.force_bias(st, th_a, th_b)
        vref = np.array([ct.conj() @ sec.one_body(prob.chol[g]) @ cpsi for g in range(prob.naux)]) / ovl
        assert np.allclose(vb, vref, atol=1e-11)
        xbar = orc.field_shift(st, vb, cap=None)
        xref = np.array([-math.sqrt(st.dt) * (ct.conj() @ (1j * sec.one_body(prob.chol[g])) @ cpsi / ovl
                                               - vbar_fci[g]) for g in range(prob.naux)])
        assert np.allclose(xbar, xref, atol=1e-12)
        # local energy <T|H|psi>/<T|psi>, half-rotated and full-G forms
        eref = (ct.conj() @ hfci @ cpsi) / ovl
        e, e1, e2 = orc.local_energy(st, th_a, th_b)
        assert abs(e - eref) < 1e-10 * max(1.0, abs(eref))
        assert abs(e1 + e2 - e) < 1e-12 * max(1.0, abs(e))
        assert abs(orc.local_energy_full_g(st, psi) - eref) < 1e-10 * max(1.0, abs(eref))


def test_trial_greens_function_idempotent():
    prob, _, _ = _fci_case()
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, 0.01)
    _, th_a, _ = orc.overlap_theta(st, prob.psiT.astype(complex))
    g = orc.greens_function(st.phi_a, th_a)
    assert np.allclose(g @ g, g, atol=1e-13) and np.allclose(g, g.T, atol=1e-13)


def _fock_propagator(prob, sec, dt, x):
    """B(x) of Eq. 8 with the mean-field shift, built from the paper's operators in Fock space."""
    ct = sec.determinant_vector(prob.psiT)
    vs = [1j * sec.one_body(prob.chol[g]) for g in range(prob.naux)]
    vbar = [(ct.conj() @ v @ ct) / (ct.conj() @ ct) for v in vs]
    v0 = sec.one_body(prob.h1e - 0.5 * np.einsum("gpr,grq->pq", prob.chol, prob.chol))
    o1 = v0 - sum(vb * v for vb, v in zip(vbar, vs))
    const = prob.ecore + 0.5 * sum(vb * vb for vb in vbar)
    half = scipy.linalg.expm(-0.5 * dt * o1)
    two = scipy.linalg.expm(-math.sqrt(dt) * sum(xg * (v - vb * np.eye(sec.dim)) for xg, v, vb in zip(x, vs, vbar)))
    return half @ two @ half * np.exp(-dt * const)


@pytest.mark.parametrize("case", CASES[:3])
def test_propagator_matches_fock_space_operator(case):
    """Thouless: the determinant update (VHS, h_eff, c_mf, E_c) equals B(x) of Eq. 8 on the FCI vector."""
    prob, sec, _ = _fci_case(**case)
    dt = 0.02
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, dt)
    rng = np.random.default_rng(5)
    psi = random_walkers(rng, 4, prob.nalpha + prob.nbeta, 1, 0.4, prob.psiT)[0]
    for _ in range(3):
        x = rng.standard_normal(prob.naux) + 0.3j * rng.standard_normal(prob.naux)
        p2, cmf = orc.propagate_determinant(st, psi, x, order=30)
        lhs = sec.determinant_vector(p2) * np.exp(cmf - dt * st.ecore_mf)
        rhs = _fock_propagator(prob, sec, dt, x) @ sec.determinant_vector(psi)
        assert np.allclose(lhs, rhs, atol=1e-12 * np.max(np.abs(rhs)))


def _gauss_hermite(naux, nodes):
    z, wq = np.polynomial.hermite_e.hermegauss(nodes)   # weight exp(-x^2/2)
    wq = wq / math.sqrt(2 * math.pi)
    pts = np.array(list(itertools.product(z, repeat=naux)))
    wts = np.prod(np.array(list(itertools.product(wq, repeat=naux))), axis=1)
    return pts, wts


def test_field_average_matches_exact_propagator_to_second_order():
    """E_x[B(x)] = exp(-dt H) + O(dt^2): error ratio ~4 per halving of dt (Eqs. 7-8)."""
    prob = tiny_problem(4, 2, 2, naux=3, seed=19)
    sec = fci.Sector(4, 2, 2)
    hfci = sec.hamiltonian(prob.h1e, fci.eri_from_cholesky(prob.chol), prob.ecore)
    rng = np.random.default_rng(1)
    psi = random_walkers(rng, 4, 4, 1, 0.3, prob.psiT)[0]
    cpsi = sec.determinant_vector(psi)
    pts, wts = _gauss_hermite(3, 12)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, dt)
        avg = np.zeros(sec.dim, dtype=complex)
        for x, wq in zip(pts, wts):
            p2, cmf = orc.propagate_determinant(st, psi, x, order=25)
            avg += wq * sec.determinant_vector(p2) * np.exp(cmf - dt * st.ecore_mf)
        exact = scipy.linalg.expm(-dt * hfci) @ cpsi
        errs.append(np.linalg.norm(avg - exact) / np.linalg.norm(exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.7 < r2 < 4.3, errs


def test_importance_sampling_identity_for_hybrid_weights():
    """Eqs. 13-16: E_x[I(x, xbar) psi'(x)/O'(x)] equals the unshifted average (change of variables).

    The hybrid weight exp(log I) of the oracle, with the force bias of a walker
    that is not the trial, must reproduce the free (unshifted) field average;
    a wrong sign or factor in x.xbar - xbar^2/2, c_mf or log O breaks it.
    """
    prob = tiny_problem(4, 2, 2, naux=3, seed=23)
    sec = fci.Sector(4, 2, 2)
    dt = 0.02
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, dt)
    rng = np.random.default_rng(9)
    psi = random_walkers(rng, 4, 4, 1, 0.5, prob.psiT)[0]
    logo, th_a, th_b = orc.overlap_theta(st, psi)
    xbar = orc.field_shift(st, orc.force_bias(st, th_a, th_b), cap=None)
    assert np.max(np.abs(xbar)) > 0.01
    pts, wts = _gauss_hermite(3, 14)
    shifted = np.zeros(sec.dim, dtype=complex)
    free = np.zeros(sec.dim, dtype=complex)
    for x, wq in zip(pts, wts):
        p2, cmf = orc.propagate_determinant(st, psi, x - xbar, order=25)
        logo2, _, _ = orc.overlap_theta(st, p2)
        _, log_i, _ = orc.weight_update(st, 1.0, logo, logo2, cmf, x, xbar, e_trial=st.ecore_mf)
        shifted += wq * np.exp(log_i) * sec.determinant_vector(p2) / np.exp(logo2)
        p0, cmf0 = orc.propagate_determinant(st, psi, x, order=25)
        free += wq * np.exp(cmf0) * sec.determinant_vector(p0) / np.exp(logo)
    assert np.linalg.norm(shifted - free) < 1e-9 * np.linalg.norm(free)


def test_phaseless_weight_real_case_and_projection():
    """With a real overlap ratio the phaseless weight equals |I|; a phase beyond pi/2 kills the walker."""
    prob = tiny_problem(4, 2, 2, naux=3, seed=23)
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, 0.01)
    x = np.array([0.3, -1.0, 0.2])
    xbar = np.array([0.01 + 0.02j, -0.03j, 0.0])
    w, log_i, theta = orc.weight_update(st, 2.0, 0.1 + 0.0j, 0.3 + 0.0j, 0.0j, x, xbar, st.ecore_mf)
    assert theta == 0.0 and abs(w - 2.0 * math.exp(log_i.real)) < 1e-14
    w, _, theta = orc.weight_update(st, 2.0, 0.1 + 0.0j, 0.3 + 2.0j, 0.0j, x, xbar, st.ecore_mf)
    assert abs(theta - 2.0) < 1e-15 and w == 0.0


def test_diagonal_eigenstate_keeps_unit_weight():
    """Closed form: H diagonal in the orbital basis and Phi_T an eigen-determinant -> w stays 1, E_L = E_var."""
    n = 3
    h1e = np.diag([0.2, 1.1, 2.5])
    chol = np.stack([np.diag([0.5, -0.2, 0.1]), np.diag([0.05, 0.3, -0.4])])
    psiT = np.eye(n)[:, [0, 0]]
    st = orc.build_setup(h1e, chol, 0.4, 1, 1, psiT, 0.01)
    # closed-form HF energy of the doubly occupied orbital 0
    l0 = chol[:, 0, 0]
    evar = 0.4 + 2 * 0.2 + 0.5 * np.sum((2 * l0) ** 2) - 0.5 * 2 * np.sum(l0 ** 2)
    assert abs(st.evar - evar) < 1e-14
    hist, wk = orc.run_phaseless(st, psiT, 5, 12, seed=3, reortho_every=5, comb_every=0)
    assert np.allclose(wk.w, 1.0, atol=1e-12)
    assert np.allclose(hist[:, 0] / hist[:, 1], evar, atol=1e-12)


def test_taylor_against_expm():
    rng = np.random.default_rng(0)
    a = 0.2 * (rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9)))
    psi = rng.standard_normal((9, 3)) + 1j * rng.standard_normal((9, 3))
    nrm = np.linalg.norm(a, 2)
    for order in (4, 6, 8):
        err = np.linalg.norm(orc.taylor_exp_apply(a, psi, order) - scipy.linalg.expm(a) @ psi, 2)
        bound = nrm ** (order + 1) / math.factorial(order + 1) * math.exp(nrm) * np.linalg.norm(psi, 2)
        assert err <= bound
        assert err > 1e-3 * bound   # the truncation really is the error


def test_qr_invariance():
    prob, _, _ = _fci_case(unrestricted=True, seed=11)
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, 0.01)
    rng = np.random.default_rng(4)
    psi = random_walkers(rng, 4, 4, 3, 0.5, prob.psiT) * 3.0
    wk = orc.Walkers(psi.copy(), np.array([orc.overlap_theta(st, p)[0] for p in psi]), np.ones(3))
    before = [orc.overlap_theta(st, p) for p in wk.psi]
    orc.reorthogonalise(st, wk)
    for i in range(3):
        logo, th_a, th_b = orc.overlap_theta(st, wk.psi[i])
        assert abs(np.exp(logo) - np.exp(wk.logo[i])) < 1e-12 * abs(np.exp(logo))
        _, b_a, b_b = before[i]
        assert np.allclose(orc.greens_function(st.phi_a, th_a), orc.greens_function(st.phi_a, b_a), atol=1e-12)
        assert np.allclose(orc.force_bias(st, th_a, th_b), orc.force_bias(st, b_a, b_b), atol=1e-12)
        assert abs(orc.local_energy(st, th_a, th_b)[0] - orc.local_energy(st, b_a, b_b)[0]) < 1e-11
        for lo, hi in ((0, 2), (2, 4)):
            q = wk.psi[i][:, lo:hi]
            assert np.allclose(q.conj().T @ q, np.eye(2), atol=1e-13)
            r = q.conj().T @ psi[i][:, lo:hi]
            assert np.all(np.diag(r).real > 0) and np.allclose(np.diag(r).imag, 0, atol=1e-12)
            assert np.allclose(np.tril(r, -1), 0, atol=1e-12)


def test_comb_copy_counts():
    rng = np.random.default_rng(8)
    w = rng.exponential(size=37)
    w[[3, 10, 11]] = 0.0
    nw = len(w)
    total = np.sum(w)
    expect = nw * w / total
    acc = np.zeros(nw)
    grid = 2000
    for k in range(grid):
        src, wnew = orc.comb_assignment(w, (k + 0.5) / grid)
        counts = np.bincount(src, minlength=nw)
        assert counts.sum() == nw
        assert np.all(counts[[3, 10, 11]] == 0)
        assert np.all((counts == np.floor(expect)) | (counts == np.ceil(expect)))
        assert np.all(np.diff(src) >= 0)
        acc += counts
        assert wnew == total / nw or abs(wnew - total / nw) < 1e-15 * total
    assert np.allclose(acc / grid, expect, atol=2.0 / grid)


def test_energy_shift_invariance_and_trajectory_sanity():
    prob = tiny_problem(4, 2, 2, naux=6, seed=7)
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, 0.01)
    h1, wk1 = orc.run_phaseless(st, prob.psiT, 16, 30, seed=99, reortho_every=5, comb_every=10)
    h2, wk2 = orc.run_phaseless(st, prob.psiT, 16, 30, seed=99, e_trial=st.evar + 1.0,
                                reortho_every=5, comb_every=10)
    e1 = h1[:, 0] / h1[:, 1]
    e2 = h2[:, 0] / h2[:, 1]
    assert np.allclose(e1, e2, rtol=1e-13, atol=0)
    assert np.allclose(wk1.psi, wk2.psi, atol=1e-13)
    ratio = wk2.w / wk1.w
    assert np.allclose(ratio, ratio[0], rtol=1e-12)
    assert np.all(np.isfinite(e1))


def test_trial_energy_follows_the_running_estimate():
    """E_T replaced at each comb by the running mixed estimate (R4 option): since the factor
    exp(dt (E_T - E_c)) multiplies every weight alike and the comb is scale-equivariant, the
    energies and walkers equal those of a fixed E_T, and the weights differ by exactly
    prod_t exp(dt (E_T(t) - E_var)) with E_T(t) rebuilt here from the measured sums."""
    prob = tiny_problem(4, 2, 2, naux=6, seed=7)
    dt = 0.01
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, dt)
    nsteps, comb = 35, 10
    h0, wk0 = orc.run_phaseless(st, prob.psiT, 16, nsteps, seed=99, reortho_every=5, comb_every=comb)
    te = orc.TrialEnergy(st.evar)
    h1, wk1 = orc.run_phaseless(st, prob.psiT, 16, nsteps, seed=99, reortho_every=5, comb_every=comb,
                                trial_energy=te)
    assert np.allclose(h1[:, 0] / h1[:, 1], h0[:, 0] / h0[:, 1], rtol=1e-13, atol=0)
    assert np.allclose(wk1.psi, wk0.psi, atol=1e-13)
    # E_T in force during step t: E_var until the first comb (after step comb-1), then the
    # mixed estimate over the measurements at the starts of steps 0 .. c-1 of the last comb at c
    # (the sums of this run: their weight totals carry the shifts applied so far)
    et = np.full(nsteps, st.evar)
    for t in range(nsteps):
        c = (t // comb) * comb
        if c > 0:
            et[t] = np.sum(h1[:c, 0]) / np.sum(h1[:c, 1])
    log_ratio = dt * np.sum(et - st.evar)
    assert abs(te.et - np.sum(h1[:30, 0]) / np.sum(h1[:30, 1])) < 1e-12 * abs(te.et)
    assert np.allclose(h1[:, 1], h0[:, 1] * np.exp(dt * np.cumsum(np.r_[0.0, et[:-1] - st.evar])),
                       rtol=1e-11, atol=0)
    assert np.allclose(wk1.w, wk0.w * math.exp(log_ratio), rtol=1e-11, atol=0)
    # the same run in two calls continues the state (sums and E_T carried over)
    te2 = orc.TrialEnergy(st.evar)
    ha, wka = orc.run_phaseless(st, prob.psiT, 16, 17, seed=99, reortho_every=5, comb_every=comb,
                                trial_energy=te2)
    hb, wkb = orc.run_phaseless(st, prob.psiT, 16, nsteps - 17, seed=99, reortho_every=5,
                                comb_every=comb, trial_energy=te2, walkers=wka)
    assert np.array_equal(np.vstack([ha, hb]), h1)
    assert np.array_equal(wkb.w, wk1.w) and te2.et == te.et


@pytest.mark.slow
def test_free_projection_converges_to_fci():
    """Free projection (Section "Free projection AFQMC") reaches E_FCI within error + Trotter bias."""
    prob = tiny_problem(4, 2, 2, naux=6, seed=7)
    sec = fci.Sector(4, 2, 2)
    hfci = sec.hamiltonian(prob.h1e, fci.eri_from_cholesky(prob.chol), prob.ecore)
    e_fci = float(np.linalg.eigvalsh(hfci)[0])
    dt = 0.025
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, dt)
    assert st.evar - e_fci > 1e-3                  # the trial is not exact
    nw, nsteps, ngroups = 240, 120, 8
    est = []
    for grp in range(ngroups):
        psi = np.repeat(prob.psiT.astype(complex)[None], nw, axis=0)
        logo = np.full(nw, orc.overlap_theta(st, psi[0])[0])
        wc = np.ones(nw, dtype=complex)
        for s in range(nsteps):
            orc.free_projection_step(st, psi, logo, wc, seed=1000 + grp, step=s, e_trial=st.evar)
            if s % 5 == 4:
                for i in range(nw):
                    q, r = np.linalg.qr(psi[i][:, :2])
                    q2, r2 = np.linalg.qr(psi[i][:, 2:])
                    psi[i] = np.hstack([q, q2])
                    # |psi>/<T|psi> is unchanged by the QR, so only log O is recomputed
                    logo[i] = orc.overlap_theta(st, psi[i])[0]
        est.append(orc.free_projection_energy(st, psi, wc).real)
    est = np.array(est)
    mean, err = est.mean(), est.std(ddof=1) / math.sqrt(ngroups)
    assert abs(mean - e_fci) < 4 * err + 2e-3, (mean, err, e_fci, st.evar)
    assert abs(mean - e_fci) < 0.5 * (st.evar - e_fci) + 4 * err


# --- planted mistakes: the pins above must catch them -------------------------------------

def test_planted_mistakes_are_detected(monkeypatch):
    prob, sec, hfci = _fci_case(unrestricted=True, seed=11)
    rng = np.random.default_rng(3)
    psi = random_walkers(rng, 4, 4, 1, 0.6, prob.psiT)[0]
    ct = sec.determinant_vector(prob.psiT)
    cpsi = sec.determinant_vector(psi)
    eref = (ct.conj() @ hfci @ cpsi) / (ct.conj() @ cpsi)
    good = orc.local_energy

    def flipped_exchange(st, th_a, th_b):
        e, e1, e2 = good(st, th_a, th_b)
        exx = sum(np.sum((st.lrot_a[g] @ th_a) * (st.lrot_a[g] @ th_a).T) +
                  np.sum((st.lrot_b[g] @ th_b) * (st.lrot_b[g] @ th_b).T) for g in range(st.naux))
        return e + exx, e1, e2 + exx

    def transposed_theta(st, th_a, th_b):
        e = st.ecore + np.sum(st.hrot_a * th_a.T) + np.sum(st.hrot_b * th_b.T)
        for g in range(st.naux):
            ta = st.lrot_a[g] @ th_a
            e += 0.5 * np.trace(ta) ** 2 - 0.5 * np.sum(ta * ta)     # T_ab T_ab instead of T_ab T_ba
        return complex(e), 0j, 0j

    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, 0.01)
    _, th_a, th_b = orc.overlap_theta(st, psi)
    assert abs(good(st, th_a, th_b)[0] - eref) < 1e-10
    for bad in (flipped_exchange, transposed_theta):
        assert abs(bad(st, th_a, th_b)[0] - eref) > 1e-4
