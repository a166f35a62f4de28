"""Pins for the oracle with complex Hamiltonians and complex Cholesky vectors (Section "Support of
complex Cholesky vectors": twice as many auxiliary fields as Cholesky vectors), against brute-force
Fock-space references built from the complex two-electron integrals (oracle.fci, which never uses
the single-determinant formulas).  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import afqmc as orc
from oracle import fci
from synthetic_inputs import make_complex_problem, random_walkers


def _case(nalpha=2, nbeta=2, unrestricted=False, npairs=3, seed=5):
    prob = make_complex_problem(4, nalpha, nbeta, npairs, 2.0, seed, unrestricted=unrestricted)
    sec = fci.Sector(4, nalpha, nbeta)
    eri = fci.eri_from_complex_cholesky(prob.chol)
    hfci = sec.hamiltonian(prob.h1e, eri, prob.ecore)
    fields = orc.hermitian_fields(prob.chol)
    return prob, sec, hfci, fields


CASES = [dict(), dict(unrestricted=True, seed=11), dict(nalpha=2, nbeta=1, unrestricted=True, seed=7, npairs=2)]


def test_complex_integrals_have_the_two_electron_symmetries():
    prob, _, _, _ = _case()
    eri = fci.eri_from_complex_cholesky(prob.chol)
    assert np.iscomplexobj(prob.chol) and np.abs(prob.chol.imag).max() > 0.1 * np.abs(prob.chol).max()
    assert np.allclose(eri, eri.transpose(2, 3, 0, 1), atol=1e-14)            # (ps|qr) = (qr|ps)
    assert np.allclose(eri, eri.transpose(1, 0, 3, 2).conj(), atol=1e-14)     # (ps|qr) = (sp|rq)*
    assert np.abs(eri.imag).max() > 1e-3                                       # genuinely complex
    # real symmetric L: the complex form reduces to Eq. 3
    lr = np.random.default_rng(1).standard_normal((3, 4, 4))
    lr = lr + lr.transpose(0, 2, 1)
    assert np.allclose(fci.eri_from_complex_cholesky(lr), fci.eri_from_cholesky(lr))


def test_hermitian_fields_are_hermitian_and_reduce_for_real_vectors():
    prob, _, _, fields = _case()
    assert fields.shape[0] == 2 * prob.chol.shape[0]
    assert np.allclose(fields, fields.conj().transpose(0, 2, 1), atol=1e-15)
    lr = np.random.default_rng(2).standard_normal((2, 4, 4))
    lr = lr + lr.transpose(0, 2, 1)
    f = orc.hermitian_fields(lr)
    assert np.allclose(f[0::2], lr) and np.allclose(f[1::2], 0.0)


def test_complex_hamiltonian_field_form_matches_eri_form():
    """Eq. 2 with complex integrals == v0 - 1/2 sum_g v_g^2 (+E0) over the 2X Hermitian fields M^g
    (v_g = i M_g, v0 = h - 1/2 sum_g M^g M^g), as Fock-space matrices."""
    prob, sec, hfci, fields = _case()
    v0 = prob.h1e - 0.5 * np.einsum("gpr,grq->pq", fields, fields)
    h2 = sec.one_body(v0) + prob.ecore * np.eye(sec.dim)
    for m in fields:
        vg = 1j * sec.one_body(m)
        h2 = h2 - 0.5 * vg @ vg
    assert np.allclose(hfci, h2, atol=1e-12)
    assert np.allclose(hfci, hfci.conj().T, atol=1e-12)
    # the field-form one-body term equals h - 1/2 sum_s (ps|sr) from the integrals
    eri = fci.eri_from_complex_cholesky(prob.chol)
    assert np.allclose(v0, prob.h1e - 0.5 * np.einsum("psqr->pr", eri * np.eye(4)[None, :, :, None]), atol=1e-13)


@pytest.mark.parametrize("case", CASES)
def test_complex_overlap_greens_function_force_bias_energy_vs_fci(case):
    prob, sec, hfci, fields = _case(**case)
    st = orc.build_setup(prob.h1e, fields, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, 0.01)
    assert np.iscomplexobj(st.phi_a) and np.isrealobj(st.lbar)
    ct = sec.determinant_vector(prob.psiT)
    evar = (ct.conj() @ hfci @ ct) / (ct.conj() @ ct)
    assert abs(evar.imag) < 1e-12 and abs(st.evar - evar.real) < 1e-12 * max(1, abs(evar))
    vbar_fci = np.array([(ct.conj() @ (1j * sec.one_body(m)) @ ct) / (ct.conj() @ ct) for m in fields])
    assert np.allclose(1j * st.lbar, vbar_fci, atol=1e-12)
    rng = np.random.default_rng(3)
    for psi in random_walkers(rng, 4, prob.nalpha + prob.nbeta, 4, spread=0.6, psiT=prob.psiT):
        cpsi = sec.determinant_vector(psi)
        ovl = ct.conj() @ cpsi
        logo, th_a, th_b = orc.overlap_theta(st, psi)
        assert abs(np.exp(logo) - ovl) < 1e-12 * abs(ovl)
        for spin, (phi, th) in enumerate(((st.phi_a, th_a), (st.phi_b, th_b))):
            if th.shape[1] == 0:
                continue
            g = orc.greens_function(phi, th)
            gref = np.array([[ct.conj() @ sec.one_body_spin(p, q, spin) @ cpsi for q in range(4)]
                             for p in range(4)]) / ovl
            assert np.allclose(g, gref, atol=1e-11)
            assert np.allclose(g @ g, g, atol=1e-11)
            assert abs(np.trace(g) - th.shape[1]) < 1e-11
        vb = orc.force_bias(st, th_a, th_b)
        vref = np.array([ct.conj() @ sec.one_body(m) @ cpsi for m in fields]) / ovl
        assert np.allclose(vb, vref, atol=1e-11)
        xbar = orc.field_shift(st, vb, cap=None)
        xref = np.array([-math.sqrt(st.dt) * (ct.conj() @ (1j * sec.one_body(m)) @ cpsi / ovl - vbar_fci[g])
                         for g, m in enumerate(fields)])
        assert np.allclose(xbar, xref, atol=1e-12)
        eref = (ct.conj() @ hfci @ cpsi) / ovl
        e, e1, e2 = orc.local_energy(st, th_a, th_b)
        assert abs(e - eref) < 1e-10 * max(1.0, abs(eref))
        assert abs(orc.local_energy_full_g(st, psi) - eref) < 1e-10 * max(1.0, abs(eref))


def test_complex_propagator_matches_fock_space_operator():
    """Thouless with complex Hermitian fields: the determinant update equals B(x) of Eq. 8 on the FCI
    vector (mean-field shift, h_eff, c_mf and E_c included)."""
    prob, sec, _, fields = _case(unrestricted=True, seed=13)
    dt = 0.02
    st = orc.build_setup(prob.h1e, fields, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, dt)
    ct = sec.determinant_vector(prob.psiT)
    vs = [1j * sec.one_body(m) for m in fields]
    vbar = [(ct.conj() @ v @ ct) / (ct.conj() @ ct) for v in vs]
    v0 = sec.one_body(prob.h1e - 0.5 * np.einsum("gpr,grq->pq", fields, fields))
    o1 = v0 - sum(vb * v for vb, v in zip(vbar, vs))
    const = prob.ecore + 0.5 * sum(vb * vb for vb in vbar)
    rng = np.random.default_rng(5)
    psi = random_walkers(rng, 4, prob.nalpha + prob.nbeta, 1, 0.4, prob.psiT)[0]
    for _ in range(2):
        x = rng.standard_normal(len(fields)) + 0.3j * rng.standard_normal(len(fields))
        p2, cmf = orc.propagate_determinant(st, psi, x, order=30)
        lhs = sec.determinant_vector(p2) * np.exp(cmf - dt * st.ecore_mf)
        half = scipy.linalg.expm(-0.5 * dt * o1)
        two = scipy.linalg.expm(-math.sqrt(dt) * sum(xg * (v - vb * np.eye(sec.dim))
                                                     for xg, v, vb in zip(x, vs, vbar)))
        rhs = half @ two @ half * np.exp(-dt * const) @ sec.determinant_vector(psi)
        assert np.allclose(lhs, rhs, atol=1e-12 * np.max(np.abs(rhs)))


def test_real_trial_formulas_would_fail_the_complex_pins():
    """A planted mistake (the trial's transpose without conjugation in the overlap) breaks the overlap
    pin, so the pins above see the conjugations the complex case needs."""
    prob, sec, _, fields = _case(unrestricted=True, seed=11)
    st = orc.build_setup(prob.h1e, fields, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, 0.01)
    psi = random_walkers(np.random.default_rng(9), 4, prob.nalpha + prob.nbeta, 1, 0.5, prob.psiT)[0]
    ovl = sec.determinant_vector(prob.psiT).conj() @ sec.determinant_vector(psi)
    wrong = np.linalg.det(st.phi_a.T @ psi[:, :prob.nalpha]) * np.linalg.det(st.phi_b.T @ psi[:, prob.nalpha:])
    assert abs(wrong - ovl) > 1e-3 * abs(ovl)
    logo, _, _ = orc.overlap_theta(st, psi)
    assert abs(np.exp(logo) - ovl) < 1e-12 * abs(ovl)
