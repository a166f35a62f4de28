"""Complex Hamiltonians with complex Cholesky vectors (Section "Support of complex Cholesky vectors":
two auxiliary fields per vector) through the C ABI, against the oracle on identical fields.

FP64: 1e-10 relative along trajectories (binary64 everywhere, sums in another order), 1e-11 per
kernel.  FP32: the mixed energy within 0.1 mHa over the horizon (binary32 contractions)."""
import math

import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from oracle import afqmc as orc
from synthetic_inputs import make_complex_problem, random_walkers

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "rhf_N8_2_2": lambda: make_complex_problem(8, 2, 2, 5, 3.0, 71),
    "uhf_N10_3_2": lambda: make_complex_problem(10, 3, 2, 6, 3.0, 72, unrestricted=True),
    "uhf_N24_5_4": lambda: make_complex_problem(24, 5, 4, 20, 8.0, 73, unrestricted=True),
}


def _setup(prob, dt=0.005):
    return orc.build_setup(prob.h1e, orc.hermitian_fields(prob.chol), prob.ecore, prob.nalpha, prob.nbeta,
                           prob.psiT, dt)


def _ctx(prob, nw, prec="fp64", seed=5, dt=0.005, **kw):
    return pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, dt=dt,
                     seed=seed, prec=prec, **kw)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_complex_setup_overlap_and_local_energy(name):
    prob = PROBLEMS[name]()
    st = _setup(prob)
    nw = 7
    ctx = _ctx(prob, nw)
    info = ctx.info()
    assert info["naux"] == 2 * prob.chol.shape[0]
    assert abs(info["e_var"] - st.evar) < 1e-11 * max(1.0, abs(st.evar))
    assert abs(info["e_core_mf"] - st.ecore_mf) < 1e-11 * max(1.0, abs(st.ecore_mf))
    rng = np.random.default_rng(4)
    if prob.nalpha == prob.nbeta and np.allclose(prob.psiT[:, :prob.nalpha], prob.psiT[:, prob.nalpha:]):
        half = random_walkers(rng, prob.norb, prob.nalpha, nw, 0.3, prob.psiT[:, :prob.nalpha])
        psi = np.concatenate([half, half], axis=2)
    else:
        psi = random_walkers(rng, prob.norb, prob.nalpha + prob.nbeta, nw, 0.3, prob.psiT)
    w = rng.uniform(0.5, 1.5, nw)
    ctx.set_walkers(psi, w, 0)
    sums, eloc = ctx.local_energy(per_walker=True)
    _, logo, _, _ = ctx.get_walkers()
    for i in range(nw):
        lo, ta, tb = orc.overlap_theta(st, psi[i])
        e = orc.local_energy(st, ta, tb)
        assert abs(logo[i].real - lo.real) < 1e-11 * max(1, abs(lo.real))
        for k in range(3):
            assert abs(eloc[i, k] - e[k]) < 1e-11 * max(1, abs(e[k])), (i, k, eloc[i, k], e[k])
    ctx.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_complex_one_step_parity(name):
    prob = PROBLEMS[name]()
    nw, seed = 9, 77
    st = _setup(prob, dt=0.01)
    ctx = _ctx(prob, nw, seed=seed, dt=0.01, fb_cap=0.5)
    psi0, logo0, w0, _ = ctx.get_walkers()
    ctx.propagate(1)
    x, xbar = ctx.get_fields()
    psi_g, logo_g, w_g, step = ctx.get_walkers()
    ctx.close()
    assert step == 1 and x.shape == (nw, 2 * prob.chol.shape[0])
    wk = orc.Walkers(psi0.copy(), np.array([orc.overlap_theta(st, p)[0] for p in psi0]), w0.copy(), 0)
    rec = []
    xref = orc.phaseless_step(st, wk, seed, st.evar, fb_cap=0.5, record=rec)
    assert np.array_equal(x.view(np.uint64), xref.view(np.uint64))
    for r in rec:
        assert np.allclose(xbar[r["walker"]], r["xbar"], rtol=0, atol=1e-12)
    assert np.allclose(psi_g, wk.psi, rtol=0, atol=1e-11)
    assert np.allclose(w_g, wk.w, rtol=1e-11, atol=0)
    assert np.allclose(logo_g.real, wk.logo.real, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_complex_trajectory_against_the_oracle(prec, tol):
    """24 walkers, 20 steps, QR every 5, comb every 10 (FP64) or no comb (FP32 horizon)."""
    prob = PROBLEMS["uhf_N10_3_2"]()
    nw, nsteps, seed = 24, 20, 240616250
    comb = 10 if prec == "fp64" else 0
    st = _setup(prob)
    ctx = _ctx(prob, nw, prec=prec, seed=seed)
    e = ctx.run(nsteps, energy_every=1, reortho_every=5, comb_every=comb)
    ctx.close()
    hist, _ = orc.run_phaseless(st, prob.psiT, nw, nsteps, seed, reortho_every=5, comb_every=comb)
    eg, er = e[:, 0] / e[:, 1], hist[:, 0] / hist[:, 1]
    if prec == "fp64":
        assert np.max(np.abs(eg - er) / np.abs(er)) < tol
        assert np.allclose(e[:, 1], hist[:, 1], rtol=tol, atol=0)
    else:
        assert np.max(np.abs(eg - er)) < tol


def test_complex_chunked_device_binary32_chunks():
    """complex64 Cholesky chunks from device memory, against afqmc_create of the same values from host."""
    import torch
    prob = PROBLEMS["uhf_N24_5_4"]()
    c64 = prob.chol.astype(np.complex64)
    out = []
    for chol in (c64.astype(np.complex128), [torch.from_numpy(c64[:7]).cuda(), torch.from_numpy(c64[7:]).cuda()]):
        ctx = pkg.Afqmc(prob.h1e, chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=8, seed=3,
                        naux=c64.shape[0])
        out.append(ctx.run(5, energy_every=1, reortho_every=5, comb_every=0))
        ctx.close()
    assert np.allclose(out[0], out[1], rtol=1e-11, atol=1e-13)


def test_complex_contexts_reject_tensor_forms_and_real_chunks():
    prob = PROBLEMS["rhf_N8_2_2"]()
    with pytest.raises(pkg.AfqmcError, match="FP64 and FP32"):
        _ctx(prob, 4, prec="bf16x3")
    lib = pkg.load()
    assert lib.afqmc_workspace_size_complex(8, 5, 2, 2, None, None, None) == 1
