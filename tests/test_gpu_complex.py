"""Complex Hamiltonians with complex Cholesky vectors (Section "Support of complex Cholesky vectors":
two auxiliary fields per vector) through the C ABI, against the oracle on identical fields.

FP64: 1e-10 relative along trajectories (binary64 everywhere, sums in another order), 1e-11 per
kernel.  FP32 and BF16x3: the mixed energy within 0.1 mHa over the horizon (binary32 contractions;
split bf16 products realified along K, ~16 significant bits each).  BF16: 1 mHa (8 bits per
operand)."""
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
    # N > 128: two M tiles of every tensor-core product, a ragged second tile
    "uhf_N136_4_3": lambda: make_complex_problem(136, 4, 3, 6, 4.0, 74, unrestricted=True),
}
HORIZON_TOL = {"fp32": 1e-4, "bf16x3": 1e-4, "bf16": 1e-3}


def _setup(prob, dt=0.005):
    return orc.build_setup(prob.h1e, orc.hermitian_fields(prob.chol), prob.ecore, prob.nalpha, prob.nbeta,
                           prob.psiT, dt)


def _ctx(prob, nw, prec="fp64", seed=5, dt=0.005, **kw):
    return pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, dt=dt,
                     seed=seed, prec=prec, **kw)


@pytest.mark.parametrize("name", [n for n in PROBLEMS if n != "uhf_N136_4_3"])
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


@pytest.mark.parametrize("name", [n for n in PROBLEMS if n != "uhf_N136_4_3"])
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


@pytest.mark.parametrize("name", ["rhf_N8_2_2", "uhf_N24_5_4", "uhf_N136_4_3"])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_complex_tensor_forms_track_the_oracle(name, prec):
    """The realified tensor-core path (exchange and force bias, VHS over 2 naux fields, propagation with
    complex E_h): 16 walkers, 10 steps, QR every 5, no comb, the same fields as the oracle."""
    prob = PROBLEMS[name]()
    nw, nsteps, seed = 16, 10, 240616251
    st = _setup(prob)
    ctx = _ctx(prob, nw, prec=prec, seed=seed)
    assert abs(ctx.info()["e_var"] - st.evar) < HORIZON_TOL[prec]
    e = ctx.run(nsteps, energy_every=1, reortho_every=5, comb_every=0)
    _, _, w_g, _ = ctx.get_walkers()
    ctx.close()
    hist, wk = orc.run_phaseless(st, prob.psiT, nw, nsteps, seed, reortho_every=5, comb_every=0)
    d = np.abs(e[:, 0] / e[:, 1] - hist[:, 0] / hist[:, 1])
    assert np.max(d) <= HORIZON_TOL[prec], d
    r = (w_g / wk.w) / np.mean(w_g / wk.w)
    assert np.max(np.abs(r - 1.0)) < (1e-4 if prec == "bf16x3" else 1e-2)


@pytest.mark.parametrize("name", ["uhf_N24_5_4", "uhf_N136_4_3"])
def test_complex_bf16x3_local_energy_and_force_bias_per_walker(name):
    """Kernel level: E_L = E1 + E_H + E_X of random walkers from the tensor-core exchange, and the
    force-bias shift of the next step, against the oracle on the same walkers."""
    prob = PROBLEMS[name]()
    st = _setup(prob)
    nw = 6
    ctx = _ctx(prob, nw, prec="bf16x3", seed=12)
    rng = np.random.default_rng(8)
    psi = random_walkers(rng, prob.norb, prob.nalpha + prob.nbeta, nw, 0.3, prob.psiT)
    ctx.set_walkers(psi, np.ones(nw), 0)
    _, eloc = ctx.local_energy(per_walker=True)
    ctx.propagate(1)
    _, xbar = ctx.get_fields()
    ctx.close()
    for i in range(nw):
        _, ta, tb = orc.overlap_theta(st, psi[i])
        e = orc.local_energy(st, ta, tb)
        for k in range(3):
            assert abs(eloc[i, k] - e[k]) < 1e-4 * max(1.0, abs(e[k])), (i, k, eloc[i, k], e[k])
        ref = orc.field_shift(st, orc.force_bias(st, ta, tb), 1.0)
        assert np.all(np.abs(xbar[i] - ref) <= 1e-4 * np.abs(ref) + 1e-6), i


def test_complex_bf16x3_propagation_paths_agree():
    """The tensor-core propagation (four complex E_h planes) and the CUDA-core propagation on the planar
    VHS give the same trajectory to the bf16 rounding of E_h and the Taylor terms."""
    prob = PROBLEMS["uhf_N24_5_4"]()
    out = []
    for path in (0, 1):
        ctx = _ctx(prob, 8, prec="bf16x3", seed=19)
        ctx.set_tuning(prop_path=path)
        out.append(ctx.run(6, energy_every=1, reortho_every=3, comb_every=0))
        ctx.close()
    assert np.max(np.abs(out[0][:, 0] / out[0][:, 1] - out[1][:, 0] / out[1][:, 1])) < 1e-4


def test_complex_contexts_reject_real_chunks_and_the_control_variate():
    prob = PROBLEMS["rhf_N8_2_2"]()
    ctx = _ctx(prob, 4, prec="bf16x3")
    with pytest.raises(pkg.AfqmcError, match="real Hamiltonians"):
        ctx.cv_attach()
    ctx.close()
    lib = pkg.load()
    assert lib.afqmc_workspace_size_complex(8, 5, 2, 2, None, None, None) == 1
