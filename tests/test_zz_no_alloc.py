"""The allocation-free comb plan (afqmc_comb_plan_noalloc) against afqmc_popcontrol.

Some callers cannot allocate device memory (their memory belongs to another
allocator, or they must avoid cudaMalloc's implicit synchronisation); the
allocation-free entry point serves them with a static device scratch array.
This file is collected last so that a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from paper_2406_16238_b300 import _lib
from synthetic_inputs import config_small

pytestmark = pytest.mark.gpu


def _popcontrol_reference(prob, nw, seed, step, w, rng):
    """Walkers after afqmc_popcontrol of a context holding distinct walkers with weights w."""
    half = prob.psiT[:, :prob.nalpha][None] + 0.3 * (rng.standard_normal((nw, prob.norb, prob.nalpha))
                                                      + 1j * rng.standard_normal((nw, prob.norb, prob.nalpha)))
    psi = np.concatenate([half, half], axis=2)
    ctx = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, seed=seed)
    ctx.set_walkers(psi, w, step)
    ctx.popcontrol()
    psi_after, _, w_after, _ = ctx.get_walkers()
    ctx.close()
    return psi, psi_after, w_after


@pytest.mark.parametrize("nw,seed,steps", [(50, 123, (30, 31)), (7, 5, (10, 10))])
def test_noalloc_comb_plan_matches_popcontrol_on_consecutive_calls(nw, seed, steps):
    import torch
    prob = config_small()
    rng = np.random.default_rng(nw)
    src = torch.full((nw,), -7, dtype=torch.int32, device="cuda")
    neww = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call, step in enumerate(steps):
        w = rng.exponential(size=nw)
        w[[0, nw // 2]] = 0.0
        psi, psi_after, w_after = _popcontrol_reference(prob, nw, seed, step, w, rng)
        wd = torch.tensor(w, dtype=torch.float64, device="cuda")
        pkg._lib.comb_plan_noalloc(wd, seed, step, src, neww)
        torch.cuda.synchronize()
        s = src.cpu().numpy().astype(np.int64)
        nwt = float(neww.item())
        assert np.array_equal(psi_after, psi[s]), f"call {call}"
        assert np.allclose(w_after, nwt, rtol=1e-15, atol=0), f"call {call}"
        assert not set(s.tolist()) & {0, nw // 2}


def test_noalloc_comb_plan_after_larger_call_and_all_zero_weights():
    import torch
    nw_big, nw = 300, 9
    src = torch.zeros(nw_big, dtype=torch.int32, device="cuda")
    neww = torch.zeros(1, dtype=torch.float64, device="cuda")
    pkg._lib.comb_plan_noalloc(torch.rand(nw_big, dtype=torch.float64, device="cuda"), 1, 2, src, neww)
    zero = torch.zeros(nw, dtype=torch.float64, device="cuda")
    pkg._lib.comb_plan_noalloc(zero, 1, 3, src[:nw], neww)
    torch.cuda.synchronize()
    assert float(neww.item()) == -1.0
    assert np.array_equal(src[:nw].cpu().numpy(), np.arange(nw))


def test_noalloc_comb_plan_rejects_oversized_batches():
    import torch
    lib = pkg.load()
    w = torch.ones(1, dtype=torch.float64, device="cuda")
    st = lib.afqmc_comb_plan_noalloc(ctypes.c_void_p(w.data_ptr()), _lib.NOALLOC_MAX_WALKERS + 1, 1, 0,
                                     ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(w.data_ptr()), None)
    assert st == 1 and "outside" in lib.afqmc_last_error().decode()


@pytest.mark.parametrize("nw", [4097, _lib.NOALLOC_MAX_WALKERS])
def test_noalloc_comb_plan_large_batches_match_the_oracle(nw):
    """Batches beyond one shared-memory tile of the kernel (2048 weights), whose prefix sums are written to
    and searched in the static array, up to its last prefix word: src and the new weight bit for bit
    against the oracle's comb (binary64 prefix in index order, the same Philox xi), with zero weights."""
    import torch
    from oracle import afqmc as orc
    from oracle import philox
    rng = np.random.default_rng(nw)
    seed, step = 99, 1234
    w = rng.exponential(size=nw)
    w[rng.choice(nw, size=nw // 7, replace=False)] = 0.0
    w[-1] = 0.0
    ref_src, ref_w = orc.comb_assignment(w, philox.comb_uniform(seed, step))
    src = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    neww = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):   # two calls in a row share the array
        pkg._lib.comb_plan_noalloc(torch.tensor(w, dtype=torch.float64, device="cuda"), seed, step, src, neww)
        torch.cuda.synchronize()
        assert np.array_equal(src.cpu().numpy().astype(np.int64), ref_src)
        assert float(neww.item()) == ref_w
