"""GPU parity of the tensor-core propagation (BF16 forms) against the FP64 oracle.

Each case propagates random walkers one step through the C ABI, reads back the fields the
GPU drew (x and the capped force bias x̄), and propagates the same walkers with the oracle's
exp(-dt/2 h_eff) Taylor_6(VHS) exp(-dt/2 h_eff) on x - x̄ (Eq. 8).  The GPU builds VHS and
every product from split-bf16 operands (about 16 significant bits per product, fp32
accumulation), so ψ agrees to a few parts in 1e6 of its largest entry; plain BF16 builds VHS
from single bf16 operands (8 bits) and is held to 5e-3.  Shapes cover one column chunk, several
chunks, N not a multiple of 8 or 16, nbeta = 0 and N = 128 (the largest the fused kernel takes);
N = 150, 200, 300 run the batched form (two or three 128-row tiles per walker).
"""
import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from oracle import afqmc as orc
from synthetic_inputs import config_medium, config_small, make_problem, random_walkers

pytestmark = pytest.mark.gpu

PSI_TOL = {"bf16x3": 2e-5, "bf16": 5e-3}

CASES = {
    "rhf_N8": lambda: config_small(),
    "uhf_N13_3_2": lambda: make_problem(13, 3, 2, 17, 5.0, 31, unrestricted=True),
    "rhf_N6_nbeta0": lambda: make_problem(6, 2, 0, 9, 3.0, 41, unrestricted=True),
    "uhf_N37_20_17": lambda: make_problem(37, 20, 17, 60, 8.0, 43, unrestricted=True),   # 2 chunks
    "uhf_N64_40_30": lambda: make_problem(64, 40, 30, 96, 12.0, 44, unrestricted=True),  # 3 chunks
    "rhf_N108": lambda: config_medium(),
    "uhf_N128_9_7": lambda: make_problem(128, 9, 7, 160, 10.0, 45, unrestricted=True),
    # N > 128: the batched form (V streamed, one launch per product)
    "rhf_N150_12": lambda: make_problem(150, 12, 12, 300, 15.0, 46),
    "uhf_N200_20_16": lambda: make_problem(200, 20, 16, 400, 20.0, 47, unrestricted=True),
    "rhf_N300_25": lambda: make_problem(300, 25, 25, 600, 60.0, 48),
}


def _restricted(prob):
    return prob.nalpha == prob.nbeta and np.array_equal(prob.psiT[:, :prob.nalpha], prob.psiT[:, prob.nalpha:])


def _state(prob, nw, seed, spread=0.2):
    rng = np.random.default_rng(seed)
    if _restricted(prob):
        half = random_walkers(rng, prob.norb, prob.nalpha, nw, spread, prob.psiT[:, :prob.nalpha])
        psi = np.concatenate([half, half], axis=2)
    else:
        psi = random_walkers(rng, prob.norb, prob.nalpha + prob.nbeta, nw, spread, prob.psiT)
    return psi, rng.uniform(0.5, 1.5, nw)


def _ctx(prob, nw, prec, **kw):
    return pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, dt=0.01,
                     seed=11, prec=prec, **kw)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_propagation_vs_oracle(prec, name):
    prob = CASES[name]()
    nw = 37
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, 0.01)
    ctx = _ctx(prob, nw, prec)
    psi, w = _state(prob, nw, seed=8)
    ctx.set_walkers(psi, w, 5)
    ctx.propagate(1)
    x, xbar = ctx.get_fields()
    psi_g, _, _, _ = ctx.get_walkers()
    ctx.close()
    worst = 0.0
    for i in range(nw):
        ref, _ = orc.propagate_determinant(st, psi[i], x[i] - xbar[i])
        worst = max(worst, np.max(np.abs(psi_g[i] - ref)) / np.max(np.abs(ref)))
    assert worst < PSI_TOL[prec], worst


@pytest.mark.parametrize("path", [0, 2])
def test_propagation_paths_agree(path):
    """Tensor-core (path 0) and fused CUDA-core (path 2) propagation on the same walkers and fields."""
    prob = config_medium()
    nw = 64
    psi, w = _state(prob, nw, seed=9)
    out = {}
    for p in (path, 1):
        ctx = _ctx(prob, nw, "bf16x3")
        ctx.set_tuning(prop_path=p)
        ctx.set_walkers(psi, w, 3)
        ctx.propagate(1)
        out[p] = ctx.get_walkers()[0]
        ctx.close()
    scale = np.max(np.abs(out[1]))
    assert np.max(np.abs(out[path] - out[1])) < 2e-5 * scale


@pytest.mark.parametrize("large", [False, True])
def test_tensor_core_propagation_skips_frozen_walkers(large):
    prob = make_problem(150, 12, 12, 300, 15.0, 46) if large else config_medium()
    nw = 150   # more walkers than SMs: some CTAs take a second walker after a frozen one
    psi, w = _state(prob, nw, seed=10)
    w[[0, 3, 148, 149]] = 0.0
    ctx = _ctx(prob, nw, "bf16x3")
    ctx.set_walkers(psi, w, 0)
    ctx.propagate(2)
    psi_g, _, w_g, _ = ctx.get_walkers()
    for i in (0, 3, 148, 149):
        assert w_g[i] == 0.0 and np.array_equal(psi_g[i], psi[i].astype(np.complex64))
    assert not np.allclose(psi_g[1], psi[1], atol=1e-6)


@pytest.mark.parametrize("graphs", [False, True])
def test_fields_drawn_by_the_exchange_warp_are_bit_exact(graphs):
    """With the energy measured, the tensor-core exchange's spare warp draws the step's normals;
    they must equal the oracle's Philox / Box-Muller draws bit for bit, as must the normals that a
    step without an energy draws itself (direct launches and CUDA-graph replays alike)."""
    from oracle import philox
    prob = config_small()
    nw, seed = 24, 77
    ctx = pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, dt=0.01,
                    seed=seed, prec="bf16x3")
    ctx.set_graphs(graphs)
    for steps, energy_every in ((1, 1), (1, 0), (3, 2), (2, 1)):
        step0 = ctx.get_walkers()[3]
        ctx.run(steps, energy_every, 0, 0)
        x, _ = ctx.get_fields()
        ref = philox.normals(seed, step0 + steps - 1, nw, prob.naux)
        assert np.array_equal(x.view(np.uint64), ref.view(np.uint64)), (steps, energy_every)
    ctx.local_energy()          # draws the normals of the current step ...
    step0 = ctx.get_walkers()[3]
    ctx.propagate(1)            # ... which this step uses
    x, _ = ctx.get_fields()
    assert np.array_equal(x.view(np.uint64), philox.normals(seed, step0, nw, prob.naux).view(np.uint64))
    ctx.close()
