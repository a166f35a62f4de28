"""GPU tests of the autotuner and of batched uneven systems (one graph launch per step)."""
import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from paper_2406_16238_b300._lib import Batch
from synthetic_inputs import config_batched, config_medium

pytestmark = pytest.mark.gpu


def _ctx(prob, nw, prec, seed):
    return pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, seed=seed,
                     prec=prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_autotune_restores_walkers_and_keeps_accuracy(prec):
    prob = config_medium()
    ref = _ctx(prob, 128, "fp64", 3)
    e_ref = ref.run(6, 1, 5, 0)
    ctx = _ctx(prob, 128, prec, 3)
    ctx.run(2, 1, 5, 0)
    before = ctx.get_walkers()
    t = ctx.autotune(steps=2)
    after = ctx.get_walkers()
    assert after[3] == before[3]
    assert np.array_equal(after[0], before[0]) and np.array_equal(after[2], before[2])
    assert t["tile_cap"] in (1, 2, 4) and t["ms_per_step"] > 0
    e = ctx.run(4, 1, 5, 0)
    d = np.abs(e[:, 0] / e[:, 1] - e_ref[2:, 0] / e_ref[2:, 1])
    assert np.max(d) < 1e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_batch_reproduces_individual_runs(prec):
    probs = config_batched(nsys=4, nmin=18, nmax=60)
    nw = 48
    seeds = [11, 12, 13, 14]
    solo = []
    for p, sd in zip(probs, seeds):
        c = _ctx(p, nw, prec, sd)
        c.set_graphs(False)
        solo.append((c.run(13, 2, 5, 10), c.get_walkers()))
        c.close()
    ctxs = [_ctx(p, nw, prec, sd) for p, sd in zip(probs, seeds)]
    b = Batch(ctxs, mode="graphs")   # the systems' own step graphs: bit for bit the solo runs
    e = b.run(13, energy_every=2, reortho_every=5, comb_every=10)
    assert e.shape == (4, 7, 4)
    for i, c in enumerate(ctxs):
        psi, logo, w, step = c.get_walkers()
        assert step == 13
        assert np.array_equal(e[i], solo[i][0])
        assert np.array_equal(psi, solo[i][1][0]) and np.array_equal(w, solo[i][1][2])
    b.close()
