"""GPU tests of the learned control variate (network kernels, training, estimator)."""
import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from oracle import afqmc as orc
from oracle import mlp
from synthetic_inputs import config_medium, config_small, random_walkers

pytestmark = pytest.mark.gpu


def _flat(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def _ctx(prob, nw, prec="fp32", seed=3):
    return pkg.Afqmc(prob.h1e, prob.chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=nw, seed=seed,
                     prec=prec)


def test_network_forward_and_gradients_match_the_oracle():
    prob = config_small()
    ctx = _ctx(prob, 16)
    ctx.cv_attach(capacity=64, batch=32)
    dim = ctx.cv_dim
    assert dim == 2 * prob.norb + 8
    params = mlp.init_params(dim, seed=4)
    ctx.cv_set_params(_flat(params))
    assert np.array_equal(ctx.cv_get_params(), _flat(params))
    rng = np.random.default_rng(0)
    x = rng.standard_normal((32, dim)).astype(np.float32)
    y = rng.standard_normal(32).astype(np.float32)
    out, loss, grads = ctx.cv_eval(x, y)
    p32 = [p.astype(np.float32).astype(np.float64) for p in params]
    ref_out, _ = mlp.forward(p32, x.astype(np.float64))
    ref_loss, ref_grads = mlp.loss_and_grads(p32, x.astype(np.float64), y.astype(np.float64))
    assert np.allclose(out, ref_out, rtol=0, atol=2e-5 * np.max(np.abs(ref_out)) + 1e-6)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    g = _flat(ref_grads)
    assert np.max(np.abs(grads - g)) < 1e-4 * np.max(np.abs(g))
    for blk_g, blk_ref in zip(np.split(grads, np.cumsum([p.size for p in params])[:-1]), ref_grads):
        assert np.linalg.norm(blk_g - blk_ref.reshape(-1)) <= 1e-4 * max(np.linalg.norm(blk_ref), 1e-12)


def test_network_on_the_tensor_cores_matches_the_oracle():
    """512-row batches run every layer's product of at least 128 x 64 x 64 on the tensor cores (split
    bf16, three products, fp32 accumulation: ~2^-16 relative per product): output, loss and gradients
    against the oracle at 1e-4 relative (the CUDA-core test above holds the binary32 path to 2e-5)."""
    prob = config_medium()
    ctx = _ctx(prob, 16)
    ctx.cv_attach(capacity=1024, batch=512)
    dim = ctx.cv_dim
    assert dim == 2 * prob.norb + 8 and dim >= 64
    params = mlp.init_params(dim, seed=5)
    ctx.cv_set_params(_flat(params))
    rng = np.random.default_rng(1)
    x = rng.standard_normal((512, dim)).astype(np.float32)
    y = rng.standard_normal(512).astype(np.float32)
    out, loss, grads = ctx.cv_eval(x, y)
    p32 = [p.astype(np.float32).astype(np.float64) for p in params]
    ref_out, _ = mlp.forward(p32, x.astype(np.float64))
    ref_loss, ref_grads = mlp.loss_and_grads(p32, x.astype(np.float64), y.astype(np.float64))
    assert np.allclose(out, ref_out, rtol=0, atol=1e-4 * np.max(np.abs(ref_out)))
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    for blk_g, blk_ref in zip(np.split(grads, np.cumsum([p.size for p in params])[:-1]), ref_grads):
        assert np.linalg.norm(blk_g - blk_ref.reshape(-1)) <= 1e-4 * max(np.linalg.norm(blk_ref), 1e-12)
    assert ctx.launch_count() > 0
    ctx.close()


def _trained_context(prec, nw=640, steps=12, epochs=40):
    prob = config_medium()
    ctx = _ctx(prob, nw, prec=prec, seed=7)
    ctx.cv_attach(capacity=nw * steps, batch=512, sample_frac=0.125, seed=2)
    n = ctx.cv_collect(steps, reortho_every=5, comb_every=10)
    assert n == nw * steps
    losses = ctx.cv_train(epochs, lr=1e-3)
    return prob, ctx, losses


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_training_reduces_the_loss(prec):
    _, ctx, losses = _trained_context(prec, epochs=30)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.1 * losses[0], losses


def test_control_variate_is_unbiased_and_the_trained_network_reduces_variance():
    prob, ctx, _ = _trained_context("fp32")
    psi, logo, w, step = ctx.get_walkers()
    ctx.set_walkers(psi, w, step)
    exact = ctx.local_energy()                       # every walker's exact exchange
    ctx.cv_enable(True)

    def draws(ndraw):
        out = []
        for k in range(ndraw):
            ctx.set_walkers(psi, w, 10000 + k)        # the subsample follows the step counter
            out.append(ctx.local_energy())
        return np.array(out)

    trained = draws(160)
    assert np.allclose(trained[:, 1], exact[1], rtol=1e-12)
    e_tr = trained[:, 0]
    se = e_tr.std(ddof=1) / np.sqrt(len(e_tr))
    assert abs(e_tr.mean() - exact[0]) < 4.0 * se + 1e-9 * abs(exact[0]), (e_tr.mean(), exact[0], se)
    # the same estimator with the untrained (randomly initialised) network: same cost, no learning
    ctx.cv_set_params(_flat(mlp.init_params(ctx.cv_dim, seed=9)))
    untrained = draws(160)[:, 0]
    se_u = untrained.std(ddof=1) / np.sqrt(len(untrained))
    assert abs(untrained.mean() - exact[0]) < 4.0 * se_u + 1e-9 * abs(exact[0])
    assert e_tr.std() < 0.5 * untrained.std(), (e_tr.std(), untrained.std())


def test_control_variate_run_tracks_the_plain_energy():
    """From the same walkers and fields, the CV run's per-step energies scatter around the plain ones."""
    prob, ctx, _ = _trained_context("bf16x3", steps=8, epochs=20)
    psi, logo, w, step = ctx.get_walkers()
    ctx.cv_enable(True)
    e_cv = ctx.run(30, energy_every=1, reortho_every=5, comb_every=0)
    ctx.cv_enable(False)
    ctx.set_walkers(psi, w, step)
    e_plain = ctx.run(30, energy_every=1, reortho_every=5, comb_every=0)
    a, b = e_cv[:, 0] / e_cv[:, 1], e_plain[:, 0] / e_plain[:, 1]
    d = a - b
    assert np.all(np.isfinite(a))
    assert abs(d.mean()) < 5 * d.std(ddof=1) / np.sqrt(len(d)) + 1e-4, (d.mean(), d.std())
    assert np.max(np.abs(d)) < 0.05


def test_async_readout_in_the_control_variate_form():
    """afqmc_local_energy_async copies the control-variate estimator's sums as the synchronous call returns them."""
    import torch
    prob, ctx, _ = _trained_context("bf16x3", steps=4, epochs=5)
    psi, logo, w, step = ctx.get_walkers()
    ctx.cv_enable(True)
    ref = ctx.local_energy()
    ctx.set_walkers(psi, w, step)
    out = torch.zeros(4, dtype=torch.float64).pin_memory().numpy()
    ctx.local_energy_async(out)
    ctx.synchronize(60.0)
    ctx.cv_enable(False)
    assert np.all(np.isfinite(out)) and out[1] > 0
    assert np.array_equal(out, ref)
