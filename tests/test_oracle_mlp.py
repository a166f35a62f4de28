"""Pins for the learned-control-variate oracle (CPU only)."""
import numpy as np

from oracle import afqmc as orc
from oracle import mlp
from synthetic_inputs import random_walkers, tiny_problem


def test_backward_matches_central_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init_params(7, seed=3, hidden=6)
    x = rng.standard_normal((5, 7))
    y = rng.standard_normal(5)
    _, grads = mlp.loss_and_grads(params, x, y)
    h = 1e-6
    for i, p in enumerate(params):
        flat = p.reshape(-1)
        for j in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[j]
            flat[j] = old + h
            lp, _ = mlp.loss_and_grads(params, x, y)
            flat[j] = old - h
            lm, _ = mlp.loss_and_grads(params, x, y)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[i].reshape(-1)[j]) < 1e-7 * max(1.0, abs(fd)), (i, j)


def test_adam_fits_a_smooth_target():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((256, 4))
    y = np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2]
    params = mlp.init_params(4, seed=2, hidden=32)
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    first = mlp.loss_and_grads(params, x, y)[0]
    for t in range(1, 1501):
        _, g = mlp.loss_and_grads(params, x, y)
        mlp.adam_step(params, g, m, v, t, 3e-3)
    last = mlp.loss_and_grads(params, x, y)[0]
    assert last < 0.02 * first


def test_features_definition():
    prob = tiny_problem(4, 2, 2, naux=6, seed=7, unrestricted=True)
    st = orc.build_setup(prob.h1e, prob.chol, prob.ecore, 2, 2, prob.psiT, 0.01)
    psi = random_walkers(np.random.default_rng(2), 4, 4, 1, 0.4, prob.psiT)[0]
    _, ta, tb = orc.overlap_theta(st, psi)
    vb = orc.force_bias(st, ta, tb)
    z = mlp.features(np.diag(orc.greens_function(st.phi_a, ta)).real,
                     np.diag(orc.greens_function(st.phi_b, tb)).real, vb)
    assert z.shape == (2 * 4 + 8,)
    assert abs(z[:4].sum() - 2) < 1e-12 and abs(z[4:8].sum() - 2) < 1e-12     # Tr G^s = n_s
    re = vb.real
    assert abs(z[8] - re.mean()) < 1e-14 and abs(z[9] - re.var()) < 1e-14
    from scipy import stats
    assert abs(z[10] - stats.skew(re)) < 1e-10 and abs(z[11] - stats.kurtosis(re, fisher=False)) < 1e-10


def test_control_variate_is_unbiased_and_reduces_to_horvitz_thompson():
    rng = np.random.default_rng(5)
    nw = 40
    w = rng.uniform(0.2, 2.0, nw)
    a = rng.normal(3.0, 0.5, nw)
    k = rng.normal(1.0, 0.3, nw)
    f = k + rng.normal(0.0, 0.02, nw)           # a good surrogate
    exact = np.sum(w * (a - k))
    pi = 0.125
    draws_cv, draws_ht = [], []
    for _ in range(40000):
        sel = rng.random(nw) < pi
        draws_cv.append(mlp.cv_numerator(w, a, k, f, sel, pi))
        draws_ht.append(mlp.cv_numerator(w, a, k, np.zeros(nw), sel, pi))
    draws_cv, draws_ht = np.array(draws_cv), np.array(draws_ht)
    assert abs(draws_cv.mean() - exact) < 4 * draws_cv.std() / np.sqrt(len(draws_cv))
    assert abs(draws_ht.mean() - exact) < 4 * draws_ht.std() / np.sqrt(len(draws_ht))
    assert draws_cv.std() < 0.1 * draws_ht.std()
    # f = 0 is exactly the Horvitz-Thompson estimate of sum w K
    sel = rng.random(nw) < pi
    ht = np.sum(w * a) - np.sum((w * k)[sel]) / pi
    assert abs(mlp.cv_numerator(w, a, k, np.zeros(nw), sel, pi) - ht) < 1e-12
