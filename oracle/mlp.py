"""Learned control variate for the exchange energy: FP64 oracle (TEST INFRASTRUCTURE ONLY).

The mixed estimator of Eq. 9 is split as E_L = A - K with A = Re(E0 + E1 + J)
(cheap: one-body, Coulomb) and K = Re(1/2 sum_{g s} Tr T T) (the exchange, the
dominant cost).  A small MLP f(z) predicts K from per-walker features z;
exact K on a random subsample keeps the estimate unbiased:

  ENumer_CV = sum_i w_i (A_i - f_i) - (1/pi) sum_{i in S} w_i (K_i - f_i),

S drawn with independent inclusion probability pi per walker, so that
E_S[ENumer_CV] = sum_i w_i (A_i - K_i) = ENumer for any f (Horvitz-Thompson
correction).  With f = 0 it is the plain Horvitz-Thompson subsample estimate.

Features z (2N + 8 values): diag Re G^alpha, diag Re G^beta, and the mean,
variance, skewness and kurtosis (non-excess, over gamma) of Re vbias and of
Im vbias.  Network: z -> 256 -> 256 -> 256 -> 1, tanh hidden activations,
linear output; parameters stored "in x out" (h = x W + b).  Loss: mean squared
error.  Optimiser: Adam (Kingma & Ba 2015) with beta1 = 0.9, beta2 = 0.999,
eps = 1e-8.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 256


def features(diag_ga, diag_gb, vbias):
    """z for one walker: diag Re G^a [N], diag Re G^b [N], vbias [X] complex."""
    out = [np.asarray(diag_ga, float), np.asarray(diag_gb, float)]
    for part in (vbias.real, vbias.imag):
        m = part.mean()
        c = part - m
        var = (c * c).mean()
        sd = np.sqrt(var)
        if sd > 0:
            skew = ((c / sd) ** 3).mean()
            kurt = ((c / sd) ** 4).mean()
        else:
            skew = kurt = 0.0
        out.append(np.array([m, var, skew, kurt]))
    return np.concatenate(out)


def init_params(dim, seed, hidden=HIDDEN):
    """Glorot-uniform weights, zero biases: [W1, b1, W2, b2, W3, b3, W4, b4]."""
    rng = np.random.default_rng(seed)
    sizes = [dim, hidden, hidden, hidden, 1]
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / (a + b))
        params.append(rng.uniform(-lim, lim, (a, b)))
        params.append(np.zeros(b))
    return params


def forward(params, x):
    """Returns (output [B], activations list)."""
    acts = [x]
    h = x
    for layer in range(3):
        h = np.tanh(h @ params[2 * layer] + params[2 * layer + 1])
        acts.append(h)
    out = (h @ params[6] + params[7])[:, 0]
    return out, acts


def loss_and_grads(params, x, y):
    """MSE loss and its gradient with respect to every parameter (manual backward)."""
    out, acts = forward(params, x)
    bsz = x.shape[0]
    r = out - y
    loss = float(np.mean(r * r))
    dz = (2.0 / bsz) * r[:, None]                    # d loss / d output
    grads = [None] * 8
    grads[6] = acts[3].T @ dz
    grads[7] = dz.sum(axis=0)
    da = dz @ params[6].T
    for layer in (2, 1, 0):
        dzl = da * (1.0 - acts[layer + 1] ** 2)      # tanh'
        grads[2 * layer] = acts[layer].T @ dzl
        grads[2 * layer + 1] = dzl.sum(axis=0)
        da = dzl @ params[2 * layer].T
    return loss, grads


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); updates params, m, v in place."""
    for i in range(len(params)):
        m[i] = b1 * m[i] + (1 - b1) * grads[i]
        v[i] = b2 * v[i] + (1 - b2) * grads[i] ** 2
        mh = m[i] / (1 - b1 ** t)
        vh = v[i] / (1 - b2 ** t)
        params[i] = params[i] - lr * mh / (np.sqrt(vh) + eps)


def cv_numerator(w, a, k, f, selected, pi):
    """ENumer_CV for one step (see module docstring); `selected` is a boolean mask."""
    w = np.asarray(w, float)
    base = np.sum(w * (a - f))
    corr = np.sum((w * (k - f))[selected]) / pi
    return base - corr
