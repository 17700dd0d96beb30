"""Pins of the FP64 MLP oracle: central finite differences of the loss
against the analytic gradients, and Adam's first step (a closed form: every
parameter moves by -lr g / (|g| + eps))."""
import numpy as np

from oracle import mlp
from paper_2405_05640_gb300 import inputs


def _params(I=12, H=8, O=6, seed=0):
    return inputs.mlp_init(I, H, O, seed)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = {k: v.astype(np.float64) for k, v in _params().items()}
    X = rng.standard_normal((10, 12))
    T = rng.standard_normal((10, 6))
    L, g = mlp.loss_and_grads(p, X, T, rows=9, outs=5)
    h = 1e-6
    for k in mlp.NAMES:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = mlp.loss_and_grads(p, X, T, rows=9, outs=5)
            flat[idx] = old - h
            Lm, _ = mlp.loss_and_grads(p, X, T, rows=9, outs=5)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (k, idx, fd, an)


def test_padding_rows_and_outputs_do_not_contribute():
    rng = np.random.default_rng(2)
    p = {k: v.astype(np.float64) for k, v in _params().items()}
    X = rng.standard_normal((10, 12))
    T = rng.standard_normal((10, 6))
    L1, g1 = mlp.loss_and_grads(p, X[:7], T[:7, :4], rows=7, outs=4)
    X2, T2 = X.copy(), T.copy()
    X2[7:] = 123.0
    T2[:, 4:] = -50.0
    L2, g2 = mlp.loss_and_grads(p, X2, T2, rows=7, outs=4)
    assert abs(L1 - L2) < 1e-14
    for k in mlp.NAMES:
        np.testing.assert_allclose(g1[k], g2[k], atol=1e-14)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(3)
    p = {k: v.astype(np.float64) for k, v in _params().items()}
    g = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    q = {k: x.copy() for k, x in p.items()}
    mlp.adam(q, g, m, v, 1, lr=1e-3)
    for k in mlp.NAMES:
        np.testing.assert_allclose(q[k] - p[k], -1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-9, atol=1e-15)
