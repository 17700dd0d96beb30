"""FP64 CPU oracle of the element-local network of the learned initial guess
(test infrastructure only; see oracle/__init__.py for who may call it).

The paper has no learned component; this follows the plain definitions:
  H1 = relu(X W1^T + b1),  H2 = relu(H1 W2^T + b2),  Y = H2 W3^T + b3
  L  = (1 / (2 R O)) sum_{r < R, o < O} (Y - T)^2       (R rows, O outputs)
and its gradients by the chain rule; Adam (Kingma & Ba 2015) with bias
correction.  The energy-norm variant replaces the mean square by
d.K(d) / (2 R O) for a symmetric positive semi-definite K (for a guess
network on a mesh: K = A_e + lambda B_e element by element).  An optional rounding function q is applied where a reduced-
precision implementation stores values (hidden activations H1, H2; the
back-propagated dY, dA2, dA1), so that both sides take the ReLU decisions on
the same values; the arithmetic stays FP64.  Pinned by a finite-difference
check in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def _ident(a):
    return a


def forward(p, X, q=_ident):
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = q(np.maximum(Z2, 0.0))
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (H1, H2)


def loss_and_grads(p, X, T, rows=None, outs=None, q=_ident, K=None):
    """Loss and gradients over the first `rows` rows and `outs` outputs.

    K (optional): a symmetric positive semi-definite linear map of the error
    block d = (Y - T)[:rows, :outs]; the loss is then the K-norm
    L = d.K(d) / (2 rows outs), whose gradient in Y is K(d) / (rows outs)
    (the mean square is K = identity)."""
    R = X.shape[0] if rows is None else rows
    O = p["W3"].shape[0] if outs is None else outs
    Y, (H1, H2) = forward(p, X, q)
    E = np.zeros_like(Y)
    E[:R, :O] = Y[:R, :O] - T[:R, :O]
    if K is None:
        L = 0.5 * float(np.sum(E * E)) / (R * O)
    else:
        KE = np.asarray(K(E[:R, :O].copy()), dtype=np.float64).reshape(R, O)
        L = 0.5 * float(np.sum(E[:R, :O] * KE)) / (R * O)
        E = np.zeros_like(Y)
        E[:R, :O] = KE
    dY = q(E / (R * O))
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dA2 = q((dY @ p["W3"]) * (H2 > 0))
    g["W2"] = dA2.T @ H1
    g["b2"] = dA2.sum(0)
    dA1 = q((dA2 @ p["W2"]) * (H1 > 0))
    g["W1"] = dA1.T @ X
    g["b1"] = dA1.sum(0)
    return L, g


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t >= 1), in place on p, m, v."""
    for k in NAMES:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
