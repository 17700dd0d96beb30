"""Pins of the FP64 MLP oracle: central finite differences of the loss
against the analytic gradients (mean square and energy norm), the energy
norm with K = identity reducing to the mean square, the element-stiffness
energy's invariants, and Adam's first step (a closed form: every parameter
moves by -lr g / (|g| + eps))."""
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


def _fd_check(p, X, T, rng, **kw):
    L, g = mlp.loss_and_grads(p, X, T, **kw)
    h = 1e-6
    for k in mlp.NAMES:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = mlp.loss_and_grads(p, X, T, **kw)
            flat[idx] = old - h
            Lm, _ = mlp.loss_and_grads(p, X, T, **kw)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (k, idx, fd, an)


def test_energy_norm_gradients_match_finite_differences():
    """K: a different random symmetric positive definite matrix per row."""
    rng = np.random.default_rng(4)
    p = {k: v.astype(np.float64) for k, v in _params().items()}
    X = rng.standard_normal((10, 12))
    T = rng.standard_normal((10, 6))
    Ms = []
    for _ in range(9):
        A = rng.standard_normal((5, 5))
        Ms.append(A @ A.T + 0.1 * np.eye(5))

    def K(d):
        return np.stack([Ms[r] @ d[r] for r in range(d.shape[0])])

    _fd_check(p, X, T, rng, rows=9, outs=5, K=K)


def test_energy_norm_with_identity_is_the_mean_square():
    rng = np.random.default_rng(5)
    p = {k: v.astype(np.float64) for k, v in _params().items()}
    X = rng.standard_normal((10, 12))
    T = rng.standard_normal((10, 6))
    L1, g1 = mlp.loss_and_grads(p, X, T, rows=8, outs=6)
    L2, g2 = mlp.loss_and_grads(p, X, T, rows=8, outs=6, K=lambda d: d)
    assert abs(L1 - L2) <= 1e-15 * L1
    for k in mlp.NAMES:
        np.testing.assert_allclose(g2[k], g1[k], rtol=1e-14, atol=1e-15)


def test_element_energy_invariants():
    """The element-stiffness energy of a guess network's error: an
    element-wise constant error costs lambda |B_e| c^2 only (constants are
    the null space of A_e), and a linear error x costs the element volume
    (|grad x|^2 = 1 integrated) -- exact for GLL quadrature, which
    integrates the degree-2N-2 product exactly on an affine element."""
    import oracle
    case = inputs.BoxCase("e", 3, (2, 2, 1), (0, 0, 0), 0, perturb_amp=0.0, seed=0)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices())
    lam = 0.7

    def K(d):
        return (om.ax_local(d.reshape(-1)) + lam * om.B.reshape(-1) * d.reshape(-1)).reshape(d.shape)

    c = np.arange(1.0, om.E + 1.0)[:, None] * np.ones((om.E, om.npt))
    Bsum = om.B.reshape(om.E, om.npt).sum(1)
    np.testing.assert_allclose(np.sum(c * K(c), axis=1), lam * Bsum * c[:, 0] ** 2, rtol=1e-12)
    x = om.xyz[0].reshape(om.E, om.npt)
    Ax = om.ax_local(x.reshape(-1)).reshape(om.E, om.npt)
    np.testing.assert_allclose(np.sum(x * Ax, axis=1), Bsum, rtol=1e-12)


def test_averaged_energy_invariants():
    """The energy of the averaged correction, K = S M^-1 (A_L + lambda B)
    M^-1 S (S: sum of the copies of every node, M: multiplicity): symmetric;
    on a continuous error it equals the element energy sum_e d_e (A_e +
    lambda B_e) d_e (M^-1 S d = d); and it depends on a discontinuous error
    only through its average."""
    import oracle
    case = inputs.BoxCase("a", 3, (2, 2, 2), (1, 0, 0), 0, perturb_amp=0.05, seed=2)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices())
    lam = 0.5

    def Ke(d):
        return om.ax_local(d) + lam * om.B.reshape(-1) * d

    def K(d):
        return om.dssum(Ke(om.dssum(d) * om.minv) * om.minv)

    rng = np.random.default_rng(6)
    u, v = rng.standard_normal(om.nloc), rng.standard_normal(om.nloc)
    assert abs(u @ K(v) - v @ K(u)) <= 1e-12 * abs(u @ K(v))
    c = om.scatter(rng.standard_normal(om.nglob))  # continuous
    assert abs(c @ K(c) - c @ Ke(c)) <= 1e-12 * abs(c @ Ke(c))
    w = om.dssum(u) * om.minv
    assert abs(u @ K(u) - w @ Ke(w)) <= 1e-12 * abs(w @ Ke(w))
