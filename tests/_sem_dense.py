"""Independent brute-force SEM assembly used to pin the oracle.

Nothing here calls the oracle's numerics: GLL nodes come from numpy's Legendre
class, Lagrange derivatives from the barycentric formula (Berrut & Trefethen,
SIAM Review 2004), the Jacobian from the analytic derivative of the trilinear
map, and global nodes are identified by matching physical coordinates.  The
element stiffness is the Galerkin form  K_e[p, q] = sum over GLL quadrature
points of  rho_i rho_j rho_k det J  grad phi_p . grad phi_q.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def gll_numpy(N: int):
    """GLL nodes (roots of P_N' plus the end points) and weights via numpy."""
    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c)))) if N > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    PN = npleg.legval(x, c)
    w = 2.0 / (N * (N + 1) * PN ** 2)
    return x, w


def bary_weights(x):
    n = len(x)
    lam = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                lam[j] /= (x[j] - x[k])
    return lam


def bary_deriv(x):
    """D_ij = l_j'(x_i) from barycentric weights."""
    lam = bary_weights(x)
    n = len(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = lam[j] / lam[i] / (x[i] - x[j])
        D[i, i] = -D[i].sum()
    return D


def trilinear_jacobian(V, r, s, t):
    """J[a, b] = d x_a / d r_b of the trilinear map of vertices V[8, 3]."""
    f = [np.array([0.5 * (1 - q), 0.5 * (1 + q)]) for q in (r, s, t)]
    df = np.array([-0.5, 0.5])
    J = np.zeros((3, 3))
    for v in range(8):
        b = (v & 1, (v >> 1) & 1, (v >> 2) & 1)
        g = [df[b[0]] * f[1][b[1]] * f[2][b[2]],
             f[0][b[0]] * df[b[1]] * f[2][b[2]],
             f[0][b[0]] * f[1][b[1]] * df[b[2]]]
        for a in range(3):
            for d in range(3):
                J[a, d] += V[v, a] * g[d]
    return J


def trilinear_point(V, r, s, t):
    f = [np.array([0.5 * (1 - q), 0.5 * (1 + q)]) for q in (r, s, t)]
    x = np.zeros(3)
    for v in range(8):
        x += V[v] * f[0][v & 1] * f[1][(v >> 1) & 1] * f[2][(v >> 2) & 1]
    return x


def element_stiffness(N, V):
    x, w = gll_numpy(N)
    D = bary_deriv(x)
    n1 = N + 1
    npt = n1 ** 3
    K = np.zeros((npt, npt))
    M = np.zeros(npt)
    # grad_r phi_p at quadrature point q: phi_p(q) = delta in two directions
    for k in range(n1):
        for j in range(n1):
            for i in range(n1):
                q = i + n1 * (j + n1 * k)
                J = trilinear_jacobian(V, x[i], x[j], x[k])
                det = np.linalg.det(J)
                Jinv = np.linalg.inv(J)  # Jinv[b, a] = d r_b / d x_a
                wq = w[i] * w[j] * w[k] * det
                M[q] = wq
                # reference gradients of all basis functions at point q
                gr = np.zeros((npt, 3))
                for kk in range(n1):
                    for jj in range(n1):
                        for ii in range(n1):
                            p = ii + n1 * (jj + n1 * kk)
                            gr[p, 0] = D[i, ii] * (j == jj) * (k == kk)
                            gr[p, 1] = (i == ii) * D[j, jj] * (k == kk)
                            gr[p, 2] = (i == ii) * (j == jj) * D[k, kk]
                gx = gr @ Jinv  # physical gradient: sum_b dphi/dr_b dr_b/dx_a
                K += wq * gx @ gx.T
    return K, M


def physical_points(N, verts):
    x, _ = gll_numpy(N)
    n1 = N + 1
    E = verts.shape[0]
    P = np.zeros((E, n1 ** 3, 3))
    for e in range(E):
        for k in range(n1):
            for j in range(n1):
                for i in range(n1):
                    P[e, i + n1 * (j + n1 * k)] = trilinear_point(verts[e], x[i], x[j], x[k])
    return P


def coordinate_numbering(P, period=None, decimals=9):
    """Global ids by matching coordinates (wrapped into the period where an
    axis is periodic)."""
    Q = P.reshape(-1, 3).copy()
    if period is not None:
        for a in range(3):
            if period[a]:
                Q[:, a] = np.mod(Q[:, a], period[a])
                Q[np.isclose(Q[:, a], period[a]), a] = 0.0
    keys = np.round(Q, decimals)
    keys[keys == 0.0] = 0.0  # fold -0.0
    _, gid = np.unique(keys, axis=0, return_inverse=True)
    return gid.reshape(-1), int(gid.max()) + 1


def assemble(N, verts, period=None):
    """Dense assembled stiffness and lumped mass over coordinate-matched nodes."""
    P = physical_points(N, verts)
    gid, ng = coordinate_numbering(P, period)
    E = verts.shape[0]
    npt = (N + 1) ** 3
    A = np.zeros((ng, ng))
    Bm = np.zeros(ng)
    for e in range(E):
        K, M = element_stiffness(N, verts[e])
        g = gid[e * npt:(e + 1) * npt]
        np.add.at(A, (g[:, None], g[None, :]), K)
        np.add.at(Bm, g, M)
    return A, Bm, gid, ng, P
