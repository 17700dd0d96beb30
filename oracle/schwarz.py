"""Oracle of the hybrid Schwarz preconditioner of the pressure solve (test
infrastructure only: imported by tests and the benchmark's CPU baseline,
never by the library).

The paper (section 3.1) solves the pressure with a Krylov method and "a
hybrid-Schwarz multigrid preconditioner" and gives no formulas; the method
it names is the overlapping Schwarz / fast-diagonalisation preconditioner of
the SEM literature it cites for the numerics (Deville, Fischer & Mund 2002).
The reading implemented here (additive, symmetric; two levels, or three
with an intermediate order M damped by w_M):

  z = M r = sum_e R_e^T A_e^{-1} R_e r  [+ w_M P_M S_M P_M^T r]  +  P A_c^{-1} P^T r

* Local solves.  Subdomain e is element e extended by one GLL point into each
  neighbour (N+3 points per direction).  Along each direction the 1-D
  stiffness and mass of the three elements (left neighbour, e, right
  neighbour; lengths from the element edges) are assembled and restricted to
  the N+3 points, i.e. homogeneous Dirichlet just beyond the overlap.  Points
  outside the domain (no neighbour) and Dirichlet boundary points are
  decoupled (identity rows, zero data).  A_e is the separable operator
  Bz x By x Ax + Bz x Ay x Bx + Az x By x Bx, inverted by fast
  diagonalisation: Ax S = Bx S Lambda with S^T Bx S = I, so
  A_e^{-1} = (Sz x Sy x Sx) diag(1 / (lz + ly + lx)) (Sz x Sy x Sx)^T.
  For axis-aligned tensor-product meshes A_e is exactly the SEM operator on
  the extended subdomain.
* Coarse level.  The trilinear (N = 1) discretisation on the element
  vertices; P interpolates vertex values to the GLL points element by
  element, P^T r sums r / mult into the vertices; A_c^{-1} by CG to 1e-12.
* Krylov.  Flexible PCG (Polak-Ribiere beta), which also tolerates the
  inexact coarse solves of the GPU path.  Restarted flexible GMRES (the
  Krylov method the paper names for the pressure) is here too, to compare
  the two on the same preconditioner.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import Mesh, deriv, gll


def element_lengths(verts: np.ndarray):
    """Mean edge lengths (hx, hy, hz) of every element (vertex v = vx + 2vy + 4vz)."""
    V = np.asarray(verts, dtype=np.float64).reshape(-1, 8, 3)
    hx = 0.25 * sum(np.linalg.norm(V[:, b + 1] - V[:, b], axis=1) for b in (0, 2, 4, 6))
    hy = 0.25 * sum(np.linalg.norm(V[:, b + 2] - V[:, b], axis=1) for b in (0, 1, 4, 5))
    hz = 0.25 * sum(np.linalg.norm(V[:, b + 4] - V[:, b], axis=1) for b in (0, 1, 2, 3))
    return hx, hy, hz


def extended_1d(N, h, hL, hR, hasL, hasR, dirL, dirR):
    """(A, B, valid) on the N+3 extended points of one element along one axis."""
    xi, rho = gll(N)
    D = deriv(N, xi)
    Ah = D.T @ np.diag(rho) @ D
    Bh = np.diag(rho)
    n1, M = N + 1, 3 * N + 1
    A = np.zeros((M, M))
    B = np.zeros((M, M))
    for off, hh in ((0, hL), (N, h), (2 * N, hR)):
        A[off:off + n1, off:off + n1] += (2.0 / hh) * Ah
        B[off:off + n1, off:off + n1] += (hh / 2.0) * Bh
    sel = list(range(N - 1, 2 * N + 2))
    A = A[np.ix_(sel, sel)]
    B = B[np.ix_(sel, sel)]
    valid = np.ones(N + 3, dtype=bool)
    dead = [d for d, c in ((0, not hasL), (1, dirL), (N + 2, not hasR), (N + 1, dirR)) if c]
    for d in dead:
        A[d, :] = 0.0
        A[:, d] = 0.0
        B[d, :] = 0.0
        B[:, d] = 0.0
        A[d, d] = 1.0
        B[d, d] = 1.0
        valid[d] = False
    return A, B, valid


class SchwarzFDM:
    """Additive overlapping Schwarz with fast-diagonalisation local solves."""

    def __init__(self, N, nel, periodic, faces, verts, mesh: Mesh | None = None):
        self.N, self.nel, self.per, self.faces = N, tuple(nel), tuple(periodic), faces
        self.m = mesh if mesh is not None else Mesh(N, nel, periodic, faces, verts)
        E = self.m.E
        n1, ne = N + 1, N + 3
        hs = element_lengths(verts)
        eidx = np.arange(E)
        coord = [eidx % nel[0], (eidx // nel[0]) % nel[1], eidx // (nel[0] * nel[1])]
        stride = [1, nel[0], nel[0] * nel[1]]
        self.S = np.zeros((E, 3, ne, ne))
        self.L = np.zeros((E, 3, ne))
        self.valid = np.zeros((E, 3, ne), dtype=bool)
        move = np.zeros((E, 3, ne, 2), dtype=np.int64)  # (element, local index) of extended point along axis
        for e in range(E):
            for a in range(3):
                c, n = int(coord[a][e]), nel[a]
                hasL, hasR = c > 0 or bool(periodic[a]), c < n - 1 or bool(periodic[a])
                dirL = (not periodic[a]) and c == 0 and bool((faces >> (2 * a)) & 1)
                dirR = (not periodic[a]) and c == n - 1 and bool((faces >> (2 * a + 1)) & 1)
                eL = e - stride[a] if c > 0 else e + (n - 1) * stride[a]
                eR = e + stride[a] if c < n - 1 else e - (n - 1) * stride[a]
                h = hs[a][e]
                hL = hs[a][eL] if hasL else h
                hR = hs[a][eR] if hasR else h
                A, B, valid = extended_1d(N, h, hL, hR, hasL, hasR, dirL, dirR)
                lam, S = sla.eigh(A, B)
                self.S[e, a], self.L[e, a], self.valid[e, a] = S, lam, valid
                for I in range(ne):
                    move[e, a, I] = (eL, N - 1) if I == 0 else ((eR, 1) if I == ne - 1 else (e, I - 1))
        gid = self.m.gid.reshape(E, n1, n1, n1)
        self.gid_ext = np.full((E, ne, ne, ne), -1, dtype=np.int64)
        for e in range(E):
            for K in range(ne):
                for J in range(ne):
                    for I in range(ne):
                        if not (self.valid[e, 0, I] and self.valid[e, 1, J] and self.valid[e, 2, K]):
                            continue
                        ex, i = move[e, 0, I]
                        ey, j = move[e, 1, J]
                        ez, k = move[e, 2, K]
                        e2 = int(ex) + (int(ey) - e) + (int(ez) - e)
                        self.gid_ext[e, K, J, I] = gid[e2, k, j, i]

    def local_solve(self, e, rext):
        """A_e^{-1} rext by fast diagonalisation (rext [K][J][I])."""
        Sx, Sy, Sz = self.S[e]
        t = np.einsum("ai,kji->kja", Sx.T, rext)
        t = np.einsum("bj,kja->kba", Sy.T, t)
        t = np.einsum("ck,kba->cba", Sz.T, t)
        lam = self.L[e, 2][:, None, None] + self.L[e, 1][None, :, None] + self.L[e, 0][None, None, :]
        t = t / lam
        t = np.einsum("ia,cba->cbi", Sx, t)
        t = np.einsum("jb,cbi->cji", Sy, t)
        return np.einsum("kc,cji->kji", Sz, t)

    def apply(self, r):
        """z = sum_e R_e^T A_e^{-1} R_e r for continuous E-layout r."""
        rg = np.zeros(self.m.nglob)
        rg[self.m.gid] = r
        zg = np.zeros(self.m.nglob)
        for e in range(self.m.E):
            g = self.gid_ext[e]
            ok = g >= 0
            rext = np.where(ok, rg[np.where(ok, g, 0)], 0.0)
            u = self.local_solve(e, rext)
            np.add.at(zg, g[ok], u[ok])
        return zg[self.m.gid]


class CoarseLevel:
    """Trilinear (N = 1) coarse correction P A_c^{-1} P^T."""

    def __init__(self, N, nel, periodic, faces, verts, mesh: Mesh):
        self.N, self.m = N, mesh
        self.mc = Mesh(1, nel, periodic, faces, verts)
        xi, _ = gll(N)
        self.J1 = np.stack([(1.0 - xi) / 2.0, (1.0 + xi) / 2.0], axis=1)  # [N+1, 2]

    def restrict(self, r):
        E, n1 = self.m.E, self.N + 1
        rl = (r / self.m.mult).reshape(E, n1, n1, n1)
        J = self.J1
        rc = np.einsum("ia,jb,kc,ekji->ecba", J, J, J, rl).reshape(-1)
        return self.mc.apply_mask(self.mc.dssum(rc))

    def prolong(self, xc):
        E, J = self.m.E, self.J1
        return np.einsum("ia,jb,kc,ecba->ekji", J, J, J, xc.reshape(E, 2, 2, 2)).reshape(-1)

    def apply(self, r, tol=1e-12):
        rc = self.restrict(r)
        if not np.any(rc):
            return np.zeros_like(r)
        xc, _, _, _ = self.mc.pcg(rc, tol=tol, max_iter=100000)
        return self.prolong(xc)


def lagrange_interp(M, N):
    """J[i, a] = l^M_a(xi^N_i): the order-M GLL Lagrange basis evaluated at the
    order-N GLL points (Lagrange's product formula; exactly 1 / 0 where the
    point sets share a node, so element faces map to faces)."""
    xm, _ = gll(M)
    xn, _ = gll(N)
    J = np.zeros((N + 1, M + 1))
    for i, x in enumerate(xn):
        for a in range(M + 1):
            if abs(x - xm[a]) < 1e-14:
                J[i, :] = 0.0
                J[i, a] = 1.0
                break
            J[i, a] = np.prod([(x - xm[b]) / (xm[a] - xm[b]) for b in range(M + 1) if b != a])
    return J


class MidLevel:
    """Intermediate level of the multigrid: the overlapping Schwarz of the
    order-M discretisation on the same elements, reached by element-wise
    interpolation.  P_M x interpolates a continuous order-M field to the
    order-N points; its adjoint in the unique-node products is
    P_M^T r = Q_M Q_M^T J^T (r / mult_N) (masked); the level applies
    P_M S_M P_M^T."""

    def __init__(self, N, M, nel, periodic, faces, verts, mesh: Mesh):
        self.N, self.M, self.m = N, M, mesh
        self.mm = Mesh(M, nel, periodic, faces, verts)
        self.sw = SchwarzFDM(M, nel, periodic, faces, verts, self.mm)
        self.J = lagrange_interp(M, N)

    def restrict(self, r):
        E, n1 = self.m.E, self.N + 1
        rl = (r / self.m.mult).reshape(E, n1, n1, n1)
        J = self.J
        rm = np.einsum("ia,jb,kc,ekji->ecba", J, J, J, rl).reshape(-1)
        return self.mm.apply_mask(self.mm.dssum(rm))

    def prolong(self, xm):
        E, m1, J = self.m.E, self.M + 1, self.J
        return np.einsum("ia,jb,kc,ecba->ekji", J, J, J, xm.reshape(E, m1, m1, m1)).reshape(-1)

    def apply(self, r):
        return self.prolong(self.sw.apply(self.restrict(r)))


class HybridSchwarz:
    """z = S_N r + w_M P_M S_M P_M^T r + P_1 A_1^{-1} P_1^T r (masked): the fine
    overlapping Schwarz, an optional intermediate order-M Schwarz level with
    weight w_M (mid_order = None: two levels) and the trilinear coarse
    level.  The levels are added (symmetric); the intermediate one is damped
    because its correction overlaps the fine level's."""

    def __init__(self, N, nel, periodic, faces, verts, mesh: Mesh | None = None, coarse=True, mid_order=None,
                 mid_weight=0.15):
        self.m = mesh if mesh is not None else Mesh(N, nel, periodic, faces, verts)
        self.sw = SchwarzFDM(N, nel, periodic, faces, verts, self.m)
        self.cl = CoarseLevel(N, nel, periodic, faces, verts, self.m) if coarse else None
        self.mid = MidLevel(N, mid_order, nel, periodic, faces, verts, self.m) if mid_order else None
        self.mid_weight = mid_weight

    def apply(self, r):
        z = self.sw.apply(r)
        if self.mid is not None:
            z = z + self.mid_weight * self.mid.apply(r)
        if self.cl is not None:
            z = z + self.cl.apply(r)
        return self.m.apply_mask(z)

    def apply_multiplicative(self, r):
        """The levels one after the other: the coarse correction x_c, then
        the local solves on the updated residual r - A x_c (one more
        operator application per preconditioning step)."""
        xc = self.m.apply_mask(self.cl.apply(r))
        return self.m.apply_mask(xc + self.sw.apply(r - self.m.apply(xc)))


def fpcg(m: Mesh, b, precond, tol=1e-10, max_iter=5000):
    """Flexible PCG (Polak-Ribiere beta); returns (x, iterations, rel_res)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = m.glsc3(r, z)
    bb = m.glsc3(b, b)
    for it in range(1, max_iter + 1):
        w = m.apply(p)
        alpha = rz / m.glsc3(p, w)
        x += alpha * p
        r_old = r.copy()
        r -= alpha * w
        rel = math.sqrt(m.glsc3(r, r) / bb)
        if rel <= tol:
            return x, it, rel
        z = precond(r)
        rz_new = m.glsc3(r, z)
        beta = (rz_new - m.glsc3(r_old, z)) / rz
        rz = rz_new
        p = z + beta * p
    return x, max_iter, rel


def fgmres(m: Mesh, b, precond, restart=30, tol=1e-10, max_iter=5000):
    """Restarted flexible GMRES(restart), right-preconditioned (the
    preconditioned directions z_j = M v_j are kept, x += Z y), modified
    Gram-Schmidt Arnoldi in the multiplicity-weighted inner product, Givens
    rotations for the least-squares problem; each cycle restarts from the
    true residual.  Returns (x, iterations, rel_res)."""
    x = np.zeros_like(b)
    bn = math.sqrt(m.glsc3(b, b))
    if bn == 0.0:
        return x, 0, 0.0
    it = 0
    while True:
        r = b - m.apply(x)
        beta = math.sqrt(m.glsc3(r, r))
        if beta <= tol * bn or it >= max_iter:
            return x, it, beta / bn
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        k = 0
        for j in range(restart):
            z = precond(V[j])
            Z.append(z)
            w = m.apply(z)
            for i in range(j + 1):
                H[i, j] = m.glsc3(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = math.sqrt(m.glsc3(w, w))
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if abs(g[j + 1]) <= tol * bn or it >= max_iter or d == 0.0:
                break
            V.append(w / math.sqrt(m.glsc3(w, w)))
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
