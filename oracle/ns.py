"""FP64 CPU oracle of one incompressible Navier-Stokes time step (test
infrastructure only; see oracle/__init__.py for who may call it).

The paper's governing equations are Eq. 1 (section 3):
    div v = 0,   dv/dt + (v . grad) v = -grad p + (1/Re) lap v + F.
Section 3.1 says the velocity and pressure are split as in Karniadakis,
Israeli & Orszag (1991) and that the pressure is solved with a Krylov method
each step, the velocity with CG; it does not give the scheme.  The reading
taken here: BDF_k / EXT_k (k = min(step+1, 2)), P_N-P_N collocation, no
dealiasing, on a fully periodic box:

  NL^n   = -(u^n . grad) u^n                          (collocation)
  S      = sum_j (b_j / dt) u^{n+1-j}                 BDF history
  F      = S + sum_j a_j NL^{n+1-j}                   EXT extrapolation
  A p    = Q Q^T wdiv(F),   wdiv(F)_i = int grad(phi_i) . F
           (singular: right-hand side projected to zero unique-node mean,
            solution shifted to zero mean)
  (nu A + (b0/dt) B) u_c = Q Q^T [B (F_c - d p/dx_c)],  c = 1..3
  BDF1: b0 = 1, b1 = 1;  EXT1: a1 = 1
  BDF2: b0 = 3/2, b1 = 2, b2 = -1/2;  EXT2: a1 = 2, a2 = -1

Derivatives along the reference directions are the contractions with D
written out with numpy.einsum; the inverse Jacobian comes from the C oracle.

Higher order and dealiasing (the splitting the paper cites is the high-order
one of Karniadakis, Israeli & Orszag 1991: BDF_k / EXT_k up to k = 3):
  BDF3: b0 = 11/6, b = (3, -3/2, 1/3);  EXT3: a = (3, -3, 1),
ramping k = 1, 2, 3 over the first steps.  Dealiased advection (over-
integration on M = 3(N+1)/2 Gauss-Legendre points per direction, the usual
3/2 rule for SEM): the weak form
  W_c[i] = int phi_i (u . grad) u_c dx
         = sum_q w_q (sum_a [sum_m detJ dr_a/dx_m u_m] d u_c / d r_a) phi_i  at the Gauss points,
with u and d u_c / d r_a interpolated from the GLL points and detJ dr_a/dx_m
= cofactor C[m][a] of the trilinear Jacobian evaluated at the Gauss points;
the advection term is then NL_c = -(Q Q^T W_c) / (Q Q^T B).
"""
from __future__ import annotations

import numpy as np

from . import Mesh, gll, inverse_jacobian

BDF = {1: (1.0, (1.0,)), 2: (1.5, (2.0, -0.5)), 3: (11.0 / 6.0, (3.0, -1.5, 1.0 / 3.0))}
EXT = {1: (1.0,), 2: (2.0, -1.0), 3: (3.0, -3.0, 1.0)}


def dealias_points(N: int) -> int:
    """M = 3(N+1)/2 Gauss points per direction (rounded up)."""
    return (3 * (N + 1) + 1) // 2


def lagrange_matrix(xi: np.ndarray, z: np.ndarray) -> np.ndarray:
    """J[q, i] = l_i(z_q), the Lagrange basis on the nodes xi at the points z
    (product formula)."""
    J = np.ones((len(z), len(xi)))
    for i in range(len(xi)):
        for j in range(len(xi)):
            if j != i:
                J[:, i] *= (z - xi[j]) / (xi[i] - xi[j])
    return J


def fine_metric(verts: np.ndarray, z: np.ndarray, w: np.ndarray) -> np.ndarray:
    """W[e, m, a, q] = w_q detJ dr_a/dx_m at the tensor points q = (qi, qj, qk)
    (qi fastest) of the 1-D points z with weights w: for the trilinear map
    x(r,s,t) = sum_v V_v prod (1 +- r)/2, detJ dr_a/dx_m is the cofactor
    C[m][a] of J_ab = dx_a/dr_b (computed from vertex offsets)."""
    verts = np.asarray(verts, dtype=np.float64).reshape(-1, 8, 3)
    M = len(z)
    r = z[None, None, :]
    s = z[None, :, None]
    t = z[:, None, None]
    lo = lambda x: 0.5 * (1.0 - x)
    hi = lambda x: 0.5 * (1.0 + x)
    f = [(lo, -0.5), (hi, 0.5)]
    J = np.zeros((verts.shape[0], 3, 3, M, M, M))
    for v in range(1, 8):
        bx, by, bz = v & 1, (v >> 1) & 1, (v >> 2) & 1
        gr = f[bx][1] * f[by][0](s) * f[bz][0](t) * np.ones_like(r)
        gs = f[bx][0](r) * f[by][1] * f[bz][0](t) * np.ones_like(s)
        gt = f[bx][0](r) * f[by][0](s) * f[bz][1] * np.ones_like(t)
        X = verts[:, v, :] - verts[:, 0, :]
        for a in range(3):
            J[:, a, 0] += X[:, a, None, None, None] * gr
            J[:, a, 1] += X[:, a, None, None, None] * gs
            J[:, a, 2] += X[:, a, None, None, None] * gt
    C = np.zeros_like(J)
    for a in range(3):
        for b in range(3):
            a1, a2 = (a + 1) % 3, (a + 2) % 3
            b1, b2 = (b + 1) % 3, (b + 2) % 3
            C[:, a, b] = J[:, a1, b1] * J[:, a2, b2] - J[:, a1, b2] * J[:, a2, b1]
    wq = (w[:, None, None] * w[None, :, None] * w[None, None, :])  # [qk, qj, qi]
    Wm = np.zeros((verts.shape[0], 3, 3, M ** 3))
    for m in range(3):
        for a in range(3):
            Wm[:, m, a] = (wq * C[:, m, a]).reshape(verts.shape[0], -1)
    return Wm


class NSOracle:
    def __init__(self, N, nel, verts, Re, periodic=(1, 1, 1), order=2, dealias=False, M=None):
        self.order, self.dealias = order, dealias
        self.m = Mesh(N, nel, periodic, 0, verts)
        self.N, self.E, self.n1 = N, self.m.E, N + 1
        self.nu = 1.0 / Re
        self.RX = inverse_jacobian(N, verts)  # [E, 9, npt]
        self.B = self.m.B.reshape(self.E, -1)
        self.u = [np.zeros(self.m.nloc) for _ in range(3)]
        self.u_hist = []   # previous velocities, most recent first
        self.nl_hist = []  # previous advection terms, most recent first
        self.p = np.zeros(self.m.nloc)
        self.steps = 0
        self.verts = np.asarray(verts, dtype=np.float64).reshape(-1, 8, 3)
        self.M = M if M is not None else dealias_points(N)
        if dealias:
            self.binv = 1.0 / self.m.dssum(self.m.B.reshape(-1))

    # ---- operators
    def _cube(self, f):
        return np.reshape(f, (self.E, self.n1, self.n1, self.n1))  # [e, k, j, i]

    def ref_derivs(self, f):
        """(df/dr, df/ds, df/dt) by contraction with D along i, j, k."""
        D, F = self.m.D, self._cube(f)
        dr = np.einsum("il,ekjl->ekji", D, F)
        ds = np.einsum("jl,ekli->ekji", D, F)
        dt = np.einsum("kl,elji->ekji", D, F)
        return [x.reshape(self.E, -1) for x in (dr, ds, dt)]

    def grad(self, f):
        """Collocation gradient: df/dx_m = sum_a (dr_a/dx_m) df/dr_a."""
        d = self.ref_derivs(f)
        return [sum(self.RX[:, 3 * a + m] * d[a] for a in range(3)).reshape(-1) for m in range(3)]

    def advect(self, u):
        """NL_c = -sum_m u_m d u_c / d x_m (collocation)."""
        out = []
        for c in range(3):
            g = self.grad(u[c])
            out.append(-(u[0] * g[0] + u[1] * g[1] + u[2] * g[2]))
        return out

    def advect_weak(self, u, M=None):
        """W_c = int phi_i (u . grad) u_c by Gauss quadrature with M points per
        direction (local, not assembled)."""
        M = self.M if M is None else M
        N1, E = self.n1, self.E
        z, w = np.polynomial.legendre.leggauss(M)
        xi = gll(self.N)[0]
        J = lagrange_matrix(xi, z)
        JD = J @ self.m.D
        Wm = fine_metric(self.verts, z, w)

        def interp(f, Ji, Jj, Jk):
            # one direction at a time (i, then j, then k)
            F = np.reshape(f, (E, N1, N1, N1))
            F = np.einsum("qi,ekji->ekjq", Ji, F)
            F = np.einsum("rj,ekjq->ekrq", Jj, F)
            return np.einsum("sk,ekrq->esrq", Jk, F).reshape(E, -1)

        uf = [interp(u[m], J, J, J) for m in range(3)]
        ct = [sum(Wm[:, m, a] * uf[m] for m in range(3)) for a in range(3)]
        out = []
        for c in range(3):
            dr = interp(u[c], JD, J, J)
            ds = interp(u[c], J, JD, J)
            dt = interp(u[c], J, J, JD)
            fq = (ct[0] * dr + ct[1] * ds + ct[2] * dt).reshape(E, M, M, M)
            g = np.einsum("sk,esrq->ekrq", J, fq)
            g = np.einsum("rj,ekrq->ekjq", J, g)
            out.append(np.einsum("qi,ekjq->ekji", J, g).reshape(-1))
        return out

    def advect_dealiased(self, u):
        """NL_c = -(Q Q^T W_c) / (Q Q^T B)."""
        W = self.advect_weak(u)
        return [-self.binv * self.m.dssum(Wc) for Wc in W]

    def wdiv(self, F):
        """Local weak divergence: int grad(phi_i) . F by GLL quadrature,
        sum_a D_a^T [B sum_m (dr_a/dx_m) F_m]."""
        D = self.m.D
        phi = [self._cube(self.B * sum(self.RX[:, 3 * a + m] * np.reshape(F[m], (self.E, -1))
                                       for m in range(3))) for a in range(3)]
        w = (np.einsum("li,ekjl->ekji", D, phi[0]) + np.einsum("lj,ekli->ekji", D, phi[1]) +
             np.einsum("lk,elji->ekji", D, phi[2]))
        return w.reshape(-1)

    def unique_mean(self, f):
        return float(np.sum(f / self.m.mult) / self.m.nglob)

    def kinetic_energy(self, u=None):
        u = self.u if u is None else u
        w = self.m.B.reshape(-1) / self.m.mult
        return 0.5 * float(sum(np.sum(w * uc * uc) for uc in u)) / float(np.sum(w))

    # ---- state
    def set_velocity(self, u):
        self.u = [np.asarray(x, dtype=np.float64).reshape(-1).copy() for x in u]
        self.u_hist, self.nl_hist, self.steps = [], [], 0

    def pressure_rhs(self, F):
        b = self.m.dssum(self.wdiv(F))
        return b - self.unique_mean(b)

    def solve_pressure(self, b, tol, p0=None):
        self.m.set_helmholtz(1.0, 0.0)
        p, it, rr, st = self.m.pcg(b, x0=p0, tol=tol, max_iter=100000)
        return p - self.unique_mean(p), it, st

    def step(self, dt, p_tol=1e-12, v_tol=1e-12):
        k = min(self.steps + 1, self.order)
        b0, bj = BDF[k]
        aj = EXT[k]
        nl = self.advect_dealiased(self.u) if self.dealias else self.advect(self.u)
        us = [self.u] + self.u_hist
        nls = [nl] + self.nl_hist
        F = []
        for c in range(3):
            S = sum((bj[j] / dt) * us[j][c] for j in range(k))
            F.append(S + sum(aj[j] * nls[j][c] for j in range(k)))
        bp = self.pressure_rhs(F)
        self.p, pit, pst = self.solve_pressure(bp, p_tol, self.p)
        gp = self.grad(self.p)
        self.m.set_helmholtz(self.nu, b0 / dt)
        unew, vits = [], []
        for c in range(3):
            rhs = self.m.dssum(self.m.B.reshape(-1) * (F[c] - gp[c]))
            uc, it, rr, st = self.m.pcg(rhs, x0=self.u[c], tol=v_tol, max_iter=100000)
            unew.append(uc)
            vits.append(it)
        self.m.set_helmholtz(1.0, 0.0)
        keep = self.order - 1
        self.u_hist = ([self.u] + self.u_hist)[:keep]
        self.nl_hist = ([nl] + self.nl_hist)[:keep]
        self.u = unew
        self.steps += 1
        return {"p_iters": pit, "p_status": pst, "v_iters": vits, "p_rhs": bp}
