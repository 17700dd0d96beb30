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
"""
from __future__ import annotations

import numpy as np

from . import Mesh, inverse_jacobian

BDF = {1: (1.0, (1.0,)), 2: (1.5, (2.0, -0.5))}
EXT = {1: (1.0,), 2: (2.0, -1.0)}


class NSOracle:
    def __init__(self, N, nel, verts, Re, periodic=(1, 1, 1)):
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
        k = min(self.steps + 1, 2)
        b0, bj = BDF[k]
        aj = EXT[k]
        nl = self.advect(self.u)
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
        self.u_hist = [self.u] + self.u_hist[:0]
        self.nl_hist = [nl] + self.nl_hist[:0]
        self.u = unew
        self.steps += 1
        return {"p_iters": pit, "p_status": pst, "v_iters": vits, "p_rhs": bp}
