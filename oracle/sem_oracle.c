/*
 * sem_oracle.c -- plain, slow, FP64 CPU oracle for the spectral-element
 * pressure-Poisson path (test infrastructure, not part of the library).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's shared object.  It shares no code, header,
 * table or constant with the CUDA library: every formula below is written
 * out from its mathematical definition.
 *
 * The paper (Karp et al., arXiv 2405.05640) states the method in prose only,
 * section 3.1 ("Neko"): E non-overlapping hexahedra, an order-N Lagrange
 * basis collocated on the Gauss-Lobatto-Legendre (GLL) points, element-by-
 * element (matrix-free) operators, a unit-depth gather-scatter that sums the
 * copies of nodes shared between elements, and a preconditioned Krylov solve
 * of Ax=b each time step.  It refers the discretisation to Deville, Fischer &
 * Mund, "High-Order Methods for Incompressible Fluid Flow" (2002); the
 * formulas here are the textbook ones:
 *
 *   GLL nodes/weights ........ or_legendre, or_gll
 *   derivative matrix ........ or_deriv
 *   geometric factors ........ or_geometry (trilinear hexahedra)
 *   box connectivity ......... or_box_numbering, or_box_mask
 *   gather-scatter (Q Q^T) ... or_dssum, or_apply_mask
 *   local stiffness .......... or_ax_local, or_helmholtz_local
 *   Jacobi diagonal .......... or_jacobi_diag_local
 *   Jacobi-PCG ............... or_pcg
 *   inverse Jacobian ......... or_inverse_jacobian (for gradients / divergence)
 *
 * Layout: a field is stored element by element, u[e][k][j][i] with i fastest
 * (local point p = i + (N+1)*(j + (N+1)*k)); geometric factors are
 * G[e][c][p], c = 0..5 for (rr, ss, tt, rs, rt, st).
 *
 * Return codes: 0 ok, -1 invalid argument, -3 bad mesh (det J <= 0),
 * -5 NaN/Inf in the right-hand side, -6 not converged.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_EMESH (-3)
#define OR_ENAN (-5)
#define OR_ENOTCONV (-6)

/* Legendre polynomial P_N(x) and its derivative by the three-term
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, and
 * P_N'(x) = sum over the same recurrence differentiated:
 * (k+1) P'_{k+1} = (2k+1) (P_k + x P'_k) - k P'_{k-1}. */
void or_legendre(int N, double x, double *P, double *dP)
{
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (N == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int k = 1; k < N; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        double d2 = ((2.0 * k + 1.0) * (p1 + x * d1) - k * d0) / (k + 1.0);
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *P = p1; *dP = d1;
}

/* GLL nodes: xi_0 = -1, xi_N = +1, interior nodes are the roots of P_N'.
 * Newton on P_N' with P_N'' from the Legendre equation
 * (1 - x^2) P'' = 2 x P' - N(N+1) P, started from the Chebyshev-Gauss-
 * Lobatto points -cos(pi i / N).  Weights rho_i = 2 / (N (N+1) P_N(xi_i)^2).
 * Returns 0, or -1 for N < 1. */
int or_gll(int N, double *xi, double *rho)
{
    if (N < 1) return OR_EINVAL;
    xi[0] = -1.0; xi[N] = 1.0;
    for (int i = 1; i < N; ++i) {
        double x = -cos(M_PI * i / N);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            or_legendre(N, x, &P, &dP);
            double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
            double dx = dP / d2P;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        xi[i] = x;
    }
    /* the node set is symmetric about 0 */
    for (int i = 0; i <= N / 2; ++i) {
        double s = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -s; xi[N - i] = s;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int i = 0; i <= N; ++i) {
        double P, dP;
        or_legendre(N, xi[i], &P, &dP);
        rho[i] = 2.0 / (N * (N + 1.0) * P * P);
    }
    return OR_OK;
}

/* Collocation derivative D_ij = l_j'(xi_i) of the GLL Lagrange basis:
 * D_ij = P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j)) for i != j,
 * D_00 = -N(N+1)/4, D_NN = +N(N+1)/4, all other diagonal entries 0.
 * D is row-major, D[i*(N+1) + j]. */
void or_deriv(int N, const double *xi, double *D)
{
    int n1 = N + 1;
    double PN[64];
    for (int i = 0; i < n1; ++i) {
        double dP;
        or_legendre(N, xi[i], &PN[i], &dP);
    }
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n1; ++j) {
            double d;
            if (i != j) d = PN[i] / (PN[j] * (xi[i] - xi[j]));
            else if (i == 0) d = -0.25 * N * (N + 1.0);
            else if (i == N) d = 0.25 * N * (N + 1.0);
            else d = 0.0;
            D[i * n1 + j] = d;
        }
}

/* Geometry of trilinear hexahedra.
 * verts[e][v][a]: vertex v = vx + 2 vy + 4 vz of element e, coordinate a.
 * Outputs (any may be NULL):
 *   xyz[a][e][p] : physical coordinates of the GLL points,
 *   G[e][c][p]   : rho_i rho_j rho_k detJ sum_m (dr_a/dx_m)(dr_b/dx_m),
 *                  c = (rr, ss, tt, rs, rt, st),
 *   B[e][p]      : rho_i rho_j rho_k detJ (diagonal mass matrix).
 * The Jacobian J_ab = dx_a/dr_b is obtained by applying D along direction b
 * to the coordinate field x_a.  Returns -3 if det J <= 0 anywhere. */
int or_geometry(int N, long E, const double *verts, const double *xi,
                const double *rho, const double *D,
                double *xyz, double *G, double *B)
{
    int n1 = N + 1;
    long npt = (long)n1 * n1 * n1;
    double *X = (double *)malloc(sizeof(double) * 3 * npt);
    int status = OR_OK;
    for (long e = 0; e < E; ++e) {
        const double *V = verts + e * 24;
        /* J is invariant under translation, so it is taken from the
         * coordinates relative to vertex 0 (same derivative, smaller
         * rounding in the D contraction far from the origin). */
        double V0[3] = {V[0], V[1], V[2]};
        /* trilinear map evaluated at the GLL points */
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    double r = xi[i], s = xi[j], t = xi[k];
                    double fr[2] = {0.5 * (1.0 - r), 0.5 * (1.0 + r)};
                    double fs[2] = {0.5 * (1.0 - s), 0.5 * (1.0 + s)};
                    double ft[2] = {0.5 * (1.0 - t), 0.5 * (1.0 + t)};
                    long p = i + n1 * (j + n1 * k);
                    for (int a = 0; a < 3; ++a) {
                        double x = 0.0;
                        for (int v = 0; v < 8; ++v)
                            x += (V[v * 3 + a] - V0[a]) * fr[v & 1] * fs[(v >> 1) & 1] * ft[(v >> 2) & 1];
                        X[a * npt + p] = x;
                    }
                }
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    long p = i + n1 * (j + n1 * k);
                    double J[3][3];
                    for (int a = 0; a < 3; ++a) {
                        const double *Xa = X + a * npt;
                        double dr = 0.0, ds = 0.0, dt = 0.0;
                        for (int l = 0; l < n1; ++l) {
                            dr += D[i * n1 + l] * Xa[l + n1 * (j + n1 * k)];
                            ds += D[j * n1 + l] * Xa[i + n1 * (l + n1 * k)];
                            dt += D[k * n1 + l] * Xa[i + n1 * (j + n1 * l)];
                        }
                        J[a][0] = dr; J[a][1] = ds; J[a][2] = dt;
                    }
                    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                    if (!(det > 0.0)) status = OR_EMESH;
                    /* inverse Jacobian: Ri[b][m] = dr_b/dx_m = cofactor(m,b)/det */
                    double Ri[3][3];
                    Ri[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
                    Ri[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
                    Ri[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
                    Ri[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
                    Ri[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
                    Ri[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
                    Ri[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
                    Ri[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
                    Ri[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
                    double wq = rho[i] * rho[j] * rho[k] * det;
                    static const int ca[6] = {0, 1, 2, 0, 0, 1};
                    static const int cb[6] = {0, 1, 2, 1, 2, 2};
                    if (G)
                        for (int c = 0; c < 6; ++c) {
                            double g = 0.0;
                            for (int m = 0; m < 3; ++m) g += Ri[ca[c]][m] * Ri[cb[c]][m];
                            G[(e * 6 + c) * npt + p] = wq * g;
                        }
                    if (B) B[e * npt + p] = wq;
                    if (xyz)
                        for (int a = 0; a < 3; ++a) {
                            double r = xi[i], s = xi[j], t = xi[k], x = 0.0;
                            for (int v = 0; v < 8; ++v)
                                x += V[v * 3 + a] * 0.125 * ((v & 1) ? 1.0 + r : 1.0 - r) *
                                     (((v >> 1) & 1) ? 1.0 + s : 1.0 - s) * (((v >> 2) & 1) ? 1.0 + t : 1.0 - t);
                            xyz[(a * E + e) * npt + p] = x;
                        }
                }
    }
    free(X);
    return status;
}

/* Connectivity of an nel[0] x nel[1] x nel[2] box of elements, element
 * e = ex + nel0 (ey + nel1 ez).  Local point (e; i,j,k) is the global node
 * (I,J,K) = (ex N + i, ey N + j, ez N + k), taken modulo nel_a N on a
 * periodic axis.  gid = I + Gx (J + Gy K) with G_a = nel_a N (+1 unless
 * periodic).  Writes gid[nloc] and returns the global node count. */
long or_box_numbering(int N, const int *nel, const int *periodic, long *gid)
{
    int n1 = N + 1;
    long Gd[3];
    for (int a = 0; a < 3; ++a) Gd[a] = (long)nel[a] * N + (periodic[a] ? 0 : 1);
    long e = 0, l = 0;
    for (int ez = 0; ez < nel[2]; ++ez)
        for (int ey = 0; ey < nel[1]; ++ey)
            for (int ex = 0; ex < nel[0]; ++ex, ++e)
                for (int k = 0; k < n1; ++k)
                    for (int j = 0; j < n1; ++j)
                        for (int i = 0; i < n1; ++i, ++l) {
                            long I = (long)ex * N + i, J = (long)ey * N + j, K = (long)ez * N + k;
                            if (periodic[0]) I %= Gd[0];
                            if (periodic[1]) J %= Gd[1];
                            if (periodic[2]) K %= Gd[2];
                            gid[l] = I + Gd[0] * (J + Gd[1] * K);
                        }
    return Gd[0] * Gd[1] * Gd[2];
}

/* Dirichlet mask of the box: bit 2a of `faces` marks the low face of axis a,
 * bit 2a+1 the high face (ignored on periodic axes).  mask[l] = 1 where the
 * local point lies on a Dirichlet face, else 0. */
void or_box_mask(int N, const int *nel, const int *periodic, int faces, unsigned char *mask)
{
    int n1 = N + 1;
    long l = 0;
    for (int ez = 0; ez < nel[2]; ++ez)
        for (int ey = 0; ey < nel[1]; ++ey)
            for (int ex = 0; ex < nel[0]; ++ex)
                for (int k = 0; k < n1; ++k)
                    for (int j = 0; j < n1; ++j)
                        for (int i = 0; i < n1; ++i, ++l) {
                            long I[3] = {(long)ex * N + i, (long)ey * N + j, (long)ez * N + k};
                            int m = 0;
                            for (int a = 0; a < 3; ++a) {
                                if (periodic[a]) continue;
                                if ((faces >> (2 * a)) & 1 && I[a] == 0) m = 1;
                                if ((faces >> (2 * a + 1)) & 1 && I[a] == (long)nel[a] * N) m = 1;
                            }
                            mask[l] = (unsigned char)m;
                        }
}

/* Direct stiffness summation u <- Q Q^T u: every local copy of a global node
 * receives the sum of all copies, accumulated in ascending local index.
 * tmp must hold nglob doubles. */
void or_dssum(long nloc, const long *gid, long nglob, double *u, double *tmp)
{
    for (long g = 0; g < nglob; ++g) tmp[g] = 0.0;
    for (long l = 0; l < nloc; ++l) tmp[gid[l]] += u[l];
    for (long l = 0; l < nloc; ++l) u[l] = tmp[gid[l]];
}

void or_apply_mask(long nloc, const unsigned char *mask, double *u)
{
    for (long l = 0; l < nloc; ++l)
        if (mask[l]) u[l] = 0.0;
}

/* Local (unassembled) stiffness, element by element:
 *   u_r(ijk) = sum_l D_il u(ljk),  u_s = sum_l D_jl u(ilk),  u_t = sum_l D_kl u(ijl)
 *   v_r = G_rr u_r + G_rs u_s + G_rt u_t   (and cyclically for v_s, v_t)
 *   w(ijk) = sum_l D_li v_r(ljk) + sum_l D_lj v_s(ilk) + sum_l D_lk v_t(ijl). */
void or_ax_local(int N, long E, const double *D, const double *G, const double *u, double *w)
{
    int n1 = N + 1;
    long npt = (long)n1 * n1 * n1;
    double *vr = (double *)malloc(sizeof(double) * npt * 3);
    double *vs = vr + npt, *vt = vs + npt;
    for (long e = 0; e < E; ++e) {
        const double *ue = u + e * npt;
        const double *Ge = G + e * 6 * npt;
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    double ur = 0.0, us = 0.0, ut = 0.0;
                    for (int l = 0; l < n1; ++l) {
                        ur += D[i * n1 + l] * ue[l + n1 * (j + n1 * k)];
                        us += D[j * n1 + l] * ue[i + n1 * (l + n1 * k)];
                        ut += D[k * n1 + l] * ue[i + n1 * (j + n1 * l)];
                    }
                    long p = i + n1 * (j + n1 * k);
                    double grr = Ge[0 * npt + p], gss = Ge[1 * npt + p], gtt = Ge[2 * npt + p];
                    double grs = Ge[3 * npt + p], grt = Ge[4 * npt + p], gst = Ge[5 * npt + p];
                    vr[p] = grr * ur + grs * us + grt * ut;
                    vs[p] = grs * ur + gss * us + gst * ut;
                    vt[p] = grt * ur + gst * us + gtt * ut;
                }
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    double s = 0.0;
                    for (int l = 0; l < n1; ++l) {
                        s += D[l * n1 + i] * vr[l + n1 * (j + n1 * k)];
                        s += D[l * n1 + j] * vs[i + n1 * (l + n1 * k)];
                        s += D[l * n1 + k] * vt[i + n1 * (j + n1 * l)];
                    }
                    w[e * npt + i + n1 * (j + n1 * k)] = s;
                }
    }
    free(vr);
}

/* Local Helmholtz operator w = h1 * (A_L u) + h2 * B u. */
void or_helmholtz_local(int N, long E, const double *D, const double *G, const double *B,
                        double h1, double h2, const double *u, double *w)
{
    long nloc = E * (long)(N + 1) * (N + 1) * (N + 1);
    or_ax_local(N, E, D, G, u, w);
    for (long l = 0; l < nloc; ++l) w[l] = h1 * w[l] + h2 * B[l] * u[l];
}

/* Diagonal of the local stiffness (coefficient of u(ijk) in w(ijk)):
 *   sum_l D_li^2 G_rr(ljk) + sum_l D_lj^2 G_ss(ilk) + sum_l D_lk^2 G_tt(ijl)
 *   + 2 D_ii D_jj G_rs(ijk) + 2 D_ii D_kk G_rt(ijk) + 2 D_jj D_kk G_st(ijk). */
void or_jacobi_diag_local(int N, long E, const double *D, const double *G, double *diag)
{
    int n1 = N + 1;
    long npt = (long)n1 * n1 * n1;
    for (long e = 0; e < E; ++e) {
        const double *Ge = G + e * 6 * npt;
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    long p = i + n1 * (j + n1 * k);
                    double s = 0.0;
                    for (int l = 0; l < n1; ++l) {
                        s += D[l * n1 + i] * D[l * n1 + i] * Ge[0 * npt + l + n1 * (j + n1 * k)];
                        s += D[l * n1 + j] * D[l * n1 + j] * Ge[1 * npt + i + n1 * (l + n1 * k)];
                        s += D[l * n1 + k] * D[l * n1 + k] * Ge[2 * npt + i + n1 * (j + n1 * l)];
                    }
                    double Di = D[i * n1 + i], Dj = D[j * n1 + j], Dk = D[k * n1 + k];
                    s += 2.0 * Di * Dj * Ge[3 * npt + p];
                    s += 2.0 * Di * Dk * Ge[4 * npt + p];
                    s += 2.0 * Dj * Dk * Ge[5 * npt + p];
                    diag[e * npt + p] = s;
                }
    }
}

/* Unique-node inner product of two continuous element-layout fields:
 * <a,b> = sum_l a_l b_l / mult_l, passed as minv = 1/mult. */
double or_glsc3(long nloc, const double *a, const double *b, const double *minv)
{
    double s = 0.0;
    for (long l = 0; l < nloc; ++l) s += a[l] * b[l] * minv[l];
    return s;
}

/* Assembled operator y = M Q Q^T (h1 A_L + h2 B) x. */
static void or_assembled(int N, long E, const double *D, const double *G, const double *B,
                         double h1, double h2, const long *gid, long nglob,
                         const unsigned char *mask, const double *x, double *y, double *tmp)
{
    long nloc = E * (long)(N + 1) * (N + 1) * (N + 1);
    if (h2 == 0.0) {
        or_ax_local(N, E, D, G, x, y);
        if (h1 != 1.0)
            for (long l = 0; l < nloc; ++l) y[l] *= h1;
    } else {
        or_helmholtz_local(N, E, D, G, B, h1, h2, x, y);
    }
    or_dssum(nloc, gid, nglob, y, tmp);
    or_apply_mask(nloc, mask, y);
}

/* Jacobi-preconditioned conjugate gradients (Hestenes-Stiefel) on the
 * assembled system M Q Q^T (h1 A_L + h2 B) x = b, b continuous and masked:
 *   r = b - A x0;  z = P r;  p = z;  rho = <r,z>
 *   repeat: w = A p; alpha = rho / <p,w>; x += alpha p; r -= alpha w;
 *           stop when ||r|| <= tol ||b||; z = P r; rho' = <r,z>;
 *           beta = rho'/rho; p = z + beta p
 * with <.,.> the unique-node product (or_glsc3) and P = dinv (0 on masked
 * nodes).  x holds the initial guess on entry.  work holds 4*nloc + nglob
 * doubles.  Returns 0 when converged, -6 when max_iter was reached, -5 when
 * b holds a NaN or Inf.  iters / rel_res receive the final state. */
int or_pcg(int N, long E, const double *D, const double *G, const double *B,
           double h1, double h2, const long *gid, long nglob, const unsigned char *mask,
           const double *minv, const double *dinv, const double *b, double *x,
           double tol, int max_iter, int *iters, double *rel_res, double *work)
{
    long nloc = E * (long)(N + 1) * (N + 1) * (N + 1);
    double *r = work, *z = r + nloc, *p = z + nloc, *w = p + nloc, *tmp = w + nloc;
    for (long l = 0; l < nloc; ++l)
        if (!isfinite(b[l])) return OR_ENAN;
    double bnorm = sqrt(or_glsc3(nloc, b, b, minv));
    or_assembled(N, E, D, G, B, h1, h2, gid, nglob, mask, x, w, tmp);
    for (long l = 0; l < nloc; ++l) r[l] = b[l] - w[l];
    double rnorm = sqrt(or_glsc3(nloc, r, r, minv));
    *iters = 0;
    *rel_res = bnorm > 0.0 ? rnorm / bnorm : rnorm;
    if (rnorm <= tol * bnorm) return OR_OK;
    for (long l = 0; l < nloc; ++l) { z[l] = dinv[l] * r[l]; p[l] = z[l]; }
    double rho = or_glsc3(nloc, r, z, minv);
    for (int it = 1; it <= max_iter; ++it) {
        or_assembled(N, E, D, G, B, h1, h2, gid, nglob, mask, p, w, tmp);
        double alpha = rho / or_glsc3(nloc, p, w, minv);
        for (long l = 0; l < nloc; ++l) { x[l] += alpha * p[l]; r[l] -= alpha * w[l]; }
        rnorm = sqrt(or_glsc3(nloc, r, r, minv));
        *iters = it;
        *rel_res = bnorm > 0.0 ? rnorm / bnorm : rnorm;
        if (rnorm <= tol * bnorm) return OR_OK;
        for (long l = 0; l < nloc; ++l) z[l] = dinv[l] * r[l];
        double rho1 = or_glsc3(nloc, r, z, minv);
        double beta = rho1 / rho;
        rho = rho1;
        for (long l = 0; l < nloc; ++l) p[l] = z[l] + beta * p[l];
    }
    return OR_ENOTCONV;
}

/* Inverse Jacobian dr_a/dx_m at every GLL point of trilinear hexahedra:
 * RX[e][3a+m][p], from J = dx/dr obtained (as in or_geometry) by applying D
 * to the vertex-relative coordinates.  Returns -3 if det J <= 0. */
int or_inverse_jacobian(int N, long E, const double *verts, const double *xi, const double *D, double *RX)
{
    int n1 = N + 1;
    long npt = (long)n1 * n1 * n1;
    double *X = (double *)malloc(sizeof(double) * 3 * npt);
    int status = OR_OK;
    for (long e = 0; e < E; ++e) {
        const double *V = verts + e * 24;
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    double fr[2] = {0.5 * (1.0 - xi[i]), 0.5 * (1.0 + xi[i])};
                    double fs[2] = {0.5 * (1.0 - xi[j]), 0.5 * (1.0 + xi[j])};
                    double ft[2] = {0.5 * (1.0 - xi[k]), 0.5 * (1.0 + xi[k])};
                    for (int a = 0; a < 3; ++a) {
                        double x = 0.0;
                        for (int v = 0; v < 8; ++v)
                            x += (V[v * 3 + a] - V[a]) * fr[v & 1] * fs[(v >> 1) & 1] * ft[(v >> 2) & 1];
                        X[a * npt + i + n1 * (j + n1 * k)] = x;
                    }
                }
        for (int k = 0; k < n1; ++k)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    long p = i + n1 * (j + n1 * k);
                    double J[3][3];
                    for (int a = 0; a < 3; ++a) {
                        const double *Xa = X + a * npt;
                        double dr = 0.0, ds = 0.0, dt = 0.0;
                        for (int l = 0; l < n1; ++l) {
                            dr += D[i * n1 + l] * Xa[l + n1 * (j + n1 * k)];
                            ds += D[j * n1 + l] * Xa[i + n1 * (l + n1 * k)];
                            dt += D[k * n1 + l] * Xa[i + n1 * (j + n1 * l)];
                        }
                        J[a][0] = dr; J[a][1] = ds; J[a][2] = dt;
                    }
                    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                    if (!(det > 0.0)) status = OR_EMESH;
                    double R[3][3];
                    R[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
                    R[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
                    R[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
                    R[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
                    R[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
                    R[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
                    R[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
                    R[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
                    R[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
                    for (int a = 0; a < 3; ++a)
                        for (int m = 0; m < 3; ++m) RX[(e * 9 + 3 * a + m) * npt + p] = R[a][m];
                }
    }
    free(X);
    return status;
}
