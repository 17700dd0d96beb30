// sem_schwarz.cu -- hybrid Schwarz preconditioner of the pressure solve.
//
// Paper section 3.1: the pressure is solved by a Krylov method with a
// hybrid-Schwarz multigrid preconditioner (the SEM overlapping Schwarz /
// fast-diagonalisation method of the literature it cites).  Two additive
// levels, symmetric:
//   z = sum_e R_e^T A_e^{-1} R_e r  +  P A_c^{-1} P^T r.
// Local solves: element e extended by one GLL point into each neighbour
// (N+3 points per direction); along each direction the 1-D stiffness and mass
// of the three elements (left neighbour, e, right neighbour; mean edge
// lengths) assembled and restricted to the N+3 points (homogeneous Dirichlet
// just beyond the overlap); points outside the domain and Dirichlet boundary
// points decoupled.  A_e = Bz(x)By(x)Ax + Bz(x)Ay(x)Bx + Az(x)By(x)Bx is inverted
// by fast diagonalisation, A S = B S Lambda with S^T B S = I:
//   A_e^{-1} = (Sz(x)Sy(x)Sx) diag(1/(lz + ly + lx)) (Sz(x)Sy(x)Sx)^T.
// Coarse level: the trilinear (N = 1) mesh on the same vertices; P^T sums
// r/mult into the vertices, P interpolates back; A_c^{-1} by a fixed number
// of Jacobi-CG iterations (device-driven).
//
// GB300 design (FP32, the inner solver's precision): the 1-D eigenproblems
// are solved once on the host (Cholesky + cyclic Jacobi) and cached by their
// key (lengths and boundary flags: a tensor-product mesh has few distinct
// ones); one CTA per element gathers the extended residual from its
// neighbours with computed indices (box topology), applies the six 1-D
// contractions through shared memory and writes the extended solution; a
// second kernel assembles each point's value from the (up to 2 x 2 x 2)
// overlapping subdomains in a fixed order (deterministic, copies identical,
// no atomics).

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "sem_common.cuh"

struct sem_schwarz {
    const sem_mesh *m, *mc;
    int N, ne, P;
    float *S;      // [P][ne][ne] eigenvectors S[l][a] (row l = point, column a = mode)
    float *L;      // [P][ne] eigenvalues
    int *prob;     // [E][3] problem id per element and axis
    float *uext;   // [E][ne^3] extended local solutions
    float *rc, *xc;  // coarse right-hand side and solution (coarse E-layout)
    void *cg_scratch;
    size_t ws_bytes;
};

namespace sem {

constexpr int kMaxNe = kMaxN1 + 2;

// ---------------------------------------------------------------- host set-up

// Generalised symmetric eigenproblem A s = lambda B s (B SPD): Cholesky B =
// G G^T, C = G^-1 A G^-T, cyclic Jacobi rotations C = V diag(l) V^T,
// S = G^-T V (so S^T B S = I, S^T A S = diag(l)).
static void gen_eig(int n, const double *A, const double *B, double *S, double *lam) {
    std::vector<double> G(n * n, 0.0), C(n * n), V(n * n, 0.0), T(n * n);
    for (int j = 0; j < n; ++j) {
        double d = B[j * n + j];
        for (int k = 0; k < j; ++k) d -= G[j * n + k] * G[j * n + k];
        G[j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double v = B[i * n + j];
            for (int k = 0; k < j; ++k) v -= G[i * n + k] * G[j * n + k];
            G[i * n + j] = v / G[j * n + j];
        }
    }
    // T = G^-1 A (forward substitution per column), C = T G^-T (per row)
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double v = A[i * n + c];
            for (int k = 0; k < i; ++k) v -= G[i * n + k] * T[k * n + c];
            T[i * n + c] = v / G[i * n + i];
        }
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < n; ++j) {
            double v = T[r * n + j];
            for (int k = 0; k < j; ++k) v -= C[r * n + k] * G[j * n + k];
            C[r * n + j] = v / G[j * n + j];
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) C[i * n + j] = C[j * n + i] = 0.5 * (C[i * n + j] + C[j * n + i]);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += C[i * n + j] * C[i * n + j];
                if (i != j) off += C[i * n + j] * C[i * n + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = C[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (C[q * n + q] - C[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double ckp = C[k * n + p], ckq = C[k * n + q];
                    C[k * n + p] = c * ckp - s * ckq;
                    C[k * n + q] = s * ckp + c * ckq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double cpk = C[p * n + k], cqk = C[q * n + k];
                    C[p * n + k] = c * cpk - s * cqk;
                    C[q * n + k] = s * cpk + c * cqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = C[i * n + i];
    // S = G^-T V: back substitution per column
    for (int c = 0; c < n; ++c)
        for (int i = n - 1; i >= 0; --i) {
            double v = V[i * n + c];
            for (int k = i + 1; k < n; ++k) v -= G[k * n + i] * S[k * n + c];
            S[i * n + c] = v / G[i * n + i];
        }
}

// Cache key of a 1-D problem: lengths on a log scale with 2^-10 relative
// resolution (exact repeats on tensor-product meshes; nearby ones merged on
// deformed meshes, a change far below what matters to a preconditioner) and
// the boundary flags.
struct FdmKey {
    long long h, hL, hR;
    int flags;
    bool operator<(const FdmKey &o) const {
        if (flags != o.flags) return flags < o.flags;
        if (h != o.h) return h < o.h;
        if (hL != o.hL) return hL < o.hL;
        return hR < o.hR;
    }
};
static long long qlen(double h) { return std::llround(std::log2(h) * 1024.0); }

// ---------------------------------------------------------------- kernels

struct SwArgs {
    int64_t E;
    int nel[3], per[3], faces;
};

// Along one axis: the (element offset, local index) of extended point I of an
// element at coordinate c of n (valid = false outside the domain).
__device__ __forceinline__ bool ext_move(int I, int N, int c, int n, int per, int &dc, int &li) {
    if (I == 0) {
        if (c == 0 && !per) return false;
        dc = c == 0 ? n - 1 : -1;
        li = N - 1;
    } else if (I == N + 2) {
        if (c == n - 1 && !per) return false;
        dc = c == n - 1 ? -(n - 1) : 1;
        li = 1;
    } else {
        dc = 0;
        li = I - 1;
    }
    return true;
}

template <int N>
__global__ void __launch_bounds__(256)
    schwarz_local_kernel(const float *__restrict__ r, const float *__restrict__ Stab, const float *__restrict__ Ltab,
                         const int *__restrict__ prob, SwArgs A, float *__restrict__ uext) {
    constexpr int N1 = N + 1, NE = N + 3, NE2 = NE * NE, NE3 = NE2 * NE, NPT = N1 * N1 * N1;
    __shared__ float sS[3][NE * NE], sL[3][NE], sa[NE3], sb[NE3];
    for (int64_t e = blockIdx.x; e < A.E; e += gridDim.x) {
        __syncthreads();
        const int ex = (int)(e % A.nel[0]), ey = (int)((e / A.nel[0]) % A.nel[1]),
                  ez = (int)(e / ((int64_t)A.nel[0] * A.nel[1]));
        for (int t = threadIdx.x; t < 3 * NE2; t += blockDim.x) {
            const int a = t / NE2;
            sS[a][t - a * NE2] = Stab[(int64_t)prob[e * 3 + a] * NE2 + (t - a * NE2)];
        }
        for (int t = threadIdx.x; t < 3 * NE; t += blockDim.x) {
            const int a = t / NE;
            sL[a][t - a * NE] = Ltab[(int64_t)prob[e * 3 + a] * NE + (t - a * NE)];
        }
        // gather the extended residual
        for (int t = threadIdx.x; t < NE3; t += blockDim.x) {
            const int I = t % NE, J = (t / NE) % NE, K = t / NE2;
            int dx, dy, dz, i, j, k;
            float v = 0.f;
            if (ext_move(I, N, ex, A.nel[0], A.per[0], dx, i) && ext_move(J, N, ey, A.nel[1], A.per[1], dy, j) &&
                ext_move(K, N, ez, A.nel[2], A.per[2], dz, k)) {
                const int64_t e2 = (ex + dx) + (int64_t)A.nel[0] * ((ey + dy) + (int64_t)A.nel[1] * (ez + dz));
                v = r[e2 * NPT + i + N1 * (j + N1 * k)];
            }
            sa[t] = v;
        }
        __syncthreads();
        // forward: along I with Sx^T, J with Sy^T, K with Sz^T
        for (int t = threadIdx.x; t < NE3; t += blockDim.x) {
            const int a = t % NE, r0 = t - a;
            float s = 0.f;
#pragma unroll
            for (int l = 0; l < NE; ++l) s = fmaf(sS[0][l * NE + a], sa[r0 + l], s);
            sb[t] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NE3; t += blockDim.x) {
            const int I = t % NE, b = (t / NE) % NE, K = t / NE2;
            float s = 0.f;
#pragma unroll
            for (int l = 0; l < NE; ++l) s = fmaf(sS[1][l * NE + b], sb[K * NE2 + l * NE + I], s);
            sa[t] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NE3; t += blockDim.x) {
            const int IJ = t % NE2, c = t / NE2;
            float s = 0.f;
#pragma unroll
            for (int l = 0; l < NE; ++l) s = fmaf(sS[2][l * NE + c], sa[l * NE2 + IJ], s);
            const int a = IJ % NE, b = IJ / NE;
            sb[t] = s / (sL[0][a] + sL[1][b] + sL[2][c]);
        }
        __syncthreads();
        // backward: along K with Sz, J with Sy, I with Sx
        for (int t = threadIdx.x; t < NE3; t += blockDim.x) {
            const int IJ = t % NE2, K = t / NE2;
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < NE; ++c) s = fmaf(sS[2][K * NE + c], sb[c * NE2 + IJ], s);
            sa[t] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NE3; t += blockDim.x) {
            const int I = t % NE, J = (t / NE) % NE, K = t / NE2;
            float s = 0.f;
#pragma unroll
            for (int b = 0; b < NE; ++b) s = fmaf(sS[1][J * NE + b], sa[K * NE2 + b * NE + I], s);
            sb[t] = s;
        }
        __syncthreads();
        float *ue = uext + e * NE3;
        for (int t = threadIdx.x; t < NE3; t += blockDim.x) {
            const int I = t % NE, r0 = t - I;
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < NE; ++a) s = fmaf(sS[0][I * NE + a], sb[r0 + a], s);
            ue[t] = s;
        }
    }
}

// Along one axis: the subdomains covering local index i of an element at
// coordinate c of n: (element offset, extended index), left to right.
// (N = 2: the middle point is covered by all three.)
__device__ __forceinline__ int cover(int i, int N, int c, int n, int per, int (&dc)[3], int (&I)[3]) {
    int m = 0;
    if (i <= 1 && (c > 0 || per)) {  // the left neighbour (its own point N, or its right extension)
        dc[m] = c == 0 ? n - 1 : -1;
        I[m++] = i + N + 1;
    }
    dc[m] = 0;
    I[m++] = i + 1;
    if (i >= N - 1 && (c < n - 1 || per)) {  // the right neighbour (its own point 0, or its left extension)
        dc[m] = c == n - 1 ? -(n - 1) : 1;
        I[m++] = i - N + 1;
    }
    return m;
}

// z(e, i, j, k) = sum over the covering subdomains (z, then y, then x from
// low to high position) of their extended solutions; 0 on Dirichlet nodes
// (dinv = 0 there).  With add, z += that sum.
template <int N>
__global__ void __launch_bounds__(256)
    schwarz_sum_kernel(const float *__restrict__ uext, const float *__restrict__ dinv, SwArgs A,
                       float *__restrict__ z) {
    constexpr int N1 = N + 1, NE = N + 3, NE2 = NE * NE, NE3 = NE2 * NE, NPT = N1 * N1 * N1;
    const int64_t n = A.E * NPT;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / NPT;
        const int p = (int)(l - e * NPT);
        const int i = p % N1, j = (p / N1) % N1, k = p / (N1 * N1);
        const int ex = (int)(e % A.nel[0]), ey = (int)((e / A.nel[0]) % A.nel[1]),
                  ez = (int)(e / ((int64_t)A.nel[0] * A.nel[1]));
        int dx[3], Ix[3], dy[3], Iy[3], dz[3], Iz[3];
        const int mx = cover(i, N, ex, A.nel[0], A.per[0], dx, Ix);
        const int my = cover(j, N, ey, A.nel[1], A.per[1], dy, Iy);
        const int mz = cover(k, N, ez, A.nel[2], A.per[2], dz, Iz);
        float s = 0.f;
        for (int c = 0; c < mz; ++c)
            for (int b = 0; b < my; ++b)
                for (int a = 0; a < mx; ++a) {
                    const int64_t e2 = (ex + dx[a]) + (int64_t)A.nel[0] * ((ey + dy[b]) + (int64_t)A.nel[1] * (ez + dz[c]));
                    s += uext[e2 * NE3 + Ix[a] + NE * (Iy[b] + NE * Iz[c])];
                }
        z[l] = dinv[l] != 0.f ? s : 0.f;
    }
}

// Coarse restriction rc[e][c][b][a] = sum_ijk J1[i][a] J1[j][b] J1[k][c] r(i,j,k) / mult,
// J1[i] = ((1 - xi_i)/2, (1 + xi_i)/2); one thread per (element, vertex).
struct J1Tab {
    float j[kMaxN1][2];
};

template <int N>
__global__ void restrict_kernel(const float *__restrict__ r, const float *__restrict__ minv, J1Tab J, int64_t E,
                                float *__restrict__ rc) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < E * 8; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / 8;
        const int v = (int)(t - e * 8), a = v & 1, b = (v >> 1) & 1, c = v >> 2;
        const float *re = r + e * NPT, *me = minv + e * NPT;
        float s = 0.f;
        for (int k = 0; k < N1; ++k)
            for (int j = 0; j < N1; ++j) {
                const float wjk = J.j[j][b] * J.j[k][c];
                float si = 0.f;
#pragma unroll
                for (int i = 0; i < N1; ++i) {
                    const int q = i + N1 * (j + N1 * k);
                    si = fmaf(J.j[i][a], re[q] * me[q], si);
                }
                s = fmaf(wjk, si, s);
            }
        rc[t] = s;
    }
}

// z += P xc (trilinear interpolation of the element's vertex values)
template <int N>
__global__ void prolong_add_kernel(const float *__restrict__ xc, J1Tab J, int64_t E, float *__restrict__ z) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < E * NPT; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / NPT;
        const int p = (int)(l - e * NPT);
        const int i = p % N1, j = (p / N1) % N1, k = p / (N1 * N1);
        const float *x = xc + e * 8;
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) s = fmaf(J.j[i][v & 1] * J.j[j][(v >> 1) & 1] * J.j[k][v >> 2], x[v], s);
        z[l] += s;
    }
}

static size_t sw_layout(const sem_mesh *m, const sem_mesh *mc, size_t *off) {
    const int ne = m->N + 3;
    const size_t P = 3 * (size_t)m->E;  // upper bound: every element and axis distinct
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = align_up(o + b); return at; };
    off[0] = take(sizeof(float) * P * ne * ne);
    off[1] = take(sizeof(float) * P * ne);
    off[2] = take(sizeof(int) * 3 * m->E);
    off[3] = take(sizeof(float) * (size_t)m->E * ne * ne * ne);
    off[4] = take(sizeof(float) * mc->nloc);
    off[5] = take(sizeof(float) * mc->nloc);
    off[6] = take(fixed_cg_scratch_bytes(mc));
    return o;
}

static SwArgs sw_args(const sem_mesh *m) {
    SwArgs A;
    A.E = m->E;
    for (int a = 0; a < 3; ++a) {
        A.nel[a] = m->nel[a];
        A.per[a] = m->periodic[a];
    }
    A.faces = m->faces;
    return A;
}

template <int N>
static int sw_apply_n(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      cudaStream_t st) {
    const sem_mesh *m = sw->m;
    const SwArgs A = sw_args(m);
    int64_t g = m->E;
    if (g > (int64_t)m->num_sms * 8) g = (int64_t)m->num_sms * 8;
    schwarz_local_kernel<N><<<(int)g, 256, 0, st>>>(r, sw->S, sw->L, sw->prob, A, sw->uext);
    SEM_CUDA_CHECK(cudaGetLastError());
    int64_t gp = (m->nloc + 255) / 256;
    if (gp > (int64_t)m->num_sms * 32) gp = (int64_t)m->num_sms * 32;
    schwarz_sum_kernel<N><<<(int)gp, 256, 0, st>>>(sw->uext, m->dinv32, A, z);
    SEM_CUDA_CHECK(cudaGetLastError());
    if (coarse_iters > 0) {
        J1Tab J{};
        for (int i = 0; i <= m->N; ++i) {
            J.j[i][0] = (float)(0.5 * (1.0 - m->xi[i]));
            J.j[i][1] = (float)(0.5 * (1.0 + m->xi[i]));
        }
        int64_t gc = (m->E * 8 + 255) / 256;
        restrict_kernel<N><<<(int)gc, 256, 0, st>>>(r, m->minv32, J, m->E, sw->rc);
        SEM_CUDA_CHECK(cudaGetLastError());
        int s = gs_launch(sw->mc, sw->rc, SEM_F32, kGsSumMask, st);
        if (s != SEM_OK) return s;
        s = fixed_cg_f32(sw->mc, sw->rc, sw->xc, coarse_iters, coarse_tol, sw->cg_scratch, st);
        if (s != SEM_OK) return s;
        prolong_add_kernel<N><<<(int)gp, 256, 0, st>>>(sw->xc, J, m->E, z);
        SEM_CUDA_CHECK(cudaGetLastError());
    }
    return SEM_OK;
}

int schwarz_apply_f32(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      cudaStream_t st) {
    switch (sw->N) {
#define SEM_SW_CASE(n) \
    case n: return sw_apply_n<n>(sw, r, z, coarse_iters, coarse_tol, st);
        SEM_SW_CASE(2) SEM_SW_CASE(3) SEM_SW_CASE(4) SEM_SW_CASE(5) SEM_SW_CASE(6) SEM_SW_CASE(7)
        SEM_SW_CASE(8) SEM_SW_CASE(9)
#undef SEM_SW_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "Schwarz preconditioner built for 2 <= N <= 9");
    }
}

}  // namespace sem

using namespace sem;

extern "C" {

size_t sem_schwarz_workspace_bytes(const sem_mesh *m, const sem_mesh *mc) {
    if (!m || !mc) return 0;
    size_t off[7];
    return sw_layout(m, mc, off);
}

int sem_schwarz_create(const sem_mesh *m, const sem_mesh *mc, void *ws, size_t bytes, void *stream,
                       sem_schwarz **out) {
    if (!m || !mc || !out) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (m->N < 2 || m->N > 9) return fail(SEM_ERR_UNSUPPORTED, "Schwarz preconditioner built for 2 <= N <= 9");
    if (!m->G32 || !mc->G32) return fail(SEM_ERR_INVALID_ARG, "both meshes need SEM_GEOM_F32");
    if (mc->N != 1 || mc->E != m->E)
        return fail(SEM_ERR_INVALID_ARG, "the coarse mesh must be the N = 1 mesh of the same elements");
    for (int a = 0; a < 3; ++a)
        if (mc->nel[a] != m->nel[a] || mc->periodic[a] != m->periodic[a])
            return fail(SEM_ERR_INVALID_ARG, "the coarse mesh must have the same topology");
    size_t off[7];
    const size_t need = sw_layout(m, mc, off);
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign || bytes < need)
        return fail(SEM_ERR_WORKSPACE, "Schwarz workspace NULL, misaligned or smaller than sem_schwarz_workspace_bytes");
    cudaStream_t st = as_stream(stream);
    const int N = m->N, n1 = N + 1, ne = N + 3;
    const int64_t E = m->E;
    // element lengths from the vertices (mean edge length per direction)
    std::vector<double> V(24 * E);
    SEM_CUDA_CHECK(cudaMemcpyAsync(V.data(), m->verts, sizeof(double) * 24 * E, cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    std::vector<double> hl[3];
    for (int a = 0; a < 3; ++a) hl[a].resize(E);
    static const int edges[3][4] = {{0, 2, 4, 6}, {0, 1, 4, 5}, {0, 1, 2, 3}};
    static const int step[3] = {1, 2, 4};
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int q = 0; q < 4; ++q) {
                const double *p0 = &V[24 * e + 3 * edges[a][q]], *p1 = &V[24 * e + 3 * (edges[a][q] + step[a])];
                s += std::sqrt((p1[0] - p0[0]) * (p1[0] - p0[0]) + (p1[1] - p0[1]) * (p1[1] - p0[1]) +
                               (p1[2] - p0[2]) * (p1[2] - p0[2]));
            }
            hl[a][e] = 0.25 * s;
        }
    // reference 1-D stiffness and mass
    std::vector<double> Ah(n1 * n1, 0.0), Bh(n1, 0.0);
    for (int i = 0; i < n1; ++i) {
        Bh[i] = m->rho[i];
        for (int j = 0; j < n1; ++j) {
            double s = 0.0;
            for (int q = 0; q < n1; ++q) s += m->D.d[q * n1 + i] * m->rho[q] * m->D.d[q * n1 + j];
            Ah[i * n1 + j] = s;
        }
    }
    std::map<FdmKey, int> cache;
    std::vector<float> Stab, Ltab;
    std::vector<int> prob(3 * E);
    const int stride[3] = {1, m->nel[0], m->nel[0] * m->nel[1]};
    std::vector<double> A(ne * ne), B(ne * ne), Sd(ne * ne), ld(ne);
    const int M3 = 3 * N + 1;
    std::vector<double> Af(M3 * M3), Bf(M3 * M3);
    for (int64_t e = 0; e < E; ++e) {
        const int coord[3] = {(int)(e % m->nel[0]), (int)((e / m->nel[0]) % m->nel[1]),
                              (int)(e / ((int64_t)m->nel[0] * m->nel[1]))};
        for (int a = 0; a < 3; ++a) {
            const int c = coord[a], n = m->nel[a], per = m->periodic[a];
            const bool hasL = c > 0 || per, hasR = c < n - 1 || per;
            const bool dirL = !per && c == 0 && ((m->faces >> (2 * a)) & 1);
            const bool dirR = !per && c == n - 1 && ((m->faces >> (2 * a + 1)) & 1);
            const int64_t eL = c > 0 ? e - stride[a] : e + (int64_t)(n - 1) * stride[a];
            const int64_t eR = c < n - 1 ? e + stride[a] : e - (int64_t)(n - 1) * stride[a];
            const double h = hl[a][e], hL = hasL ? hl[a][eL] : h, hR = hasR ? hl[a][eR] : h;
            const FdmKey key{qlen(h), qlen(hL), qlen(hR),
                             (hasL ? 1 : 0) | (hasR ? 2 : 0) | (dirL ? 4 : 0) | (dirR ? 8 : 0)};
            auto it = cache.find(key);
            if (it != cache.end()) {
                prob[3 * e + a] = it->second;
                continue;
            }
            std::fill(Af.begin(), Af.end(), 0.0);
            std::fill(Bf.begin(), Bf.end(), 0.0);
            const double hh[3] = {hL, h, hR};
            for (int q = 0; q < 3; ++q)
                for (int i = 0; i < n1; ++i) {
                    const int gi = q * N + i;
                    Bf[gi * M3 + gi] += 0.5 * hh[q] * Bh[i];
                    for (int j = 0; j < n1; ++j) Af[gi * M3 + q * N + j] += (2.0 / hh[q]) * Ah[i * n1 + j];
                }
            for (int i = 0; i < ne; ++i)
                for (int j = 0; j < ne; ++j) {
                    A[i * ne + j] = Af[(N - 1 + i) * M3 + (N - 1 + j)];
                    B[i * ne + j] = Bf[(N - 1 + i) * M3 + (N - 1 + j)];
                }
            const int dead[4] = {!hasL ? 0 : -1, dirL ? 1 : -1, !hasR ? ne - 1 : -1, dirR ? ne - 2 : -1};
            for (int d : dead) {
                if (d < 0) continue;
                for (int q = 0; q < ne; ++q) {
                    A[d * ne + q] = A[q * ne + d] = 0.0;
                    B[d * ne + q] = B[q * ne + d] = 0.0;
                }
                A[d * ne + d] = B[d * ne + d] = 1.0;
            }
            gen_eig(ne, A.data(), B.data(), Sd.data(), ld.data());
            const int id = (int)(Ltab.size() / ne);
            for (int q = 0; q < ne * ne; ++q) Stab.push_back((float)Sd[q]);
            for (int q = 0; q < ne; ++q) Ltab.push_back((float)ld[q]);
            cache[key] = id;
            prob[3 * e + a] = id;
        }
    }
    sem_schwarz *sw = new (std::nothrow) sem_schwarz();
    if (!sw) return fail(SEM_ERR_INVALID_ARG, "host allocation failed");
    char *base = static_cast<char *>(ws);
    sw->m = m;
    sw->mc = mc;
    sw->N = N;
    sw->ne = ne;
    sw->P = (int)(Ltab.size() / ne);
    sw->S = reinterpret_cast<float *>(base + off[0]);
    sw->L = reinterpret_cast<float *>(base + off[1]);
    sw->prob = reinterpret_cast<int *>(base + off[2]);
    sw->uext = reinterpret_cast<float *>(base + off[3]);
    sw->rc = reinterpret_cast<float *>(base + off[4]);
    sw->xc = reinterpret_cast<float *>(base + off[5]);
    sw->cg_scratch = base + off[6];
    sw->ws_bytes = need;
    cudaError_t ce = cudaMemcpyAsync(sw->S, Stab.data(), sizeof(float) * Stab.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sw->L, Ltab.data(), sizeof(float) * Ltab.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sw->prob, prob.data(), sizeof(int) * prob.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        delete sw;
        return cuda_fail(ce, "sem_schwarz_create upload");
    }
    *out = sw;
    return SEM_OK;
}

int sem_schwarz_destroy(sem_schwarz *sw) {
    delete sw;
    return SEM_OK;
}

int sem_schwarz_problems(const sem_schwarz *sw) { return sw ? sw->P : -1; }

int sem_schwarz_apply(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      void *stream) {
    if (!sw || !r || !z) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (r == z) return fail(SEM_ERR_INVALID_ARG, "r and z must not overlap");
    if (coarse_iters < 0) return fail(SEM_ERR_INVALID_ARG, "coarse_iters < 0");
    return schwarz_apply_f32(sw, r, z, coarse_iters, coarse_tol, as_stream(stream));
}

}  // extern "C"
