// sem_ns.cu -- incompressible Navier-Stokes building blocks and time
// stepper on a fully periodic box mesh.
//
// Paper section 3 (Eq. 1): div v = 0, dv/dt + (v.grad)v = -grad p +
// (1/Re) lap v + F.  Section 3.1: the velocity and pressure are split
// (Karniadakis, Israeli & Orszag 1991), a Krylov method solves the pressure
// system each step and CG the velocity systems.  The scheme written here is
// BDF_k / EXT_k (k = min(step+1, 2)), P_N-P_N collocation without
// dealiasing by default; sem_ns_set_scheme raises the order to 3 (BDF3 /
// EXT3, the high-order splitting the paper cites) and switches the advection
// to its dealiased weak form (sem_dealias.cu):
//   F   = sum_j (b_j/dt) u^{n+1-j} + sum_j a_j NL^{n+1-j},   NL = -(u.grad)u
//   A p = Q Q^T wdiv(F) - mean  (singular periodic Poisson; p has zero mean)
//   (nu A + (b0/dt) B) u_c = Q Q^T [B (F_c - dp/dx_c)]
//
// Element kernels: one element per CTA iteration (grid-stride over
// elements), the element's fields staged in shared memory, one thread per
// point (or several points per thread for large N); derivatives along the
// reference directions are contractions with D from shared memory and are
// mapped to physical space with the stored inverse Jacobian dr_a/dx_m.

#include <cmath>
#include <vector>

#include "sem_common.cuh"

struct sem_ns {
    const sem_mesh *m;
    double nu;
    int steps;
    int order;      // highest BDF/EXT order (1..3); step n uses k = min(n+1, order)
    int dealias;    // advection by the dealiased weak form
    int k;          // order of the step begun
    double *W;      // fine-point factors of the dealiased advection (caller buffer)
    double *binv;   // 1 / (Q Q^T B)
    double *u[3], *uprev[3], *uprev2[3], *unew[3];
    double *nl[3], *nlprev[3], *nlprev2[3];
    double *F[3];
    double *ph[3];  // p^n, p^{n-1}, p^{n-2}
    double *bp;     // last pressure right-hand side (assembled, zero mean)
    double *vr[3];  // velocity right-hand sides
    double *dA;     // local Poisson diagonal
    double *dh;     // inverse assembled Helmholtz diagonal
    double *red;    // reduction partials and results
    double last_h2;
    size_t ws_bytes;
    int begun;        // sem_ns_step_begin done, finish pending
    double begun_dt;
};

namespace sem {

constexpr int kNsRedBlocks = 1184;
constexpr int kNsRedThreads = 256;

template <int N>
__host__ __device__ constexpr int ns_threads() {
    return ((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32 > 512 ? 512
                                                            : ((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32;
}

// derivative of the slab f (element-local, [k][j][i]) along direction a at (i,j,k)
template <int N1>
__device__ __forceinline__ double dref(const double *sD, const double *f, int a, int i, int j, int k) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < N1; ++l) {
        if (a == 0) s = fma(sD[i * N1 + l], f[l + N1 * (j + N1 * k)], s);
        else if (a == 1) s = fma(sD[j * N1 + l], f[i + N1 * (l + N1 * k)], s);
        else s = fma(sD[k * N1 + l], f[i + N1 * (j + N1 * l)], s);
    }
    return s;
}

// gradient of the shared slab f at point p of element e: g_m = sum_a rx[a][m] D_a f
template <int N1>
__device__ __forceinline__ void grad_at(const double *sD, const double *f, const double *__restrict__ rxe,
                                        int npt, int p, double g[3]) {
    const int i = p % N1, j = (p / N1) % N1, k = p / (N1 * N1);
    const double d0 = dref<N1>(sD, f, 0, i, j, k), d1 = dref<N1>(sD, f, 1, i, j, k),
                 d2 = dref<N1>(sD, f, 2, i, j, k);
#pragma unroll
    for (int m = 0; m < 3; ++m)
        g[m] = rxe[m * npt + p] * d0 + rxe[(3 + m) * npt + p] * d1 + rxe[(6 + m) * npt + p] * d2;
}

template <int N>
__global__ void __launch_bounds__(ns_threads<N>())
    grad_kernel(const double *__restrict__ f, const double *__restrict__ rx, DMat Dm, int E,
                double *__restrict__ g) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    __shared__ double sD[N1 * N1], sf[NPT];
    for (int q = threadIdx.x; q < N1 * N1; q += blockDim.x) sD[q] = Dm.d[q];
    const int64_t nloc = (int64_t)E * NPT;
    for (int e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        for (int p = threadIdx.x; p < NPT; p += blockDim.x) sf[p] = f[(int64_t)e * NPT + p];
        __syncthreads();
        const double *rxe = rx + (int64_t)e * 9 * NPT;
        for (int p = threadIdx.x; p < NPT; p += blockDim.x) {
            double gg[3];
            grad_at<N1>(sD, sf, rxe, NPT, p, gg);
            for (int m = 0; m < 3; ++m) g[m * nloc + (int64_t)e * NPT + p] = gg[m];
        }
    }
}

// nl[c] = -sum_m u[m] d u[c] / dx_m
template <int N>
__global__ void __launch_bounds__(ns_threads<N>())
    advect_kernel(const double *__restrict__ u0, const double *__restrict__ u1, const double *__restrict__ u2,
                  const double *__restrict__ rx, DMat Dm, int E, double *__restrict__ n0,
                  double *__restrict__ n1, double *__restrict__ n2) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    __shared__ double sD[N1 * N1], su[3][NPT];
    for (int q = threadIdx.x; q < N1 * N1; q += blockDim.x) sD[q] = Dm.d[q];
    const double *uu[3] = {u0, u1, u2};
    double *nn[3] = {n0, n1, n2};
    for (int e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        for (int p = threadIdx.x; p < NPT; p += blockDim.x)
            for (int c = 0; c < 3; ++c) su[c][p] = uu[c][(int64_t)e * NPT + p];
        __syncthreads();
        const double *rxe = rx + (int64_t)e * 9 * NPT;
        for (int p = threadIdx.x; p < NPT; p += blockDim.x) {
            const double v0 = su[0][p], v1 = su[1][p], v2 = su[2][p];
            for (int c = 0; c < 3; ++c) {
                double g[3];
                grad_at<N1>(sD, su[c], rxe, NPT, p, g);
                nn[c][(int64_t)e * NPT + p] = -(v0 * g[0] + v1 * g[1] + v2 * g[2]);
            }
        }
    }
}

// Forcing F_c = sum_{j<k} (s_j u^{n-j}_c + a_j NL^{n-j}_c), stored; then the
// local weak divergence w = sum_a D_a^T [B sum_m rx[a][m] F_m].  With k = 0,
// F is an input.
struct NsForce {
    const double *u[3][3];   // [level j][component]
    const double *nl[3][3];
    double s[3], a[3];
    int k;
};

template <int N>
__global__ void __launch_bounds__(ns_threads<N>())
    force_wdiv_kernel(const NsForce H, double *__restrict__ F0, double *__restrict__ F1, double *__restrict__ F2,
                      const double *__restrict__ Bm, const double *__restrict__ rx, DMat Dm, int E,
                      double *__restrict__ w) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    __shared__ double sD[N1 * N1], sphi[3][NPT];
    for (int q = threadIdx.x; q < N1 * N1; q += blockDim.x) sD[q] = Dm.d[q];
    for (int e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        const double *rxe = rx + (int64_t)e * 9 * NPT;
        for (int p = threadIdx.x; p < NPT; p += blockDim.x) {
            const int64_t l = (int64_t)e * NPT + p;
            double f[3];
            if (H.k > 0) {
                for (int c = 0; c < 3; ++c) {
                    double v = 0.0;
                    for (int j = 0; j < H.k; ++j) v += H.s[j] * H.u[j][c][l] + H.a[j] * H.nl[j][c][l];
                    f[c] = v;
                }
                F0[l] = f[0];
                F1[l] = f[1];
                F2[l] = f[2];
            } else {
                f[0] = F0[l];
                f[1] = F1[l];
                f[2] = F2[l];
            }
            const double b = Bm[l];
            for (int a = 0; a < 3; ++a)
                sphi[a][p] = b * (rxe[(3 * a) * NPT + p] * f[0] + rxe[(3 * a + 1) * NPT + p] * f[1] +
                                  rxe[(3 * a + 2) * NPT + p] * f[2]);
        }
        __syncthreads();
        for (int p = threadIdx.x; p < NPT; p += blockDim.x) {
            const int i = p % N1, j = (p / N1) % N1, k = p / (N1 * N1);
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < N1; ++q) {
                s = fma(sD[q * N1 + i], sphi[0][q + N1 * (j + N1 * k)], s);
                s = fma(sD[q * N1 + j], sphi[1][i + N1 * (q + N1 * k)], s);
                s = fma(sD[q * N1 + k], sphi[2][i + N1 * (j + N1 * q)], s);
            }
            w[(int64_t)e * NPT + p] = s;
        }
    }
}

// nl <- -binv * nl (the assembled weak advection to its strong, continuous form)
__global__ void scale_neg_kernel(double *__restrict__ a, const double *__restrict__ binv, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        a[l] = -binv[l] * a[l];
}

// velocity right-hand sides vr_c = B (F_c - d p / d x_c) (local)
template <int N>
__global__ void __launch_bounds__(ns_threads<N>())
    vrhs_kernel(const double *__restrict__ pr, const double *__restrict__ F0, const double *__restrict__ F1,
                const double *__restrict__ F2, const double *__restrict__ Bm, const double *__restrict__ rx,
                DMat Dm, int E, double *__restrict__ v0, double *__restrict__ v1, double *__restrict__ v2) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    __shared__ double sD[N1 * N1], sp[NPT];
    for (int q = threadIdx.x; q < N1 * N1; q += blockDim.x) sD[q] = Dm.d[q];
    for (int e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        for (int p = threadIdx.x; p < NPT; p += blockDim.x) sp[p] = pr[(int64_t)e * NPT + p];
        __syncthreads();
        const double *rxe = rx + (int64_t)e * 9 * NPT;
        for (int p = threadIdx.x; p < NPT; p += blockDim.x) {
            const int64_t l = (int64_t)e * NPT + p;
            double g[3];
            grad_at<N1>(sD, sp, rxe, NPT, p, g);
            const double b = Bm[l];
            v0[l] = b * (F0[l] - g[0]);
            v1[l] = b * (F1[l] - g[1]);
            v2[l] = b * (F2[l] - g[2]);
        }
    }
}

// Two-stage deterministic reduction: block partials of out[0] = sum_l w_l a_l
// (times b_l if given) and out[1] = sum_l w_l, then one block sums them in
// block order.
__global__ void __launch_bounds__(kNsRedThreads)
    red_stage1(const double *__restrict__ w, const double *__restrict__ a, const double *__restrict__ b, int64_t n,
               double *__restrict__ part) {
    __shared__ double sh[2][kNsRedThreads / 32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double t = a[l] * (b ? b[l] : 1.0);
        s0 = fma(w[l], t, s0);
        s1 += w[l];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int q = 0; q < kNsRedThreads / 32; ++q) {
            t0 += sh[0][q];
            t1 += sh[1][q];
        }
        part[blockIdx.x] = t0;
        part[kNsRedBlocks + blockIdx.x] = t1;
    }
}

// sum (B/mult)(u0^2 + u1^2 + u2^2) and sum B/mult, block partials
__global__ void __launch_bounds__(kNsRedThreads)
    energy_stage1(const double *__restrict__ Bm, const double *__restrict__ minv, const double *__restrict__ u0,
                  const double *__restrict__ u1, const double *__restrict__ u2, int64_t n, double *__restrict__ part) {
    __shared__ double sh[2][kNsRedThreads / 32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double w = Bm[l] * minv[l];
        s0 = fma(w, u0[l] * u0[l] + u1[l] * u1[l] + u2[l] * u2[l], s0);
        s1 += w;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int q = 0; q < kNsRedThreads / 32; ++q) {
            t0 += sh[0][q];
            t1 += sh[1][q];
        }
        part[blockIdx.x] = t0;
        part[kNsRedBlocks + blockIdx.x] = t1;
    }
}

__global__ void red_stage2(const double *__restrict__ part, double *__restrict__ out) {
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int q = 0; q < kNsRedBlocks; ++q) {
            t0 += part[q];
            t1 += part[kNsRedBlocks + q];
        }
        out[0] = t0;
        out[1] = t1;
    }
}

// f -= out[0] / count  (count given on the host)
__global__ void sub_mean_kernel(double *__restrict__ f, int64_t n, const double *__restrict__ sum, double inv_count) {
    const double mu = sum[0] * inv_count;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        f[l] -= mu;
}

__global__ void helm_diag_kernel(const double *__restrict__ dA, const double *__restrict__ Bm, double h1, double h2,
                                 int64_t n, double *__restrict__ dh) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        dh[l] = h1 * dA[l] + h2 * Bm[l];
}

__global__ void invert_kernel_ns(double *__restrict__ d, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        d[l] = 1.0 / d[l];
}

static int grid_pts(const sem_mesh *m) {
    int64_t g = (m->nloc + 255) / 256;
    if (g > (int64_t)m->num_sms * 32) g = (int64_t)m->num_sms * 32;
    return (int)(g < 1 ? 1 : g);
}

static int grid_el(const sem_mesh *m) {
    int64_t g = m->E;
    if (g > (int64_t)m->num_sms * 16) g = (int64_t)m->num_sms * 16;
    return (int)g;
}

#define SEM_NS_DISPATCH(KERNEL, ...)                                                                   \
    switch (m->N) {                                                                                     \
        case 1: KERNEL<1><<<grid_el(m), ns_threads<1>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 2: KERNEL<2><<<grid_el(m), ns_threads<2>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 3: KERNEL<3><<<grid_el(m), ns_threads<3>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 4: KERNEL<4><<<grid_el(m), ns_threads<4>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 5: KERNEL<5><<<grid_el(m), ns_threads<5>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 6: KERNEL<6><<<grid_el(m), ns_threads<6>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 7: KERNEL<7><<<grid_el(m), ns_threads<7>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 8: KERNEL<8><<<grid_el(m), ns_threads<8>(), 0, st>>>(__VA_ARGS__); break;                  \
        case 9: KERNEL<9><<<grid_el(m), ns_threads<9>(), 0, st>>>(__VA_ARGS__); break;                  \
        default: return fail(SEM_ERR_UNSUPPORTED, "Navier-Stokes kernels are built for N <= 9");       \
    }                                                                                                   \
    SEM_CUDA_CHECK(cudaGetLastError());

static int need_rx(const sem_mesh *m) {
    if (!m) return fail(SEM_ERR_INVALID_ARG, "NULL mesh");
    if (!m->rx) return fail(SEM_ERR_INVALID_ARG, "mesh built without SEM_GEOM_RX");
    if (m->N > 9) return fail(SEM_ERR_UNSUPPORTED, "Navier-Stokes kernels are built for N <= 9");
    return SEM_OK;
}

static int launch_grad(const sem_mesh *m, const double *f, double *g, cudaStream_t st) {
    SEM_NS_DISPATCH(grad_kernel, f, m->rx, m->D, (int)m->E, g)
    return SEM_OK;
}

static int launch_advect(const sem_mesh *m, const double *const u[3], double *const nl[3], cudaStream_t st) {
    SEM_NS_DISPATCH(advect_kernel, u[0], u[1], u[2], m->rx, m->D, (int)m->E, nl[0], nl[1], nl[2])
    return SEM_OK;
}

static int launch_force_wdiv(const sem_mesh *m, const NsForce &H, double *const F[3], double *w, cudaStream_t st) {
    SEM_NS_DISPATCH(force_wdiv_kernel, H, F[0], F[1], F[2], m->B, m->rx, m->D, (int)m->E, w)
    return SEM_OK;
}

static int launch_vrhs(const sem_mesh *m, const double *p, double *const F[3], double *const v[3],
                       cudaStream_t st) {
    SEM_NS_DISPATCH(vrhs_kernel, p, F[0], F[1], F[2], m->B, m->rx, m->D, (int)m->E, v[0], v[1], v[2])
    return SEM_OK;
}

// out[0] = sum w a (b), out[1] = sum w
static int reduce(const sem_mesh *m, const double *w, const double *a, const double *b, double *part,
                  double *out, cudaStream_t st) {
    red_stage1<<<kNsRedBlocks, kNsRedThreads, 0, st>>>(w, a, b, m->nloc, part);
    red_stage2<<<1, 32, 0, st>>>(part, out);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

// f <- f - (unique-node mean of f)
static int remove_mean(const sem_mesh *m, double *f, double *red, cudaStream_t st) {
    int s = reduce(m, m->minv, f, nullptr, red, red + 2 * kNsRedBlocks, st);
    if (s != SEM_OK) return s;
    sub_mean_kernel<<<grid_pts(m), 256, 0, st>>>(f, m->nloc, red + 2 * kNsRedBlocks, 1.0 / (double)m->nglob);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

static size_t ns_red_bytes() { return align_up(sizeof(double) * (2 * kNsRedBlocks + 8)); }

}  // namespace sem

// The state's advection form on u (3 fields) into nl: collocation, or the
// dealiased weak form assembled and divided by the assembled mass.
static int ns_advect_into(const sem_ns *ns, const double *const u[3], double *const nl[3], cudaStream_t st) {
    using namespace sem;
    const sem_mesh *m = ns->m;
    if (!ns->dealias) return launch_advect(m, u, nl, st);
    int s = advect_weak_launch(m, ns->W, u, nl, st);
    if (s != SEM_OK) return s;
    for (int c = 0; c < 3; ++c) {
        s = gs_launch(m, nl[c], SEM_F64, kGsSum, st);
        if (s != SEM_OK) return s;
        scale_neg_kernel<<<grid_pts(m), 256, 0, st>>>(nl[c], ns->binv, m->nloc);
        SEM_CUDA_CHECK(cudaGetLastError());
    }
    return SEM_OK;
}

using namespace sem;

static double *ns_slot(const sem_ns *ns, int which);

extern "C" {

int sem_gradient(const sem_mesh *m, const double *f, double *g, void *stream) {
    int s = need_rx(m);
    if (s != SEM_OK) return s;
    if (!f || !g) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    return launch_grad(m, f, g, as_stream(stream));
}

int sem_advect(const sem_mesh *m, const double *u, double *nl, void *stream) {
    int s = need_rx(m);
    if (s != SEM_OK) return s;
    if (!u || !nl) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    const double *uu[3] = {u, u + m->nloc, u + 2 * m->nloc};
    double *nn[3] = {nl, nl + m->nloc, nl + 2 * m->nloc};
    return launch_advect(m, uu, nn, as_stream(stream));
}

int sem_weak_div(const sem_mesh *m, const double *F, double *w, void *stream) {
    int s = need_rx(m);
    if (s != SEM_OK) return s;
    if (!F || !w) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    NsForce H{};
    H.k = 0;  // F is the input
    double *FF[3] = {const_cast<double *>(F), const_cast<double *>(F + m->nloc), const_cast<double *>(F + 2 * m->nloc)};
    return launch_force_wdiv(m, H, FF, w, as_stream(stream));
}

// 34 fields: per component u, u^{n-1}, u^{n-2}, u^{n+1}, NL, NL^{n-1},
// NL^{n-2}, F, pressure history slot, velocity right-hand side; plus bp, dA,
// dh, binv; then reductions.
constexpr int kNsFields = 34;

size_t sem_ns_workspace_bytes(const sem_mesh *m) {
    if (!m) return 0;
    return kNsFields * align_up(sizeof(double) * m->nloc) + ns_red_bytes();
}

int sem_ns_create(const sem_mesh *m, double Re, void *ws, size_t bytes, void *stream, sem_ns **out) {
    int s = need_rx(m);
    if (s != SEM_OK) return s;
    if (!out || !(Re > 0.0)) return fail(SEM_ERR_INVALID_ARG, "out NULL or Re <= 0");
    for (int a = 0; a < 3; ++a)
        if (!m->periodic[a]) return fail(SEM_ERR_UNSUPPORTED, "the stepper needs a fully periodic box");
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign || bytes < sem_ns_workspace_bytes(m))
        return fail(SEM_ERR_WORKSPACE, "NS workspace NULL, misaligned or smaller than sem_ns_workspace_bytes");
    sem_ns *ns = new sem_ns();
    ns->m = m;
    ns->nu = 1.0 / Re;
    ns->steps = 0;
    ns->last_h2 = -1.0;
    ns->ws_bytes = sem_ns_workspace_bytes(m);
    char *p = static_cast<char *>(ws);
    const size_t vb = align_up(sizeof(double) * m->nloc);
    auto take = [&]() { double *q = reinterpret_cast<double *>(p); p += vb; return q; };
    for (int c = 0; c < 3; ++c) {
        ns->u[c] = take();
        ns->uprev[c] = take();
        ns->uprev2[c] = take();
        ns->unew[c] = take();
        ns->nl[c] = take();
        ns->nlprev[c] = take();
        ns->nlprev2[c] = take();
        ns->F[c] = take();
        ns->ph[c] = take();
        ns->vr[c] = take();
    }
    ns->bp = take();
    ns->dA = take();
    ns->dh = take();
    ns->binv = take();
    ns->order = 2;
    ns->dealias = 0;
    ns->k = 1;
    ns->W = nullptr;
    ns->red = reinterpret_cast<double *>(p);  // after the kNsFields slots
    cudaStream_t st = as_stream(stream);
    s = jacobi_diag_launch(m, ns->dA, st);
    if (s != SEM_OK) {
        delete ns;
        return s;
    }
    for (int c = 0; c < 3; ++c) {
        cudaError_t e = cudaMemsetAsync(ns->ph[c], 0, sizeof(double) * m->nloc, st);
        if (e != cudaSuccess) {
            delete ns;
            return cuda_fail(e, "cudaMemsetAsync");
        }
    }
    *out = ns;
    return SEM_OK;
}

size_t sem_ns_dealias_bytes(const sem_mesh *m) { return dealias_metric_bytes(m); }

int sem_ns_set_scheme(sem_ns *ns, int order, int dealias, void *d_dealias, size_t bytes, void *stream) {
    if (!ns || order < 1 || order > 3) return fail(SEM_ERR_INVALID_ARG, "NULL state or order outside 1..3");
    const sem_mesh *m = ns->m;
    cudaStream_t st = as_stream(stream);
    if (dealias) {
        if (!d_dealias || reinterpret_cast<uintptr_t>(d_dealias) % kAlign || bytes < dealias_metric_bytes(m))
            return fail(SEM_ERR_WORKSPACE, "dealias buffer NULL, misaligned or smaller than sem_ns_dealias_bytes");
        double *W = static_cast<double *>(d_dealias);
        int s = dealias_metric_launch(m, W, st);
        if (s != SEM_OK) return s;
        // 1 / (Q Q^T B)
        SEM_CUDA_CHECK(cudaMemcpyAsync(ns->binv, m->B, sizeof(double) * m->nloc, cudaMemcpyDeviceToDevice, st));
        s = gs_launch(m, ns->binv, SEM_F64, kGsSum, st);
        if (s != SEM_OK) return s;
        invert_kernel_ns<<<grid_pts(m), 256, 0, st>>>(ns->binv, m->nloc);
        SEM_CUDA_CHECK(cudaGetLastError());
        ns->W = W;
    } else {
        ns->W = nullptr;
    }
    ns->order = order;
    ns->dealias = dealias ? 1 : 0;
    return SEM_OK;
}

int sem_ns_advect(const sem_ns *ns, const double *u, double *nl, void *stream) {
    if (!ns || !u || !nl) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    const int64_t n = ns->m->nloc;
    const double *uu[3] = {u, u + n, u + 2 * n};
    double *nn[3] = {nl, nl + n, nl + 2 * n};
    return ns_advect_into(ns, uu, nn, as_stream(stream));
}

int sem_ns_destroy(sem_ns *ns) {
    delete ns;
    return SEM_OK;
}

int sem_ns_set_velocity(sem_ns *ns, const double *u, void *stream) {
    if (!ns || !u) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    const sem_mesh *m = ns->m;
    cudaStream_t st = as_stream(stream);
    for (int c = 0; c < 3; ++c) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(ns->u[c], u + c * m->nloc, sizeof(double) * m->nloc,
                                       cudaMemcpyDeviceToDevice, st));
        SEM_CUDA_CHECK(cudaMemsetAsync(ns->ph[c], 0, sizeof(double) * m->nloc, st));
    }
    ns->steps = 0;
    return SEM_OK;
}

int sem_ns_get(const sem_ns *ns, int which, double *dst, void *stream) {
    if (!ns || !dst) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    const double *src = ns_slot(ns, which);
    if (!src) return fail(SEM_ERR_INVALID_ARG, "unknown field");
    SEM_CUDA_CHECK(cudaMemcpyAsync(dst, src, sizeof(double) * ns->m->nloc, cudaMemcpyDeviceToDevice,
                                   as_stream(stream)));
    return SEM_OK;
}

size_t sem_ns_scratch_bytes(const sem_ns *ns, const sem_pcg_opts *popts, const sem_pcg_opts *vopts) {
    if (!ns) return 0;
    size_t a = sem_pcg_scratch_bytes(ns->m, popts), b = sem_pcg_scratch_bytes(ns->m, vopts);
    return a > b ? a : b;
}

int sem_ns_step_begin(sem_ns *ns, double dt, void *stream) {
    NvtxRange nvtx_range("NS step: advection, pressure right-hand side");
    if (!ns || !(dt > 0.0)) return fail(SEM_ERR_INVALID_ARG, "NULL state or dt <= 0");
    const sem_mesh *m = ns->m;
    cudaStream_t st = as_stream(stream);
    const int k = ns->steps + 1 < ns->order ? ns->steps + 1 : ns->order;
    // BDF_k history weights b_j (b0 in step_finish) and EXT_k weights a_j
    static const double kB[4][3] = {{0, 0, 0}, {1.0, 0, 0}, {2.0, -0.5, 0}, {3.0, -1.5, 1.0 / 3.0}};
    static const double kA[4][3] = {{0, 0, 0}, {1.0, 0, 0}, {2.0, -1.0, 0}, {3.0, -3.0, 1.0}};
    // advection at t^n, forcing, weak divergence -> pressure right-hand side
    int s = ns_advect_into(ns, ns->u, ns->nl, st);
    if (s != SEM_OK) return s;
    NsForce H{};
    H.k = k;
    for (int c = 0; c < 3; ++c) {
        H.u[0][c] = ns->u[c];
        H.u[1][c] = ns->uprev[c];
        H.u[2][c] = ns->uprev2[c];
        H.nl[0][c] = ns->nl[c];
        H.nl[1][c] = ns->nlprev[c];
        H.nl[2][c] = ns->nlprev2[c];
    }
    for (int j = 0; j < 3; ++j) {
        H.s[j] = kB[k][j] / dt;
        H.a[j] = kA[k][j];
    }
    s = launch_force_wdiv(m, H, ns->F, ns->bp, st);
    if (s != SEM_OK) return s;
    ns->k = k;
    s = gs_launch(m, ns->bp, SEM_F64, kGsSum, st);
    if (s != SEM_OK) return s;
    s = remove_mean(m, ns->bp, ns->red, st);
    if (s != SEM_OK) return s;
    ns->begun = 1;
    ns->begun_dt = dt;
    return SEM_OK;
}

int sem_ns_step_finish(sem_ns *ns, const sem_pcg_opts *popts, const sem_pcg_opts *vopts, const double *p_guess,
                       sem_pcg_stats *pstats, sem_pcg_stats *vstats, void *scratch, size_t scratch_bytes,
                       void *stream) {
    NvtxRange nvtx_range("NS step: pressure and velocity solves");
    if (!ns || !popts || !vopts || !pstats || !vstats || !scratch) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (!ns->begun) return fail(SEM_ERR_INVALID_ARG, "sem_ns_step_finish without sem_ns_step_begin");
    const sem_mesh *m = ns->m;
    cudaStream_t st = as_stream(stream);
    const double dt = ns->begun_dt;
    const double b0 = ns->k == 1 ? 1.0 : (ns->k == 2 ? 1.5 : 11.0 / 6.0);
    int s;
    // pressure: solve into the oldest history slot
    double *pn = ns->ph[2];
    sem_pcg_opts po = *popts;
    po.h1 = 1.0;
    po.h2 = 0.0;
    po.dinv = nullptr;
    if (p_guess) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(pn, p_guess, sizeof(double) * m->nloc, cudaMemcpyDeviceToDevice, st));
        po.use_initial_guess = 1;
    } else if (popts->use_initial_guess) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(pn, ns->ph[0], sizeof(double) * m->nloc, cudaMemcpyDeviceToDevice, st));
    }
    s = sem_pcg_solve(m, ns->bp, pn, &po, pstats, scratch, scratch_bytes, stream);
    if (s != SEM_OK) return s;
    s = remove_mean(m, pn, ns->red, st);
    if (s != SEM_OK) return s;
    // velocity right-hand sides and Helmholtz solves
    s = launch_vrhs(m, pn, ns->F, ns->vr, st);
    if (s != SEM_OK) return s;
    const double h2 = b0 / dt;
    if (h2 != ns->last_h2) {
        helm_diag_kernel<<<grid_pts(m), 256, 0, st>>>(ns->dA, m->B, ns->nu, h2, m->nloc, ns->dh);
        SEM_CUDA_CHECK(cudaGetLastError());
        s = gs_launch(m, ns->dh, SEM_F64, kGsSum, st);
        if (s != SEM_OK) return s;
        invert_kernel_ns<<<grid_pts(m), 256, 0, st>>>(ns->dh, m->nloc);
        SEM_CUDA_CHECK(cudaGetLastError());
        ns->last_h2 = h2;
    }
    sem_pcg_opts vo = *vopts;
    vo.h1 = ns->nu;
    vo.h2 = h2;
    vo.dinv = ns->dh;
    vo.precision = SEM_PCG_F64;
    vo.use_initial_guess = 1;
    for (int c = 0; c < 3; ++c) {
        s = gs_launch(m, ns->vr[c], SEM_F64, kGsSum, st);
        if (s != SEM_OK) return s;
        SEM_CUDA_CHECK(cudaMemcpyAsync(ns->unew[c], ns->u[c], sizeof(double) * m->nloc, cudaMemcpyDeviceToDevice, st));
        s = sem_pcg_solve(m, ns->vr[c], ns->unew[c], &vo, &vstats[c], scratch, scratch_bytes, stream);
        if (s != SEM_OK) return s;
    }
    // history: u^{n-2} <- u^{n-1} <- u^n <- u^{n+1};  NL^{n-2} <- NL^{n-1} <- NL^n;  p ring
    for (int c = 0; c < 3; ++c) {
        double *t = ns->uprev2[c];
        ns->uprev2[c] = ns->uprev[c];
        ns->uprev[c] = ns->u[c];
        ns->u[c] = ns->unew[c];
        ns->unew[c] = t;
        double *q = ns->nlprev2[c];
        ns->nlprev2[c] = ns->nlprev[c];
        ns->nlprev[c] = ns->nl[c];
        ns->nl[c] = q;
    }
    double *pold = ns->ph[2];
    ns->ph[2] = ns->ph[1];
    ns->ph[1] = ns->ph[0];
    ns->ph[0] = pold;
    ns->steps += 1;
    ns->begun = 0;
    return SEM_OK;
}

int sem_ns_step(sem_ns *ns, double dt, const sem_pcg_opts *popts, const sem_pcg_opts *vopts,
                const double *p_guess, sem_pcg_stats *pstats, sem_pcg_stats *vstats, void *scratch,
                size_t scratch_bytes, void *stream) {
    int s = sem_ns_step_begin(ns, dt, stream);
    if (s != SEM_OK) return s;
    return sem_ns_step_finish(ns, popts, vopts, p_guess, pstats, vstats, scratch, scratch_bytes, stream);
}

}  // extern "C"

static double *ns_slot(const sem_ns *ns, int which) {
    if (which >= 0 && which < 3) return ns->u[which];
    if (which >= 3 && which < 6) return ns->ph[which - 3];
    if (which == 6) return ns->bp;
    if (which >= 7 && which < 10) return ns->uprev[which - 7];
    if (which >= 10 && which < 13) return ns->nlprev[which - 10];
    if (which >= 13 && which < 16) return ns->uprev2[which - 13];
    if (which >= 16 && which < 19) return ns->nlprev2[which - 16];
    return nullptr;
}

extern "C" {

int sem_ns_set(sem_ns *ns, int which, const double *src, void *stream) {
    if (!ns || !src) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    double *dst = ns_slot(ns, which);
    if (!dst) return fail(SEM_ERR_INVALID_ARG, "unknown field");
    SEM_CUDA_CHECK(cudaMemcpyAsync(dst, src, sizeof(double) * ns->m->nloc, cudaMemcpyDeviceToDevice,
                                   as_stream(stream)));
    return SEM_OK;
}

int sem_ns_get_steps(const sem_ns *ns) { return ns ? ns->steps : -1; }

int sem_ns_set_steps(sem_ns *ns, int steps) {
    if (!ns || steps < 0) return fail(SEM_ERR_INVALID_ARG, "NULL state or steps < 0");
    ns->steps = steps;
    ns->begun = 0;
    return SEM_OK;
}

int sem_ns_kinetic_energy(const sem_ns *ns, double *energy, void *scratch, size_t scratch_bytes, void *stream) {
    if (!ns || !energy || !scratch) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (scratch_bytes < ns_red_bytes()) return fail(SEM_ERR_WORKSPACE, "scratch too small");
    const sem_mesh *m = ns->m;
    cudaStream_t st = as_stream(stream);
    double *part = static_cast<double *>(scratch);
    double *res = part + 2 * kNsRedBlocks;
    // res[0] = sum (B/mult) |u|^2, res[1] = sum B/mult (the volume)
    energy_stage1<<<kNsRedBlocks, kNsRedThreads, 0, st>>>(m->B, m->minv, ns->u[0], ns->u[1], ns->u[2], m->nloc,
                                                          part);
    red_stage2<<<1, 32, 0, st>>>(part, res);
    SEM_CUDA_CHECK(cudaGetLastError());
    double h[2];
    SEM_CUDA_CHECK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    *energy = 0.5 * h[0] / h[1];
    return SEM_OK;
}

}  // extern "C"
