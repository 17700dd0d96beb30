// sem_dealias.cu -- dealiased (over-integrated) advection for the
// Navier-Stokes stepper.
//
// The advection term of Eq. 1 (section 3) is quadratic in the velocity; on
// the GLL collocation points its product aliases.  The stepper can instead
// integrate its weak form exactly on M = 3(N+1)/2 Gauss-Legendre points per
// direction (the 3/2 rule), element by element:
//   W_c[i] = int phi_i (u . grad) u_c dx
//          = sum_q w_q [sum_a (sum_m C[m][a] u_m) d u_c / d r_a] phi_i,
// C[m][a] = det J dr_a/dx_m (the cofactor of the trilinear Jacobian, a
// polynomial), u and d u_c / d r_a interpolated from the GLL points.  For
// trilinear elements the integrand is a polynomial of degree <= 3N + 2 per
// direction, so the quadrature is exact.  The stepper then forms
// NL_c = -(Q Q^T W_c) / (Q Q^T B).
//
// GB300 design: FP64 throughout (an explicit term of the FP64 stepper); one
// element per CTA iteration, sum-factorised contractions one direction at a
// time through shared memory; the fine-point factors w_q C[m][a] (9 per
// point) are computed once per mesh into a caller buffer and streamed.
// FP64-pipe bound (~0.45 M FMA per element at N = 7).

#include <cmath>
#include <vector>

#include "sem_common.cuh"

namespace sem {

constexpr int kMaxM = (3 * 10 + 1) / 2;  // N <= 9

__host__ __device__ constexpr int dealias_points(int N) { return (3 * (N + 1) + 1) / 2; }

struct DealiasMats {
    double J[kMaxM * kMaxN1];   // J[q][i] = l_i(z_q)
    double JD[kMaxM * kMaxN1];  // (J D)[q][l] = l_l'(z_q)
    double z[kMaxM], w[kMaxM];  // Gauss-Legendre points and weights
};

// Gauss-Legendre points and weights on [-1, 1]: Newton on P_M from cosine
// guesses, P_M and P_M' by the three-term recurrence.
static void gauss_legendre(int M, double *z, double *w) {
    for (int i = 0; i < M; ++i) {
        double x = -std::cos(3.14159265358979323846 * (i + 0.75) / (M + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int n = 2; n <= M; ++n) {
                const double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            const double dp = M * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int n = 2; n <= M; ++n) {
            const double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        const double dp = M * (x * p1 - p0) / (x * x - 1.0);
        z[i] = x;
        w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

// J (Lagrange basis on the GLL nodes at the Gauss points, barycentric form)
// and J D.
static DealiasMats dealias_mats(const sem_mesh *m) {
    DealiasMats A{};
    const int N1 = m->n1, M = dealias_points(m->N);
    gauss_legendre(M, A.z, A.w);
    double bw[kMaxN1];
    for (int j = 0; j < N1; ++j) {
        double p = 1.0;
        for (int k = 0; k < N1; ++k)
            if (k != j) p *= (m->xi[j] - m->xi[k]);
        bw[j] = 1.0 / p;
    }
    for (int q = 0; q < M; ++q) {
        // a Gauss point on a GLL node (both sets hold 0 when M and N+1 are
        // odd: N = 2, 6): the row is the unit vector of that node
        int hit = -1;
        for (int j = 0; j < N1; ++j)
            if (std::fabs(A.z[q] - m->xi[j]) < 1e-15) hit = j;
        if (hit >= 0) {
            for (int j = 0; j < N1; ++j) A.J[q * N1 + j] = j == hit ? 1.0 : 0.0;
            continue;
        }
        double den = 0.0, t[kMaxN1];
        for (int j = 0; j < N1; ++j) {
            t[j] = bw[j] / (A.z[q] - m->xi[j]);
            den += t[j];
        }
        for (int j = 0; j < N1; ++j) A.J[q * N1 + j] = t[j] / den;
    }
    for (int q = 0; q < M; ++q)
        for (int l = 0; l < N1; ++l) {
            double s = 0.0;
            for (int i = 0; i < N1; ++i) s += A.J[q * N1 + i] * m->D.d[i * N1 + l];
            A.JD[q * N1 + l] = s;
        }
    return A;
}

// W[e][3m+a][q] = w_qi w_qj w_qk C[m][a] at the Gauss points (vertex-relative
// trilinear Jacobian, as in the GLL geometry).
__global__ void dealias_metric_kernel(const double *__restrict__ verts, int64_t E, int M, DealiasMats A,
                                      double *__restrict__ W) {
    const int64_t M3 = (int64_t)M * M * M, n = E * M3;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / M3;
        const int q = (int)(l - e * M3);
        const int qi = q % M, qj = (q / M) % M, qk = q / (M * M);
        const double r = A.z[qi], s = A.z[qj], t = A.z[qk];
        const double fr[2] = {0.5 * (1.0 - r), 0.5 * (1.0 + r)};
        const double fs[2] = {0.5 * (1.0 - s), 0.5 * (1.0 + s)};
        const double ft[2] = {0.5 * (1.0 - t), 0.5 * (1.0 + t)};
        const double df[2] = {-0.5, 0.5};
        double J[3][3] = {};
        const double *V = verts + e * 24;
        for (int v = 1; v < 8; ++v) {
            const int bx = v & 1, by = (v >> 1) & 1, bz = (v >> 2) & 1;
            const double gr = df[bx] * fs[by] * ft[bz];
            const double gs = fr[bx] * df[by] * ft[bz];
            const double gt = fr[bx] * fs[by] * df[bz];
            for (int a = 0; a < 3; ++a) {
                const double X = V[v * 3 + a] - V[a];
                J[a][0] += X * gr;
                J[a][1] += X * gs;
                J[a][2] += X * gt;
            }
        }
        const double wq = A.w[qi] * A.w[qj] * A.w[qk];
        double *We = W + e * 9 * M3;
        for (int mm = 0; mm < 3; ++mm) {
            const int m1 = (mm + 1) % 3, m2 = (mm + 2) % 3;
            for (int a = 0; a < 3; ++a) {
                const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
                const double C = J[m1][a1] * J[m2][a2] - J[m1][a2] * J[m2][a1];
                We[(3 * mm + a) * M3 + q] = wq * C;
            }
        }
    }
}

// ---- sum-factorised contractions through shared memory (all threads) ----
// A 3-D array is indexed [x2][x1][x0], x0 fastest.

// out[x2][x1][o] = sum_i mat[o][i] in[x2][x1][i]          (along x0)
template <int NI, int NO, int D1, int D2>
__device__ __forceinline__ void along0(const double *__restrict__ in, double *__restrict__ out, const double *mat) {
    for (int t = threadIdx.x; t < NO * D1 * D2; t += blockDim.x) {
        const int o = t % NO, r = t / NO;
        const double *src = in + r * NI;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NI; ++i) s = fma(mat[o * NI + i], src[i], s);
        out[t] = s;
    }
}
// out[x2][o][x0] = sum_i mat[o][i] in[x2][i][x0]           (along x1)
template <int NI, int NO, int D0, int D2>
__device__ __forceinline__ void along1(const double *__restrict__ in, double *__restrict__ out, const double *mat) {
    for (int t = threadIdx.x; t < D0 * NO * D2; t += blockDim.x) {
        const int x0 = t % D0, o = (t / D0) % NO, x2 = t / (D0 * NO);
        const double *src = in + (x2 * NI) * D0 + x0;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NI; ++i) s = fma(mat[o * NI + i], src[i * D0], s);
        out[t] = s;
    }
}
// out[o][x1][x0] = sum_i mat[o][i] in[i][x1][x0]           (along x2)
template <int NI, int NO, int D0, int D1>
__device__ __forceinline__ void along2(const double *__restrict__ in, double *__restrict__ out, const double *mat) {
    for (int t = threadIdx.x; t < D0 * D1 * NO; t += blockDim.x) {
        const int x01 = t % (D0 * D1), o = t / (D0 * D1);
        const double *src = in + x01;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NI; ++i) s = fma(mat[o * NI + i], src[i * D0 * D1], s);
        out[t] = s;
    }
}

template <int N>
struct DealiasShape {
    static constexpr int N1 = N + 1, M = dealias_points(N);
    static constexpr int NPT = N1 * N1 * N1, M3 = M * M * M;
    static constexpr int NNM = N1 * N1 * M, NMM = N1 * M * M;
    // doubles: J, J^T, JD, JD-transposed not needed; su[3], ct[3], Y0, Y1, Z00, Z01, Z10, F
    static constexpr int doubles = 3 * M * N1 + 3 * NPT + 3 * M3 + 2 * NNM + 3 * NMM + M3;
    static constexpr int smem = doubles * 8;
};

// W_c (local weak advection, c = 0..2) for every element.
template <int N>
__global__ void __launch_bounds__(256)
    advect_weak_kernel(const double *__restrict__ u0, const double *__restrict__ u1, const double *__restrict__ u2,
                       const double *__restrict__ W, DealiasMats A, int64_t E, double *__restrict__ o0,
                       double *__restrict__ o1, double *__restrict__ o2) {
    using S = DealiasShape<N>;
    constexpr int N1 = S::N1, M = S::M, NPT = S::NPT, M3 = S::M3;
    extern __shared__ __align__(16) double sm[];
    double *J = sm, *JT = J + M * N1, *JD = JT + M * N1;  // JT[i][q] = J[q][i]
    double *su = JD + M * N1;                             // [3][NPT]
    double *ct = su + 3 * NPT;                            // [3][M3]
    double *Y0 = ct + 3 * M3, *Y1 = Y0 + S::NNM;
    double *Z00 = Y1 + S::NNM, *Z01 = Z00 + S::NMM, *Z10 = Z01 + S::NMM;
    double *F = Z10 + S::NMM;
    for (int t = threadIdx.x; t < M * N1; t += blockDim.x) {
        J[t] = A.J[t];
        JD[t] = A.JD[t];
        JT[(t % N1) * M + t / N1] = A.J[t];
    }
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        for (int t = threadIdx.x; t < NPT; t += blockDim.x) {
            su[t] = u0[e * NPT + t];
            su[NPT + t] = u1[e * NPT + t];
            su[2 * NPT + t] = u2[e * NPT + t];
        }
        for (int t = threadIdx.x; t < 3 * M3; t += blockDim.x) ct[t] = 0.0;
        __syncthreads();
        const double *We = W + e * 9 * M3;
        // ct_a = sum_m w C[m][a] u_m at the Gauss points
        for (int m = 0; m < 3; ++m) {
            along0<N1, M, N1, N1>(su + m * NPT, Y0, J);
            __syncthreads();
            along1<N1, M, M, N1>(Y0, Z00, J);
            __syncthreads();
            along2<N1, M, M, M>(Z00, F, J);
            __syncthreads();
            for (int q = threadIdx.x; q < M3; q += blockDim.x) {
                const double f = F[q];
#pragma unroll
                for (int a = 0; a < 3; ++a) ct[a * M3 + q] = fma(We[(3 * m + a) * M3 + q], f, ct[a * M3 + q]);
            }
            __syncthreads();
        }
        for (int c = 0; c < 3; ++c) {
            const double *uc = su + c * NPT;
            along0<N1, M, N1, N1>(uc, Y0, J);   // J along r
            along0<N1, M, N1, N1>(uc, Y1, JD);  // J D along r
            __syncthreads();
            along1<N1, M, M, N1>(Y0, Z00, J);   // (J, J)
            along1<N1, M, M, N1>(Y0, Z01, JD);  // (J, JD)
            along1<N1, M, M, N1>(Y1, Z10, J);   // (JD, J)
            __syncthreads();
            // (u . grad) u_c weighted: F = ct_0 d_r + ct_1 d_s + ct_2 d_t at the Gauss points
            for (int q = threadIdx.x; q < M3; q += blockDim.x) {
                const int x01 = q % (M * M), sk = q / (M * M);
                double dr = 0.0, ds = 0.0, dt = 0.0;
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const int src = k * M * M + x01;
                    dr = fma(J[sk * N1 + k], Z10[src], dr);
                    ds = fma(J[sk * N1 + k], Z01[src], ds);
                    dt = fma(JD[sk * N1 + k], Z00[src], dt);
                }
                F[q] = ct[q] * dr + ct[M3 + q] * ds + ct[2 * M3 + q] * dt;
            }
            __syncthreads();
            // project back with J^T, one direction at a time: k, j, i
            along2<M, N1, M, M>(F, Z00, JT);
            __syncthreads();
            along1<M, N1, M, N1>(Z00, Y0, JT);
            __syncthreads();
            double *out = (c == 0 ? o0 : (c == 1 ? o1 : o2)) + e * NPT;
            for (int t = threadIdx.x; t < NPT; t += blockDim.x) {
                const double *src = Y0 + (t / N1) * M;
                const int i = t % N1;
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < M; ++q) s = fma(JT[i * M + q], src[q], s);
                out[t] = s;
            }
            __syncthreads();
        }
    }
}

size_t dealias_metric_bytes(const sem_mesh *m) {
    if (!m || m->N > 9) return 0;
    const int64_t M = dealias_points(m->N);
    return align_up(sizeof(double) * 9 * (size_t)(m->E * M * M * M));
}

int dealias_metric_launch(const sem_mesh *m, double *W, cudaStream_t st) {
    const DealiasMats A = dealias_mats(m);
    const int M = dealias_points(m->N);
    const int64_t n = m->E * (int64_t)M * M * M;
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)m->num_sms * 32) g = (int64_t)m->num_sms * 32;
    dealias_metric_kernel<<<(int)g, 256, 0, st>>>(m->verts, m->E, M, A, W);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

template <int N>
static int launch_weak_n(const sem_mesh *m, const double *W, const double *const u[3], double *const out[3],
                         cudaStream_t st) {
    using S = DealiasShape<N>;
    auto kern = advect_weak_kernel<N>;
    int dev_max = 0;
    SEM_CUDA_CHECK(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    if (S::smem > dev_max) return fail(SEM_ERR_UNSUPPORTED, "dealiasing: element does not fit in shared memory");
    SEM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::smem));
    int per_sm = 0;
    SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, S::smem));
    int64_t grid = (int64_t)m->num_sms * (per_sm > 0 ? per_sm : 1);
    if (grid > m->E) grid = m->E;
    kern<<<(int)grid, 256, S::smem, st>>>(u[0], u[1], u[2], W, dealias_mats(m), m->E, out[0], out[1], out[2]);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int advect_weak_launch(const sem_mesh *m, const double *W, const double *const u[3], double *const out[3],
                       cudaStream_t st) {
    switch (m->N) {
#define SEM_DA_CASE(n) \
    case n: return launch_weak_n<n>(m, W, u, out, st);
        SEM_DA_CASE(1) SEM_DA_CASE(2) SEM_DA_CASE(3) SEM_DA_CASE(4) SEM_DA_CASE(5)
        SEM_DA_CASE(6) SEM_DA_CASE(7) SEM_DA_CASE(8) SEM_DA_CASE(9)
#undef SEM_DA_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "dealiased advection is built for N <= 9");
    }
}

}  // namespace sem
