// sem_ax64.cu -- the FP64 local stiffness / Helmholtz operator with
// even/odd ("centro-antisymmetric") derivative contractions.
//
// Paper section 3.1: every operator except the gather-scatter is applied
// element by element, matrix free, on the order-N GLL Lagrange basis.  Per
// element e:
//   u_r = D u (along r), u_s, u_t likewise;
//   (v_r, v_s, v_t) = G (u_r, u_s, u_t), G the six symmetric geometric factors;
//   w = D^T v_r + D^T v_s + D^T v_t   [Helmholtz: w = h1 w + h2 B u].
//
// Why a kernel of its own: on GB300 FP64 arithmetic, not HBM, bounds this
// operator.  The FP64 FMA pipe retires ~1.9 FMAs per clock per SM (1.2
// TFLOP/s), FP64 MMA (mma.sync m8n8k4) shares that unit (1.05 TFLOP/s alone,
// 1.03 together), so the tensor cores add nothing, and the operator's 64
// bytes per point would need ~12 TFLOP/s to be bandwidth bound.  The time is
// the number of FP64 instructions per point, so this kernel minimises it:
//  - the GLL derivative matrix is centro-antisymmetric, D[N-i][N-l] =
//    -D[i][l] (so is D^T).  With e_l = x_l + x_{N-l}, o_l = x_l - x_{N-l}
//    (l < H = (N+1)/2 rounded down) a line y = M x splits into
//        P_i = sum_l A_il e_l (+ M[i][m] x_m, middle point m, odd N+1),
//        Q_i = sum_l B_il o_l,   A_il = (M[i][l] + M[i][N-l]) / 2,
//                                B_il = (M[i][l] - M[i][N-l]) / 2,
//        y_i = P_i + Q_i,  y_{N-i} = Q_i - P_i   (i < H),
//        y_m = sum_l M[m][l] o_l                  (odd N+1);
//    at N = 7 a line costs 8 + 32 + 8 = 48 instead of 64 FP64 operations;
//  - one thread owns a whole line in each contraction pass (it needs every
//    input of the line for e and o), so the coefficients are the same for
//    all threads: they sit in the kernel parameters and enter every FMA as
//    a constant-bank operand (no registers, no shared-memory loads);
//  - per point: 18 forward + 9 geometric-factor + 18 backward + 2 summing
//    FP64 operations = 47 (the direct form: 59); the fused CG form adds 3.
// Everything else (addresses, shared memory, the bulk copies) runs on other
// units and is hidden behind the FP64 pipe.
//
// Layout: a persistent grid, one element per CTA at a time, one thread per
// line ((N+1)^2 lines per direction).  The element's input slab(s) arrive in
// shared memory by 1-D bulk copies (TMA), the buffer refilled with the next
// element's slabs as soon as it has been consumed; the contiguous [6][npt]
// geometric factors are read from global memory in the column pass that
// uses them.  Passes per element, with a CTA barrier after each (after pass
// 1 only in the CG form, which writes the new search direction there):
//   1. column pass (thread = (i, j) column along t): the operand (CG: the
//      new search direction) into registers, the t-derivative in registers;
//   2. r and s derivatives (thread = one r-line, then one s-line) into two
//      work fields;
//   3. column pass: v = G (u_r, u_s, u_t) (v_r, v_s in place), D^T along t
//      in registers;
//   4. D^T along r and s, in place;
//   5. column pass: w = sum of the three, stored to global memory.
// Every mbarrier wait is bounded in time; on time-out the kernel records
// kDevTimeoutTma in the mesh error word, all CTAs leave the loop and each
// drains its copies still in flight.

#include <cmath>

#include "sem_common.cuh"

namespace sem {

// Even/odd coefficients of one line contraction y = M x (M = D or D^T).
template <int N1>
struct EoMat {
    static constexpr int H = N1 / 2;
    double a[H * H];     // A_il, i, l < H
    double b[H * H];     // B_il
    double c[H + 1];     // odd N1: M[i][m], i < H (middle column)
    double mr[H + 1];    // odd N1: M[m][l], l < H (middle row)
};

template <int N1>
struct Eo64 {
    EoMat<N1> f, bk;  // forward D, backward D^T
    // 1, -1 and -0 as run-time values: every FP64 add, subtract and multiply
    // of the kernel is issued as an FMA with one of them (x + y = fma(x, 1, y),
    // x - y = fma(y, -1, x), a b = fma(a, b, -0), bit-identical results), since
    // GB300 retires FP64 FMAs at 1.89 per clock per SM but adds and multiplies
    // at 1.59; being kernel parameters, the compiler cannot fold them back.
    double one, mone, mzero;
};

// FP64 add / subtract / multiply as FMAs with run-time unit constants.
struct F64Ops {
    double one, mone, mzero;
    __device__ __forceinline__ double add(double x, double y) const { return fma(x, one, y); }
    __device__ __forceinline__ double sub(double x, double y) const { return fma(y, mone, x); }
    __device__ __forceinline__ double mul(double a, double b) const { return fma(a, b, mzero); }
};

template <int N>
__host__ __device__ constexpr int ax64_threads() {
    return ((N + 1) * (N + 1) + 31) / 32 * 32;
}

// One line: y = M x in even/odd form (see the file header); every
// operation an FMA.
template <int N1>
__device__ __forceinline__ void eo_line(const double (&x)[N1], double (&y)[N1], const EoMat<N1> &M,
                                        const F64Ops &f) {
    constexpr int H = N1 / 2;
    constexpr bool ODD = (N1 % 2) != 0;
    double e[H], o[H];
#pragma unroll
    for (int l = 0; l < H; ++l) {
        e[l] = f.add(x[l], x[N1 - 1 - l]);
        o[l] = f.sub(x[l], x[N1 - 1 - l]);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        double P = ODD ? f.mul(M.c[i], x[H]) : 0.0;
        double Q = 0.0;
#pragma unroll
        for (int l = 0; l < H; ++l) {
            P = (ODD || l > 0) ? fma(M.a[i * H + l], e[l], P) : f.mul(M.a[i * H], e[0]);
            Q = l > 0 ? fma(M.b[i * H + l], o[l], Q) : f.mul(M.b[i * H], o[0]);
        }
        y[i] = f.add(P, Q);
        y[N1 - 1 - i] = f.sub(Q, P);
    }
    if constexpr (ODD) {
        double m = 0.0;
#pragma unroll
        for (int l = 0; l < H; ++l) m = l > 0 ? fma(M.mr[l], o[l], m) : f.mul(M.mr[0], o[0]);
        y[H] = m;
    }
}

// Shared-memory bytes: one stage of the inputs (u; CG: r, dinv, p), two work
// fields (r and s derivatives), the mbarrier and the reduction scratch.
template <int N, bool CG>
__host__ __device__ constexpr int ax64_in_bytes() {
    constexpr int NPT = (N + 1) * (N + 1) * (N + 1);
    return ((CG ? 3 : 1) * NPT * 8 + 15) / 16 * 16;
}
template <int N, bool CG>
__host__ __device__ constexpr int ax64_smem_bytes() {
    constexpr int NPT = (N + 1) * (N + 1) * (N + 1);
    return ax64_in_bytes<N, CG>() + ((2 * NPT * 8 + 15) / 16 * 16) + 2 * 8 + 16 * 8;
}

struct Ax64Args {
    int64_t E;
    int use_tma;       // 1: bulk-copy staging; 0: plain cooperative loads
    double h1, h2;     // Helmholtz coefficients
    const int *guard;  // if set, the kernel runs only when *guard == guard_value
    int guard_value;
};

// Modes: plain / HELM: w = A_L u (or h1 A_L u + h2 B u); CG: p <- dinv r +
// beta p (written back; dinv == nullptr: p <- r + beta p), w = A_L p (or the
// Helmholtz form), and sum_l p_l w_l reduced over the grid into alpha =
// rho / pw (per-CTA partials; the last CTA sums them in a fixed order).
//
// Staging: the inputs (read along lines of all three directions) go through
// one shared-memory buffer, refilled with the next element's slabs by bulk
// copies as soon as pass 2 has consumed them; G (and B), read once per point
// in a column pass, come straight from global memory (each warp reads 32
// consecutive doubles per factor and k).  The footprint stays small (12 KB
// at N = 7, 20 KB in the CG form), so many CTAs are resident and the FP64
// pipe stays fed across the barriers between passes.  Lines are read from
// the unpadded slabs: the bank conflicts of the r-lines cost a few dozen
// shared-memory cycles per pass against thousands of FP64 cycles.
template <int N, bool HELM, bool CG>
__global__ void __launch_bounds__(ax64_threads<N>())
    ax64_kernel(const double *__restrict__ u, double *__restrict__ w, const double *__restrict__ G,
                const double *__restrict__ Bm, const Eo64<N + 1> K, const Ax64Args args, const CgFuse<double> cg,
                int *__restrict__ err) {
    constexpr int N1 = N + 1, NL = N1 * N1, NPT = NL * N1;
    constexpr int INB = ax64_in_bytes<N, CG>();
    constexpr int NIN = CG ? 3 : 1;
    constexpr int T = ax64_threads<N>();
    extern __shared__ __align__(128) unsigned char smem[];
    if (CG && cg.scal->done) return;                            // uniform: the solve has converged
    if (args.guard && *args.guard != args.guard_value) return;  // uniform: not this phase
    double *sin = reinterpret_cast<double *>(smem);        // inputs (CG: r, dinv, p -> new p)
    double *R = reinterpret_cast<double *>(smem + INB);    // u_r -> v_r -> D^T v_r
    double *Sf = R + NPT;                                   // u_s -> v_s -> D^T v_s
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + INB + (2 * NPT * 8 + 15) / 16 * 16);
    double *sred = reinterpret_cast<double *>(bar + 2);
    double *su = sin + (CG ? 2 * NPT : 0);  // the operand of the contractions
    const int tid = threadIdx.x;
    const bool act = tid < NL;
    // column pass: thread = (i, j); r pass: (j, k); s pass: (i, k)
    const int ta = tid % N1, tb = tid / N1;
    const int rln = N1 * tid;          // (0, j, k), step 1
    const int sln = ta + NL * tb;      // (i, 0, k), step N1

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t E = args.E, stride = gridDim.x;
    const uint32_t ub = NPT * 8;
    const bool jac = CG && cg.dinv != nullptr;
    auto issue_in = [&](int64_t e) {
        unsigned char *st = smem;
        mbar_arrive_expect_tx(&bar[0], (jac ? NIN : (CG ? 2 : 1)) * ub);
        if (CG) {
            bulk_g2s(st, cg.r + e * NPT, ub, &bar[0]);
            if (jac) bulk_g2s(st + ub, cg.dinv + e * NPT, ub, &bar[0]);
            bulk_g2s(st + 2 * ub, cg.p + e * NPT, ub, &bar[0]);
        } else {
            bulk_g2s(st, u + e * NPT, ub, &bar[0]);
        }
    };
    if (args.use_tma && tid == 0 && (int64_t)blockIdx.x < E) issue_in(blockIdx.x);

    const double beta = CG ? cg.scal->beta : 0.0;
    const F64Ops f{K.one, K.mone, K.mzero};
    double pw_acc = 0.0;
    int it = 0;
    bool ok = true;
    for (int64_t e = blockIdx.x; e < E; e += stride, ++it) {
        const int64_t en = e + stride;
        if (args.use_tma) {
            const bool mine = mbar_wait_bounded(&bar[0], it & 1, err, kDevTimeoutTma);
            ok = __syncthreads_and(mine);
            if (!ok) break;
        } else {
            __syncthreads();  // the previous element's readers of the buffer are done
            for (int q = tid; q < NPT; q += T) {
                if (CG) {
                    sin[q] = cg.r[e * NPT + q];
                    if (jac) sin[NPT + q] = cg.dinv[e * NPT + q];
                    sin[2 * NPT + q] = cg.p[e * NPT + q];
                } else {
                    sin[q] = u[e * NPT + q];
                }
            }
            __syncthreads();
        }
        const double *ge = G + e * 6 * NPT;

        // 1. column pass: the operand (CG: the new search direction, written
        //    over the old one) and D along t
        double ru[N1], ut[N1];
        if (act) {
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                const int q = tid + NL * k;
                double x;
                if (CG) {
                    x = fma(beta, sin[2 * NPT + q], jac ? f.mul(sin[NPT + q], sin[q]) : sin[q]);
                    cg.p[e * NPT + q] = x;
                    su[q] = x;
                } else {
                    x = su[q];
                }
                ru[k] = x;
            }
            eo_line<N1>(ru, ut, K.f, f);
        }
        // the CG form wrote the new search direction into the buffer; the
        // plain form wrote nothing (the barrier before pass 1 already covers
        // the previous element's readers of R and Sf)
        if (CG) __syncthreads();
        // 2. D along r and along s
        if (act) {
            double x[N1], y[N1];
#pragma unroll
            for (int l = 0; l < N1; ++l) x[l] = su[rln + l];
            eo_line<N1>(x, y, K.f, f);
#pragma unroll
            for (int l = 0; l < N1; ++l) R[rln + l] = y[l];
#pragma unroll
            for (int l = 0; l < N1; ++l) x[l] = su[sln + N1 * l];
            eo_line<N1>(x, y, K.f, f);
#pragma unroll
            for (int l = 0; l < N1; ++l) Sf[sln + N1 * l] = y[l];
        }
        __syncthreads();  // the inputs are consumed: fetch the next element's
        if (args.use_tma && tid == 0 && en < E) {
            fence_proxy_async_smem();
            issue_in(en);
        }
        // 3. column pass: v = G (u_r, u_s, u_t); D^T along t
        double wt[N1], bq[N1];
        if (act) {
            double vt[N1];
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                const int q = tid + NL * k;
                const double ur = R[q], us = Sf[q], uu = ut[k];
                const double g0 = __ldg(ge + q), g1 = __ldg(ge + NPT + q), g2 = __ldg(ge + 2 * NPT + q);
                const double g3 = __ldg(ge + 3 * NPT + q), g4 = __ldg(ge + 4 * NPT + q);
                const double g5 = __ldg(ge + 5 * NPT + q);
                R[q] = fma(g4, uu, fma(g3, us, f.mul(g0, ur)));
                Sf[q] = fma(g5, uu, fma(g1, us, f.mul(g3, ur)));
                vt[k] = fma(g2, uu, fma(g5, us, f.mul(g4, ur)));
                if (HELM) bq[k] = __ldg(Bm + e * NPT + q);
            }
            eo_line<N1>(vt, wt, K.bk, f);
        }
        __syncthreads();
        // 4. D^T along r and along s, in place
        if (act) {
            double x[N1], y[N1];
#pragma unroll
            for (int l = 0; l < N1; ++l) x[l] = R[rln + l];
            eo_line<N1>(x, y, K.bk, f);
#pragma unroll
            for (int l = 0; l < N1; ++l) R[rln + l] = y[l];
#pragma unroll
            for (int l = 0; l < N1; ++l) x[l] = Sf[sln + N1 * l];
            eo_line<N1>(x, y, K.bk, f);
#pragma unroll
            for (int l = 0; l < N1; ++l) Sf[sln + N1 * l] = y[l];
        }
        __syncthreads();
        // 5. column pass: w = D^T v_r + D^T v_s + D^T v_t
        if (act) {
            double *we = w + e * NPT;
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                const int q = tid + NL * k;
                double acc = f.add(f.add(R[q], Sf[q]), wt[k]);
                if (HELM) acc = fma(args.h1, acc, f.mul(f.mul(args.h2, bq[k]), ru[k]));
                we[q] = acc;
                if (CG) pw_acc = fma(ru[k], acc, pw_acc);
            }
        }
        // the barrier after pass 1 of the next element protects R and Sf
    }
    if (!ok && args.use_tma && tid == 0) {
        // a wait gave up: drain the copies this CTA still has in flight (bounded)
        const int64_t e = blockIdx.x + (int64_t)it * stride;
        if (e < E) mbar_wait_bounded(&bar[0], it & 1, err, kDevTimeoutTma);
    }
    if (CG) {
        // grid reduction of p.w: per-CTA partials; the last CTA to arrive sums
        // them with all its threads in a fixed order
        __shared__ int s_last;
        const int lane = tid & 31, wid = tid >> 5;
        constexpr int NW = T / 32;
        double v = pw_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) sred[wid] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NW; ++q) t += sred[q];
            cg.partial[blockIdx.x] = t;
            __threadfence();
            s_last = atomicAdd(&cg.scal->cnt[3], 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double t = 0.0;
            for (int q = tid; q < (int)gridDim.x; q += T) t += __ldcg(cg.partial + q);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) sred[wid] = t;  // thread 0 read sred before the barrier above
            __syncthreads();
            if (tid == 0) {
                double pw = 0.0;
                for (int q = 0; q < NW; ++q) pw += sred[q];
                cg.scal->pw = pw;
                cg.scal->alpha = cg.scal->rho / pw;
                cg.scal->cnt[3] = 0u;
            }
        }
    }
}

// ---------------------------------------------------------------- host

// Even/odd coefficients of M (row-major (N+1)^2): see the file header.
template <int N1>
static void eo_coefs(const double *M, EoMat<N1> &out) {
    constexpr int H = N1 / 2, m = N1 / 2;
    for (int i = 0; i < H; ++i)
        for (int l = 0; l < H; ++l) {
            out.a[i * H + l] = 0.5 * (M[i * N1 + l] + M[i * N1 + (N1 - 1 - l)]);
            out.b[i * H + l] = 0.5 * (M[i * N1 + l] - M[i * N1 + (N1 - 1 - l)]);
        }
    for (int i = 0; i <= H; ++i) {
        out.c[i] = (N1 % 2 && i < H) ? M[i * N1 + m] : 0.0;
        out.mr[i] = (N1 % 2 && i < H) ? M[m * N1 + i] : 0.0;
    }
}

template <int N, bool HELM, bool CG>
static int launch_ax64_n(const sem_mesh *m, const double *u, double *w, double h1, double h2, const CgFuse<double> &cg,
                         const int *guard, int gval, cudaStream_t st) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    constexpr int threads = ax64_threads<N>();
    Eo64<N1> K;
    double Dt[N1 * N1];
    for (int i = 0; i < N1; ++i)
        for (int l = 0; l < N1; ++l) Dt[i * N1 + l] = m->D.d[l * N1 + i];
    eo_coefs<N1>(m->D.d, K.f);
    eo_coefs<N1>(Dt, K.bk);
    K.one = 1.0;
    K.mone = -1.0;
    K.mzero = -0.0;
    auto kern = ax64_kernel<N, HELM, CG>;
    int dev_max = 0;
    SEM_CUDA_CHECK(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    const AxTune tune = g_ax_tune[0][HELM][CG][0][N];
    const int smem = ax64_smem_bytes<N, CG>();
    if (smem > dev_max) return fail(SEM_ERR_UNSUPPORTED, "element does not fit in shared memory");
    SEM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    if (tune.per_sm_cap > 0 && per_sm > tune.per_sm_cap) per_sm = tune.per_sm_cap;
    int64_t grid = (int64_t)m->num_sms * per_sm;
    if (grid > kAxMaxGrid) grid = kAxMaxGrid;
    if (grid > m->E) grid = m->E;
    Ax64Args a;
    a.E = m->E;
    a.h1 = h1;
    a.h2 = h2;
    a.guard = guard;
    a.guard_value = gval;
    uintptr_t al = 0;
    if (CG)
        al |= reinterpret_cast<uintptr_t>(cg.r) | reinterpret_cast<uintptr_t>(cg.dinv) | reinterpret_cast<uintptr_t>(cg.p);
    else
        al |= reinterpret_cast<uintptr_t>(u);
    a.use_tma = ((NPT * 8) % 16 == 0) && (al % 16 == 0);
    kern<<<(int)grid, threads, smem, st>>>(u, w, m->G, m->B, K, a, cg, m->d_err);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

template <bool HELM, bool CG>
static int dispatch_ax64(const sem_mesh *m, const double *u, double *w, double h1, double h2, const CgFuse<double> &cg,
                         const int *guard, int gval, cudaStream_t st) {
    switch (m->N) {
#define SEM_AX64_CASE(n) \
    case n: return launch_ax64_n<n, HELM, CG>(m, u, w, h1, h2, cg, guard, gval, st);
        SEM_AX64_CASE(1) SEM_AX64_CASE(2) SEM_AX64_CASE(3) SEM_AX64_CASE(4) SEM_AX64_CASE(5)
        SEM_AX64_CASE(6) SEM_AX64_CASE(7) SEM_AX64_CASE(8) SEM_AX64_CASE(9) SEM_AX64_CASE(10) SEM_AX64_CASE(11)
#undef SEM_AX64_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "order N not built");
    }
}

int ax_launch_f64(const sem_mesh *m, const double *u, double *w, double h1, double h2, cudaStream_t st,
                  const int *guard, int gval) {
    const CgFuse<double> none{};
    if (h2 != 0.0 || h1 != 1.0) return dispatch_ax64<true, false>(m, u, w, h1, h2, none, guard, gval, st);
    return dispatch_ax64<false, false>(m, u, w, 1.0, 0.0, none, guard, gval, st);
}

int ax_cg_launch_f64(const sem_mesh *m, const CgFuse<double> &cg, double *w, double h1, double h2, cudaStream_t st) {
    if (h2 != 0.0 || h1 != 1.0) return dispatch_ax64<true, true>(m, nullptr, w, h1, h2, cg, nullptr, 0, st);
    return dispatch_ax64<false, true>(m, nullptr, w, 1.0, 0.0, cg, nullptr, 0, st);
}

}  // namespace sem
