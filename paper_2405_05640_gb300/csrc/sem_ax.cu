// sem_ax.cu -- matrix-free local stiffness / Helmholtz operator.
//
// Paper section 3.1: every operator except the gather-scatter is applied
// element by element ("matrix-free"), with identical cost per element; the
// basis is the order-N Lagrange basis on the GLL points.  Per element e:
//   u_r = D u (along r), u_s, u_t likewise;
//   (v_r, v_s, v_t) = G (u_r, u_s, u_t), G the symmetric 3x3 geometric factors;
//   w = D^T v_r + D^T v_s + D^T v_t  [+ Helmholtz: w = h1 w + h2 B u].
//
// GB300 design: a persistent grid (a few CTAs per SM), each CTA owning one
// element at a time.  The element's u slab and its six geometric-factor slabs
// (contiguous in the [E][6][npt] layout) are brought into shared memory by
// 1-D bulk copies on the TMA engine, completing on an mbarrier; a ring of
// stages lets the copies of the next element overlap the contraction of the
// current one.  Threads are laid out (i, j) over the (N+1)^2 columns and loop
// over k, holding their u column and the t-direction results in registers.
// Every mbarrier wait is bounded in time; on time-out the kernel records
// kDevTimeoutTma in the mesh error word and all CTAs leave the loop.
// This kernel serves the FP32 operator (plain, fused CG, affine and BF16-
// factor forms); the FP64 operator has its own kernel (sem_ax64.cu).

#include <cuda_bf16.h>

#include <type_traits>

#include "sem_common.cuh"

namespace sem {

// Slabs per stage: the input field (u; or r, dinv, p in the fused CG mode),
// the six geometric factors (AFF: the element's 4 affine scalars instead),
// and B (Helmholtz, FP64).
// A CTA works on EPC consecutive elements at a time (the "block shape"; 1
// by default, 2 or 4 where (N+1)^2 threads leave a warp half empty, chosen by
// the autotuner).  Their slabs are contiguous in every array, so each bulk
// copy simply covers EPC elements.
template <int N, typename T, bool HELM, bool CG, bool AFF, bool G16 = false, int EPC = 1>
__host__ __device__ constexpr int ax_stage_bytes() {
    constexpr int NPT = (N + 1) * (N + 1) * (N + 1);
    constexpr int gsize = AFF ? 16 : 6 * NPT * (G16 ? 2 : (int)sizeof(T));
    return (EPC * (NPT * (CG ? 3 : 1) * (int)sizeof(T) + gsize + (HELM ? NPT * 8 : 0)) + 15) / 16 * 16;
}

template <int N, typename T, bool HELM, bool CG, bool AFF, bool G16 = false, int EPC = 1>
__host__ __device__ constexpr int ax_smem_bytes(int nst) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    return nst * ax_stage_bytes<N, T, HELM, CG, AFF, G16, EPC>() + 2 * EPC * NPT * (int)sizeof(T) +
           ((N1 * N1 * (int)sizeof(T) + 15) / 16 * 16) + 4 * 8 + 32 * 8;
}

template <int N, int EPC = 1>
__host__ __device__ constexpr int ax_threads() {
    return (EPC * (N + 1) * (N + 1) + 31) / 32 * 32;
}

// N1 consecutive shared-memory values into registers: 16-byte vector loads
// when a line is a whole number of 16-byte vectors (lines start 16-byte
// aligned: every slab is), else scalar loads.
template <typename T, int N1>
__device__ __forceinline__ void smem_line(const T *a, T (&v)[N1]) {
    if constexpr ((N1 * sizeof(T)) % 16 == 0) {
        constexpr int V = 16 / sizeof(T);
#pragma unroll
        for (int c = 0; c < N1; c += V) {
            if constexpr (sizeof(T) == 4) {
                const float4 q = *reinterpret_cast<const float4 *>(a + c);
                v[c] = q.x;
                v[c + 1] = q.y;
                v[c + 2] = q.z;
                v[c + 3] = q.w;
            } else {
                const double2 q = *reinterpret_cast<const double2 *>(a + c);
                v[c] = q.x;
                v[c + 1] = q.y;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < N1; ++c) v[c] = a[c];
    }
}

struct AxArgs {
    int64_t E;
    int nst;      // pipeline stages (1..3)
    int use_tma;  // 1: bulk-copy staging; 0: plain cooperative loads
    double h1, h2;
    const int *guard;  // if set, the kernel runs only when *guard == guard_value
    int guard_value;
    float rho[kMaxN1];  // GLL weights (affine mode: G = rho_i rho_j rho_k (a, b, c)_e)
};

// Launch shape of the operator per (precision, Helmholtz, fused CG, N):
// pipeline stages, a cap on resident CTAs per SM (0 = occupancy limit) and
// the elements per CTA (FP32).  Defaults: 2 stages, no cap, 1 element;
// sem_autotune_operator measures and sets them.
AxTune g_ax_tune[2][2][2][2][kMaxN1] = {};

static AxTune tune_for(int dt, bool helm, bool cg, bool aff, int N) {
    AxTune t = g_ax_tune[dt][helm][cg][aff][N];
    if (t.nst <= 0) t.nst = 2;
    if (t.epc <= 0) t.epc = 1;
    return t;
}

// One element per CTA at a time (persistent grid).  Modes:
//   plain / HELM: w = A_L u  (or h1 A_L u + h2 B u);
//   CG: p <- dinv r + beta p (written back), w = A_L p (or Helmholtz), and
//       sum_l p_l w_l reduced over the grid into alpha = rho / pw;
//   AFF (axis-aligned box elements): G is diagonal and factorises, G_rr =
//       rho_i rho_j rho_k a_e etc.; G points at the [E][4] scalars (a, b, c, 0);
//   G16 (FP32 operator): the six factors are stored in BF16 ([E][6][npt],
//       12 bytes per point) and widened to FP32 in shared memory reads.
template <int N, typename T, bool HELM, bool CG, bool AFF, typename DM, bool G16 = false, int EPC = 1>
__global__ void __launch_bounds__(ax_threads<N, EPC>())
    ax_kernel(const T *__restrict__ u, T *__restrict__ w, const void *__restrict__ Gv,
              const double *__restrict__ Bm, const DM Dm, const AxArgs args, const CgFuse<T> cg,
              int *__restrict__ err) {
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    constexpr int SB = ax_stage_bytes<N, T, HELM, CG, AFF, G16, EPC>();
    using GT = typename std::conditional<G16, __nv_bfloat16, T>::type;
    const GT *__restrict__ G = static_cast<const GT *>(Gv);
    // Vector r-line loads and D_kl as constant-bank operands cut the shared-
    // memory instructions; measured faster for the FP32 plain and affine
    // forms, slower for the general fused CG form and FP64, which keep
    // scalar loads and D from shared memory.
    constexpr bool kLineLoads = sizeof(T) == 4 && (AFF || !CG);
    constexpr int NIN = CG ? 3 : 1;  // input slabs
    extern __shared__ __align__(128) unsigned char smem[];
    if (CG && cg.scal->done) return;  // uniform: the solve has converged or paused
    if (args.guard && *args.guard != args.guard_value) return;  // uniform: not this phase
    const int nst = args.nst;
    T *svr0 = reinterpret_cast<T *>(smem + nst * SB);
    T *svs0 = svr0 + EPC * NPT;
    T *sD = svs0 + EPC * NPT;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + nst * SB + 2 * EPC * NPT * sizeof(T) +
                                                 ((N1 * N1 * sizeof(T) + 15) / 16 * 16));
    double *sred = reinterpret_cast<double *>(bar + 4);  // 32 doubles: per-warp partials
    const int tid = threadIdx.x;
    const int slot = tid / (N1 * N1);             // element of the CTA's group
    const bool active = slot < EPC;
    const int lt = tid - slot * N1 * N1;
    const int i = lt % N1, j = lt / N1;
    T *svr = svr0 + (active ? slot : 0) * NPT;
    T *svs = svs0 + (active ? slot : 0) * NPT;

    for (int q = tid; q < N1 * N1; q += blockDim.x) sD[q] = (T)Dm.d[q];
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    T rDi[N1], rDj[N1], rDti[N1], rDtj[N1];
#pragma unroll
    for (int l = 0; l < N1; ++l) {
        rDi[l] = active ? sD[i * N1 + l] : T(0);
        rDj[l] = active ? sD[j * N1 + l] : T(0);
        rDti[l] = active ? sD[l * N1 + i] : T(0);
        rDtj[l] = active ? sD[l * N1 + j] : T(0);
    }
    const T beta = CG ? (T)cg.scal->beta : T(0);
    T rij = T(0);  // rho_i rho_j (affine mode); unrolled selects keep the parameters in the constant bank
    if (AFF && active) {
        T ri = T(0), rj = T(0);
#pragma unroll
        for (int q = 0; q < N1; ++q) {
            ri = q == i ? (T)args.rho[q] : ri;
            rj = q == j ? (T)args.rho[q] : rj;
        }
        rij = ri * rj;
    }

    const int64_t E = args.E;
    const int64_t C = (E + EPC - 1) / EPC;  // element groups
    const int64_t stride = gridDim.x;
    const uint32_t ubytes = NPT * sizeof(T), gbytes = AFF ? 16 : 6 * NPT * sizeof(GT);
    const uint32_t bbytes = HELM ? NPT * sizeof(double) : 0;
    // stage layout: each input slab holds EPC elements, then EPC G slabs, then EPC B slabs
    const uint32_t inoff = EPC * ubytes, goff = NIN * EPC * ubytes, boff = goff + EPC * gbytes;

    // CG with dinv == nullptr: the preconditioned residual z comes in r and
    // p <- z + beta p (general preconditioner); the dinv slab is not loaded
    const bool jac = CG && cg.dinv != nullptr;
    auto stage_ptr = [&](int s) { return smem + s * SB; };
    auto group_size = [&](int64_t c) { return (int)((E - c * EPC) < EPC ? (E - c * EPC) : EPC); };
    auto issue = [&](int64_t c, int s) {
        unsigned char *st = stage_ptr(s);
        const int64_t e = c * EPC;
        const uint32_t nv = (uint32_t)group_size(c);
        mbar_arrive_expect_tx(&bar[s], nv * (NIN * ubytes + gbytes + bbytes - (CG && !jac ? ubytes : 0)));
        if (CG) {
            bulk_g2s(st, cg.r + e * NPT, nv * ubytes, &bar[s]);
            if (jac) bulk_g2s(st + inoff, cg.dinv + e * NPT, nv * ubytes, &bar[s]);
            bulk_g2s(st + 2 * inoff, cg.p + e * NPT, nv * ubytes, &bar[s]);
        } else {
            bulk_g2s(st, u + e * NPT, nv * ubytes, &bar[s]);
        }
        bulk_g2s(st + goff, AFF ? G + e * 4 : G + e * 6 * NPT, nv * gbytes, &bar[s]);
        if (HELM) bulk_g2s(st + boff, Bm + e * NPT, nv * bbytes, &bar[s]);
    };

    if (args.use_tma && tid == 0) {
        for (int s = 0; s < nst; ++s) {
            const int64_t c = blockIdx.x + s * stride;
            if (c < C) issue(c, s);
        }
    }

    T pw_acc = T(0);
    int it = 0;
    bool ok = true;
    for (int64_t c = blockIdx.x; c < C; c += stride, ++it) {
        const int s = it % nst;
        const uint32_t parity = (it / nst) & 1;
        unsigned char *st = stage_ptr(s);
        const int nv = group_size(c);
        const bool mine_el = active && slot < nv;  // this thread's element exists
        const int64_t e = c * EPC + (active ? slot : 0);
        if (args.use_tma) {
            bool mine = mbar_wait_bounded(&bar[s], parity, err, kDevTimeoutTma);
            ok = __syncthreads_and(mine);
            if (!ok) break;
        } else {
            const int64_t e0 = c * EPC;
            T *dst = reinterpret_cast<T *>(st);
            if (CG) {
                for (int q = tid; q < nv * NPT; q += blockDim.x) {
                    dst[q] = cg.r[e0 * NPT + q];
                    if (jac) dst[EPC * NPT + q] = cg.dinv[e0 * NPT + q];
                    dst[2 * EPC * NPT + q] = cg.p[e0 * NPT + q];
                }
            } else {
                for (int q = tid; q < nv * NPT; q += blockDim.x) dst[q] = u[e0 * NPT + q];
            }
            const GT *gs = AFF ? G + e0 * 4 : G + e0 * 6 * NPT;
            GT *gd = reinterpret_cast<GT *>(st + goff);
            for (int q = tid; q < nv * (AFF ? 4 : 6 * NPT); q += blockDim.x) gd[q] = gs[q];
            if (HELM) {
                double *db = reinterpret_cast<double *>(st + boff);
                for (int q = tid; q < nv * NPT; q += blockDim.x) db[q] = Bm[e0 * NPT + q];
            }
            __syncthreads();
        }
        // the operand: u, or the updated search direction p (CG); this
        // thread's element's slabs
        const int sl = active ? slot : 0;
        T *su = reinterpret_cast<T *>(st) + (CG ? 2 * EPC * NPT : 0) + sl * NPT;
        const GT *sg = reinterpret_cast<const GT *>(st + goff) + sl * (AFF ? 4 : 6 * NPT);
        const double *sb = reinterpret_cast<const double *>(st + boff) + sl * NPT;
        if (CG) {
            const T *sr = reinterpret_cast<const T *>(st) + sl * NPT;
            const T *sdi = sr + EPC * NPT;
            T *pe = cg.p + e * NPT;
            if (mine_el) {
#pragma unroll
                for (int k = 0; k < N1; ++k) {
                    const int q = i + N1 * (j + N1 * k);
                    const T pn = fma(beta, su[q], jac ? sdi[q] * sr[q] : sr[q]);
                    su[q] = pn;
                    pe[q] = pn;
                }
            }
            __syncthreads();
        }

        T ru[N1], rvt[N1];
        if (mine_el) {
#pragma unroll
            for (int k = 0; k < N1; ++k) ru[k] = su[i + N1 * (j + N1 * k)];
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                T ur = T(0), us = T(0), ut = T(0);
                if constexpr (kLineLoads) {
                    T line[N1];  // the r-line (., j, k): vector loads; D_kl from the constant bank
                    smem_line<T, N1>(su + N1 * (j + N1 * k), line);
#pragma unroll
                    for (int l = 0; l < N1; ++l) {
                        ur = fma(rDi[l], line[l], ur);
                        us = fma(rDj[l], su[i + N1 * (l + N1 * k)], us);
                        ut = fma((T)Dm.d[k * N1 + l], ru[l], ut);
                    }
                } else {
#pragma unroll
                    for (int l = 0; l < N1; ++l) {
                        ur = fma(rDi[l], su[l + N1 * (j + N1 * k)], ur);
                        us = fma(rDj[l], su[i + N1 * (l + N1 * k)], us);
                        ut = fma(sD[k * N1 + l], ru[l], ut);
                    }
                }
                const int p = i + N1 * (j + N1 * k);
                if (AFF) {
                    const T wq = rij * (T)args.rho[k];
                    svr[p] = (wq * (T)sg[0]) * ur;
                    svs[p] = (wq * (T)sg[1]) * us;
                    rvt[k] = (wq * (T)sg[2]) * ut;
                } else {
                    const T g0 = (T)sg[p], g1 = (T)sg[NPT + p], g2 = (T)sg[2 * NPT + p];
                    const T g3 = (T)sg[3 * NPT + p], g4 = (T)sg[4 * NPT + p], g5 = (T)sg[5 * NPT + p];
                    svr[p] = g0 * ur + g3 * us + g4 * ut;
                    svs[p] = g3 * ur + g1 * us + g5 * ut;
                    rvt[k] = g4 * ur + g5 * us + g2 * ut;
                }
            }
        }
        __syncthreads();
        if (mine_el) {
            T *we = w + e * NPT;
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                // three independent accumulation chains (one per direction)
                T ar = T(0), as = T(0), at = T(0);
                if constexpr (kLineLoads) {
                    T line[N1];
                    smem_line<T, N1>(svr + N1 * (j + N1 * k), line);
#pragma unroll
                    for (int l = 0; l < N1; ++l) {
                        ar = fma(rDti[l], line[l], ar);
                        as = fma(rDtj[l], svs[i + N1 * (l + N1 * k)], as);
                        at = fma((T)Dm.d[l * N1 + k], rvt[l], at);
                    }
                } else {
#pragma unroll
                    for (int l = 0; l < N1; ++l) {
                        ar = fma(rDti[l], svr[l + N1 * (j + N1 * k)], ar);
                        as = fma(rDtj[l], svs[i + N1 * (l + N1 * k)], as);
                        at = fma(sD[l * N1 + k], rvt[l], at);
                    }
                }
                T acc = (ar + as) + at;
                const int p = i + N1 * (j + N1 * k);
                if (HELM) acc = (T)(args.h1 * (double)acc + args.h2 * sb[p] * (double)ru[k]);
                we[p] = acc;
                if (CG) pw_acc = fma(ru[k], acc, pw_acc);
            }
        }
        __syncthreads();  // stage s and svr/svs free again
        if (args.use_tma && tid == 0) {
            const int64_t cn = c + nst * stride;
            if (cn < C) {
                fence_proxy_async_smem();
                issue(cn, s);
            }
        }
    }
    if (!ok && args.use_tma && tid == 0) {
        // a wait gave up: drain the copies this CTA still has in flight (bounded)
        for (int s = 0; s < nst; ++s) {
            const int itn = it + ((s - it % nst) + nst) % nst;
            const int64_t cn = blockIdx.x + (int64_t)itn * stride;
            if (cn < C) mbar_wait_bounded(&bar[s], (itn / nst) & 1, err, kDevTimeoutTma);
        }
    }
    if (CG) {
        // grid reduction of p.w: per-CTA partials; the last CTA to arrive sums
        // them with all its threads (thread t takes partials t, t + blockDim,
        // ... in order, then a fixed shuffle tree and the warps in order: the
        // same order on every run)
        __shared__ int s_last;
        const int lane = tid & 31, wid = tid >> 5, nw = (int)(blockDim.x >> 5);
        double v = (double)pw_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sred[wid] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < nw; ++q) t += sred[q];
            cg.partial[blockIdx.x] = t;
            __threadfence();
            s_last = atomicAdd(&cg.scal->cnt[3], 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double t = 0.0;
            for (int q = tid; q < (int)gridDim.x; q += blockDim.x) t += __ldcg(cg.partial + q);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) sred[wid] = t;  // thread 0 read sred before the barrier above
            __syncthreads();
            if (tid == 0) {
                double pw = 0.0;
                for (int q = 0; q < nw; ++q) pw += sred[q];
                cg.scal->pw = pw;
                cg.scal->alpha = cg.scal->rho / pw;
                cg.scal->cnt[3] = 0u;
            }
        }
    }
}

// ---------------------------------------------------------------- launch

template <int N, typename T, bool HELM, bool CG, bool AFF, typename DM, bool G16, int EPC>
static int launch_ax_epc(const sem_mesh *m, const T *u, T *w, const void *G, double h1, double h2, const DM &Dm,
                         const CgFuse<T> &cg, const int *guard, int gval, cudaStream_t st, const AxTune &tune) {
    constexpr int NPT = (N + 1) * (N + 1) * (N + 1);
    constexpr int threads = ax_threads<N, EPC>();
    auto kern = ax_kernel<N, T, HELM, CG, AFF, DM, G16, EPC>;
    int dev_max = 0;
    SEM_CUDA_CHECK(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    int nst = tune.nst < 1 ? 1 : (tune.nst > 3 ? 3 : tune.nst);
    while (nst > 1 && ax_smem_bytes<N, T, HELM, CG, AFF, G16, EPC>(nst) > dev_max) --nst;
    const int smem = ax_smem_bytes<N, T, HELM, CG, AFF, G16, EPC>(nst);
    if (smem > dev_max) return fail(SEM_ERR_UNSUPPORTED, "element group does not fit in shared memory");
    SEM_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    if (tune.per_sm_cap > 0 && per_sm > tune.per_sm_cap) per_sm = tune.per_sm_cap;
    const int64_t groups = (m->E + EPC - 1) / EPC;
    int64_t grid = (int64_t)m->num_sms * per_sm;
    if (grid > kAxMaxGrid) grid = kAxMaxGrid;
    if (grid > groups) grid = groups;
    AxArgs a;
    a.E = m->E;
    a.nst = nst;
    a.h1 = h1;
    a.h2 = h2;
    a.guard = guard;
    a.guard_value = gval;
    for (int q = 0; q < kMaxN1; ++q) a.rho[q] = q <= m->N ? (float)m->rho[q] : 0.f;
    uintptr_t al = reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(m->B);
    if (CG)
        al |= reinterpret_cast<uintptr_t>(cg.r) | reinterpret_cast<uintptr_t>(cg.dinv) |
              reinterpret_cast<uintptr_t>(cg.p);
    else
        al |= reinterpret_cast<uintptr_t>(u);
    a.use_tma = ((NPT * sizeof(T)) % 16 == 0) && ((NPT * sizeof(double)) % 16 == 0) && (al % 16 == 0);
    kern<<<(int)grid, threads, smem, st>>>(u, w, G, m->B, Dm, a, cg, m->d_err);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

// Element groups of 2 and 4 are built for the FP32 operator of the general
// and the BF16-factor forms (the solvers' inner loops, incl. the batched
// one) at the orders whose (N+1)^2 lines leave warps partly empty.
template <int N, typename T, bool AFF>
constexpr bool ax_has_groups() {
    return sizeof(T) == 4 && !AFF && N >= 2 && N <= 9 && ((N + 1) * (N + 1)) % 32 != 0;
}

template <int N, typename T, bool HELM, bool CG, bool AFF, typename DM, bool G16>
static int launch_ax_n(const sem_mesh *m, const T *u, T *w, const void *G, double h1, double h2,
                       const DM &Dm, const CgFuse<T> &cg, const int *guard, int gval, cudaStream_t st) {
    const AxTune tune = tune_for(sizeof(T) == 8 ? 0 : 1, HELM, CG, AFF, N);
    if constexpr (ax_has_groups<N, T, AFF>() && !HELM) {
        if (tune.epc == 2)
            return launch_ax_epc<N, T, HELM, CG, AFF, DM, G16, 2>(m, u, w, G, h1, h2, Dm, cg, guard, gval, st, tune);
        if (tune.epc == 4)
            return launch_ax_epc<N, T, HELM, CG, AFF, DM, G16, 4>(m, u, w, G, h1, h2, Dm, cg, guard, gval, st, tune);
    }
    return launch_ax_epc<N, T, HELM, CG, AFF, DM, G16, 1>(m, u, w, G, h1, h2, Dm, cg, guard, gval, st, tune);
}

template <typename T, bool HELM, bool CG, typename DM, bool AFF = false, bool G16 = false>
static int dispatch_ax(const sem_mesh *m, const T *u, T *w, const void *G, double h1, double h2,
                       const DM &Dm, const CgFuse<T> &cg, cudaStream_t st, const int *guard = nullptr,
                       int gval = 0) {
    switch (m->N) {
#define SEM_AX_CASE(n) \
    case n: return launch_ax_n<n, T, HELM, CG, AFF, DM, G16>(m, u, w, G, h1, h2, Dm, cg, guard, gval, st);
        SEM_AX_CASE(1) SEM_AX_CASE(2) SEM_AX_CASE(3) SEM_AX_CASE(4) SEM_AX_CASE(5)
        SEM_AX_CASE(6) SEM_AX_CASE(7) SEM_AX_CASE(8) SEM_AX_CASE(9) SEM_AX_CASE(10) SEM_AX_CASE(11)
#undef SEM_AX_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "order N not built");
    }
}

int ax_launch_f32(const sem_mesh *m, const float *u, float *w, cudaStream_t st, const int *guard, int gval) {
    if (!m->G32) return fail(SEM_ERR_INVALID_ARG, "mesh built without SEM_GEOM_F32");
    const CgFuse<float> none{};
    if (m->aff32)
        return dispatch_ax<float, false, false, DMatF, true>(m, u, w, m->aff32, 1.0, 0.0, m->Df, none, st, guard,
                                                             gval);
    if (m->G16)
        return dispatch_ax<float, false, false, DMatF, false, true>(m, u, w, m->G16, 1.0, 0.0, m->Df, none, st,
                                                                    guard, gval);
    return dispatch_ax<float, false, false>(m, u, w, m->G32, 1.0, 0.0, m->Df, none, st, guard, gval);
}

int ax_cg_launch_f32(const sem_mesh *m, const CgFuse<float> &cg, float *w, cudaStream_t st) {
    if (!m->G32) return fail(SEM_ERR_INVALID_ARG, "mesh built without SEM_GEOM_F32");
    if (m->aff32)
        return dispatch_ax<float, false, true, DMatF, true>(m, nullptr, w, m->aff32, 1.0, 0.0, m->Df, cg, st);
    if (m->G16)
        return dispatch_ax<float, false, true, DMatF, false, true>(m, nullptr, w, m->G16, 1.0, 0.0, m->Df, cg, st);
    return dispatch_ax<float, false, true>(m, nullptr, w, m->G32, 1.0, 0.0, m->Df, cg, st);
}

// ---------------------------------------------------------------- Jacobi diagonal

// diag(A_L) at (i,j,k): sum_l D_li^2 G_rr(ljk) + sum_l D_lj^2 G_ss(ilk)
//   + sum_l D_lk^2 G_tt(ijl) + 2 D_ii D_jj G_rs + 2 D_ii D_kk G_rt + 2 D_jj D_kk G_st.
__global__ void jacobi_diag_kernel(const double *__restrict__ G, int64_t E, int N, DMat Dm,
                                   double *__restrict__ diag) {
    const int n1 = N + 1;
    const int64_t npt = (int64_t)n1 * n1 * n1;
    const int64_t nloc = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nloc;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int p = (int)(l - e * npt);
        const int i = p % n1, j = (p / n1) % n1, k = p / (n1 * n1);
        const double *Ge = G + e * 6 * npt;
        double s = 0.0;
        for (int q = 0; q < n1; ++q) {
            const double a = Dm.d[q * n1 + i], b = Dm.d[q * n1 + j], c = Dm.d[q * n1 + k];
            s += a * a * Ge[q + n1 * (j + n1 * k)];
            s += b * b * Ge[npt + i + n1 * (q + n1 * k)];
            s += c * c * Ge[2 * npt + i + n1 * (j + n1 * q)];
        }
        const double di = Dm.d[i * n1 + i], dj = Dm.d[j * n1 + j], dk = Dm.d[k * n1 + k];
        s += 2.0 * di * dj * Ge[3 * npt + p] + 2.0 * di * dk * Ge[4 * npt + p] +
             2.0 * dj * dk * Ge[5 * npt + p];
        diag[l] = s;
    }
}

int jacobi_diag_launch(const sem_mesh *m, double *diag, cudaStream_t st) {
    int64_t g = (m->nloc + 255) / 256;
    if (g > (int64_t)m->num_sms * 64) g = (int64_t)m->num_sms * 64;
    jacobi_diag_kernel<<<(int)g, 256, 0, st>>>(m->G, m->E, m->N, m->D, diag);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

// ---------------------------------------------------------------- autotuner

// Time `reps` launches of the operator of mesh m (mode: plain or fused CG,
// FP32 or FP64) with the current table entry; returns ms per launch.
template <typename T, bool CG, typename DM>
static int time_operator(const sem_mesh *m, const T *G, const DM &Dm, T *bufs, PcgScal *scal, double *partial,
                         int reps, cudaStream_t st, float *ms) {
    const int64_t n = m->nloc;
    T *u = bufs, *w = bufs + n, *dinv = bufs + 2 * n, *pp = bufs + 3 * n;
    CgFuse<T> cg{u, dinv, pp, scal, partial};
    // the same dispatch as the solvers (FP32: the affine form on affine meshes)
    auto once = [&]() {
        if (sizeof(T) == 4)
            return CG ? ax_cg_launch_f32(m, reinterpret_cast<const CgFuse<float> &>(cg), reinterpret_cast<float *>(w), st)
                      : ax_launch_f32(m, reinterpret_cast<const float *>(u), reinterpret_cast<float *>(w), st);
        return CG ? ax_cg_launch_f64(m, reinterpret_cast<const CgFuse<double> &>(cg), reinterpret_cast<double *>(w),
                                     1.0, 0.0, st)
                  : ax_launch_f64(m, reinterpret_cast<const double *>(u), reinterpret_cast<double *>(w), 1.0, 0.0, st);
    };
    for (int q = 0; q < 2; ++q) {
        int s = once();
        if (s != SEM_OK) return s;
    }
    cudaEvent_t a, b;
    SEM_CUDA_CHECK(cudaEventCreate(&a));
    SEM_CUDA_CHECK(cudaEventCreate(&b));
    cudaEventRecord(a, st);
    int s = SEM_OK;
    for (int q = 0; q < reps && s == SEM_OK; ++q) s = once();
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != SEM_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
    *ms = t / reps;
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

size_t sem_autotune_scratch_bytes(const sem_mesh *m) {
    if (!m) return 0;
    return align_up(sizeof(double) * 4 * m->nloc) + align_up(sizeof(PcgScal)) + align_up(sizeof(double) * kAxMaxGrid);
}

int sem_autotune_operator(const sem_mesh *m, int dtype, int fused_cg, void *scratch, size_t bytes, void *stream,
                          sem_tune_result *out) {
    if (!m || !scratch || !out) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (dtype != SEM_F64 && dtype != SEM_F32) return fail(SEM_ERR_INVALID_ARG, "unknown dtype");
    if (dtype == SEM_F32 && !m->G32) return fail(SEM_ERR_INVALID_ARG, "mesh built without SEM_GEOM_F32");
    if (bytes < sem_autotune_scratch_bytes(m) || reinterpret_cast<uintptr_t>(scratch) % kAlign)
        return fail(SEM_ERR_WORKSPACE, "scratch smaller than sem_autotune_scratch_bytes or misaligned");
    cudaStream_t st = as_stream(stream);
    char *p = static_cast<char *>(scratch);
    SEM_CUDA_CHECK(cudaMemsetAsync(p, 0, sem_autotune_scratch_bytes(m), st));
    void *bufs = p;
    PcgScal *scal = reinterpret_cast<PcgScal *>(p + align_up(sizeof(double) * 4 * m->nloc));
    double *partial = reinterpret_cast<double *>(p + align_up(sizeof(double) * 4 * m->nloc) + align_up(sizeof(PcgScal)));
    const int dt = dtype == SEM_F64 ? 0 : 1, cg = fused_cg ? 1 : 0, N = m->N;
    AxTune &slot = g_ax_tune[dt][0][cg][dt == 1 && m->aff32 ? 1 : 0][N];
    const AxTune saved = slot;
    // the FP64 operator keeps one element per CTA and stages nothing across
    // elements: only its CTA cap is tuned; the FP32 one sweeps pipeline depth
    // x CTA cap x elements per CTA (groups where (N+1)^2 lines leave warps
    // partly empty; see ax_has_groups)
    const bool groups = dt == 1 && !m->aff32 && N >= 2 && N <= 9 && ((N + 1) * (N + 1)) % 32 != 0;
    const int stages[3] = {1, 2, 3}, caps[4] = {0, 1, 2, 4}, epcs[3] = {1, 2, 4};
    const int na = dt == 0 ? 1 : 3, ne = groups ? 3 : 1;
    float best = 1e30f;
    AxTune bt{2, 0, 1};
    out->configs = 0;
    for (int a = 0; a < na; ++a)
        for (int c = 0; c < 4; ++c)
            for (int g = 0; g < ne; ++g) {
                slot = AxTune{dt == 0 ? 2 : stages[a], caps[c], epcs[g]};
                float ms = 0.f;
                int s;
                if (dt == 1 && cg)
                    s = time_operator<float, true>(m, m->G32, m->Df, static_cast<float *>(bufs), scal, partial, 10, st,
                                                   &ms);
                else if (dt == 1)
                    s = time_operator<float, false>(m, m->G32, m->Df, static_cast<float *>(bufs), scal, partial, 10, st,
                                                    &ms);
                else if (cg)
                    s = time_operator<double, true>(m, m->G, m->D, static_cast<double *>(bufs), scal, partial, 5, st, &ms);
                else
                    s = time_operator<double, false>(m, m->G, m->D, static_cast<double *>(bufs), scal, partial, 5, st,
                                                     &ms);
                if (s != SEM_OK) {
                    slot = saved;
                    return s;
                }
                if (out->configs < SEM_TUNE_MAX_CONFIGS) {
                    out->stages[out->configs] = slot.nst;
                    out->caps[out->configs] = caps[c];
                    out->epcs[out->configs] = epcs[g];
                    out->ms[out->configs] = ms;
                }
                ++out->configs;
                if (ms < best) {
                    best = ms;
                    bt = slot;
                }
            }
    slot = bt;
    out->best_stages = bt.nst;
    out->best_cap = bt.per_sm_cap;
    out->best_epc = bt.epc;
    out->best_ms = best;
    return SEM_OK;
}

int sem_autotune_set(const sem_mesh *m, int dtype, int fused_cg, int stages, int per_sm_cap, int epc) {
    if (!m) return fail(SEM_ERR_INVALID_ARG, "NULL mesh");
    if (dtype != SEM_F64 && dtype != SEM_F32) return fail(SEM_ERR_INVALID_ARG, "unknown dtype");
    if (stages < 1 || stages > 3 || per_sm_cap < 0 || (epc != 1 && epc != 2 && epc != 4))
        return fail(SEM_ERR_INVALID_ARG, "stages 1..3, per_sm_cap >= 0, epc 1, 2 or 4");
    const int dt = dtype == SEM_F64 ? 0 : 1;
    g_ax_tune[dt][0][fused_cg ? 1 : 0][dt == 1 && m->aff32 ? 1 : 0][m->N] = AxTune{stages, per_sm_cap, epc};
    return SEM_OK;
}

int sem_autotune_reset(void) {
    for (auto &a : g_ax_tune)
        for (auto &b : a)
            for (auto &c : b)
                for (auto &d : c)
                    for (auto &f : d) f = AxTune{0, 0, 0};
    return SEM_OK;
}

}  // extern "C"


extern "C" {

int sem_ax(const sem_mesh *m, const void *u, void *w, int dtype, void *stream) {
    if (!m || !u || !w) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (u == w) return fail(SEM_ERR_INVALID_ARG, "u and w must not overlap");
    if (dtype == SEM_F64)
        return ax_launch_f64(m, static_cast<const double *>(u), static_cast<double *>(w), 1.0, 0.0,
                             as_stream(stream));
    if (dtype == SEM_F32)
        return ax_launch_f32(m, static_cast<const float *>(u), static_cast<float *>(w), as_stream(stream));
    if (dtype == SEM_F64_PAIR)
        return ax_launch_pair(m, static_cast<const double *>(u), static_cast<double *>(w), as_stream(stream));
    return fail(SEM_ERR_INVALID_ARG, "unknown dtype");
}

int sem_helmholtz(const sem_mesh *m, double h1, double h2, const double *u, double *w, void *stream) {
    if (!m || !u || !w) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (u == w) return fail(SEM_ERR_INVALID_ARG, "u and w must not overlap");
    return ax_launch_f64(m, u, w, h1, h2, as_stream(stream));
}

}  // extern "C"
