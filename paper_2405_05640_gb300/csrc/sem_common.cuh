// sem_common.cuh -- internal declarations shared by the library's CUDA
// translation units: the mesh object, error plumbing, and the inline-PTX
// helpers for the bulk-copy (TMA) + mbarrier pipeline.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/sem.h"
#include <nvtx3/nvToolsExt.h>

namespace sem {

constexpr int kMaxN = SEM_MAX_ORDER;
constexpr int kMaxN1 = kMaxN + 1;
constexpr int kAlign = 256;

// Derivative matrix passed by value to kernels (copied to shared memory).
struct DMat {
    double d[kMaxN1 * kMaxN1];  // row-major D[i][j] = l_j'(xi_i)
};
struct DMatF {
    float d[kMaxN1 * kMaxN1];
};

// Device-resident scalars of one CG solve (read by the fused kernels).
struct PcgScal {
    double bb, rr, rho, pw, alpha, beta, tol2, rr0;
    double scale;       // mixed precision: 1/||r|| of the outer residual (inner init)
    double scale_prev;  // mixed precision: the previous 1/||r||
    double rho_prev;    // rho of the iteration before the last update
    double prev_rr;     // batched solver: FP64 residual of the previous refinement
    int iter, done, status, max_iter;
    int phase;          // batched solver: kBt* state of this solve
    int rounds;         // batched solver: rounds executed by this solve
    int inner_done;     // batched solver: inner iterations of the inner solves already restarted
    unsigned cnt[4];  // arrival counters of the grid reductions (cnt[3]: fused operator)
};

// Inner relative tolerance of a refinement round: delta, or with theta > 0
// the larger theta * target / ||r|| (target^2 = the outer tol2, ||r||^2 =
// the outer rr of `so`), capped at 0.5 so that every round iterates: a round
// that starts near the outer target stops once the target is within reach.
__device__ __forceinline__ double inner_delta(const PcgScal *__restrict__ so, double delta, double theta) {
    if (theta > 0.0 && so->rr > 0.0) {
        const double a = fmin(0.5, theta * sqrt(so->tol2 / so->rr));
        if (a > delta) return a;
    }
    return delta;
}

// Arguments of the fused CG operator: p <- dinv r + beta p, w = A_L p,
// alpha = rho / sum_l p_l w_l (grid reduction over per-CTA partials).
template <typename T>
struct CgFuse {
    const T *r;
    const T *dinv;
    T *p;
    PcgScal *scal;
    double *partial;  // >= gridDim.x doubles
};

// Error word values written by kernels into mesh->d_err.
enum DevErr : int { kDevOk = 0, kDevTimeoutTma = 1, kDevTimeoutFlag = 2 };

}  // namespace sem

struct sem_mesh {
    int N, n1, npt;
    int64_t E, nloc, nglob;
    int nel[3], periodic[3], faces;
    int geom_flags;
    // host copies of the 1-D GLL data
    double xi[sem::kMaxN1], rho[sem::kMaxN1];
    sem::DMat D;
    sem::DMatF Df;
    // device arrays (inside the caller's workspace)
    double *verts;       // [E][8][3]
    double *G;           // [E][6][npt]
    float *G32;          // [E][6][npt] FP32 geometric factors, or nullptr
    float2 *G2;          // [E][6][npt] FP32-pair (hi, lo) geometric factors, or nullptr
    float *aff32;        // [E][4] affine elements: (a, b, c, 0), G_rr = rho_i rho_j rho_k a, ... or nullptr
    void *G16;           // [E][6][npt] BF16 geometric factors for the FP32 operator, or nullptr
    double *B;           // [E][npt]
    double *mult;        // [nloc]
    double *minv;        // [nloc] 1/mult
    double *dinv;        // [nloc] inverse assembled Jacobi diagonal (0 on Dirichlet)
    float *dinv32;       // [nloc] same in FP32 (SEM_GEOM_F32)
    float *minv32;       // [nloc]
    double *rx;          // [E][9][npt] dr_a/dx_m (a-major) or nullptr
    int *gs_idx;         // group copies, bucketed by group size (see sem_mesh.cu)
    int *d_err;          // device error word
    int64_t ngroups, nmasked, nentries;
    int64_t gs_n[4], gs_nm[4], gs_start[4];  // bucket b (2^b copies): groups, masked groups, first int
    size_t ws_bytes;
    int device;
    int num_sms;
};

namespace sem {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);

#define SEM_CUDA_CHECK(call)                                  \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return sem::cuda_fail(_e, #call); \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- shared PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion counted in bytes on
// `bar`.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar`, giving up after `limit_ns` of global time.
// On give-up writes `code` into *err (first writer wins) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  int code, uint64_t limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

// Grid-wide barrier of a kernel whose CTAs are all resident (cooperative
// launch): each CTA adds one arrival to *bar and thread 0 waits until it
// reaches `target`, giving up after `limit_ns` of global time or at once when
// another CTA has given up (*err != 0); a give-up writes kDevTimeoutFlag into
// *err (first writer wins).  Returns false (on every thread of the CTA) when
// the wait gave up.
__device__ __forceinline__ bool grid_barrier_bounded(unsigned *bar, unsigned target, int *err,
                                                     uint64_t limit_ns = 1000000000ull) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int good = 1;
        uint64_t t0 = 0;
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (*reinterpret_cast<volatile int *>(err) != 0) {
                good = 0;
                break;
            }
            const uint64_t t = global_timer_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > limit_ns) {
                atomicCAS(err, 0, (int)kDevTimeoutFlag);
                good = 0;
                break;
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// A named range on a profiler's CPU timeline (NVTX; a no-op when no tool is
// attached): solves, refinement rounds, Krylov cycles, NS phases, network
// passes.  ncu can select the kernels of a range (--nvtx --nvtx-include).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------- host helpers
int ax_launch_f64(const sem_mesh *m, const double *u, double *w, double h1, double h2,
                  cudaStream_t st, const int *guard = nullptr, int gval = 0);
int ax_launch_f32(const sem_mesh *m, const float *u, float *w, cudaStream_t st, const int *guard = nullptr,
                  int gval = 0);
// FP64 operator in FP32-pair arithmetic (sem_ax_pair.cu); needs m->G2.
int ax_launch_pair(const sem_mesh *m, const double *u, double *w, cudaStream_t st);
// Fused CG operator (see CgFuse); w receives the local (unassembled) A_L p.
int ax_cg_launch_f64(const sem_mesh *m, const CgFuse<double> &cg, double *w, double h1, double h2,
                     cudaStream_t st);
int ax_cg_launch_f32(const sem_mesh *m, const CgFuse<float> &cg, float *w, cudaStream_t st);
// Fused CG form of the FP32-pair FP64 operator (sem_ax_pair.cu).
int ax_cg_launch_pair(const sem_mesh *m, const CgFuse<double> &cg, double *w, cudaStream_t st);
constexpr int kAxMaxGrid = 152 * 32;  // upper bound of the operator grid (partials of the fused kernel)
int gs_launch(const sem_mesh *m, void *u, int dtype, int mode, cudaStream_t st, const int *guard = nullptr,
              int gval = 0);

// Operator launch shape (see sem_ax.cu); g_ax_tune[dtype][helm][cg][affine][N].
struct AxTune {
    int nst;         // pipeline stages, 0 = default (2)
    int per_sm_cap;  // resident CTAs per SM cap, 0 = occupancy limit
    int epc;         // FP32 operator: elements per CTA (1, 2, 4), 0 = default (1)
};
extern AxTune g_ax_tune[2][2][2][2][kMaxN1];
int jacobi_diag_launch(const sem_mesh *m, double *diag, cudaStream_t st);

// Box topology for the arithmetic (index-free) gather-scatter of the CG loop:
// element e = ex + nel0 (ey + nel1 ez), local point i + N1 (j + N1 k).
struct BoxTopo {
    int N, N1, NPT;
    int nel[3], per[3];
    int faces;  // Dirichlet face bits (2a: low face of axis a, 2a+1: high face)
    int64_t E;
};
inline BoxTopo box_topo(const sem_mesh *m) {
    BoxTopo b;
    b.N = m->N;
    b.N1 = m->n1;
    b.NPT = m->npt;
    for (int a = 0; a < 3; ++a) {
        b.nel[a] = m->nel[a];
        b.per[a] = m->periodic[a];
    }
    b.faces = m->faces;
    b.E = m->E;
    return b;
}
// Sum the copies shared across y- and z-element faces (edges included), in
// place, no mask: the first two passes of the axis-by-axis gather-scatter;
// the x pass and the Dirichlet mask are applied by the CG update that reads
// the field (sem_pcg.cu).
int gs_yz_launch(const sem_mesh *m, void *u, int dtype, cudaStream_t st, const int *guard = nullptr,
                 int gval = 0);

// Dealiased advection (sem_dealias.cu): fine-point factors w_q det J dr_a/dx_m
// ([E][9][M^3], M = 3(N+1)/2 Gauss points per direction) and the local weak
// form W_c = int phi_i (u . grad) u_c.  N <= 9.
size_t dealias_metric_bytes(const sem_mesh *m);
int dealias_metric_launch(const sem_mesh *m, double *W, cudaStream_t st);
int advect_weak_launch(const sem_mesh *m, const double *W, const double *const u[3], double *const out[3],
                       cudaStream_t st);

// Host GLL data of order N (sem_mesh.cu): nodes, weights, D_ij = l_j'(xi_i)
// (row-major, (N+1)^2).
void gll_host(int N, double *xi, double *rho);
void deriv_host(int N, const double *x, double *D);

// Hybrid Schwarz preconditioner (sem_schwarz.cu): z = M r in FP32; done
// (optional device flag): set -> the kernels return at once; coop: the
// coarse CG as one cooperative kernel (grid barriers), else as separate
// launches (for graphs whose branches run concurrently).
int schwarz_apply_f32(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      const int *done, cudaStream_t st, bool coop = true);
// The (fine) mesh a Schwarz object was built on.
const sem_mesh *schwarz_mesh(const sem_schwarz *sw);
// Intermediate (order-M) level of the Schwarz multigrid (sem_schwarz.cu):
// z += w P_M S_M P_M^T r; work: schwarz_mid_work_bytes; done: guard flag.
size_t schwarz_mid_work_bytes(const sem_schwarz *mid);
int schwarz_mid_check(const sem_schwarz *sw, const sem_schwarz *mid);
int schwarz_mid_apply_add(const sem_schwarz *sw, const sem_schwarz *mid, double w, const float *r, float *z,
                          void *work, const int *done, cudaStream_t st);

// Flexible GMRES inner solve (sem_gmres.cu): one cycle of at most `restart`
// iterations on A d = r64 * so->scale from d = 0, preconditioned by the
// hybrid Schwarz object sw (plus the intermediate level mid), or by the FP32
// Jacobi diagonal when sw is null; stops when the Arnoldi residual estimate
// has fallen by inner_delta(so, delta, theta); writes d.  work:
// gmres_work_bytes(m, restart).
constexpr int kGmMaxRestart = 128;
struct GmresArgs {
    int restart, max_iter, check;
    double delta, theta;
    const sem_schwarz *sw;
    int coarse_iters;
    double coarse_tol;
    const sem_schwarz *mid;
    double mid_w;
    void *mid_work;
};
struct GmresResult {
    int iters, converged, status, launches, ax_launches;
};
size_t gmres_work_bytes(const sem_mesh *m, int restart);
int gmres_cycle(const sem_mesh *m, const double *r64, const PcgScal *so, float *d, const GmresArgs &a, void *work,
                cudaStream_t st, GmresResult *out);

// gather-scatter modes
constexpr int kGsSum = 0;       // sum copies
constexpr int kGsSumMask = 1;   // sum copies, then zero Dirichlet nodes
constexpr int kGsMaskOnly = 2;  // zero Dirichlet nodes only

}  // namespace sem
