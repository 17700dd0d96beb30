// sem_pcg.cu -- Jacobi-preconditioned conjugate gradients on the assembled
// SEM system, with fused vector updates and deterministic reductions.
//
// Paper section 3.1: a preconditioned Krylov method solves Ax = b each time
// step; the operator is applied matrix-free and followed by the gather-
// scatter.  The iteration is the Hestenes-Stiefel CG with a Jacobi (inverse
// assembled diagonal) preconditioner:
//   r = b - A x0; z = P r; p = z; rho = <r,z>
//   loop: w = A p; alpha = rho/<p,w>; x += alpha p; r -= alpha w;
//         stop if ||r|| <= tol ||b||; z = P r; rho' = <r,z>; p = z + (rho'/rho) p
// with <a,b> = sum_l a_l b_l / mult_l the unique-node product.
//
// GB300 design: per iteration four stream-ordered kernels -- the persistent
// TMA operator kernel, the gather-scatter, a fused p.w reduction, and one
// fused update kernel (x, r, z, both dot products, beta, convergence flag);
// the p update is fused into the next iteration's reduction kernel.  All
// scalars stay on the device; the host reads a convergence flag every
// `check_every` iterations, and kernels launched after convergence return at
// once.  Reductions are two-level (block partials, summed in block order by
// the last block), so results are run-to-run deterministic.

#include <chrono>
#include <cmath>
#include <vector>

#include "sem_common.cuh"

namespace sem {

constexpr int kPThreads = 256;
constexpr int kPBlocks = 1184;  // 152 SMs x 8 blocks: fixed so the reduction order is fixed

struct PcgScal {
    double bb, rr, rho, pw, alpha, beta, tol2, rr0;
    int iter, done, status, max_iter;
    unsigned cnt[4];
};

struct PcgWork {
    double *r, *p, *w;
    double *partial;  // [4][kPBlocks]
    PcgScal *scal;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-reduce NV values, publish block partials, and let the last block to
// arrive sum all partials in block order.  Returns true on thread 0 of the
// last block, with the totals in `tot`.
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double *partial, unsigned *counter, double (&tot)[NV]) {
    __shared__ double sh[NV][kPThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = wsum(v[q]);
        if (lane == 0) sh[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = 0.0;
            for (int k = 0; k < kPThreads / 32; ++k) t += sh[q][k];
            partial[q * kPBlocks + blockIdx.x] = t;
        }
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = 0.0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) t += partial[q * kPBlocks + k];
        t = wsum(t);
        __syncthreads();
        if (lane == 0) sh[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return false;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = 0.0;
        for (int k = 0; k < kPThreads / 32; ++k) t += sh[q][k];
        tot[q] = t;
    }
    *counter = 0u;
    return true;
}

// r = b - Ax0 (or b), z = dinv r, p = z; bb, rr, rho.
__global__ void __launch_bounds__(kPThreads)
    pcg_init_kernel(const double *__restrict__ b, const double *__restrict__ ax0, const double *__restrict__ dinv,
                    const double *__restrict__ minv, int64_t n, PcgWork W, double tol, int rel, int max_iter) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double bl = b[l];
        const double r = ax0 ? bl - ax0[l] : bl;
        const double z = dinv[l] * r;
        W.r[l] = r;
        W.p[l] = z;
        const double mi = minv[l];
        v[0] = fma(bl * bl, mi, v[0]);
        v[1] = fma(r * r, mi, v[1]);
        v[2] = fma(r * z, mi, v[2]);
    }
    double t[3];
    if (grid_reduce<3>(v, W.partial, &W.scal->cnt[0], t)) {
        PcgScal *s = W.scal;
        s->bb = t[0];
        s->rr = t[1];
        s->rr0 = t[1];
        s->rho = t[2];
        s->tol2 = rel ? tol * tol * t[0] : tol * tol;
        s->iter = 0;
        s->max_iter = max_iter;
        s->beta = 0.0;
        if (!isfinite(t[0]) || !isfinite(t[1])) {
            s->done = 1;
            s->status = SEM_ERR_NAN;
        } else if (t[1] <= s->tol2) {
            s->done = 1;
            s->status = SEM_OK;
        } else {
            s->done = 0;
            s->status = SEM_ERR_NOT_CONVERGED;
        }
    }
}

// pw = <p, w>, alpha = rho / pw.
__global__ void __launch_bounds__(kPThreads)
    pcg_pw_kernel(const double *__restrict__ minv, int64_t n, PcgWork W) {
    if (W.scal->done) return;
    double v[1] = {0.0};
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        v[0] = fma(W.p[l] * W.w[l], minv[l], v[0]);
    double t[1];
    if (grid_reduce<1>(v, W.partial + kPBlocks, &W.scal->cnt[1], t)) {
        W.scal->pw = t[0];
        W.scal->alpha = W.scal->rho / t[0];
    }
}

// x += alpha p; r -= alpha w; z = dinv r; rr = <r,r>; rz = <r,z>;
// last block: beta = rz/rho, rho = rz, iteration count and convergence flag.
__global__ void __launch_bounds__(kPThreads)
    pcg_update_kernel(double *__restrict__ x, const double *__restrict__ dinv, const double *__restrict__ minv,
                      int64_t n, PcgWork W) {
    if (W.scal->done) return;
    const double alpha = W.scal->alpha;
    double v[2] = {0.0, 0.0};
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double p = W.p[l];
        x[l] = fma(alpha, p, x[l]);
        const double r = fma(-alpha, W.w[l], W.r[l]);
        W.r[l] = r;
        const double mi = minv[l];
        v[0] = fma(r * r, mi, v[0]);
        v[1] = fma(r * (dinv[l] * r), mi, v[1]);
    }
    double t[2];
    if (grid_reduce<2>(v, W.partial + 2 * kPBlocks, &W.scal->cnt[2], t)) {
        PcgScal *s = W.scal;
        s->rr = t[0];
        s->beta = t[1] / s->rho;
        s->rho = t[1];
        s->iter += 1;
        if (!isfinite(t[0])) {
            s->done = 1;
            s->status = SEM_ERR_NAN;
        } else if (t[0] <= s->tol2) {
            s->done = 1;
            s->status = SEM_OK;
        } else if (s->iter >= s->max_iter) {
            s->done = 1;
            s->status = SEM_ERR_NOT_CONVERGED;
        }
    }
}

// p = dinv r + beta p.
__global__ void __launch_bounds__(kPThreads)
    pcg_p_kernel(const double *__restrict__ dinv, int64_t n, PcgWork W) {
    if (W.scal->done) return;
    const double beta = W.scal->beta;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        W.p[l] = fma(beta, W.p[l], dinv[l] * W.r[l]);
}

static size_t pcg_scratch(const sem_mesh *m) {
    return align_up(sizeof(double) * m->nloc) * 3 + align_up(sizeof(double) * 4 * kPBlocks) +
           align_up(sizeof(PcgScal));
}

static PcgWork carve(const sem_mesh *m, void *scratch) {
    char *p = static_cast<char *>(scratch);
    PcgWork W;
    const size_t vb = align_up(sizeof(double) * m->nloc);
    W.r = reinterpret_cast<double *>(p);
    W.p = reinterpret_cast<double *>(p + vb);
    W.w = reinterpret_cast<double *>(p + 2 * vb);
    W.partial = reinterpret_cast<double *>(p + 3 * vb);
    W.scal = reinterpret_cast<PcgScal *>(p + 3 * vb + align_up(sizeof(double) * 4 * kPBlocks));
    return W;
}

// Event pairs recorded on the launching stream around selected kernels;
// harvested after each host synchronisation.
struct EvTimer {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    int used = 0;
    double total_ms = 0.0;
    int init(bool enable, int pairs) {
        on = enable;
        if (!on) return SEM_OK;
        ev.resize(2 * pairs);
        for (auto &e : ev) SEM_CUDA_CHECK(cudaEventCreate(&e));
        return SEM_OK;
    }
    void start(cudaStream_t st) {
        if (on && used < (int)ev.size() / 2) cudaEventRecord(ev[2 * used], st);
    }
    void stop(cudaStream_t st) {
        if (on && used < (int)ev.size() / 2) cudaEventRecord(ev[2 * used + 1], st), ++used;
    }
    void harvest() {
        for (int q = 0; q < used; ++q) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]) == cudaSuccess) total_ms += ms;
        }
        used = 0;
    }
    ~EvTimer() {
        for (auto &e : ev) cudaEventDestroy(e);
    }
};

struct SolveCtx {
    EvTimer tax, tgs;
    int launches = 0, ax_launches = 0;
};

static int apply_assembled_timed(const sem_mesh *m, const double *x, double *y, double h1, double h2,
                                 cudaStream_t st, SolveCtx &c) {
    c.tax.start(st);
    int s = ax_launch_f64(m, x, y, h1, h2, st);
    c.tax.stop(st);
    if (s != SEM_OK) return s;
    c.tgs.start(st);
    s = gs_launch(m, y, SEM_F64, kGsSumMask, st);
    c.tgs.stop(st);
    c.launches += 2;
    c.ax_launches += 1;
    return s;
}

static int pcg_f64(const sem_mesh *m, const double *b, double *x, const sem_pcg_opts *o, sem_pcg_stats *stats,
                   void *scratch, cudaStream_t st) {
    PcgWork W = carve(m, scratch);
    const int64_t n = m->nloc;
    const int check = o->check_every > 0 ? o->check_every : 16;
    SolveCtx c;
    int s0 = c.tax.init(o->profile != 0, check + 1);
    if (s0 == SEM_OK) s0 = c.tgs.init(o->profile != 0, check + 1);
    if (s0 != SEM_OK) return s0;
    SEM_CUDA_CHECK(cudaMemsetAsync(W.scal, 0, sizeof(PcgScal), st));
    const double *ax0 = nullptr;
    if (o->use_initial_guess) {
        int s = apply_assembled_timed(m, x, W.w, o->h1, o->h2, st, c);
        if (s != SEM_OK) return s;
        ax0 = W.w;
    } else {
        SEM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    }
    pcg_init_kernel<<<kPBlocks, kPThreads, 0, st>>>(b, ax0, m->dinv, m->minv, n, W, o->tol,
                                                    o->tol_is_relative, o->max_iter);
    SEM_CUDA_CHECK(cudaGetLastError());
    c.launches += 1;
    PcgScal h{};
    int launched = 0;
    while (true) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(&h, W.scal, sizeof(h), cudaMemcpyDeviceToHost, st));
        SEM_CUDA_CHECK(cudaStreamSynchronize(st));
        c.tax.harvest();
        c.tgs.harvest();
        if (h.done || launched >= o->max_iter) break;
        for (int q = 0; q < check && launched < o->max_iter; ++q, ++launched) {
            int s = apply_assembled_timed(m, W.p, W.w, o->h1, o->h2, st, c);
            if (s != SEM_OK) return s;
            pcg_pw_kernel<<<kPBlocks, kPThreads, 0, st>>>(m->minv, n, W);
            pcg_update_kernel<<<kPBlocks, kPThreads, 0, st>>>(x, m->dinv, m->minv, n, W);
            pcg_p_kernel<<<kPBlocks, kPThreads, 0, st>>>(m->dinv, n, W);
            SEM_CUDA_CHECK(cudaGetLastError());
            c.launches += 3;
        }
    }
    int derr = 0;
    SEM_CUDA_CHECK(cudaMemcpyAsync(&derr, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    stats->iters = h.iter;
    stats->outer_iters = 0;
    stats->bnorm = std::sqrt(h.bb);
    stats->abs_res = std::sqrt(h.rr);
    stats->rel_res = h.bb > 0 ? std::sqrt(h.rr / h.bb) : stats->abs_res;
    stats->ax_ms = c.tax.total_ms;
    stats->gs_ms = c.tgs.total_ms;
    stats->ax_launches = c.ax_launches;
    stats->kernel_launches = c.launches;
    int status = h.done ? h.status : SEM_ERR_NOT_CONVERGED;
    if (derr != 0) status = SEM_ERR_TIMEOUT;
    return status;
}

static int check_opts(const sem_pcg_opts *o) {
    if (o->precision != SEM_PCG_F64) return fail(SEM_ERR_UNSUPPORTED, "precision mode not built");
    if (!(o->tol > 0.0) || o->max_iter < 1) return fail(SEM_ERR_INVALID_ARG, "tol must be > 0, max_iter >= 1");
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

size_t sem_pcg_scratch_bytes(const sem_mesh *m, const sem_pcg_opts *o) {
    if (!m) return 0;
    (void)o;
    return pcg_scratch(m);
}

size_t sem_pcg_host_scratch_bytes(const sem_mesh *m, const sem_pcg_opts *o) {
    if (!m) return 0;
    return sem_pcg_scratch_bytes(m, o) + 2 * align_up(sizeof(double) * m->nloc);
}

int sem_pcg_solve(const sem_mesh *m, const double *b, double *x, const sem_pcg_opts *o, sem_pcg_stats *stats,
                  void *scratch, size_t scratch_bytes, void *stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!m || !b || !x || !o || !stats || !scratch) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    *stats = sem_pcg_stats{};
    int s = check_opts(o);
    if (s != SEM_OK) return s;
    if (scratch_bytes < sem_pcg_scratch_bytes(m, o) || reinterpret_cast<uintptr_t>(scratch) % kAlign)
        return fail(SEM_ERR_WORKSPACE, "scratch smaller than sem_pcg_scratch_bytes or not 256-byte aligned");
    s = pcg_f64(m, b, x, o, stats, scratch, as_stream(stream));
    stats->status = s;
    stats->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (s != SEM_OK && s != SEM_ERR_CUDA) set_error(sem_status_string(s));
    return s;
}

int sem_pcg_solve_host(const sem_mesh *m, const double *hb, double *hx, const sem_pcg_opts *o,
                       sem_pcg_stats *stats, void *scratch, size_t scratch_bytes, void *stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!m || !hb || !hx || !o || !stats || !scratch) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    *stats = sem_pcg_stats{};
    int s = check_opts(o);
    if (s != SEM_OK) return s;
    if (scratch_bytes < sem_pcg_host_scratch_bytes(m, o) || reinterpret_cast<uintptr_t>(scratch) % kAlign)
        return fail(SEM_ERR_WORKSPACE, "scratch smaller than sem_pcg_host_scratch_bytes or not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    const size_t vb = align_up(sizeof(double) * m->nloc);
    char *p = static_cast<char *>(scratch);
    double *db = reinterpret_cast<double *>(p);
    double *dx = reinterpret_cast<double *>(p + vb);
    void *inner = p + 2 * vb;
    SEM_CUDA_CHECK(cudaMemcpyAsync(db, hb, sizeof(double) * m->nloc, cudaMemcpyHostToDevice, st));
    if (o->use_initial_guess)
        SEM_CUDA_CHECK(cudaMemcpyAsync(dx, hx, sizeof(double) * m->nloc, cudaMemcpyHostToDevice, st));
    s = pcg_f64(m, db, dx, o, stats, inner, st);
    if (s == SEM_OK || s == SEM_ERR_NOT_CONVERGED) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(hx, dx, sizeof(double) * m->nloc, cudaMemcpyDeviceToHost, st));
        SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    }
    stats->status = s;
    stats->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (s != SEM_OK && s != SEM_ERR_CUDA) set_error(sem_status_string(s));
    return s;
}

}  // extern "C"
