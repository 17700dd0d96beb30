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
// GB300 design: per iteration three stream-ordered kernels -- the persistent
// TMA operator kernel fused with the search-direction update p = z + beta p
// and the <p, A p> reduction (alpha); the y and z passes of the gather-
// scatter; and one line-wise update kernel (the x pass of the gather-scatter,
// the Dirichlet mask, x, r, z, both dot products, beta, convergence flag).  All
// scalars stay on the device; the host reads a convergence flag every
// `check_every` iterations, and kernels launched after convergence return at
// once.  Reductions are two-level (block partials, summed in block order by
// the last block), so results are run-to-run deterministic.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "sem_common.cuh"

namespace sem {

constexpr int kPThreads = 256;
constexpr int kPBlocks = 1184;  // 152 SMs x 8 blocks: fixed so the reduction order is fixed

// Vectors of one CG iteration space in precision T.
template <typename T>
struct PcgWork {
    T *r, *p, *w;
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

__device__ __forceinline__ void set_start_flags(PcgScal *s, double bb, double rr) {
    if (!isfinite(bb) || !isfinite(rr)) {
        s->done = 1;
        s->status = SEM_ERR_NAN;
    } else if (rr <= s->tol2) {
        s->done = 1;
        s->status = SEM_OK;
    } else {
        s->done = 0;
        s->status = SEM_ERR_NOT_CONVERGED;
    }
}

// Start of a CG solve in precision T: r = scale * (b - Ax0) (ax0 may be
// null), z = dinv r, p = z; bb = <b,b>, rr = <r,r>, rho = <r,z>.
// In the mixed solver b is the FP64 outer residual and `scale` = 1/||b||
// comes from the outer scalars (scale_src), so the inner system is O(1).
template <typename T, typename TB>
__device__ __forceinline__ bool pcg_init_body(const TB *__restrict__ b, const T *__restrict__ ax0,
                                              const T *__restrict__ dinv, const T *__restrict__ minv, int64_t n,
                                              PcgWork<T> W, const PcgScal *__restrict__ scale_src, double tol,
                                              int rel, int max_iter, double theta = 0.0);

template <typename T, typename TB>
__global__ void __launch_bounds__(kPThreads)
    pcg_init_kernel(const TB *__restrict__ b, const T *__restrict__ ax0, const T *__restrict__ dinv,
                    const T *__restrict__ minv, int64_t n, PcgWork<T> W, const PcgScal *__restrict__ scale_src,
                    double tol, int rel, int max_iter, double theta = 0.0) {
    pcg_init_body<T, TB>(b, ax0, dinv, minv, n, W, scale_src, tol, rel, max_iter, theta);
}

// Returns true on the thread that wrote the scalars.
template <typename T, typename TB>
__device__ __forceinline__ bool pcg_init_body(const TB *__restrict__ b, const T *__restrict__ ax0,
                                              const T *__restrict__ dinv, const T *__restrict__ minv, int64_t n,
                                              PcgWork<T> W, const PcgScal *__restrict__ scale_src, double tol,
                                              int rel, int max_iter, double theta) {
    const double sc = scale_src ? scale_src->scale : 1.0;
    if (scale_src) tol = inner_delta(scale_src, tol, theta);
    double v[3] = {0.0, 0.0, 0.0};
    T f[3] = {T(0), T(0), T(0)};  // per-thread partials in T (FP32: no FP64 pipe per element)
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const T bl = scale_src ? (T)((double)b[l] * sc) : (T)b[l];
        const T r = ax0 ? bl - ax0[l] : bl;
        const T z = dinv[l] * r;
        W.r[l] = r;
        W.p[l] = z;
        const T mi = minv[l];
        if (sizeof(T) == 8) {
            v[0] = fma((double)(bl * bl), (double)mi, v[0]);
            v[1] = fma((double)(r * r), (double)mi, v[1]);
            v[2] = fma((double)(r * z), (double)mi, v[2]);
        } else {
            f[0] = fmaf(bl * bl, mi, f[0]);
            f[1] = fmaf(r * r, mi, f[1]);
            f[2] = fmaf(r * z, mi, f[2]);
        }
    }
    if (sizeof(T) == 4)
        for (int q = 0; q < 3; ++q) v[q] = (double)f[q];
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
        set_start_flags(s, t[0], t[1]);
        return true;
    }
    return false;
}

// 16-byte vector of T (float4 / double2) as an array.
template <typename T>
struct V16 {
    static constexpr int n = 16 / sizeof(T);
    T a[16 / sizeof(T)];
};
template <typename T>
__device__ __forceinline__ V16<T> ld16(const T *p) {
    V16<T> v;
    if (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        reinterpret_cast<float4 &>(v) = q;
    } else {
        const double2 q = *reinterpret_cast<const double2 *>(p);
        reinterpret_cast<double2 &>(v) = q;
    }
    return v;
}
template <typename T>
__device__ __forceinline__ void st16(T *p, const V16<T> &v) {
    if (sizeof(T) == 4)
        *reinterpret_cast<float4 *>(p) = reinterpret_cast<const float4 &>(v);
    else
        *reinterpret_cast<double2 *>(p) = reinterpret_cast<const double2 &>(v);
}

// One point of the update: x += alpha p; r -= alpha w; rr and rz partials
// (per-thread in T for FP32, FP64 for FP64).
template <typename T>
__device__ __forceinline__ void update_point(T alpha, T p, T w, T mi, T di, T &x, T &r, double (&v)[2], T &f0,
                                             T &f1) {
    x = fma(alpha, p, x);
    r = fma(-alpha, w, r);
    if (sizeof(T) == 8) {
        v[0] = fma((double)(r * r), (double)mi, v[0]);
        v[1] = fma((double)(r * (di * r)), (double)mi, v[1]);
    } else {
        f0 = fma(r * r, mi, f0);
        f1 = fma(r * (di * r), mi, f1);
    }
}

static bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// N1 consecutive values of a line into registers (16-byte vectors when VEC).
template <typename T, int N1, bool VEC>
__device__ __forceinline__ void load_line(const T *__restrict__ a, T (&v)[N1]) {
    if (VEC) {
#pragma unroll
        for (int c = 0; c < N1; c += V16<T>::n) {
            const V16<T> q = ld16(a + c);
#pragma unroll
            for (int d = 0; d < V16<T>::n; ++d) v[c + d] = q.a[d];
        }
    } else {
#pragma unroll
        for (int c = 0; c < N1; ++c) v[c] = a[c];
    }
}
template <typename T, int N1, bool VEC>
__device__ __forceinline__ void store_line(T *__restrict__ a, const T (&v)[N1]) {
    if (VEC) {
#pragma unroll
        for (int c = 0; c < N1; c += V16<T>::n) {
            V16<T> q;
#pragma unroll
            for (int d = 0; d < V16<T>::n; ++d) q.a[d] = v[c + d];
            st16(a + c, q);
        }
    } else {
#pragma unroll
        for (int c = 0; c < N1; ++c) a[c] = v[c];
    }
}

// Shared / Dirichlet status of a face point along one axis: the point sits on
// the low (lo = true) or high face of element index e of nel.
__device__ __forceinline__ void face_status(int e, int nel, int per, bool lo, int dir_bit_lo, int dir_bit_hi,
                                           int faces, int &shared, bool &dirichlet) {
    if (lo) {
        shared = (e > 0 || per) ? 1 : 0;
        dirichlet = !per && e == 0 && (faces & dir_bit_lo);
    } else {
        shared = (e < nel - 1 || per) ? 1 : 0;
        dirichlet = !per && e == nel - 1 && (faces & dir_bit_hi);
    }
}

// CG update with the last gather-scatter pass folded in.  w holds A_L p after
// the y and z passes (gs_yz_launch); one thread per r-line (e, j, k):
//   w(e,0)  <- w(left, N) + w(e, 0)      if e has a left neighbour in x,
//   w(e,N)  <- w(e, N) + w(right, 0)     if it has a right one
// (the neighbour's thread forms the same sum from the same operands in the
// same order, so all copies stay bit-identical); w <- 0 on Dirichlet nodes;
// then x += alpha p, r -= alpha w and the <r,r>, <r,z> partials with the
// weight 1/mult computed from the point's position (a power of two, the same
// value as the mesh's stored 1/mult).
// WRITEW: the assembled, masked w is also written to wout (the flexible CG of
// a general preconditioner needs <z, A p> in the next iteration), and dinv is
// not read (the <r, D^-1 r> partial is then 0; the preconditioner's own
// kernel forms rho).  wout must not be W.w: the x pass of this launch reads
// W.w's raw line ends.
template <typename T, int N, bool VEC, bool WRITEW = false>
__global__ void __launch_bounds__(kPThreads)
    pcg_update_box_kernel(T *__restrict__ x, const T *__restrict__ dinv, BoxTopo B, PcgWork<T> W,
                          T *__restrict__ wout = nullptr) {
    if (W.scal->done) return;
    constexpr int N1 = N + 1, NL = N1 * N1, NPT = NL * N1;
    const T alpha = (T)W.scal->alpha;
    double v[2] = {0.0, 0.0};
    T f0 = T(0), f1 = T(0);
    const int nx = B.nel[0], ny = B.nel[1];
    const int64_t nlines = B.E * NL;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < nlines;
         L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = L / NL;
        const int jk = (int)(L - e * NL);
        const int j = jk % N1, k = jk / N1;
        const int ex = (int)(e % nx);
        const int64_t eyz = e / nx;
        const int ey = (int)(eyz % ny), ez = (int)(eyz / ny);
        const int64_t base = L * N1;
        T p[N1], w[N1], xv[N1], r[N1], di[N1];
        load_line<T, N1, VEC>(W.p + base, p);
        load_line<T, N1, VEC>(W.w + base, w);
        load_line<T, N1, VEC>(x + base, xv);
        load_line<T, N1, VEC>(W.r + base, r);
        if (WRITEW) {  // flexible CG: z comes from the preconditioner, <r, D^-1 r> is not used
#pragma unroll
            for (int i = 0; i < N1; ++i) di[i] = T(0);
        } else {
            load_line<T, N1, VEC>(dinv + base, di);
        }
        // y and z status of the whole line
        int sy = 0, sz = 0;
        bool dy = false, dz = false;
        if (j == 0 || j == N) face_status(ey, ny, B.per[1], j == 0, 4, 8, B.faces, sy, dy);
        if (k == 0 || k == N) face_status(ez, B.nel[2], B.per[2], k == 0, 16, 32, B.faces, sz, dz);
        // x pass at the two ends (neighbour values read before any change)
        int sx0 = 0, sxN = 0;
        bool dx0 = false, dxN = false;
        face_status(ex, nx, B.per[0], true, 1, 2, B.faces, sx0, dx0);
        face_status(ex, nx, B.per[0], false, 1, 2, B.faces, sxN, dxN);
        const T wl = sx0 ? W.w[(ex > 0 ? e - 1 : e + nx - 1) * NPT + (int64_t)jk * N1 + N] : T(0);
        const T wr = sxN ? W.w[(ex < nx - 1 ? e + 1 : e - (nx - 1)) * NPT + (int64_t)jk * N1] : T(0);
        const T w0 = w[0], wN = w[N];
        if (sx0) w[0] = wl + w0;
        if (sxN) w[N] = wN + wr;
        const bool dyz = dy || dz;
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int sx = i == 0 ? sx0 : (i == N ? sxN : 0);
            const bool dd = dyz || (i == 0 && dx0) || (i == N && dxN);
            const int sh = sx + sy + sz;
            const T mi = sh == 0 ? T(1) : (sh == 1 ? T(0.5) : (sh == 2 ? T(0.25) : T(0.125)));
            const T wt = dd ? T(0) : w[i];
            if (WRITEW) w[i] = wt;
            update_point(alpha, p[i], wt, mi, di[i], xv[i], r[i], v, f0, f1);
        }
        store_line<T, N1, VEC>(x + base, xv);
        store_line<T, N1, VEC>(W.r + base, r);
        if (WRITEW) store_line<T, N1, VEC>(wout + base, w);
    }
    if (sizeof(T) == 4) {
        v[0] = (double)f0;
        v[1] = (double)f1;
    }
    double t[2];
    if (grid_reduce<2>(v, W.partial + 2 * kPBlocks, &W.scal->cnt[2], t)) {
        PcgScal *s = W.scal;
        s->rr = t[0];
        s->beta = t[1] / s->rho;
        s->rho_prev = s->rho;
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

template <typename T, int N>
static int launch_update_box_n(const sem_mesh *m, T *x, const T *dinv, const PcgWork<T> &W, cudaStream_t st,
                               T *wout) {
    const bool writew = wout != nullptr;
    constexpr int N1 = N + 1;
    const BoxTopo B = box_topo(m);
    const bool vec = (N1 * sizeof(T)) % 16 == 0 && al16(x) && al16(dinv) && al16(W.p) && al16(W.w) && al16(W.r) &&
                     (!writew || al16(wout));
    auto kv = pcg_update_box_kernel<T, N, ((N1 * sizeof(T)) % 16 == 0)>;
    auto ks = pcg_update_box_kernel<T, N, false>;
    auto kvw = pcg_update_box_kernel<T, N, ((N1 * sizeof(T)) % 16 == 0), true>;
    auto ksw = pcg_update_box_kernel<T, N, false, true>;
    auto kern = writew ? (vec ? kvw : ksw) : (vec ? kv : ks);
    // one wave: every resident block takes an equal share of the lines
    int per_sm = 0;
    SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, 0));
    int grid = m->num_sms * (per_sm > 0 ? per_sm : 1);
    if (grid > kPBlocks) grid = kPBlocks;
    kern<<<grid, kPThreads, 0, st>>>(x, dinv, B, W, wout);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

template <typename T>
static int launch_update_box(const sem_mesh *m, T *x, const T *dinv, const PcgWork<T> &W, cudaStream_t st,
                             T *wout = nullptr) {
    switch (m->N) {
#define SEM_UB_CASE(n) \
    case n: return launch_update_box_n<T, n>(m, x, dinv, W, st, wout);
        SEM_UB_CASE(1) SEM_UB_CASE(2) SEM_UB_CASE(3) SEM_UB_CASE(4) SEM_UB_CASE(5)
        SEM_UB_CASE(6) SEM_UB_CASE(7) SEM_UB_CASE(8) SEM_UB_CASE(9) SEM_UB_CASE(10) SEM_UB_CASE(11)
#undef SEM_UB_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "order N not built");
    }
}

// ---- FP64 outer loop of the mixed solver ----

// r = b - w (w = A x, or null for x = 0); rr = <r,r>, bb = <b,b>; the
// convergence flag of the outer loop; scale = 1/||r|| for the inner start.
__global__ void __launch_bounds__(kPThreads)
    ir_residual_kernel(const double *__restrict__ b, const double *__restrict__ w, double *__restrict__ r,
                       const double *__restrict__ minv, int64_t n, double *partial, PcgScal *s, double tol,
                       int rel) {
    double v[2] = {0.0, 0.0};
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double bl = b[l];
        const double rl = w ? bl - w[l] : bl;
        r[l] = rl;
        const double mi = minv[l];
        v[0] = fma(bl * bl, mi, v[0]);
        v[1] = fma(rl * rl, mi, v[1]);
    }
    double t[2];
    if (grid_reduce<2>(v, partial, &s->cnt[0], t)) {
        s->bb = t[0];
        s->rr = t[1];
        s->tol2 = rel ? tol * tol * t[0] : tol * tol;
        s->scale_prev = s->scale;
        s->scale = t[1] > 0.0 ? 1.0 / sqrt(t[1]) : 0.0;
        s->iter += 1;
        set_start_flags(s, t[0], t[1]);
    }
}

// x += ||r|| d  (d: the inner FP32 solution of A d = r / ||r||).
__global__ void __launch_bounds__(kPThreads)
    ir_correct_kernel(double *__restrict__ x, float *__restrict__ d, int64_t n, const PcgScal *__restrict__ s) {
    const double nr = s->scale > 0.0 ? 1.0 / s->scale : 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        x[l] = fma((double)d[l], nr, x[l]);
        d[l] = 0.0f;
    }
}

// Refinement without restart: the FP32 residual becomes the new FP64
// residual r / ||r||; the FP32 search direction is rescaled by
// c = ||r_old|| / ||r_new|| to stay consistent with it; rho and beta are
// recomputed from the new residual (beta = rho / (rho_prev c^2)); the inner
// loop resumes until its residual has fallen by `delta` again.
__global__ void __launch_bounds__(kPThreads)
    ir_reliable_kernel(const double *__restrict__ r64, const float *__restrict__ dinv, const float *__restrict__ minv,
                       int64_t n, PcgWork<float> W, const PcgScal *__restrict__ so, double delta, double theta) {
    delta = inner_delta(so, delta, theta);
    const double inv = so->scale;
    const float c = (float)(so->scale / so->scale_prev);
    float f0 = 0.f, f1 = 0.f;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const float r = (float)(r64[l] * inv);
        W.r[l] = r;
        W.p[l] *= c;
        const float mi = minv[l];
        f0 = fmaf(r * r, mi, f0);
        f1 = fmaf(r * (dinv[l] * r), mi, f1);
    }
    double v[2] = {(double)f0, (double)f1}, t[2];
    if (grid_reduce<2>(v, W.partial + 2 * kPBlocks, &W.scal->cnt[2], t)) {
        PcgScal *s = W.scal;
        const double cc = (double)c * (double)c;
        s->rr = t[0];
        s->beta = t[1] / (s->rho_prev * cc);
        s->rho = t[1];
        s->tol2 = delta * delta * t[0];
        if (!isfinite(t[0])) {
            s->done = 1;
            s->status = SEM_ERR_NAN;
        } else {
            s->done = 0;
            s->status = SEM_ERR_NOT_CONVERGED;
        }
    }
}

// block partials of the vector kernels ([4][kPBlocks]) and of the fused operator
constexpr size_t kPartialBytes = sizeof(double) * (4 * kPBlocks + kAxMaxGrid);

static size_t pcg_scratch_f64(const sem_mesh *m) {
    return align_up(sizeof(double) * m->nloc) * 3 + align_up(kPartialBytes) + align_up(sizeof(PcgScal));
}

// mixed: FP64 r, w; FP32 d, r, p, w; two partial blocks; two scalar blocks
static size_t pcg_scratch_mixed(const sem_mesh *m) {
    return align_up(sizeof(double) * m->nloc) * 2 + align_up(sizeof(float) * m->nloc) * 6 +
           2 * align_up(kPartialBytes) + 2 * align_up(sizeof(PcgScal));
}

static int gmres_restart(const sem_pcg_opts *o) { return o->gmres_restart > 0 ? o->gmres_restart : 30; }

static size_t mid_bytes(const sem_pcg_opts *o) {
    return o->schwarz && o->schwarz_mid ? align_up(schwarz_mid_work_bytes(o->schwarz_mid)) : 0;
}

static size_t pcg_scratch(const sem_mesh *m, const sem_pcg_opts *o) {
    if (o && o->precision == SEM_PCG_MIXED)
        return pcg_scratch_mixed(m) + mid_bytes(o) +
               (o->krylov == SEM_KRYLOV_FGMRES ? gmres_work_bytes(m, gmres_restart(o)) : 0);
    return pcg_scratch_f64(m);
}

static PcgWork<double> carve_f64(const sem_mesh *m, void *scratch) {
    char *p = static_cast<char *>(scratch);
    PcgWork<double> W;
    const size_t vb = align_up(sizeof(double) * m->nloc);
    W.r = reinterpret_cast<double *>(p);
    W.p = reinterpret_cast<double *>(p + vb);
    W.w = reinterpret_cast<double *>(p + 2 * vb);
    W.partial = reinterpret_cast<double *>(p + 3 * vb);
    W.scal = reinterpret_cast<PcgScal *>(p + 3 * vb + align_up(kPartialBytes));
    return W;
}

struct MixedWork {
    double *r64, *w64;
    float *d32;
    float *z32;  // preconditioned residual (general preconditioner)
    float *wa32; // assembled A p of the last iteration (general preconditioner)
    double *partial_out;
    PcgScal *scal_out;
    PcgWork<float> in;
};

static MixedWork carve_mixed(const sem_mesh *m, void *scratch) {
    char *p = static_cast<char *>(scratch);
    const size_t vd = align_up(sizeof(double) * m->nloc), vf = align_up(sizeof(float) * m->nloc);
    const size_t pb = align_up(kPartialBytes), sb = align_up(sizeof(PcgScal));
    MixedWork M;
    M.r64 = reinterpret_cast<double *>(p);
    M.w64 = reinterpret_cast<double *>(p + vd);
    p += 2 * vd;
    M.d32 = reinterpret_cast<float *>(p);
    M.in.r = reinterpret_cast<float *>(p + vf);
    M.in.p = reinterpret_cast<float *>(p + 2 * vf);
    M.in.w = reinterpret_cast<float *>(p + 3 * vf);
    M.z32 = reinterpret_cast<float *>(p + 4 * vf);
    M.wa32 = reinterpret_cast<float *>(p + 5 * vf);
    p += 6 * vf;
    M.partial_out = reinterpret_cast<double *>(p);
    M.in.partial = reinterpret_cast<double *>(p + pb);
    p += 2 * pb;
    M.scal_out = reinterpret_cast<PcgScal *>(p);
    M.in.scal = reinterpret_cast<PcgScal *>(p + sb);
    return M;
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

// Assembled operator y = M Q Q^T (h1 A_L + h2 B) x in precision T, timed.
template <typename T>
static int apply_assembled_timed(const sem_mesh *m, const T *x, T *y, double h1, double h2, cudaStream_t st,
                                 SolveCtx &c, bool pair = false) {
    c.tax.start(st);
    int s;
    if (sizeof(T) == 8 && pair)
        s = ax_launch_pair(m, reinterpret_cast<const double *>(x), reinterpret_cast<double *>(y), st);
    else if (sizeof(T) == 8)
        s = ax_launch_f64(m, reinterpret_cast<const double *>(x), reinterpret_cast<double *>(y), h1, h2, st);
    else
        s = ax_launch_f32(m, reinterpret_cast<const float *>(x), reinterpret_cast<float *>(y), st);
    c.tax.stop(st);
    if (s != SEM_OK) return s;
    c.tgs.start(st);
    s = gs_launch(m, y, sizeof(T) == 8 ? SEM_F64 : SEM_F32, kGsSumMask, st);
    c.tgs.stop(st);
    c.launches += 2;
    c.ax_launches += 1;
    return s;
}


// CG iterations after an init kernel: three kernels per iteration (fused
// operator, gather-scatter, fused update), with a host check every `check`
// iterations.  Leaves the final scalars in *h.
template <typename T>
static int cg_loop(const sem_mesh *m, PcgWork<T> W, T *x, const T *dinv, int max_iter, int check, double h1,
                   double h2, cudaStream_t st, SolveCtx &c, PcgScal *h, bool pair = false) {
    NvtxRange nvtx_range("PCG iterations");
    CgFuse<T> cg{W.r, dinv, W.p, W.scal, W.partial + 4 * kPBlocks};
    int launched = 0;
    while (true) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(h, W.scal, sizeof(PcgScal), cudaMemcpyDeviceToHost, st));
        SEM_CUDA_CHECK(cudaStreamSynchronize(st));
        c.tax.harvest();
        c.tgs.harvest();
        if (h->done || launched >= max_iter) break;
        for (int q = 0; q < check && launched < max_iter; ++q, ++launched) {
            // p <- dinv r + beta p; w = A_L p; alpha = rho / <p, w>   (one kernel)
            c.tax.start(st);
            int s;
            if constexpr (sizeof(T) == 4)
                s = ax_cg_launch_f32(m, cg, W.w, st);
            else
                s = pair ? ax_cg_launch_pair(m, cg, W.w, st) : ax_cg_launch_f64(m, cg, W.w, h1, h2, st);
            c.tax.stop(st);
            if (s != SEM_OK) return s;
            // w <- M Q Q^T w, axis by axis: the y and z passes here, the x
            // pass and the mask inside the update
            c.tgs.start(st);
            s = gs_yz_launch(m, W.w, sizeof(T) == 8 ? SEM_F64 : SEM_F32, st);
            c.tgs.stop(st);
            if (s != SEM_OK) return s;
            // x += alpha p; r -= alpha w; rr, rz; beta; convergence flag
            s = launch_update_box<T>(m, x, dinv, W, st);
            if (s != SEM_OK) return s;
            c.launches += 3;
            c.ax_launches += 1;
        }
    }
    return SEM_OK;
}

// Flexible CG with a general preconditioner z = M r: rho = <r, z> and the
// Polak-Ribiere beta = <z, r_new - r_old> / rho_old = -alpha <z, A p> / rho_old
// (A p assembled in wa by the update; rho_old kept in rho_prev by the update),
// line-wise on the box topology (one thread per r-line, as the update): 1/mult
// from the point's position instead of a stored array, so only r, z and wa are
// read.
template <int N, bool VEC>
__global__ void __launch_bounds__(kPThreads)
    fpcg_dots_box_kernel(const float *__restrict__ r, const float *__restrict__ z, const float *__restrict__ wa,
                         BoxTopo B, PcgWork<float> W, int first) {
    if (W.scal->done) return;
    if (first < 0) first = W.scal->iter == 0 ? 1 : 0;  // uniform
    constexpr int N1 = N + 1, NL = N1 * N1;
    float f0 = 0.f, f1 = 0.f;
    const int nx = B.nel[0], ny = B.nel[1];
    const int64_t nlines = B.E * NL;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < nlines;
         L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = L / NL;
        const int jk = (int)(L - e * NL);
        const int j = jk % N1, k = jk / N1;
        const int ex = (int)(e % nx);
        const int64_t eyz = e / nx;
        const int ey = (int)(eyz % ny), ez = (int)(eyz / ny);
        const int64_t base = L * N1;
        float rv[N1], zv[N1], wv[N1];
        load_line<float, N1, VEC>(r + base, rv);
        load_line<float, N1, VEC>(z + base, zv);
        if (!first) load_line<float, N1, VEC>(wa + base, wv);
        int sy = 0, sz = 0, sx0 = 0, sxN = 0;
        bool dd = false;
        if (j == 0 || j == N) face_status(ey, ny, B.per[1], j == 0, 4, 8, B.faces, sy, dd);
        if (k == 0 || k == N) face_status(ez, B.nel[2], B.per[2], k == 0, 16, 32, B.faces, sz, dd);
        face_status(ex, nx, B.per[0], true, 1, 2, B.faces, sx0, dd);
        face_status(ex, nx, B.per[0], false, 1, 2, B.faces, sxN, dd);
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int sh = (i == 0 ? sx0 : (i == N ? sxN : 0)) + sy + sz;
            const float mi = sh == 0 ? 1.f : (sh == 1 ? 0.5f : (sh == 2 ? 0.25f : 0.125f));
            f0 = fmaf(rv[i] * zv[i], mi, f0);
            if (!first) f1 = fmaf(wv[i] * zv[i], mi, f1);
        }
    }
    double v[2] = {(double)f0, (double)f1}, t[2];
    if (grid_reduce<2>(v, W.partial, &W.scal->cnt[0], t)) {
        PcgScal *s = W.scal;
        s->beta = first ? 0.0 : -s->alpha * t[1] / s->rho_prev;
        s->rho = t[0];
    }
}

template <int N>
static int launch_fpcg_dots_box_n(const sem_mesh *m, const float *r, const float *z, const float *wa,
                                  const PcgWork<float> &W, int first, cudaStream_t st) {
    constexpr int N1 = N + 1;
    const BoxTopo B = box_topo(m);
    const bool vec = ((N1 * sizeof(float)) % 16 == 0);
    auto kv = fpcg_dots_box_kernel<N, ((N1 * sizeof(float)) % 16 == 0)>;
    auto ks = fpcg_dots_box_kernel<N, false>;
    auto kern = vec ? kv : ks;
    int per_sm = 0;
    SEM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, 0));
    int grid = m->num_sms * (per_sm > 0 ? per_sm : 1);
    if (grid > kPBlocks) grid = kPBlocks;
    kern<<<grid, kPThreads, 0, st>>>(r, z, wa, B, W, first);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

static int launch_fpcg_dots_box(const sem_mesh *m, const float *r, const float *z, const float *wa,
                                const PcgWork<float> &W, int first, cudaStream_t st) {
    switch (m->N) {
#define SEM_FD_CASE(n) \
    case n: return launch_fpcg_dots_box_n<n>(m, r, z, wa, W, first, st);
        SEM_FD_CASE(2) SEM_FD_CASE(3) SEM_FD_CASE(4) SEM_FD_CASE(5) SEM_FD_CASE(6) SEM_FD_CASE(7)
        SEM_FD_CASE(8) SEM_FD_CASE(9)
#undef SEM_FD_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "order N not built");
    }
}

// Inner FP32 flexible CG with the hybrid Schwarz preconditioner, after an
// init kernel: per iteration z = M r, the dots, the fused operator with
// p = z + beta p, the y/z gather-scatter, the update (x pass, mask; writes
// the assembled A p); host check every `check` iterations.
static int cg_loop_schwarz(const sem_mesh *m, PcgWork<float> W, float *z, float *wa, float *x, const sem_schwarz *sw,
                           int coarse_iters, double coarse_tol, int max_iter, int check, cudaStream_t st, SolveCtx &c,
                           PcgScal *h, const sem_schwarz *mid = nullptr, double mid_w = 0.0, void *mid_work = nullptr) {
    NvtxRange nvtx_range("flexible CG iterations (Schwarz)");
    CgFuse<float> cg{z, nullptr, W.p, W.scal, W.partial + 4 * kPBlocks};
    int launched = 0;
    while (true) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(h, W.scal, sizeof(PcgScal), cudaMemcpyDeviceToHost, st));
        SEM_CUDA_CHECK(cudaStreamSynchronize(st));
        c.tax.harvest();
        c.tgs.harvest();
        if (h->done || launched >= max_iter) break;
        for (int q = 0; q < check && launched < max_iter; ++q, ++launched) {
            int s = schwarz_apply_f32(sw, W.r, z, coarse_iters, coarse_tol, &W.scal->done, st);
            if (s != SEM_OK) return s;
            if (mid) {  // the intermediate level of the multigrid
                s = schwarz_mid_apply_add(sw, mid, mid_w, W.r, z, mid_work, &W.scal->done, st);
                if (s != SEM_OK) return s;
                c.launches += 4;
            }
            s = launch_fpcg_dots_box(m, W.r, z, wa, W, launched == 0 ? 1 : 0, st);
            if (s != SEM_OK) return s;
            c.tax.start(st);
            s = ax_cg_launch_f32(m, cg, W.w, st);
            c.tax.stop(st);
            if (s != SEM_OK) return s;
            c.tgs.start(st);
            s = gs_yz_launch(m, W.w, SEM_F32, st);
            c.tgs.stop(st);
            if (s != SEM_OK) return s;
            s = launch_update_box<float>(m, x, m->dinv32, W, st, wa);
            if (s != SEM_OK) return s;
            c.launches += coarse_iters > 0 ? 7 : 6;
            c.ax_launches += 1;
        }
    }
    return SEM_OK;
}

static int finish_stats(const sem_mesh *m, cudaStream_t st, sem_pcg_stats *stats, const SolveCtx &c, int status) {
    int derr = 0;
    SEM_CUDA_CHECK(cudaMemcpyAsync(&derr, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    stats->ax_ms = c.tax.total_ms;
    stats->gs_ms = c.tgs.total_ms;
    stats->ax_launches = c.ax_launches;
    stats->kernel_launches = c.launches;
    if (derr != 0) status = SEM_ERR_TIMEOUT;
    return status;
}

static int pcg_f64(const sem_mesh *m, const double *b, double *x, const sem_pcg_opts *o, sem_pcg_stats *stats,
                   void *scratch, cudaStream_t st) {
    PcgWork<double> W = carve_f64(m, scratch);
    const int64_t n = m->nloc;
    const int check = o->check_every > 0 ? o->check_every : 16;
    SolveCtx c;
    int s0 = c.tax.init(o->profile != 0, check + 1);
    if (s0 == SEM_OK) s0 = c.tgs.init(o->profile != 0, check + 1);
    if (s0 != SEM_OK) return s0;
    SEM_CUDA_CHECK(cudaMemsetAsync(W.scal, 0, sizeof(PcgScal), st));
    const bool pair = o->precision == SEM_PCG_F64_PAIR;
    const double *ax0 = nullptr;
    if (o->use_initial_guess) {
        int s = apply_assembled_timed<double>(m, x, W.w, o->h1, o->h2, st, c, pair);
        if (s != SEM_OK) return s;
        ax0 = W.w;
    } else {
        SEM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    }
    const double *dinv = o->dinv ? o->dinv : m->dinv;
    pcg_init_kernel<double, double><<<kPBlocks, kPThreads, 0, st>>>(b, ax0, dinv, m->minv, n, W, nullptr,
                                                                    o->tol, o->tol_is_relative, o->max_iter);
    SEM_CUDA_CHECK(cudaGetLastError());
    c.launches += 1;
    PcgScal h{};
    int s = cg_loop<double>(m, W, x, dinv, o->max_iter, check, o->h1, o->h2, st, c, &h, pair);
    if (s != SEM_OK) return s;
    stats->iters = h.iter;
    stats->outer_iters = 0;
    stats->init_rel_res = h.bb > 0 ? std::sqrt(h.rr0 / h.bb) : std::sqrt(h.rr0);
    stats->bnorm = std::sqrt(h.bb);
    stats->abs_res = std::sqrt(h.rr);
    stats->rel_res = h.bb > 0 ? std::sqrt(h.rr / h.bb) : stats->abs_res;
    return finish_stats(m, st, stats, c, h.done ? h.status : SEM_ERR_NOT_CONVERGED);
}

// FP64 iterative refinement around FP32 Jacobi-PCG:
//   r = b - A x (FP64);  repeat { solve A d = r/||r|| in FP32 to inner_tol;
//   x += ||r|| d (FP64);  r = b - A x (FP64) }  until ||r|| <= tol ||b||.
static int pcg_mixed(const sem_mesh *m, const double *b, double *x, const sem_pcg_opts *o, sem_pcg_stats *stats,
                     void *scratch, cudaStream_t st) {
    MixedWork M = carve_mixed(m, scratch);
    const int64_t n = m->nloc;
    const int check = o->check_every > 0 ? o->check_every : 16;
    const double inner_tol = o->inner_tol > 0.0 ? o->inner_tol : 1e-4;
    SolveCtx c, cin;
    int s0 = c.tax.init(o->profile != 0, 4);
    if (s0 == SEM_OK) s0 = c.tgs.init(o->profile != 0, 4);
    if (s0 == SEM_OK) s0 = cin.tax.init(o->profile != 0, check + 1);
    if (s0 == SEM_OK) s0 = cin.tgs.init(o->profile != 0, check + 1);
    if (s0 != SEM_OK) return s0;
    SEM_CUDA_CHECK(cudaMemsetAsync(M.scal_out, 0, sizeof(PcgScal), st));
    SEM_CUDA_CHECK(cudaMemsetAsync(M.in.scal, 0, sizeof(PcgScal), st));
    const double *w0 = nullptr;
    if (o->use_initial_guess) {
        int s = apply_assembled_timed<double>(m, x, M.w64, o->h1, o->h2, st, c, o->outer_pair != 0);
        if (s != SEM_OK) return s;
        w0 = M.w64;
    } else {
        SEM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    }
    ir_residual_kernel<<<kPBlocks, kPThreads, 0, st>>>(b, w0, M.r64, m->minv, n, M.partial_out, M.scal_out, o->tol,
                                                       o->tol_is_relative);
    SEM_CUDA_CHECK(cudaGetLastError());
    c.launches += 1;
    PcgScal ho{}, hi{};
    int inner_total = 0, outer = 0, status = SEM_ERR_NOT_CONVERGED;
    double prev_rr = -1.0, guard = 0.25;
    while (true) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(&ho, M.scal_out, sizeof(PcgScal), cudaMemcpyDeviceToHost, st));
        SEM_CUDA_CHECK(cudaStreamSynchronize(st));
        if (outer == 0) stats->init_rel_res = ho.bb > 0 ? std::sqrt(ho.rr / ho.bb) : std::sqrt(ho.rr);
        c.tax.harvest();
        c.tgs.harvest();
        if (ho.done) {
            status = ho.status;
            break;
        }
        if (inner_total >= o->max_iter) break;
        // stagnation guard: the FP64 residual must keep falling
        if (prev_rr >= 0.0 && !(ho.rr < guard * prev_rr)) break;
        prev_rr = ho.rr;
        const sem_schwarz *sw = static_cast<const sem_schwarz *>(o->schwarz);
        if (o->krylov == SEM_KRYLOV_FGMRES) {
            // one flexible GMRES cycle on A d = r / ||r||, from d = 0
            char *mid_work = static_cast<char *>(scratch) + pcg_scratch_mixed(m);
            GmresArgs ga{gmres_restart(o), o->max_iter - inner_total, check, inner_tol, o->inner_adapt, sw,
                         o->coarse_iters, o->coarse_tol > 0 ? o->coarse_tol : 1e-2,
                         static_cast<const sem_schwarz *>(o->schwarz_mid),
                         o->mid_weight > 0.0 ? o->mid_weight : 0.15, mid_work};
            GmresResult gr{};
            int s = gmres_cycle(m, M.r64, M.scal_out, M.d32, ga, mid_work + mid_bytes(o), st, &gr);
            if (s != SEM_OK) return s;
            cin.launches += gr.launches;
            cin.ax_launches += gr.ax_launches;
            inner_total += gr.iters;
            if (gr.status == SEM_ERR_NAN) {
                status = SEM_ERR_NAN;
                break;
            }
            // a cycle that stopped at its restart length must still lower the
            // FP64 residual, one that met its tolerance by the usual factor
            guard = gr.converged ? 0.25 : 1.0;
        } else if (outer == 0 || o->mixed_restart || sw) {
            // inner FP32 solve of A d = r / ||r||, from d = 0
            SEM_CUDA_CHECK(cudaMemsetAsync(M.d32, 0, sizeof(float) * n, st));
            pcg_init_kernel<float, double><<<kPBlocks, kPThreads, 0, st>>>(
                M.r64, nullptr, m->dinv32, m->minv32, n, M.in, M.scal_out, inner_tol, 1, o->max_iter - inner_total,
                o->inner_adapt);
        } else {
            // keep the search direction: swap in the FP64 residual and go on
            ir_reliable_kernel<<<kPBlocks, kPThreads, 0, st>>>(M.r64, m->dinv32, m->minv32, n, M.in, M.scal_out,
                                                               inner_tol, o->inner_adapt);
        }
        SEM_CUDA_CHECK(cudaGetLastError());
        cin.launches += 1;
        int s = SEM_OK;
        if (o->krylov == SEM_KRYLOV_FGMRES)
            ;  // the cycle above
        else if (sw)
            s = cg_loop_schwarz(m, M.in, M.z32, M.wa32, M.d32, sw, o->coarse_iters, o->coarse_tol > 0 ? o->coarse_tol : 1e-2,
                                o->max_iter - inner_total, check, st, cin, &hi, o->schwarz_mid,
                                o->mid_weight > 0.0 ? o->mid_weight : 0.15,
                                static_cast<char *>(scratch) + pcg_scratch_mixed(m));
        else
            s = cg_loop<float>(m, M.in, M.d32, m->dinv32, o->max_iter - inner_total, check, o->h1, o->h2, st, cin,
                               &hi);
        if (s != SEM_OK) return s;
        if (o->krylov != SEM_KRYLOV_FGMRES)
            inner_total = (o->mixed_restart || sw) ? inner_total + hi.iter : hi.iter;
        // x += ||r|| d; r = b - A x in FP64
        ir_correct_kernel<<<kPBlocks, kPThreads, 0, st>>>(x, M.d32, n, M.scal_out);
        s = apply_assembled_timed<double>(m, x, M.w64, o->h1, o->h2, st, c, o->outer_pair != 0);
        if (s != SEM_OK) return s;
        ir_residual_kernel<<<kPBlocks, kPThreads, 0, st>>>(b, M.w64, M.r64, m->minv, n, M.partial_out, M.scal_out,
                                                           o->tol, o->tol_is_relative);
        SEM_CUDA_CHECK(cudaGetLastError());
        c.launches += 2;
        ++outer;
    }
    stats->iters = inner_total;
    stats->outer_iters = outer;
    stats->bnorm = std::sqrt(ho.bb);
    stats->abs_res = std::sqrt(ho.rr);
    stats->rel_res = ho.bb > 0 ? std::sqrt(ho.rr / ho.bb) : stats->abs_res;
    // the operator timings: inner FP32 launches (ax_ms) and FP64 outer ones
    SolveCtx tot;
    tot.launches = c.launches + cin.launches;
    tot.ax_launches = cin.ax_launches;
    tot.tax.total_ms = cin.tax.total_ms;
    tot.tgs.total_ms = cin.tgs.total_ms;
    stats->outer_ax_ms = c.tax.total_ms;
    stats->outer_ax_launches = c.ax_launches;
    return finish_stats(m, st, stats, tot, status);
}

static int check_opts(const sem_mesh *m, const sem_pcg_opts *o) {
    if (o->precision != SEM_PCG_F64 && o->precision != SEM_PCG_MIXED && o->precision != SEM_PCG_F64_PAIR)
        return fail(SEM_ERR_UNSUPPORTED, "unknown precision mode");
    if (o->schwarz && o->precision != SEM_PCG_MIXED)
        return fail(SEM_ERR_UNSUPPORTED, "the Schwarz preconditioner is used by SEM_PCG_MIXED");
    if (o->schwarz && schwarz_mesh(o->schwarz) != m)
        return fail(SEM_ERR_INVALID_ARG, "the Schwarz preconditioner was built on another mesh");
    if (o->schwarz && (o->h2 != 0.0 || o->h1 != 1.0 || o->dinv))
        return fail(SEM_ERR_UNSUPPORTED, "the Schwarz preconditioner is built for the Poisson operator");
    if (o->schwarz_mid && !o->schwarz)
        return fail(SEM_ERR_INVALID_ARG, "schwarz_mid is the intermediate level of a Schwarz preconditioner");
    if (o->schwarz_mid) {
        int s = schwarz_mid_check(o->schwarz, o->schwarz_mid);
        if (s != SEM_OK) return s;
        if (o->mid_weight < 0.0) return fail(SEM_ERR_INVALID_ARG, "mid_weight < 0");
    }
    if (o->precision == SEM_PCG_F64_PAIR && !m->G2)
        return fail(SEM_ERR_INVALID_ARG, "SEM_PCG_F64_PAIR needs a mesh built with SEM_GEOM_PAIR");
    if (o->precision == SEM_PCG_F64_PAIR && (o->h2 != 0.0 || o->h1 != 1.0))
        return fail(SEM_ERR_UNSUPPORTED, "SEM_PCG_F64_PAIR solves the Poisson operator (h1 = 1, h2 = 0)");
    if (o->outer_pair && (o->precision != SEM_PCG_MIXED || !m->G2))
        return fail(SEM_ERR_INVALID_ARG, "outer_pair: SEM_PCG_MIXED on a mesh built with SEM_GEOM_PAIR");
    if (o->precision == SEM_PCG_MIXED && !m->G32)
        return fail(SEM_ERR_INVALID_ARG, "SEM_PCG_MIXED needs a mesh built with SEM_GEOM_F32");
    if (o->precision == SEM_PCG_MIXED && (o->h2 != 0.0 || o->h1 != 1.0 || o->dinv))
        return fail(SEM_ERR_UNSUPPORTED, "SEM_PCG_MIXED solves the Poisson operator (h1 = 1, h2 = 0, mesh diagonal)");
    if (!(o->inner_adapt >= 0.0 && o->inner_adapt < 1.0))
        return fail(SEM_ERR_INVALID_ARG, "inner_adapt must be in [0, 1)");
    if (o->krylov != SEM_KRYLOV_CG && o->krylov != SEM_KRYLOV_FGMRES)
        return fail(SEM_ERR_INVALID_ARG, "unknown krylov method");
    if (o->krylov == SEM_KRYLOV_FGMRES && o->precision != SEM_PCG_MIXED)
        return fail(SEM_ERR_UNSUPPORTED, "flexible GMRES is the inner solver of SEM_PCG_MIXED");
    if (o->gmres_restart < 0 || o->gmres_restart > kGmMaxRestart)
        return fail(SEM_ERR_INVALID_ARG, "gmres_restart outside [0, 128]");
    if (!(o->tol > 0.0) || o->max_iter < 1) return fail(SEM_ERR_INVALID_ARG, "tol must be > 0, max_iter >= 1");
    return SEM_OK;
}

static int solve_dispatch(const sem_mesh *m, const double *b, double *x, const sem_pcg_opts *o,
                          sem_pcg_stats *stats, void *scratch, cudaStream_t st) {
    NvtxRange nvtx_range("sem_pcg_solve");
    // every solve reports the timeouts of its own kernels: an earlier call's
    // give-up (already reported by that call, or read with
    // sem_mesh_check_device_error) is cleared here
    SEM_CUDA_CHECK(cudaMemsetAsync(m->d_err, 0, sizeof(int), st));
    if (o->precision == SEM_PCG_MIXED) return pcg_mixed(m, b, x, o, stats, scratch, st);
    return pcg_f64(m, b, x, o, stats, scratch, st);
}

// ---------------------------------------------------------------- batched solves
//
// Many independent mixed-precision solves run in ONE graph launch.  Every
// decision of the solver runs on the device, per solve, as a phase:
//   kBtIterate  FP32 CG iterations (the kernels return at once when the
//               inner solve has paused: its residual fell by inner_tol);
//   kBtRefine   x += ||r|| d (FP64), r = b - A x (FP64), convergence /
//               stagnation / budget decision;
//   kBtReliable swap the FP64 residual into the FP32 iteration, rescale p,
//               recompute beta, resume;
//   kBtFinished nothing more to do.
// Per solve the graph holds the start kernels and a WHILE conditional node
// whose body is one round: K FP32 iterations, the guarded refinement stage,
// and a kernel that counts the round and sets the node's condition -- loop
// again unless the solve has finished, its round budget is spent or a
// bounded wait of one of its kernels gave up (mesh error word).  The solves
// are parallel branches of the graph, so each iterates at its own pace (a
// small solve is done after its own rounds, not after the largest one's) and
// the host waits once, for the whole batch.  The last kernel of each solve
// records its completion time from the global timer.

constexpr int kBtIterate = 0, kBtRefine = 1, kBtReliable = 2, kBtFinished = 3;

__global__ void bt_pause_kernel(const PcgScal *__restrict__ in, PcgScal *__restrict__ out) {
    if (threadIdx.x == 0 && out->phase == kBtIterate && in->done) {
        if (in->status == SEM_ERR_NAN) {
            out->phase = kBtFinished;
            out->status = SEM_ERR_NAN;
        } else {
            out->phase = kBtRefine;
        }
    }
}

__global__ void __launch_bounds__(kPThreads)
    bt_correct_kernel(double *__restrict__ x, float *__restrict__ d, int64_t n, const PcgScal *__restrict__ s) {
    if (s->phase != kBtRefine) return;
    const double nr = s->scale > 0.0 ? 1.0 / s->scale : 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        x[l] = fma((double)d[l], nr, x[l]);
        d[l] = 0.0f;
    }
}

// r = b - w (FP64); decide: converged -> finished (OK); inner budget spent
// or no progress -> finished (not converged); else -> reliable update.
__global__ void __launch_bounds__(kPThreads)
    bt_residual_kernel(const double *__restrict__ b, const double *__restrict__ w, double *__restrict__ r,
                       const double *__restrict__ minv, int64_t n, double *partial, PcgScal *s,
                       const PcgScal *__restrict__ in) {
    if (s->phase != kBtRefine) return;
    double v[1] = {0.0};
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const double rl = b[l] - w[l];
        r[l] = rl;
        v[0] = fma(rl * rl, minv[l], v[0]);
    }
    double t[1];
    if (grid_reduce<1>(v, partial, &s->cnt[0], t)) {
        const double rr = t[0];
        s->rr = rr;
        s->scale_prev = s->scale;
        s->scale = rr > 0.0 ? 1.0 / sqrt(rr) : 0.0;
        s->iter += 1;  // refinements
        if (!isfinite(rr)) {
            s->phase = kBtFinished;
            s->status = SEM_ERR_NAN;
        } else if (rr <= s->tol2) {
            s->phase = kBtFinished;
            s->status = SEM_OK;
        } else if (in->iter >= in->max_iter || (s->prev_rr > 0.0 && !(rr < 0.25 * s->prev_rr))) {
            s->phase = kBtFinished;
            s->status = SEM_ERR_NOT_CONVERGED;
        } else {
            s->phase = kBtReliable;
        }
        s->prev_rr = rr;
    }
}

// the reliable update of ir_reliable_kernel, run only in phase kBtReliable;
// the last block resumes the iteration.
__global__ void __launch_bounds__(kPThreads)
    bt_reliable_kernel(const double *__restrict__ r64, const float *__restrict__ dinv, const float *__restrict__ minv,
                       int64_t n, PcgWork<float> W, PcgScal *so, double delta, double theta) {
    if (so->phase != kBtReliable) return;
    delta = inner_delta(so, delta, theta);
    const double inv = so->scale;
    const float c = (float)(so->scale / so->scale_prev);
    float f0 = 0.f, f1 = 0.f;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const float r = (float)(r64[l] * inv);
        W.r[l] = r;
        W.p[l] *= c;
        const float mi = minv[l];
        f0 = fmaf(r * r, mi, f0);
        f1 = fmaf(r * (dinv[l] * r), mi, f1);
    }
    double v[2] = {(double)f0, (double)f1}, t[2];
    if (grid_reduce<2>(v, W.partial + 2 * kPBlocks, &W.scal->cnt[2], t)) {
        PcgScal *s = W.scal;
        const double cc = (double)c * (double)c;
        s->rr = t[0];
        s->beta = t[1] / (s->rho_prev * cc);
        s->rho = t[1];
        s->tol2 = delta * delta * t[0];
        s->done = 0;
        s->status = SEM_ERR_NOT_CONVERGED;
        so->phase = kBtIterate;
    }
}

// Start of the graph: the reference time of the completion times.
__global__ void bt_clock_kernel(unsigned long long *t0) {
    if (threadIdx.x == 0) *t0 = global_timer_ns();
}

// After the start: a solve whose right-hand side is already converged (or
// holds a NaN) is finished, the others iterate; the loop condition follows.
__global__ void bt_start_kernel(PcgScal *s, cudaGraphConditionalHandle h, unsigned long long *tdone) {
    if (threadIdx.x == 0) {
        s->prev_rr = s->rr;
        s->rounds = 0;
        s->phase = s->done ? kBtFinished : kBtIterate;
        if (s->phase == kBtFinished) *tdone = global_timer_ns();
        cudaGraphSetConditional(h, s->phase == kBtFinished ? 0u : 1u);
    }
}

// End of a round: count it; finish the solve when its round budget is spent
// or a bounded wait of one of its kernels gave up; record the completion
// time; loop again unless finished.
__global__ void bt_round_end_kernel(PcgScal *s, const int *__restrict__ err, int max_rounds,
                                    cudaGraphConditionalHandle h, unsigned long long *tdone) {
    if (threadIdx.x != 0) return;
    s->rounds += 1;
    if (s->phase != kBtFinished) {
        if (*err != 0) {
            s->phase = kBtFinished;
            s->status = SEM_ERR_TIMEOUT;
        } else if (s->rounds >= max_rounds) {
            s->phase = kBtFinished;
            s->status = SEM_ERR_NOT_CONVERGED;
        }
    }
    const bool fin = s->phase == kBtFinished;
    if (fin) *tdone = global_timer_ns();
    cudaGraphSetConditional(h, fin ? 0u : 1u);
}

// Schwarz inner solve (flexible CG, restarted at every refinement): in
// phase kBtReliable the inner FP32 iteration starts again from the new FP64
// residual (the init of the single-solve path), then the solve iterates.
__global__ void __launch_bounds__(kPThreads)
    bt_restart_kernel(const double *__restrict__ r64, const float *__restrict__ dinv, const float *__restrict__ minv,
                      int64_t n, PcgWork<float> W, PcgScal *so, double delta, int max_iter, double theta) {
    if (so->phase != kBtReliable) return;  // uniform
    const int before = W.scal->iter;  // read before the last block resets it
    if (pcg_init_body<float, double>(r64, nullptr, dinv, minv, n, W, so, delta, 1, max_iter, theta)) {
        so->inner_done += before;
        so->phase = W.scal->done && W.scal->status == SEM_ERR_NAN ? kBtFinished : kBtIterate;
    }
}

struct BtSolve {
    const sem_mesh *m;
    const double *b;
    double *x;
    MixedWork M;
    const sem_schwarz *sw;  // hybrid Schwarz inner preconditioner, or nullptr (Jacobi)
};

// One round of solve i on stream st: K FP32 iterations, then the guarded
// refinement stage.  Launch-time host work only; all state on the device.
static int bt_round(BtSolve &S, const sem_pcg_opts *o, int K, cudaStream_t st) {
    const sem_mesh *m = S.m;
    const int64_t n = m->nloc;
    const double itol = o->inner_tol > 0.0 ? o->inner_tol : 1e-2;
    if (S.sw) {
        // flexible CG with the hybrid Schwarz preconditioner (coarse CG as
        // separate launches: the branches of the graph run concurrently)
        CgFuse<float> cgs{S.M.z32, nullptr, S.M.in.p, S.M.in.scal, S.M.in.partial + 4 * kPBlocks};
        const double ctol = o->coarse_tol > 0 ? o->coarse_tol : 1e-2;
        for (int q = 0; q < K; ++q) {
            int s = schwarz_apply_f32(S.sw, S.M.in.r, S.M.z32, o->coarse_iters, ctol, &S.M.in.scal->done, st, false);
            if (s != SEM_OK) return s;
            s = launch_fpcg_dots_box(m, S.M.in.r, S.M.z32, S.M.wa32, S.M.in, -1, st);
            if (s != SEM_OK) return s;
            s = ax_cg_launch_f32(m, cgs, S.M.in.w, st);
            if (s != SEM_OK) return s;
            s = gs_yz_launch(m, S.M.in.w, SEM_F32, st, &S.M.in.scal->done, 0);
            if (s != SEM_OK) return s;
            s = launch_update_box<float>(m, S.M.d32, m->dinv32, S.M.in, st, S.M.wa32);
            if (s != SEM_OK) return s;
        }
    }
    CgFuse<float> cg{S.M.in.r, m->dinv32, S.M.in.p, S.M.in.scal, S.M.in.partial + 4 * kPBlocks};
    for (int q = 0; q < (S.sw ? 0 : K); ++q) {
        int s = ax_cg_launch_f32(m, cg, S.M.in.w, st);
        if (s != SEM_OK) return s;
        // axis-by-axis gather-scatter: y and z passes (guarded by the solve's
        // done flag), the x pass and the mask inside the update
        s = gs_yz_launch(m, S.M.in.w, SEM_F32, st, &S.M.in.scal->done, 0);
        if (s != SEM_OK) return s;
        s = launch_update_box<float>(m, S.M.d32, m->dinv32, S.M.in, st);
        if (s != SEM_OK) return s;
    }
    bt_pause_kernel<<<1, 32, 0, st>>>(S.M.in.scal, S.M.scal_out);
    bt_correct_kernel<<<kPBlocks, kPThreads, 0, st>>>(S.x, S.M.d32, n, S.M.scal_out);
    int s = ax_launch_f64(m, S.x, S.M.w64, 1.0, 0.0, st, &S.M.scal_out->phase, kBtRefine);
    if (s != SEM_OK) return s;
    s = gs_launch(m, S.M.w64, SEM_F64, kGsSumMask, st, &S.M.scal_out->phase, kBtRefine);
    if (s != SEM_OK) return s;
    bt_residual_kernel<<<kPBlocks, kPThreads, 0, st>>>(S.b, S.M.w64, S.M.r64, m->minv, n, S.M.partial_out,
                                                       S.M.scal_out, S.M.in.scal);
    if (S.sw)
        bt_restart_kernel<<<kPBlocks, kPThreads, 0, st>>>(S.M.r64, m->dinv32, m->minv32, n, S.M.in, S.M.scal_out,
                                                          itol, o->max_iter, o->inner_adapt);
    else
        bt_reliable_kernel<<<kPBlocks, kPThreads, 0, st>>>(S.M.r64, m->dinv32, m->minv32, n, S.M.in, S.M.scal_out,
                                                           itol, o->inner_adapt);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

size_t sem_pcg_scratch_bytes(const sem_mesh *m, const sem_pcg_opts *o) {
    if (!m) return 0;
    return pcg_scratch(m, o);
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
    int s = check_opts(m, o);
    if (s != SEM_OK) return s;
    if (scratch_bytes < sem_pcg_scratch_bytes(m, o) || reinterpret_cast<uintptr_t>(scratch) % kAlign)
        return fail(SEM_ERR_WORKSPACE, "scratch smaller than sem_pcg_scratch_bytes or not 256-byte aligned");
    s = solve_dispatch(m, b, x, o, stats, scratch, as_stream(stream));
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
    int s = check_opts(m, o);
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
    s = solve_dispatch(m, db, dx, o, stats, inner, st);
    if (s == SEM_OK || s == SEM_ERR_NOT_CONVERGED) {
        SEM_CUDA_CHECK(cudaMemcpyAsync(hx, dx, sizeof(double) * m->nloc, cudaMemcpyDeviceToHost, st));
        SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    }
    stats->status = s;
    stats->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (s != SEM_OK && s != SEM_ERR_CUDA) set_error(sem_status_string(s));
    return s;
}


size_t sem_pcg_batched_scratch_bytes(const sem_mesh *const *meshes, int nsolve, const sem_pcg_opts *o) {
    if (!meshes || nsolve <= 0) return 0;
    size_t t = align_up(sizeof(unsigned long long) * (nsolve + 1));  // start time, completion times
    for (int i = 0; i < nsolve; ++i) {
        if (!meshes[i]) return 0;
        t += align_up(pcg_scratch_mixed(meshes[i]));
    }
    (void)o;
    return t;
}

}  // extern "C"

namespace sem {

// Streams, events and the graph of one batched call, released on every exit.
struct BtGraph {
    std::vector<cudaStream_t> ss, bss;
    std::vector<cudaEvent_t> ev;
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool capturing = false;
    ~BtGraph() {
        if (capturing) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
            if (junk) cudaGraphDestroy(junk);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        for (auto q : ss) cudaStreamDestroy(q);
        for (auto q : bss) cudaStreamDestroy(q);
        for (auto e : ev) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
        cudaGetLastError();  // errors of a failed capture are reported by the caller
    }
};

// Capture solve S on stream q (already part of the capture): the start
// kernels, then a WHILE node whose body is one round.
static int bt_capture_solve(BtSolve &S, const sem_pcg_opts *o, int K, int max_rounds, cudaStream_t q,
                            cudaStream_t bs, unsigned long long *tdone) {
    const sem_mesh *m = S.m;
    const int64_t n = m->nloc;
    const double itol = o->inner_tol > 0.0 ? o->inner_tol : 1e-2;
    SEM_CUDA_CHECK(cudaMemsetAsync(S.M.scal_out, 0, sizeof(PcgScal), q));
    SEM_CUDA_CHECK(cudaMemsetAsync(S.M.in.scal, 0, sizeof(PcgScal), q));
    SEM_CUDA_CHECK(cudaMemsetAsync(S.x, 0, sizeof(double) * n, q));
    SEM_CUDA_CHECK(cudaMemsetAsync(S.M.d32, 0, sizeof(float) * n, q));
    ir_residual_kernel<<<kPBlocks, kPThreads, 0, q>>>(S.b, nullptr, S.M.r64, m->minv, n, S.M.partial_out,
                                                      S.M.scal_out, o->tol, o->tol_is_relative);
    pcg_init_kernel<float, double><<<kPBlocks, kPThreads, 0, q>>>(S.M.r64, nullptr, m->dinv32, m->minv32, n, S.M.in,
                                                                  S.M.scal_out, itol, 1, o->max_iter,
                                                                  o->inner_adapt);
    SEM_CUDA_CHECK(cudaGetLastError());
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    SEM_CUDA_CHECK(cudaStreamGetCaptureInfo(q, &cst, nullptr, &g));
    cudaGraphConditionalHandle h;
    SEM_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    bt_start_kernel<<<1, 32, 0, q>>>(S.M.scal_out, h, tdone);
    SEM_CUDA_CHECK(cudaGetLastError());
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    SEM_CUDA_CHECK(cudaStreamGetCaptureInfo(q, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    SEM_CUDA_CHECK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
    SEM_CUDA_CHECK(cudaStreamUpdateCaptureDependencies(q, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    // the loop body: one round of this solve
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    SEM_CUDA_CHECK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int s = bt_round(S, o, K, bs);
    if (s == SEM_OK) {
        bt_round_end_kernel<<<1, 32, 0, bs>>>(S.M.scal_out, m->d_err, max_rounds, h, tdone);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(e, "bt_round_end_kernel");
    }
    cudaGraph_t out = nullptr;
    cudaError_t ce = cudaStreamEndCapture(bs, &out);
    if (s != SEM_OK) return s;
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (round body)");
    return SEM_OK;
}

}  // namespace sem

extern "C" {

}  // extern "C"

namespace sem {

// The batched solve; sws: per-solve hybrid Schwarz objects (nullptr: Jacobi).
static int batched_impl(const sem_mesh *const *meshes, const sem_schwarz *const *sws, int nsolve,
                        const double *const *b, double *const *x, const sem_pcg_opts *o, sem_pcg_stats *stats,
                        void *scratch, size_t scratch_bytes, void *stream) {
    NvtxRange nvtx_range("batched solves (one graph)");
    const auto t0 = std::chrono::steady_clock::now();
    if (!meshes || nsolve <= 0 || !b || !x || !o || !stats || !scratch)
        return fail(SEM_ERR_INVALID_ARG, "NULL argument or nsolve <= 0");
    if (o->precision != SEM_PCG_MIXED) return fail(SEM_ERR_UNSUPPORTED, "batched solves use SEM_PCG_MIXED");
    if (o->use_initial_guess) return fail(SEM_ERR_UNSUPPORTED, "batched solves start from x = 0");
    if (o->schwarz || o->schwarz_mid || o->outer_pair)
        return fail(SEM_ERR_UNSUPPORTED, "batched solves use the Jacobi inner solver");
    if (o->krylov != SEM_KRYLOV_CG) return fail(SEM_ERR_UNSUPPORTED, "batched solves use CG inner solves");
    if (!(o->inner_adapt >= 0.0 && o->inner_adapt < 1.0))
        return fail(SEM_ERR_INVALID_ARG, "inner_adapt must be in [0, 1)");
    if (!(o->tol > 0.0) || o->max_iter < 1) return fail(SEM_ERR_INVALID_ARG, "tol must be > 0, max_iter >= 1");
    for (int i = 0; i < nsolve; ++i) {
        if (!meshes[i] || !b[i] || !x[i]) return fail(SEM_ERR_INVALID_ARG, "NULL mesh, b or x");
        if (!meshes[i]->G32) return fail(SEM_ERR_INVALID_ARG, "batched solves need meshes built with SEM_GEOM_F32");
        if (meshes[i]->device != meshes[0]->device) return fail(SEM_ERR_INVALID_ARG, "meshes on different devices");
    }
    if (scratch_bytes < sem_pcg_batched_scratch_bytes(meshes, nsolve, o) ||
        reinterpret_cast<uintptr_t>(scratch) % kAlign)
        return fail(SEM_ERR_WORKSPACE, "scratch smaller than sem_pcg_batched_scratch_bytes or misaligned");
    cudaStream_t st = as_stream(stream);
    for (int i = 0; i < nsolve; ++i) SEM_CUDA_CHECK(cudaMemsetAsync(meshes[i]->d_err, 0, sizeof(int), st));
    char *p = static_cast<char *>(scratch);
    unsigned long long *d_t = reinterpret_cast<unsigned long long *>(p);  // [0]: start, [1 + i]: solve i done
    p += align_up(sizeof(unsigned long long) * (nsolve + 1));
    std::vector<BtSolve> S(nsolve);
    for (int i = 0; i < nsolve; ++i) {
        S[i].m = meshes[i];
        S[i].b = b[i];
        S[i].x = x[i];
        S[i].M = carve_mixed(meshes[i], p);
        S[i].sw = sws ? sws[i] : nullptr;
        p += align_up(pcg_scratch_mixed(meshes[i]));
    }
    const int K = o->check_every > 0 ? o->check_every : 16;
    const int max_rounds = o->max_iter / K + 64;

    // Shortest job first: every solve's kernels carry a scheduling priority
    // from the rank of its estimated work, local points x elements along an
    // axis x N (CG iterations grow like 1/h ~ nel N), the smallest work the
    // greatest priority, spread evenly over the device's priority levels.
    // The block scheduler then serves the small solves first: their latency
    // drops while the batch's total work and end time stay the same.
    int prio_least = 0, prio_greatest = 0;
    SEM_CUDA_CHECK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    const int levels = prio_least - prio_greatest + 1;
    std::vector<int> order(nsolve), prio(nsolve);
    std::vector<double> work(nsolve);
    for (int i = 0; i < nsolve; ++i) {
        const sem_mesh *m = meshes[i];
        const int nmax = std::max(m->nel[0], std::max(m->nel[1], m->nel[2]));
        work[i] = (double)m->nloc * nmax * m->N;
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work[a] < work[c]; });
    for (int r = 0; r < nsolve; ++r) prio[order[r]] = prio_greatest + (int)((int64_t)r * levels / nsolve);

    // Build the graph by capture on streams of our own (the caller's may be
    // the legacy default stream, which cannot be captured): a clock kernel,
    // then one branch per solve (captured on a stream of the solve's
    // priority, the loop body too), joined at the end.
    BtGraph G;
    G.ss.resize(nsolve);
    G.bss.resize(levels);
    G.ev.resize(nsolve + 1);
    for (int i = 0; i < nsolve; ++i)
        SEM_CUDA_CHECK(cudaStreamCreateWithPriority(&G.ss[i], cudaStreamNonBlocking, prio[i]));
    for (int l = 0; l < levels; ++l)
        SEM_CUDA_CHECK(cudaStreamCreateWithPriority(&G.bss[l], cudaStreamNonBlocking, prio_greatest + l));
    for (auto &e : G.ev) SEM_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    SEM_CUDA_CHECK(cudaStreamCreateWithFlags(&G.cs, cudaStreamNonBlocking));
    SEM_CUDA_CHECK(cudaStreamBeginCapture(G.cs, cudaStreamCaptureModeRelaxed));
    G.capturing = true;
    bt_clock_kernel<<<1, 32, 0, G.cs>>>(d_t);
    SEM_CUDA_CHECK(cudaGetLastError());
    SEM_CUDA_CHECK(cudaEventRecord(G.ev[nsolve], G.cs));
    for (int i = 0; i < nsolve; ++i) {
        SEM_CUDA_CHECK(cudaStreamWaitEvent(G.ss[i], G.ev[nsolve], 0));
        int s = bt_capture_solve(S[i], o, K, max_rounds, G.ss[i], G.bss[prio[i] - prio_greatest], d_t + 1 + i);
        if (s != SEM_OK) return s;
        SEM_CUDA_CHECK(cudaEventRecord(G.ev[i], G.ss[i]));
        SEM_CUDA_CHECK(cudaStreamWaitEvent(G.cs, G.ev[i], 0));
    }
    G.capturing = false;
    SEM_CUDA_CHECK(cudaStreamEndCapture(G.cs, &G.g));
    SEM_CUDA_CHECK(cudaGraphInstantiate(&G.exec, G.g, cudaGraphInstantiateFlagUseNodePriority));
    // the one launch of the batch, and the one wait
    SEM_CUDA_CHECK(cudaGraphLaunch(G.exec, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));

    // per-solve statistics
    std::vector<unsigned long long> ht(nsolve + 1, 0ull);
    SEM_CUDA_CHECK(cudaMemcpy(ht.data(), d_t, sizeof(unsigned long long) * (nsolve + 1), cudaMemcpyDeviceToHost));
    // kernels of one round body (Schwarz: local solves, coarse CG launches,
    // overlap sums, dots, operator, gather-scatter, update per iteration)
    const int per_round = (sws ? (7 + 2 * o->coarse_iters) * K : 3 * K) + 7;
    int status = SEM_OK, derr = 0;
    for (int i = 0; i < nsolve; ++i) {
        PcgScal ho{}, hi{};
        SEM_CUDA_CHECK(cudaMemcpy(&ho, S[i].M.scal_out, sizeof(PcgScal), cudaMemcpyDeviceToHost));
        SEM_CUDA_CHECK(cudaMemcpy(&hi, S[i].M.in.scal, sizeof(PcgScal), cudaMemcpyDeviceToHost));
        int e = 0;
        SEM_CUDA_CHECK(cudaMemcpy(&e, meshes[i]->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        derr |= e;
        sem_pcg_stats &t = stats[i];
        t = sem_pcg_stats{};
        t.iters = hi.iter + ho.inner_done;
        t.outer_iters = ho.iter > 0 ? ho.iter - 1 : 0;
        t.bnorm = std::sqrt(ho.bb);
        t.abs_res = std::sqrt(ho.rr);
        t.rel_res = ho.bb > 0 ? std::sqrt(ho.rr / ho.bb) : t.abs_res;
        t.init_rel_res = 1.0;
        t.status = ho.phase == kBtFinished ? ho.status : SEM_ERR_NOT_CONVERGED;
        if (e) t.status = SEM_ERR_TIMEOUT;
        // device time from the start of the batch's graph to this solve's last round
        t.wall_ms = ht[1 + i] >= ht[0] ? (double)(ht[1 + i] - ht[0]) * 1e-6 : -1.0;
        t.kernel_launches = 6 + ho.rounds * per_round;
        t.ax_launches = ho.rounds;  // rounds of the device-side loop
        if (t.status != SEM_OK && status == SEM_OK) status = t.status;
    }
    if (derr) status = SEM_ERR_TIMEOUT;
    if (status != SEM_OK) set_error(sem_status_string(status));
    (void)t0;
    return status;
}

}  // namespace sem

extern "C" {

int sem_pcg_solve_batched(const sem_mesh *const *meshes, int nsolve, const double *const *b, double *const *x,
                          const sem_pcg_opts *o, sem_pcg_stats *stats, void *scratch, size_t scratch_bytes,
                          void *stream) {
    return batched_impl(meshes, nullptr, nsolve, b, x, o, stats, scratch, scratch_bytes, stream);
}

int sem_pcg_solve_batched_schwarz(const sem_mesh *const *meshes, const sem_schwarz *const *sws, int nsolve,
                                  const double *const *b, double *const *x, const sem_pcg_opts *o,
                                  sem_pcg_stats *stats, void *scratch, size_t scratch_bytes, void *stream) {
    if (!meshes || !sws || nsolve <= 0) return fail(SEM_ERR_INVALID_ARG, "NULL argument or nsolve <= 0");
    for (int i = 0; i < nsolve; ++i) {
        if (!sws[i] || schwarz_mesh(sws[i]) != meshes[i])
            return fail(SEM_ERR_INVALID_ARG, "Schwarz object i must be built on meshes[i]");
    }
    if (o && o->coarse_iters < 0) return fail(SEM_ERR_INVALID_ARG, "coarse_iters < 0");
    return batched_impl(meshes, sws, nsolve, b, x, o, stats, scratch, scratch_bytes, stream);
}

}  // extern "C"
