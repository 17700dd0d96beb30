// sem_gmres.cu -- flexible restarted GMRES as the FP32 inner solver of the
// mixed-precision pressure solve.
//
// The paper's pressure solver is restarted GMRES with a hybrid-Schwarz
// multigrid preconditioner (Sec. 3.1).  Here one GMRES cycle is one
// refinement round of the mixed solver: the cycle solves A d = r / ||r||
// in FP32 from d = 0 (r: the FP64 outer residual) with right preconditioning
// that may change from one iteration to the next (flexible: the
// preconditioned directions z_j are kept, d = Z y), and the next round
// restarts from the FP64 true residual -- the restart is the refinement.
//
// Arnoldi in the multiplicity-weighted inner product (sum over unique
// nodes), classical Gram-Schmidt: the projections of w = A z_j on all basis
// vectors come from one fused multi-dot pass and are removed in one fused
// update pass that also forms ||w'||; a second pass is made only when the
// first cancelled all but 1 % of ||w|| (decided on the device): a single
// pass keeps the FP32 basis orthogonal well below the inner tolerance
// otherwise, and a second one on every column would double the traffic
// over the basis.  Givens rotations, the convergence
// test on the Arnoldi residual estimate |g_{j+1}| and the back substitution
// run in single-thread kernels; the host only launches and, every `check`
// iterations, reads the state.  Every kernel of an iteration is a no-op once
// the cycle is done, so a batch of launched iterations may overrun the
// convergence point.

#include <cmath>

#include "sem_common.cuh"

namespace sem {

constexpr int kGmThreads = 256;
constexpr int kGmBlocks = 152 * 8;  // fixed: the reduction order is fixed
constexpr int kGmGroup = 8;         // basis vectors per multi-dot block

struct GmState {
    double H[(kGmMaxRestart + 1) * kGmMaxRestart];  // H[i + (kGmMaxRestart + 1) j]
    double cs[kGmMaxRestart], sn[kGmMaxRestart], g[kGmMaxRestart + 1], y[kGmMaxRestart];
    double h[kGmMaxRestart + 1];   // projections of this column (both passes)
    double hp[kGmMaxRestart + 1];  // projections of the current pass
    double ww, wn2, beta, tol, inv;
    int j, done, conv, reorth, iter, status;
};

struct GmWork {
    GmState *S;
    double *partial;  // [kGmMaxRestart + 2][kGmBlocks]
    float *V, *Z, *w;
    size_t ldv;       // floats between consecutive basis vectors
};

static size_t vec_floats(const sem_mesh *m) { return align_up(sizeof(float) * m->nloc) / sizeof(float); }

size_t gmres_work_bytes(const sem_mesh *m, int restart) {
    const size_t vf = align_up(sizeof(float) * m->nloc);
    return align_up(sizeof(GmState)) + align_up(sizeof(double) * (kGmMaxRestart + 2) * kGmBlocks) +
           vf * (2 * (size_t)restart + 2);
}

static GmWork carve(const sem_mesh *m, int restart, void *work) {
    char *p = static_cast<char *>(work);
    GmWork W;
    W.S = reinterpret_cast<GmState *>(p);
    p += align_up(sizeof(GmState));
    W.partial = reinterpret_cast<double *>(p);
    p += align_up(sizeof(double) * (kGmMaxRestart + 2) * kGmBlocks);
    W.ldv = vec_floats(m);
    W.V = reinterpret_cast<float *>(p);
    W.Z = W.V + (size_t)(restart + 1) * W.ldv;
    W.w = W.Z + (size_t)restart * W.ldv;
    return W;
}

// Block sums of K doubles per thread: thread k < K writes sum k to out[k * stride].
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *out, int stride) {
    __shared__ double sh[kGmThreads / 32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int q = 0; q < kGmThreads / 32; ++q) t += sh[q][threadIdx.x];
        out[threadIdx.x * (size_t)stride] = t;
    }
    __syncthreads();
}

// Sum of one row of block partials by a whole block (thread-strided, then a
// fixed tree): the same order every call.
__device__ __forceinline__ double row_sum(const double *__restrict__ row) {
    __shared__ double sh[kGmThreads / 32];
    double t = 0.0;
    for (int b = threadIdx.x; b < kGmBlocks; b += blockDim.x) t += row[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < kGmThreads / 32; ++q) r += sh[q];
    return r;  // valid on thread 0
}

// ---- cycle start: v_0 = (float)(r64 * scale) / beta ----

__global__ void __launch_bounds__(kGmThreads)
    gm_start_kernel(const double *__restrict__ r64, const PcgScal *__restrict__ so, const float *__restrict__ minv,
                    int64_t n, float *__restrict__ v0, double *__restrict__ partial) {
    const double sc = so->scale;
    float f = 0.f;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)(r64[l] * sc);
        v0[l] = v;
        f = fmaf(v * v, minv[l], f);
    }
    double d[1] = {(double)f};
    block_sum<1>(d, partial + blockIdx.x, kGmBlocks);
}

__global__ void __launch_bounds__(kGmThreads)
    gm_start_finish_kernel(GmState *S, const double *__restrict__ partial, const PcgScal *__restrict__ so,
                           double delta, double theta) {
    const double t = row_sum(partial);
    if (threadIdx.x != 0) return;
    const double beta = sqrt(t);
    S->beta = beta;
    S->g[0] = beta;
    S->j = 0;
    S->iter = 0;
    S->reorth = 0;
    S->conv = 0;
    S->tol = inner_delta(so, delta, theta) * beta;
    S->inv = beta > 0.0 ? 1.0 / beta : 0.0;
    S->status = isfinite(beta) ? SEM_OK : SEM_ERR_NAN;
    S->done = (beta > 0.0 && isfinite(beta)) ? 0 : 1;
    if (beta == 0.0) S->conv = 1;
}

// v *= S->inv (the new basis vector); guard: cycle not done.
__global__ void __launch_bounds__(kGmThreads)
    gm_scale_kernel(float *__restrict__ v, const float *__restrict__ src, int64_t n, const GmState *__restrict__ S) {
    if (S->done) return;
    const float s = (float)S->inv;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        v[l] = src[l] * s;
}

// Jacobi preconditioner z = dinv v; guard: cycle not done.
__global__ void __launch_bounds__(kGmThreads)
    gm_jacobi_kernel(const float *__restrict__ v, const float *__restrict__ dinv, int64_t n, float *__restrict__ z,
                     const GmState *__restrict__ S) {
    if (S->done) return;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        z[l] = dinv[l] * v[l];
}


// ---- Gram-Schmidt passes ----

// Partials of <w, v_i> (i < nv, weighted by minv) and, in pass 0, <w, w>:
// block (x, y) covers basis vectors 8y .. 8y + 7.  Four points per thread
// and load (float4; the vectors start on 16-byte boundaries), the ragged
// tail (nloc % 4) one by one.  pass 0 runs while the
// cycle is not done, pass 1 only when a second pass was asked for.
__global__ void __launch_bounds__(kGmThreads)
    gm_mdot_kernel(const float *__restrict__ w, const float *__restrict__ V, size_t ldv, int nv,
                   const float *__restrict__ minv, int64_t n, double *__restrict__ partial,
                   const GmState *__restrict__ S, int pass) {
    if (pass == 0 ? S->done != 0 : S->reorth == 0) return;
    const int g0 = blockIdx.y * kGmGroup;
    const int kn = nv - g0 < kGmGroup ? nv - g0 : kGmGroup;
    float acc[kGmGroup + 1];
#pragma unroll
    for (int k = 0; k <= kGmGroup; ++k) acc[k] = 0.f;
    const int64_t n4 = n >> 2;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    const float4 *w4 = reinterpret_cast<const float4 *>(w), *m4 = reinterpret_cast<const float4 *>(minv);
    for (int64_t q = tid; q < n4; q += nth) {
        const float4 wv = w4[q], mv = m4[q];
        const float4 wm = make_float4(wv.x * mv.x, wv.y * mv.y, wv.z * mv.z, wv.w * mv.w);
#pragma unroll
        for (int k = 0; k < kGmGroup; ++k)
            if (k < kn) {
                const float4 v = reinterpret_cast<const float4 *>(V + (size_t)(g0 + k) * ldv)[q];
                acc[k] = fmaf(wm.x, v.x, fmaf(wm.y, v.y, fmaf(wm.z, v.z, fmaf(wm.w, v.w, acc[k]))));
            }
        acc[kGmGroup] = fmaf(wm.x, wv.x, fmaf(wm.y, wv.y, fmaf(wm.z, wv.z, fmaf(wm.w, wv.w, acc[kGmGroup]))));
    }
    for (int64_t l = 4 * n4 + tid; l < n; l += nth) {
        const float wv = w[l], wm = wv * minv[l];
#pragma unroll
        for (int k = 0; k < kGmGroup; ++k)
            if (k < kn) acc[k] = fmaf(wm, V[(size_t)(g0 + k) * ldv + l], acc[k]);
        acc[kGmGroup] = fmaf(wm, wv, acc[kGmGroup]);
    }
    __shared__ double sh[kGmThreads / 32][kGmGroup + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k <= kGmGroup; ++k) {
        double x = (double)acc[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x <= kGmGroup) {
        double t = 0.0;
        for (int q = 0; q < kGmThreads / 32; ++q) t += sh[q][threadIdx.x];
        const int k = threadIdx.x;
        if (k < kGmGroup && g0 + k < nv) partial[(size_t)(g0 + k) * kGmBlocks + blockIdx.x] = t;
        if (k == kGmGroup && blockIdx.y == 0) partial[(size_t)(kGmMaxRestart + 1) * kGmBlocks + blockIdx.x] = t;
    }
}

// w <- w - sum_i hp_i v_i (i < nv); partial of ||w||^2 (weighted) in slot 0.
__global__ void __launch_bounds__(kGmThreads)
    gm_update_kernel(float *__restrict__ w, const float *__restrict__ V, size_t ldv, int nv,
                     const float *__restrict__ minv, int64_t n, double *__restrict__ partial,
                     const GmState *__restrict__ S, int pass) {
    if (pass == 0 ? S->done != 0 : S->reorth == 0) return;
    __shared__ float hs[kGmMaxRestart + 1];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = (float)S->hp[i];
    __syncthreads();
    float f = 0.f;
    const int64_t n4 = n >> 2;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    float4 *w4 = reinterpret_cast<float4 *>(w);
    const float4 *m4 = reinterpret_cast<const float4 *>(minv);
    for (int64_t q = tid; q < n4; q += nth) {
        float4 x = w4[q];
#pragma unroll 4
        for (int i = 0; i < nv; ++i) {
            const float4 v = reinterpret_cast<const float4 *>(V + (size_t)i * ldv)[q];
            const float h = -hs[i];
            x.x = fmaf(h, v.x, x.x);
            x.y = fmaf(h, v.y, x.y);
            x.z = fmaf(h, v.z, x.z);
            x.w = fmaf(h, v.w, x.w);
        }
        w4[q] = x;
        const float4 mv = m4[q];
        f = fmaf(x.x * x.x, mv.x, fmaf(x.y * x.y, mv.y, fmaf(x.z * x.z, mv.z, fmaf(x.w * x.w, mv.w, f))));
    }
    for (int64_t l = 4 * n4 + tid; l < n; l += nth) {
        float x = w[l];
        for (int i = 0; i < nv; ++i) x = fmaf(-hs[i], V[(size_t)i * ldv + l], x);
        w[l] = x;
        f = fmaf(x * x, minv[l], f);
    }
    double d[1] = {(double)f};
    block_sum<1>(d, partial + blockIdx.x, kGmBlocks);
}

// Sums of the partials, one block per row, in a fixed order.  mode 0 (after
// the first multi-dot; nv + 1 blocks): hp = h = the projections, ww =
// ||w||^2; mode 1 (after the first update; 1 block): wn2 = ||w'||^2, ask for
// a second pass when all but 1 % of ||w|| was cancelled (wn2 < 1e-4 ww);
// mode 2 (second multi-dot; nv blocks): hp = the new projections, h += hp;
// mode 3 (second update; 1 block): wn2, no more passes.
__global__ void __launch_bounds__(kGmThreads)
    gm_reduce_kernel(const double *__restrict__ partial, int nv, GmState *S, int mode) {
    if (mode <= 1 ? S->done != 0 : S->reorth == 0) return;
    const int i = blockIdx.x;
    const bool proj = mode == 0 || mode == 2;
    const int row = proj ? (i < nv ? i : kGmMaxRestart + 1) : 0;
    const double t = row_sum(partial + (size_t)row * kGmBlocks);
    if (threadIdx.x != 0) return;
    if (proj) {
        if (i < nv) {
            S->hp[i] = t;
            S->h[i] = mode == 0 ? t : S->h[i] + t;
        } else {
            S->ww = t;
        }
    } else {
        S->wn2 = t;
        S->reorth = mode == 1 ? (t < 1e-4 * S->ww ? 1 : 0) : 0;
    }
}

// Column j of the Hessenberg matrix, the previous Givens rotations applied
// to it, its own rotation, the residual estimate |g_{j+1}|; the cycle is done
// when it meets the tolerance, on breakdown (the Krylov space is invariant:
// the least-squares solution is exact), or at the restart length.
__global__ void gm_finish_kernel(GmState *S, int restart) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || S->done) return;
    constexpr int L = kGmMaxRestart + 1;
    const int j = S->j;
    double *Hc = S->H + (size_t)L * j;
    for (int i = 0; i <= j; ++i) Hc[i] = S->h[i];
    const double hn = sqrt(fmax(S->wn2, 0.0));
    Hc[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = S->cs[i] * Hc[i] + S->sn[i] * Hc[i + 1];
        Hc[i + 1] = -S->sn[i] * Hc[i] + S->cs[i] * Hc[i + 1];
        Hc[i] = a;
    }
    const double dd = hypot(Hc[j], hn);
    const double c = dd > 0.0 ? Hc[j] / dd : 1.0, sgn = dd > 0.0 ? hn / dd : 0.0;
    S->cs[j] = c;
    S->sn[j] = sgn;
    Hc[j] = dd;
    Hc[j + 1] = 0.0;
    S->g[j + 1] = -sgn * S->g[j];
    S->g[j] = c * S->g[j];
    S->j = j + 1;
    S->iter += 1;
    S->inv = hn > 0.0 ? 1.0 / hn : 0.0;
    const double res = fabs(S->g[j + 1]);
    if (!isfinite(dd) || !isfinite(res)) {
        S->status = SEM_ERR_NAN;
        S->done = 1;
    } else if (res <= S->tol || hn == 0.0) {
        S->conv = 1;
        S->done = 1;
    } else if (j + 1 >= restart) {
        S->done = 1;
    }
}

// y from the triangular system R y = g (k = S->j columns).
__global__ void gm_solve_kernel(GmState *S) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    constexpr int L = kGmMaxRestart + 1;
    const int k = S->j;
    const bool bad = S->status != SEM_OK;
    for (int i = k - 1; i >= 0; --i) {
        double t = S->g[i];
        for (int c = i + 1; c < k; ++c) t -= S->H[(size_t)L * c + i] * S->y[c];
        const double dii = S->H[(size_t)L * i + i];
        S->y[i] = (bad || dii == 0.0) ? 0.0 : t / dii;
    }
}

// d = sum_{i < k} y_i z_i.
__global__ void __launch_bounds__(kGmThreads)
    gm_combine_kernel(const float *__restrict__ Z, size_t ldv, int64_t n, const GmState *__restrict__ S,
                      float *__restrict__ d) {
    __shared__ float ys[kGmMaxRestart];
    const int k = S->j;
    for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = (float)S->y[i];
    __syncthreads();
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        float x = 0.f;
        for (int i = 0; i < k; ++i) x = fmaf(ys[i], Z[(size_t)i * ldv + l], x);
        d[l] = x;
    }
}


// ---- host: one cycle ----

static int gm_iteration(const sem_mesh *m, const GmWork &W, int jj, const GmresArgs &a, cudaStream_t st,
                        int *launches) {
    const int64_t n = m->nloc;
    const float *vj = W.V + (size_t)jj * W.ldv;
    float *zj = W.Z + (size_t)jj * W.ldv;
    float *vn = W.V + (size_t)(jj + 1) * W.ldv;
    const int *done = &W.S->done;
    const int nv = jj + 1;
    int s;
    if (a.sw) {
        s = schwarz_apply_f32(a.sw, vj, zj, a.coarse_iters, a.coarse_tol, done, st);
        if (s != SEM_OK) return s;
        if (a.mid) {
            s = schwarz_mid_apply_add(a.sw, a.mid, a.mid_w, vj, zj, a.mid_work, done, st);
            if (s != SEM_OK) return s;
        }
    } else {
        gm_jacobi_kernel<<<kGmBlocks, kGmThreads, 0, st>>>(vj, m->dinv32, n, zj, W.S);
    }
    s = ax_launch_f32(m, zj, W.w, st, done, 0);
    if (s != SEM_OK) return s;
    s = gs_launch(m, W.w, SEM_F32, kGsSumMask, st, done, 0);
    if (s != SEM_OK) return s;
    const dim3 mgrid(kGmBlocks, (nv + kGmGroup - 1) / kGmGroup);
    for (int pass = 0; pass < 2; ++pass) {
        gm_mdot_kernel<<<mgrid, kGmThreads, 0, st>>>(W.w, W.V, W.ldv, nv, m->minv32, n, W.partial, W.S, pass);
        gm_reduce_kernel<<<pass == 0 ? nv + 1 : nv, kGmThreads, 0, st>>>(W.partial, nv, W.S, 2 * pass);
        gm_update_kernel<<<kGmBlocks, kGmThreads, 0, st>>>(W.w, W.V, W.ldv, nv, m->minv32, n, W.partial, W.S, pass);
        gm_reduce_kernel<<<1, kGmThreads, 0, st>>>(W.partial, nv, W.S, 2 * pass + 1);
    }
    gm_finish_kernel<<<1, 32, 0, st>>>(W.S, a.restart);
    gm_scale_kernel<<<kGmBlocks, kGmThreads, 0, st>>>(vn, W.w, n, W.S);
    SEM_CUDA_CHECK(cudaGetLastError());
    *launches += 13;
    return SEM_OK;
}

int gmres_cycle(const sem_mesh *m, const double *r64, const PcgScal *so, float *d, const GmresArgs &a, void *work,
                cudaStream_t st, GmresResult *out) {
    NvtxRange nvtx_range("GMRES cycle");
    if (a.restart < 1 || a.restart > kGmMaxRestart) return fail(SEM_ERR_INVALID_ARG, "restart outside [1, 128]");
    const int64_t n = m->nloc;
    GmWork W = carve(m, a.restart, work);
    gm_start_kernel<<<kGmBlocks, kGmThreads, 0, st>>>(r64, so, m->minv32, n, W.V, W.partial);
    gm_start_finish_kernel<<<1, kGmThreads, 0, st>>>(W.S, W.partial, so, a.delta, a.theta);
    gm_scale_kernel<<<kGmBlocks, kGmThreads, 0, st>>>(W.V, W.V, n, W.S);
    SEM_CUDA_CHECK(cudaGetLastError());
    int launches = 3, launched = 0;
    const int check = a.check > 0 ? a.check : 8;
    struct Tail {
        int j, done, conv, reorth, iter, status;
    } h{};
    while (true) {
        for (int q = 0; q < check && launched < a.restart && launched < a.max_iter; ++q, ++launched) {
            int s = gm_iteration(m, W, launched, a, st, &launches);
            if (s != SEM_OK) return s;
        }
        SEM_CUDA_CHECK(cudaMemcpyAsync(&h, &W.S->j, sizeof(Tail), cudaMemcpyDeviceToHost, st));
        SEM_CUDA_CHECK(cudaStreamSynchronize(st));
        if (h.done || launched >= a.restart || launched >= a.max_iter) break;
    }
    gm_solve_kernel<<<1, 32, 0, st>>>(W.S);
    gm_combine_kernel<<<kGmBlocks, kGmThreads, 0, st>>>(W.Z, W.ldv, n, W.S, d);
    SEM_CUDA_CHECK(cudaGetLastError());
    out->iters = h.iter;
    out->converged = h.conv;
    out->status = h.status;
    out->launches = launches + 2;
    out->ax_launches = launched;
    return SEM_OK;
}

}  // namespace sem
