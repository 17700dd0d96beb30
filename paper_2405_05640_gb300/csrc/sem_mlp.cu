// sem_mlp.cu -- element-local network for the learned initial guess of the
// pressure solve: training and inference on the tensor cores.
//
// Not from the paper (which has no learned component): a 3-layer MLP applied
// to every element independently,
//   H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3,
// loss L = (1/(2 R O)) sum (Y - T)^2 over the R real rows and O real outputs,
// gradients by the chain rule, Adam with bias correction.  All five weight
// and activation contractions run on sem_gemm_bf16 (tcgen05, BF16 operands,
// FP32 accumulation); the FP32 master parameters, gradients and Adam moments
// live in one flat array [W1, b1, W2, b2, W3, b3].
//
// The guess corrects the cubic extrapolation p_ext = 3 p1 - 3 p2 + p3 of the
// last three pressures; the sem_guess_* kernels at the end of this file form
// the residual r = b - A p_ext, the per-element features ((p1-p2), (p2-p3),
// r and the previous third difference, each with its own scale), the
// training target (p - p_ext)/se and the continuous guess p_ext + se Y.

#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "sem_common.cuh"

namespace sem {
int gemm_tn_bf16(const void *A, const void *B, int M, int N, int K, const float *bias, int act, float *c32,
                 void *c16, int ldc, int *d_err, cudaStream_t st, float *ws, size_t ws_floats);
}

struct sem_mlp {
    int I, H, O, R;
    size_t P, oW1, ob1, oW2, ob2, oW3, ob3;
    float *p, *g, *m, *v;
    __nv_bfloat16 *W1h, *W2h, *W3h, *W2t, *W3t;
    __nv_bfloat16 *XT, *H1, *H1T, *H2, *H2T, *dY, *dYT, *dA2, *dA2T, *dA1, *dA1T;
    float *Y, *dH2, *dH1;
    float *part;
    float *wsk;          // split-K partials of the weight-gradient GEMMs
    size_t wsk_floats;
    int *err;
    int t;
};

namespace sem {

using bf16 = __nv_bfloat16;
constexpr int kColChunks = 64;

__global__ void f32_to_bf16_kernel(const float *__restrict__ s, bf16 *__restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = __float2bfloat16_rn(s[i]);
}

// dst[c][r] = src[r][c] for src [rows x cols]; 32x32 tiles through shared memory.
template <typename TS, typename TD>
__global__ void transpose_kernel(const TS *__restrict__ src, TD *__restrict__ dst, int rows, int cols) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int r = r0 + q, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[q][threadIdx.x] = (float)src[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int c = c0 + q, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(size_t)c * rows + r] = (TD)tile[threadIdx.x][q];
    }
}

// dY = (Y - T)/(R_real O_real) on real rows/outputs (0 elsewhere, BF16);
// block partials of sum (Y - T)^2.
__global__ void loss_grad_kernel(const float *__restrict__ Y, const float *__restrict__ T, int rows, int outs,
                                 int rows_real, int outs_real, bf16 *__restrict__ dY, float *__restrict__ part) {
    __shared__ float sh[8];
    const float sc = 1.0f / ((float)rows_real * (float)outs_real);
    float acc = 0.f;
    const int64_t n = (int64_t)rows * outs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / outs), o = (int)(i - (int64_t)r * outs);
        float d = 0.f;
        if (r < rows_real && o < outs_real) d = Y[i] - T[i];
        acc = fmaf(d, d, acc);
        dY[i] = __float2bfloat16_rn(d * sc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        part[blockIdx.x] = t;
    }
}

__global__ void sum_partials_kernel(const float *__restrict__ part, int n, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < n; ++q) t += part[q];
        *out = t;
    }
}

// Energy-norm loss: delta = Y - T for the E elements (rows) and npt points
// (outputs) of a mesh, in the element-local layout [E][npt] of its fields.
__global__ void energy_delta_kernel(const float *__restrict__ Y, const float *__restrict__ T, int ld, int64_t E,
                                    int npt, float *__restrict__ D) {
    const int64_t n = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int q = (int)(l - e * npt);
        D[l] = Y[e * ld + q] - T[e * ld + q];
    }
}

// x *= w (FP32 by an FP32 weight)
__global__ void scale_f32_kernel(float *__restrict__ x, const float *__restrict__ w, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        x[l] *= w[l];
}

// K-norm pieces: g = A_L delta + lambda B delta (W = A_L delta, element by
// element); sum delta g into the block partials; g stays in W when
// `keep`, else dY = g / (E npt) (BF16) on real entries, 0 elsewhere.
__global__ void energy_grad_kernel(const float *__restrict__ D, float *__restrict__ W,
                                   const double *__restrict__ Bm, float lambda, int rows, int outs, int64_t E,
                                   int npt, bool keep, bf16 *__restrict__ dY, float *__restrict__ part) {
    __shared__ float sh[8];
    const float sc = 1.0f / ((float)E * (float)npt);
    float acc = 0.f;
    if (keep) {
        const int64_t n = E * npt;
        for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
             l += (int64_t)gridDim.x * blockDim.x) {
            const float d = D[l];
            const float g = fmaf(lambda * (float)Bm[l], d, W[l]);
            W[l] = g;
            acc = fmaf(d, g, acc);
        }
    } else {
        const int64_t n = (int64_t)rows * outs;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int r = (int)(i / outs), o = (int)(i - (int64_t)r * outs);
            float g = 0.f;
            if (r < E && o < npt) {
                const int64_t l = (int64_t)r * npt + o;
                const float d = D[l];
                g = fmaf(lambda * (float)Bm[l], d, W[l]);
                acc = fmaf(d, g, acc);
            }
            dY[i] = __float2bfloat16_rn(g * sc);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        part[blockIdx.x] = t;
    }
}

// dY = G / (E npt) (BF16) on real entries (G in the element layout), 0 elsewhere.
__global__ void energy_dy_kernel(const float *__restrict__ G, int rows, int outs, int64_t E, int npt,
                                 bf16 *__restrict__ dY) {
    const float sc = 1.0f / ((float)E * (float)npt);
    const int64_t n = (int64_t)rows * outs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / outs), o = (int)(i - (int64_t)r * outs);
        dY[i] = __float2bfloat16_rn(r < E && o < npt ? G[(int64_t)r * npt + o] * sc : 0.f);
    }
}

// dA = dH * (H > 0) (ReLU derivative from the post-activation), BF16
__global__ void relu_mask_kernel(const float *__restrict__ dH, const bf16 *__restrict__ H, bf16 *__restrict__ dA,
                                 int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dA[i] = __float2bfloat16_rn(__bfloat162float(H[i]) > 0.f ? dH[i] : 0.f);
}

// column sums of A [rows x cols] (BF16) in two deterministic passes
__global__ void colsum_partial_kernel(const bf16 *__restrict__ A, int rows, int cols, float *__restrict__ part) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    const int chunk = (rows + kColChunks - 1) / kColChunks;
    const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += __bfloat162float(A[(size_t)r * cols + c]);
    part[(size_t)blockIdx.y * cols + c] = s;
}

__global__ void colsum_final_kernel(const float *__restrict__ part, int cols, float *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int q = 0; q < kColChunks; ++q) s += part[(size_t)q * cols + c];
    out[c] = s;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static int gridn(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g));
}

template <typename TS, typename TD>
static void transpose(const TS *src, TD *dst, int rows, int cols, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_kernel<TS, TD><<<grid, block, 0, st>>>(src, dst, rows, cols);
}

static void colsum(const bf16 *A, int rows, int cols, float *part, float *out, cudaStream_t st) {
    dim3 grid((cols + 127) / 128, kColChunks);
    colsum_partial_kernel<<<grid, 128, 0, st>>>(A, rows, cols, part);
    colsum_final_kernel<<<(cols + 127) / 128, 128, 0, st>>>(part, cols, out);
}

// BF16 working copies of the weights (and the transposes the backward pass needs)
static int refresh_bf16(sem_mlp *n, cudaStream_t st) {
    f32_to_bf16_kernel<<<gridn((int64_t)n->H * n->I), 256, 0, st>>>(n->p + n->oW1, n->W1h, (int64_t)n->H * n->I);
    f32_to_bf16_kernel<<<gridn((int64_t)n->H * n->H), 256, 0, st>>>(n->p + n->oW2, n->W2h, (int64_t)n->H * n->H);
    f32_to_bf16_kernel<<<gridn((int64_t)n->O * n->H), 256, 0, st>>>(n->p + n->oW3, n->W3h, (int64_t)n->O * n->H);
    transpose<float, bf16>(n->p + n->oW2, n->W2t, n->H, n->H, st);
    transpose<float, bf16>(n->p + n->oW3, n->W3t, n->O, n->H, st);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

// Split-K work space of the weight-gradient GEMMs (M x N = O x H, H x H,
// H x I; K = the rows): up to 16 slices of the largest.
static size_t splitk_floats(int I, int H, int O) {
    size_t mn = (size_t)O * H;
    if ((size_t)H * H > mn) mn = (size_t)H * H;
    if ((size_t)H * I > mn) mn = (size_t)H * I;
    return 16 * mn;
}

static size_t mlp_bytes(int I, int H, int O, int R, size_t *P_out) {
    const size_t P = (size_t)H * I + H + (size_t)H * H + H + (size_t)O * H + O;
    if (P_out) *P_out = P;
    size_t b = 4 * align_up(4 * P);                                       // p, g, m, v
    b += align_up(2 * (size_t)H * I) + 2 * align_up(2 * (size_t)H * H) + 2 * align_up(2 * (size_t)O * H);
    b += align_up(2 * (size_t)I * R);                                     // XT
    b += 8 * align_up(2 * (size_t)R * H);                                 // H1 H1T H2 H2T dA2 dA2T dA1 dA1T
    b += 2 * align_up(2 * (size_t)R * O);                                 // dY dYT
    b += align_up(4 * (size_t)R * O) + 2 * align_up(4 * (size_t)R * H);  // Y dH2 dH1
    b += align_up(4 * ((size_t)kColChunks * (I > O ? (I > H ? I : H) : (O > H ? O : H)) + 4096));
    b += align_up(4 * splitk_floats(I, H, O));
    b += align_up(64);
    return b;
}

static int check_dims(int I, int H, int O, int R) {
    if (I <= 0 || H <= 0 || O <= 0 || R <= 0 || I % 128 || H % 128 || O % 128 || R % 128)
        return fail(SEM_ERR_INVALID_ARG, "network dimensions and rows must be positive multiples of 128");
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

size_t sem_mlp_workspace_bytes(int n_in, int n_hidden, int n_out, int max_rows) {
    if (check_dims(n_in, n_hidden, n_out, max_rows) != SEM_OK) return 0;
    return mlp_bytes(n_in, n_hidden, n_out, max_rows, nullptr);
}

int sem_mlp_create(int n_in, int n_hidden, int n_out, int max_rows, void *ws, size_t bytes, sem_mlp **out) {
    int s = check_dims(n_in, n_hidden, n_out, max_rows);
    if (s != SEM_OK) return s;
    if (!out) return fail(SEM_ERR_INVALID_ARG, "out is NULL");
    size_t P = 0;
    const size_t need = mlp_bytes(n_in, n_hidden, n_out, max_rows, &P);
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign || bytes < need)
        return fail(SEM_ERR_WORKSPACE, "MLP workspace NULL, misaligned or smaller than sem_mlp_workspace_bytes");
    sem_mlp *n = new sem_mlp();
    n->I = n_in;
    n->H = n_hidden;
    n->O = n_out;
    n->R = max_rows;
    n->P = P;
    n->oW1 = 0;
    n->ob1 = n->oW1 + (size_t)n->H * n->I;
    n->oW2 = n->ob1 + n->H;
    n->ob2 = n->oW2 + (size_t)n->H * n->H;
    n->oW3 = n->ob2 + n->H;
    n->ob3 = n->oW3 + (size_t)n->O * n->H;
    char *p = static_cast<char *>(ws);
    auto take = [&](size_t b) { char *q = p; p += align_up(b); return q; };
    n->p = reinterpret_cast<float *>(take(4 * P));
    n->g = reinterpret_cast<float *>(take(4 * P));
    n->m = reinterpret_cast<float *>(take(4 * P));
    n->v = reinterpret_cast<float *>(take(4 * P));
    n->W1h = reinterpret_cast<bf16 *>(take(2 * (size_t)n->H * n->I));
    n->W2h = reinterpret_cast<bf16 *>(take(2 * (size_t)n->H * n->H));
    n->W2t = reinterpret_cast<bf16 *>(take(2 * (size_t)n->H * n->H));
    n->W3h = reinterpret_cast<bf16 *>(take(2 * (size_t)n->O * n->H));
    n->W3t = reinterpret_cast<bf16 *>(take(2 * (size_t)n->O * n->H));
    n->XT = reinterpret_cast<bf16 *>(take(2 * (size_t)n->I * n->R));
    bf16 **acts[8] = {&n->H1, &n->H1T, &n->H2, &n->H2T, &n->dA2, &n->dA2T, &n->dA1, &n->dA1T};
    for (auto a : acts) *a = reinterpret_cast<bf16 *>(take(2 * (size_t)n->R * n->H));
    n->dY = reinterpret_cast<bf16 *>(take(2 * (size_t)n->R * n->O));
    n->dYT = reinterpret_cast<bf16 *>(take(2 * (size_t)n->R * n->O));
    n->Y = reinterpret_cast<float *>(take(4 * (size_t)n->R * n->O));
    n->dH2 = reinterpret_cast<float *>(take(4 * (size_t)n->R * n->H));
    n->dH1 = reinterpret_cast<float *>(take(4 * (size_t)n->R * n->H));
    const int wide = n->I > n->O ? (n->I > n->H ? n->I : n->H) : (n->O > n->H ? n->O : n->H);
    n->part = reinterpret_cast<float *>(take(4 * ((size_t)kColChunks * wide + 4096)));
    n->wsk_floats = splitk_floats(n_in, n_hidden, n_out);
    n->wsk = reinterpret_cast<float *>(take(4 * n->wsk_floats));
    n->err = reinterpret_cast<int *>(take(64));
    n->t = 0;
    cudaError_t e = cudaMemset(ws, 0, need);
    if (e != cudaSuccess) {
        delete n;
        return cuda_fail(e, "cudaMemset");
    }
    *out = n;
    return SEM_OK;
}

int sem_mlp_destroy(sem_mlp *n) {
    delete n;
    return SEM_OK;
}

size_t sem_mlp_num_params(const sem_mlp *n) { return n ? n->P : 0; }

int sem_mlp_set_params(sem_mlp *n, const float *host, void *stream) {
    if (!n || !host) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = as_stream(stream);
    SEM_CUDA_CHECK(cudaMemcpyAsync(n->p, host, 4 * n->P, cudaMemcpyHostToDevice, st));
    SEM_CUDA_CHECK(cudaMemsetAsync(n->m, 0, 4 * n->P, st));
    SEM_CUDA_CHECK(cudaMemsetAsync(n->v, 0, 4 * n->P, st));
    n->t = 0;
    int s = refresh_bf16(n, st);
    if (s != SEM_OK) return s;
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    return SEM_OK;
}

int sem_mlp_get_params(const sem_mlp *n, float *host, void *stream) {
    if (!n || !host) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = as_stream(stream);
    SEM_CUDA_CHECK(cudaMemcpyAsync(host, n->p, 4 * n->P, cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    return SEM_OK;
}

int sem_mlp_get_grads(const sem_mlp *n, float *host, void *stream) {
    if (!n || !host) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = as_stream(stream);
    SEM_CUDA_CHECK(cudaMemcpyAsync(host, n->g, 4 * n->P, cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    return SEM_OK;
}

static int fwd(sem_mlp *n, const void *X, int rows, cudaStream_t st) {
    int s = gemm_tn_bf16(X, n->W1h, rows, n->H, n->I, n->p + n->ob1, 1, nullptr, n->H1, n->H, n->err, st, nullptr, 0);
    if (s == SEM_OK) s = gemm_tn_bf16(n->H1, n->W2h, rows, n->H, n->H, n->p + n->ob2, 1, nullptr, n->H2, n->H, n->err, st, nullptr, 0);
    if (s == SEM_OK) s = gemm_tn_bf16(n->H2, n->W3h, rows, n->O, n->H, n->p + n->ob3, 0, n->Y, nullptr, n->O, n->err, st, nullptr, 0);
    return s;
}

int sem_mlp_forward(sem_mlp *n, const void *X, int rows, float *Y, void *stream) {
    NvtxRange nvtx_range("network forward");
    if (!n || !X || !Y) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (rows <= 0 || rows % 128 || rows > n->R) return fail(SEM_ERR_INVALID_ARG, "rows must be a multiple of 128, <= max_rows");
    cudaStream_t st = as_stream(stream);
    int s = fwd(n, X, rows, st);
    if (s != SEM_OK) return s;
    SEM_CUDA_CHECK(cudaMemcpyAsync(Y, n->Y, 4 * (size_t)rows * n->O, cudaMemcpyDeviceToDevice, st));
    return SEM_OK;
}

// Backward pass from the BF16 output gradient in n->dY: the weight and bias
// gradients into n->g.
static int mlp_backward(sem_mlp *n, const void *X, int R, cudaStream_t st) {
    const int I = n->I, H = n->H, O = n->O;
    // layer 3
    transpose<bf16, bf16>(n->dY, n->dYT, R, O, st);
    transpose<bf16, bf16>(n->H2, n->H2T, R, H, st);
    int s = gemm_tn_bf16(n->dYT, n->H2T, O, H, R, nullptr, 0, n->g + n->oW3, nullptr, H, n->err, st, n->wsk,
                         n->wsk_floats);
    if (s != SEM_OK) return s;
    colsum(n->dY, R, O, n->part, n->g + n->ob3, st);
    s = gemm_tn_bf16(n->dY, n->W3t, R, H, O, nullptr, 0, n->dH2, nullptr, H, n->err, st, nullptr, 0);
    if (s != SEM_OK) return s;
    relu_mask_kernel<<<gridn((int64_t)R * H), 256, 0, st>>>(n->dH2, n->H2, n->dA2, (int64_t)R * H);
    // layer 2
    transpose<bf16, bf16>(n->dA2, n->dA2T, R, H, st);
    transpose<bf16, bf16>(n->H1, n->H1T, R, H, st);
    s = gemm_tn_bf16(n->dA2T, n->H1T, H, H, R, nullptr, 0, n->g + n->oW2, nullptr, H, n->err, st, n->wsk,
                     n->wsk_floats);
    if (s != SEM_OK) return s;
    colsum(n->dA2, R, H, n->part, n->g + n->ob2, st);
    s = gemm_tn_bf16(n->dA2, n->W2t, R, H, H, nullptr, 0, n->dH1, nullptr, H, n->err, st, nullptr, 0);
    if (s != SEM_OK) return s;
    relu_mask_kernel<<<gridn((int64_t)R * H), 256, 0, st>>>(n->dH1, n->H1, n->dA1, (int64_t)R * H);
    // layer 1
    transpose<bf16, bf16>(n->dA1, n->dA1T, R, H, st);
    transpose<bf16, bf16>(static_cast<const bf16 *>(X), n->XT, R, I, st);
    s = gemm_tn_bf16(n->dA1T, n->XT, H, I, R, nullptr, 0, n->g + n->oW1, nullptr, I, n->err, st, n->wsk,
                     n->wsk_floats);
    if (s != SEM_OK) return s;
    colsum(n->dA1, R, H, n->part, n->g + n->ob1, st);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

// The loss sum (dloss, reduced from the partials before the backward pass
// reuses n->part) and the GEMMs' timeout flag, read after the pass:
// *loss = 0.5 sum / norm.
static int mlp_finish(sem_mlp *n, const double *dloss, double norm, double *loss, cudaStream_t st) {
    double h = 0.0;
    int herr = 0;
    SEM_CUDA_CHECK(cudaMemcpyAsync(&h, dloss, sizeof(double), cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaMemcpyAsync(&herr, n->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SEM_CUDA_CHECK(cudaStreamSynchronize(st));
    if (herr) return fail(SEM_ERR_TIMEOUT, "a GEMM wait timed out");
    *loss = 0.5 * h / norm;
    return SEM_OK;
}

int sem_mlp_grad(sem_mlp *n, const void *X, const float *T, int rows, int rows_real, int outs_real, double *loss,
                 void *stream) {
    NvtxRange nvtx_range("network forward + backward");
    if (!n || !X || !T || !loss) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (rows <= 0 || rows % 128 || rows > n->R || rows_real <= 0 || rows_real > rows || outs_real <= 0 ||
        outs_real > n->O)
        return fail(SEM_ERR_INVALID_ARG, "bad row / output counts");
    cudaStream_t st = as_stream(stream);
    int s = fwd(n, X, rows, st);
    if (s != SEM_OK) return s;
    const int lblocks = 1024;
    loss_grad_kernel<<<lblocks, 256, 0, st>>>(n->Y, T, rows, n->O, rows_real, outs_real, n->dY, n->part);
    double *dloss = reinterpret_cast<double *>(n->err + 8);
    sum_partials_kernel<<<1, 32, 0, st>>>(n->part, lblocks, dloss);
    s = mlp_backward(n, X, rows, st);
    if (s != SEM_OK) return s;
    return mlp_finish(n, dloss, (double)rows_real * outs_real, loss, st);
}

int sem_mlp_grad_energy(sem_mlp *n, const sem_mesh *m, const void *X, const float *T, int rows, double lambda,
                        int assembled, float *work, size_t work_floats, double *loss, void *stream) {
    NvtxRange nvtx_range("network forward + backward (energy norm)");
    if (!n || !m || !X || !T || !work || !loss) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (rows <= 0 || rows % 128 || rows > n->R || m->E > rows || m->npt > n->O)
        return fail(SEM_ERR_INVALID_ARG, "rows must be a multiple of 128 with E <= rows <= max_rows, npt <= n_out");
    if (!m->G32) return fail(SEM_ERR_INVALID_ARG, "the energy norm needs a mesh built with SEM_GEOM_F32");
    if (!(lambda >= 0.0)) return fail(SEM_ERR_INVALID_ARG, "lambda must be >= 0");
    if (work_floats < 2 * (size_t)m->nloc) return fail(SEM_ERR_WORKSPACE, "work holds fewer than 2 nloc floats");
    cudaStream_t st = as_stream(stream);
    int s = fwd(n, X, rows, st);
    if (s != SEM_OK) return s;
    float *D = work, *W = work + m->nloc;
    energy_delta_kernel<<<gridn(m->nloc), 256, 0, st>>>(n->Y, T, n->O, m->E, m->npt, D);
    SEM_CUDA_CHECK(cudaGetLastError());
    if (assembled) {
        // the averaged correction's error: D <- M^-1 S D (S: sum of the copies)
        s = gs_launch(m, D, SEM_F32, kGsSum, st);
        if (s != SEM_OK) return s;
        scale_f32_kernel<<<gridn(m->nloc), 256, 0, st>>>(D, m->minv32, m->nloc);
    }
    s = ax_launch_f32(m, D, W, st);
    if (s != SEM_OK) return s;
    const int lblocks = 1024;
    energy_grad_kernel<<<lblocks, 256, 0, st>>>(D, W, m->B, (float)lambda, rows, n->O, m->E, m->npt, assembled != 0,
                                                n->dY, n->part);
    double *dloss = reinterpret_cast<double *>(n->err + 8);
    sum_partials_kernel<<<1, 32, 0, st>>>(n->part, lblocks, dloss);
    if (assembled) {
        // gradient S M^-1 (A_L + lambda B) M^-1 S delta
        scale_f32_kernel<<<gridn(m->nloc), 256, 0, st>>>(W, m->minv32, m->nloc);
        s = gs_launch(m, W, SEM_F32, kGsSum, st);
        if (s != SEM_OK) return s;
        energy_dy_kernel<<<gridn((int64_t)rows * n->O), 256, 0, st>>>(W, rows, n->O, m->E, m->npt, n->dY);
    }
    SEM_CUDA_CHECK(cudaGetLastError());
    s = mlp_backward(n, X, rows, st);
    if (s != SEM_OK) return s;
    return mlp_finish(n, dloss, (double)m->E * m->npt, loss, st);
}

int sem_mlp_adam(sem_mlp *n, double lr, double beta1, double beta2, double eps, void *stream) {
    if (!n) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = as_stream(stream);
    n->t += 1;
    const float c1 = (float)(1.0 - std::pow(beta1, n->t)), c2 = (float)(1.0 - std::pow(beta2, n->t));
    adam_kernel<<<gridn((int64_t)n->P), 256, 0, st>>>(n->p, n->g, n->m, n->v, (int64_t)n->P, (float)lr, (float)beta1,
                                                     (float)beta2, (float)eps, c1, c2);
    SEM_CUDA_CHECK(cudaGetLastError());
    return refresh_bf16(n, st);
}

}  // extern "C"

// ---------------------------------------------------------------- guess features

namespace sem {

// X[e][q], q < 4 npt: (p1 - p2)/sd, (p2 - p3)/sd, r/sr and
// (p1 - 3 p2 + 3 p3 - p4)/s3 (p1/s3 when p4 is null) of element e; columns
// beyond 4 npt are left as they are (zero from the caller).
__global__ void guess_features_kernel(const double *__restrict__ p1, const double *__restrict__ p2,
                                      const double *__restrict__ p3, const double *__restrict__ p4,
                                      const double *__restrict__ r, int64_t E, int npt, double isd, double isr,
                                      double is3, bf16 *__restrict__ X, int ldx) {
    const int64_t n = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int q = (int)(l - e * npt);
        bf16 *row = X + e * ldx;
        row[q] = __float2bfloat16_rn((float)((p1[l] - p2[l]) * isd));
        row[npt + q] = __float2bfloat16_rn((float)((p2[l] - p3[l]) * isd));
        row[2 * npt + q] = __float2bfloat16_rn((float)(r[l] * isr));
        const double f4 = p4 ? p1[l] - 3.0 * p2[l] + 3.0 * p3[l] - p4[l] : p1[l];
        row[3 * npt + q] = __float2bfloat16_rn((float)(f4 * is3));
    }
}

__global__ void extrap_kernel(const double *__restrict__ p1, const double *__restrict__ p2,
                              const double *__restrict__ p3, int64_t n, double *__restrict__ out) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        out[l] = 3.0 * p1[l] - 3.0 * p2[l] + p3[l];
}

__global__ void sub_kernel(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                           double *__restrict__ out) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        out[l] = a[l] - b[l];
}

// T[e][q] = (p - (3 p1 - 3 p2 + p3)) / pscale
__global__ void guess_target_kernel(const double *__restrict__ p, const double *__restrict__ p1,
                                    const double *__restrict__ p2, const double *__restrict__ p3, int64_t E, int npt,
                                    double ips, float *__restrict__ T, int ldt) {
    const int64_t n = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int q = (int)(l - e * npt);
        T[e * ldt + q] = (float)((p[l] - (3.0 * p1[l] - 3.0 * p2[l] + p3[l])) * ips);
    }
}

// guess (local) = (3 p1 - 3 p2 + p3) + pscale * Y  (before averaging)
__global__ void guess_apply_kernel(const float *__restrict__ Y, int ldy, const double *__restrict__ p1,
                                   const double *__restrict__ p2, const double *__restrict__ p3, int64_t E, int npt,
                                   double ps, double *__restrict__ g) {
    const int64_t n = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int q = (int)(l - e * npt);
        g[l] = 3.0 * p1[l] - 3.0 * p2[l] + p3[l] + ps * (double)Y[e * ldy + q];
    }
}

__global__ void scale_by_kernel(double *__restrict__ g, const double *__restrict__ w, int64_t n) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        g[l] *= w[l];
}

}  // namespace sem

extern "C" {

static int guess_residual(const sem_mesh *m, const double *b, const double *p1, const double *p2, const double *p3,
                          double *r, double *work, bool pair, void *stream) {
    if (!m || !b || !p1 || !p2 || !p3 || !r || !work || r == work) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (pair && !m->G2) return fail(SEM_ERR_INVALID_ARG, "the FP32-pair operator needs a mesh built with SEM_GEOM_PAIR");
    cudaStream_t st = as_stream(stream);
    extrap_kernel<<<gridn(m->nloc), 256, 0, st>>>(p1, p2, p3, m->nloc, work);
    SEM_CUDA_CHECK(cudaGetLastError());
    int s = pair ? ax_launch_pair(m, work, r, st) : ax_launch_f64(m, work, r, 1.0, 0.0, st);
    if (s != SEM_OK) return s;
    s = gs_launch(m, r, SEM_F64, kGsSumMask, st);
    if (s != SEM_OK) return s;
    sub_kernel<<<gridn(m->nloc), 256, 0, st>>>(b, r, m->nloc, r);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int sem_guess_residual(const sem_mesh *m, const double *b, const double *p1, const double *p2, const double *p3,
                       double *r, double *work, void *stream) {
    return guess_residual(m, b, p1, p2, p3, r, work, false, stream);
}

int sem_guess_residual_pair(const sem_mesh *m, const double *b, const double *p1, const double *p2,
                            const double *p3, double *r, double *work, void *stream) {
    return guess_residual(m, b, p1, p2, p3, r, work, true, stream);
}

int sem_guess_features(const sem_mesh *m, const double *p1, const double *p2, const double *p3, const double *p4,
                       const double *r, double sd, double sr, double s3, void *X, int ldx, void *stream) {
    if (!m || !p1 || !p2 || !p3 || !r || !X) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (ldx < 4 * m->npt || !(sd > 0) || !(sr > 0) || !(s3 > 0))
        return fail(SEM_ERR_INVALID_ARG, "ldx < 4 npt or a scale <= 0");
    guess_features_kernel<<<gridn(m->nloc), 256, 0, as_stream(stream)>>>(
        p1, p2, p3, p4, r, m->E, m->npt, 1.0 / sd, 1.0 / sr, 1.0 / s3, static_cast<bf16 *>(X), ldx);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int sem_guess_target(const sem_mesh *m, const double *p, const double *p1, const double *p2, const double *p3,
                     double pscale, float *T, int ldt, void *stream) {
    if (!m || !p || !p1 || !p2 || !p3 || !T) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (ldt < m->npt || !(pscale > 0)) return fail(SEM_ERR_INVALID_ARG, "ldt < npt or scale <= 0");
    guess_target_kernel<<<gridn(m->nloc), 256, 0, as_stream(stream)>>>(p, p1, p2, p3, m->E, m->npt, 1.0 / pscale, T, ldt);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int sem_guess_apply(const sem_mesh *m, const float *Y, int ldy, const double *p1, const double *p2, const double *p3,
                    double pscale, double *guess, void *stream) {
    if (!m || !Y || !p1 || !p2 || !p3 || !guess) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (ldy < m->npt) return fail(SEM_ERR_INVALID_ARG, "ldy < npt");
    cudaStream_t st = as_stream(stream);
    guess_apply_kernel<<<gridn(m->nloc), 256, 0, st>>>(Y, ldy, p1, p2, p3, m->E, m->npt, pscale, guess);
    SEM_CUDA_CHECK(cudaGetLastError());
    // continuous: average the copies of every node (Q Q^T g / mult)
    int s = gs_launch(m, guess, SEM_F64, kGsSum, st);
    if (s != SEM_OK) return s;
    scale_by_kernel<<<gridn(m->nloc), 256, 0, st>>>(guess, m->minv, m->nloc);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

}  // extern "C"
