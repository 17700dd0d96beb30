// sem_gs.cu -- gather-scatter (direct stiffness summation), scatter from the
// global numbering, and the unique-node inner product.
//
// Paper section 3.1: because the method is globally unstructured but locally
// structured, only a unit-depth exchange is needed -- the gather-scatter
// phase, which sums the contributions of all elements sharing a node (face,
// edge or corner) and hands the sum back to each copy.  Section 4.2 names it
// the communication kernel and the strong-scaling bottleneck.
//
// Data structure: "groups" = global nodes that have more than one local copy
// or lie on a Dirichlet face.  gs_off/gs_idx is a CSR list of the local
// indices of each group, ascending; groups [0, nmasked) are the Dirichlet
// ones.  Interior element nodes are never touched.  One thread per group sums
// its copies in ascending local index (deterministic; every copy receives
// bit-identical values) and writes the sum back.

#include <mutex>

#include "sem_common.cuh"

namespace sem {

template <typename T>
__global__ void gs_kernel(T *__restrict__ u, const int *__restrict__ off, const int *__restrict__ idx,
                          int64_t ngroups, int64_t nmasked, int mode, const int *__restrict__ guard, int gval) {
    if (guard && *guard != gval) return;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int a = off[g], b = off[g + 1];
        const bool masked = g < nmasked;
        if (masked && mode != kGsSum) {
            for (int q = a; q < b; ++q) u[idx[q]] = T(0);
        } else if (mode != kGsMaskOnly && b - a > 1) {
            T s = u[idx[a]];
            for (int q = a + 1; q < b; ++q) s += u[idx[q]];
            for (int q = a; q < b; ++q) u[idx[q]] = s;
        }
    }
}

int gs_launch(const sem_mesh *m, void *u, int dtype, int mode, cudaStream_t st, const int *guard, int gval) {
    const int64_t n = (mode == kGsMaskOnly) ? m->nmasked : m->ngroups;
    if (n == 0) return SEM_OK;
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)m->num_sms * 32) g = (int64_t)m->num_sms * 32;
    if (dtype == SEM_F64)
        gs_kernel<double><<<(int)g, 256, 0, st>>>(static_cast<double *>(u), m->gs_off, m->gs_idx, n,
                                                  m->nmasked, mode, guard, gval);
    else if (dtype == SEM_F32)
        gs_kernel<float><<<(int)g, 256, 0, st>>>(static_cast<float *>(u), m->gs_off, m->gs_idx, n,
                                                 m->nmasked, mode, guard, gval);
    else
        return fail(SEM_ERR_INVALID_ARG, "unknown dtype");
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

__global__ void scatter_kernel(const double *__restrict__ ug, double *__restrict__ ul, int64_t E, int N,
                               int nx, int ny, int64_t Gx, int64_t Gy, int64_t Gz, int px, int py, int pz) {
    const int n1 = N + 1;
    const int64_t npt = (int64_t)n1 * n1 * n1;
    const int64_t nloc = E * npt;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nloc;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = l / npt;
        const int p = (int)(l - e * npt);
        const int i = p % n1, j = (p / n1) % n1, k = p / (n1 * n1);
        const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
        int64_t I = ex * N + i, J = ey * N + j, K = ez * N + k;
        if (px && I >= Gx) I -= Gx;
        if (py && J >= Gy) J -= Gy;
        if (pz && K >= Gz) K -= Gz;
        ul[l] = ug[I + Gx * (J + Gy * K)];
    }
}

// Deterministic two-level reduction of sum_l a_l b_l w_l: fixed-size grid of
// block partials, summed in block order by the last block to finish.
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kRedThreads)
    glsc3_kernel(const double *__restrict__ a, const double *__restrict__ b, const double *__restrict__ w,
                 int64_t n, double *__restrict__ partial, unsigned *__restrict__ counter,
                 double *__restrict__ result) {
    __shared__ double sh[kRedThreads / 32];
    __shared__ bool last;
    double s = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[l] * b[l], w[l], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) {
            partial[blockIdx.x] = t;
            __threadfence();
            last = (atomicAdd(counter, 1u) == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t = 0.0;
        for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) t += partial[q];
        t = warp_sum(t);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
            for (int q = 0; q < kRedThreads / 32; ++q) r += sh[q];
            *result = r;
            *counter = 0u;
        }
    }
}

// ---- allocation-free inner product ------------------------------------
// Scratch of sem_glsc3_noalloc: the 1024 block partials and the arrival
// counter of glsc3_kernel, in a file-scope device array.  Every device that
// loads the library holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = 8448;  // 1024 doubles + counter, rounded to 256
static_assert(sizeof(double) * kRedBlocks + sizeof(unsigned) <= kNoAllocScratchBytes,
              "static scratch too small for the reduction");
static __device__ __align__(256) unsigned char g_glsc3_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static void *g_noalloc_addr[kNoAllocMaxDevices];  // device address of the array, per device
static std::mutex g_noalloc_mutex;

// The array's name is only a host-side stand-in; its device address must be
// looked up once per device with that device current.
static int noalloc_scratch_for_current_device(void **out) {
    int dev = 0;
    SEM_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SEM_ERR_UNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_glsc3_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_glsc3_noalloc_scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

int sem_dssum(const sem_mesh *m, void *u, int dtype, int apply_mask, void *stream) {
    if (!m || !u) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    return gs_launch(m, u, dtype, apply_mask ? kGsSumMask : kGsSum, as_stream(stream));
}

int sem_scatter(const sem_mesh *m, const double *ug, double *ul, void *stream) {
    if (!m || !ug || !ul) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    const int64_t Gx = (int64_t)m->nel[0] * m->N + (m->periodic[0] ? 0 : 1);
    const int64_t Gy = (int64_t)m->nel[1] * m->N + (m->periodic[1] ? 0 : 1);
    const int64_t Gz = (int64_t)m->nel[2] * m->N + (m->periodic[2] ? 0 : 1);
    int64_t g = (m->nloc + 255) / 256;
    if (g > (int64_t)m->num_sms * 64) g = (int64_t)m->num_sms * 64;
    scatter_kernel<<<(int)g, 256, 0, as_stream(stream)>>>(ug, ul, m->E, m->N, m->nel[0], m->nel[1], Gx, Gy, Gz,
                                                          m->periodic[0], m->periodic[1], m->periodic[2]);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int sem_glsc3(const sem_mesh *m, const double *a, const double *b, double *d_result, void *d_scratch,
              size_t scratch_bytes, void *stream) {
    if (!m || !a || !b || !d_result || !d_scratch) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    const size_t need = sizeof(double) * kRedBlocks + 64;
    if (scratch_bytes < need || (reinterpret_cast<uintptr_t>(d_scratch) % 16))
        return fail(SEM_ERR_WORKSPACE, "glsc3 scratch too small or misaligned");
    double *partial = static_cast<double *>(d_scratch);
    unsigned *counter = reinterpret_cast<unsigned *>(partial + kRedBlocks);
    cudaStream_t st = as_stream(stream);
    SEM_CUDA_CHECK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    glsc3_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(a, b, m->minv, m->nloc, partial, counter, d_result);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

// Same reduction as sem_glsc3, with its scratch in g_glsc3_noalloc_scratch
// instead of a caller buffer; no cudaMalloc, cudaFree or allocating library
// call.  The first call on a device looks up the array's device address.
int sem_glsc3_noalloc(const sem_mesh *m, const double *a, const double *b, double *d_result, void *stream) {
    if (!m || !a || !b || !d_result) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    const size_t need = sizeof(double) * kRedBlocks + sizeof(unsigned);
    if (need > kNoAllocScratchBytes)
        return fail(SEM_ERR_WORKSPACE, "sem_glsc3_noalloc: reduction needs " + std::to_string(need) +
                                           " bytes, static scratch holds " + std::to_string(kNoAllocScratchBytes));
    if (m->nloc >= (int64_t(1) << 31))
        return fail(SEM_ERR_INVALID_ARG, "sem_glsc3_noalloc: more than 2^31-1 points");
    void *scratch = nullptr;
    int s = noalloc_scratch_for_current_device(&scratch);
    if (s != SEM_OK) return s;
    double *partial = static_cast<double *>(scratch);
    unsigned *counter = reinterpret_cast<unsigned *>(partial + kRedBlocks);
    cudaStream_t st = as_stream(stream);
    // the counter must start at 0 (a previous call leaves it at 0, but a
    // call cut short would not): clear it every time
    SEM_CUDA_CHECK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    glsc3_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(a, b, m->minv, m->nloc, partial, counter, d_result);
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

}  // extern "C"
