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
// or lie on a Dirichlet face, stored by size in four buckets (2^b copies in
// bucket b; size 1 only for masked nodes), the local indices of each group
// ascending, each bucket's Dirichlet groups first.  Interior element nodes are
// never touched.  One thread per group: it loads the group's indices with one
// vector load (int2 / int4 / two int4), all copies at once, sums them in
// ascending local index (deterministic; every copy receives bit-identical
// values) and writes the sum back -- two dependent memory levels.

#include <mutex>

#include "sem_common.cuh"

namespace sem {

struct GsPlan {
    const int *idx;
    int64_t start[4];  // first int of bucket b
    int64_t nm[4];     // masked groups at the head of bucket b
    int64_t t0[5];     // bucket b's groups [0, t0[b+1] - t0[b]) run on threads [t0[b], t0[b+1])
};

template <typename T>
__global__ void __launch_bounds__(256)
    gs_kernel(T *__restrict__ u, GsPlan P, int mode, const int *__restrict__ guard, int gval) {
    if (guard && *guard != gval) return;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= P.t0[4]) return;
    const bool zero_masked = mode != kGsSum;
    if (t < P.t0[1]) {  // single copies: always Dirichlet
        u[P.idx[P.start[0] + (t - P.t0[0])]] = T(0);
    } else if (t < P.t0[2]) {
        const int64_t g = t - P.t0[1];
        const int2 q = *reinterpret_cast<const int2 *>(P.idx + P.start[1] + 2 * g);
        if (zero_masked && g < P.nm[1]) {
            u[q.x] = T(0);
            u[q.y] = T(0);
        } else {
            const T a0 = u[q.x], a1 = u[q.y];
            const T s = a0 + a1;
            u[q.x] = s;
            u[q.y] = s;
        }
    } else if (t < P.t0[3]) {
        const int64_t g = t - P.t0[2];
        const int4 q = *reinterpret_cast<const int4 *>(P.idx + P.start[2] + 4 * g);
        if (zero_masked && g < P.nm[2]) {
            u[q.x] = T(0);
            u[q.y] = T(0);
            u[q.z] = T(0);
            u[q.w] = T(0);
        } else {
            const T a0 = u[q.x], a1 = u[q.y], a2 = u[q.z], a3 = u[q.w];
            const T s = ((a0 + a1) + a2) + a3;
            u[q.x] = s;
            u[q.y] = s;
            u[q.z] = s;
            u[q.w] = s;
        }
    } else {
        const int64_t g = t - P.t0[3];
        const int4 *q4 = reinterpret_cast<const int4 *>(P.idx + P.start[3] + 8 * g);
        const int4 q = q4[0], r = q4[1];
        if (zero_masked && g < P.nm[3]) {
            u[q.x] = T(0);
            u[q.y] = T(0);
            u[q.z] = T(0);
            u[q.w] = T(0);
            u[r.x] = T(0);
            u[r.y] = T(0);
            u[r.z] = T(0);
            u[r.w] = T(0);
        } else {
            const T a0 = u[q.x], a1 = u[q.y], a2 = u[q.z], a3 = u[q.w];
            const T a4 = u[r.x], a5 = u[r.y], a6 = u[r.z], a7 = u[r.w];
            const T s = ((((((a0 + a1) + a2) + a3) + a4) + a5) + a6) + a7;
            u[q.x] = s;
            u[q.y] = s;
            u[q.z] = s;
            u[q.w] = s;
            u[r.x] = s;
            u[r.y] = s;
            u[r.z] = s;
            u[r.w] = s;
        }
    }
}

int gs_launch(const sem_mesh *m, void *u, int dtype, int mode, cudaStream_t st, const int *guard, int gval) {
    GsPlan P;
    P.idx = m->gs_idx;
    P.t0[0] = 0;
    for (int b = 0; b < 4; ++b) {
        P.start[b] = m->gs_start[b];
        P.nm[b] = m->gs_nm[b];
        int64_t cnt;
        if (mode == kGsMaskOnly)
            cnt = m->gs_nm[b];
        else if (mode == kGsSum)
            cnt = b == 0 ? 0 : m->gs_n[b];
        else
            cnt = m->gs_n[b];  // bucket 0 holds masked groups only
        P.t0[b + 1] = P.t0[b] + cnt;
    }
    const int64_t n = P.t0[4];
    if (n == 0) return SEM_OK;
    const int64_t g = (n + 255) / 256;
    if (dtype == SEM_F64)
        gs_kernel<double><<<(unsigned)g, 256, 0, st>>>(static_cast<double *>(u), P, mode, guard, gval);
    else if (dtype == SEM_F32)
        gs_kernel<float><<<(unsigned)g, 256, 0, st>>>(static_cast<float *>(u), P, mode, guard, gval);
    else
        return fail(SEM_ERR_INVALID_ARG, "unknown dtype");
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

// ---- axis-by-axis gather-scatter on the box topology (CG loop) --------
// Summing the copies of every node can be done one axis at a time: after the
// y pass each copy holds the sum over its y-neighbours, after the z pass over
// its y and z neighbours, after the x pass over all.  The y and z passes run
// together here, one thread per (y, z) node group of one x position: the
// group's 2 or 4 copies are read, summed in a fixed order and written back
// (every copy gets the same bits).  Indices are computed, not loaded; the
// fastest thread index runs along x (i, then ex), so each group of N+1
// threads reads whole 32-byte sectors.

// Copies along one axis of global node index G (0 <= G < nel N + !per):
// 1 copy (e0, i0) or 2 copies (e0, N) and (e1, 0) on an element boundary.
__device__ __forceinline__ int axis_copies(int G, int nel, int per, int N, int &e0, int &i0, int &e1) {
    if (!per && G == nel * N) {
        e0 = nel - 1;
        i0 = N;
        e1 = -1;
        return 1;
    }
    const int e = G / N, i = G - e * N;
    if (i == 0 && (e > 0 || per)) {
        e0 = e > 0 ? e - 1 : nel - 1;
        i0 = N;
        e1 = e;
        return 2;
    }
    e0 = e;
    i0 = i;
    e1 = -1;
    return 1;
}

// Block row y = one (J, K) node group: y < nA: J = the (y / Gz)-th shared y
// boundary, K = y mod Gz; else J = any y node that is not shared (shared ones
// are skipped: they belong to the first set), K = a shared z boundary.
// Threads along x run over the x positions (ex, i).  N is a template
// parameter, so the index arithmetic per thread is a few multiplies.
template <typename T, int N>
__global__ void __launch_bounds__(256)
    gs_yz_kernel(T *__restrict__ u, BoxTopo B, int nA, int nrows, int nKs, const int *__restrict__ guard, int gval) {
    if (guard && *guard != gval) return;
    constexpr int N1 = N + 1, NPT = N1 * N1 * N1;
    const int nxl = B.nel[0] * N1;  // x positions (ex, i)
    const int Gz = B.nel[2] * N + (B.per[2] ? 0 : 1);
    for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
        int J, K;
        if (row < nA) {
            const int a = row / Gz;
            K = row - a * Gz;
            J = (B.per[1] ? a : a + 1) * N;
        } else {
            const int b = row - nA;
            const int jj = b / nKs;
            J = jj;
            K = (B.per[2] ? b - jj * nKs : b - jj * nKs + 1) * N;
        }
        int ey[2], jy[1], ez[2], kz[1];
        const int ny = axis_copies(J, B.nel[1], B.per[1], N, ey[0], jy[0], ey[1]);
        if (row >= nA && ny == 2) continue;  // a shared y node: done in the first set (uniform per block)
        const int nz = axis_copies(K, B.nel[2], B.per[2], N, ez[0], kz[0], ez[1]);
        if (ny * nz < 2) continue;
        for (int xi = blockIdx.x * blockDim.x + threadIdx.x; xi < nxl; xi += gridDim.x * blockDim.x) {
            const int ex = xi / N1, i = xi - ex * N1;
            auto at = [&](int ay, int bz, int jj2, int kk) {
                const int64_t e = ex + (int64_t)B.nel[0] * (ey[ay] + (int64_t)B.nel[1] * ez[bz]);
                return e * NPT + i + N1 * (jj2 + N1 * kk);
            };
            // copies in the order (y0,z0), (y1,z0), (y0,z1), (y1,z1); y1 / z1 sit at j / k = 0
            const int64_t i00 = at(0, 0, jy[0], kz[0]);
            if (ny == 2 && nz == 2) {
                const int64_t i10 = at(1, 0, 0, kz[0]), i01 = at(0, 1, jy[0], 0), i11 = at(1, 1, 0, 0);
                const T s = ((u[i00] + u[i10]) + u[i01]) + u[i11];
                u[i00] = s;
                u[i10] = s;
                u[i01] = s;
                u[i11] = s;
            } else {
                const int64_t i1 = ny == 2 ? at(1, 0, 0, kz[0]) : at(0, 1, jy[0], 0);
                const T s = u[i00] + u[i1];
                u[i00] = s;
                u[i1] = s;
            }
        }
    }
}

template <typename T>
static int gs_yz_dispatch(const sem_mesh *m, T *u, const BoxTopo &B, int nA, int nrows, int nKs, dim3 grid,
                          cudaStream_t st, const int *guard, int gval) {
    switch (m->N) {
#define SEM_GSYZ_CASE(n) \
    case n: gs_yz_kernel<T, n><<<grid, 256, 0, st>>>(u, B, nA, nrows, nKs, guard, gval); break;
        SEM_GSYZ_CASE(1) SEM_GSYZ_CASE(2) SEM_GSYZ_CASE(3) SEM_GSYZ_CASE(4) SEM_GSYZ_CASE(5)
        SEM_GSYZ_CASE(6) SEM_GSYZ_CASE(7) SEM_GSYZ_CASE(8) SEM_GSYZ_CASE(9) SEM_GSYZ_CASE(10) SEM_GSYZ_CASE(11)
#undef SEM_GSYZ_CASE
        default: return fail(SEM_ERR_UNSUPPORTED, "order N not built");
    }
    SEM_CUDA_CHECK(cudaGetLastError());
    return SEM_OK;
}

int gs_yz_launch(const sem_mesh *m, void *u, int dtype, cudaStream_t st, const int *guard, int gval) {
    const BoxTopo B = box_topo(m);
    const int64_t Gy = (int64_t)B.nel[1] * B.N + (B.per[1] ? 0 : 1);
    const int64_t Gz = (int64_t)B.nel[2] * B.N + (B.per[2] ? 0 : 1);
    const int nJs = B.per[1] ? B.nel[1] : B.nel[1] - 1;
    const int nKs = B.per[2] ? B.nel[2] : B.nel[2] - 1;
    const int64_t nxl = (int64_t)B.nel[0] * B.N1;
    const int64_t nA = (int64_t)nJs * Gz;
    const int64_t nrows = nA + Gy * nKs;
    if (nrows == 0 || nxl == 0) return SEM_OK;
    if (nrows >= (int64_t(1) << 31)) return fail(SEM_ERR_UNSUPPORTED, "gs_yz: too many node rows");
    dim3 grid((unsigned)((nxl + 255) / 256), (unsigned)(nrows < 65535 ? nrows : 65535));
    if (dtype == SEM_F64)
        return gs_yz_dispatch<double>(m, static_cast<double *>(u), B, (int)nA, (int)nrows, nKs, grid, st, guard, gval);
    if (dtype == SEM_F32)
        return gs_yz_dispatch<float>(m, static_cast<float *>(u), B, (int)nA, (int)nrows, nKs, grid, st, guard, gval);
    return fail(SEM_ERR_INVALID_ARG, "unknown dtype");
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
