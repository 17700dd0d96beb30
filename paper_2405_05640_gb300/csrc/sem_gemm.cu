// sem_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05).
//
// C[M x N] = act(A[M x K] . B[N x K]^T + bias), A and B row-major BF16 with K
// contiguous ("TN"), FP32 accumulation in tensor memory (TMEM), output FP32
// and/or BF16.  Used by the element-local network of the learned initial
// guess (forward: activations x weights^T; backward: transposed operands).
//
// Design (one CTA of 4 warps per 128 x BN output tile):
//  - warp 0, one thread: TMA producer.  2-D tiled bulk-tensor copies of the
//    A tile (128 x 64) and B tile (BN x 64) with the 128-byte swizzle into a
//    ring of STAGES shared-memory stages; completion counted in bytes on a
//    "full" mbarrier per stage.
//  - warp 1, one thread: MMA issuer.  Waits for a full stage, issues four
//    tcgen05.mma (K = 16 each) reading both operands from shared memory
//    through matrix descriptors and accumulating into a 128 x BN FP32 TMEM
//    tile, then tcgen05.commit to the stage's "empty" mbarrier so the
//    producer can refill it; a final commit signals the epilogue.
//  - all 4 warps: epilogue.  Warp w reads TMEM lanes 32w..32w+31 (rows of the
//    tile) with tcgen05.ld, adds the bias, applies the activation and stores.
// Every mbarrier wait is bounded by the global timer; on time-out the kernel
// records an error word, drains what it issued (bounded), frees its TMEM and
// returns.

#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "sem_common.cuh"

namespace sem {

constexpr int kGemmBM = 128, kGemmBK = 64, kGemmStages = 4, kGemmThreads = 128;
constexpr uint32_t kTileABytes = kGemmBM * kGemmBK * 2;  // 16 KB

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D(tmem) (+)= A(smem desc) . B(smem desc)^T, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// 32 lanes x 32 columns of 32-bit TMEM cells: thread t gets row (lane) t,
// columns col .. col+31.
__device__ __forceinline__ void tmem_ld_32x32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle (rows of 64 BF16 = 128 B, 8-row groups 1024 B apart):
// start address >> 4 in bits 0-13, leading offset (unused here) in 16-29,
// stride offset 1024 >> 4 in 32-45, descriptor version 1 in 46-47, layout
// "128-byte swizzle" (2) in 61-63.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int BN>
__host__ __device__ constexpr int gemm_smem_bytes() {
    return 1024 /*alignment slack*/ + kGemmStages * (int)(kTileABytes + BN * kGemmBK * 2) + 256;
}

struct GemmEpi {
    const float *bias;  // [N] or null
    int act;            // 0 identity, 1 ReLU
    float *c32;         // [M][ldc] or null
    __nv_bfloat16 *c16; // [M][ldc] or null
    int ldc;
    float *ws;          // split-K: [splits][M][N] FP32 partial tiles (no bias, no activation), or null
    int M, N;
};

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_tn_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K,
                        GemmEpi epi, int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    // align the operand ring to 1024 bytes (the swizzle pattern period)
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    unsigned char *sA = smem;
    unsigned char *sB = smem + kGemmStages * kTileABytes;
    constexpr uint32_t kTileBBytes = BN * kGemmBK * 2;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + kGemmStages * kTileBBytes);
    uint64_t *empty = full + kGemmStages;
    uint64_t *done = empty + kGemmStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.x * BN;
    // split-K: CTA z takes the K-blocks [kb0, kb0 + KT) of its slice
    const int KTall = K / kGemmBK, per = (KTall + gridDim.z - 1) / gridDim.z;
    const int kb0 = blockIdx.z * per;
    const int KT = KTall - kb0 < per ? KTall - kb0 : per;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    __syncwarp();  // tcgen05.alloc is warp-aligned
    if (warp == 0) {
        tmem_alloc(tmem_slot, (uint32_t)BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    if (warp == 0 && lane == 0) {
        // producer
        int kt = 0;
        for (; kt < KT; ++kt) {
            const int s = kt % kGemmStages;
            if (kt >= kGemmStages && !mbar_wait_bounded(&empty[s], ((kt / kGemmStages) - 1) & 1, err, kDevTimeoutTma)) {
                ok = false;
                break;
            }
            mbar_arrive_expect_tx(&full[s], kTileABytes + kTileBBytes);
            tma_load_2d(sA + s * kTileABytes, &tmA, (kb0 + kt) * kGemmBK, m0, &full[s]);
            tma_load_2d(sB + s * kTileBBytes, &tmB, (kb0 + kt) * kGemmBK, n0, &full[s]);
        }
        if (!ok) {
            // drain the stages still being filled (bounded)
            for (int q = (kt > kGemmStages ? kt - kGemmStages : 0); q < kt; ++q)
                mbar_wait_bounded(&full[q % kGemmStages], (q / kGemmStages) & 1, err, kDevTimeoutTma);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16_f32(kGemmBM, BN);
        int kt = 0;
        for (; kt < KT; ++kt) {
            const int s = kt % kGemmStages;
            if (!mbar_wait_bounded(&full[s], (kt / kGemmStages) & 1, err, kDevTimeoutTma)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * kTileABytes), b0 = smem_u32(sB + s * kTileBBytes);
#pragma unroll
            for (int kk = 0; kk < kGemmBK / 16; ++kk)
                umma_bf16(tmem, sw128_kmajor_desc(a0 + kk * 32), sw128_kmajor_desc(b0 + kk * 32), idesc,
                          (kt | kk) != 0);
            umma_commit(&empty[s]);
        }
        umma_commit(done);  // fires when every MMA issued above has completed
    }
    __syncwarp();

    // epilogue: warp w owns rows 32w .. 32w+31 of the tile (TMEM lanes)
    const bool have = mbar_wait_bounded(done, 0, err, kDevTimeoutTma);
    tc_fence_after();
    // tcgen05.ld is warp-aligned: decide for the whole block
    const bool go = __syncthreads_and(have && ok);
    if (go) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld_32x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            const int col = n0 + c;
            if (epi.ws) {  // split-K partial: raw FP32 tile
                float4 *dst = reinterpret_cast<float4 *>(epi.ws + ((size_t)blockIdx.z * epi.M + row) * epi.N + col);
#pragma unroll
                for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                continue;
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                float x = v[q];
                if (epi.bias) x += epi.bias[col + q];
                if (epi.act == 1) x = fmaxf(x, 0.0f);
                v[q] = x;
            }
            if (epi.c32) {
                float4 *dst = reinterpret_cast<float4 *>(epi.c32 + (size_t)row * epi.ldc + col);
#pragma unroll
                for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            if (epi.c16) {
                __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(epi.c16 + (size_t)row * epi.ldc + col);
#pragma unroll
                for (int q = 0; q < 16; ++q) dst[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)BN);
}

// Split-K reduction: C = act(sum over the slices, in slice order, + bias).
__global__ void gemm_splitk_reduce_kernel(const float *__restrict__ ws, int splits, GemmEpi epi) {
    const int64_t MN = (int64_t)epi.M * epi.N;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < MN; q += (int64_t)gridDim.x * blockDim.x) {
        float x = 0.f;
        for (int s = 0; s < splits; ++s) x += ws[s * MN + q];
        const int row = (int)(q / epi.N), col = (int)(q - (int64_t)row * epi.N);
        if (epi.bias) x += epi.bias[col];
        if (epi.act == 1) x = fmaxf(x, 0.0f);
        if (epi.c32) epi.c32[(size_t)row * epi.ldc + col] = x;
        if (epi.c16) epi.c16[(size_t)row * epi.ldc + col] = __float2bfloat16_rn(x);
    }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D BF16 row-major [rows][cols] tensor map with a (64 x box_rows) box and
// the 128-byte swizzle.
static int make_tmap(CUtensorMap *tm, const void *ptr, int rows, int cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(SEM_ERR_CUDA, "cuTensorMapEncodeTiled not available from the driver");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SEM_ERR_INVALID_ARG, "cuTensorMapEncodeTiled rejected the operand");
    return SEM_OK;
}

// Split count for a workspace of ws_floats: slices of K when the output
// tiles alone fill less than the SMs (at least 8 K-blocks per slice, at most
// 16 slices), else 1.
int gemm_splits(int M, int N, int K, size_t ws_floats, int num_sms) {
    const int BN = (N % 256 == 0) ? 256 : 128;
    const int tiles = (M / kGemmBM) * (N / BN);
    const int KT = K / kGemmBK;
    int s = (num_sms + tiles - 1) / tiles;
    s = s < 16 ? s : 16;
    s = s < KT / 8 ? s : KT / 8;
    while (s > 1 && (size_t)s * M * N > ws_floats) --s;
    if (s <= 1) return 1;
    // every slice non-empty: the kernel gives slice z the K-blocks from
    // z * ceil(KT / s), so s is the number of slices of that length
    const int per = (KT + s - 1) / s;
    return (KT + per - 1) / per;
}

int gemm_tn_bf16(const void *A, const void *B, int M, int N, int K, const float *bias, int act, float *c32,
                 void *c16, int ldc, int *d_err, cudaStream_t st, float *ws, size_t ws_floats) {
    if (!A || !B || (!c32 && !c16) || !d_err) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
    if (M <= 0 || N <= 0 || K <= 0 || M % kGemmBM || K % kGemmBK || N % 128)
        return fail(SEM_ERR_INVALID_ARG, "GEMM needs M % 128 == 0, N % 128 == 0, K % 64 == 0");
    if (ldc < N || ldc % 4) return fail(SEM_ERR_INVALID_ARG, "ldc must be >= N and a multiple of 4");
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) % 16)
        return fail(SEM_ERR_INVALID_ARG, "A and B must be 16-byte aligned");
    const int BN = (N % 256 == 0) ? 256 : 128;
    CUtensorMap ta, tb;
    int s = make_tmap(&ta, A, M, K, kGemmBM);
    if (s != SEM_OK) return s;
    s = make_tmap(&tb, B, N, K, BN);
    if (s != SEM_OK) return s;
    int dev = 0, sms = 148;
    SEM_CUDA_CHECK(cudaGetDevice(&dev));
    SEM_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int splits = ws ? gemm_splits(M, N, K, ws_floats, sms) : 1;
    GemmEpi epi{bias, act, c32, static_cast<__nv_bfloat16 *>(c16), ldc, splits > 1 ? ws : nullptr, M, N};
    dim3 grid(N / BN, M / kGemmBM, splits);
    if (BN == 256) {
        constexpr int smem = gemm_smem_bytes<256>();
        SEM_CUDA_CHECK(cudaFuncSetAttribute(gemm_tn_bf16_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        gemm_tn_bf16_kernel<256><<<grid, kGemmThreads, smem, st>>>(ta, tb, K, epi, d_err);
    } else {
        constexpr int smem = gemm_smem_bytes<128>();
        SEM_CUDA_CHECK(cudaFuncSetAttribute(gemm_tn_bf16_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        gemm_tn_bf16_kernel<128><<<grid, kGemmThreads, smem, st>>>(ta, tb, K, epi, d_err);
    }
    SEM_CUDA_CHECK(cudaGetLastError());
    if (splits > 1) {
        const int64_t MN = (int64_t)M * N;
        const int g = (int)((MN + 255) / 256 < (int64_t)sms * 8 ? (MN + 255) / 256 : (int64_t)sms * 8);
        gemm_splitk_reduce_kernel<<<g, 256, 0, st>>>(ws, splits, epi);
        SEM_CUDA_CHECK(cudaGetLastError());
    }
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

int sem_gemm_bf16(const void *A, const void *B, int M, int N, int K, const float *bias, int act, float *C32,
                  void *C16, int ldc, int *d_err, void *stream) {
    return gemm_tn_bf16(A, B, M, N, K, bias, act, C32, C16, ldc, d_err, as_stream(stream), nullptr, 0);
}

size_t sem_gemm_bf16_splitk_work_bytes(int M, int N, int K) {
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    return sizeof(float) * 16 * (size_t)M * N;
}

int sem_gemm_bf16_splitk(const void *A, const void *B, int M, int N, int K, const float *bias, int act, float *C32,
                         void *C16, int ldc, void *d_work, size_t work_bytes, int *d_err, void *stream) {
    if (d_work && reinterpret_cast<uintptr_t>(d_work) % 16)
        return fail(SEM_ERR_WORKSPACE, "split-K work space must be 16-byte aligned");
    return gemm_tn_bf16(A, B, M, N, K, bias, act, C32, C16, ldc, d_err, as_stream(stream),
                        static_cast<float *>(d_work), d_work ? work_bytes / sizeof(float) : 0);
}

}  // extern "C"
