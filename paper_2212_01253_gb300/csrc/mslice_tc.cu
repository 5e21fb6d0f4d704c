// mslice_tc.cu -- dense layers of the learned initialiser on the 5th-generation
// tensor cores: C = beta C + A B^T (+ bias, ReLU) with BF16 operands and FP32
// accumulation in tensor memory (tcgen05.mma kind::f16, M = 128, N = 256),
// operand tiles moved by TMA (cp.async.bulk.tensor, 128-byte swizzle, this
// GPU's memory only, no multicast) through a 4-stage mbarrier pipeline.
//
// One CTA of 4 warps per 128 x 256 output tile (tiles in groups of 8 row
// blocks, for L2 reuse): lane 0 of warp 0 issues the
// TMA loads, lane 0 of warp 1 issues the MMAs (4 per 64-wide k step) and
// commits each stage back to the loader, and all four warps read the
// accumulator out of tensor memory (warp w owns rows 32w..32w+31) for the
// epilogue.  Every wait on an mbarrier is bounded (about one second of
// %globaltimer); a wait that runs out records MSLICE_ETIMEDOUT in the status
// word and the CTA leaves after freeing its tensor memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "mslice.h"

namespace {

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 4;
constexpr int kStageA = kBM * kBK * 2, kStageB = kBN * kBK * 2;   // bytes per stage
constexpr int kSmemBytes = kStages * (kStageA + kStageB) + 1024;   // + 1024 for the alignment of the tiles
constexpr int kTmemCols = 256;                                      // FP32 accumulator, one column per n
constexpr int kGroupM = 8;                                          // row blocks per group of the tile order
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}

// 2-D tiled TMA load of box {x (k), y (row)} into shared memory, completing
// on the mbarrier's transaction count
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor of a K-major operand tile with the 128-byte
// swizzle: rows of 128 bytes (64 BF16 of k), 8-row atoms 1024 bytes apart
// (stride byte offset), leading byte offset unused for this layout (1),
// descriptor version 1, layout type 2 (128-byte swizzle)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3fffu);
    d |= (uint64_t)1u << 16;                       // leading byte offset (unused), 16 B
    d |= (uint64_t)((1024u >> 4) & 0x3fffu) << 32; // stride byte offset, 1024 B
    d |= (uint64_t)1u << 46;                       // version
    d |= (uint64_t)2u << 61;                       // 128-byte swizzle
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes (lane l
// of the warp gets lane 32 w + l); the wait is in the same statement, so no
// use of the registers can move above it
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// the status word of the tensor-core GEMM: MSLICE_ETIMEDOUT bits after a
// bounded wait ran out (read and cleared by mslice_nn_gemm_bf16_status)
__device__ unsigned g_tc_status;

__device__ __forceinline__ void store_row32(float* o, const float (&v)[32], int n_valid, const float* bias,
                                            int relu, float beta, bool vec) {
    float r[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        float x = v[i];
        if (bias && i < n_valid) x += __ldg(bias + i);
        if (relu) x = fmaxf(x, 0.f);
        r[i] = x;
    }
    if (vec && n_valid == 32) {
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
            float4 x = make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
            if (beta != 0.f) {
                const float4 c = *reinterpret_cast<const float4*>(o + i);
                x = make_float4(fmaf(beta, c.x, x.x), fmaf(beta, c.y, x.y), fmaf(beta, c.z, x.z), fmaf(beta, c.w, x.w));
            }
            *reinterpret_cast<float4*>(o + i) = x;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i < n_valid) o[i] = beta != 0.f ? fmaf(beta, o[i], r[i]) : r[i];
    }
}

// C[m][n] = beta C[m][n] + sum_k A[m][k] B[n][k] (+ bias[n]) (ReLU if relu):
// one 128 x 256 tile of C per CTA, A and B BF16 K-major through the tensor maps
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap mapA,
                                                    const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
                                                    float* __restrict__ C, long long ldc,
                                                    const float* __restrict__ bias, int relu, float beta) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], acc_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tiles = (smem_u32(smem_raw) + 1023u) & ~1023u;   // 1024-byte aligned for the swizzle atoms
    // tile order: CTAs in launch order walk groups of kGroupM row blocks, all
    // column blocks of a group before the next, so that the tiles in flight
    // at once share a few A row blocks and a band of B column blocks in L2
    const int nbn = gridDim.x, nbm = gridDim.y;
    const int lin = blockIdx.y * nbn + blockIdx.x;
    const int first_m = (lin / (kGroupM * nbn)) * kGroupM;
    const int gm = nbm - first_m < kGroupM ? nbm - first_m : kGroupM;
    const int within = lin - first_m * nbn;
    const int m0 = (first_m + within % gm) * kBM, n0 = (within / gm) * kBN;
    const int kt_n = (K + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&acc_bar), 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // loader: stage s is free once the MMAs that read it have completed
        for (int kt = 0; kt < kt_n; ++kt) {
            const int s = kt % kStages;
            const uint32_t ph = (uint32_t)(kt / kStages) & 1u;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u)) {
                s_fail = 1;
                break;
            }
            const uint32_t fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, (uint32_t)(kStageA + kStageB));
            tma_load_2d(tiles + s * kStageA, &mapA, kt * kBK, m0, fb);
            tma_load_2d(tiles + kStages * kStageA + s * kStageB, &mapB, kt * kBK, n0, fb);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: four k = 16 steps per stage, the descriptors advanced by
        // 32 bytes along the swizzled 128-byte rows
        for (int kt = 0; kt < kt_n; ++kt) {
            const int s = kt % kStages;
            const uint32_t ph = (uint32_t)(kt / kStages) & 1u;
            if (s_fail || !mbar_wait(smem_u32(&full_bar[s]), ph)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = tiles + s * kStageA, b0 = tiles + kStages * kStageA + s * kStageB;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                mma_f16(tmem, sw128_desc(a0 + 32 * kk), sw128_desc(b0 + 32 * kk), (kt | kk) != 0 ? 1u : 0u);
            mma_commit(smem_u32(&empty_bar[s]));
        }
        mma_commit(smem_u32(&acc_bar));   // the accumulator is complete when every MMA above is
    }
    __syncwarp();
    const bool ok = mbar_wait(smem_u32(&acc_bar), 0u);
    tc_fence_after();
    // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile in its lanes
    const int m = m0 + 32 * warp + lane;
    const bool vec = ((ldc & 3) == 0) && ((((uintptr_t)C) & 15) == 0);
#pragma unroll 1
    for (int c = 0; c < kBN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c), v);
        const int nb = n0 + 32 * c;
        if (ok && m < M && nb < N) {
            const int nv = N - nb < 32 ? N - nb : 32;
            store_row32(C + (long long)m * ldc + nb, v, nv, bias ? bias + nb : nullptr, relu, beta, vec);
        }
    }
    if (threadIdx.x == 0 && (!ok || s_fail)) atomicOr(&g_tc_status, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTmemCols)
                     : "memory");
}

// dst[r][k] = BF16(src[r * s_row + k * s_k]) (nearest even) for k < K, 0 for K <= k < ld
__global__ void k_pack_bf16(const float* __restrict__ src, long long s_row, long long s_k, int rows, int K,
                            uint16_t* __restrict__ dst, long long ld) {
    const long long n = (long long)rows * ld;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / ld, k = i - r * ld;
        float x = 0.f;
        if (k < K) x = src[r * s_row + k * s_k];
        uint32_t b;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(b) : "f"(0.f), "f"(x));
        dst[i] = (uint16_t)(b & 0xffffu);
    }
}

// cuTensorMapEncodeTiled from the driver, found once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// tensor map of a row-major [rows][ld] BF16 matrix read as K-major tiles of
// box_rows x 64 with the 128-byte swizzle; columns past K read as zero
bool make_map(CUtensorMap* map, const void* base, int rows, int K, long long ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int configure_tc() {
    static int done[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MSLICE_ELAUNCH;
    if (!done[dev]) {
        if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
            return MSLICE_ELAUNCH;
        done[dev] = 1;
    }
    return MSLICE_OK;
}

}  // namespace

extern "C" {

int mslice_nn_pack_bf16(const float* src, long long s_row, long long s_k, int rows, int K, void* dst, long long ld,
                        void* stream) {
    if (!src || !dst || rows < 1 || K < 1 || ld < K || ((uintptr_t)dst & 1)) return MSLICE_EINVAL;
    const long long n = (long long)rows * ld;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_pack_bf16<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(src, s_row, s_k, rows, K, (uint16_t*)dst, ld);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_nn_gemm_bf16(int M, int N, int K, const void* A, long long lda, const void* B, long long ldb, float* C,
                        long long ldc, const float* bias, int relu, float beta, void* stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || ldc < N || lda < K || ldb < K) return MSLICE_EINVAL;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (lda & 7) || (ldb & 7) || ((uintptr_t)C & 3))
        return MSLICE_EINVAL;
    if ((M + kBM - 1) / kBM > 65535) return MSLICE_EUNSUPPORTED;
    int rc = configure_tc();
    if (rc) return rc;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, lda, kBM) || !make_map(&mb, B, N, K, ldb, kBN)) return MSLICE_EUNSUPPORTED;
    const dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
    k_gemm_tc<<<grid, 128, kSmemBytes, (cudaStream_t)stream>>>(ma, mb, M, N, K, C, ldc, bias, relu, beta);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_nn_gemm_bf16_status(void* stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return MSLICE_ELAUNCH;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(v)) != cudaSuccess) return MSLICE_ELAUNCH;
    if (v) {
        const unsigned zero = 0;
        if (cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(zero)) != cudaSuccess) return MSLICE_ELAUNCH;
        return MSLICE_ETIMEDOUT;
    }
    return MSLICE_OK;
}

}  // extern "C"
