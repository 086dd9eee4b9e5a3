// gemm_tc.cu -- BF16 tensor-core GEMM for sm_103a: D[M x N] = A[M x K] . B[N x K]^T
// with FP32 accumulation in tensor memory, and fused epilogues.
//
// Both operands are K-major (rows of K contiguous elements).  Tiles of
// 128 x 64 (A) and BN x 64 (B) elements are moved by TMA into 128-byte
// swizzled shared memory through a 3-stage (BN = 128) or 2-stage (BN = 256) mbarrier
// pipeline (two CTAs fit on an SM, so one CTA's epilogue overlaps the other's main
// loop); one thread
// issues tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulator of 128 lanes x
// BN columns in TMEM); after the last K tile the eight warps of the CTA read
// the accumulator with tcgen05.ld (warp w may read the lanes 32 (w mod 4) ..
// 32 (w mod 4) + 31, its tile rows; warps w and w + 4 split the columns in
// halves) and apply the epilogue.  Every wait on an mbarrier is bounded: on expiry the kernel
// records a timeout in a status word, stops issuing work, waits (bounded) for
// the copies it issued, frees its TMEM and returns.  The abort path is exact
// only when those second waits complete: if the wait for the issued matrix
// operations (or for the issued copies) also runs out, the kernel still frees
// its TMEM and exits, and what it leaves behind (tensor memory or shared
// memory written late) is undefined.  SA_ETIMEOUT is reported either way.
//
// Shapes: M multiple of 128, N multiple of BN, K multiple of 64 (callers pad).
#include <cstdint>
#include <cstdlib>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gelu.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
// Pipeline depth per tile width: 3 stages of a 128 x 128 pair (96 KB) or 2 of a
// 128 x 256 pair (96 KB), so that two CTAs share an SM.
template <int BN>
__host__ __device__ constexpr int stages_for() { return BN >= 256 ? 2 : 3; }
constexpr int kThreads = 256;  // 8 warps: all of them run the epilogue, two per TMEM lane quadrant
constexpr uint32_t kSpin = 1u << 20;  // bounded waits (each try_wait itself blocks for a while)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; with an abort flag it also gives up once another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int* abort_flag = nullptr) {
    for (uint32_t i = 0; i < kSpin; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *(const volatile int*)abort_flag) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row atoms of 1024 bytes (stride-dimension byte offset).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                     // leading-dimension byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride-dimension byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 columns of 32-bit accumulator -> 16 registers per thread (its row).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// test_stall: 0, except in the test of the timeout path: then the matrix-unit
// thread first waits on a barrier that nothing ever arrives on (polled without
// blocking, a bounded number of times), so that wait runs out while every
// copy the producer issued still completes normally.
template <int BN, class Epi>
__global__ void __launch_bounds__(kThreads, 2)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K, Epi epi,
                     int* status, uint32_t test_stall) {
    constexpr int kATile = kBM * kBK * 2;
    constexpr int kBTile = BN * kBK * 2;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;  // TMEM columns (power of two >= 32)
    constexpr int kStages = stages_for<BN>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = base + kStages * kATile;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBTile);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint64_t* never = done + 1;  // test_stall: armed by nobody
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int KT = K / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        mbar_init(never, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int issued = 0;
        for (int kt = 0; kt < KT; ++kt) {
            const int s = kt % kStages;
            if (kt >= kStages && !mbar_wait(&empty[s], ((kt / kStages) - 1) & 1, abort_flag)) {
                atomicExch(abort_flag, 1);
                break;
            }
            if (*(volatile int*)abort_flag) break;
            mbar_expect_tx(&full[s], kATile + kBTile);
            tma_load_2d(sA + s * kATile, &tmA, &full[s], kt * kBK, m0);
            tma_load_2d(sB + s * kBTile, &tmB, &full[s], kt * kBK, n0);
            issued = kt + 1;
        }
        // on abort: wait (bounded) for every copy issued, so none lands after the CTA exits
        if (*(volatile int*)abort_flag)
            for (int kt = (issued > kStages ? issued - kStages : 0); kt < issued; ++kt)
                mbar_wait(&full[kt % kStages], (kt / kStages) & 1);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t idesc = idesc_bf16(kBM, BN);
        bool ok = true;
        if (test_stall) {
            bool got = false;
            for (int i = 0; i < 4096 && !got; ++i) got = mbar_test_wait(never, 0);
            if (!got) {
                atomicExch(abort_flag, 1);
                ok = false;
            }
        }
        for (int kt = 0; kt < KT && ok; ++kt) {
            const int s = kt % kStages;
            if (!mbar_wait(&full[s], (kt / kStages) & 1) || *(volatile int*)abort_flag) {
                atomicExch(abort_flag, 1);
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = sdesc(smem_u32(sA + s * kATile));
            const uint64_t db = sdesc(smem_u32(sB + s * kBTile));
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)  // K = 16 per MMA: advance 32 bytes inside the swizzled row
                umma_bf16(tmem, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, (kt | kk) != 0 ? 1u : 0u);
            umma_commit(&empty[s]);
        }
        umma_commit(done);  // arrives once every MMA issued above has completed
    }
    __syncwarp();

    // ---- epilogue: warp w reads accumulator lanes 32 q .. 32 q + 31 (tile rows), q = w mod 4,
    // and the columns [h BN/2, (h + 1) BN/2), h = w / 4
    __shared__ float red[kBM];  // reducing epilogues: the second column half's sum per row
    const int quad = warp & 3, half = warp >> 2;
    const int row = m0 + quad * 32 + lane;
    float acc = 0.0f;
    const bool have = mbar_wait(done, 0);
    if (!have) atomicExch(abort_flag, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have && !*(volatile int*)abort_flag) {
#pragma unroll 1
        for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
            epi(row, n0 + c, v, acc);
        }
        if (Epi::kReduces && half == 1) red[quad * 32 + lane] = acc;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // the row's sum: first half + second half, in that order
    if (Epi::kReduces && half == 0 && have && !*(volatile int*)abort_flag) epi.finish(row, n0, acc + red[quad * 32 + lane]);
    // SA_ETIMEOUT, unless an earlier error of the run is already recorded
    if (threadIdx.x == 0 && *(volatile int*)abort_flag && status) atomicCAS(status, 0, 4);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// ---- epilogues ------------------------------------------------------------
// Each epilogue takes 16 accumulator columns of one row; a reducing one (kReduces)
// adds into acc, and finish() stores the row's sum over the tile.
struct EpiStoreF32 {
    static constexpr bool kReduces = false;
    float* D;
    int ldd;
    __device__ __forceinline__ void finish(int, int, float) const {}
    __device__ __forceinline__ void operator()(int row, int col, const float* v, float&) const {
        float4* p = reinterpret_cast<float4*>(D + (size_t)row * ldd + col);
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
};

// Surrogate layer: z = acc + bias; stores gelu(z) as BF16 (and z as FP32 when Z != nullptr).
struct EpiBiasGelu {
    static constexpr bool kReduces = false;
    const float* bias;
    __nv_bfloat16* A;
    int lda;
    float* Z;
    int ldz;
    __device__ __forceinline__ void finish(int, int, float) const {}
    __device__ __forceinline__ void operator()(int row, int col, const float* v, float&) const {
        __align__(16) __nv_bfloat16 a[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float z = v[j] + bias[col + j];
            if (Z) Z[(size_t)row * ldz + col + j] = z;
            a[j] = __float2bfloat16_rn(gelu_f(z));
        }
        uint4* dst = reinterpret_cast<uint4*>(A + (size_t)row * lda + col);
        dst[0] = reinterpret_cast<const uint4*>(a)[0];
        dst[1] = reinterpret_cast<const uint4*>(a)[1];
    }
};

// Surrogate output head: part[row][n0 / BN] = sum over the tile's columns of
// gelu(acc + b) w, in a fixed order (per 16 columns sequentially, the chunks of
// each column half in turn, then first half + second half), so it is
// deterministic; stores z as FP32 when Z != nullptr.
struct EpiBiasGeluDot {
    static constexpr bool kReduces = true;
    const float* bias;
    const float* w;
    float* part;
    int nparts;
    int tile;
    float* Z;
    int ldz;
    __device__ __forceinline__ void finish(int row, int n0, float total) const {
        part[(size_t)row * nparts + n0 / tile] = total;
    }
    __device__ __forceinline__ void operator()(int row, int col, const float* v, float& acc) const {
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float z = v[j] + bias[col + j];
            if (Z) Z[(size_t)row * ldz + col + j] = z;
            s = fmaf(gelu_f(z), w[col + j], s);
        }
        acc += s;
    }
};

// ---- host side ------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Tensor map of a row-major [rows x K] BF16 matrix with leading dimension ld
// (elements), boxes of box_rows x 64 elements, 128-byte swizzle.
bool make_tmap(CUtensorMap* m, const void* ptr, int rows, int K, int ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
size_t gemm_smem() {
    constexpr int kStages = stages_for<BN>();
    return 1024 + (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + (2 * kStages + 2) * 8 + 16;
}

template <int BN, class Epi>
cudaError_t launch_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const Epi& epi, int* status,
                        cudaStream_t s) {
    if (M % kBM || N % BN || K % kBK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (lda * 2) % 16 || (ldb * 2) % 16) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, A, M, K, lda, kBM) || !make_tmap(&tb, B, N, K, ldb, BN)) return cudaErrorInvalidValue;
    const size_t smem = gemm_smem<BN>();
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(N / BN, M / kBM);
    // Test of the timeout path only: SA_GEMM_TEST_STALL=1 makes one wait of the
    // matrix-unit thread run out (see test_stall), so the kernel must report SA_ETIMEOUT.
    const char* t = std::getenv("SA_GEMM_TEST_STALL");
    const uint32_t test_stall = (t && t[0] == '1') ? 1u : 0u;
    gemm_bf16_kernel<BN, Epi><<<grid, kThreads, smem, s>>>(ta, tb, K, epi, status, test_stall);
    return cudaGetLastError();
}

__device__ int g_gemm_status;  // status word of the kernel-level entry point

}  // namespace

// D (FP32, [M x N], leading dimension ldd) = A [M x K] . B [N x K]^T (BF16, K-major).
cudaError_t launch_gemm_bf16_f32(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K,
                                 int* status, cudaStream_t s) {
    EpiStoreF32 epi{D, ldd};
    if (N % 256 == 0) return launch_gemm<256>(A, lda, B, ldb, M, N, K, epi, status, s);
    if (N % 128 == 0) return launch_gemm<128>(A, lda, B, ldb, M, N, K, epi, status, s);
    return launch_gemm<64>(A, lda, B, ldb, M, N, K, epi, status, s);
}

cudaError_t launch_gemm_bias_gelu(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const float* bias,
                                  void* out_bf16, int ldo, float* Z, int ldz, int* status, cudaStream_t s) {
    EpiBiasGelu epi{bias, static_cast<__nv_bfloat16*>(out_bf16), ldo, Z, ldz};
    if (N % 128 == 0) return launch_gemm<128>(A, lda, B, ldb, M, N, K, epi, status, s);
    return launch_gemm<64>(A, lda, B, ldb, M, N, K, epi, status, s);
}

cudaError_t launch_gemm_bias_gelu_dot(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                                      const float* bias, const float* w, float* part, float* Z, int ldz, int* status,
                                      cudaStream_t s) {
    if (N % 128) return cudaErrorInvalidValue;
    EpiBiasGeluDot epi{bias, w, part, N / 128, 128, Z, ldz};
    return launch_gemm<128>(A, lda, B, ldb, M, N, K, epi, status, s);
}

int* gemm_status_ptr() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gemm_status) != cudaSuccess) return nullptr;
    return static_cast<int*>(p);
}

}  // namespace sa
