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
#include "tc_sm103.cuh"

namespace sa {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
// Pipeline depth per tile width: 3 stages of a 128 x 128 pair (96 KB) or 2 of a
// 128 x 256 pair (96 KB), so that two CTAs share an SM.
template <int BN>
__host__ __device__ constexpr int stages_for() { return BN >= 256 ? 2 : 3; }
constexpr int kThreads = 256;  // 8 warps: all of them run the epilogue, two per TMEM lane quadrant
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
    static_assert(!Epi::kStaged || kThreads * 17 * 4 <= kStages * kATile, "staging area beyond the A stages");
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
            if constexpr (Epi::kStaged) {
                if (epi.dual) {  // two products: B's rows b_row1 + .. and b_row2 + .. of one output column tile
                    const int nc = blockIdx.x * (BN / 2);
                    tma_load_2d(sB + s * kBTile, &tmB, &full[s], kt * kBK, epi.b_row1 + nc);
                    tma_load_2d(sB + s * kBTile + kBTile / 2, &tmB, &full[s], kt * kBK, epi.b_row2 + nc);
                } else {
                    tma_load_2d(sB + s * kBTile, &tmB, &full[s], kt * kBK, n0);
                }
            } else {
                tma_load_2d(sB + s * kBTile, &tmB, &full[s], kt * kBK, n0);
            }
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
    if constexpr (Epi::kStaged)
        if (warp >= 2) {
            if (epi.dual) epi.prefetch(m0, blockIdx.x * (BN / 2), BN / 2, threadIdx.x - 64, kThreads - 64);
            else epi.prefetch(m0, n0, BN, threadIdx.x - 64, kThreads - 64);
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
        // a staging epilogue gets 32 x 17 floats per warp of the pipeline's shared
        // memory, idle once every matrix operation has completed
        float* scratch = reinterpret_cast<float*>(base) + warp * (32 * 17);
        const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
        bool dual = false;
        if constexpr (Epi::kStaged) dual = epi.dual;
        if (dual) {
            // columns [0, BN/2) and [BN/2, BN) hold two products of the same output
            // columns: the second (the smaller) is added first
            if constexpr (Epi::kStaged) {
                const int nc = blockIdx.x * (BN / 2);
#pragma unroll 1
                for (int c = half * (BN / 4); c < (half + 1) * (BN / 4); c += 16) {
                    float v[16];
                    tmem_ld16(tl + (uint32_t)(c + BN / 2), v);
                    epi.staged(m0 + quad * 32, nc + c, v, scratch, lane, epi.shift2);
                    tmem_ld16(tl + (uint32_t)c, v);
                    epi.staged(m0 + quad * 32, nc + c, v, scratch, lane, epi.shift);
                }
            }
        } else {
#pragma unroll 1
            for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 16) {
                float v[16];
                tmem_ld16(tl + (uint32_t)c, v);
                if constexpr (Epi::kStaged)
                    epi.staged(m0 + quad * 32, n0 + c, v, scratch, lane, epi.shift);
                else
                    epi(row, n0 + c, v, acc);
            }
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
    static constexpr bool kStaged = false;
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
    static constexpr bool kStaged = false;
    const float* bias;
    __nv_bfloat16* A;
    int lda;
    float* Z;
    int ldz;
    __device__ __forceinline__ void finish(int, int, float) const {}
    __device__ __forceinline__ void operator()(int row, int col, const float* v, float&) const {
        uint32_t a[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const f32x2_t z = f2_add(f2_pack(v[j], v[j + 1]), f2_pack(bias[col + j], bias[col + j + 1]));
            const float2 g = f2_unpack(gelu2(z));
            if (Z) {
                const float2 zz = f2_unpack(z);
                Z[(size_t)row * ldz + col + j] = zz.x;
                Z[(size_t)row * ldz + col + j + 1] = zz.y;
            }
            const __nv_bfloat162 h = __floats2bfloat162_rn(g.x, g.y);
            a[j / 2] = *reinterpret_cast<const uint32_t*>(&h);
        }
        uint4* dst = reinterpret_cast<uint4*>(A + (size_t)row * lda + col);
        dst[0] = make_uint4(a[0], a[1], a[2], a[3]);
        dst[1] = make_uint4(a[4], a[5], a[6], a[7]);
    }
};

// Surrogate output head: part[row][n0 / BN] = sum over the tile's columns of
// gelu(acc + b) w, in a fixed order (per 16 columns: the even and the odd columns
// each in order, then even + odd; the 16-column groups of each column half in
// turn; then first half + second half), so it is deterministic; stores z as FP32
// when Z != nullptr.
struct EpiBiasGeluDot {
    static constexpr bool kReduces = true;
    static constexpr bool kStaged = false;
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
        f32x2_t s = f2_splat(0.0f);  // even and odd columns, each summed in order
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const f32x2_t z = f2_add(f2_pack(v[j], v[j + 1]), f2_pack(bias[col + j], bias[col + j + 1]));
            if (Z) {
                const float2 zz = f2_unpack(z);
                Z[(size_t)row * ldz + col + j] = zz.x;
                Z[(size_t)row * ldz + col + j + 1] = zz.y;
            }
            s = f2_fma(gelu2(z), f2_pack(w[col + j], w[col + j + 1]), s);
        }
        const float2 se = f2_unpack(s);
        acc += se.x + se.y;
    }
};

// Exact split product (the rotated costs' level-0 transform): Y (double-float
// pairs (hi, lo), [M x N], leading dimension ldy) += (A . B^T) 2^(er[row] +
// fq[col] - shift).  A and B hold BF16 integer slices of magnitude <= 128, so
// every product is an integer of magnitude <= 2^14 and, for K <= 1024, every
// partial sum of the FP32 accumulator is an integer of magnitude <= 2^24: the
// accumulator is exact, and so is its scaling by a power of two.  The pair
// takes it by TwoSum and Fast2Sum (explicitly rounded, never contracted).
__device__ __forceinline__ float2 dd_add(float2 a, float b) {
    const float s = __fadd_rn(a.x, b);
    const float bb = __fsub_rn(s, a.x);
    const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const float t = __fadd_rn(a.y, e);
    const float hi = __fadd_rn(s, t);
    return make_float2(hi, __fsub_rn(t, __fsub_rn(hi, s)));
}
struct EpiAccumPair {
    static constexpr bool kReduces = false;
    static constexpr bool kStaged = true;
    float2* Y;
    int ldy;
    const int* er;
    const int* fq;
    int shift;
    // two products per tile (B's rows b_row1 + c and b_row2 + c for output column c,
    // scaled by shift and shift2), or one (B's rows = the output columns)
    bool dual;
    int b_row1, b_row2, shift2, b_rows;  // b_rows: rows of B (its tensor map)
    __device__ __forceinline__ void finish(int, int, float) const {}
    // 2^e as an FP32 number, for e >= -126 (smaller scales flush to zero: below the pairs' range)
    __device__ __forceinline__ static float pow2(int e) { return e < -126 ? 0.0f : __int_as_float((e + 127) << 23); }
    // The warp's 32 rows row0 .. row0 + 31 (lane i holds row row0 + i) and the 16
    // columns col .. col + 15 go through shared memory (rows 17 floats apart: no
    // bank conflicts either way), so that each half-warp reads and writes one
    // row's 16 pairs, 128 contiguous bytes, instead of 32 rows 8 KB apart.
    __device__ __forceinline__ void staged(int row0, int col, const float* v, float* s, int lane, int sh) const {
#pragma unroll
        for (int j = 0; j < 16; ++j) s[lane * 17 + j] = v[j];
        __syncwarp();
        const int j = lane & 15, h = lane >> 4;
        const int f = fq[col + j] - sh;
        float2* y = Y + (size_t)(row0 + 16 * h) * ldy + col + j;  // rows i and i + 16: banks 17 i + j, 17 i + 16 + j
        float2 cur[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) cur[i] = y[(size_t)i * ldy];  // all loads in flight before the first store
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int r = i + 16 * h;
            y[(size_t)i * ldy] = dd_add(cur[i], __fmul_rn(s[r * 17 + j], pow2(er[row0 + r] + f)));
        }
        __syncwarp();
    }
    // Issued by the warps idle during the main loop: the tile's rows of Y into L2,
    // so the epilogue's reads find them there.
    __device__ __forceinline__ void prefetch(int m0, int n0, int bn, int t, int nt) const {
        for (int r = t; r < 128; r += nt)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Y + (size_t)(m0 + r) * ldy + n0),
                         "r"((unsigned)(bn * sizeof(float2)))
                         : "memory");
    }
};

// ---- host side ------------------------------------------------------------
template <int BN>
size_t gemm_smem() {
    constexpr int kStages = stages_for<BN>();
    return 1024 + (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + (2 * kStages + 2) * 8 + 16;
}

template <int BN, class Epi>
cudaError_t launch_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const Epi& epi, int* status,
                        cudaStream_t s) {
    bool dual = false;
    int b_rows = N;
    if constexpr (Epi::kStaged) {
        dual = epi.dual;
        if (dual) b_rows = epi.b_rows;
    }
    const int bn = dual ? BN / 2 : BN;  // output columns per tile
    if (M % kBM || N % bn || K % kBK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (lda * 2) % 16 || (ldb * 2) % 16) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, A, M, K, lda, kBM) || !make_tmap(&tb, B, b_rows, K, ldb, dual ? BN / 2 : BN))
        return cudaErrorInvalidValue;
    const size_t smem = gemm_smem<BN>();
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(N / bn, M / kBM);
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

cudaError_t launch_gemm_accum_pair(const void* A, int lda, const void* B, int ldb, float2* Y, int ldy, int M, int N,
                                   int K, const int* er, const int* fq, int shift, int* status, cudaStream_t s) {
    if (K > 1024) return cudaErrorInvalidValue;  // beyond it the accumulator is no longer exact
    EpiAccumPair epi{Y, ldy, er, fq, shift, false, 0, 0, 0, N};
    if (N % 128 == 0) return launch_gemm<128>(A, lda, B, ldb, M, N, K, epi, status, s);
    return launch_gemm<64>(A, lda, B, ldb, M, N, K, epi, status, s);
}

// Two products of one launch: Y += (A . B1^T) 2^(er + fq - shift2), then
// Y += (A . B2^T) 2^(er + fq - shift1), B1 = B's rows b_row2 .. b_row2 + N - 1 and
// B2 = its rows b_row1 .. (B has b_rows rows); one pass over Y in HBM (the
// second addition finds the rows in L2).  N multiple of 128.
cudaError_t launch_gemm_accum_pair2(const void* A, int lda, const void* B, int ldb, int b_rows, int b_row1, int b_row2,
                                    float2* Y, int ldy, int M, int N, int K, const int* er, const int* fq, int shift1,
                                    int shift2, int* status, cudaStream_t s) {
    if (K > 1024 || N % 128) return cudaErrorInvalidValue;
    if (b_row1 < 0 || b_row2 < 0 || b_row1 + N > b_rows || b_row2 + N > b_rows) return cudaErrorInvalidValue;
    EpiAccumPair epi{Y, ldy, er, fq, shift1, true, b_row1, b_row2, shift2, b_rows};
    return launch_gemm<256>(A, lda, B, ldb, M, N, K, epi, status, s);
}

int* gemm_status_ptr() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gemm_status) != cudaSuccess) return nullptr;
    return static_cast<int*>(p);
}

}  // namespace sa
