// mlp_fused.cu -- the surrogate's forward pass for inference as one persistent
// tensor-core kernel.  For each tile of 128 rows of the BF16 inputs X [rows x np]:
//   Z1 = X W1^T + b1,  A1 = g(Z1) rounded to BF16           (layer 1)
//   part[row][j] = sum_{h in chunk j} g((A1 W2^T)_h + b2_h) w3_h   (layer 2 + head)
// for the four chunks j of 128 hidden units, g the erf-form GELU of gelu.cuh.
// The hidden activations A1 (128 x 512 BF16, 128 KB) stay in shared memory in
// the 128-byte-swizzled K-major layout that tcgen05.mma reads, instead of
// going to HBM and back between two GEMMs.  The arithmetic is that of the two
// GEMMs with the bias + GELU and bias + GELU + head epilogues of gemm_tc.cu:
// the same FP32 accumulators, the same BF16 rounding of A1, and the head's
// sums in the same order (per 16 columns the even and the odd ones, each in
// order, then even + odd; the four 16-column groups of each column half in
// turn; then first half + second half).
//
// Roles (one CTA of 18 warps per SM, persistent over the row tiles):
//   warp 0, one lane   TMA: the tile's X (into A1's last blocks, free once the
//                      previous tile's layer 2 is done with them), then the
//                      weights in 256 x 64 blocks through a 2-stage ring (W1,
//                      then W2);
//   warp 1, one lane   tcgen05.mma, 128 x 256 x 16 per instruction, into two
//                      256-column accumulators in tensor memory (512 columns):
//                      a "pair" is 256 hidden units, two chunks; layer 1's two
//                      pairs, then layer 2's, each waiting for its accumulator
//                      to be drained;
//   warps 2-17         the epilogue: warp w reads accumulator lanes 32 (w mod 4)
//                      .. + 31 (its tile rows) and a quarter of each pair's
//                      columns, i.e. one half of a chunk (b1, b2 and w3 are
//                      read from shared memory as broadcasts).  Layer 1's pair p
//                      becomes A1's blocks 4p .. 4p + 3 in shared memory while
//                      the next pair is multiplied; layer 2 waits only for the
//                      A1 blocks it reads.
// Products of 128 x 256 move 12 KB of operands per 2^19 multiply-adds where
// 128 x 128 ones move 8 KB per 2^18; the MMAs of this kernel are bound by that
// operand traffic (111 us with 128-column products, 90 us with these, both
// without the GELU work).
// Every wait is bounded (as in gemm_tc.cu): on expiry the kernel records
// SA_ETIMEOUT in the status word, every role stops, the copies and matrix
// operations already issued are waited for (bounded), and tensor memory is freed.
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

constexpr int kEpiWarps = 16;               // four per TMEM lane quadrant, a quarter of a pair's columns each
constexpr int kFWarps = 2 + kEpiWarps;
constexpr int kFThreads = 32 * kFWarps;
constexpr int kBlk = 128 * 64 * 2;          // one 128 x 64 BF16 block, 128-byte swizzled: 16 KB
constexpr int kWBlk = 2 * kBlk;             // one 256 x 64 weight block: 32 KB
constexpr int kRing = 2;                    // weight blocks in flight
constexpr int kHid = kMlpHidden;            // 512 hidden units per layer
constexpr int kPairs = kHid / 256;          // accumulators (256 columns each) per layer
constexpr int kA1Blocks = kHid / 64;        // A1: 8 blocks of 64 hidden units
static_assert(kHid == 512, "the fused forward pass is laid out for 512 hidden units");

struct FusedBars {
    uint64_t full[kRing], empty[kRing];  // weight ring
    uint64_t xfull;                      // the tile's X has landed
    uint64_t accf[kPairs], acce[kPairs];  // accumulator p written / drained
    uint64_t a1f[kPairs];                // A1 blocks 4p .. 4p + 3 written (layer 1's pair p)
    uint64_t a1e;                        // every layer-2 product of the tile has completed
    uint64_t hsf[kPairs], hse[kPairs];   // the head's second-half sums handed over / taken
    uint64_t mma_done;                   // abort path: every issued product has completed
    uint32_t tmem;
    int abort_flag;
};

constexpr size_t kFusedSmem = 1024 + (size_t)kA1Blocks * kBlk + (size_t)kRing * kWBlk + sizeof(FusedBars) +
                              (kPairs * 2 * 128 + 3 * kHid) * sizeof(float);
static_assert(kFusedSmem <= 232448, "beyond the shared memory of one CTA");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// 32 accumulator columns of the warp's 32 lanes, without the wait.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// 64 accumulator columns (two loads, one wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
    uint32_t r[64];
    tmem_ld32_async(taddr, r);
    tmem_ld32_async(taddr + 32u, r + 32);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 64; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(kFThreads, 1)
    mlp_fused_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                     const __grid_constant__ CUtensorMap tmW2, int xb, int ntiles, const float* __restrict__ b1,
                     const float* __restrict__ b2, const float* __restrict__ w3, float* __restrict__ part,
                     int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA1 = base;                      // 8 blocks; X occupies the last xb of them
    uint8_t* sW = sA1 + kA1Blocks * kBlk;     // ring
    FusedBars* B = reinterpret_cast<FusedBars*>(sW + kRing * kWBlk);
    float* hs = reinterpret_cast<float*>(B + 1);  // [kPairs][2][128]
    float* sb1 = hs + kPairs * 2 * 128;            // b1, b2, w3 (the epilogue's broadcast reads)
    float* sb2 = sb1 + kHid;
    float* sw3 = sb2 + kHid;
    uint8_t* sX = sA1 + (kA1Blocks - xb) * kBlk;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* abort_flag = &B->abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&B->full[s], 1);
            mbar_init(&B->empty[s], 1);
        }
        mbar_init(&B->xfull, 1);
        for (int p = 0; p < kPairs; ++p) {
            mbar_init(&B->accf[p], 1);
            mbar_init(&B->acce[p], kEpiWarps);
            mbar_init(&B->a1f[p], kEpiWarps);
            mbar_init(&B->hsf[p], kEpiWarps / 2);  // the warps of the second chunk halves
            mbar_init(&B->hse[p], kEpiWarps / 2);  // the warps of the first halves
        }
        mbar_init(&B->a1e, 1);
        mbar_init(&B->mma_done, 1);
        B->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        sb1[i] = b1[i];
        sb2[i] = b2[i];
        sw3[i] = w3[i];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&B->tmem)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = B->tmem;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        uint32_t g = 0;  // weight blocks issued
        bool ok = true;
        int t = 0, x_issued = -1;  // the last tile whose X was issued
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
            // X lives in A1's last blocks: wait until the previous tile's layer 2 is done with them
            if (t > 0 && !mbar_wait(&B->a1e, (t - 1) & 1, abort_flag)) { ok = false; break; }
            mbar_expect_tx(&B->xfull, xb * kBlk);
            for (int kb = 0; kb < xb; ++kb) tma_load_2d(sX + kb * kBlk, &tmX, &B->xfull, kb * 64, tile * 128);
            x_issued = t;
            for (int layer = 0; layer < 2 && ok; ++layer)
                for (int p = 0; p < kPairs && ok; ++p)
                    for (int kb = 0; kb < (layer == 0 ? xb : kA1Blocks); ++kb, ++g) {
                        const int s = (int)(g % kRing);
                        if (g >= (uint32_t)kRing && !mbar_wait(&B->empty[s], ((g / kRing) - 1) & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&B->full[s], kWBlk);
                        tma_load_2d(sW + s * kWBlk, layer == 0 ? &tmW1 : &tmW2, &B->full[s], kb * 64, p * 256);
                    }
        }
        if (!ok) {
            atomicExch(abort_flag, 1);
            // the copies still in flight land before the CTA exits (bounded)
            for (uint32_t q = (g > (uint32_t)kRing ? g - kRing : 0); q < g; ++q)
                mbar_wait(&B->full[q % kRing], (q / kRing) & 1);
            if (x_issued >= 0) mbar_wait(&B->xfull, x_issued & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t idesc = idesc_bf16(128, 256);
        uint32_t g = 0;
        bool ok = true;
        int t = 0;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
            if (!mbar_wait(&B->xfull, t & 1, abort_flag)) { ok = false; break; }
            for (int layer = 0; layer < 2 && ok; ++layer)
                for (int p = 0; p < kPairs && ok; ++p) {
                    const int use = 2 * t + layer;  // of accumulator p
                    if (use > 0 && !mbar_wait(&B->acce[p], (use - 1) & 1, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int kbs = layer == 0 ? xb : kA1Blocks;
                    for (int kb = 0; kb < kbs; ++kb, ++g) {
                        // layer 2's first pair reads A1 blocks 4q .. 4q + 3 once layer 1's pair q is written
                        if (layer == 1 && p == 0 && (kb & 3) == 0 && !mbar_wait(&B->a1f[kb >> 2], t & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        const int s = (int)(g % kRing);
                        if (!mbar_wait(&B->full[s], (g / kRing) & 1, abort_flag)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t da = sdesc(smem_u32((layer == 0 ? sX : sA1) + kb * kBlk));
                        const uint64_t db = sdesc(smem_u32(sW + s * kWBlk));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            umma_bf16(tmem + (uint32_t)(p * 256), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk),
                                      idesc, (kb | kk) != 0 ? 1u : 0u);
                        umma_commit(&B->empty[s]);
                    }
                    if (ok) umma_commit(&B->accf[p]);
                }
            if (ok) umma_commit(&B->a1e);
        }
        if (!ok) atomicExch(abort_flag, 1);
        umma_commit(&B->mma_done);  // arrives once every product issued above has completed
        mbar_wait(&B->mma_done, 0);
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads the lanes of quadrant w mod 4 (its 32 tile rows) and the
        // columns 64 qq .. 64 qq + 63 of each pair, qq = (w - 2) / 4: half qq mod 2 of chunk
        // 2p + qq / 2, hidden units 256 p + 64 qq .. (A1 block 4p + qq)
        const int quad = warp & 3, qq = (warp - 2) >> 2;
        const int r = quad * 32 + lane;  // tile row
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        int t = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
            // layer 1: A1 = g(acc + b1) as BF16, the row's 128 bytes of block 4p + qq
            for (int p = 0; p < kPairs && ok; ++p) {
                if (!mbar_wait(&B->accf[p], 0, abort_flag)) { ok = false; break; }  // use 2t: even
                // A1 blocks of this tile overwrite the previous tile's, read by its layer 2
                if (p == 0 && t > 0 && !mbar_wait(&B->a1e, (t - 1) & 1, abort_flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float v[64];
                tmem_ld64(tmem + lane_base + (uint32_t)(p * 256 + qq * 64), v);
                const float* bb = sb1 + p * 256 + qq * 64;
                uint8_t* row = sA1 + (4 * p + qq) * kBlk + r * 128;
#pragma unroll
                for (int u = 0; u < 8; ++u) {  // 16-byte unit u of the row: 8 hidden units
                    uint32_t pk[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int c = 8 * u + 2 * i;
                        const float2 b = *reinterpret_cast<const float2*>(bb + c);
                        const float2 g2 = f2_unpack(gelu2(f2_add(f2_pack(v[c], v[c + 1]), f2_pack(b.x, b.y))));
                        pk[i] = pack_bf16x2(g2.x, g2.y);
                    }
                    // swizzled by the row's index mod 8
                    *reinterpret_cast<uint4*>(row + ((u ^ (r & 7)) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // for the tensor core's reads
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&B->acce[p]);
                    mbar_arrive(&B->a1f[p]);
                }
            }
            // layer 2 and the head: the warp's half of chunk 2p + qq / 2 summed over its four
            // 16-column groups in order; part = first half + second half
            for (int p = 0; p < kPairs && ok; ++p) {
                if (!mbar_wait(&B->accf[p], 1, abort_flag)) { ok = false; break; }  // use 2t + 1: odd
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float h = 0.0f;
                {
                    float v[64];
                    tmem_ld64(tmem + lane_base + (uint32_t)(p * 256 + qq * 64), v);
                    const float* bb = sb2 + p * 256 + qq * 64;
                    const float* ww = sw3 + p * 256 + qq * 64;
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        f32x2_t sum = f2_splat(0.0f);  // even and odd columns of the group, each in order
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int c = 16 * cc + 2 * i;
                            const float2 b = *reinterpret_cast<const float2*>(bb + c);
                            const float2 w = *reinterpret_cast<const float2*>(ww + c);
                            const f32x2_t g2 = gelu2(f2_add(f2_pack(v[c], v[c + 1]), f2_pack(b.x, b.y)));
                            sum = f2_fma(g2, f2_pack(w.x, w.y), sum);
                        }
                        const float2 se = f2_unpack(sum);
                        h += se.x + se.y;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&B->acce[p]);
                float* hp = hs + (p * 2 + (qq >> 1)) * 128 + r;  // this chunk's hand-over slot of row r
                if (qq & 1) {
                    if (t > 0 && !mbar_wait(&B->hse[p], (t - 1) & 1, abort_flag)) { ok = false; break; }
                    *hp = h;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&B->hsf[p]);
                } else {
                    if (!mbar_wait(&B->hsf[p], t & 1, abort_flag)) { ok = false; break; }
                    const float second = *hp;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&B->hse[p]);
                    part[((size_t)tile * 128 + r) * 4 + 2 * p + (qq >> 1)] = h + second;
                }
            }
        }
        if (!ok) atomicExch(abort_flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int*)abort_flag && status) atomicCAS(status, 0, 4);  // SA_ETIMEOUT
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

}  // namespace

bool mlp_fused_ok(int np, int rows) { return (np == 64 || np == 128) && rows > 0 && rows % 128 == 0; }

// part [rows x 4] (FP32) from X (BF16 [rows x np]), W1 (BF16 [512 x np]), W2 (BF16 [512 x 512]).
cudaError_t launch_mlp_fused(const void* X, int np, int rows, const void* W1, const void* W2, const float* b1,
                             const float* b2, const float* w3, float* part, int* status, cudaStream_t s) {
    if (!mlp_fused_ok(np, rows)) return cudaErrorInvalidValue;
    if (((uintptr_t)X & 15) || ((uintptr_t)W1 & 15) || ((uintptr_t)W2 & 15)) return cudaErrorInvalidValue;
    CUtensorMap tx, t1, t2;
    if (!make_tmap(&tx, X, rows, np, np, 128) || !make_tmap(&t1, W1, kHid, np, np, 256) ||
        !make_tmap(&t2, W2, kHid, kHid, kHid, 256))
        return cudaErrorInvalidValue;
    static bool attr = false;
    static int sms = 0;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kFusedSmem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = rows / 128;
    const int grid = ntiles < sms ? ntiles : sms;
    mlp_fused_kernel<<<grid, kFThreads, kFusedSmem, s>>>(tx, t1, t2, np / 64, ntiles, b1, b2, w3, part, status);
    return cudaGetLastError();
}

}  // namespace sa
