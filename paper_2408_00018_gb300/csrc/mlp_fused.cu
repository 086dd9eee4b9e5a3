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
//   warp 0, one lane   TMA: the tile's X (its own buffer, refilled as soon as
//                      layer 1's products are done with it), then the weights
//                      in 128 x 64 blocks through a 3-stage ring (W1, then W2);
//   warp 1, one lane   tcgen05.mma into four 128-column accumulators in tensor
//                      memory (512 columns): layer 1's chunks, then layer 2's,
//                      each waiting for its accumulator to be drained;
//   warps 2-17         the epilogue: warp w reads accumulator lanes 32 (w mod 4)
//                      .. + 31 (its tile rows) and a quarter of each chunk's
//                      columns (b1, b2 and w3 are read from shared memory, one
//                      broadcast per four columns).  Layer 1's chunk j
//                      becomes A1's blocks 2j and 2j + 1 in shared memory while
//                      the next chunks are multiplied; layer 2 waits only for
//                      the A1 blocks it reads.
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

constexpr int kEpiWarps = 16;             // four per TMEM lane quadrant, a quarter of a chunk's columns each
constexpr int kFWarps = 2 + kEpiWarps;
constexpr int kFThreads = 32 * kFWarps;
constexpr int kBlk = 128 * 64 * 2;    // one 128 x 64 BF16 block, 128-byte swizzled: 16 KB
constexpr int kRing = 3;              // weight blocks in flight
constexpr int kXBlocks = 2;           // X: up to 128 input columns
constexpr int kHid = kMlpHidden;      // 512 hidden units per layer
constexpr int kChunks = kHid / 128;   // accumulator chunks per layer (and TMEM buffers)
constexpr int kA1Blocks = kHid / 64;  // A1: 8 blocks of 64 hidden units
static_assert(kHid == 512, "the fused forward pass is laid out for 512 hidden units");

struct FusedBars {
    uint64_t full[kRing], empty[kRing];  // weight ring
    uint64_t xfull, xempty;              // the tile's X has landed / layer 1's products are done with it
    uint64_t accf[kChunks], acce[kChunks];  // accumulator j written / drained
    uint64_t a1f[kChunks];               // A1 blocks 2j, 2j + 1 written (layer 1's chunk j)
    uint64_t a1e;                        // every layer-2 product of the tile has completed
    uint64_t hsf[2], hse[2];             // the head's partial sums handed to the first quarter
    uint64_t mma_done;                   // abort path: every issued product has completed
    uint32_t tmem;
    int abort_flag;
};

constexpr int kHand = 5;  // partial sums a row hands over per chunk (see the head below)
constexpr size_t kFusedSmem = 1024 + (size_t)(kA1Blocks + kXBlocks + kRing) * kBlk + sizeof(FusedBars) +
                              (2 * kHand * 128 + 3 * kHid) * sizeof(float);
static_assert(kFusedSmem <= 232448, "beyond the shared memory of one CTA");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(kFThreads, 1)
    mlp_fused_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                     const __grid_constant__ CUtensorMap tmW2, int xb, int ntiles, const float* __restrict__ b1,
                     const float* __restrict__ b2, const float* __restrict__ w3, float* __restrict__ part,
                     int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA1 = base;                      // 8 blocks
    uint8_t* sX = sA1 + kA1Blocks * kBlk;     // xb blocks
    uint8_t* sW = sX + kXBlocks * kBlk;       // ring
    FusedBars* B = reinterpret_cast<FusedBars*>(sW + kRing * kBlk);
    float* hs = reinterpret_cast<float*>(B + 1);  // [2][kHand][128]
    float* sb1 = hs + 2 * kHand * 128;             // b1, b2, w3 (the epilogue's broadcast reads)
    float* sb2 = sb1 + kHid;
    float* sw3 = sb2 + kHid;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* abort_flag = &B->abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&B->full[s], 1);
            mbar_init(&B->empty[s], 1);
        }
        mbar_init(&B->xfull, 1);
        mbar_init(&B->xempty, 1);
        for (int j = 0; j < kChunks; ++j) {
            mbar_init(&B->accf[j], 1);
            mbar_init(&B->acce[j], kEpiWarps);
            mbar_init(&B->a1f[j], kEpiWarps);
        }
        mbar_init(&B->a1e, 1);
        for (int k = 0; k < 2; ++k) {
            mbar_init(&B->hsf[k], 12);  // the warps of quarters 1-3
            mbar_init(&B->hse[k], 4);   // the warps of quarter 0
        }
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
            // the previous tile's layer 1 is done with the X buffer
            if (t > 0 && !mbar_wait(&B->xempty, (t - 1) & 1, abort_flag)) { ok = false; break; }
            mbar_expect_tx(&B->xfull, xb * kBlk);
            for (int kb = 0; kb < xb; ++kb) tma_load_2d(sX + kb * kBlk, &tmX, &B->xfull, kb * 64, tile * 128);
            x_issued = t;
            for (int layer = 0; layer < 2 && ok; ++layer)
                for (int j = 0; j < kChunks && ok; ++j)
                    for (int kb = 0; kb < (layer == 0 ? xb : kA1Blocks); ++kb, ++g) {
                        const int s = (int)(g % kRing);
                        if (g >= (uint32_t)kRing && !mbar_wait(&B->empty[s], ((g / kRing) - 1) & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&B->full[s], kBlk);
                        tma_load_2d(sW + s * kBlk, layer == 0 ? &tmW1 : &tmW2, &B->full[s], kb * 64, j * 128);
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
        constexpr uint32_t idesc = idesc_bf16(128, 128);
        uint32_t g = 0;
        bool ok = true;
        int t = 0;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
            if (!mbar_wait(&B->xfull, t & 1, abort_flag)) { ok = false; break; }
            for (int layer = 0; layer < 2 && ok; ++layer)
                for (int j = 0; j < kChunks && ok; ++j) {
                    const int use = 2 * t + layer;  // of accumulator j
                    if (use > 0 && !mbar_wait(&B->acce[j], (use - 1) & 1, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int kbs = layer == 0 ? xb : kA1Blocks;
                    for (int kb = 0; kb < kbs; ++kb, ++g) {
                        if (layer == 1 && j == 0 && (kb & 1) == 0 && !mbar_wait(&B->a1f[kb >> 1], t & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        const int s = (int)(g % kRing);
                        if (!mbar_wait(&B->full[s], (g / kRing) & 1, abort_flag)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t da = sdesc(smem_u32((layer == 0 ? sX : sA1) + kb * kBlk));
                        const uint64_t db = sdesc(smem_u32(sW + s * kBlk));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            umma_bf16(tmem + (uint32_t)(j * 128), da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk),
                                      idesc, (kb | kk) != 0 ? 1u : 0u);
                        umma_commit(&B->empty[s]);
                    }
                    if (ok) umma_commit(&B->accf[j]);
                    if (ok && layer == 0 && j == kChunks - 1) umma_commit(&B->xempty);
                }
            if (ok) umma_commit(&B->a1e);
        }
        if (!ok) atomicExch(abort_flag, 1);
        umma_commit(&B->mma_done);  // arrives once every product issued above has completed
        mbar_wait(&B->mma_done, 0);
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads the lanes of quadrant w mod 4 (its 32 tile rows) and
        // the quarter qq = (w - 2) / 4 of each chunk's 128 columns
        const int quad = warp & 3, qq = (warp - 2) >> 2;
        const int r = quad * 32 + lane;  // tile row
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        int t = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
            // layer 1: A1 chunk j = g(acc + b1) as BF16 (columns 32 qq .. 32 qq + 31 of the chunk:
            // block 2j + qq / 2, 16-byte units 4 (qq mod 2) .. + 3 of the row)
            for (int j = 0; j < kChunks && ok; ++j) {
                if (!mbar_wait(&B->accf[j], (2 * t) & 1, abort_flag)) { ok = false; break; }
                // A1 blocks 0.. of this tile overwrite the previous tile's, read by its layer 2
                if (j == 0 && t > 0 && !mbar_wait(&B->a1e, (t - 1) & 1, abort_flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint8_t* blk = sA1 + (2 * j + (qq >> 1)) * kBlk + r * 128;
                float v[32];
                tmem_ld32(tmem + lane_base + (uint32_t)(j * 128 + qq * 32), v);
                const float* bb = sb1 + j * 128 + qq * 32;
                uint32_t pk[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float2 b = *reinterpret_cast<const float2*>(bb + 2 * i);
                    const float2 g = f2_unpack(gelu2(f2_add(f2_pack(v[2 * i], v[2 * i + 1]), f2_pack(b.x, b.y))));
                    pk[i] = pack_bf16x2(g.x, g.y);
                }
                // 16-byte units u .. u + 3 of the row, swizzled by the row's index mod 8
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int u = 4 * (qq & 1) + k;
                    *reinterpret_cast<uint4*>(blk + ((u ^ (r & 7)) << 4)) =
                        make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // for the tensor core's reads
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&B->acce[j]);
                    mbar_arrive(&B->a1f[j]);
                }
            }
            // layer 2 and the head.  The sums of the chunk's eight 16-column groups s0 .. s7
            // (each over its columns in order) combine as (((s0 + s1) + s2) + s3) +
            // (((s4 + s5) + s6) + s7): quarter 0 holds s0, s1 and receives s2, s3 (quarter 1),
            // s4 + s5 (quarter 2) and s6, s7 (quarter 3).
            for (int j = 0; j < kChunks && ok; ++j) {
                if (!mbar_wait(&B->accf[j], (2 * t + 1) & 1, abort_flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float sg[2];
                {
                    float v[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(j * 128 + qq * 32), v);
                    const float* bb = sb2 + j * 128 + qq * 32;
                    const float* ww = sw3 + j * 128 + qq * 32;
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        f32x2_t sum = f2_splat(0.0f);  // even and odd columns of the group, each in order
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int c = 16 * cc + 2 * i;
                            const float2 b = *reinterpret_cast<const float2*>(bb + c);
                            const float2 w = *reinterpret_cast<const float2*>(ww + c);
                            const f32x2_t g = gelu2(f2_add(f2_pack(v[c], v[c + 1]), f2_pack(b.x, b.y)));
                            sum = f2_fma(g, f2_pack(w.x, w.y), sum);
                        }
                        const float2 se = f2_unpack(sum);
                        sg[cc] = se.x + se.y;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&B->acce[j]);
                const int hb = j & 1, use = 2 * t + (j >> 1);  // of hand-over buffer hb
                float* h = hs + hb * kHand * 128 + r;          // [kHand][128] of buffer hb
                if (qq != 0) {
                    if (use > 0 && !mbar_wait(&B->hse[hb], (use - 1) & 1, abort_flag)) { ok = false; break; }
                    if (qq == 1) { h[0] = sg[0]; h[128] = sg[1]; }
                    else if (qq == 2) { h[256] = sg[0] + sg[1]; }
                    else { h[384] = sg[0]; h[512] = sg[1]; }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&B->hsf[hb]);
                } else {
                    if (!mbar_wait(&B->hsf[hb], use & 1, abort_flag)) { ok = false; break; }
                    const float first = ((sg[0] + sg[1]) + h[0]) + h[128];
                    const float second = (h[256] + h[384]) + h[512];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&B->hse[hb]);
                    part[((size_t)tile * 128 + r) * kChunks + j] = first + second;
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
    if (!make_tmap(&tx, X, rows, np, np, 128) || !make_tmap(&t1, W1, kHid, np, np, 128) ||
        !make_tmap(&t2, W2, kHid, kHid, kHid, 128))
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
