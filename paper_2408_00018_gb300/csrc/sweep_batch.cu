// sweep_batch.cu -- one launch per temperature level for a batch of independent
// FP32 problems of uneven dimension and chain count (the synchronous SA of Sec.
// 2.2.2 run for many problems at once, each with its own restart).
//
// The launch holds every tile of every problem, largest problems first, in
// blocks of 256 threads whose shared memory is sized for the largest tile.  A
// tile's layout follows its problem: separable costs without global sums take
// the group layout (2 lanes per chain up to n = 128, 4 up to 256, 8 above: 128,
// 64 or 32 chains per tile, about 64 KiB of state each); Ackley, whose running
// sums tie every step of a chain to the previous one, takes one chain per
// thread with as many chains as 64 KiB of state hold, and above n = 128, where
// that leaves most warps without a chain, those warps draw the chains' Philox
// blocks, deviates and thresholds ahead into a shared-memory ring, so that a
// chain's thread runs only the dependent part of its steps.  So every tile holds
// about the same shared memory, three blocks fit on an SM whatever their
// problem, and the block scheduler balances the uneven problems over the GPU
// in one grid.
//
// The end of a problem's level needs no further launch: each tile reduces the
// FP64 values of its chains to one (value, chain) partial, and the last tile of
// the problem to finish (a last-block-done counter; no block waits for another)
// combines the partials, writes the restart point, incumbent and log of the
// problem; the last problem to finish advances the level index, which cools T.
#include "restart.cuh"
#include "sweep_group.cuh"
#include "sweep_thread.cuh"

namespace sa {
namespace {

constexpr size_t kTileStateBytes = 64 * 1024;  // chain state per tile (about three blocks per SM)

// Shared memory of a one-chain-per-thread tile of S chains (the carve-up of sweep_f32.cu).
__host__ __device__ inline size_t thread_tile_bytes(int n, int S) {
    return 72 * sizeof(double) + (kMaxBlock + 4) * sizeof(int) + ((size_t)n * S + 3 * (size_t)n) * sizeof(float);
}

// One chain per thread, one step at a time (the register budget of this kernel
// is sized for the group layout); S = the tile's chain count.  PD: the warps past the
// chains draw the chains' randomness ahead (sweep_tile's producer/consumer form).
template <bool PD>
__device__ void thread_tile(const SweepArgs& A, const ProbDev& P, const WorkItem& it, int S, int level,
                            unsigned char* smem_raw) {
    const int n = P.n;
    double* red = reinterpret_cast<double*>(smem_raw);
    int* cand = reinterpret_cast<int*>(smem_raw + 72 * sizeof(double));
    int* ncand = cand + kMaxBlock;
    float* xs = reinterpret_cast<float*>(smem_raw + 72 * sizeof(double) + (kMaxBlock + 4) * sizeof(int));
    float* slo = xs + (size_t)n * S;
    float* shi = slo + n;
    float* ssig = shi + n;
    float* ring = ssig + n;
    const bool ub = P.uniform != 0, up = A.proposal == 1;
#define SA_TILE(COST)                                                                                                 \
    (ub ? (up ? sweep_tile<COST, true, 1, true, 1, PD>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, ring)   \
              : sweep_tile<COST, true, 1, false, 1, PD>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, ring)) \
        : (up ? sweep_tile<COST, false, 1, true, 1, PD>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, ring)  \
              : sweep_tile<COST, false, 1, false, 1, PD>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, ring)))
    switch (P.cost) {
    case kSchwefel: SA_TILE(kSchwefel); break;
    case kRastrigin: SA_TILE(kRastrigin); break;
    case kAckley: SA_TILE(kAckley); break;
    case kRosenbrock: SA_TILE(kRosenbrock); break;
    default: if (threadIdx.x == 0) A.run->status = 1; break;
    }
#undef SA_TILE
}

__global__ void __launch_bounds__(kBatchThreads, 3) batch_level_kernel(SweepArgs A, int num_probs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ GroupShared gsh;
    __shared__ VI red_vi[32];
    __shared__ double s_red2[64];
    __shared__ double s_old_inc;
    __shared__ bool last;
    const WorkItem it = A.items[blockIdx.x];
    const ProbDev& P = A.probs[it.problem];
    const int level = A.run->level;
    switch (it.lanes) {
    case 2: group_tile<2, false>(A, P, it, level, smem_raw, gsh); break;
    case 4: group_tile<4, false>(A, P, it, level, smem_raw, gsh); break;
    case 8: group_tile<8, false>(A, P, it, level, smem_raw, gsh); break;
    case 1: thread_tile<true>(A, P, it, it.count, level, smem_raw); break;
    default: thread_tile<false>(A, P, it, it.count, level, smem_raw); break;
    }
    // this tile's partial argmin over the FP64 values its chains were given
    __syncthreads();
    VI a{CUDART_INF, INT64_MAX};
    const double* F = A.F + P.chain_base;
    for (int j = threadIdx.x; j < it.count; j += blockDim.x) {
        const int64_t i = it.c0 + j;
        const double v = F[i];
        if (better(v, i, a.v, a.i)) { a.v = v; a.i = i; }
    }
    a = block_argmin(a, red_vi);
    if (threadIdx.x == 0) {
        P.part_val[it.slot] = a.v;
        P.part_idx[it.slot] = a.i;
        __threadfence();
        last = atomicAdd(P.done, 1u) == (unsigned)P.items - 1u;
    }
    __syncthreads();
    if (!last) return;
    // ---- the problem's last tile: its level ends here
    __threadfence();
    VI b{CUDART_INF, INT64_MAX};
    const volatile double* pv = P.part_val;
    const volatile int64_t* pi = P.part_idx;
    for (int k = threadIdx.x; k < P.items; k += blockDim.x) {
        const double v = pv[k];
        const int64_t i = pi[k];
        if (better(v, i, b.v, b.i)) { b.v = v; b.i = i; }
    }
    b = block_argmin(b, red_vi);
    finish_problem_level(P, A, 1, b, s_red2, &s_old_inc);  // (resets the tile counter)
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&A.run->probs_done, 1) == num_probs - 1) {  // the batch's last problem: cool
            A.run->probs_done = 0;
            A.run->level = level + 1;
        }
    }
}

}  // namespace

// A problem's tile layout and capacity (chains per tile) in the batched level kernel.
int batch_tile_capacity(int cost, int n, int* lanes) {
    if (cost == kSchwefel || cost == kRastrigin || cost == kRosenbrock) {
        *lanes = n <= 128 ? 2 : (n <= 256 ? 4 : 8);
        return kBatchThreads / *lanes;
    }
    // Ackley: one chain per thread; where the state leaves most warps without a
    // chain (n > 128: 64 chains or fewer), those warps draw the chains' randomness
    // ahead (lanes = 1).  Up to n = 128 the plain tile is faster (measured).
    if (n <= 128) {
        *lanes = 0;
        int S = (int)(kTileStateBytes / (4 * (size_t)n));
        S = S >= kBatchThreads ? kBatchThreads : (S / 32) * 32;
        return S < 32 ? 32 : S;
    }
    *lanes = 1;
    const int S = (int)(kTileStateBytes / (4 * (size_t)n + kPdRingBytes(1)));
    return S < 1 ? 1 : S;
}

size_t batch_smem_bytes(int cost, int n) {
    int lanes = 0;
    const int cap = batch_tile_capacity(cost, n, &lanes);
    if (lanes > 1) return ((size_t)cap * (n + 1) + 3 * (size_t)n) * sizeof(float);
    return thread_tile_bytes(n, cap) + (lanes == 1 ? kPdRingBytes(cap) : 0);
}

cudaError_t batch_set_smem(size_t bytes) {
    static size_t current = 0;  // the limit only grows, so earlier graphs stay valid
    if (bytes <= current) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(batch_level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

cudaError_t launch_batch_level(const SweepArgs& a, int num_items, int num_probs, size_t smem, cudaStream_t s) {
    batch_level_kernel<<<num_items, kBatchThreads, smem, s>>>(a, num_probs);
    return cudaGetLastError();
}

}  // namespace sa
