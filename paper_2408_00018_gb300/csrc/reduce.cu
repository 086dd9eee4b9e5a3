// reduce.cu -- the synchronisation step of the synchronous approach (Sec. 2.2.2,
// Listing 3): argmin over the chains' final values with the lowest index
// winning ties, restart of every chain from the winner, incumbent update and
// the per-level log.  One grid per level: blockIdx.y = problem; each block
// reduces a contiguous slice, and the last block to finish (last-block-done
// counter; no thread ever waits on another block) combines the partial minima
// and performs the restart.  The temperature is cooled by advancing the
// level index (temperatures are tabulated by repeated multiplication).
#include <cmath>
#include <cstdint>
#include <math_constants.h>

#include "restart.cuh"
#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

__global__ void __launch_bounds__(kArgminThreads) argmin_restart_kernel(const ProbDev* __restrict__ probs, SweepArgs A,
                                                                        int precision) {
    __shared__ VI red[32];
    __shared__ bool last;
    __shared__ double s_old_inc;
    __shared__ double s_red2[64];
    const ProbDev P = probs[blockIdx.y];
    if ((int)blockIdx.x >= P.nblk_argmin) return;
    const int t = threadIdx.x;
    const int64_t C = P.chains;
    const double* F = A.F + P.chain_base;
    const int64_t span = (int64_t)kArgminThreads * kArgminPerThread;
    const int64_t beg = (int64_t)blockIdx.x * span;
    const int64_t end = beg + span < C ? beg + span : C;
    VI a{CUDART_INF, INT64_MAX};
    for (int64_t i = beg + t; i < end; i += kArgminThreads) {
        const double v = F[i];
        if (better(v, i, a.v, a.i)) { a.v = v; a.i = i; }
    }
    a = block_argmin(a, red);
    if (t == 0) {
        P.part_val[blockIdx.x] = a.v;
        P.part_idx[blockIdx.x] = a.i;
        __threadfence();
        const unsigned int ticket = atomicAdd(P.done, 1u);
        last = (ticket == (unsigned int)P.nblk_argmin - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();

    // ---- last block: combine the partial minima --------------------------------
    VI b{CUDART_INF, INT64_MAX};
    const volatile double* pv = P.part_val;
    const volatile int64_t* pi = P.part_idx;
    for (int k = t; k < P.nblk_argmin; k += kArgminThreads) {
        const double v = pv[k];
        const int64_t i = pi[k];
        if (better(v, i, b.v, b.i)) { b.v = v; b.i = i; }
    }
    b = block_argmin(b, red);
    finish_problem_level(P, A, precision, b, s_red2, &s_old_inc);
}

__global__ void level_end_kernel(RunDev* run) {
    if (threadIdx.x == 0 && blockIdx.x == 0) run->level += 1;
}

// Rewind every problem of a handle to level 0.
__global__ void reset_kernel(ProbDev* probs, int num_probs, RunDev* run) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < num_probs) {
        const ProbDev& P = probs[p];
        for (int k = 0; k < kNumScalars; ++k) P.scal[k] = 0.0;
        P.scal[kFBest] = CUDART_INF;
        P.scal[kFInc] = CUDART_INF;
        *P.level_min = 0xFFF0000000000000ull;
        *P.done = 0u;
        *P.accepts = 0ull;
        if (P.rechecks) *P.rechecks = 0ull;
    }
    if (p == 0) {
        run->level = 0;
        run->status = 0;
        run->probs_done = 0;
    }
}

__global__ void stamp_start_kernel(RunDev* run) {
    if (threadIdx.x == 0 && blockIdx.x == 0) run->t_start = globaltimer_ns();
}

__global__ void philox_fill_kernel(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                   int64_t count, uint4* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(make_uint4(c0 + (uint32_t)i, c1, c2, c3), k0, k1);
}

// Stand-alone argmin, pass 1: one (value, index) partial per block into scratch.
__global__ void __launch_bounds__(kArgminThreads) argmin_partial_kernel(const double* __restrict__ F, int64_t count,
                                                                        VI* __restrict__ part) {
    __shared__ VI red[32];
    const int64_t span = (int64_t)kArgminThreads * kArgminPerThread;
    const int64_t beg = (int64_t)blockIdx.x * span;
    const int64_t end = beg + span < count ? beg + span : count;
    VI a{CUDART_INF, INT64_MAX};
    for (int64_t i = beg + threadIdx.x; i < end; i += kArgminThreads) {
        const double v = F[i];
        if (better(v, i, a.v, a.i)) { a.v = v; a.i = i; }
    }
    a = block_argmin(a, red);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// Stand-alone argmin, pass 2: one block combines the partials.
__global__ void __launch_bounds__(kArgminThreads) argmin_final_kernel(const VI* __restrict__ part, int nparts,
                                                                      const double* __restrict__ F, int64_t* idx,
                                                                      double* val) {
    __shared__ VI red[32];
    VI a{CUDART_INF, INT64_MAX};
    for (int k = threadIdx.x; k < nparts; k += kArgminThreads)
        if (better(part[k].v, part[k].i, a.v, a.i)) a = part[k];
    a = block_argmin(a, red);
    if (threadIdx.x == 0) {
        const int64_t i = (a.i == INT64_MAX) ? 0 : a.i;  // all NaN: index 0 (its value is NaN)
        *idx = i;
        *val = F[i];
    }
}

}  // namespace

cudaError_t launch_argmin_restart(const SweepArgs& a, const ProbDev* probs, int num_probs, int max_blocks,
                                  int precision, cudaStream_t s) {
    dim3 grid((unsigned)max_blocks, (unsigned)num_probs);
    argmin_restart_kernel<<<grid, kArgminThreads, 0, s>>>(probs, a, precision);
    return cudaGetLastError();
}

cudaError_t launch_level_end(RunDev* run, cudaStream_t s) {
    level_end_kernel<<<1, 32, 0, s>>>(run);
    return cudaGetLastError();
}

cudaError_t launch_reset(ProbDev* probs, int num_probs, RunDev* run, cudaStream_t s) {
    reset_kernel<<<(num_probs + 127) / 128, 128, 0, s>>>(probs, num_probs, run);
    return cudaGetLastError();
}

cudaError_t launch_stamp_start(RunDev* run, cudaStream_t s) {
    stamp_start_kernel<<<1, 32, 0, s>>>(run);
    return cudaGetLastError();
}

cudaError_t launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                               int64_t count, uint32_t* out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    philox_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(c0, c1, c2, c3, k0, k1, count, reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

int64_t argmin_num_parts(int64_t count) {
    const int64_t span = (int64_t)kArgminThreads * kArgminPerThread;
    return (count + span - 1) / span;
}

cudaError_t launch_argmin_f64(const double* F, int64_t count, int64_t* idx, double* val, void* scratch,
                              cudaStream_t s) {
    const int64_t parts = argmin_num_parts(count);
    VI* part = reinterpret_cast<VI*>(scratch);
    argmin_partial_kernel<<<(unsigned)parts, kArgminThreads, 0, s>>>(F, count, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    argmin_final_kernel<<<1, kArgminThreads, 0, s>>>(part, (int)parts, F, idx, val);
    return cudaGetLastError();
}

}  // namespace sa
