// restart.cuh -- the end of a level for one problem (Sec. 2.2.2, Listing 3):
// the restart point, incumbent and per-level log from the level's best chain.
// Used by the argmin/restart kernel's last block and by the batched level
// kernel's last block of each problem.
#pragma once
#include <cmath>
#include <cstdint>
#include <math_constants.h>

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

struct VI {
    double v;
    int64_t i;
};

// (v, i) better than (w, j): smaller value, then smaller index; NaN never wins.
__device__ __forceinline__ bool better(double v, int64_t i, double w, int64_t j) {
    return v < w || (v == w && i < j);
}

__device__ __forceinline__ VI warp_argmin(VI a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, a.v, o);
        const long long j = __shfl_xor_sync(0xffffffffu, (long long)a.i, o);
        if (better(w, j, a.v, a.i)) { a.v = w; a.i = j; }
    }
    return a;
}

// Block argmin; result valid in every thread.
__device__ VI block_argmin(VI a, VI* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_argmin(a);
    __syncthreads();
    if (lane == 0) red[wid] = a;
    __syncthreads();
    VI b = red[0];
    for (int k = 1; k < nw; ++k)
        if (better(red[k].v, red[k].i, b.v, b.i)) b = red[k];
    return b;
}

__device__ __forceinline__ long long globaltimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The rest of the level's end for one problem, by every thread of one block:
// b = the level's best (FP64 value, chain) of the problem; restart point,
// incumbent, Ackley's sums of the restart point, scalars, per-level log, and
// the level's candidate threshold and block counter reset for the next level.
// s_red2: 64 doubles of shared memory; s_old_inc: one double of shared memory.
__device__ void finish_problem_level(const ProbDev& P, const SweepArgs& A, int precision, VI b, double* s_red2,
                                     double* s_old_inc) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int64_t C = P.chains;
    const int level = A.run->level;
    if (t == 0) *s_old_inc = P.scal[kFInc];
    __syncthreads();
    const double old_inc = *s_old_inc;
    const bool ok = (b.i != INT64_MAX) && isfinite(b.v);
    const int n = P.n;
    if (ok) {
        const bool improve = b.v < old_inc;
        double p1 = 0.0, p2 = 0.0;
        for (int k = t; k < n; k += nt) {
            double xb;
            if (precision == 0) {
                xb = A.X64[P.x_base + (size_t)k * (size_t)C + (size_t)b.i];
                P.x_best64[k] = xb;
            } else {
                const float xf = A.X32[P.x_base + (size_t)k * (size_t)C + (size_t)b.i];
                P.x_best32[k] = xf;
                xb = (double)xf;
            }
            if (improve) P.x_inc[k] = xb;
            if (P.cost == kAckley) {
                p1 += xb * xb;
                p2 += cos(6.283185307179586 * xb);
            }
        }
        if (P.cost == kAckley) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                p1 += __shfl_xor_sync(0xffffffffu, p1, o);
                p2 += __shfl_xor_sync(0xffffffffu, p2, o);
            }
            if ((t & 31) == 0) { s_red2[t >> 5] = p1; s_red2[32 + (t >> 5)] = p2; }
            __syncthreads();
            if (t == 0) {
                double q1 = 0.0, q2 = 0.0;
                for (int k = 0; k < nt / 32; ++k) { q1 += s_red2[k]; q2 += s_red2[32 + k]; }
                P.scal[kS1] = q1;
                P.scal[kS2] = q2;
            }
        }
        if (t == 0) {
            P.scal[kFBest] = b.v;
            if (improve) P.scal[kFInc] = b.v;
        }
    } else if (t == 0) {
        atomicCAS(&A.run->status, 0, 5);  // SA_ENUMERIC (the first error raised in a run is kept)
    }
    if (t == 0) {
        P.log_argmin[level] = ok ? b.i : -1;
        P.log_f[level] = ok ? b.v : CUDART_NAN;
        P.log_finc[level] = (ok && b.v < old_inc) ? b.v : old_inc;
        P.log_t[level] = globaltimer_ns();
        *P.level_min = 0xFFF0000000000000ull;  // ordered key of +inf
        *P.done = 0u;
    }
}

}  // namespace
}  // namespace sa
