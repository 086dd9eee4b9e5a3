// sweep_rot.cu -- Metropolis sweep for rotated costs f(x) = F(y), y = Q x
// (orthogonal Q), one Markov chain per warp.
//
// A single-coordinate move x_d -> x_d + delta changes every rotated
// coordinate: y' = y + delta Q[:, d].  Each warp keeps its chain's x (FP32)
// and y in shared memory; y is a double-float pair (y_hi + y_lo) updated by
// the rank-1 correction with Q split into FP32 hi + lo parts, so that it
// follows the FP64 product Q x to about 2^-46 of |y| per update.  Lanes own
// the rotated coordinates i = lane + 32 j.
//
// Energy difference in FP32 with a rigorous bound B on its error (relative to
// real arithmetic on the pair state y_hi + y_lo and the exact move):
//   rotated Rastrigin, per coordinate (Delta_i = delta Q_id):
//     g(y + Delta) - g(y) = Delta (2y + Delta) + 20 sin(2 pi (y + Delta/2)) sin(pi Delta)
//   (product-to-sum form; sin(pi Delta) by an odd Taylor polynomial where
//   |pi Delta| < 1/2), so the error is proportional to |Delta|;
//   rotated Schwefel: h(y + Delta) - h(y), both terms from y_hi, scaled by -1/n.
// Metropolis test (Eq. of the acceptance probability, k_B = 1): accept iff
// dF <= 0 or u3 < exp(-dF/T), i.e. dF < tau = -T ln u3.  When
// |dF - tau| <= B (+ the error of tau) the decision is re-taken in FP64 from
// y_hi + y_lo and the FP64 Q, so every decision equals the FP64 decision on
// the pair state.  Level 0 starts from X0 and Y0 = X0 Q^T (FP64, rot_prep.cu);
// later levels start from x_best and y_best = Q x_best, F(y_best) computed
// once per level by the restart transform.
#include <cmath>
#include <cstdint>
#include <math_constants.h>

#include "rot_step.cuh"
#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kWarpsR = 4;
constexpr int kBlockR = 32 * kWarpsR;

template <int COST>
__device__ __forceinline__ double f_from_sum(double s, int n) {
    return COST == kRotRastrigin ? 10.0 * (double)n + s : -(s / (double)n);
}

struct RotEnd {
    double Fa, ec;
    unsigned nacc, nre;
};

template <int COST>
__device__ RotEnd rot_chain(const SweepArgs& A, const ProbDev& P, int64_t c, int level, float* x, float* yh, float* yl) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    const int64_t gc = P.chain_base + c;
    const double T = A.T_tab[level];
    const float sl = (float)A.s_tab[level];

    // ---- state at the start of the level
    double Fs;
    float edrift = 0.0f;  // bound on the FP64 value drift of the pair updates (the same in every lane)
    if (level == 0 || own_start(A, level)) {  // own-start levels continue from the chain's own x, y
        const float* xr = P.x0 + (size_t)c * n;
        const float2* yr = P.y0 + (size_t)c * n;
        double part = 0.0;
        for (int k = lane; k < n; k += 32) {
            x[k] = xr[k];
            const float2 v = yr[k];
            yh[k] = v.x;
            yl[k] = v.y;
            part += rot_g64<COST>((double)v.x + (double)v.y);
        }
        Fs = f_from_sum<COST>(rot_wsumd(part), n);
    } else {
        for (int k = lane; k < n; k += 32) {
            x[k] = P.x_best32[k];
            yh[k] = P.ybest_hi[k];
            yl[k] = P.ybest_lo[k];
        }
        Fs = P.scal[kFRot];
    }
    __syncwarp();

    const float neg_T_ln2 = (float)(-T * 0.69314718055994531);
    const float tau_abs = (float)(T * 4.0e-7);
    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    uint32_t* mybits = tracing ? A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)gc) * (size_t)A.words : nullptr;
    double dS = 0.0, e = 0.0;
    unsigned nacc = 0, nre = 0, bw = 0;
    for (int s = 0; s < A.L; ++s) {
        // randomness of step s (the same block in every lane)
        const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)level, (uint32_t)c + P.cid0, P.pid), A.key0, A.key1);
        const RotMove mv = rot_propose(w, x, P, sl, A.boundary, A.proposal, neg_T_ln2);
        const int d = mv.d;
        const float xo = mv.xo, xp = mv.xp, dh = mv.dh, dl = mv.dl, tau = mv.tau;
        // ---- FP32 energy difference and its error bound
        float dF, B;
        rot_eval32<COST>(P, yh, yl, d, dh, n, lane, dF, B);
        for (int rep = 1; rep < A.cost_repeat; ++rep) {  // the expensive-cost knob: the same evaluation again
            float dF2, B2;
            rot_eval32<COST>(P, yh, yl, d, dh + opaque_zero(), n, lane, dF2, B2);
            asm volatile("" ::"f"(dF2), "f"(B2));
        }
        B += 1.0e-6f * fabsf(tau) + tau_abs;  // with the error of tau
        bool acc;
        double dF_used = (double)dF;
        double e_step = (double)B;
        if (dF < tau - B) {
            acc = true;
        } else if (dF > tau + B) {
            acc = false;
        } else {
            // ---- FP64 re-check of a decision inside the bound
            const double dF64 = rot_eval64<COST>(P, yh, yl, d, xp, xo, n, lane, e_step);
            acc = (dF64 <= 0.0) || (u23d(w.w) < exp(-dF64 / T));
            dF_used = dF64;
            ++nre;
        }
        if (acc) {
            if (lane == 0) x[d] = xp;
            rot_update<COST>(P, yh, yl, d, dh, dl, n, lane, edrift);
            dS += dF_used;
            e += e_step;
            ++nacc;
        }
        __syncwarp();
        if (tracing) {
            bw |= (acc ? 1u : 0u) << (s & 31);
            if (((s & 31) == 31 || s == A.L - 1) && lane == 0) mybits[s >> 5] = bw;
            if ((s & 31) == 31) bw = 0;
        }
    }
    RotEnd r;
    r.Fa = Fs + dS;
    r.ec = e + (double)edrift + 1e-13 * (fabs(Fs) + fabs(dS) + 1.0);
    r.nacc = nacc;
    r.nre = nre;
    return r;
}

template <int COST>
__device__ void rot_finish(const SweepArgs& A, const ProbDev& P, int64_t c, int level, const float* x, const float* yh,
                           const float* yl, const RotEnd& r, double M) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    const int64_t gc = P.chain_base + c;
    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    const bool finite = isfinite(r.Fa);
    if (finite && (tracing || level == A.full_level || A.crossover || r.Fa - r.ec <= M)) {
        double part = 0.0;
        for (int i = lane; i < n; i += 32) part += rot_g64<COST>((double)yh[i] + (double)yl[i]);
        part = rot_wsumd(part);
        if (lane == 0) A.F[gc] = f_from_sum<COST>(part, n);
        float* dst = A.X32 + P.x_base + c;
        for (int k = lane; k < n; k += 32) dst[(size_t)k * (size_t)P.chains] = x[k];
    } else if (lane == 0) {
        A.F[gc] = finite ? CUDART_INF : CUDART_NAN;
    }
    if (keep_states(A)) {  // every chain's x and y pair may start its next level
        float* xr = const_cast<float*>(P.x0) + (size_t)c * n;
        float2* yr = const_cast<float2*>(P.y0) + (size_t)c * n;
        for (int k = lane; k < n; k += 32) {
            xr[k] = x[k];
            yr[k] = make_float2(yh[k], yl[k]);
        }
    }
}

template <int COST>
__device__ void rot_tile(const SweepArgs& A, const ProbDev& P, const WorkItem& it, float* smem) {
    __shared__ double block_hi[kWarpsR];
    __shared__ double block_M;
    __shared__ unsigned block_acc, block_re;
    const int level = A.run->level;
    const int n = P.n;
    const int warp = threadIdx.x >> 5;
    float* base = smem + (size_t)warp * 3 * n;
    float *x = base, *yh = base + n, *yl = base + 2 * n;
    if (threadIdx.x == 0) { block_acc = 0u; block_re = 0u; }
    if (threadIdx.x < kWarpsR) block_hi[threadIdx.x] = CUDART_INF;
    __syncthreads();
    const bool mine = warp < it.count;
    const int64_t c = it.c0 + warp;
    RotEnd r{0.0, 0.0, 0u, 0u};
    if (mine) {
        r = rot_chain<COST>(A, P, c, level, x, yh, yl);
        if ((threadIdx.x & 31) == 0) block_hi[warp] = isfinite(r.Fa) ? r.Fa + r.ec : CUDART_INF;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bmin = block_hi[0];
        for (int w2 = 1; w2 < kWarpsR; ++w2) bmin = fmin(bmin, block_hi[w2]);
        double M = bmin;
        if (bmin < CUDART_INF) M = fmin(M, key_dbl(atomicMin(P.level_min, dbl_key(bmin))));
        else M = key_dbl(*(volatile unsigned long long*)P.level_min);
        block_M = M;
    }
    __syncthreads();
    if (mine) {
        rot_finish<COST>(A, P, c, level, x, yh, yl, r, block_M);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&block_acc, r.nacc);
            atomicAdd(&block_re, r.nre);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (block_acc) atomicAdd(P.accepts, (unsigned long long)block_acc);
        if (block_re) atomicAdd(P.rechecks, (unsigned long long)block_re);
    }
}

// COSTS: the rotated costs the launch's problems use (bit 0 Rastrigin, bit 1
// Schwefel), so that a launch of one cost gets a register allocation of its own.
template <int COSTS>
__global__ void __launch_bounds__(kBlockR) sweep_rot_kernel(SweepArgs A) {
    extern __shared__ __align__(16) float smem_rot[];
    const WorkItem it = A.items[blockIdx.x];
    const ProbDev& P = A.probs[it.problem];
    if (COSTS == 1) rot_tile<kRotRastrigin>(A, P, it, smem_rot);
    else if (COSTS == 2) rot_tile<kRotSchwefel>(A, P, it, smem_rot);
    else if (P.cost == kRotRastrigin) rot_tile<kRotRastrigin>(A, P, it, smem_rot);
    else rot_tile<kRotSchwefel>(A, P, it, smem_rot);
}

template <int COSTS>
cudaError_t set_smem_rot(size_t bytes) {
    static size_t current = 0;  // the limit only grows, so earlier graphs stay valid
    if (bytes <= current) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(sweep_rot_kernel<COSTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

}  // namespace

size_t sweep_rot_smem_bytes(int n) { return (size_t)kWarpsR * 3 * (size_t)n * sizeof(float); }
int sweep_rot_chains_per_block() { return kWarpsR; }

cudaError_t sweep_rot_set_smem(size_t bytes) {
    cudaError_t e = set_smem_rot<1>(bytes);
    if (e == cudaSuccess) e = set_smem_rot<2>(bytes);
    if (e == cudaSuccess) e = set_smem_rot<3>(bytes);
    return e;
}

cudaError_t launch_sweep_rot(const SweepArgs& a, int num_items, size_t smem, int costs, cudaStream_t s) {
    if (costs == 1) sweep_rot_kernel<1><<<num_items, kBlockR, smem, s>>>(a);
    else if (costs == 2) sweep_rot_kernel<2><<<num_items, kBlockR, smem, s>>>(a);
    else sweep_rot_kernel<3><<<num_items, kBlockR, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sa
