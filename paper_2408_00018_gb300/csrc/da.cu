// da.cu -- delayed-acceptance Metropolis sweep with the learned surrogate, for
// the rotated costs (an extension: the paper has no surrogate).
//
// Two-stage delayed acceptance (Christen & Fox 2005): a proposal x' first
// passes stage 1 with probability min(1, exp(-(f~(x') - f~(x)) / T)), drawn
// with word 0 of the Philox block (step, level, chain, problem) of stream tag
// 3; only then is the true difference dF evaluated (the rank-1 evaluation of
// rot_step.cuh) and the move accepted with probability
// min(1, exp(-(dF - (f~(x') - f~(x))) / T)), drawn with the sweep's u3.  The
// pair of stages satisfies detailed balance for exp(-f/T) whatever f~ is, as
// long as f~ is a fixed function of the state during the level: here
// f~(x) = mu + sigma MLP(bf16((x - mid) / half)) with the weights, mu and sigma
// frozen for the level.
//
// The chains advance in lockstep, one step per round of launches, so that the
// surrogate of every chain's proposal is one pair of tensor-core GEMMs:
//   patch      x'_d into the chain's BF16 input row (one thread per chain)
//   GEMM 1     A1 = gelu(Xs W1^T + b1)           (fused epilogue, BF16 out)
//   GEMM 2     part = per-tile sums of gelu(A1 W2^T + b2) w3   (fused epilogue)
//   step       stage 1, the true difference for survivors, stage 2, update or
//              restore the input row (one warp per chain)
// Chain state lives in global memory between rounds: x [C][n], y_hi, y_lo
// [C][n], the input rows Xs [Cp][np] (BF16), F, its error bound and f~(x).
// The level ends like the plain rotated sweep (candidate band, FP64 values of
// the candidates); the chains' end states and values then enter a ring buffer
// of (x, f) pairs, and before the next level the network takes a few Adam
// steps on batches drawn from it.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>
#include <math_constants.h>

#include "rot_step.cuh"
#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kWarpsDA = 4;
constexpr int kDaInserts = 4;  // buffer insertions per level, evenly spaced over the steps

__device__ __forceinline__ __nv_bfloat16 std_bf16(float x, float mid, float inv_half) {
    return __float2bfloat16_rn((x - mid) * inv_half);
}

template <int COST>
__device__ __forceinline__ double f_of_sum(double s, int n) {
    return COST == kRotRastrigin ? 10.0 * (double)n + s : -(s / (double)n);
}

// Level start: every chain's x, y pair, input row, F and error bound.
template <int COST>
__device__ void start_chain(const SweepArgs& A, const ProbDev& P, const DaDev& D, int64_t c, int level) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    float* x = D.xf + (size_t)c * n;
    float* yh = D.yh + (size_t)c * n;
    float* yl = D.yl + (size_t)c * n;
    __nv_bfloat16* xs = D.xs + (size_t)c * D.np;
    double part = 0.0;
    for (int k = lane; k < n; k += 32) {
        float xv, h, l;
        if (level == 0) {
            xv = P.x0[(size_t)c * n + k];
            const float2 v = P.y0[(size_t)c * n + k];
            h = v.x;
            l = v.y;
            part += rot_g64<COST>((double)h + (double)l);
        } else {
            xv = P.x_best32[k];
            h = P.ybest_hi[k];
            l = P.ybest_lo[k];
        }
        x[k] = xv;
        yh[k] = h;
        yl[k] = l;
        xs[k] = std_bf16(xv, D.mid[k], D.inv_half[k]);
    }
    for (int k = n + lane; k < D.np; k += 32) xs[k] = __float2bfloat16_rn(0.0f);
    part = rot_wsumd(part);
    if (lane == 0) {
        D.Fa[c] = level == 0 ? f_of_sum<COST>(part, n) : P.scal[kFRot];
        D.Ea[c] = 0.0;
    }
}

__global__ void __launch_bounds__(32 * kWarpsDA) da_start_kernel(SweepArgs A, DaDev D) {
    const ProbDev& P = A.probs[D.problem];
    const int64_t c = (int64_t)blockIdx.x * kWarpsDA + (threadIdx.x >> 5);
    if (c >= P.chains) return;
    const int level = A.run->level;
    if (P.cost == kRotRastrigin) start_chain<kRotRastrigin>(A, P, D, c, level);
    else start_chain<kRotSchwefel>(A, P, D, c, level);
}

// f~ from the output head's four partial sums q and the output bias: the sum in a
// fixed order, then mu + sigma * sum as one FMA, all by explicit round-to-nearest
// intrinsics so that every kernel that forms f~ rounds it the same way.
__device__ __forceinline__ float surrogate_of(const DaDev& D, const float* q, float b3) {
    const float t = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(q[0], q[1]), q[2]), q[3]), b3);
    return __fmaf_rn(D.ms[1], t, D.ms[0]);
}

// f~ of every chain's start state (from the head's partial sums).
__global__ void da_ft_kernel(SweepArgs A, DaDev D, const float* __restrict__ b3) {
    const ProbDev& P = A.probs[D.problem];
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= P.chains) return;
    const float* q = D.part + (size_t)c * 4;
    const float v = surrogate_of(D, q, *b3);
    D.fts[c] = v;
    const int level = A.run->level;
    if (D.trace_ft0 && level < A.trace_levels) D.trace_ft0[(size_t)level * P.chains + c] = v;
}

// Put step s's proposal into each chain's input row.
__global__ void da_patch_kernel(SweepArgs A, DaDev D, int s) {
    const ProbDev& P = A.probs[D.problem];
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= P.chains) return;
    const int level = A.run->level;
    const int n = P.n;
    const double T = A.T_tab[level];
    const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)level, (uint32_t)c + P.cid0, P.pid), A.key0, A.key1);
    const RotMove mv = rot_propose(w, D.xf + (size_t)c * n, P, (float)A.s_tab[level], A.boundary, 0,
                                   (float)(-T * 0.69314718055994531));
    D.xs[(size_t)c * D.np + mv.d] = std_bf16(mv.xp, D.mid[mv.d], D.inv_half[mv.d]);
}

// One 4-byte asynchronous copy from global into shared memory (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The level's constants of a step, formed once per thread and launch.
struct StepConst {
    double T;                 // temperature
    float Tf, neg_T_ln2, sl;  // T and -T ln 2 in FP32; sl = sqrt(T / T0)
};

// One lockstep step of chain c.  sy: the warp's 2n floats of shared memory.  The
// chain's pair state is copied into it asynchronously before the step's draws
// (the copies do not depend on them), the step reads and updates it there, and
// an accepted move writes it back.  The copies are lane-strided (k = lane + 32 j)
// and the evaluation and update may take coordinates in pairs, so a warp
// barrier separates each from the next.
template <int COST>
__device__ void step_chain(const SweepArgs& A, const ProbDev& P, const DaDev& D, int64_t c, int level, int s,
                           const StepConst& K, float* sy, unsigned& nacc, unsigned& nev, unsigned& nre) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    float* x = D.xf + (size_t)c * n;
    float* yhg = D.yh + (size_t)c * n;
    float* ylg = D.yl + (size_t)c * n;
    float* yh = sy;
    float* yl = sy + n;
    for (int k = lane; k < n; k += 32) {
        cp_async4(yh + k, yhg + k);
        cp_async4(yl + k, ylg + k);
    }
    // the running value and its error bound (lane 0 updates them on acceptance)
    const double Fa0 = D.Fa[c], Ea0 = D.Ea[c];
    const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)level, (uint32_t)c + P.cid0, P.pid), A.key0, A.key1);
    const RotMove mv = rot_propose(w, x, P, K.sl, A.boundary, 0, K.neg_T_ln2);
    // surrogate at the proposal (fixed summation order) and at the current state
    const float* q = D.part + (size_t)c * 4;
    const float ftp = surrogate_of(D, q, D.b3[0]);
    const float ftc = D.fts[c];
    const bool tracing = level < A.trace_levels;
    if (tracing && D.trace_ftp && lane == 0) D.trace_ftp[((size_t)level * A.L + s) * P.chains + c] = ftp;
    // ---- stage 1 (surrogate only): pass iff u < exp(-dFs/T), dFs = f~(x') - f~(x), i.e.
    // dFs < tau1 = -T ln u.  FP32 decides outside a margin that covers the error of
    // tau1 (1e-6 tau1 + 4e-7 T), the roundings of the FP32 difference, of the margin
    // and of the comparison; inside it the FP64 tests decide, so the decision is the
    // FP64 one everywhere (this GPU's FP64 rate is a small fraction of its FP32 rate).
    const uint4 wd = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)level, (uint32_t)c + P.cid0, P.pid), D.dkey0, D.dkey1);
    const float d32 = ftp - ftc;
    bool pass1;
    if (ftp <= ftc) {  // dFs <= 0 exactly
        pass1 = true;
    } else {
        const float t1 = K.neg_T_ln2 * lg2_approx(u23f(wd.x));
        const float M1 = fmaf(1.1e-6f, t1, fmaf(4.4e-7f, K.Tf, 2.4e-7f * d32));
        if (d32 < t1 - M1) {
            pass1 = true;
        } else if (d32 > t1 + M1) {
            pass1 = false;
        } else {
            const double dFs = (double)ftp - (double)ftc;
            const double tau1 = (double)t1;
            const double m1 = 1.0e-6 * tau1 + 4.0e-7 * K.T;
            if (dFs < tau1 - m1) pass1 = true;
            else if (dFs > tau1 + m1) pass1 = false;
            else pass1 = u23d(wd.x) < exp(-dFs / K.T);
        }
    }
    bool acc = false;
    cp_async_wait_all();
    __syncwarp();
    if (pass1) {
        ++nev;
        // ---- stage 2: accept iff dF - dFs <= 0 or u3 < exp(-(dF - dFs)/T), i.e. dF < dFs + tau
        float dF, B;
        rot_eval32<COST>(P, yh, yl, mv.d, mv.dh, n, lane, dF, B);
        for (int rep = 1; rep < A.cost_repeat; ++rep) {  // the expensive-cost knob
            float dF2, B2;
            rot_eval32<COST>(P, yh, yl, mv.d, mv.dh + opaque_zero(), n, lane, dF2, B2);
            asm volatile("" ::"f"(dF2), "f"(B2));
        }
        // FP32 decides outside B widened by the error of tau and the roundings of the
        // FP32 threshold and comparison; inside it the FP64 tests below decide (the
        // FP64 decision everywhere, as in stage 1)
        const float thr32 = d32 + mv.tau;
        const float Bt32 = fmaf(1.00001f, B, fmaf(1.2e-6f, fabsf(mv.tau),
                                                  fmaf(4.8e-7f, K.Tf, 4.0e-7f * (fabsf(d32) + fabsf(thr32)))));
        bool rechecked = false;
        double dF64 = 0.0, e64 = 0.0;
        if (dF < thr32 - Bt32) {
            acc = true;
        } else if (dF > thr32 + Bt32) {
            acc = false;
        } else {
            const double dFs = (double)ftp - (double)ftc;
            const double thr = dFs + (double)mv.tau;
            const double Bt = (double)B + 1.0e-6 * fabs((double)mv.tau) + 4.0e-7 * K.T + 1e-12 * fabs(dFs);
            if ((double)dF < thr - Bt) {
                acc = true;
            } else if ((double)dF > thr + Bt) {
                acc = false;
            } else {
                dF64 = rot_eval64<COST>(P, yh, yl, mv.d, mv.xp, mv.xo, n, lane, e64);
                const double r = dF64 - dFs;
                acc = (r <= 0.0) || (u23d(mv.w3) < exp(-r / K.T));
                rechecked = true;
                ++nre;
            }
        }
        if (acc) {
            float edrift = 0.0f;
            rot_update<COST>(P, yh, yl, mv.d, mv.dh, mv.dl, n, lane, edrift);
            __syncwarp();  // the update may write a coordinate another lane copies back
            for (int k = lane; k < n; k += 32) {
                yhg[k] = yh[k];
                ylg[k] = yl[k];
            }
            if (lane == 0) {
                const double dF_used = rechecked ? dF64 : (double)dF;
                const double e_step = rechecked ? e64 : (double)B;
                x[mv.d] = mv.xp;
                D.Fa[c] = Fa0 + dF_used;
                D.Ea[c] = Ea0 + (e_step + (double)edrift);
                D.fts[c] = ftp;
            }
            ++nacc;
        }
    }
    // the input row keeps x'_d only if the move was accepted
    if (!acc && lane == 0) D.xs[(size_t)c * D.np + mv.d] = std_bf16(mv.xo, D.mid[mv.d], D.inv_half[mv.d]);
    if (tracing && A.bits && lane == 0 && acc) {
        uint32_t* word = A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)(P.chain_base + c)) * A.words + (s >> 5);
        *word |= 1u << (s & 31);  // one chain per warp, steps in order: no other writer
    }
    __syncwarp();
}

// A grid sized to the resident blocks; each warp takes chains blockIdx * kWarpsDA +
// warp + j * (gridDim * kWarpsDA), so that the counters take one global atomic per block.
__global__ void __launch_bounds__(32 * kWarpsDA, 6) da_step_kernel(SweepArgs A, DaDev D, int s) {
    extern __shared__ __align__(16) float smem_da[];
    __shared__ unsigned sacc, sev, sre;
    const ProbDev& P = A.probs[D.problem];
    if (threadIdx.x == 0) sacc = sev = sre = 0u;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    float* sy = smem_da + (size_t)warp * 2 * P.n;
    const int level = A.run->level;
    StepConst K;
    K.T = A.T_tab[level];
    K.Tf = (float)K.T;
    K.neg_T_ln2 = (float)(-K.T * 0.69314718055994531);
    K.sl = (float)A.s_tab[level];
    unsigned nacc = 0, nev = 0, nre = 0;
    const int64_t stride = (int64_t)gridDim.x * kWarpsDA;
    for (int64_t c = (int64_t)blockIdx.x * kWarpsDA + warp; c < P.chains; c += stride) {
        if (P.cost == kRotRastrigin) step_chain<kRotRastrigin>(A, P, D, c, level, s, K, sy, nacc, nev, nre);
        else step_chain<kRotSchwefel>(A, P, D, c, level, s, K, sy, nacc, nev, nre);
    }
    if ((threadIdx.x & 31) == 0 && (nacc | nev | nre)) {
        atomicAdd(&sacc, nacc);
        atomicAdd(&sev, nev);
        atomicAdd(&sre, nre);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sacc) atomicAdd(P.accepts, (unsigned long long)sacc);
        if (sev) atomicAdd(D.evals, (unsigned long long)sev);
        if (sre) atomicAdd(P.rechecks, (unsigned long long)sre);
    }
}

// Zero the traced level's accept bits before its steps set them.
__global__ void da_clear_bits_kernel(SweepArgs A, DaDev D) {
    const ProbDev& P = A.probs[D.problem];
    const int level = A.run->level;
    if (!A.bits || level >= A.trace_levels) return;
    const size_t count = (size_t)P.chains * A.words;
    uint32_t* base = A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)P.chain_base) * A.words;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        base[i] = 0u;
}

// Level end: candidate band (as the plain rotated sweep), FP64 values of the
// candidates, their states in the [n][chains] block; every chain's (x, F) into
// the ring buffer at slots (level C + c) mod cap.
template <int COST>
__device__ void finish_chain(const SweepArgs& A, const ProbDev& P, const DaDev& D, int64_t c, int level, double M) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    const int64_t gc = P.chain_base + c;
    const float* x = D.xf + (size_t)c * n;
    const float* yh = D.yh + (size_t)c * n;
    const float* yl = D.yl + (size_t)c * n;
    const double Fa = D.Fa[c], ec = D.Ea[c] + 1e-13 * (fabs(Fa) + 1.0);
    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    const bool finite = isfinite(Fa);
    if (finite && (tracing || level == A.full_level || Fa - ec <= M)) {
        double part = 0.0;
        for (int i = lane; i < n; i += 32) part += rot_g64<COST>((double)yh[i] + (double)yl[i]);
        part = rot_wsumd(part);
        if (lane == 0) A.F[gc] = f_of_sum<COST>(part, n);
        float* dst = A.X32 + P.x_base + c;
        for (int k = lane; k < n; k += 32) dst[(size_t)k * (size_t)P.chains] = x[k];
    } else if (lane == 0) {
        A.F[gc] = finite ? CUDART_INF : CUDART_NAN;
    }
}

// Chains' current (x, F) into the ring buffer: insertion j of the level goes to
// rows ((level kDaInserts + j) C + c) mod cap.
__global__ void da_insert_kernel(SweepArgs A, DaDev D, int j) {
    const ProbDev& P = A.probs[D.problem];
    const int level = A.run->level;
    const int n = P.n;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (row >= P.chains) return;
    const int lane = threadIdx.x & 31;
    const int64_t slot = (((int64_t)level * kDaInserts + j) * P.chains + row) % D.cap;
    for (int k = lane; k < n; k += 32) D.rx[(size_t)slot * n + k] = D.xf[(size_t)row * n + k];
    if (lane == 0) D.rf[slot] = (float)D.Fa[row];
}

__global__ void __launch_bounds__(32 * kWarpsDA) da_finish_kernel(SweepArgs A, DaDev D) {
    __shared__ double block_hi[kWarpsDA];
    __shared__ double block_M;
    const ProbDev& P = A.probs[D.problem];
    const int level = A.run->level;
    const int warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kWarpsDA + warp;
    const bool mine = c < P.chains;
    if ((threadIdx.x & 31) == 0) {
        double v = CUDART_INF;
        if (mine) {
            const double Fa = D.Fa[c];
            if (isfinite(Fa)) v = Fa + D.Ea[c] + 1e-13 * (fabs(Fa) + 1.0);
        }
        block_hi[warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bmin = block_hi[0];
        for (int w2 = 1; w2 < kWarpsDA; ++w2) bmin = fmin(bmin, block_hi[w2]);
        double M = bmin;
        if (bmin < CUDART_INF) M = fmin(M, key_dbl(atomicMin(P.level_min, dbl_key(bmin))));
        else M = key_dbl(*(volatile unsigned long long*)P.level_min);
        block_M = M;
    }
    __syncthreads();
    if (!mine) return;
    if (P.cost == kRotRastrigin) finish_chain<kRotRastrigin>(A, P, D, c, level, block_M);
    else finish_chain<kRotSchwefel>(A, P, D, c, level, block_M);
}

// ---- training ---------------------------------------------------------------
// Mean and standard deviation of the buffer's values (one block, fixed order).
__global__ void da_stats_kernel(SweepArgs A, DaDev D) {
    __shared__ double red[256];
    const ProbDev& P = A.probs[D.problem];
    const int level = A.run->level;
    const int64_t filled = min((int64_t)level * kDaInserts * P.chains, (int64_t)D.cap);
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < filled; i += blockDim.x) s += (double)D.rf[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = filled > 0 ? red[0] / (double)filled : 0.0;
    __syncthreads();
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < filled; i += blockDim.x) {
        const double e = (double)D.rf[i] - mean;
        v += e * e;
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sd = filled > 1 ? sqrt(red[0] / (double)(filled - 1)) : 1.0;
        D.ms[0] = (float)mean;
        D.ms[1] = (float)(sd > 1e-12 ? sd : 1.0);
        *D.train_on = filled > 0 ? 1 : 0;
    }
}

// One training batch (Philox stream tag 4, counter (row, epoch step, level,
// problem)): even rows uniformly from the filled buffer, odd rows from the states
// the previous level inserted (the region the chains are in now); standardised
// inputs and targets.
__global__ void da_sample_kernel(SweepArgs A, DaDev D, int e) {
    const ProbDev& P = A.probs[D.problem];
    const int level = A.run->level;
    const int64_t filled = min((int64_t)level * kDaInserts * P.chains, (int64_t)D.cap);
    const int64_t recent = min((int64_t)kDaInserts * P.chains, filled);
    const int64_t recent0 = ((int64_t)(level > 0 ? level - 1 : 0) * kDaInserts * P.chains) % D.cap;
    const int n = P.n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)D.batch * D.np;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / D.np), k = (int)(t % D.np);
        float v = 0.0f;
        int64_t j = 0;
        if (filled > 0) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)e, (uint32_t)level, P.pid), D.tkey0, D.tkey1);
            const uint64_t r = ((uint64_t)w.y << 32) | w.x;
            j = (b & 1) ? (recent0 + (int64_t)(r % (uint64_t)recent)) % D.cap : (int64_t)(r % (uint64_t)filled);
            if (k < n) v = (D.rx[(size_t)j * n + k] - D.mid[k]) * D.inv_half[k];
        }
        D.work.Xb[t] = __float2bfloat16_rn(v);
        if (k == 0) D.bt[b] = filled > 0 ? (D.rf[j] - D.ms[0]) / D.ms[1] : 0.0f;
    }
}

// Adam with the step count and the switch in device memory (so a captured level
// can be replayed): no update while the buffer is empty.
__global__ void da_adam_kernel(DaDev D, int64_t count, float lr, float b1, float b2, float eps) {
    if (*D.train_on == 0) return;
    const int step = *D.adam_step + 1;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = D.grad[i];
        const float mi = fmaf(b1, D.m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, D.v[i], (1.0f - b2) * gi * gi);
        D.m[i] = mi;
        D.v[i] = vi;
        D.mlp.p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}
__global__ void da_adam_count_kernel(DaDev D) {
    if (*D.train_on) *D.adam_step += 1;
}

__global__ void da_reset_kernel(DaDev D, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        D.m[i] = 0.0f;
        D.v[i] = 0.0f;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *D.adam_step = 0;
        *D.evals = 0ull;
    }
}

int grid_for(int64_t work, int block) {
    int64_t g = (work + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 152 * 64 ? 152 * 64 : g));
}

size_t da_step_smem(int n) { return (size_t)kWarpsDA * 2 * (size_t)n * sizeof(float); }

}  // namespace

// The step kernel's shared memory (above the default 48 KB from n = 1537 on) and grid:
// the blocks that fit on the device at once, at most one per 4 chains.
cudaError_t da_prepare(DaDev& D, int64_t chains) {
    const size_t smem = da_step_smem(D.mlp.n);
    static size_t current = 0;  // only ever raised: a smaller handle must not lower a larger one's limit
    cudaError_t e = cudaSuccess;
    if (smem > current) {
        e = cudaFuncSetAttribute(da_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) current = smem;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, da_step_kernel, 32 * kWarpsDA, smem);
    if (e != cudaSuccess) return e;
    const int64_t need = (chains + kWarpsDA - 1) / kWarpsDA;
    D.step_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(1, per_sm) * sms));
    return cudaSuccess;
}

// Before level 0 of a run: fresh network (seeded), zero moments and counters.
cudaError_t da_run_start(const DaDev& D, uint64_t seed, cudaStream_t s) {
    cudaError_t e = mlp_init(D.mlp.p, D.mlp.n, seed, s);
    if (e != cudaSuccess) return e;
    const int64_t count = mlp_offsets(D.mlp.n).total;
    da_reset_kernel<<<grid_for(count, 256), 256, 0, s>>>(D, count);
    return cudaGetLastError();
}

// One level of the delayed-acceptance sweep (launch sequence; also captured as a graph).
cudaError_t launch_da_level(const SweepArgs& A, const DaDev& Dc, int64_t chains, int L, int train_steps, float lr,
                            int* status, cudaStream_t s) {
    DaDev D = Dc;
    const int64_t count = mlp_offsets(D.mlp.n).total;
    const MlpOffsets o = mlp_offsets(D.mlp.n);
    cudaError_t e = cudaSuccess;
    // training on the buffer filled by the previous levels (no update at level 0)
    da_stats_kernel<<<1, 256, 0, s>>>(A, D);
    for (int t = 0; t < train_steps && e == cudaSuccess; ++t) {
        da_sample_kernel<<<grid_for((int64_t)D.batch * D.np, 256), 256, 0, s>>>(A, D, t);
        e = mlp_cast(D.mlp, s);
        if (e == cudaSuccess) e = mlp_loss_grad(D.mlp, D.work.Xb, D.batch, D.batch, D.bt, D.work, D.grad, nullptr, status, s);
        if (e == cudaSuccess) {
            da_adam_kernel<<<grid_for(count, 256), 256, 0, s>>>(D, count, lr, 0.9f, 0.999f, 1e-8f);
            da_adam_count_kernel<<<1, 1, 0, s>>>(D);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return e;
    // the level's network: BF16 weights, then the start states and their f~
    e = mlp_cast(D.mlp, s);
    if (e != cudaSuccess) return e;
    const int cblocks = (int)((chains + kWarpsDA - 1) / kWarpsDA);
    da_clear_bits_kernel<<<grid_for(chains * A.words, 256), 256, 0, s>>>(A, D);
    da_start_kernel<<<cblocks, 32 * kWarpsDA, 0, s>>>(A, D);
    e = mlp_infer(D.mlp, D.xs, D.Cp, D.A1, D.part, status, s);
    if (e != cudaSuccess) return e;
    da_ft_kernel<<<(int)((chains + 255) / 256), 256, 0, s>>>(A, D, D.mlp.p + o.b3);
    for (int st = 0; st < L && e == cudaSuccess; ++st) {
        da_patch_kernel<<<(int)((chains + 255) / 256), 256, 0, s>>>(A, D, st);
        e = mlp_infer(D.mlp, D.xs, D.Cp, D.A1, D.part, status, s);
        if (e == cudaSuccess) {
            da_step_kernel<<<D.step_blocks, 32 * kWarpsDA, da_step_smem(D.mlp.n), s>>>(A, D, st);
            // states along the level (and at its end) feed the training buffer
            for (int j = 0; j < kDaInserts; ++j)  // exactly kDaInserts insertions per level
                if (std::max(1, (j + 1) * L / kDaInserts) - 1 == st)
                    da_insert_kernel<<<cblocks, 32 * kWarpsDA, 0, s>>>(A, D, j);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return e;
    da_finish_kernel<<<cblocks, 32 * kWarpsDA, 0, s>>>(A, D);
    return cudaGetLastError();
}

}  // namespace sa
