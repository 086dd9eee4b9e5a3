// sweep_f32w.cu -- Metropolis sweep of one temperature level, FP32 state,
// one Markov chain per warp.
//
// The 32 lanes of a warp run 32 consecutive steps s0 .. s0+31 of the same
// chain (the kernel of Listing 4, one step per lane): each lane draws its
// Philox block, proposes its move and evaluates its energy difference from
// the chain's state at the start of the group.  The group is then committed
// in step order.  A lane whose coordinate (for Rosenbrock: the coordinate or
// a neighbour) is also touched by an earlier lane of the group is "pending":
// the earlier lanes are decided first, then the pending lanes are
// re-evaluated one at a time, in step order, from the state those decisions
// left.  Every other lane's speculative evaluation read exactly the state
// the sequential chain would have read, so the decisions equal those of the
// one-step-at-a-time chain.  With n coordinates about 31*32/(2n) lanes per
// group are pending, so this layout is used for n >= 48.
//
// The chain's state is one row x[0..n) of shared memory per warp.  Only
// separable costs without global running sums use this kernel (Schwefel,
// Rastrigin, Rosenbrock); Ackley keeps one chain per thread.
//
// End of level: as in the chain-per-thread kernel, each chain holds
// F_start + dS and a running bound e on its FP32 error; the chains whose
// interval can contain the level minimum are re-evaluated in FP64 (lanes over
// coordinates) and write their state for the argmin.
#include <cfloat>
#include <cmath>
#include <math_constants.h>

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kBlock = 256;
#ifndef SA_F32W_MIN_BLOCKS
#define SA_F32W_MIN_BLOCKS 3  // resident blocks per SM the register budget is sized for
#endif
constexpr int kWarps = kBlock / 32;
constexpr unsigned kFull = 0xffffffffu;

// A register copy the compiler cannot trace back to the kernel-parameter
// bank, so loop invariants stay in registers instead of being reloaded with
// constant loads inside the step loop.
__device__ __forceinline__ uint32_t opaque(uint32_t v) {
    uint32_t r;
    asm volatile("mov.b32 %0, %1;" : "=r"(r) : "r"(v));
    return r;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

struct WStep {
    int d;
    float z, tau, xo, xp, dF, xm, xq, hp;
};

// Term of one coordinate in the separable costs that keep a per-coordinate
// cache: Schwefel h(t) = t sin sqrt|t| (f = -(1/n) sum h), Rastrigin
// g(t) = t^2 - 10 cos 2 pi t.  The cache holds exactly this function's value
// at the stored coordinate, so reading it equals recomputing it.
template <int COST>
__device__ __forceinline__ float term(float t) {
    if (COST == kSchwefel) return t * sin_reduced(sqrt_approx(fabsf(t)));
    return g_rastrigin(t);
}

struct WCtx {
    float* xw;  // the warp's chain state, x[0..n)
    float* hw;  // Schwefel/Rastrigin: term(x[k]) for every coordinate
    int n;
    float inv_n;
    float lo_u, hi_u, sig_u;
    const float *slo, *shi, *ssig;
    int boundary;
    float neg_T_ln2;
    PhiloxFixed pf;
    const uint32_t* rk;  // Philox round keys (kernel parameters)
};

// UP: the move is a uniform redraw of the coordinate (z = u2) instead of a Gaussian step.
template <bool UP>
__device__ __forceinline__ void wpropose(const WCtx& C, uint32_t s, WStep& p) {
    const uint4 w = philox_step(s, C.pf, C.rk);
    p.d = coord_of(w.x, C.n);
    const float u1 = u23f(w.y), u2 = u23f(w.z), u3 = u23f(w.w);
    if (UP) {
        p.z = u2;  // uniform redraw: x' = lo + u2 (hi - lo)
    } else {
        // Box-Muller, cosine branch: z = sqrt(-2 ln u1) cos(2 pi u2) = -sqrt(..) cos(2 pi (u2 - 1/2)).
        const float r = sqrt_approx(-1.3862943611198906f * __log2f(u1));
        p.z = -r * __cosf(6.28318530717958648f * (u2 - 0.5f));
    }
    // u3 < exp(-dF/T)  <=>  dF < tau = -T ln u3
    p.tau = C.neg_T_ln2 * __log2f(u3);
}

// Move and energy difference from the chain's current state.
template <int COST, bool UB, bool UP>
__device__ __forceinline__ void wevaluate(const WCtx& C, WStep& p) {
    const int d = p.d;
    const float xo = C.xw[d];
    float lo, hi, sg;
    if (UB) { lo = C.lo_u; hi = C.hi_u; sg = C.sig_u; }
    else { lo = C.slo[d]; hi = C.shi[d]; sg = C.ssig[d]; }
    float xp = UP ? fmaf(hi - lo, p.z, lo) : fmaf(sg, p.z, xo);
    if (C.boundary == 0) xp = xp < lo ? 2.0f * lo - xp : (xp > hi ? 2.0f * hi - xp : xp);
    xp = fminf(fmaxf(xp, lo), hi);
    p.xo = xo;
    p.xp = xp;
    if (COST == kSchwefel) {
        p.hp = term<COST>(xp);
        p.dF = (C.hw[d] - p.hp) * C.inv_n;
    } else if (COST == kRastrigin) {
        p.hp = term<COST>(xp);
        p.dF = p.hp - C.hw[d];
    } else {
        float dummy = 0.0f, before = 0.0f, after = 0.0f;
        p.xm = d > 0 ? C.xw[d - 1] : 0.0f;
        p.xq = d + 1 < C.n ? C.xw[d + 1] : 0.0f;
        if (d > 0) { before += rosen_term(p.xm, xo, dummy); after += rosen_term(p.xm, xp, dummy); }
        if (d + 1 < C.n) { before += rosen_term(xo, p.xq, dummy); after += rosen_term(xp, p.xq, dummy); }
        p.dF = after - before;
    }
}

// Rosenbrock: FP32 error bound of one step's dF from the values involved.
__device__ __forceinline__ float rosen_bound(const WCtx& C, const WStep& p) {
    float eb = 0.0f, s = 0.0f;
    if (p.d > 0) { s += rosen_term(p.xm, p.xo, eb); s += rosen_term(p.xm, p.xp, eb); }
    if (p.d + 1 < C.n) { s += rosen_term(p.xo, p.xq, eb); s += rosen_term(p.xp, p.xq, eb); }
    return eb + (s + fabsf(p.dF)) * 1.2e-7f;
}

template <int COST>
__device__ __forceinline__ void partial64(const float* xw, int n, int k, double& p1) {
    const double x = (double)xw[k];
    if (COST == kSchwefel) p1 += h64_schwefel(x);
    else if (COST == kRastrigin) p1 += g64_rastrigin(x);
    else if (k + 1 < n) p1 += rosen64(x, (double)xw[k + 1]);
}

struct ChainEnd {
    double Fa, ec;   // F_start + dS and the bound on its error
    unsigned nacc;   // accepted moves
};

template <int COST, bool UB, bool UP>
__device__ ChainEnd warp_chain(const SweepArgs& A, const ProbDev& P, int64_t c, int level, float* xw, float* hw,
                               const float* slo, const float* shi, const float* ssig, double* block_hi) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    const int64_t gc = P.chain_base + c;
    const double T = A.T_tab[level];
    const float sl = (float)A.s_tab[level];
    const float inv_n = 1.0f / (float)n;

    // ---- state at the start of the level
    if (level == 0) {
        for (int k = 4 * lane; k < n; k += 128) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(k >> 2), 0u, (uint32_t)c + P.cid0, P.pid), A.ikey0, A.ikey1);
            const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (k + j < n) {
                    const double lo = P.lo[k + j], hi = P.hi[k + j];
                    float x = (float)(lo + u23d(ww[j]) * (hi - lo));
                    xw[k + j] = fminf(fmaxf(x, P.lo32[k + j]), P.hi32[k + j]);
                }
            }
        }
    } else if (own_start(A, level)) {  // the chain's own state (no exchange before this level)
        for (int k = lane; k < n; k += 32) xw[k] = A.X32[P.x_base + (size_t)k * (size_t)P.chains + (size_t)c];
    } else {
        for (int k = lane; k < n; k += 32) xw[k] = P.x_best32[k];
    }
    __syncwarp();
    if (COST == kSchwefel || COST == kRastrigin) {
        for (int k = lane; k < n; k += 32) hw[k] = term<COST>(xw[k]);
        __syncwarp();
    }

    double Fs;
    float es = 0.0f;
    if (level == 0 || own_start(A, level)) {
        // FP32 value of f at the start point with a bound on its error
        float sum = 0.0f, sabs = 0.0f, e = 0.0f;
        for (int k = lane; k < n; k += 32) {
            const float x = xw[k];
            float g;
            if (COST == kSchwefel) {
                g = hw[k];
                e += fabsf(x) * fmaf(sqrt_approx(fabsf(x)), 4.8e-7f, 2.6e-6f);
            } else if (COST == kRastrigin) {
                g = hw[k];
                e += 2.4e-5f + fabsf(g) * 1.2e-7f;
            } else {
                g = k + 1 < n ? rosen_term(x, xw[k + 1], e) : 0.0f;
            }
            sum += g;
            sabs += fabsf(g);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(kFull, sum, o);
            sabs += __shfl_xor_sync(kFull, sabs, o);
            e += __shfl_xor_sync(kFull, e, o);
        }
        const float rnd = ((float)(n / 32) + 6.0f) * 1.2e-7f;  // sequential + tree summation rounding
        if (COST == kSchwefel) {
            const float F = -sum * inv_n;
            Fs = (double)F;
            es = (e + rnd * sabs) * inv_n + fabsf(F) * 1.2e-7f;
        } else if (COST == kRastrigin) {
            const float F = 10.0f * (float)n + sum;
            Fs = (double)F;
            es = e + rnd * (sabs + 10.0f * (float)n);
        } else {
            Fs = (double)sum;
            es = e + rnd * sabs;
        }
    } else {
        Fs = P.scal[kFBest];
    }

    WCtx C;
    C.xw = xw;
    C.hw = hw;
    C.n = n;
    C.inv_n = inv_n;
    C.lo_u = P.lo_u;
    C.hi_u = P.hi_u;
    C.sig_u = P.sig_u * sl;
    C.slo = slo;
    C.shi = shi;
    C.ssig = ssig;
    C.boundary = (int)opaque((uint32_t)A.boundary);
    C.neg_T_ln2 = (float)(-T * 0.69314718055994531);
    // Round keys in registers for the whole level: reading them from the
    // kernel-parameter bank inside the loop would issue constant loads, which
    // share a low-throughput pipe with divergent branches.
    uint32_t rk[20];
#pragma unroll
    for (int i = 0; i < 20; ++i) rk[i] = opaque(A.rk[i]);
    C.pf = philox_prep((uint32_t)level, (uint32_t)c + P.cid0, P.pid, rk);
    C.rk = rk;
    const float kappa = P.kappa;

    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    uint32_t* mybits = tracing ? A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)gc) * (size_t)A.words : nullptr;
    const unsigned lt = lanemask_lt();
    // Per-lane sums of the accepted differences (lane l holds the steps
    // s = l mod 32) and of the bounds on their FP32 errors; reduced once at the end.
    float dS = 0.0f, e = 0.0f;
    unsigned nacc = 0;
    const int L = (int)opaque((uint32_t)A.L);
    for (int s0 = 0; s0 < L; s0 += 32) {
        const int s = s0 + lane;
        const bool live = s < L;
        WStep p;
        wpropose<UP>(C, (uint32_t)s, p);
        wevaluate<COST, UB, UP>(C, p);
        // earlier lanes of the group whose step can change what this lane's evaluation read
        unsigned earlier;
        const int key = live ? p.d : -1 - lane;
        if (COST == kRosenbrock) {
            earlier = 0u;
            for (int k = 0; k < 31; ++k) {
                const int dk = __shfl_sync(kFull, key, k);
                earlier |= ((k < lane) && dk >= p.d - 1 && dk <= p.d + 1) ? (1u << k) : 0u;
            }
        } else {
            earlier = __match_any_sync(kFull, key) & lt;  // every lane takes part, live or not
        }
        const bool pend = live && earlier != 0u;
        bool acc = live && !pend && (p.dF < p.tau);
        __syncwarp();  // every speculative read happens before any write
        // Branch-free commit: lanes that do not accept write to the scratch
        // slot n of their row.  Accepting lanes write distinct coordinates
        // (each is the first lane of the group to touch its coordinate).
        int slot = acc ? p.d : n;
        xw[slot] = p.xp;
        if (COST == kSchwefel || COST == kRastrigin) hw[slot] = p.hp;
        // pending lanes, in rounds: a lane goes once every earlier conflicting
        // lane is decided; the whole warp evaluates, the going lanes keep it
        unsigned undecided = __ballot_sync(kFull, pend);
        while (undecided) {
            __syncwarp();
            const bool go = ((undecided >> lane) & 1u) && (earlier & undecided) == 0u;
            WStep q = p;
            wevaluate<COST, UB, UP>(C, q);
            const bool a2 = q.dF < q.tau;
            if (go) p = q;
            acc = go ? a2 : acc;
            __syncwarp();
            slot = (go && a2) ? q.d : n;
            xw[slot] = q.xp;
            if (COST == kSchwefel || COST == kRastrigin) hw[slot] = q.hp;
            undecided &= ~__ballot_sync(kFull, go);
        }
        __syncwarp();
        const float bnd = COST == kRosenbrock ? rosen_bound(C, p) : kappa;
        dS += acc ? p.dF : 0.0f;
        e += acc ? bnd + fabsf(dS) * 1.2e-7f : 0.0f;
        nacc += acc ? 1u : 0u;
        if (tracing) {
            const unsigned accm = __ballot_sync(kFull, acc);
            if (lane == 0) mybits[s0 >> 5] = accm;
        }
    }
    // lane sums -> chain sums (five tree levels: their rounding is bounded by 5 u sum|dS_lane|)
    float dabs = fabsf(dS);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dS += __shfl_xor_sync(kFull, dS, o);
        dabs += __shfl_xor_sync(kFull, dabs, o);
        e += __shfl_xor_sync(kFull, e, o);
        nacc += __shfl_xor_sync(kFull, nacc, o);
    }
    e += 5.0f * 1.2e-7f * dabs;

    // ---- candidates for the FP64 argmin
    const double Fa = Fs + (double)dS;
    const double ec = (double)es + (double)e;
    const bool finite = isfinite(Fa);
    if (lane == 0) block_hi[threadIdx.x >> 5] = finite ? Fa + ec : CUDART_INF;
    return ChainEnd{Fa, ec, nacc};
}

// After every warp of the block has finished its chain: one atomicMin per
// block on the device-wide threshold, then each warp's candidate test.
template <int COST>
__device__ void warp_chain_finish(const SweepArgs& A, const ProbDev& P, int64_t c, int level, const float* xw,
                                  double Fa, double ec, double M, unsigned nacc, unsigned* block_acc) {
    const int lane = threadIdx.x & 31;
    const int n = P.n;
    const int64_t gc = P.chain_base + c;
    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    const bool finite = isfinite(Fa);
    if (finite && (tracing || level == A.full_level || A.crossover || Fa - ec <= M)) {
        double p1 = 0.0;
        for (int k = lane; k < n; k += 32) partial64<COST>(xw, n, k, p1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p1 += __shfl_xor_sync(kFull, p1, o);
        if (lane == 0) {
            A.F[gc] = COST == kSchwefel ? -(p1 / (double)n) : (COST == kRastrigin ? 10.0 * (double)n + p1 : p1);
        }
        float* dst = A.X32 + P.x_base + c;
        for (int k = lane; k < n; k += 32) dst[(size_t)k * (size_t)P.chains] = xw[k];
    } else {
        if (lane == 0) A.F[gc] = finite ? CUDART_INF : CUDART_NAN;
        if (keep_states(A)) {  // every chain keeps its state for the next level
            float* dst = A.X32 + P.x_base + c;
            for (int k = lane; k < n; k += 32) dst[(size_t)k * (size_t)P.chains] = xw[k];
        }
    }
    if (lane == 0) atomicAdd(block_acc, nacc);
}

__global__ void __launch_bounds__(kBlock, SA_F32W_MIN_BLOCKS) sweep_f32w_kernel(SweepArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned block_acc;
    __shared__ double block_hi[kWarps];
    __shared__ double block_M;
    const WorkItem it = A.items[blockIdx.x];
    const ProbDev& P = A.probs[it.problem];
    const int level = A.run->level;
    const int n = P.n;
    const int warp = threadIdx.x >> 5;
    float* xs = reinterpret_cast<float*>(smem_raw);       // [kWarps][n] states
    float* hs = xs + (size_t)kWarps * (n + 1);             // [kWarps][n + 1] cached terms
    float* slo = hs + (size_t)kWarps * (n + 1);
    float* shi = slo + n;
    float* ssig = shi + n;
    const bool ub = P.uniform != 0;
    const bool up = A.proposal == 1;
    if (threadIdx.x == 0) block_acc = 0u;
    if (threadIdx.x < kWarps) block_hi[threadIdx.x] = CUDART_INF;
    if (!ub) {
        const float sl = (float)A.s_tab[level];
        for (int k = threadIdx.x; k < n; k += kBlock) { slo[k] = P.lo32[k]; shi[k] = P.hi32[k]; ssig[k] = P.sig32[k] * sl; }
    }
    __syncthreads();
    const bool mine = warp < it.count;
    float* xw = xs + (size_t)warp * (n + 1);  // row of n coordinates plus the scratch slot n
    float* hw = hs + (size_t)warp * (n + 1);
    const int64_t c = it.c0 + warp;
    ChainEnd end{0.0, 0.0, 0u};
    if (mine) {
        switch (P.cost) {
        case kSchwefel:
            end = up ? (ub ? warp_chain<kSchwefel, true, true>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi)
                           : warp_chain<kSchwefel, false, true>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi))
                     : (ub ? warp_chain<kSchwefel, true, false>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi)
                           : warp_chain<kSchwefel, false, false>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi));
            break;
        case kRastrigin:
            end = up ? (ub ? warp_chain<kRastrigin, true, true>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi)
                           : warp_chain<kRastrigin, false, true>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi))
                     : (ub ? warp_chain<kRastrigin, true, false>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi)
                           : warp_chain<kRastrigin, false, false>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi));
            break;
        case kRosenbrock:
            end = up ? (ub ? warp_chain<kRosenbrock, true, true>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi)
                           : warp_chain<kRosenbrock, false, true>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi))
                     : (ub ? warp_chain<kRosenbrock, true, false>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi)
                           : warp_chain<kRosenbrock, false, false>(A, P, c, level, xw, hw, slo, shi, ssig, block_hi));
            break;
        default:
            if ((threadIdx.x & 31) == 0) A.run->status = 1;
            break;
        }
    }
    __syncthreads();
    // one atomicMin per block on the device-wide threshold M = min(F + e)
    if (threadIdx.x == 0) {
        double bmin = block_hi[0];
        for (int w = 1; w < kWarps; ++w) bmin = fmin(bmin, block_hi[w]);
        double M = bmin;
        if (bmin < CUDART_INF) {
            const unsigned long long old = atomicMin(P.level_min, dbl_key(bmin));
            M = fmin(M, key_dbl(old));
        } else {
            M = key_dbl(*(volatile unsigned long long*)P.level_min);
        }
        block_M = M;
    }
    __syncthreads();
    if (mine) {
        switch (P.cost) {
        case kSchwefel: warp_chain_finish<kSchwefel>(A, P, c, level, xw, end.Fa, end.ec, block_M, end.nacc, &block_acc); break;
        case kRastrigin: warp_chain_finish<kRastrigin>(A, P, c, level, xw, end.Fa, end.ec, block_M, end.nacc, &block_acc); break;
        case kRosenbrock: warp_chain_finish<kRosenbrock>(A, P, c, level, xw, end.Fa, end.ec, block_M, end.nacc, &block_acc); break;
        default: break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && block_acc) atomicAdd(P.accepts, (unsigned long long)block_acc);
}

}  // namespace

int sweep_f32w_chains_per_block() { return kWarps; }

size_t sweep_f32w_smem_bytes(int n) { return (2 * (size_t)kWarps * (n + 1) + 3 * (size_t)n) * sizeof(float); }

cudaError_t sweep_f32w_set_smem(size_t bytes) {
    static size_t current = 0;
    if (bytes <= current) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(sweep_f32w_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

cudaError_t launch_sweep_f32w(const SweepArgs& a, int num_items, size_t smem, cudaStream_t s) {
    sweep_f32w_kernel<<<num_items, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sa
