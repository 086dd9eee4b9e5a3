// sweep_group.cuh -- the group layout of the FP32 sweep (device code shared
// by the group-layout kernel and the batched level kernel).
//
// Metropolis sweep of one temperature level, FP32 state,
// one Markov chain per group of G lanes (G = 2, 4, 8 or 32; G = 32 is one
// chain per warp).
//
// The G lanes of a group run G consecutive steps s0 .. s0+G-1 of the same
// chain (the kernel of Listing 4, one step per lane): each lane draws its
// Philox block, proposes its move and evaluates its energy difference from
// the chain's state at the start of the group.  The group is then committed
// in step order.  A lane whose coordinate (for Rosenbrock: the coordinate or
// a neighbour) is also touched by an earlier lane of its group is "pending":
// the earlier lanes are decided first, then the pending lanes are
// re-evaluated one at a time, in step order, from the state those decisions
// left.  Every other lane's speculative evaluation read exactly the state
// the sequential chain would have read, so the decisions equal those of the
// one-step-at-a-time chain.  With n coordinates about G(G-1)/(2n) lanes per
// group are pending.
//
// The group size trades the two limits of the sweep against each other.  A
// chain's state (n floats, plus n cached terms) lives in shared memory, so
// the shared memory of an SM bounds the chains it holds; G lanes per chain
// multiply the warps that hide the latency of the step's dependent Philox
// rounds and SFU functions by G, while the pending lanes' re-evaluations
// grow with G.  At n = 256 one chain per thread leaves ~1.5 warps per
// scheduler; G = 4 gives four times as many at ~2% pending lanes.
//
// The chain's state is one row x[0..n) of shared memory per group (slot n
// absorbs masked writes), optionally with the cache h[k] = term(x[k]) of the
// separable costs (CACHE).  Only separable costs without global running sums
// use this kernel (Schwefel, Rastrigin, Rosenbrock); Ackley keeps one chain
// per thread.
//
// End of level: as in the chain-per-thread kernel, each chain holds
// F_start + dS and a running bound e on its FP32 error; the chains whose
// interval can contain the level minimum are re-evaluated in FP64, one warp
// per candidate with the lane-strided partial sums and butterfly of the
// chain-per-thread kernel (so the FP64 value does not depend on the layout),
// and write their state for the argmin.
#pragma once
#include <cfloat>
#include <cmath>
#include <math_constants.h>
#include <type_traits>

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {


constexpr int kGroupMaxBlock = 256;
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

template <int G> struct Log2;
template <> struct Log2<2> { static constexpr int v = 1; };
template <> struct Log2<4> { static constexpr int v = 2; };
template <> struct Log2<8> { static constexpr int v = 3; };
template <> struct Log2<32> { static constexpr int v = 5; };

struct WStep {
    int d;
    float z, tau, xo, xp, dF, xm, xq, hp;
};

// Term of one coordinate in the separable costs that keep a per-coordinate
// cache: Schwefel h(t) = t sin sqrt|t| (f = -(1/n) sum h), Rastrigin
// g(t) = t^2 - 10 cos 2 pi t.  The product is rounded on its own
// (__fmul_rn is never merged into a later addition), so the value is the
// same whether it is read from the cache or recomputed inside a difference.
template <int COST>
__device__ __forceinline__ float term(float t) {
    if (COST == kSchwefel) return __fmul_rn(t, sin_reduced(sqrt_approx(fabsf(t))));
    return g_rastrigin(t);
}

struct WCtx {
    float* xw;  // the group's chain state, x[0..n)
    float* hw;  // Schwefel/Rastrigin with the cache: term(x[k]) for every coordinate
    int n;
    float inv_n;
    float lo_u, hi_u, sig_u;
    const float *slo, *shi, *ssig;
    int boundary;
    float neg_T_ln2;
    PhiloxFixed pf;
    const uint32_t* rk;  // Philox round keys (kernel parameters)
};

// The move of one step from its Philox block w.
// UP: the move is a uniform redraw of the coordinate (z = u2) instead of a Gaussian step.
template <bool UP>
__device__ __forceinline__ void wpropose(const WCtx& C, const uint4& w, WStep& p) {
    p.d = coord_of(w.x, C.n);
    const float u1 = u23f(w.y), u2 = u23f(w.z), u3 = u23f(w.w);
    if (UP) {
        p.z = u2;  // uniform redraw: x' = lo + u2 (hi - lo)
    } else {
        // Box-Muller, cosine branch: z = sqrt(-2 ln u1) cos(2 pi u2) = -sqrt(..) cos(2 pi (u2 - 1/2)).
        const float r = sqrt_approx(-1.3862943611198906f * lg2_approx(u1));
        p.z = -r * cos_approx(6.28318530717958648f * (u2 - 0.5f));
    }
    // u3 < exp(-dF/T)  <=>  dF < tau = -T ln u3
    p.tau = C.neg_T_ln2 * lg2_approx(u3);
}

// Move and energy difference from the chain's current state.
template <int COST, bool UB, bool UP, bool CACHE>
__device__ __forceinline__ void wevaluate(const WCtx& C, WStep& p) {
    const int d = p.d;
    const float xo = C.xw[d];
    float lo, hi, sg;
    if (UB) { lo = C.lo_u; hi = C.hi_u; sg = C.sig_u; }
    else { lo = C.slo[d]; hi = C.shi[d]; sg = C.ssig[d]; }
    float xp = UP ? fmaf(hi - lo, p.z, lo) : fmaf(sg, p.z, xo);
    xp = reflect_clip(xp, lo, hi, C.boundary == 0);
    p.xo = xo;
    p.xp = xp;
    if (COST == kSchwefel || COST == kRastrigin) {
        const float ho = CACHE ? C.hw[d] : term<COST>(xo);
        p.hp = term<COST>(xp);
        p.dF = COST == kSchwefel ? (ho - p.hp) * C.inv_n : p.hp - ho;
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

// Sum over the G lanes of a group (every lane of the group receives it).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

struct ChainEnd {
    double Fa, ec;   // F_start + dS and the bound on its error
    unsigned nacc;   // accepted moves
};

// One level of the chain c held by the calling group (all 32 lanes of the
// warp call it together; `mine` is false for a group without a chain, whose
// lanes take part in the warp-wide votes only).
template <int COST, bool UB, bool UP, int G, bool CACHE>
__device__ ChainEnd group_chain(const SweepArgs& A, const ProbDev& P, int64_t c, bool mine, int level, float* xw,
                                float* hw, const float* slo, const float* shi, const float* ssig) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);      // position in the group = step offset
    const int gi = lane / G;            // group within the warp
    const int n = P.n;
    const int64_t gc = P.chain_base + c;
    const double T = A.T_tab[level];
    const float sl = (float)A.s_tab[level];
    const float inv_n = 1.0f / (float)n;

    // ---- state at the start of the level
    if (!mine) {
        for (int k = gl; k <= n; k += G) xw[k] = 0.0f;
    } else if (level == 0) {
        for (int k = 4 * gl; k < n; k += 4 * G) {
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
        for (int k = gl; k < n; k += G) xw[k] = A.X32[P.x_base + (size_t)k * (size_t)P.chains + (size_t)c];
    } else {
        for (int k = gl; k < n; k += G) xw[k] = P.x_best32[k];
    }
    __syncwarp();
    if (CACHE && (COST == kSchwefel || COST == kRastrigin)) {
        for (int k = gl; k < n; k += G) hw[k] = term<COST>(xw[k]);
        __syncwarp();
    }

    double Fs = 0.0;
    float es = 0.0f;
    if (level == 0 || own_start(A, level)) {  // warp-uniform
        // FP32 value of f at the start point with a bound on its error; the
        // group sums run on every lane of the warp (a group without a chain adds zeros)
        float sum = 0.0f, sabs = 0.0f, e = 0.0f;
        if (mine) {
            for (int k = gl; k < n; k += G) {
                const float x = xw[k];
                float g;
                if (COST == kSchwefel) {
                    g = term<COST>(x);
                    e += fabsf(x) * fmaf(sqrt_approx(fabsf(x)), 4.8e-7f, 2.6e-6f);
                } else if (COST == kRastrigin) {
                    g = term<COST>(x);
                    e += 2.4e-5f + fabsf(g) * 1.2e-7f;
                } else {
                    g = k + 1 < n ? rosen_term(x, xw[k + 1], e) : 0.0f;
                }
                sum += g;
                sabs += fabsf(g);
            }
        }
        sum = group_sum<G>(sum);
        sabs = group_sum<G>(sabs);
        e = group_sum<G>(e);
        // sequential sums of ceil(n/G) terms, then log2 G tree levels
        const float rnd = ((float)((n + G - 1) / G) + (float)Log2<G>::v + 1.0f) * 1.2e-7f;
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

    const bool trace_on = (A.bits != nullptr) && level < A.trace_levels;  // warp-uniform
    const bool tracing = mine && trace_on;
    uint32_t* mybits = tracing ? A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)gc) * (size_t)A.words : nullptr;
    const unsigned lt = lanemask_lt();
    const unsigned gmask = G == 32 ? kFull : ((1u << G) - 1u) << (gi * G);
    // Per-lane sums of the accepted differences (lane gl holds the steps
    // s = gl mod G) and of the bounds on their FP32 errors; reduced once at the end.
    // Each accepted step adds its difference's bound plus u |dS| for the rounding
    // of the running sum.  Where the difference's bound is the constant kappa
    // (Schwefel, Rastrigin) the lane keeps sum |dS| over its accepted steps and
    // forms nacc kappa + u sum |dS| once at the end.
    float dS = 0.0f, e = 0.0f, sabs_acc = 0.0f;
    unsigned nacc = 0, bw = 0;
    const int L = (int)opaque((uint32_t)A.L);
    // Each lane draws the Philox block of its next round's step while the
    // current round evaluates: the block depends on the step counter alone, so
    // its ten dependent rounds of products fill the latency of this round's
    // loads, shuffles and SFU functions.  (The block drawn in the last round
    // belongs to a step past L and is not used.)
    uint4 wn = philox_step((uint32_t)gl, C.pf, C.rk);
    // one round: steps s0 .. s0 + G - 1, one per lane (live: the lane's step exists;
    // trace_c: std::true_type when the level records its accept bits)
    auto round = [&](int s0, bool live, auto trace_c) {
        constexpr bool kTrace = decltype(trace_c)::value;
        const int s = s0 + gl;
        const uint4 w = wn;
        wn = philox_step((uint32_t)(s + G), C.pf, C.rk);
        WStep p;
        wpropose<UP>(C, w, p);
        wevaluate<COST, UB, UP, CACHE>(C, p);
        bool acc, pend;
        if (G < 32) {
            // pending: an earlier lane of the group touches what this lane's evaluation
            // read -- its coordinate, or for Rosenbrock a neighbour (G - 1 shuffles
            // within the group; a warp-wide match costs far more on this GPU).  Keying
            // the test on the earlier lanes' speculative acceptances instead would
            // leave fewer lanes pending for the separable costs, but at this
            // schedule's acceptance rates (about 50 to 90%) it measured slower.
            const int key = live ? p.d : -1 - lane;
            bool hit = false;
#pragma unroll
            for (int k = 1; k < G; ++k) {
                const int dk = __shfl_up_sync(kFull, key, k, G);
                hit |= (gl >= k) && (COST == kRosenbrock ? (dk >= p.d - 1 && dk <= p.d + 1) : dk == p.d);
            }
            pend = live && hit;
            acc = live && !pend && (p.dF < p.tau);
            // Branch-free commit, with no barrier after the speculative reads:
            // lanes that do not accept write to the scratch slot n of their row,
            // and an accepting lane is the first of its group to touch its
            // coordinate, so no other lane's speculative read of this round saw
            // it (a later lane that did is pending and reads again below).
            const int slot = acc ? p.d : n;
            xw[slot] = p.xp;
            if (CACHE && (COST == kSchwefel || COST == kRastrigin)) hw[slot] = p.hp;
            // pending lanes, by position in the group: the lane at position j reads
            // again once the lanes before it have committed
            const unsigned pendm = __ballot_sync(kFull, pend);
            if (pendm) {
                constexpr unsigned kRep = G == 2 ? 0x55555555u : (G == 4 ? 0x11111111u : 0x01010101u);
#pragma unroll 1
                for (int pos = 1; pos < G; ++pos) {
                    if (!(pendm & (kRep << pos))) continue;
                    __syncwarp();
                    WStep q = p;
                    wevaluate<COST, UB, UP, CACHE>(C, q);
                    const bool go = pend && gl == pos;
                    const bool a2 = q.dF < q.tau;
                    if (go) p = q;
                    acc = go ? a2 : acc;
                    __syncwarp();
                    const int slot2 = (go && a2) ? q.d : n;
                    xw[slot2] = q.xp;
                    if (CACHE && (COST == kSchwefel || COST == kRastrigin)) hw[slot2] = q.hp;
                }
            }
        } else {
            // one chain per warp: the lanes sharing a coordinate, by a warp-wide match
            const int key = live ? p.d : -1 - lane;
            unsigned earlier;
            if (COST == kRosenbrock) {
                earlier = 0u;
                for (int k = 0; k < 31; ++k) {
                    const int dk = __shfl_sync(kFull, key, k);
                    earlier |= ((k < lane) && dk >= p.d - 1 && dk <= p.d + 1) ? (1u << k) : 0u;
                }
            } else {
                earlier = __match_any_sync(kFull, key) & lt;  // every lane takes part, live or not
            }
            pend = live && earlier != 0u;
            acc = live && !pend && (p.dF < p.tau);
            __syncwarp();  // every speculative read happens before any write
            int slot = acc ? p.d : n;
            xw[slot] = p.xp;
            if (CACHE && (COST == kSchwefel || COST == kRastrigin)) hw[slot] = p.hp;
            // pending lanes, in rounds: a lane goes once every earlier conflicting
            // lane is decided; the whole warp evaluates, the going lanes keep it
            unsigned undecided = __ballot_sync(kFull, pend);
            while (undecided) {
                __syncwarp();
                const bool go = ((undecided >> lane) & 1u) && (earlier & undecided) == 0u;
                WStep q = p;
                wevaluate<COST, UB, UP, CACHE>(C, q);
                const bool a2 = q.dF < q.tau;
                if (go) p = q;
                acc = go ? a2 : acc;
                __syncwarp();
                slot = (go && a2) ? q.d : n;
                xw[slot] = q.xp;
                if (CACHE && (COST == kSchwefel || COST == kRastrigin)) hw[slot] = q.hp;
                undecided &= ~__ballot_sync(kFull, go);
            }
        }
        __syncwarp();  // this round's writes before the next round's reads
        dS += acc ? p.dF : 0.0f;
        if (COST == kRosenbrock) e += acc ? rosen_bound(C, p) + fabsf(dS) * 1.2e-7f : 0.0f;
        else sabs_acc += acc ? fabsf(dS) : 0.0f;
        nacc += acc ? 1u : 0u;
        if (kTrace) {
            const unsigned accm = __ballot_sync(kFull, acc) & gmask;
            bw |= (G == 32 ? accm : accm >> (gi * G)) << (s0 & 31);
            if (((s0 & 31) + G == 32) || s0 + G >= L) {
                if (tracing && gl == 0) mybits[s0 >> 5] = bw;
                bw = 0;
            }
        }
    };
    // The level's rounds, with the choices that hold for the whole level taken
    // once: tracing or not, and whether every group of the warp holds a chain.
    auto rounds = [&](auto trace_c) {
        int s0 = 0;
        if (__all_sync(kFull, mine)) {
            for (; s0 + G <= L; s0 += G) round(s0, true, trace_c);  // full rounds
        } else {
            for (; s0 + G <= L; s0 += G) round(s0, mine, trace_c);
        }
        if (s0 < L) round(s0, mine && s0 + gl < L, trace_c);  // the last, partial round
    };
    if (trace_on) rounds(std::true_type{});
    else rounds(std::false_type{});
    (void)gmask;
    if (COST != kRosenbrock) e = fmaf((float)nacc, kappa, sabs_acc * 1.2e-7f);
    // lane sums -> chain sums (log2 G tree levels: their rounding is bounded by log2(G) u sum|dS_lane|)
    float dabs = group_sum<G>(fabsf(dS));
    dS = group_sum<G>(dS);
    e = group_sum<G>(e);
    nacc = group_sum<G>(nacc);
    e += (float)Log2<G>::v * 1.2e-7f * dabs;

    const double Fa = Fs + (double)dS;
    const double ec = (double)es + (double)e;
    return ChainEnd{Fa, ec, nacc};
}

template <int COST, int G, bool CACHE>
__device__ __forceinline__ ChainEnd dispatch_chain(const SweepArgs& A, const ProbDev& P, int64_t c, bool mine, int level,
                                                   float* xw, float* hw, const float* slo, const float* shi,
                                                   const float* ssig, bool ub, bool up) {
    if (up) {
        return ub ? group_chain<COST, true, true, G, CACHE>(A, P, c, mine, level, xw, hw, slo, shi, ssig)
                  : group_chain<COST, false, true, G, CACHE>(A, P, c, mine, level, xw, hw, slo, shi, ssig);
    }
    return ub ? group_chain<COST, true, false, G, CACHE>(A, P, c, mine, level, xw, hw, slo, shi, ssig)
              : group_chain<COST, false, false, G, CACHE>(A, P, c, mine, level, xw, hw, slo, shi, ssig);
}

// Block-level scratch of a group tile (static shared memory of the calling kernel),
// for up to MAXC chains per block: sized by the layout, since a few hundred bytes
// decide whether one more block fits on an SM.
template <int MAXC>
struct GroupSharedN {
    unsigned block_acc;
    int ncand;
    double block_M;
    double chain_hi[MAXC];
    int cand[MAXC];
};
using GroupShared = GroupSharedN<kGroupMaxBlock / 2>;  // any layout (G >= 2)

// One tile of chains in the group layout: G lanes per chain, blockDim.x / G chains.
// smem_raw: the dynamic shared memory (state rows, cached terms, box arrays).
template <int G, bool CACHE, int MAXC>
__device__ void group_tile(const SweepArgs& A, const ProbDev& P, const WorkItem& it, int level, unsigned char* smem_raw,
                           GroupSharedN<MAXC>& sh) {
    constexpr int kMaxChains = kGroupMaxBlock / G;
    static_assert(MAXC >= kMaxChains, "block scratch smaller than the layout's chains");
    unsigned& block_acc = sh.block_acc;
    double* chain_hi = sh.chain_hi;
    double& block_M = sh.block_M;
    int* cand = sh.cand;
    int& ncand = sh.ncand;
    const int n = P.n;
    const int CB = blockDim.x / G;              // chains per block
    const int cb = threadIdx.x / G;             // this group's chain
    const int gl = threadIdx.x & (G - 1);
    float* xs = reinterpret_cast<float*>(smem_raw);                    // [CB][n + 1] states
    float* hs = xs + (size_t)CB * (n + 1);                             // [CB][n + 1] cached terms (CACHE)
    float* slo = hs + (CACHE ? (size_t)CB * (n + 1) : 0);
    float* shi = slo + n;
    float* ssig = shi + n;
    const bool ub = P.uniform != 0;
    const bool up = A.proposal == 1;
    if (threadIdx.x == 0) { block_acc = 0u; ncand = 0; }
    if (!ub) {
        const float sl = (float)A.s_tab[level];
        for (int k = threadIdx.x; k < n; k += blockDim.x) { slo[k] = P.lo32[k]; shi[k] = P.hi32[k]; ssig[k] = P.sig32[k] * sl; }
    }
    __syncthreads();
    const bool mine = cb < it.count;
    const bool warp_busy = (threadIdx.x & ~31) / G < it.count;  // the warp's first group has a chain
    float* xw = xs + (size_t)cb * (n + 1);  // row of n coordinates plus the scratch slot n
    float* hw = hs + (size_t)cb * (n + 1);
    const int64_t c = it.c0 + cb;
    ChainEnd end{CUDART_INF, 0.0, 0u};
    if (warp_busy) {
        switch (P.cost) {
        case kSchwefel: end = dispatch_chain<kSchwefel, G, CACHE>(A, P, c, mine, level, xw, hw, slo, shi, ssig, ub, up); break;
        case kRastrigin: end = dispatch_chain<kRastrigin, G, CACHE>(A, P, c, mine, level, xw, hw, slo, shi, ssig, ub, up); break;
        case kRosenbrock: end = dispatch_chain<kRosenbrock, G, CACHE>(A, P, c, mine, level, xw, hw, slo, shi, ssig, ub, up); break;
        default:
            if ((threadIdx.x & 31) == 0) A.run->status = 1;
            break;
        }
    }
    const bool finite = mine && isfinite(end.Fa);
    if (gl == 0 && cb < kMaxChains) chain_hi[cb] = finite ? end.Fa + end.ec : CUDART_INF;
    __syncthreads();
    // one atomicMin per block on the device-wide threshold M = min(F + e)
    if (threadIdx.x == 0) {
        double bmin = chain_hi[0];
        for (int j = 1; j < CB; ++j) bmin = fmin(bmin, chain_hi[j]);
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
    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    const int64_t gc = P.chain_base + c;
    if (mine) {
        if (finite && (tracing || level == A.full_level || A.crossover || end.Fa - end.ec <= block_M)) {
            if (gl == 0) cand[atomicAdd(&ncand, 1)] = cb;
        } else {
            if (gl == 0) A.F[gc] = finite ? CUDART_INF : CUDART_NAN;
            if (keep_states(A)) {  // every chain keeps its state for the next level
                float* dst = A.X32 + P.x_base + c;
                for (int k = gl; k < n; k += G) dst[(size_t)k * (size_t)P.chains] = xw[k];
            }
        }
        if (gl == 0) atomicAdd(&block_acc, end.nacc);
    }
    __syncthreads();
    // one warp per candidate: lane-strided FP64 partial sums in index order, then the butterfly
    const int lane = threadIdx.x & 31;
    const int nc = ncand;
    for (int j = threadIdx.x >> 5; j < nc; j += blockDim.x >> 5) {
        const int tc = cand[j];
        const float* xr = xs + (size_t)tc * (n + 1);
        double p1 = 0.0;
        switch (P.cost) {
        case kSchwefel: for (int k = lane; k < n; k += 32) partial64<kSchwefel>(xr, n, k, p1); break;
        case kRastrigin: for (int k = lane; k < n; k += 32) partial64<kRastrigin>(xr, n, k, p1); break;
        default: for (int k = lane; k < n; k += 32) partial64<kRosenbrock>(xr, n, k, p1); break;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p1 += __shfl_xor_sync(kFull, p1, o);
        const int64_t cc = it.c0 + tc;
        if (lane == 0) {
            A.F[P.chain_base + cc] = P.cost == kSchwefel ? -(p1 / (double)n)
                                   : (P.cost == kRastrigin ? 10.0 * (double)n + p1 : p1);
        }
        float* dst = A.X32 + P.x_base + cc;
        for (int k = lane; k < n; k += 32) dst[(size_t)k * (size_t)P.chains] = xr[k];
    }
    if (threadIdx.x == 0 && block_acc) atomicAdd(P.accepts, (unsigned long long)block_acc);
}

}  // namespace
}  // namespace sa
