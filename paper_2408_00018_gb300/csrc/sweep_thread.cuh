// sweep_thread.cuh -- the chain-per-thread FP32 sweep of one tile of chains
// (device code shared by the chain-per-thread kernel and the batched level
// kernel).
//
// One thread runs one Markov chain for the L steps of a level (the kernel of
// Listing 4): pick a coordinate, Gaussian move, reflect/clip into the box,
// energy difference, Boltzmann acceptance (Eq. "proba", k_b = 1).  The
// chain's state lives in shared memory as x[d][lane] (bank = lane, so the
// random coordinate of each lane never conflicts).  Separable costs use the
// O(1) difference of the terms that touch coordinate d instead of the
// paper's full recompute of f(x1).
//
// Steps of one chain are independent except through the coordinates they
// touch, so U consecutive steps are proposed and evaluated together (their
// Philox blocks, transcendental functions and state loads interleave), then
// committed in order; a step whose coordinate (or, for Rosenbrock, a
// neighbour; for Ackley, any coordinate) was changed by an earlier accepted
// step of the same group is re-evaluated from the current state before its
// decision.  The decisions are exactly those of the one-step-at-a-time chain.
//
// At the end of the level every chain holds F_start + dS with a running
// bound e on its FP32 error.  The block takes part in a device-wide
// threshold M = min(F + e) (atomicMin on an ordered key); only chains with
// F - e <= M can hold the level's minimum, and only those are re-evaluated
// in FP64 and have their state written to global memory.  The FP64 argmin
// over those candidates (reduce.cu) is therefore exact.

#pragma once
#include <type_traits>
#include <cfloat>
#include <cmath>
#include <math_constants.h>

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kMaxBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sums of two doubles; every thread receives the totals.
__device__ void block_sum2(double& a, double& b, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    __syncthreads();
    if (lane == 0) { red[wid] = a; red[32 + wid] = b; }
    __syncthreads();
    double sa_ = 0.0, sb = 0.0;
    for (int i = 0; i < nw; ++i) { sa_ += red[i]; sb += red[32 + i]; }
    a = sa_;
    b = sb;
}

__device__ double block_min(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_min(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double m = red[0];
    for (int i = 1; i < nw; ++i) m = fmin(m, red[i]);
    return m;
}

// FP64 partial sums of the cost at x (coordinate k of column tc of xs), strided over the block.
template <int COST>
__device__ void partials64(const float* xs, int B, int n, int tc, double& p1, double& p2) {
    p1 = 0.0;
    p2 = 0.0;
    for (int k = threadIdx.x; k < n; k += B) {
        const double x = (double)xs[k * B + tc];
        if (COST == kSchwefel) p1 += h64_schwefel(x);
        else if (COST == kRastrigin) p1 += g64_rastrigin(x);
        else if (COST == kAckley) { p1 += x * x; p2 += cos(6.283185307179586 * x); }
        else if (COST == kRosenbrock) { if (k + 1 < n) p1 += rosen64(x, (double)xs[(k + 1) * B + tc]); }
    }
}
template <int COST>
__device__ __forceinline__ double assemble64(int n, double p1, double p2) {
    if (COST == kSchwefel) return -(p1 / (double)n);
    if (COST == kRastrigin) return 10.0 * (double)n + p1;
    if (COST == kAckley) return ackley64(n, p1, p2);
    return p1;
}

// FP32 value of the cost at the chain's own column, with an error bound (level 0 start).
template <int COST>
__device__ float start_value32(const float* xs, int B, int n, int t, float inv_n, float& eb, SepState& st) {
    float s = 0.0f, sabs = 0.0f, e = 0.0f;
    st.s1 = 0.0f;
    st.s2 = 0.0f;
    for (int k = 0; k < n; ++k) {
        const float x = xs[k * B + t];
        if (COST == kSchwefel) {
            const float r = sqrt_approx(fabsf(x));
            const float g = x * sin_reduced(r);
            e += fabsf(x) * fmaf(r, 4.8e-7f, 2.6e-6f);
            s += g;
            sabs += fabsf(g);
        } else if (COST == kRastrigin) {
            const float g = g_rastrigin(x);
            e += 2.4e-5f + fabsf(g) * 1.2e-7f;
            s += g;
            sabs += fabsf(g);
        } else if (COST == kAckley) {
            st.s1 = fmaf(x, x, st.s1);
            st.s2 += cos2pi(x);
        } else if (COST == kRosenbrock) {
            if (k + 1 < n) {
                const float g = rosen_term(x, xs[(k + 1) * B + t], e);
                s += g;
                sabs += g;
            }
        }
    }
    float F;
    if (COST == kSchwefel) {
        F = -s * inv_n;
        eb = (e + sabs * 1.2e-7f * (float)n) * inv_n + fabsf(F) * 1.2e-7f;
    } else if (COST == kRastrigin) {
        F = 10.0f * (float)n + s;
        eb = e + (sabs + 10.0f * n) * 1.2e-7f * (float)n;
    } else if (COST == kAckley) {
        st.a = ackley_value(st.s1, st.s2, inv_n);
        F = st.a;
        eb = 1e-4f + 2.4e-7f * (float)n * 50.0f;
    } else {
        F = s;
        eb = e + sabs * 1.2e-7f * (float)n;
    }
    return F;
}

// Producer/consumer form of the chain-per-thread tile (PD below): steps drawn ahead per
// phase, and the ring's size for S chains (two phases of coordinate, deviate, threshold).
constexpr int kPdSteps = 8;
__host__ __device__ constexpr size_t kPdRingBytes(int S) { return (size_t)2 * kPdSteps * S * 12; }

// One proposed step.  a, b: cost-specific values kept for the error bound
// (Schwefel: sqrt|xo|, sqrt|xp|; Rastrigin: g(xo), g(xp); Rosenbrock: the
// neighbours x_{d-1}, x_{d+1}; Ackley: the candidate sums).
struct Step {
    int d;
    float z, tau, xo, xp, dF, a, b, ap;
    float co, cp;  // Ackley: cos 2 pi xo, cos 2 pi xp
};

struct Ctx {
    float* xcol;       // this chain's column (stride B)
    int B, n;
    float inv_n;
    float lo_u, hi_u, sig_u;         // uniform box (sig_u already scaled by sqrt(T/T0))
    const float *slo, *shi, *ssig;   // per-coordinate box (ssig scaled)
    int boundary;
    float neg_T_ln2;  // -T ln 2: tau = -T ln u3 = neg_T_ln2 * log2(u3)
    float kappa;      // bound on the FP32 error of any accepted step's dF over the box (Schwefel, Rastrigin)
    PhiloxFixed pf;     // the parts of the step's Philox rounds 1-2 fixed for the chain and level
    const uint32_t* rk; // the sweep key of every Philox round (kernel parameters)
};

// Randomness of step s: coordinate, Gaussian deviate, acceptance threshold.
// UP: the move is a uniform redraw of the coordinate (z = u2) instead of a Gaussian step.
template <bool UP>
__device__ __forceinline__ void propose(const Ctx& C, uint32_t s, Step& p) {
    // = philox4x32_10((s, level, chain, problem), key) bit for bit
    const uint4 w = philox_step(s, C.pf, C.rk);
    p.d = coord_of(w.x, C.n);
    const float u1 = u23f(w.y), u2 = u23f(w.z), u3 = u23f(w.w);
    if (UP) {
        p.z = u2;  // uniform redraw: x' = lo + u2 (hi - lo)
    } else {
        // Box-Muller, cosine branch: z = sqrt(-2 ln u1) cos(2 pi u2) = -sqrt(..) cos(2 pi (u2 - 1/2)).
        const float r = sqrt_approx(-1.3862943611198906f * lg2_approx(u1));
        p.z = -r * cos_approx(6.28318530717958648f * (u2 - 0.5f));
    }
    // u3 < exp(-dF/T)  <=>  dF < tau = -T ln u3   (tau > 0, so dF <= 0 is always accepted)
    p.tau = C.neg_T_ln2 * lg2_approx(u3);
}

// The proposed step's move from the chain's current state: p.xo, p.xp.
template <bool UB, bool UP>
__device__ __forceinline__ void move_to(const Ctx& C, Step& p) {
    const int d = p.d;
    const float xo = C.xcol[d * C.B];
    float lo, hi, sg;
    if (UB) { lo = C.lo_u; hi = C.hi_u; sg = C.sig_u; }
    else { lo = C.slo[d]; hi = C.shi[d]; sg = C.ssig[d]; }
    float xp = UP ? fmaf(hi - lo, p.z, lo) : fmaf(sg, p.z, xo);
    xp = reflect_clip(xp, lo, hi, C.boundary == 0);
    p.xo = xo;
    p.xp = xp;
}

// Ackley: the part of a step's difference that depends on the running sums.
__device__ __forceinline__ void ackley_dep(const Ctx& C, const SepState& st, Step& p) {
    p.a = fmaf(p.xp - p.xo, p.xp + p.xo, st.s1);
    p.b = st.s2 + (p.cp - p.co);
    p.ap = ackley_value(p.a, p.b, C.inv_n);
    p.dF = p.ap - st.a;
}

// Move and energy difference of a proposed step from the chain's current state.
template <int COST, bool UB, bool UP>
__device__ __forceinline__ void evaluate(const Ctx& C, const SepState& st, Step& p) {
    move_to<UB, UP>(C, p);
    const int d = p.d;
    const float xo = p.xo, xp = p.xp;
    if (COST == kSchwefel) {
        const float ro = sqrt_approx(fabsf(xo)), rp = sqrt_approx(fabsf(xp));
        p.dF = (xo * sin_reduced(ro) - xp * sin_reduced(rp)) * C.inv_n;
        p.a = ro;
        p.b = rp;
    } else if (COST == kRastrigin) {
        const float go = g_rastrigin(xo), gp = g_rastrigin(xp);
        p.dF = gp - go;
        p.a = go;
        p.b = gp;
    } else if (COST == kAckley) {
        p.co = cos2pi(xo);
        p.cp = cos2pi(xp);
        ackley_dep(C, st, p);
    } else {
        float dummy = 0.0f, before = 0.0f, after = 0.0f;
        const float xm = d > 0 ? C.xcol[(d - 1) * C.B] : 0.0f;
        const float xq = d + 1 < C.n ? C.xcol[(d + 1) * C.B] : 0.0f;
        if (d > 0) { before += rosen_term(xm, xo, dummy); after += rosen_term(xm, xp, dummy); }
        if (d + 1 < C.n) { before += rosen_term(xo, xq, dummy); after += rosen_term(xp, xq, dummy); }
        p.dF = after - before;
        p.a = xm;
        p.b = xq;
        p.ap = before + after;
    }
}

// Bound on the FP32 error of an accepted step's dF (see sa_device.cuh for the constants).
template <int COST>
__device__ __forceinline__ float step_bound(const Ctx& C, const Step& p) {
    if (COST == kSchwefel)
        return (fabsf(p.xo) * fmaf(p.a, 4.8e-7f, 2.6e-6f) + fabsf(p.xp) * fmaf(p.b, 4.8e-7f, 2.6e-6f)) * C.inv_n +
               fabsf(p.dF) * 2.4e-7f;
    if (COST == kRastrigin) return 4.8e-5f + (fabsf(p.a) + fabsf(p.b) + fabsf(p.dF)) * 1.2e-7f;
    if (COST == kAckley) return 1e-4f + fabsf(p.dF) * 2.4e-7f;
    float eb = 0.0f;
    if (p.d > 0) { rosen_term(p.a, p.xo, eb); rosen_term(p.a, p.xp, eb); }
    if (p.d + 1 < C.n) { rosen_term(p.xo, p.b, eb); rosen_term(p.xp, p.b, eb); }
    return eb + (p.ap + fabsf(p.dF)) * 1.2e-7f;
}

// Does an accepted earlier step k invalidate the speculative evaluation of step j?
template <int COST>
__device__ __forceinline__ bool conflicts(int dk, int dj) {
    if (COST == kAckley) return true;                              // global sums changed
    if (COST == kRosenbrock) return dk >= dj - 1 && dk <= dj + 1;  // neighbour terms
    return dk == dj;
}

// R: steps whose randomness (Philox block, coordinate, Gaussian deviate,
// acceptance threshold) is drawn together before any of them is evaluated.
// The randomness does not depend on the chain's state, so the R draws are
// independent of each other and of the evaluations: drawing them as one batch
// gives the integer-multiply pipe (the 32 x 32 -> 64-bit products of Philox)
// R independent instruction streams per thread, where the sweep otherwise
// has only the U speculative steps.  The decisions are unchanged.
// S: the tile's chain capacity, the stride of the state columns (<= blockDim.x;
// threads from S on hold no chain and take part in the block's reductions only).
// PD (U = R = 1): the warps from ceil(S / 32) on hold no chain; they draw every chain's
// randomness kPdSteps steps ahead into a double-buffered ring (`ring`, kPdRingBytes(S)),
// and the chains' threads take it from there, so a chain's step is only its dependent
// part (evaluation and commit).  The proposals are those propose() makes for the chain,
// so the decisions equal the chain-per-thread ones bit for bit.
template <int COST, bool UB, int U, bool UP, int R, bool PD = false>
__device__ void sweep_tile(const SweepArgs& A, const ProbDev& P, const WorkItem& it, int S, int level,
                           float* xs, float* slo, float* shi, float* ssig, double* red, int* cand, int* ncand,
                           float* ring = nullptr) {
    const int t = threadIdx.x, NT = blockDim.x, B = S, n = P.n;
    const bool active = t < it.count && t < S;
    const int64_t c = it.c0 + t;
    const int64_t gc = P.chain_base + c;
    const double T = A.T_tab[level];
    const float sl = (float)A.s_tab[level];
    const float inv_n = 1.0f / (float)n;

    if (!UB)
        for (int k = t; k < n; k += NT) { slo[k] = P.lo32[k]; shi[k] = P.hi32[k]; ssig[k] = P.sig32[k] * sl; }
    if (level == 0) {
        if (active) {
            for (int k = 0; k < n; k += 4) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)(k >> 2), 0u, (uint32_t)c + P.cid0, P.pid), A.ikey0, A.ikey1);
                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (k + j < n) {
                        const double lo = P.lo[k + j], hi = P.hi[k + j];
                        float x = (float)(lo + u23d(ww[j]) * (hi - lo));
                        x = fminf(fmaxf(x, P.lo32[k + j]), P.hi32[k + j]);
                        xs[(k + j) * B + t] = x;
                    }
                }
            }
        }
    } else if (own_start(A, level)) {  // the chain's own state (no exchange before this level)
        if (active)
            for (int k = 0; k < n; ++k) xs[k * B + t] = A.X32[P.x_base + (size_t)k * (size_t)P.chains + (size_t)c];
    } else if (t < S) {
        for (int k = 0; k < n; ++k) xs[k * B + t] = P.x_best32[k];
    }
    __syncthreads();

    double Fs = 0.0;
    float es = 0.0f;
    SepState st{0.0f, 0.0f, 0.0f};
    if (level == 0 || own_start(A, level)) {
        if (active) Fs = (double)start_value32<COST>(xs, B, n, t, inv_n, es, st);
    } else {
        Fs = P.scal[kFBest];
        if (COST == kAckley) {
            st.s1 = (float)P.scal[kS1];
            st.s2 = (float)P.scal[kS2];
            st.a = ackley_value(st.s1, st.s2, inv_n);
            es = 1e-4f;
        }
    }

    Ctx C;
    C.xcol = xs + t;
    C.B = B;
    C.n = n;
    C.inv_n = inv_n;
    C.lo_u = P.lo_u;
    C.hi_u = P.hi_u;
    C.sig_u = P.sig_u * sl;
    C.slo = slo;
    C.shi = shi;
    C.ssig = ssig;
    C.boundary = A.boundary;
    C.neg_T_ln2 = (float)(-T * 0.69314718055994531);
    C.kappa = P.kappa;
    C.rk = A.rk;
    C.pf = philox_prep((uint32_t)level, (uint32_t)c + P.cid0, P.pid, A.rk);

    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    uint32_t* mybits = tracing ? A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)gc) * (size_t)A.words : nullptr;
    float dS = 0.0f, e = 0.0f;
    uint32_t nacc = 0;
    // The level's steps; trace_c is std::true_type when the level records its
    // accept bits, so the untraced levels carry no per-step test for it.
    auto run_steps = [&](auto trace_c) {
        constexpr bool kTrace = decltype(trace_c)::value;
        uint32_t bw = 0;
        const int L = A.L;
        int s = 0;
        auto commit = [&](Step& p, int sidx) -> bool {
            const bool acc = p.dF < p.tau;
            if (COST == kSchwefel || COST == kRastrigin) {
                // without a divergent branch (12% faster at n = 256): a rejected step
                // stores the value it read, and the error grows by the box-wide
                // per-step bound kappa
                C.xcol[p.d * B] = acc ? p.xp : p.xo;
                dS += acc ? p.dF : 0.0f;
                e += acc ? fmaf(fabsf(dS), 1.2e-7f, C.kappa) : 0.0f;
                nacc += acc ? 1u : 0u;
            } else if (acc) {
                C.xcol[p.d * B] = p.xp;
                dS += p.dF;
                e += step_bound<COST>(C, p) + fabsf(dS) * 1.2e-7f;
                ++nacc;
                if (COST == kAckley) { st.s1 = p.a; st.s2 = p.b; st.a = p.ap; }
            }
            if (kTrace) {
                bw |= (acc ? 1u : 0u) << (sidx & 31);
                if ((sidx & 31) == 31 || sidx == L - 1) { mybits[sidx >> 5] = bw; bw = 0; }
            }
            return acc;
        };
        if (PD) {
            // ring: proposals [2][kPdSteps][S] as coordinates, deviates, thresholds
            int* rd = reinterpret_cast<int*>(ring);
            float* rz = ring + 2 * kPdSteps * S;
            float* rt = rz + 2 * kPdSteps * S;
            const int DW = (S + 31) >> 5;           // warps holding chains
            const bool producer = (t >> 5) >= DW;  // warp-uniform
            const int tp = t - 32 * DW, NP = NT - 32 * DW;
            const int phases = (L + kPdSteps - 1) / kPdSteps;
            auto produce = [&](int ph) {  // steps ph kPdSteps .. of every chain of the tile
                const int buf = ph & 1, s0 = ph * kPdSteps;
                const int cnt = min(kPdSteps, L - s0);
                for (int q = tp; q < cnt * S; q += NP) {
                    const int j = q / S, ch = q - j * S;
                    if (ch >= it.count) continue;
                    Ctx Cq = C;
                    Cq.pf = philox_prep((uint32_t)level, (uint32_t)(it.c0 + ch) + P.cid0, P.pid, A.rk);
                    Step p;
                    propose<UP>(Cq, (uint32_t)(s0 + j), p);
                    const int o = (buf * kPdSteps + j) * S + ch;
                    rd[o] = p.d;
                    rz[o] = p.z;
                    rt[o] = p.tau;
                }
            };
            if (producer) produce(0);
            __syncthreads();
            for (int ph = 0; ph < phases; ++ph) {  // every thread of the block: one barrier per phase
                if (producer) {
                    if (ph + 1 < phases) produce(ph + 1);
                } else if (active) {
                    const int buf = ph & 1, s0 = ph * kPdSteps;
                    const int cnt = min(kPdSteps, L - s0);
                    auto fetch = [&](int j, Step& p) {
                        const int o = (buf * kPdSteps + j) * S + t;
                        p.d = rd[o];
                        p.z = rz[o];
                        p.tau = rt[o];
                    };
                    for (int j = 0; j < cnt; ++j) {
                        Step p;
                        fetch(j, p);
                        evaluate<COST, UB, UP>(C, st, p);
                        commit(p, s0 + j);
                    }
                }
                __syncthreads();
            }
            s = L;
        }
        if (!PD && R > U) {
            for (; s + R <= L; s += R) {
                Step p[R];
#pragma unroll
                for (int j = 0; j < R; ++j) propose<UP>(C, (uint32_t)(s + j), p[j]);
#pragma unroll
                for (int g = 0; g < R; g += U) {
#pragma unroll
                    for (int j = 0; j < U; ++j) evaluate<COST, UB, UP>(C, st, p[g + j]);
                    bool acc[U];
#pragma unroll
                    for (int j = 0; j < U; ++j) {
                        bool dirty = false;
#pragma unroll
                        for (int k = 0; k < j; ++k) dirty |= acc[k] && conflicts<COST>(p[g + k].d, p[g + j].d);
                        if (dirty) evaluate<COST, UB, UP>(C, st, p[g + j]);
                        acc[j] = commit(p[g + j], s + g + j);
                    }
                }
            }
        }
        if (U > 1) {
            for (; s + U <= L; s += U) {
                Step p[U];
#pragma unroll
                for (int j = 0; j < U; ++j) propose<UP>(C, (uint32_t)(s + j), p[j]);
#pragma unroll
                for (int j = 0; j < U; ++j) evaluate<COST, UB, UP>(C, st, p[j]);
                bool acc[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    bool dirty = false;
#pragma unroll
                    for (int k = 0; k < j; ++k) dirty |= acc[k] && conflicts<COST>(p[k].d, p[j].d);
                    if (dirty) evaluate<COST, UB, UP>(C, st, p[j]);
                    acc[j] = commit(p[j], s + j);
                }
            }
        }
        for (; s < L; ++s) {
            Step p;
            propose<UP>(C, (uint32_t)s, p);
            evaluate<COST, UB, UP>(C, st, p);
            commit(p, s);
        }
    };
    if (active || PD) {
        if (tracing) run_steps(std::true_type{});
        else run_steps(std::false_type{});
    }

    // ---- candidates for the FP64 argmin -------------------------------------
    const double Fa = Fs + (double)dS;
    const double ec = (double)es + (double)e;
    const bool finite = active && isfinite(Fa);
    const double lo_c = finite ? Fa - ec : CUDART_INF;
    const double hi_c = finite ? Fa + ec : CUDART_INF;
    double bmin = block_min(hi_c, red);
    if (t == 0) {
        *ncand = 0;
        double M = bmin;
        if (bmin < CUDART_INF) {
            const unsigned long long old = atomicMin(P.level_min, dbl_key(bmin));
            M = fmin(M, key_dbl(old));
        } else {
            M = key_dbl(*(volatile unsigned long long*)P.level_min);
        }
        red[64] = M;
    }
    __syncthreads();
    const double M = red[64];
    const bool is_cand = finite && (tracing || level == A.full_level || A.crossover || lo_c <= M);
    if (is_cand) cand[atomicAdd(ncand, 1)] = t;
    else if (active) {
        A.F[gc] = finite ? CUDART_INF : CUDART_NAN;
        if (keep_states(A))  // every chain keeps its state for the next level
            for (int k = 0; k < n; ++k) A.X32[P.x_base + (size_t)k * (size_t)P.chains + (size_t)c] = xs[k * B + t];
    }
    __syncthreads();
    // One warp per candidate: lane-strided partial sums in index order, then a
    // fixed butterfly, so the FP64 value does not depend on the block shape
    // (the chain-per-warp kernel evaluates candidates in the same order).
    const int nc = *ncand;
    const int lane = t & 31;
    for (int j = t >> 5; j < nc; j += (NT + 31) >> 5) {
        const int tc = cand[j];
        double p1 = 0.0, p2 = 0.0;
        for (int k = lane; k < n; k += 32) {
            const double x = (double)xs[k * B + tc];
            if (COST == kSchwefel) p1 += h64_schwefel(x);
            else if (COST == kRastrigin) p1 += g64_rastrigin(x);
            else if (COST == kAckley) { p1 += x * x; p2 += cos(6.283185307179586 * x); }
            else if (k + 1 < n) p1 += rosen64(x, (double)xs[(k + 1) * B + tc]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p1 += __shfl_xor_sync(0xffffffffu, p1, o);
            p2 += __shfl_xor_sync(0xffffffffu, p2, o);
        }
        if (lane == 0) A.F[P.chain_base + it.c0 + tc] = assemble64<COST>(n, p1, p2);
        float* dst = A.X32 + P.x_base + it.c0 + tc;
        for (int k = lane; k < n; k += 32) dst[(size_t)k * (size_t)P.chains] = xs[k * B + tc];
    }
    // accepted-move count of the tile
    double a1 = (double)nacc, a2 = 0.0;
    block_sum2(a1, a2, red);
    if (t == 0) atomicAdd(P.accepts, (unsigned long long)a1);
}

template <int COST, bool UB, bool UP, int R>
__device__ __forceinline__ void dispatch_r(const SweepArgs& A, const ProbDev& P, const WorkItem& it, int S, int level,
                                           float* xs, float* slo, float* shi, float* ssig, double* red, int* cand,
                                           int* ncand, int u) {
    if (UP || COST == kAckley || u <= 1)
        sweep_tile<COST, UB, 1, UP, R>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand);
    else if (u >= 4 && R == 1)  // (a batch of randomness takes U = 2)
        sweep_tile<COST, UB, 4, UP, 1>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand);
    else
        sweep_tile<COST, UB, 2, UP, R>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand);
}

template <int COST>
__device__ __forceinline__ void dispatch_u(const SweepArgs& A, const ProbDev& P, const WorkItem& it, int S, int level,
                                           float* xs, float* slo, float* shi, float* ssig, double* red, int* cand,
                                           int* ncand) {
    const bool ub = P.uniform != 0;
    const int u = (COST == kAckley) ? 1 : P.unroll;
    const bool batch = P.rand_batch > 1;
    if (A.proposal == 1) {  // uniform redraws: one step at a time
        if (batch) {
            if (ub) dispatch_r<COST, true, true, 16>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, 1);
            else dispatch_r<COST, false, true, 16>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, 1);
        } else {
            if (ub) dispatch_r<COST, true, true, 1>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, 1);
            else dispatch_r<COST, false, true, 1>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, 1);
        }
    } else if (batch) {
        if (ub) dispatch_r<COST, true, false, 16>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, u);
        else dispatch_r<COST, false, false, 16>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, u);
    } else {
        if (ub) dispatch_r<COST, true, false, 1>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, u);
        else dispatch_r<COST, false, false, 1>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand, u);
    }
}

}  // namespace
}  // namespace sa
