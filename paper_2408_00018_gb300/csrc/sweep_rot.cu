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

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kWarpsR = 4;
constexpr int kBlockR = 32 * kWarpsR;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float wsumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double wsumd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// sin(pi a) for |pi a| < 1/2: Taylor polynomial to degree 7 (truncation below
// 1.1e-8 relative).
__device__ __forceinline__ float sinpi_small(float a) {
    const float x = 3.14159265358979f * a;
    const float x2 = x * x;
    const float p = fmaf(x2, fmaf(x2, fmaf(x2, -1.98412698e-4f, 8.33333333e-3f), -1.66666667e-1f), 1.0f);
    return x * p;
}
// sin(2 pi r) for |r| < 2^22: r - rint(r) is exact, the SFU sine then runs on [-pi, pi].
__device__ __forceinline__ float sin2pi(float r) {
    const float f = r - rintf(r);
    return __sinf(6.28318530717958648f * f);
}

template <int COST>
__device__ __forceinline__ double g64_rot(double y) {
    return COST == kRotRastrigin ? g64_rastrigin(y) : h64_schwefel(y);
}
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
    float edrift = 0.0f;  // bound on the FP64 value drift of the pair updates (per lane)
    if (level == 0) {
        const float* xr = P.x0 + (size_t)c * n;
        const float2* yr = P.y0 + (size_t)c * n;
        double part = 0.0;
        for (int k = lane; k < n; k += 32) {
            x[k] = xr[k];
            const float2 v = yr[k];
            yh[k] = v.x;
            yl[k] = v.y;
            part += g64_rot<COST>((double)v.x + (double)v.y);
        }
        Fs = f_from_sum<COST>(wsumd(part), n);
    } else {
        for (int k = lane; k < n; k += 32) {
            x[k] = P.x_best32[k];
            yh[k] = P.ybest_hi[k];
            yl[k] = P.ybest_lo[k];
        }
        Fs = P.scal[kFRot];
    }
    __syncwarp();

    const float sig = P.sig_u * sl, lo = P.lo_u, hi = P.hi_u;
    const float neg_T_ln2 = (float)(-T * 0.69314718055994531);
    const float tau_abs = (float)(T * 4.0e-7);
    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    uint32_t* mybits = tracing ? A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)gc) * (size_t)A.words : nullptr;
    const float qmax_pi = P.qmax * 3.14159265f;
    const float inv_n = 1.0f / (float)n;
    const float nsum = ((float)((n + 31) / 32) + 6.0f) * 1.2e-7f;  // summation rounding per unit of sum |t_i|
    double dS = 0.0, e = 0.0;
    unsigned nacc = 0, nre = 0, bw = 0;
    for (int s = 0; s < A.L; ++s) {
        // randomness of step s (the same block in every lane)
        const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)level, (uint32_t)c, P.pid), A.key0, A.key1);
        const int d = coord_of(w.x, n);
        const float r = sqrt_approx(-1.3862943611198906f * __log2f(u23f(w.y)));
        const float z = -r * __cosf(6.28318530717958648f * (u23f(w.z) - 0.5f));  // cos(2 pi u2)
        const float tau = neg_T_ln2 * __log2f(u23f(w.w));
        const float xo = x[d];
        float xp = fmaf(sig, z, xo);
        if (A.boundary == 0) xp = xp < lo ? 2.0f * lo - xp : (xp > hi ? 2.0f * hi - xp : xp);
        xp = fminf(fmaxf(xp, lo), hi);
        // delta = xp - xo exactly, as dh + dl (TwoSum)
        const float dh = xp - xo;
        const float bb = dh - xp;
        const float dl = (xp - (dh - bb)) + (-xo - bb);
        // ---- FP32 energy difference and its error bound
        const float* qcol = P.qt_hi + (size_t)d * n;
        float sum = 0.0f, sabs = 0.0f, bnd = 0.0f;
        if (COST == kRotRastrigin) {
            const bool any_big = fabsf(dh) * qmax_pi >= 0.5f;  // some |pi Delta_i| may reach 1/2
            for (int i = lane; i < n; i += 32) {
                const float yv = yh[i];
                const float Dl = dh * qcol[i];
                const float m = (yv - rintf(yv)) + fmaf(0.5f, Dl, yl[i]);  // y + Delta/2 modulo 1
                const float s1 = sin2pi(m);
                float s2 = sinpi_small(Dl);
                float c = 2.0e-4f;
                if (any_big && fabsf(Dl) * 3.14159265f >= 0.5f) {
                    s2 = sin2pi(0.5f * Dl);
                    c = 5.0e-4f;
                }
                const float t = fmaf(Dl, fmaf(2.0f, yv, Dl), 20.0f * s1 * s2);
                sum += t;
                sabs += fabsf(t);
                const float aD = fabsf(Dl);
                bnd = fmaf(aD, fmaf(fabsf(yv), 9.0e-7f, fmaf(aD, 6.0e-5f, c)), bnd);
            }
        } else {
            for (int i = lane; i < n; i += 32) {
                const float yv = yh[i];
                const float Dl = dh * qcol[i];
                const float yp = fmaf(dh, qcol[i], yv);
                const float ro = sqrt_approx(fabsf(yv)), rp = sqrt_approx(fabsf(yp));
                const float t = yp * sin_reduced(rp) - yv * sin_reduced(ro);
                sum += t;
                sabs += fabsf(t);
                const float ay = fabsf(yv), ap = fabsf(yp);
                // evaluation of both terms, then their arguments' errors times |h'| <= 1 + sqrt|t|/2
                const float ev = ay * fmaf(ro, 4.8e-7f, 2.6e-6f) + ap * fmaf(rp, 4.8e-7f, 2.6e-6f);
                const float ar = fmaf(0.5f, rp, 1.0f) * (6.0e-8f * (ap + ay) + 1.8e-7f * fabsf(Dl)) +
                                 fmaf(0.5f, ro, 1.0f) * 6.0e-8f * ay;
                bnd += 1.5f * (ev + ar);
            }
        }
        sum = wsumf(sum);
        sabs = wsumf(sabs);
        bnd = wsumf(bnd);
        float dF, B;
        if (COST == kRotRastrigin) {
            dF = sum;
            B = bnd + nsum * sabs;
        } else {
            dF = -sum * inv_n;
            B = (bnd + nsum * sabs) * inv_n + 2.4e-7f * fabsf(dF);
        }
        B = 1.01f * B + 1.0e-6f * fabsf(tau) + tau_abs;  // with the error of tau
        bool acc;
        double dF_used = (double)dF;
        double e_step = (double)B;
        if (dF < tau - B) {
            acc = true;
        } else if (dF > tau + B) {
            acc = false;
        } else {
            // ---- FP64 re-check of a decision inside the bound
            const double d64 = (double)xp - (double)xo;
            const double* q64 = P.qt64 + (size_t)d * n;
            double s64 = 0.0, a64 = 0.0;
            for (int i = lane; i < n; i += 32) {
                const double y64 = (double)yh[i] + (double)yl[i];
                const double gn = g64_rot<COST>(y64 + d64 * q64[i]), go = g64_rot<COST>(y64);
                s64 += gn - go;
                a64 += fabs(gn) + fabs(go);
            }
            s64 = wsumd(s64);
            a64 = wsumd(a64);
            const double dF64 = COST == kRotRastrigin ? s64 : -(s64 / (double)n);
            acc = (dF64 <= 0.0) || (u23d(w.w) < exp(-dF64 / T));
            dF_used = dF64;
            // FP64 evaluation and summation error (4 ulp per term, the rest per addition)
            e_step = 2.3e-16 * ((double)((n + 31) / 32) + 10.0) * a64 / (COST == kRotRastrigin ? 1.0 : (double)n);
            ++nre;
        }
        if (acc) {
            if (lane == 0) x[d] = xp;
            const float* qlcol = P.qt_lo + (size_t)d * n;
            for (int i = lane; i < n; i += 32) {
                // (yh, yl) += (dh + dl)(qh + ql), compensated (TwoProd by FMA, TwoSum)
                const float qh = qcol[i], ql = qlcol[i];
                const float ph = dh * qh;
                const float pl = fmaf(dh, qh, -ph);
                const float corr = fmaf(dh, ql, dl * qh);
                const float a = yh[i];
                const float sh = a + ph;
                const float t2 = sh - a;
                const float err = (a - (sh - t2)) + (ph - t2);
                const float lo2 = yl[i] + (pl + corr + err);
                const float nh = sh + lo2;
                yh[i] = nh;
                yl[i] = lo2 - (nh - sh);
                // the pair moves by at most 2^-45 (|y'| + |Delta|) from the exact
                // update; F by |g'| times that
                const float an = fabsf(nh);
                const float gp = COST == kRotRastrigin ? fmaf(2.0f, an, 64.0f) : fmaf(0.5f, sqrt_approx(an), 1.0f) * inv_n;
                edrift = fmaf(gp, (an + fabsf(ph)) * 2.9e-14f, edrift);
            }
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
    r.ec = e + (double)wsumf(edrift) + 1e-13 * (fabs(Fs) + fabs(dS) + 1.0);
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
    if (finite && (tracing || level == A.full_level || r.Fa - r.ec <= M)) {
        double part = 0.0;
        for (int i = lane; i < n; i += 32) part += g64_rot<COST>((double)yh[i] + (double)yl[i]);
        part = wsumd(part);
        if (lane == 0) A.F[gc] = f_from_sum<COST>(part, n);
        float* dst = A.X32 + P.x_base + c;
        for (int k = lane; k < n; k += 32) dst[(size_t)k * (size_t)P.chains] = x[k];
    } else if (lane == 0) {
        A.F[gc] = finite ? CUDART_INF : CUDART_NAN;
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

__global__ void __launch_bounds__(kBlockR) sweep_rot_kernel(SweepArgs A) {
    extern __shared__ __align__(16) float smem_rot[];
    const WorkItem it = A.items[blockIdx.x];
    const ProbDev& P = A.probs[it.problem];
    if (P.cost == kRotRastrigin) rot_tile<kRotRastrigin>(A, P, it, smem_rot);
    else rot_tile<kRotSchwefel>(A, P, it, smem_rot);
}

}  // namespace

size_t sweep_rot_smem_bytes(int n) { return (size_t)kWarpsR * 3 * (size_t)n * sizeof(float); }
int sweep_rot_chains_per_block() { return kWarpsR; }

cudaError_t sweep_rot_set_smem(size_t bytes) {
    static size_t current = 0;
    if (bytes <= current) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(sweep_rot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

cudaError_t launch_sweep_rot(const SweepArgs& a, int num_items, size_t smem, cudaStream_t s) {
    sweep_rot_kernel<<<num_items, kBlockR, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sa
