// rot_step.cuh -- one Metropolis step's energy difference for the rotated
// costs f(x) = F(Q x), evaluated by a warp on a chain whose rotated state
// y = Q x is held as an FP32 pair (y_hi + y_lo).  Lanes own the rotated
// coordinates i = lane + 32 j; the move x_d -> x_d + (dh + dl) changes every
// y_i by Delta_i = delta Q_id.  Used by the plain rotated sweep (state in
// shared memory) and by the delayed-acceptance sweep (state in global memory).
//
// rot_eval32 returns the FP32 difference and a bound B on its error against
// real arithmetic on the pair state and the exact move:
//   rotated Rastrigin, per coordinate:
//     g(y + Delta) - g(y) = Delta (2y + Delta) + 20 sin(2 pi (y + Delta/2)) sin(pi Delta)
//   rotated Schwefel, per coordinate (a = sqrt|y + Delta|, b = sqrt|y|):
//     h(y + Delta) - h(y) = Delta sin a + 2 y cos((a + b)/2) sin((a - b)/2),
//     a - b = (|y + Delta| - |y|) / (a + b), with |y + Delta| - |y| = +-Delta
//     when the sign does not change;
// both are product-to-sum forms whose error scales with |Delta| instead of
// with the size of the terms.  For an even n the hot loops take coordinate
// pairs in packed f32x2 arithmetic (the same operations per coordinate).
// rot_eval64 is the FP64 difference from
// y_hi + y_lo and the FP64 Q (the re-check); rot_update applies an accepted
// move to the pair with compensated arithmetic (TwoProd by FMA, TwoSum).
#pragma once
#include <cmath>
#include <cstdint>

#include "f32x2.cuh"
#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {

__device__ __forceinline__ float rot_wsumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double rot_wsumd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sin(x) for |x| < 1/2: Taylor polynomial to degree 7 (truncation below 1.1e-8 relative).
__device__ __forceinline__ float sin_taylor(float x) {
    const float x2 = x * x;
    const float p = fmaf(x2, fmaf(x2, fmaf(x2, -1.98412698e-4f, 8.33333333e-3f), -1.66666667e-1f), 1.0f);
    return x * p;
}
// sin(2 pi r) for |r| < 2^22: r - rint(r) is exact, the SFU sine then runs on [-pi, pi].
__device__ __forceinline__ float sin2pi_red(float r) {
    const float f = r - rintf(r);
    return sin_approx(6.28318530717958648f * f);
}
// cos(r) for |r| < ~64, reduced like sin_reduced.
__device__ __forceinline__ float cos_reduced(float r) {
    const float k = rintf(r * 0.15915494309189535f);
    float t = fmaf(-k, 6.28318548202514648f, r);
    t = fmaf(-k, -1.7484555314695172e-7f, t);
    return cos_approx(t);
}

// The proposal of step s (Sec. 2.1, Step 2): coordinate d, Gaussian step of the
// coordinate by the cosine branch of Box-Muller, reflect once then clip (or clip);
// tau = -T ln u3 is the Metropolis threshold.  The same FP32 arithmetic in every
// sweep, so that kernels which recompute a proposal get the same bits.
struct RotMove {
    int d;
    float xo, xp, dh, dl, tau;
    uint32_t w3;  // the word of u3
};
// P: the box (uniform scalars, or per coordinate when P.uniform == 0); sl = sqrt(T / T0).
// uprop: 1 = uniform redraw of the coordinate (x' = lo + u2 (hi - lo)), 0 = Gaussian step.
__device__ __forceinline__ RotMove rot_propose(uint4 w, const float* x, const ProbDev& P, float sl, int boundary,
                                               int uprop, float neg_T_ln2) {
    RotMove m;
    const int n = P.n;
    m.d = coord_of(w.x, n);
    float sig, lo, hi;
    if (P.uniform) { sig = P.sig_u * sl; lo = P.lo_u; hi = P.hi_u; }
    else { sig = P.sig32[m.d] * sl; lo = P.lo32[m.d]; hi = P.hi32[m.d]; }
    m.tau = neg_T_ln2 * lg2_approx(u23f(w.w));
    m.w3 = w.w;
    m.xo = x[m.d];
    float xp;
    if (uprop) {
        xp = fmaf(hi - lo, u23f(w.z), lo);
    } else {
        const float r = sqrt_approx(-1.3862943611198906f * lg2_approx(u23f(w.y)));
        const float z = -r * cos_approx(6.28318530717958648f * (u23f(w.z) - 0.5f));  // cos(2 pi u2)
        xp = fmaf(sig, z, m.xo);
    }
    m.xp = reflect_clip(xp, lo, hi, boundary == 0);
    // delta = xp - xo exactly, as dh + dl (TwoSum)
    m.dh = m.xp - m.xo;
    const float bb = m.dh - m.xp;
    m.dl = (m.xp - (m.dh - bb)) + (-m.xo - bb);
    return m;
}

// 0.0f that the compiler cannot see through (repeats an evaluation on purpose).
__device__ __forceinline__ float opaque_zero() {
    float z;
    asm volatile("mov.b32 %0, 0;" : "=f"(z));
    return z;
}

template <int COST>
__device__ __forceinline__ double rot_g64(double y) {
    return COST == kRotRastrigin ? g64_rastrigin(y) : h64_schwefel(y);
}

// FP32 difference dF and its error bound B (without the error of the test's threshold).
template <int COST>
__device__ __forceinline__ void rot_eval32(const ProbDev& P, const float* yh, const float* yl, int d, float dh, int n,
                                           int lane, float& dF, float& B) {
    const float* qcol = P.qt_hi + (size_t)d * n;
    const float nsum = ((float)((n + 31) / 32) + 6.0f) * 1.2e-7f;  // summation rounding per unit of sum |t_i|
    float sum = 0.0f, bnd = 0.0f;
    if (COST == kRotRastrigin) {
        const bool any_big = fabsf(dh) * P.qmax * 3.14159265f >= 0.5f;  // some |pi Delta_i| may reach 1/2
        if (!any_big && (n & 1) == 0) {
            // lanes own coordinate pairs (i, i + 1), i = 2 lane + 64 j, in packed
            // arithmetic: the same operations per coordinate as below; each lane sums
            // its even and its odd coordinates apart, then adds the two (no more
            // rounding steps than the loop below: ceil(n / 64) + 1 <= ceil(n / 32))
            const f32x2_t dh2 = f2_splat(dh), half = f2_splat(0.5f), two = f2_splat(2.0f), k20 = f2_splat(20.0f);
            const f32x2_t pi = f2_splat(3.14159265358979f), tpi = f2_splat(6.28318530717958648f);
            const f32x2_t c7 = f2_splat(-1.98412698e-4f), c5 = f2_splat(8.33333333e-3f), c3 = f2_splat(-1.66666667e-1f);
            const f32x2_t one = f2_splat(1.0f), k9 = f2_splat(9.0e-7f), k6 = f2_splat(6.0e-5f), kc = f2_splat(2.0e-4f);
            const f32x2_t ns = f2_splat(nsum);
            f32x2_t sum2 = f2_splat(0.0f), bnd2 = f2_splat(0.0f);
            // four iterations' loads of the Q column (from L2) in flight per lane: one at a
            // time left the warp waiting on L2 latency (95.7 -> 78.3 ms per level at n = 1024)
            #pragma unroll 4
            for (int i = 2 * lane; i < n; i += 64) {
                const f32x2_t Y = f2_ld(yh + i), YL = f2_ld(yl + i), D = f2_mul(dh2, f2_ld(qcol + i));
                const float2 y = f2_unpack(Y);
                const f32x2_t M = f2_add(f2_sub(Y, f2_pack(rintf(y.x), rintf(y.y))), f2_fma(half, D, YL));
                const float2 m = f2_unpack(M);
                const float2 ang = f2_unpack(f2_mul(tpi, f2_sub(M, f2_pack(rintf(m.x), rintf(m.y)))));
                const f32x2_t S1 = f2_pack(sin_approx(ang.x), sin_approx(ang.y));
                const f32x2_t X = f2_mul(pi, D), X2 = f2_mul(X, X);
                const f32x2_t S2 = f2_mul(X, f2_fma(X2, f2_fma(X2, f2_fma(X2, c7, c5), c3), one));
                const f32x2_t T = f2_fma(D, f2_fma(two, Y, D), f2_mul(f2_mul(k20, S1), S2));
                sum2 = f2_add(sum2, T);
                const f32x2_t aD = f2_abs(D);
                bnd2 = f2_fma(aD, f2_fma(f2_abs(Y), k9, f2_fma(aD, k6, kc)), f2_fma(ns, f2_abs(T), bnd2));
            }
            const float2 sp = f2_unpack(sum2), bp = f2_unpack(bnd2);
            sum = sp.x + sp.y;
            bnd = bp.x + bp.y;
        } else {
        #pragma unroll 4
        for (int i = lane; i < n; i += 32) {
            const float yv = yh[i];
            const float Dl = dh * qcol[i];
            const float m = (yv - rintf(yv)) + fmaf(0.5f, Dl, yl[i]);  // y + Delta/2 modulo 1
            const float s1 = sin2pi_red(m);
            float s2 = sin_taylor(3.14159265358979f * Dl);
            float c = 2.0e-4f;
            if (any_big && fabsf(Dl) * 3.14159265f >= 0.5f) {
                s2 = sin2pi_red(0.5f * Dl);
                c = 5.0e-4f;
            }
            const float t = fmaf(Dl, fmaf(2.0f, yv, Dl), 20.0f * s1 * s2);
            sum += t;
            const float aD = fabsf(Dl);
            // the term's error plus its share of the summation's rounding
            bnd = fmaf(aD, fmaf(fabsf(yv), 9.0e-7f, fmaf(aD, 6.0e-5f, c)), fmaf(nsum, fabsf(t), bnd));
        }
        }
        sum = rot_wsumf(sum);
        bnd = rot_wsumf(bnd);
        dF = sum;
        B = 1.01f * bnd;
    } else {
        // caps of the square roots' argument errors, valid for every coordinate of
        // this move (|y| <= ymax over the box, |Delta_i| <= |dh| qmax):
        // |sqrt u - sqrt v| <= sqrt|u - v|
        const float capA = 1.01f * sqrt_approx(fmaf(1.2e-7f, P.ymax, 2.4e-7f * fabsf(dh) * P.qmax)) + 1e-15f;
        const float capB = 1.01f * sqrt_approx(6.0e-8f * P.ymax) + 1e-15f;
        #pragma unroll 4
        for (int i = lane; i < n; i += 32) {
            const float yv = yh[i];
            const float Dl = dh * qcol[i];
            const float yp = yv + Dl;
            const float ay = fabsf(yv), ap = fabsf(yp);
            const float rb = rsqrtf(fmaxf(ay, 1e-30f)), ra = rsqrtf(fmaxf(ap, 1e-30f));
            const float b = ay * rb, a = ap * ra;  // sqrt|y|, sqrt|y'|
            const float num = (yv * yp > 0.0f) ? (yv > 0.0f ? Dl : -Dl) : (ap - ay);  // |y'| - |y|
            const float apb = a + b;
            const float inv = __fdividef(1.0f, fmaxf(apb, 1e-30f));  // 2 ulp, inside the bound's margin
            const float hh = 0.5f * num * inv;  // (a - b) / 2
            const bool small = fabsf(hh) < 0.5f;
            const float S2 = small ? sin_taylor(hh) : sin_reduced(hh);
            const float C = cos_reduced(0.5f * apb);
            const float Sa = sin_reduced(a);
            const float y2S2 = 2.0f * yv * S2;
            const float t = fmaf(Dl, Sa, y2S2 * C);
            sum += t;
            // errors of a and b from their arguments' errors (the pair's low part,
            // the rounding of y', the rounding of the move) and of the square roots
            const float ep = 6.0e-8f * (ap + ay) + 1.8e-7f * fabsf(Dl);
            const float eo = 6.0e-8f * ay;
            // (|sqrt u - sqrt v| <= |u - v| / sqrt v, and the caps above; arguments
            // below 1e-30 are taken as 0, which costs at most 1e-15)
            const float ea = fminf(ep * ra, capA) + 4.8e-7f * a + 1e-15f;
            const float eb = fminf(eo * rb, capB) + 4.8e-7f * b + 1e-15f;
            const float eD = fabsf(hh) * (9.6e-7f + (ea + eb) * inv) + 6.0e-7f * fabsf(Dl) * inv;  // of (a - b)/2
            const float eS2 = eD + (small ? 2.4e-7f * fabsf(hh) : 2.0e-6f);
            const float e1 = fabsf(Dl) * (2.4e-6f + ea);
            const float e2 = 2.0f * ay * (fabsf(S2) * (2.0e-6f + 0.5f * (ea + eb)) + eS2);
            bnd += fmaf(nsum, fabsf(t), 1.5f * (e1 + e2) + 3.6e-7f * (fabsf(Dl * Sa) + fabsf(y2S2)));
        }
        sum = rot_wsumf(sum);
        bnd = rot_wsumf(bnd);
        const float inv_n = 1.0f / (float)n;
        dF = -sum * inv_n;
        B = 1.01f * (bnd * inv_n + 2.4e-7f * fabsf(dF));
    }
}

// FP64 difference from the pair state and the FP64 Q; e_out bounds its rounding.
template <int COST>
__device__ __forceinline__ double rot_eval64(const ProbDev& P, const float* yh, const float* yl, int d, float xp, float xo,
                                             int n, int lane, double& e_out) {
    const double d64 = (double)xp - (double)xo;
    const double* q64 = P.qt64 + (size_t)d * n;
    double s64 = 0.0, a64 = 0.0;
        #pragma unroll 4
        for (int i = lane; i < n; i += 32) {
        const double y64 = (double)yh[i] + (double)yl[i];
        const double gn = rot_g64<COST>(y64 + d64 * q64[i]), go = rot_g64<COST>(y64);
        s64 += gn - go;
        a64 += fabs(gn) + fabs(go);
    }
    s64 = rot_wsumd(s64);
    a64 = rot_wsumd(a64);
    // FP64 evaluation (4 ulp per term) and summation error
    e_out = 2.3e-16 * ((double)((n + 31) / 32) + 10.0) * a64 / (COST == kRotRastrigin ? 1.0 : (double)n);
    return COST == kRotRastrigin ? s64 : -(s64 / (double)n);
}

// (yh, yl) += (dh + dl)(Q_hi + Q_lo)[:, d]; edrift (every lane) grows by a bound
// on the change of F caused by the update's rounding: 2^-45 (|y'| + |Delta|) per
// coordinate times |g'|, taken at |y| <= ymax, |Delta| <= |dh| qmax over the n
// coordinates.
template <int COST>
__device__ __forceinline__ void rot_update(const ProbDev& P, float* yh, float* yl, int d, float dh, float dl, int n,
                                           int lane, float& edrift) {
    const float* qcol = P.qt_hi + (size_t)d * n;
    const float* qlcol = P.qt_lo + (size_t)d * n;
    const float ym = P.ymax, dm = fabsf(dh) * P.qmax;
    const float gmax = COST == kRotRastrigin ? fmaf(2.0f, ym + dm, 64.0f)
                                             : fmaf(0.5f, sqrt_approx(ym + dm), 1.0f) / (float)n;
    edrift = fmaf((float)n * gmax, (ym + 2.0f * dm) * 2.9e-14f, edrift);
    if ((n & 1) == 0) {
        // coordinate pairs in packed arithmetic: lane for lane the operations below
        const f32x2_t dh2 = f2_splat(dh), dl2 = f2_splat(dl);
        #pragma unroll 2
        for (int i = 2 * lane; i < n; i += 64) {
            const f32x2_t qh = f2_ld(qcol + i), ql = f2_ld(qlcol + i);
            const f32x2_t ph = f2_mul(dh2, qh);  // packed products are never merged into an FMA
            const f32x2_t pl = f2_fma(dh2, qh, f2_neg(ph));
            const f32x2_t corr = f2_fma(dh2, ql, f2_mul(dl2, qh));
            const f32x2_t a = f2_ld(yh + i);
            const f32x2_t sh = f2_add(a, ph);
            const f32x2_t t2 = f2_sub(sh, a);
            const f32x2_t err = f2_add(f2_sub(a, f2_sub(sh, t2)), f2_sub(ph, t2));
            const f32x2_t lo2 = f2_add(f2_ld(yl + i), f2_add(f2_add(pl, corr), err));
            const f32x2_t nh = f2_add(sh, lo2);
            f2_st(yh + i, nh);
            f2_st(yl + i, f2_sub(lo2, f2_sub(nh, sh)));
        }
        return;
    }
        #pragma unroll 4
        for (int i = lane; i < n; i += 32) {
        const float qh = qcol[i], ql = qlcol[i];
        // the rounded product by an intrinsic that is never merged into an FMA: the
        // TwoSum below (a + ph and ph - t2) is error-free only for this very ph
        const float ph = __fmul_rn(dh, qh);
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
    }
}

}  // namespace sa
