// sa_device.cuh -- device building blocks of the annealing sweep (sm_103a).
//
// Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), one 128-bit
// block per (step, level, chain, problem); key = (seed_lo, seed_hi ^ stream tag).
// The paper draws three uniforms per step from CURAND (Sec. 2.1 Step 3 and the
// remark on CURAND in Sec. 3.3); a counter-based generator makes every step
// reproducible and lets a run resume bit-for-bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sa {

enum CostId : int32_t {
    kSchwefel = 0, kRastrigin = 1, kAckley = 2, kRosenbrock = 3, kRotRastrigin = 4, kRotSchwefel = 5,
    // the rest of the Appendix's tests (FP64, full evaluation)
    kBranin = 6, kCosineMixture = 7, kDekkersAarts = 8, kEasom = 9, kExponential = 10, kGoldsteinPrice = 11,
    kGriewank = 12, kHimmelblau = 13, kLevyMontalvo = 14, kLangerman = 15, kMichalewicz = 16, kSalomon = 17,
    kSixHumpCamel = 18, kShubert = 19, kShekel = 20, kFoxholes = 21
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        // one 32x32 -> 64-bit product per multiplier gives both halves
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// The same generator for a fixed (c1, c2, c3) and a varying step counter c0:
// the parts of rounds 1 and 2 that do not depend on c0 are computed once per
// chain and level (philox_prep), the rest per step (philox_step).  The output
// equals philox4x32_10(make_uint4(c0, c1, c2, c3), k0, k1) bit for bit.
// rk: the key of every round, rk[2r] and rk[2r+1] for round r (the schedule
// k + r (W0, W1) tabulated once on the host and passed as kernel parameters).
struct PhiloxFixed {
    uint32_t w0, w1;        // words 0, 1 after round 1 (independent of c0)
    uint32_t hi2, lo2;      // round 2's product of word 0
    uint32_t c3;
};
__device__ __forceinline__ PhiloxFixed philox_prep(uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t* rk) {
    PhiloxFixed f;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
    f.w0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk[0];
    f.w1 = (uint32_t)p1;
    const unsigned long long q0 = (unsigned long long)0xD2511F53u * f.w0;
    f.hi2 = (uint32_t)(q0 >> 32);
    f.lo2 = (uint32_t)q0;
    f.c3 = c3;
    return f;
}
__device__ __forceinline__ uint4 philox_step(uint32_t c0, const PhiloxFixed& f, const uint32_t* rk) {
    // round 1 (words 2, 3 depend on c0)
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
    const uint32_t w2 = (uint32_t)(p0 >> 32) ^ f.c3 ^ rk[1];
    const uint32_t w3 = (uint32_t)p0;
    // round 2
    const unsigned long long q1 = (unsigned long long)0xCD9E8D57u * w2;
    uint4 c = make_uint4((uint32_t)(q1 >> 32) ^ f.w1 ^ rk[2], (uint32_t)q1, f.hi2 ^ w3 ^ rk[3], f.lo2);
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const unsigned long long a = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long b = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(b >> 32) ^ c.y ^ rk[2 * r], (uint32_t)b, (uint32_t)(a >> 32) ^ c.w ^ rk[2 * r + 1],
                       (uint32_t)a);
    }
    return c;
}

// Uniform in (0,1) from the top 23 bits of a word; exact in FP32 and FP64.
// FP32 form without an integer-to-float conversion: the top 23 bits become the
// mantissa of a number in [1, 2); subtracting 1 - 2^-24 is exact and gives (k + 1/2) 2^-23.
// The bits 0x3F800000 | (w >> 9) come from one funnel shift of the pair
// (0x7F, w) right by 9: the exponent field 0x7F lands above the 23 bits.
__device__ __forceinline__ float u23f(uint32_t w) {
    return __uint_as_float(__funnelshift_r(w, 0x7Fu, 9)) - 0.999999940395355225f;
}
__device__ __forceinline__ double u23d(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }
// Coordinate d = (w n) >> 32, uniform over [0, n).
__device__ __forceinline__ int coord_of(uint32_t w, int n) { return (int)__umulhi(w, (uint32_t)n); }

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// The SFU's sine, cosine and base-2 logarithm with subnormal inputs and
// results flushed to zero (one SFU instruction each, without the fix-ups the
// subnormal-preserving forms add).  Every argument here is a normal number
// or zero except by a coincidence of size below 2^-126, where flushing moves
// the result by less than 2^-126: far inside every error bound of the sweep.
__device__ __forceinline__ float sin_approx(float x) {
    float r;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float cos_approx(float x) {
    float r;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Box handling of a proposal (Sec. 2.1, Step 2): reflect once at the face it
// crossed, then clip to [lo, hi]; or clip only.  The reflection is branch-free:
// with a = 2 lo - xp and b = 2 hi - xp, min(max(xp, a), max(b, lo)) is a for
// xp < lo, xp inside the box and max(b, lo) for xp > hi (the reflected point
// already clipped from below), and it is never below lo, so the clip reduces
// to min(., hi).  2 lo and 2 hi are exact, so a and b are the reflected points
// rounded once, as in the case-by-case form.
__device__ __forceinline__ float reflect_clip(float xp, float lo, float hi, bool reflect) {
    if (reflect) {
        const float a = 2.0f * lo - xp, b = 2.0f * hi - xp;
        return fminf(fminf(fmaxf(xp, a), fmaxf(b, lo)), hi);
    }
    return fminf(fmaxf(xp, lo), hi);
}

// sin(r) for 0 <= r <= ~64: two-constant Cody-Waite reduction by 2 pi, then the
// SFU sine on [-pi, pi].
__device__ __forceinline__ float sin_reduced(float r) {
    const float k = rintf(r * 0.15915494309189535f);
    float t = fmaf(-k, 6.28318548202514648f, r);
    t = fmaf(-k, -1.7484555314695172e-7f, t);
    return sin_approx(t);
}
// cos(2 pi t) for any |t| < 2^22: t - rint(t) is exact, the SFU cosine then runs on [-pi, pi].
__device__ __forceinline__ float cos2pi(float t) {
    const float f = t - rintf(t);
    return cos_approx(6.28318530717958648f * f);
}

// ---------------------------------------------------------------------------
// FP32 energy differences of one single-coordinate move x_d: xo -> xp.
// Each returns dF and a bound eb on |dF_computed - dF_exact| (exact = real
// arithmetic at the same FP32 inputs).  Constants: unit roundoff u = 2^-24,
// SFU sine/cosine absolute error <= 2^-21.41 on [-pi, pi] (taken as 2^-20),
// approximate square root relative error taken as 2^-22 (measured on this
// GPU: <= 2^-23.25 over [1e-3, 500]); every bound carries a further factor 2
// of margin.
// ---------------------------------------------------------------------------
struct SepState {   // per-chain running sums that some costs keep (Ackley)
    float s1, s2, a;  // sum x^2, sum cos(2 pi x), current Ackley value from (s1, s2)
};

// Normalised Schwefel: h(t) = t sin(sqrt|t|); dF = (h(xo) - h(xp)) / n.
__device__ __forceinline__ float h_schwefel(float t) { return t * sin_reduced(sqrt_approx(fabsf(t))); }

// Rastrigin: g(t) = t^2 - 10 cos(2 pi t).
__device__ __forceinline__ float g_rastrigin(float t) { return fmaf(t, t, -10.0f * cos2pi(t)); }

__device__ __forceinline__ float ackley_value(float s1, float s2, float inv_n) {
    return -20.0f * __expf(-0.2f * sqrt_approx(s1 * inv_n)) - __expf(s2 * inv_n) + 22.718281828459045f;
}

// Rosenbrock term T(a, b) = 100 (b - a^2)^2 + (1 - a)^2 and its FP32 error bound.
__device__ __forceinline__ float rosen_term(float a, float b, float& eb) {
    const float v = b - a * a, w = 1.0f - a;
    const float t = fmaf(100.0f * v, v, w * w);
    eb += 1.2e-7f * (200.0f * fabsf(v) * (a * a + 2.0f * fabsf(v)) + 300.0f * v * v + 4.0f * w * w + 2.0f * fabsf(w) * fabsf(a) + 2.0f);
    return t;
}

// ---------------------------------------------------------------------------
// FP64 cost functions (the definitions, summed in index order).  Used by the
// FP64 sweep and by the FP64 re-evaluation of argmin candidates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double h64_schwefel(double t) { return t * sin(sqrt(fabs(t))); }
__device__ __forceinline__ double g64_rastrigin(double t) { return t * t - 10.0 * cos(6.283185307179586 * t); }
__device__ __forceinline__ double ackley64(int n, double s1, double s2) {
    return -20.0 * exp(-0.2 * sqrt(s1 / (double)n)) - exp(s2 / (double)n) + 20.0 + 2.718281828459045;
}
__device__ __forceinline__ double rosen64(double a, double b) {
    const double t = b - a * a, u = 1.0 - a;
    return 100.0 * t * t + u * u;
}

// Ordered encoding of doubles as unsigned 64-bit keys (for atomicMin).
__device__ __forceinline__ unsigned long long dbl_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_dbl(unsigned long long k) {
    const unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

}  // namespace sa
