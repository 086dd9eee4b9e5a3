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

enum CostId : int32_t { kSchwefel = 0, kRastrigin = 1, kAckley = 2, kRosenbrock = 3, kRotRastrigin = 4, kRotSchwefel = 5 };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Uniform in (0,1) from the top 23 bits of a word; exact in FP32 and FP64.
__device__ __forceinline__ float u23f(uint32_t w) { return __uint2float_rn(w >> 9) * 1.1920928955078125e-7f + 5.9604644775390625e-8f; }
__device__ __forceinline__ double u23d(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }
// Coordinate d = (w n) >> 32, uniform over [0, n).
__device__ __forceinline__ int coord_of(uint32_t w, int n) { return (int)__umulhi(w, (uint32_t)n); }

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// sin(r) for 0 <= r <= ~64: two-constant Cody-Waite reduction by 2 pi, then the
// SFU sine on [-pi, pi].
__device__ __forceinline__ float sin_reduced(float r) {
    const float k = rintf(r * 0.15915494309189535f);
    float t = fmaf(-k, 6.28318548202514648f, r);
    t = fmaf(-k, -1.7484555314695172e-7f, t);
    return __sinf(t);
}
// cos(2 pi t) for any |t| < 2^22: t - rint(t) is exact, the SFU cosine then runs on [-pi, pi].
__device__ __forceinline__ float cos2pi(float t) {
    const float f = t - rintf(t);
    return __cosf(6.28318530717958648f * f);
}

// ---------------------------------------------------------------------------
// FP32 energy differences of one single-coordinate move x_d: xo -> xp.
// Each returns dF and a bound eb on |dF_computed - dF_exact| (exact = real
// arithmetic at the same FP32 inputs).  Constants: unit roundoff u = 2^-24,
// SFU sine/cosine absolute error <= 2^-21.41 on [-pi, pi] (taken as 2^-20),
// approximate square root relative error taken as 2^-21; every bound carries
// a further factor 2 of margin.
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
