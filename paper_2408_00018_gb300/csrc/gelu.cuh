// gelu.cuh -- the surrogate network's activation, shared by the tensor-core
// GEMM epilogues (forward pass) and the training kernels (backward pass), so
// the gradient is taken of the function the forward pass evaluates.
#pragma once
#include <cuda_runtime.h>

#include "f32x2.cuh"

namespace sa {

// erf by Hastings' rational approximation (Abramowitz and Stegun, formula 7.1.26):
// erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2), t = 1 / (1 + p x), x >= 0,
// odd in x; its error is at most 1.5e-7, and this FP32 evaluation (approximate reciprocal
// and exponential) adds a few units of 1e-7.  The epilogues round GELU to BF16 (8
// significant bits) or sum it against the head's weights in FP32, far above that error.
__device__ __forceinline__ float erf_hastings(float x) {
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    return copysignf(fmaf(-poly, __expf(-ax * ax), 1.0f), x);
}
// GELU, erf form: z Phi(z) = z/2 (1 + erf(z / sqrt 2)), with Hastings' erf.  For
// a = |z| / sqrt 2 and t = 1 / (1 + p a), 1 - erf(a) = poly(t) e^(-a^2) for both signs
// of z, so z Phi(z) = max(z, 0) - |z| poly(t)/2 e^(-z^2/2): one reciprocal, one base-2
// exponential (e^x = 2^(x log2 e)), and no sign or branch.  The constants are Hastings'
// scaled by exact powers of two (-1/2) or rounded once (p / sqrt 2, -log2(e) / 2).
constexpr float kGeluP = 0.3275911f * 0.70710678118654752f;
constexpr float kGeluB1 = -0.5f * 0.254829592f, kGeluB2 = -0.5f * -0.284496736f, kGeluB3 = -0.5f * 1.421413741f,
                kGeluB4 = -0.5f * -1.453152027f, kGeluB5 = -0.5f * 1.061405429f;
constexpr float kGeluC = -0.72134752044448170f;  // -log2(e) / 2

__device__ __forceinline__ float gelu_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float gelu_ex2(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Every operation explicitly rounded (never contracted), so that gelu2 below, which
// takes the same operations two lanes at a time, gives the same bits.
__device__ __forceinline__ float gelu_f(float z) {
    const float az = fabsf(z);
    const float t = gelu_rcp(fmaf(kGeluP, az, 1.0f));
    const float q = __fmul_rn(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, kGeluB5, kGeluB4), kGeluB3), kGeluB2), kGeluB1));
    const float e = gelu_ex2(__fmul_rn(__fmul_rn(z, kGeluC), z));
    return fmaf(az, __fmul_rn(q, e), fmaxf(z, 0.0f));
}


// gelu_f of both lanes of z, bit for bit.
__device__ __forceinline__ f32x2_t gelu2(f32x2_t z) {
    const float2 zz = f2_unpack(z);
    const f32x2_t az = f2_pack(fabsf(zz.x), fabsf(zz.y));
    const float2 d = f2_unpack(f2_fma(f2_splat(kGeluP), az, f2_splat(1.0f)));
    const f32x2_t t = f2_pack(gelu_rcp(d.x), gelu_rcp(d.y));
    f32x2_t q = f2_fma(t, f2_splat(kGeluB5), f2_splat(kGeluB4));
    q = f2_fma(t, q, f2_splat(kGeluB3));
    q = f2_fma(t, q, f2_splat(kGeluB2));
    q = f2_fma(t, q, f2_splat(kGeluB1));
    q = f2_mul(t, q);
    const float2 x = f2_unpack(f2_mul(f2_mul(z, f2_splat(kGeluC)), z));
    const f32x2_t e = f2_pack(gelu_ex2(x.x), gelu_ex2(x.y));
    return f2_fma(az, f2_mul(q, e), f2_pack(fmaxf(zz.x, 0.0f), fmaxf(zz.y, 0.0f)));
}
// Its derivative Phi(z) + z phi(z), with Phi from the same erf and the exact
// normal density phi: the derivative of the approximated Phi differs from phi
// by the derivative of the approximation's error (a few units of 1e-7 in
// this range), far below the BF16 rounding of the backward pass's operands.
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erf_hastings(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

}  // namespace sa
