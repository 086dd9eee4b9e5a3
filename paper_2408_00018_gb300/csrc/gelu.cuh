// gelu.cuh -- the surrogate network's activation, shared by the tensor-core
// GEMM epilogues (forward pass) and the training kernels (backward pass), so
// the gradient is taken of the function the forward pass evaluates.
#pragma once
#include <cuda_runtime.h>

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
// GELU, erf form: z Phi(z) = z/2 (1 + erf(z / sqrt 2)).
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erf_hastings(z * 0.70710678118654752f)); }
// Its derivative Phi(z) + z phi(z), with Phi from the same erf and the exact
// normal density phi: the derivative of the approximated Phi differs from phi
// by the derivative of the approximation's error (a few units of 1e-7 in
// this range), far below the BF16 rounding of the backward pass's operands.
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erf_hastings(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

}  // namespace sa
