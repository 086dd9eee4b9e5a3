// f32x2.cuh -- pairs of FP32 values in one 64-bit register and the packed
// arithmetic of sm_100-class GPUs (add, sub, mul, fma .rn.f32x2: one instruction,
// both lanes rounded as the scalar operation would round them).
#pragma once
#include <cuda_runtime.h>

namespace sa {

typedef unsigned long long f32x2_t;
__device__ __forceinline__ f32x2_t f2_pack(float a, float b) {
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(f32x2_t r) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    return make_float2(a, b);
}
__device__ __forceinline__ f32x2_t f2_fma(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2_t f2_mul(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_add(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_splat(float a) { return f2_pack(a, a); }
__device__ __forceinline__ f32x2_t f2_sub(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// |a| and -a of both lanes (sign bits, exact)
__device__ __forceinline__ f32x2_t f2_abs(f32x2_t a) { return a & 0x7fffffff7fffffffull; }
__device__ __forceinline__ f32x2_t f2_neg(f32x2_t a) { return a ^ 0x8000000080000000ull; }
// 8-byte loads and stores of two consecutive floats (p 8-byte aligned)
__device__ __forceinline__ f32x2_t f2_ld(const float* p) { return *reinterpret_cast<const f32x2_t*>(p); }
__device__ __forceinline__ void f2_st(float* p, f32x2_t v) { *reinterpret_cast<f32x2_t*>(p) = v; }

}  // namespace sa
