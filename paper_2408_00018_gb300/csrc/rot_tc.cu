// rot_tc.cu -- the rotated costs' level-0 transform Y0 = X0 Q^T on the tensor
// cores, exact to the double-float pairs the rotated sweep starts from.
//
// The method is the error-free splitting of a matrix product into products of
// low-precision slices (Ozaki, Ogita, Oishi and Rump, 2012), with integer slices.
// Every row of X0 (a chain's FP32 state) and of Q (FP64) is split into S = 6
// slices of integers of magnitude <= 128, held exactly in BF16, on a common
// power-of-two scale per row:
//   x_rj = sum_k a_k[r][j] 2^(E_r - 7 - 8(k - 1)) + rx,  |rx| <= 2^(E_r - 8 S)
//   q_ij = sum_l b_l[i][j] 2^(F_i - 7 - 8(l - 1)) + rq,  |rq| <= 2^(F_i - 8 S)
// with max_j |x_rj| < 2^E_r and max_j |q_ij| < 2^F_i.  Each product of two
// slices is an integer below 2^14, so an FP32 tensor-core accumulator over
// K <= 1024 holds every partial sum exactly; the products of the 21 slice
// pairs with k + l <= 7 are scaled by their powers of two and summed into the
// double-float pairs (TwoSum, then Fast2Sum), smallest first (12 launches: a pair
// (k, l) shares its pass over the pairs with (k, l - 1)).  Against the
// exact product the result errs by the dropped pairs (k + l >= 8: at most
// 5.02 K 2^(E_r + F_i - 48)) and the slices' remainders (2 K 2^(E_r + F_i - 48)),
// plus the rounding of the pairs' sums -- a relative error near 2^-45 of the
// row's scale, where one BF16 or FP32 product would give 2^-8 or 2^-24; the
// test of sa_rotate_rows restates the bound on the host.
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>

#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kSlices = 6;
constexpr int kMaxOrder = 7;  // slice pairs with k + l <= kMaxOrder

// One warp per row of an FP32 matrix X [rows x n] (row-major): the row's
// exponent E (max |x| < 2^E; 0 for a zero row) and its slices, exact in FP32.
__global__ void slice_rows_f32_kernel(const float* __restrict__ X, int64_t rows, int n,
                                      __nv_bfloat16* __restrict__ out, int* __restrict__ er) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const float* x = X + r * n;
    float m = 0.0f;
    for (int j = lane; j < n; j += 32) m = fmaxf(m, fabsf(x[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int E = 0;
    if (m > 0.0f) frexpf(m, &E);  // m = f 2^E, 1/2 <= f < 1
    for (int j = lane; j < n; j += 32) {
        float res = ldexpf(x[j], 7 - E);  // |res| < 128, exact
#pragma unroll
        for (int k = 0; k < kSlices; ++k) {
            const float a = rintf(res);
            out[((size_t)k * rows + r) * n + j] = __float2bfloat16_rn(a);  // an integer <= 128: exact
            res = (res - a) * 256.0f;  // exact: |res - a| <= 1/2 and its bits are res's own
        }
    }
    if (lane == 0) er[r] = E;
}

// The same for an FP64 matrix (Q), in FP64.
__global__ void slice_rows_f64_kernel(const double* __restrict__ X, int rows, int n, __nv_bfloat16* __restrict__ out,
                                      int* __restrict__ er) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const double* x = X + (size_t)r * n;
    double m = 0.0;
    for (int j = lane; j < n; j += 32) m = fmax(m, fabs(x[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int E = 0;
    if (m > 0.0) frexp(m, &E);
    for (int j = lane; j < n; j += 32) {
        double res = ldexp(x[j], 7 - E);
#pragma unroll
        for (int k = 0; k < kSlices; ++k) {
            const double a = rint(res);
            out[((size_t)k * rows + r) * n + j] = __float2bfloat16_rn((float)a);
            res = (res - a) * 256.0;
        }
    }
    if (lane == 0) er[r] = E;
}

}  // namespace

size_t rot_tc_work_bytes(int64_t C, int n) {
    return (size_t)kSlices * ((size_t)C + (size_t)n) * (size_t)n * sizeof(__nv_bfloat16) +
           ((size_t)C + (size_t)n) * sizeof(int) + 256;
}

bool rot_tc_shape_ok(int64_t C, int n) { return n % 64 == 0 && n <= 1024 && C % 128 == 0 && C <= ((int64_t)1 << 30); }

// Y [C x n] (pairs) = X [C x n] (FP32) . Q^T (Q [n x n] FP64, row-major), exactly split.
cudaError_t launch_rot_tc(const float* X, int64_t C, int n, const double* Q, float2* Y, void* work, int* status,
                          cudaStream_t s) {
    if (!rot_tc_shape_ok(C, n)) return cudaErrorInvalidValue;
    __nv_bfloat16* xs = static_cast<__nv_bfloat16*>(work);
    __nv_bfloat16* qs = xs + (size_t)kSlices * C * n;
    int* er = reinterpret_cast<int*>(qs + (size_t)kSlices * n * n);
    int* fq = er + C;
    slice_rows_f32_kernel<<<(unsigned)((C + 7) / 8), 256, 0, s>>>(X, C, n, xs, er);
    slice_rows_f64_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(Q, n, n, qs, fq);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(Y, 0, (size_t)C * n * sizeof(float2), s);
    // The slice pairs (k, l) by decreasing order m = k + l, so the smallest terms are
    // summed first: at each order, pair (k, l) shares its launch (and its pass over Y)
    // with (k, l - 1), one order lower, added after it.
    bool done[kSlices + 1][kSlices + 1] = {};
    for (int m = kMaxOrder; m >= 2 && e == cudaSuccess; --m)
        for (int k = 1; k <= kSlices && e == cudaSuccess; ++k) {
            const int l = m - k;
            if (l < 1 || l > kSlices || done[k][l]) continue;
            const __nv_bfloat16* a = xs + (size_t)(k - 1) * C * n;
            const int sh = 14 + 8 * (m - 2);
            if (l >= 2 && n % 128 == 0) {
                e = launch_gemm_accum_pair2(a, n, qs, n, kSlices * n, (l - 2) * n, (l - 1) * n, Y, n, (int)C, n, n, er,
                                            fq, sh - 8, sh, status, s);
                done[k][l - 1] = true;
            } else {
                e = launch_gemm_accum_pair(a, n, qs + (size_t)(l - 1) * n * n, n, Y, n, (int)C, n, n, er, fq, sh,
                                           status, s);
            }
            done[k][l] = true;
        }
    return e;
}

}  // namespace sa
