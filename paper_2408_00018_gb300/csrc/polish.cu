// polish.cu -- local minimiser of the hybrid SA: box-projected gradient
// descent with Armijo backtracking, in FP64, one warp per start point.
//
// The paper stops SA early and hands its point to Nelder-Mead (Sec. 4.2 and
// Table 10); here the k best final states of the last level are polished by
//   x <- P_I(x - alpha grad f(x)),  alpha = 1, 1/2, 1/4, ... until
//   f(x_new) <= f(x) + c grad f(x) . (x_new - x)   (Armijo, c = 1e-4),
// (the first search starts at alpha = 1, each later one at twice the last
// accepted step), stopping when the projected gradient's infinity norm P_I(x - g) - x falls
// below tol, when no step of the 30 halvings decreases f, or after max_iter
// iterations.  Sums over coordinates use a fixed lane-strided order and a
// butterfly, so results differ from a sequential sum only by rounding.
#include <cmath>
#include <cstdint>
#include <math_constants.h>

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ double dh64_schwefel(double t) {
    const double r = sqrt(fabs(t));
    return sin(r) + 0.5 * r * cos(r);
}

__device__ __forceinline__ double rot_term(int cost, double y) {
    return cost == kRotRastrigin ? g64_rastrigin(y) : h64_schwefel(y);
}

// y = Q x (Q row-major [n x n]); lanes own rows, each row summed in index order.
__device__ void protate(int n, const double* __restrict__ Q, const double* x, double* y) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < n; i += 32) {
        const double* q = Q + (size_t)i * n;
        double s = 0.0;
        for (int j = 0; j < n; ++j) s = fma(q[j], x[j], s);
        y[i] = s;
    }
    __syncwarp();
}

// f at x (warp-cooperative, lanes over coordinates); every lane gets the value.
// Rotated costs evaluate the formula at y = Q x (y: n doubles of workspace).
__device__ double pcost(int cost, int n, const double* x, const double* Q, double* y) {
    const int lane = threadIdx.x & 31;
    if (cost == kRotRastrigin || cost == kRotSchwefel) {
        protate(n, Q, x, y);
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += rot_term(cost, y[i]);
        s = warp_sum(s);
        return cost == kRotRastrigin ? 10.0 * (double)n + s : -(s / (double)n);
    }
    double s1 = 0.0, s2 = 0.0;
    for (int k = lane; k < n; k += 32) {
        const double t = x[k];
        if (cost == kSchwefel) s1 += h64_schwefel(t);
        else if (cost == kRastrigin) s1 += g64_rastrigin(t);
        else if (cost == kAckley) { s1 += t * t; s2 += cos(6.283185307179586 * t); }
        else if (k + 1 < n) s1 += rosen64(t, x[k + 1]);
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (cost == kSchwefel) return -(s1 / (double)n);
    if (cost == kRastrigin) return 10.0 * (double)n + s1;
    if (cost == kAckley) return ackley64(n, s1, s2);
    return s1;
}

// gradient of f at x into g (warp-cooperative); rotated costs: Q^T g'(y), y = Q x
// (y, gy: n doubles of workspace each).
__device__ void pgrad(int cost, int n, const double* x, double* g, const double* Q, double* y, double* gy) {
    const int lane = threadIdx.x & 31;
    if (cost == kRotRastrigin || cost == kRotSchwefel) {
        protate(n, Q, x, y);
        for (int i = lane; i < n; i += 32) {
            const double t = y[i];
            gy[i] = cost == kRotRastrigin ? 2.0 * t + 20.0 * CUDART_PI * sin(6.283185307179586 * t)
                                          : -dh64_schwefel(t) / (double)n;
        }
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s = fma(Q[(size_t)i * n + j], gy[i], s);
            g[j] = s;
        }
        return;
    }
    if (cost == kAckley) {
        double s1 = 0.0, s2 = 0.0;
        for (int k = lane; k < n; k += 32) { s1 += x[k] * x[k]; s2 += cos(6.283185307179586 * x[k]); }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        const double r = sqrt(s1 / (double)n);
        const double e1 = exp(-0.2 * r), e2 = exp(s2 / (double)n);
        for (int k = lane; k < n; k += 32) {
            const double a = r > 0.0 ? 4.0 * e1 * x[k] / ((double)n * r) : 0.0;
            g[k] = a + 2.0 * CUDART_PI * sin(6.283185307179586 * x[k]) * e2 / (double)n;
        }
        return;
    }
    for (int k = lane; k < n; k += 32) {
        const double t = x[k];
        if (cost == kSchwefel) g[k] = -dh64_schwefel(t) / (double)n;
        else if (cost == kRastrigin) g[k] = 2.0 * t + 20.0 * CUDART_PI * sin(6.283185307179586 * t);
        else {
            double gi = 0.0;
            if (k + 1 < n) gi += -400.0 * t * (x[k + 1] - t * t) - 2.0 * (1.0 - t);
            if (k > 0) gi += 200.0 * (t - x[k - 1] * x[k - 1]);
            g[k] = gi;
        }
    }
}

// One warp polishes one start point.  smem per warp: 5 n doubles (x, g, x_new and,
// for rotated costs, y and g'(y)).
__global__ void pgd_kernel(int cost, int n, const double* __restrict__ lo, const double* __restrict__ hi,
                           const double* __restrict__ Q, int k_points, const double* __restrict__ x0,
                           double* __restrict__ x_out, double* __restrict__ f_out, int* __restrict__ it_out,
                           int max_iter, double tol, double armijo_c, int max_halvings) {
    extern __shared__ double psm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + warp;
    if (w >= k_points) return;
    double* x = psm + (size_t)warp * 5 * n;
    double* g = x + n;
    double* xn = g + n;
    double* y = xn + n;
    double* gy = y + n;
    for (int k = lane; k < n; k += 32) x[k] = fmin(fmax(x0[(size_t)w * n + k], lo[k]), hi[k]);
    __syncwarp();
    double f = pcost(cost, n, x, Q, y);
    double alpha_next = 1.0;  // first search from 1, later ones from twice the last accepted step
    int it = 0;
    for (; it < max_iter; ++it) {
        pgrad(cost, n, x, g, Q, y, gy);
        __syncwarp();
        double pg = 0.0;
        for (int k = lane; k < n; k += 32) pg = fmax(pg, fabs(fmin(fmax(x[k] - g[k], lo[k]), hi[k]) - x[k]));
        pg = warp_max(pg);
        if (pg < tol) break;
        double alpha = alpha_next, fn = f;
        bool ok = false;
        for (int hh = 0; hh < max_halvings; ++hh) {
            double slope = 0.0;
            for (int k = lane; k < n; k += 32) {
                xn[k] = fmin(fmax(x[k] - alpha * g[k], lo[k]), hi[k]);
                slope += g[k] * (xn[k] - x[k]);
            }
            slope = warp_sum(slope);
            __syncwarp();
            fn = pcost(cost, n, xn, Q, y);
            if (fn <= f + armijo_c * slope) { ok = true; break; }
            alpha = 0.5 * alpha;
            __syncwarp();
        }
        if (!ok) break;
        for (int k = lane; k < n; k += 32) x[k] = xn[k];
        __syncwarp();
        f = fn;
        alpha_next = fmin(2.0 * alpha, 1e12);
    }
    for (int k = lane; k < n; k += 32) x_out[(size_t)w * n + k] = x[k];
    if (lane == 0) {
        f_out[w] = f;
        if (it_out) it_out[w] = it;
    }
}

// Top-k of the level's FP64 values (lowest value, then lowest index), one block;
// destroys the copy it works on by marking winners with +inf.
__global__ void topk_kernel(double* F, int64_t count, int k, int64_t* idx_out) {
    __shared__ double sv[32];
    __shared__ int64_t si[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < k; ++j) {
        double bv = CUDART_INF;
        int64_t bi = INT64_MAX;
        for (int64_t i = t; i < count; i += blockDim.x) {
            const double v = F[i];
            if (v < bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_xor_sync(kFull, bv, o);
            const long long i = __shfl_xor_sync(kFull, (long long)bi, o);
            if (v < bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
        if (lane == 0) { sv[wid] = bv; si[wid] = bi; }
        __syncthreads();
        if (t == 0) {
            for (int w = 1; w < nw; ++w)
                if (sv[w] < sv[0] || (sv[w] == sv[0] && si[w] < si[0])) { sv[0] = sv[w]; si[0] = si[w]; }
            idx_out[j] = si[0] == INT64_MAX ? -1 : si[0];
            if (si[0] != INT64_MAX) F[si[0]] = CUDART_INF;
        }
        __syncthreads();
    }
}

// Gather the selected chains' states (FP32 or FP64 storage, [n][chains] layout) as FP64 starts.
__global__ void gather_kernel(const float* X32, const double* X64, int64_t x_base, int64_t chains, int n,
                              const int64_t* idx, int k, double* out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)k * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), d = (int)(e % n);
        const int64_t c = idx[j] < 0 ? 0 : idx[j];
        const size_t off = (size_t)x_base + (size_t)d * (size_t)chains + (size_t)c;
        out[e] = X64 ? X64[off] : (double)X32[off];
    }
}

// Keep the best polished point if it improves the incumbent.
__global__ void polish_update_kernel(ProbDev* probs, int problem, const double* xs, const double* fs, int k) {
    __shared__ int best;
    const ProbDev& P = probs[problem];
    if (threadIdx.x == 0) {
        best = -1;
        double bf = P.scal[kFInc];
        for (int j = 0; j < k; ++j)
            if (fs[j] < bf) { bf = fs[j]; best = j; }
        if (best >= 0) P.scal[kFInc] = bf;
    }
    __syncthreads();
    if (best >= 0)
        for (int d = threadIdx.x; d < P.n; d += blockDim.x) P.x_inc[d] = xs[(size_t)best * P.n + d];
}

}  // namespace

size_t pgd_smem_bytes(int n, int warps) { return (size_t)warps * 5 * (size_t)n * sizeof(double); }

cudaError_t launch_pgd(int cost, int n, const double* lo, const double* hi, const double* Q, int k, const double* x0,
                       double* x_out, double* f_out, int* it_out, int max_iter, double tol, cudaStream_t s) {
    const int warps = n > 1024 ? 1 : 4;  // 5 n doubles per warp
    const size_t smem = pgd_smem_bytes(n, warps);
    cudaError_t e = cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    pgd_kernel<<<(k + warps - 1) / warps, 32 * warps, smem, s>>>(cost, n, lo, hi, Q, k, x0, x_out, f_out, it_out,
                                                                  max_iter, tol, 1e-4, 30);
    return cudaGetLastError();
}

cudaError_t launch_topk(double* F, int64_t count, int k, int64_t* idx, cudaStream_t s) {
    topk_kernel<<<1, 1024, 0, s>>>(F, count, k, idx);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float* X32, const double* X64, int64_t x_base, int64_t chains, int n, const int64_t* idx,
                          int k, double* out, cudaStream_t s) {
    gather_kernel<<<64, 256, 0, s>>>(X32, X64, x_base, chains, n, idx, k, out);
    return cudaGetLastError();
}

cudaError_t launch_polish_update(ProbDev* probs, int problem, const double* xs, const double* fs, int k, cudaStream_t s) {
    polish_update_kernel<<<1, 256, 0, s>>>(probs, problem, xs, fs, k);
    return cudaGetLastError();
}

}  // namespace sa
