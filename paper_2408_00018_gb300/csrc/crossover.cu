// crossover.cu -- the stochastic crossover at an exchange: Boltzmann selection.
//
// The paper's synchronous scheme restarts every chain from the minimum over the
// chains (Sec. 2.2.2) and names, as the alternative, an exchange whose
// crossover operator is random (the SOS scheme it cites).  Here chain c
// restarts from chain j's final state with probability w_j / sum_k w_k,
// w_j = exp(-(F_j - F_min) / T) at the finished level's temperature (0 for a
// non-finite F_j): the weights and their running sum S_j over the chains are
// formed on the device (block sums, a scan of the block sums, block-local
// scans), then each chain inverts the running sum at t = u_c S_{C-1} by binary
// search, u_c from word 0 of the Philox block (0, level, chain id, problem) of
// stream tag 5, and the drawn states are gathered into the start states of the
// next level.  The kernels run before each level's sweep and do nothing unless
// an exchange follows the previous level (they read the level from the device),
// so the sequence is captured once in the level graph and the previous level's
// final states stay readable until the next level starts.  The sums are formed in a fixed order, so a
// draw differs from a sequential running sum only where t lies within rounding
// of some S_j.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <math_constants.h>

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kXoBlock = 1024;
constexpr unsigned kFull = 0xffffffffu;

// The level whose final states are drawn from: the one before the level about to run.
__device__ __forceinline__ int xo_level(const SweepArgs& A) { return A.run->level - 1; }
__device__ __forceinline__ bool xo_active(const SweepArgs& A) {
    return A.run->level > 0 && exchange_after(A, xo_level(A));
}

// Inclusive scan of one value per thread over the block (Hillis-Steele in shared
// memory, a fixed order of additions); sh: kXoBlock doubles.
__device__ double block_inclusive_scan(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < kXoBlock; off <<= 1) {
        const double a = t >= off ? sh[t - off] : 0.0;
        __syncthreads();
        sh[t] += a;
        __syncthreads();
    }
    return sh[t];
}

__global__ void __launch_bounds__(kXoBlock) xo_weights_kernel(SweepArgs A, const ProbDev* Pp, double* w, double* bsum) {
    if (!xo_active(A)) return;
    const ProbDev& P = *Pp;
    const double T = A.T_tab[xo_level(A)];
    const double Fmin = P.scal[kFBest];
    const int64_t j = (int64_t)blockIdx.x * kXoBlock + threadIdx.x;
    double v = 0.0;
    if (j < P.chains) {
        const double f = A.F[P.chain_base + j];
        v = isfinite(f) ? exp(-(f - Fmin) / T) : 0.0;
        w[j] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __shared__ double ws[kXoBlock / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kXoBlock / 32; ++k) s += ws[k];
        bsum[blockIdx.x] = s;
    }
}

// bsum[0..nb) -> their exclusive running sum; bsum[nb] = the total.  One block.
__global__ void __launch_bounds__(kXoBlock) xo_scan_kernel(SweepArgs A, int64_t nb, double* bsum) {
    if (!xo_active(A)) return;
    __shared__ double sh[kXoBlock];
    __shared__ double carry;
    if (threadIdx.x == 0) carry = 0.0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kXoBlock) {
        const int64_t b = base + threadIdx.x;
        const double v = b < nb ? bsum[b] : 0.0;
        block_inclusive_scan(v, sh);
        const double excl = threadIdx.x > 0 ? sh[threadIdx.x - 1] : 0.0;
        const double c0 = carry;
        __syncthreads();
        if (b < nb) bsum[b] = c0 + excl;
        if (threadIdx.x == 0) carry = c0 + sh[kXoBlock - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kXoBlock) xo_prefix_kernel(SweepArgs A, const ProbDev* Pp, const double* w,
                                                             const double* bsum, double* S) {
    if (!xo_active(A)) return;
    __shared__ double sh[kXoBlock];
    const int64_t C = Pp->chains;
    const int64_t j = (int64_t)blockIdx.x * kXoBlock + threadIdx.x;
    const double incl = block_inclusive_scan(j < C ? w[j] : 0.0, sh);
    if (j < C) S[j] = bsum[blockIdx.x] + incl;
}

__global__ void xo_pick_kernel(SweepArgs A, const ProbDev* Pp, int64_t nb, const double* bsum, const double* S,
                               int64_t* src, uint32_t k0, uint32_t k1) {
    if (!xo_active(A)) return;
    const ProbDev& P = *Pp;
    const int64_t C = P.chains;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const uint4 r = philox4x32_10(make_uint4(0u, (uint32_t)xo_level(A), (uint32_t)c + P.cid0, P.pid), k0, k1);
    const double t = u23d(r.x) * bsum[nb];
    int64_t a = 0, b = C - 1;
    while (a < b) {
        const int64_t m = a + (b - a) / 2;
        if (S[m] > t) b = m;
        else a = m + 1;
    }
    src[c] = a;
}

// [n][chains] blocks (FP32 or FP64 states): tmp = X[:, src], then X = tmp.
template <class T>
__global__ void xo_gather_cols_kernel(SweepArgs A, const ProbDev* Pp, T* X, const int64_t* src, T* tmp) {
    if (!xo_active(A)) return;
    const ProbDev& P = *Pp;
    const int64_t C = P.chains, total = C * (int64_t)P.n;
    T* base = X + P.x_base;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / C, c = e - k * C;
        tmp[e] = base[k * C + src[c]];
    }
}
template <class T>
__global__ void xo_copy_back_kernel(SweepArgs A, const ProbDev* Pp, T* X, const T* tmp) {
    if (!xo_active(A)) return;
    const ProbDev& P = *Pp;
    const int64_t total = P.chains * (int64_t)P.n;
    T* base = X + P.x_base;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        base[e] = tmp[e];
}

// Rotated costs: the [chains][n] rows of x0 and of the (hi, lo) pairs y0 = Q x0.
__global__ void xo_gather_rows_kernel(SweepArgs A, const ProbDev* Pp, const int64_t* src, float* tx, float2* ty) {
    if (!xo_active(A)) return;
    const ProbDev& P = *Pp;
    const int64_t n = P.n, total = P.chains * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, k = e - c * n;
        tx[e] = P.x0[src[c] * n + k];
        ty[e] = P.y0[src[c] * n + k];
    }
}
__global__ void xo_copy_rows_kernel(SweepArgs A, const ProbDev* Pp, const float* tx, const float2* ty) {
    if (!xo_active(A)) return;
    const ProbDev& P = *Pp;
    const int64_t total = P.chains * (int64_t)P.n;
    float* x0 = const_cast<float*>(P.x0);
    float2* y0 = const_cast<float2*>(P.y0);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        x0[e] = tx[e];
        y0[e] = ty[e];
    }
}

}  // namespace

size_t crossover_blocks(int64_t chains) { return (size_t)((chains + kXoBlock - 1) / kXoBlock); }

cudaError_t launch_crossover(const SweepArgs& a, const ProbDev* dprob, const ProbDev& hprob, int precision, bool rot,
                             uint32_t xkey0, uint32_t xkey1, const CrossoverWork& w, cudaStream_t s) {
    const int64_t C = hprob.chains;
    const int64_t nb = (int64_t)crossover_blocks(C);
    const int64_t total = C * (int64_t)hprob.n;
    const int gblocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    xo_weights_kernel<<<(unsigned)nb, kXoBlock, 0, s>>>(a, dprob, w.w, w.bsum);
    xo_scan_kernel<<<1, kXoBlock, 0, s>>>(a, nb, w.bsum);
    xo_prefix_kernel<<<(unsigned)nb, kXoBlock, 0, s>>>(a, dprob, w.w, w.bsum, w.S);
    xo_pick_kernel<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(a, dprob, nb, w.bsum, w.S, w.src, xkey0, xkey1);
    if (rot) {
        float* tx = static_cast<float*>(w.xtmp);
        float2* ty = reinterpret_cast<float2*>(tx + total + (total & 1));  // 8-byte aligned after tx
        xo_gather_rows_kernel<<<gblocks, 256, 0, s>>>(a, dprob, w.src, tx, ty);
        xo_copy_rows_kernel<<<gblocks, 256, 0, s>>>(a, dprob, tx, ty);
    } else if (precision == 0) {
        xo_gather_cols_kernel<double><<<gblocks, 256, 0, s>>>(a, dprob, a.X64, w.src, static_cast<double*>(w.xtmp));
        xo_copy_back_kernel<double><<<gblocks, 256, 0, s>>>(a, dprob, a.X64, static_cast<const double*>(w.xtmp));
    } else {
        xo_gather_cols_kernel<float><<<gblocks, 256, 0, s>>>(a, dprob, a.X32, w.src, static_cast<float*>(w.xtmp));
        xo_copy_back_kernel<float><<<gblocks, 256, 0, s>>>(a, dprob, a.X32, static_cast<const float*>(w.xtmp));
    }
    return cudaGetLastError();
}

}  // namespace sa
