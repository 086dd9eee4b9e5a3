// rot_prep.cu -- FP64 transforms of the rotated costs f(x) = F(Q x):
//   * level 0: the chains' random initial points X0 (FP32, [chains][n]) and
//     Y0 = X0 Q^T, stored as double-float pairs: on the tensor cores by the
//     exact split product of rot_tc.cu where the shape allows, else in FP64
//     (tiled GEMM);
//   * every restart: y_best = Q x_best in FP64 and F(y_best) (one thread per
//     rotated coordinate, partial sums reduced by the last block to finish).
// Every dot product runs over j = 0..n-1 in index order.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;   // chains x rotated coordinates x K per tile
constexpr int kGemmThreads = 256;              // 16 x 16 threads, 4 x 4 outputs each
constexpr int kRestartThreads = 128;

// Initial points of level 0 (Sec. 2.1, Step 1): x_k uniform in [l_k, u_k] from
// word k mod 4 of Philox block (k / 4, 0, chain, problem) of the init stream,
// rounded to FP32 inside the box.
__global__ void rot_init_kernel(const ProbDev* pp, uint32_t ikey0, uint32_t ikey1, float* x0) {
    const ProbDev& P = *pp;
    const int n = P.n;
    const int nq = (n + 3) / 4;
    const int64_t total = P.chains * (int64_t)nq;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / nq;
        const int k = (int)(t - c * nq) * 4;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(k >> 2), 0u, (uint32_t)c + P.cid0, P.pid), ikey0, ikey1);
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k + j < n) {
                const double lo = P.lo[k + j], hi = P.hi[k + j];
                const float x = (float)(lo + u23d(ww[j]) * (hi - lo));
                x0[c * n + k + j] = fminf(fmaxf(x, P.lo32[k + j]), P.hi32[k + j]);
            }
        }
    }
}

// Y0[c][i] = sum_j X0[c][j] Q[i][j] in FP64; output as (hi, lo) FP32 pairs.
__global__ void __launch_bounds__(kGemmThreads) rot_y0_kernel(const ProbDev* pp, const float* __restrict__ x0,
                                                              float2* __restrict__ y0) {
    __shared__ double As[kBK][kBM + 1];
    __shared__ double Bs[kBK][kBN + 1];
    const ProbDev& P = *pp;
    const int n = P.n;
    const int64_t C = P.chains;
    const int i0 = blockIdx.x * kBN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int64_t c0 = (int64_t)blockIdx.y * kBM; c0 < C; c0 += (int64_t)gridDim.y * kBM) {
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] = 0.0;
    for (int k0 = 0; k0 < n; k0 += kBK) {
#pragma unroll
        for (int q = 0; q < (kBM * kBK) / kGemmThreads; ++q) {
            const int e = threadIdx.x + q * kGemmThreads;
            const int m = e / kBK, kk = e % kBK;
            const int64_t c = c0 + m;
            const int k = k0 + kk;
            As[kk][m] = (c < C && k < n) ? (double)x0[c * n + k] : 0.0;
            const int i = i0 + m;
            Bs[kk][m] = (i < n && k < n) ? P.q64[(size_t)i * n + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int s = 0; s < 4; ++s) b[s] = Bs[kk][tx * 4 + s];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], b[s], acc[r][s]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t c = c0 + ty * 4 + r;
        if (c >= C) continue;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = i0 + tx * 4 + s;
            if (i < n) {
                const float h = (float)acc[r][s];
                y0[c * n + i] = make_float2(h, (float)(acc[r][s] - (double)h));
            }
        }
    }
    }
}

// y_best = Q x_best (FP64, index order) as pairs, and F(y_best) from the pairs.
__global__ void __launch_bounds__(kRestartThreads) rot_restart_kernel(ProbDev* pp) {
    __shared__ double part[kRestartThreads];
    __shared__ bool last;
    ProbDev& P = *pp;
    const int n = P.n;
    const int i = blockIdx.x * kRestartThreads + threadIdx.x;
    double g = 0.0;
    if (i < n) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s = fma(P.qt64[(size_t)j * n + i], (double)P.x_best32[j], s);
        const float h = (float)s;
        const float l = (float)(s - (double)h);
        P.ybest_hi[i] = h;
        P.ybest_lo[i] = l;
        const double y = (double)h + (double)l;
        g = P.cost == kRotRastrigin ? g64_rastrigin(y) : h64_schwefel(y);
    }
    part[threadIdx.x] = g;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int t = 0; t < kRestartThreads; ++t) b += part[t];
        P.rot_part[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(P.rot_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile double*)P.rot_part)[b];
        P.scal[kFRot] = P.cost == kRotRastrigin ? 10.0 * (double)n + s : -(s / (double)n);
        *P.rot_done = 0u;
    }
}

}  // namespace

cudaError_t launch_rot_level0(const ProbDev* d_prob, const ProbDev& hp, const SweepArgs& a, float* x0, float2* y0,
                              void* tc_work, int* status, cudaStream_t s) {
    const int64_t work = hp.chains * (int64_t)((hp.n + 3) / 4);
    const int64_t blocks = std::min<int64_t>((work + 255) / 256, 152 * 16);
    rot_init_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_prob, a.ikey0, a.ikey1, x0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (tc_work) return launch_rot_tc(x0, hp.chains, hp.n, hp.q64, y0, tc_work, status, s);
    const dim3 grid((unsigned)((hp.n + kBN - 1) / kBN), (unsigned)std::min<int64_t>((hp.chains + kBM - 1) / kBM, 65535));
    rot_y0_kernel<<<grid, kGemmThreads, 0, s>>>(d_prob, x0, y0);
    return cudaGetLastError();
}

int rot_restart_blocks(int n) { return (n + kRestartThreads - 1) / kRestartThreads; }

cudaError_t launch_rot_restart(const ProbDev* d_prob, int n, cudaStream_t s) {
    rot_restart_kernel<<<rot_restart_blocks(n), kRestartThreads, 0, s>>>(const_cast<ProbDev*>(d_prob));
    return cudaGetLastError();
}

}  // namespace sa
