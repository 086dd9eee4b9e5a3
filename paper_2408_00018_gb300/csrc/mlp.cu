// mlp.cu -- the learned surrogate f~(x) = w3 . g(W2 g(W1 x + b1) + b2) + b3
// (g = erf-form GELU, hidden widths 512 and 512) on the tensor cores, and its
// training: mean squared error, gradients by the chain rule, Adam (Kingma & Ba
// 2015).  The paper has no surrogate; it serves the delayed-acceptance sweep.
//
// Parameters are kept in FP32 (flat vector: W1 [512 x n], b1, W2 [512 x 512],
// b2, w3, b3); the GEMMs take BF16 copies (W1 padded to np = n rounded up to 64
// columns, W2 and its transpose) and accumulate in FP32 (gemm_tc.cu).
//   forward:  Z1 = X W1^T + b1, A1 = g(Z1)       (GEMM, fused bias + GELU, BF16 out)
//             f~ = sum_j g(A1 W2^T + b2)_j w3_j + b3   (GEMM, fused bias + GELU + dot)
//   backward: dy = (f~ - t) / B
//             dZ2 = dy w3^T o g'(Z2);  dW2 = dZ2^T A1;  dA1 = dZ2 W2
//             dZ1 = dA1 o g'(Z1);     dW1 = dZ1^T X
// Column sums (bias gradients, dw3) and the loss are reduced in fixed order.
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/sa.h"
#include "gelu.cuh"
#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kH = kMlpHidden;
constexpr uint32_t kTagMlpInit = 2u;

// GELU and its derivative: the forms of gelu.cuh, which the GEMM epilogues evaluate.
__device__ __forceinline__ float gelu(float z) { return gelu_f(z); }
__device__ __forceinline__ float gelu_grad(float z) { return gelu_grad_f(z); }

__global__ void cast_kernel(const float* __restrict__ p, int n, int np, __nv_bfloat16* W1b, __nv_bfloat16* W2b,
                            __nv_bfloat16* W2tb) {
    const MlpOffsets o = mlp_offsets(n);
    const int64_t n1 = (int64_t)kH * np, n2 = (int64_t)kH * kH;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n1 + 2 * n2;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n1) {
            const int i = (int)(t / np), k = (int)(t % np);
            W1b[t] = __float2bfloat16_rn(k < n ? p[o.W1 + (int64_t)i * n + k] : 0.0f);
        } else if (t < n1 + n2) {
            W2b[t - n1] = __float2bfloat16_rn(p[o.W2 + (t - n1)]);
        } else {
            const int64_t u = t - n1 - n2;
            const int j = (int)(u / kH), k = (int)(u % kH);  // W2t[j][k] = W2[k][j]
            W2tb[u] = __float2bfloat16_rn(p[o.W2 + (int64_t)k * kH + j]);
        }
    }
}

// X (FP32, [B x n]) -> BF16 [Bp x np], zero padding in both directions.
__global__ void pack_kernel(const float* __restrict__ X, int B, int n, int Bp, int np, __nv_bfloat16* Xb) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)Bp * np;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / np), k = (int)(t % np);
        Xb[t] = __float2bfloat16_rn(b < B && k < n ? X[(int64_t)b * n + k] : 0.0f);
    }
}

__global__ void finish_y_kernel(const float* __restrict__ part, const float* __restrict__ b3, int B, float* y) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        const float* q = part + (size_t)b * (kH / 128);
        float s = 0.0f;
#pragma unroll
        for (int t = 0; t < kH / 128; ++t) s += q[t];
        y[b] = s + *b3;
    }
}

// BF16 transpose of a [R x C] row-major matrix (R, C multiples of 32) into [C x R].
__global__ void transpose_kernel(const __nv_bfloat16* __restrict__ in, int R, int C, __nv_bfloat16* __restrict__ out) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) tile[k][threadIdx.x] = in[(size_t)(r0 + k) * C + c0 + threadIdx.x];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) out[(size_t)(c0 + k) * R + r0 + threadIdx.x] = tile[threadIdx.x][k];
}

// dy_b = (f~_b - t_b) / B for real rows (0 for padding); dZ2 = dy w3 o g'(Z2) as BF16.
__global__ void head_bwd_kernel(const float* __restrict__ y, const float* __restrict__ t, int B, int Bp,
                                const float* __restrict__ Z2, const float* __restrict__ w3, float* dy,
                                __nv_bfloat16* dZ2b) {
    const int b = blockIdx.x;
    const float d = b < B ? (y[b] - t[b]) / (float)B : 0.0f;
    if (threadIdx.x == 0) dy[b] = d;
    for (int j = threadIdx.x; j < kH; j += blockDim.x)
        dZ2b[(size_t)b * kH + j] = __float2bfloat16_rn(d * w3[j] * gelu_grad(Z2[(size_t)b * kH + j]));
    (void)Bp;
}

// Column reductions over the batch: rows are split into chunks of kRowChunk
// (one block column of threads per chunk, rows in order inside a chunk), and a
// second pass adds the chunks' partial sums in chunk order, so the result does
// not depend on scheduling.
//   head:  dw3_j = sum_b dy_b g(Z2_bj),  db2_j = sum_b dy_b w3_j g'(Z2_bj)
//   layer 1:  db1_j = sum_b dA1_bj g'(Z1_bj)
constexpr int kRowChunk = 64;

__global__ void col_head_part_kernel(const float* __restrict__ Z2, const float* __restrict__ dy,
                                     const float* __restrict__ w3, int Bp, float* part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (j >= kH) return;
    float s3 = 0.0f, s2 = 0.0f;
    const int b1 = min(Bp, (chunk + 1) * kRowChunk);
    for (int b = chunk * kRowChunk; b < b1; ++b) {
        const float z = Z2[(size_t)b * kH + j];
        s3 = fmaf(dy[b], gelu(z), s3);
        s2 = fmaf(dy[b] * w3[j], gelu_grad(z), s2);
    }
    part[((size_t)chunk * 2 + 0) * kH + j] = s3;
    part[((size_t)chunk * 2 + 1) * kH + j] = s2;
}

__global__ void col_b1_part_kernel(const float* __restrict__ dA1, const float* __restrict__ Z1, int Bp, float* part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (j >= kH) return;
    float s = 0.0f;
    const int b1 = min(Bp, (chunk + 1) * kRowChunk);
    for (int b = chunk * kRowChunk; b < b1; ++b) s = fmaf(dA1[(size_t)b * kH + j], gelu_grad(Z1[(size_t)b * kH + j]), s);
    part[(size_t)chunk * kH + j] = s;
}

// out_v[j] = sum over chunks (in order) of part[(chunk * stride + v) * kH + j], for v < nv.
__global__ void col_finish_kernel(const float* __restrict__ part, int chunks, int stride, int nv, float* out0,
                                  float* out1) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kH) return;
    for (int v = 0; v < nv; ++v) {
        float s = 0.0f;
        for (int c = 0; c < chunks; ++c) s += part[((size_t)c * stride + v) * kH + j];
        (v == 0 ? out0 : out1)[j] = s;
    }
}

__global__ void dz1_kernel(const float* __restrict__ dA1, const float* __restrict__ Z1, int Bp, __nv_bfloat16* dZ1b) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < (int64_t)Bp * kH;
         u += (int64_t)gridDim.x * blockDim.x)
        dZ1b[u] = __float2bfloat16_rn(dA1[u] * gelu_grad(Z1[u]));
}

// W1's gradient: the first n of the np columns of dW1full; the loss and db3 (one block).
__global__ void finish_grad_kernel(const float* __restrict__ dW1full, int n, int np, float* gW1) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)kH * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), k = (int)(t % n);
        gW1[t] = dW1full[(size_t)i * np + k];
    }
}

__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ dy, int B,
                            int Bp, float* loss, float* db3) {
    __shared__ float s1[256], s2[256];
    float a = 0.0f, c = 0.0f;
    for (int b = threadIdx.x; b < Bp; b += blockDim.x) {
        if (b < B) {
            const float r = y[b] - t[b];
            a = fmaf(r, r, a);
        }
        c += dy[b];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (loss) *loss = 0.5f * s1[0] / (float)B;
        *db3 = s2[0];
    }
}

__global__ void adam_kernel(float* p, const float* __restrict__ g, float* m, float* v, int64_t count, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// He-style normal initialisation from Philox (stream tag 2), zero biases.
__global__ void init_kernel(float* p, int n, uint32_t k0, uint32_t k1) {
    const MlpOffsets o = mlp_offsets(n);
    const int64_t total = o.total;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        float scale = 0.0f;
        if (i < o.b1) scale = sqrtf(2.0f / (float)n);
        else if (i >= o.W2 && i < o.b2) scale = sqrtf(2.0f / (float)kH);
        else if (i >= o.w3 && i < o.b3) scale = sqrtf(1.0f / (float)kH);
        float val = 0.0f;
        if (scale > 0.0f) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 0u), k0, k1);
            const float r = sqrtf(-2.0f * logf(u23f(w.x)));
            val = scale * r * cosf(6.283185307179586f * u23f(w.y));
        }
        p[i] = val;
    }
}

int grid_for(int64_t work, int block = 256) {
    int64_t g = (work + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

cudaError_t mlp_cast(const MlpDev& m, cudaStream_t s) {
    cast_kernel<<<grid_for((int64_t)kH * m.np + 2 * (int64_t)kH * kH), 256, 0, s>>>(m.p, m.n, m.np, m.W1b, m.W2b, m.W2tb);
    return cudaGetLastError();
}

cudaError_t mlp_init(float* p, int n, uint64_t seed, cudaStream_t s) {
    const MlpOffsets o = mlp_offsets(n);
    init_kernel<<<grid_for(o.total), 256, 0, s>>>(p, n, (uint32_t)seed, (uint32_t)(seed >> 32) ^ kTagMlpInit);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpDev& m, const void* Xb, int Bp, MlpWork& w, float* part, int* status, cudaStream_t s) {
    const MlpOffsets o = mlp_offsets(m.n);
    cudaError_t e = launch_gemm_bias_gelu(Xb, m.np, m.W1b, m.np, Bp, kH, m.np, m.p + o.b1, w.A1, kH, w.Z1, kH, status, s);
    if (e != cudaSuccess) return e;
    return launch_gemm_bias_gelu_dot(w.A1, kH, m.W2b, kH, Bp, kH, kH, m.p + o.b2, m.p + o.w3, part, w.Z2, kH, status, s);
}

// The fused forward pass where it applies, unless SA_MLP_FUSED=0 selects the two GEMMs.
bool mlp_use_fused(int np, int Bp) {
    const char* env = std::getenv("SA_MLP_FUSED");
    return !(env && env[0] == '0') && mlp_fused_ok(np, Bp);
}

cudaError_t mlp_infer(const MlpDev& m, const void* Xb, int Bp, __nv_bfloat16* A1, float* part, int* status,
                      cudaStream_t s) {
    const MlpOffsets o = mlp_offsets(m.n);
    if (mlp_use_fused(m.np, Bp))
        return launch_mlp_fused(Xb, m.np, Bp, m.W1b, m.W2b, m.p + o.b1, m.p + o.b2, m.p + o.w3, part, status, s);
    if (!A1) return cudaErrorInvalidValue;  // no workspace for the hidden activations
    cudaError_t e = launch_gemm_bias_gelu(Xb, m.np, m.W1b, m.np, Bp, kH, m.np, m.p + o.b1, A1, kH, nullptr, 0, status, s);
    if (e != cudaSuccess) return e;
    return launch_gemm_bias_gelu_dot(A1, kH, m.W2b, kH, Bp, kH, kH, m.p + o.b2, m.p + o.w3, part, nullptr, 0, status, s);
}

cudaError_t mlp_finish_y(const MlpDev& m, const float* part, int B, float* y, cudaStream_t s) {
    const MlpOffsets o = mlp_offsets(m.n);
    finish_y_kernel<<<(B + 255) / 256, 256, 0, s>>>(part, m.p + o.b3, B, y);
    return cudaGetLastError();
}

cudaError_t mlp_loss_grad(const MlpDev& m, const void* Xb, int B, int Bp, const float* t, MlpWork& w, float* grad,
                          float* loss, int* status, cudaStream_t s) {
    const MlpOffsets o = mlp_offsets(m.n);
    cudaError_t e = mlp_forward(m, Xb, Bp, w, w.part, status, s);
    if (e == cudaSuccess) e = mlp_finish_y(m, w.part, Bp, w.y, s);
    if (e != cudaSuccess) return e;
    head_bwd_kernel<<<Bp, 128, 0, s>>>(w.y, t, B, Bp, w.Z2, m.p + o.w3, w.dy, w.dZ2b);
    const int chunks = (Bp + kRowChunk - 1) / kRowChunk;
    col_head_part_kernel<<<dim3(kH / 128, chunks), 128, 0, s>>>(w.Z2, w.dy, m.p + o.w3, Bp, w.colpart);
    col_finish_kernel<<<kH / 128, 128, 0, s>>>(w.colpart, chunks, 2, 2, grad + o.w3, grad + o.b2);
    loss_kernel<<<1, 256, 0, s>>>(w.y, t, w.dy, B, Bp, loss, grad + o.b3);
    const dim3 tb(32, 8);
    transpose_kernel<<<dim3(kH / 32, Bp / 32), tb, 0, s>>>(w.dZ2b, Bp, kH, w.dZ2T);
    transpose_kernel<<<dim3(kH / 32, Bp / 32), tb, 0, s>>>(w.A1, Bp, kH, w.A1T);
    transpose_kernel<<<dim3(m.np / 32, Bp / 32), tb, 0, s>>>(static_cast<const __nv_bfloat16*>(Xb), Bp, m.np, w.XT);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // dW2 = dZ2^T A1 (K = batch), straight into the gradient vector
    e = launch_gemm_bf16_f32(w.dZ2T, Bp, w.A1T, Bp, grad + o.W2, kH, kH, kH, Bp, status, s);
    // dA1 = dZ2 W2
    if (e == cudaSuccess) e = launch_gemm_bf16_f32(w.dZ2b, kH, m.W2tb, kH, w.dA1, kH, Bp, kH, kH, status, s);
    if (e != cudaSuccess) return e;
    dz1_kernel<<<grid_for((int64_t)Bp * kH), 256, 0, s>>>(w.dA1, w.Z1, Bp, w.dZ1b);
    col_b1_part_kernel<<<dim3(kH / 128, chunks), 128, 0, s>>>(w.dA1, w.Z1, Bp, w.colpart);
    col_finish_kernel<<<kH / 128, 128, 0, s>>>(w.colpart, chunks, 1, 1, grad + o.b1, nullptr);
    transpose_kernel<<<dim3(kH / 32, Bp / 32), tb, 0, s>>>(w.dZ1b, Bp, kH, w.dZ1T);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // dW1 = dZ1^T X (K = batch), then its first n columns
    e = launch_gemm_bf16_f32(w.dZ1T, Bp, w.XT, Bp, w.dW1, m.np, kH, m.np, Bp, status, s);
    if (e != cudaSuccess) return e;
    finish_grad_kernel<<<grid_for((int64_t)kH * m.n), 256, 0, s>>>(w.dW1, m.n, m.np, grad + o.W1);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float* p, const float* g, float* mo, float* vo, int64_t count, int step, float lr, float b1, float b2,
                     float eps, cudaStream_t s) {
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<grid_for(count), 256, 0, s>>>(p, g, mo, vo, count, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t mlp_pack(const float* X, int B, int n, int Bp, int np, void* Xb, cudaStream_t s) {
    pack_kernel<<<grid_for((int64_t)Bp * np), 256, 0, s>>>(X, B, n, Bp, np, static_cast<__nv_bfloat16*>(Xb));
    return cudaGetLastError();
}

size_t mlp_work_bytes(int Bp, int np) {
    const size_t b = (size_t)Bp;
    const size_t chunks = (b + kRowChunk - 1) / kRowChunk;
    return b * np * 2 * 2 + b * kH * (4 + 2 + 2 + 4 + 2 + 2 + 4 + 2 + 2) + b * (4 + 4 + 4 * 4) + (size_t)kH * np * 4 +
           chunks * 2 * kH * 4 + 16 * 256;
}

void mlp_work_carve(void* base, int Bp, int np, MlpWork& w) {
    auto take = [&base](size_t bytes) {
        void* r = base;
        base = static_cast<char*>(base) + ((bytes + 255) & ~(size_t)255);
        return r;
    };
    const size_t b = (size_t)Bp;
    w.Xb = static_cast<__nv_bfloat16*>(take(b * np * 2));
    w.XT = static_cast<__nv_bfloat16*>(take(b * np * 2));
    w.Z1 = static_cast<float*>(take(b * kH * 4));
    w.A1 = static_cast<__nv_bfloat16*>(take(b * kH * 2));
    w.A1T = static_cast<__nv_bfloat16*>(take(b * kH * 2));
    w.Z2 = static_cast<float*>(take(b * kH * 4));
    w.dZ2b = static_cast<__nv_bfloat16*>(take(b * kH * 2));
    w.dZ2T = static_cast<__nv_bfloat16*>(take(b * kH * 2));
    w.dA1 = static_cast<float*>(take(b * kH * 4));
    w.dZ1b = static_cast<__nv_bfloat16*>(take(b * kH * 2));
    w.dZ1T = static_cast<__nv_bfloat16*>(take(b * kH * 2));
    w.y = static_cast<float*>(take(b * 4));
    w.dy = static_cast<float*>(take(b * 4));
    w.part = static_cast<float*>(take(b * 4 * 4));
    w.dW1 = static_cast<float*>(take((size_t)kH * np * 4));
    w.colpart = static_cast<float*>(take(((b + kRowChunk - 1) / kRowChunk) * 2 * kH * 4));
}

}  // namespace sa

using namespace sa;

namespace {

struct Scratch {
    void* base = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2tb = nullptr;
    MlpWork w{};
};

// Device buffers of one kernel-level call: BF16 weights and the batch workspace.
cudaError_t scratch_alloc(Scratch& sc, MlpDev& m, int Bp, cudaStream_t s) {
    const size_t wbytes = ((size_t)kH * m.np + 2 * (size_t)kH * kH) * 2;
    const size_t bytes = wbytes + 1024 + mlp_work_bytes(Bp, m.np);
    cudaError_t e = cudaMallocAsync(&sc.base, bytes, s);
    if (e != cudaSuccess) return e;
    char* p = static_cast<char*>(sc.base);
    m.W1b = reinterpret_cast<__nv_bfloat16*>(p);
    m.W2b = m.W1b + (size_t)kH * m.np;
    m.W2tb = m.W2b + (size_t)kH * kH;
    void* rest = reinterpret_cast<void*>(((uintptr_t)(p + wbytes) + 1023) & ~(uintptr_t)1023);
    mlp_work_carve(rest, Bp, m.np, sc.w);
    return cudaSuccess;
}

// The same for inference only: BF16 weights, the packed inputs, the head's partial
// sums and, where the two-GEMM forward pass runs, its hidden activations.
cudaError_t infer_alloc(Scratch& sc, MlpDev& m, int Bp, cudaStream_t s) {
    const size_t wbytes = ((size_t)kH * m.np + 2 * (size_t)kH * kH) * 2;
    const size_t xbytes = (size_t)Bp * m.np * 2, pbytes = (size_t)Bp * 4 * sizeof(float);
    const bool fused = mlp_use_fused(m.np, Bp);
    const size_t abytes = fused ? 0 : (size_t)Bp * kH * 2;
    auto up = [](size_t b) { return (b + 1023) & ~(size_t)1023; };
    cudaError_t e = cudaMallocAsync(&sc.base, up(wbytes) + up(xbytes) + up(pbytes) + abytes, s);
    if (e != cudaSuccess) return e;
    char* p = static_cast<char*>(sc.base);
    m.W1b = reinterpret_cast<__nv_bfloat16*>(p);
    m.W2b = m.W1b + (size_t)kH * m.np;
    m.W2tb = m.W2b + (size_t)kH * kH;
    p += up(wbytes);
    sc.w.Xb = reinterpret_cast<__nv_bfloat16*>(p);
    p += up(xbytes);
    sc.w.part = reinterpret_cast<float*>(p);
    p += up(pbytes);
    sc.w.A1 = abytes ? reinterpret_cast<__nv_bfloat16*>(p) : nullptr;
    return cudaSuccess;
}

sa_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return SA_OK;
    if (e == cudaErrorInvalidValue) { cudaGetLastError(); return SA_EINVAL; }
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return SA_ENOMEM; }
    return SA_ECUDA;
}

}  // namespace

extern "C" {

int64_t sa_mlp_param_count(int32_t n) { return n < 1 ? -1 : mlp_offsets(n).total; }

sa_status sa_mlp_init(float* d_params, int32_t n, uint64_t seed, void* stream) {
    if (!d_params || n < 1 || n > 4096) return SA_EINVAL;
    return to_status(mlp_init(d_params, n, seed, static_cast<cudaStream_t>(stream)));
}

sa_status sa_mlp_forward(const float* d_params, int32_t n, const float* d_X, int32_t B, float* d_y, void* stream) {
    if (!d_params || !d_X || !d_y || n < 1 || n > 4096 || B < 1) return SA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MlpDev m{};
    m.n = n;
    m.np = (n + 63) / 64 * 64;
    m.p = const_cast<float*>(d_params);
    const int Bp = (B + 127) / 128 * 128;
    Scratch sc;
    cudaError_t e = infer_alloc(sc, m, Bp, s);
    if (e != cudaSuccess) return to_status(e);
    int* st = gemm_status_ptr();
    e = mlp_cast(m, s);
    if (e == cudaSuccess) e = mlp_pack(d_X, B, n, Bp, m.np, sc.w.Xb, s);
    if (e == cudaSuccess) e = mlp_infer(m, sc.w.Xb, Bp, sc.w.A1, sc.w.part, st, s);
    if (e == cudaSuccess) e = mlp_finish_y(m, sc.w.part, B, d_y, s);
    cudaFreeAsync(sc.base, s);
    return to_status(e);
}

sa_status sa_mlp_loss_grad(const float* d_params, int32_t n, const float* d_X, const float* d_t, int32_t B,
                           float* d_grad, float* d_loss, void* stream) {
    if (!d_params || !d_X || !d_t || !d_grad || n < 1 || n > 4096 || B < 1) return SA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MlpDev m{};
    m.n = n;
    m.np = (n + 63) / 64 * 64;
    m.p = const_cast<float*>(d_params);
    const int Bp = (B + 127) / 128 * 128;
    Scratch sc;
    cudaError_t e = scratch_alloc(sc, m, Bp, s);
    if (e != cudaSuccess) return to_status(e);
    int* st = gemm_status_ptr();
    e = mlp_cast(m, s);
    if (e == cudaSuccess) e = mlp_pack(d_X, B, n, Bp, m.np, sc.w.Xb, s);
    if (e == cudaSuccess) e = mlp_loss_grad(m, sc.w.Xb, B, Bp, d_t, sc.w, d_grad, d_loss, st, s);
    cudaFreeAsync(sc.base, s);
    return to_status(e);
}

sa_status sa_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t count, int32_t step,
                      float lr, float beta1, float beta2, float eps, void* stream) {
    if (!d_params || !d_grad || !d_m || !d_v || count < 1 || step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return SA_EINVAL;
    return to_status(mlp_adam(d_params, d_grad, d_m, d_v, count, step, lr, beta1, beta2, eps,
                              static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
