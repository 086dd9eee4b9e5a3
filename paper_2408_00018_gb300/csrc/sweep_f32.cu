// sweep_f32.cu -- Metropolis sweep of one temperature level, FP32 state, one
// Markov chain per thread (the tile code is in sweep_thread.cuh).
#include "sweep_thread.cuh"

namespace sa {
namespace {

__global__ void __launch_bounds__(kMaxBlock, 1) sweep_f32_kernel(SweepArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const WorkItem it = A.items[blockIdx.x];
    const ProbDev& P = A.probs[it.problem];
    const int level = A.run->level;
    const int n = P.n, B = blockDim.x, S = B;
    double* red = reinterpret_cast<double*>(smem_raw);                    // 72 doubles
    int* cand = reinterpret_cast<int*>(smem_raw + 72 * sizeof(double));  // B ints
    int* ncand = cand + kMaxBlock;
    float* xs = reinterpret_cast<float*>(smem_raw + 72 * sizeof(double) + (kMaxBlock + 4) * sizeof(int));
    float* slo = xs + (size_t)n * B;
    float* shi = slo + n;
    float* ssig = shi + n;
    switch (P.cost) {
    case kSchwefel: dispatch_u<kSchwefel>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand); break;
    case kRastrigin: dispatch_u<kRastrigin>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand); break;
    case kAckley: dispatch_u<kAckley>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand); break;
    case kRosenbrock: dispatch_u<kRosenbrock>(A, P, it, S, level, xs, slo, shi, ssig, red, cand, ncand); break;
    default: if (threadIdx.x == 0) A.run->status = 1; break;
    }
}

}  // namespace

size_t sweep_f32_smem_bytes(int n, int block) {
    return 72 * sizeof(double) + (kMaxBlock + 4) * sizeof(int) + ((size_t)n * block + 3 * (size_t)n) * sizeof(float);
}

cudaError_t sweep_f32_set_smem(size_t bytes) {
    // The limit only grows, so a later handle never invalidates an earlier handle's graphs.
    static size_t current = 0;
    if (bytes <= current) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(sweep_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

cudaError_t launch_sweep_f32(const SweepArgs& a, int num_items, int block, size_t smem, cudaStream_t s) {
    if (block > kMaxBlock) return cudaErrorInvalidValue;
    sweep_f32_kernel<<<num_items, block, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sa
