// sweep_f32w.cu -- the group-layout FP32 sweep kernel (G lanes per chain; the
// tile code is in sweep_group.cuh).
#include "sweep_group.cuh"

#ifndef SA_F32W_MIN_BLOCKS
#define SA_F32W_MIN_BLOCKS 3  // resident blocks of 256 threads per SM the register budget is sized for
#endif

namespace sa {
namespace {

template <int G, bool CACHE>
__global__ void __launch_bounds__(kGroupMaxBlock, SA_F32W_MIN_BLOCKS) sweep_f32g_kernel(SweepArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ GroupSharedN<kGroupMaxBlock / G> sh;
    const WorkItem it = A.items[blockIdx.x];
    group_tile<G, CACHE>(A, A.probs[it.problem], it, A.run->level, smem_raw, sh);
}

// The instantiated (G, CACHE) layouts.
template <int G, bool CACHE>
cudaError_t launch_g(const SweepArgs& a, int num_items, int block, size_t smem, cudaStream_t s) {
    sweep_f32g_kernel<G, CACHE><<<num_items, block, smem, s>>>(a);
    return cudaGetLastError();
}
template <int G, bool CACHE>
cudaError_t set_smem_g(size_t bytes) {
    static size_t current = 0;  // the limit only grows, so earlier graphs stay valid
    if (bytes <= current) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(sweep_f32g_kernel<G, CACHE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

}  // namespace

bool sweep_f32w_layout_ok(int lanes, bool cache) {
    return (lanes == 32 && cache) || ((lanes == 2 || lanes == 4 || lanes == 8) && !cache) ||
           ((lanes == 4 || lanes == 8) && cache);
}

int sweep_f32w_chains_per_block(int lanes, int block) { return block / lanes; }

// Static shared memory of the layout's kernel (its block scratch).
size_t sweep_f32w_static_bytes(int lanes) {
    switch (lanes) {
    case 2: return sizeof(GroupSharedN<kGroupMaxBlock / 2>);
    case 4: return sizeof(GroupSharedN<kGroupMaxBlock / 4>);
    case 8: return sizeof(GroupSharedN<kGroupMaxBlock / 8>);
    default: return sizeof(GroupSharedN<kGroupMaxBlock / 32>);
    }
}

size_t sweep_f32w_smem_bytes(int n, int lanes, bool cache, int block) {
    const size_t cb = (size_t)(block / lanes);
    return ((cache ? 2 : 1) * cb * (size_t)(n + 1) + 3 * (size_t)n) * sizeof(float);
}

cudaError_t sweep_f32w_set_smem(int lanes, bool cache, size_t bytes) {
    if (lanes == 32) return set_smem_g<32, true>(bytes);
    if (lanes == 8) return cache ? set_smem_g<8, true>(bytes) : set_smem_g<8, false>(bytes);
    if (lanes == 4) return cache ? set_smem_g<4, true>(bytes) : set_smem_g<4, false>(bytes);
    if (lanes == 2 && !cache) return set_smem_g<2, false>(bytes);
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_f32w(const SweepArgs& a, int num_items, int lanes, bool cache, int block, size_t smem,
                              cudaStream_t s) {
    if (block < 32 || block > kGroupMaxBlock || (block & 31) != 0 || !sweep_f32w_layout_ok(lanes, cache))
        return cudaErrorInvalidValue;
    if (lanes == 32) return launch_g<32, true>(a, num_items, block, smem, s);
    if (lanes == 8) return cache ? launch_g<8, true>(a, num_items, block, smem, s) : launch_g<8, false>(a, num_items, block, smem, s);
    if (lanes == 4) return cache ? launch_g<4, true>(a, num_items, block, smem, s) : launch_g<4, false>(a, num_items, block, smem, s);
    return launch_g<2, false>(a, num_items, block, smem, s);
}

}  // namespace sa
