// argmin_static.cu -- the argmin of sa_argmin_f64 for callers that cannot
// allocate device memory.
//
// sa_argmin_f64 asks its caller for a scratch buffer (one 16-byte partial
// minimum per 2048 inputs).  Some callers cannot provide one: code running
// inside a host framework whose allocator owns the device's memory, code that
// must not call cudaMalloc because it implicitly synchronises the device (a
// latency-critical loop), or code that must never fail for lack of memory
// half-way through a run.  For them this file keeps the scratch in a
// file-scope device array of fixed size, so the call allocates nothing.
//
// The array lives in every GPU that loads this library, until the process
// exits.  All calls share it: two calls whose kernels overlap on the GPU (on
// different streams, or from different host threads without ordering) race
// on it and may return wrong results.  Nothing in it has to start at zero:
// each call writes every partial it reads.
//
// The device address of the array is looked up once per device and kept for
// the life of the process.  cudaDeviceReset destroys the array with the
// context, so a process that resets a device must not call this entry point
// on that device again (start a new process instead).
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/sa.h"
#include "sa_internal.h"

namespace sa {
cudaError_t launch_argmin_f64(const double* F, int64_t count, int64_t* idx, double* val, void* scratch, cudaStream_t s);
int64_t argmin_num_parts(int64_t count);
}  // namespace sa

namespace {

constexpr int64_t kMaxCount = SA_ARGMIN_STATIC_MAX_COUNT;
constexpr int64_t kPartBytes = 16;  // one (double value, int64 index) partial
// inputs reduced into one partial by launch_argmin_f64 (one block of its first pass)
constexpr int64_t kSpan = (int64_t)sa::kArgminThreads * sa::kArgminPerThread;
constexpr int64_t kMaxParts = (kMaxCount + kSpan - 1) / kSpan;

// The shared scratch.  In host code this name is only a stand-in for the
// device symbol, never a device address: the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_argmin_scratch[kMaxParts * kPartBytes];
static_assert(kMaxParts * kPartBytes == sizeof(g_argmin_scratch), "scratch holds every partial of the largest count");
static_assert(kMaxParts * kPartBytes == ((int64_t)1 << 20), "the documented size of the scratch is 1 MiB");

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_argmin_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sa_status sa_argmin_f64_static(const double* d_F, int64_t count, int64_t* d_index, double* d_value,
                                          void* stream) {
    if (count < 1 || !d_F || !d_index || !d_value) return SA_EINVAL;
    if (count > kMaxCount) return SA_EINVAL;
    // the partials launch_argmin_f64 writes for this count must fit the array
    if (sa::argmin_num_parts(count) * kPartBytes > (int64_t)sizeof(g_argmin_scratch)) return SA_EINVAL;
    void* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return SA_ECUDA;
    return sa::launch_argmin_f64(d_F, count, d_index, d_value, scratch, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SA_OK : SA_ECUDA;
}
