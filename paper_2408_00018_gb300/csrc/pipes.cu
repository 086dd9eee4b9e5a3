// pipes.cu -- measured throughput of the arithmetic pipes a Metropolis step uses.
//
// The sweep's roofline is the minimum over pipes of (the pipe's rate / the
// step's algorithmic operations on it).  Unit counts give nominal rates; this
// file measures them on the GPU at hand: one kernel per operation, every
// thread running eight independent dependency chains of that one operation
// (so the pipe, not the latency, is the limit) at full occupancy, in one
// wave.  The rate is the operations of the whole grid over the launch's time
// (CUDA events); block 0 also reads the SM clock and the global timer at its
// start and end, which gives the clock the SMs ran at, and with it the rate
// per clock per SM.  The operations
// are issued as the PTX instructions the sweep uses (sin/cos/lg2/ex2/sqrt
// approximations on the SFU; 32 x 32 -> 64-bit products, their high and low halves and
// 3-input logic on the integer pipes; FP32 and FP64 fused multiply-adds), and
// a whole Philox4x32-10 block (Salmon et al., SC'11) as the unit of the
// sweep's randomness.  These are rate measurements of documented
// instructions, nothing more.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sa.h"
#include "sa_device.cuh"

namespace sa {
namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;   // independent dependency chains per thread
constexpr int kRepeat = 4;   // operations per chain per loop iteration

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int OP>
__device__ __forceinline__ void op_f(float& x, float b, float c) {
    if (OP == SA_PIPE_SIN) asm("sin.approx.ftz.f32 %0, %0;" : "+f"(x));
    else if (OP == SA_PIPE_COS) asm("cos.approx.ftz.f32 %0, %0;" : "+f"(x));
    else if (OP == SA_PIPE_LG2) asm("lg2.approx.ftz.f32 %0, %0;" : "+f"(x));
    else if (OP == SA_PIPE_EX2) asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x));
    else if (OP == SA_PIPE_SQRT) asm("sqrt.approx.ftz.f32 %0, %0;" : "+f"(x));
    else if (OP == SA_PIPE_RSQRT) asm("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x));
    else asm("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x) : "f"(b), "f"(c));
}

template <int OP>
__device__ __forceinline__ void op_u(uint32_t& x, unsigned long long& acc, uint32_t b, uint32_t c) {
    if (OP == SA_PIPE_IMAD_WIDE) {
        asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(x), "r"(b));
        x = (uint32_t)acc;
    } else if (OP == SA_PIPE_IMAD_HI) {
        asm("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(b), "r"(c));
    } else if (OP == SA_PIPE_IMAD_LO) {
        asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(b), "r"(c));
    } else {  // SA_PIPE_LOP3
        asm("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(b), "r"(c));
    }
}

template <int OP>
__global__ void __launch_bounds__(kThreads) pipe_kernel(int iters, uint32_t seed, long long* cycles, uint32_t* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t out = 0;
    __syncthreads();
    const long long t0 = clock64();
    const unsigned long long g0 = global_ns();
    if (OP == SA_PIPE_SIN || OP == SA_PIPE_COS || OP == SA_PIPE_LG2 || OP == SA_PIPE_EX2 || OP == SA_PIPE_SQRT ||
        OP == SA_PIPE_RSQRT || OP == SA_PIPE_FFMA) {
        float x[kChains];
        const float b = 0.999f + 1e-9f * (float)(seed & 7), c = 1e-3f * (float)(t & 15);
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = 0.5f + 0.01f * (float)j + 1e-6f * (float)(t & 1023);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kRepeat; ++r)
#pragma unroll
                for (int j = 0; j < kChains; ++j) op_f<OP>(x[j], b, c);
        }
#pragma unroll
        for (int j = 0; j < kChains; ++j) out ^= __float_as_uint(x[j]);
    } else if (OP == SA_PIPE_DFMA) {
        double x[kChains];
        const double b = 0.999 + 1e-12 * (double)(seed & 7), c = 1e-3 * (double)(t & 15);
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = 0.5 + 0.01 * j + 1e-9 * (double)(t & 1023);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kRepeat; ++r)
#pragma unroll
                for (int j = 0; j < kChains; ++j) asm("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[j]) : "d"(b), "d"(c));
        }
#pragma unroll
        for (int j = 0; j < kChains; ++j) out ^= (uint32_t)__double_as_longlong(x[j]);
    } else if (OP == SA_PIPE_PHILOX) {
        // two independent blocks per iteration, kRepeat iterations unrolled
        uint32_t a = 0, b2 = 0;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kRepeat; ++r) {
                const uint4 w0 = philox4x32_10(make_uint4((uint32_t)(i * kRepeat + r), 0u, t, 0u), seed, 0x1234u);
                const uint4 w1 = philox4x32_10(make_uint4((uint32_t)(i * kRepeat + r), 1u, t, 0u), seed, 0x1234u);
                a ^= w0.x ^ w0.y ^ w0.z ^ w0.w;
                b2 += w1.x ^ w1.y ^ w1.z ^ w1.w;
            }
        }
        out = a ^ b2;
    } else {
        uint32_t x[kChains];
        unsigned long long acc[kChains];
        const uint32_t b = 0x9E3779B9u ^ seed, c = 0x7F4A7C15u + t;
#pragma unroll
        for (int j = 0; j < kChains; ++j) { x[j] = t * 2654435761u + (uint32_t)j; acc[j] = x[j]; }
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kRepeat; ++r)
#pragma unroll
                for (int j = 0; j < kChains; ++j) op_u<OP>(x[j], acc[j], b, c);
        }
#pragma unroll
        for (int j = 0; j < kChains; ++j) out ^= x[j] ^ (uint32_t)(acc[j] >> 32);
    }
    __syncthreads();
    const long long t1 = clock64();
    const unsigned long long g1 = global_ns();
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // SM cycles and nanoseconds of block 0
        cycles[0] = t1 - t0;
        cycles[1] = (long long)(g1 - g0);
    }
    if (out == 0x5A5A5A5Au && seed == 0xFFFFFFFFu) sink[t] = out;  // keeps the work observable
}

template <int OP>
cudaError_t launch_pipe(int blocks, int iters, uint32_t seed, long long* cycles, uint32_t* sink, cudaStream_t s) {
    pipe_kernel<OP><<<blocks, kThreads, 0, s>>>(iters, seed, cycles, sink);
    return cudaGetLastError();
}

template <int OP>
int occupancy() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pipe_kernel<OP>, kThreads, 0) != cudaSuccess) return 0;
    return b;
}

cudaError_t launch_op(int op, int blocks, int iters, uint32_t seed, long long* cycles, uint32_t* sink, cudaStream_t s) {
    switch (op) {
    case SA_PIPE_SIN: return launch_pipe<SA_PIPE_SIN>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_COS: return launch_pipe<SA_PIPE_COS>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_LG2: return launch_pipe<SA_PIPE_LG2>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_EX2: return launch_pipe<SA_PIPE_EX2>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_SQRT: return launch_pipe<SA_PIPE_SQRT>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_RSQRT: return launch_pipe<SA_PIPE_RSQRT>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_IMAD_WIDE: return launch_pipe<SA_PIPE_IMAD_WIDE>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_IMAD_HI: return launch_pipe<SA_PIPE_IMAD_HI>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_IMAD_LO: return launch_pipe<SA_PIPE_IMAD_LO>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_LOP3: return launch_pipe<SA_PIPE_LOP3>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_FFMA: return launch_pipe<SA_PIPE_FFMA>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_DFMA: return launch_pipe<SA_PIPE_DFMA>(blocks, iters, seed, cycles, sink, s);
    case SA_PIPE_PHILOX: return launch_pipe<SA_PIPE_PHILOX>(blocks, iters, seed, cycles, sink, s);
    default: return cudaErrorInvalidValue;
    }
}

int op_occupancy(int op) {
    switch (op) {
    case SA_PIPE_SIN: return occupancy<SA_PIPE_SIN>();
    case SA_PIPE_COS: return occupancy<SA_PIPE_COS>();
    case SA_PIPE_LG2: return occupancy<SA_PIPE_LG2>();
    case SA_PIPE_EX2: return occupancy<SA_PIPE_EX2>();
    case SA_PIPE_SQRT: return occupancy<SA_PIPE_SQRT>();
    case SA_PIPE_RSQRT: return occupancy<SA_PIPE_RSQRT>();
    case SA_PIPE_IMAD_WIDE: return occupancy<SA_PIPE_IMAD_WIDE>();
    case SA_PIPE_IMAD_HI: return occupancy<SA_PIPE_IMAD_HI>();
    case SA_PIPE_IMAD_LO: return occupancy<SA_PIPE_IMAD_LO>();
    case SA_PIPE_LOP3: return occupancy<SA_PIPE_LOP3>();
    case SA_PIPE_FFMA: return occupancy<SA_PIPE_FFMA>();
    case SA_PIPE_DFMA: return occupancy<SA_PIPE_DFMA>();
    case SA_PIPE_PHILOX: return occupancy<SA_PIPE_PHILOX>();
    default: return 0;
    }
}

// Operations one thread performs per loop iteration.
double ops_per_iter(int op) {
    if (op == SA_PIPE_PHILOX) return 2.0 * kRepeat;           // Philox blocks
    return (double)kChains * kRepeat;
}

}  // namespace
}  // namespace sa

extern "C" sa_status sa_pipe_rate(int32_t op, int32_t iters, void* stream, double* ops_per_clock_per_sm,
                                  double* ops_per_second) {
    if (op < 0 || op >= SA_PIPE_COUNT || iters < 1 || iters > (1 << 20) || !ops_per_clock_per_sm) return SA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SA_ECUDA;
    const int occ = sa::op_occupancy(op);
    if (occ < 1) return SA_ECUDA;
    const int blocks = occ * sms;  // one full wave
    long long* d_cyc = nullptr;
    uint32_t* d_sink = nullptr;
    if (cudaMallocAsync(&d_cyc, sizeof(long long) * 2, s) != cudaSuccess) return SA_ENOMEM;
    if (cudaMallocAsync(&d_sink, sizeof(uint32_t) * blocks * sa::kThreads, s) != cudaSuccess) {
        cudaFreeAsync(d_cyc, s);
        return SA_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sa_status st = SA_OK;
    float ms = 0.0f;
    long long h_cyc[2] = {0, 0};
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        sa::launch_op(op, blocks, iters / 8 + 1, 1u, d_cyc, d_sink, s) != cudaSuccess ||  // warm-up
        cudaEventRecord(e0, s) != cudaSuccess || sa::launch_op(op, blocks, iters, 1u, d_cyc, d_sink, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaMemcpyAsync(h_cyc, d_cyc, sizeof(long long) * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        st = SA_ECUDA;
    if (st == SA_OK) {
        const double per_s = sa::ops_per_iter(op) * iters * sa::kThreads * blocks / (ms * 1e-3);
        const double hz = h_cyc[1] > 0 ? (double)h_cyc[0] / (double)h_cyc[1] * 1e9 : 0.0;  // SM clock of block 0
        *ops_per_clock_per_sm = hz > 0.0 ? per_s / (hz * sms) : 0.0;
        if (ops_per_second) *ops_per_second = per_s;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(d_sink, s);
    cudaFreeAsync(d_cyc, s);
    return st;
}
