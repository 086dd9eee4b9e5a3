// sweep_f64.cu -- Metropolis sweep of one temperature level, FP64 state.
//
// The kernel of Listing 4 in double precision: one thread per chain, state in
// shared memory x[d][lane], and -- as in the paper -- f(x1) recomputed in full
// at every step, summed in index order.  It serves every cost, including the
// Appendix's Tests 2-12 and 15-19 (appendix.cuh).  This translation unit is compiled
// with -fmad=false: every product and sum is rounded as written, so the only
// differences from a correctly rounded evaluation are the last-ulp errors of
// the math library's log, cos, sin and exp.
#include <cmath>
#include <math_constants.h>

#include "appendix.cuh"
#include "sa_device.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kMaxBlock = 256;

// Coordinate i of the chain's column, with coordinate d replaced by xd (d < 0: none).
struct ColX {
    const double* col;
    int B, d;
    double xd;
    __device__ __forceinline__ double operator()(int i) const { return i == d ? xd : col[(size_t)i * B]; }
};

// f at the chain's column, with coordinate d replaced by xd_new (d < 0: none).
template <int COST>
__device__ __forceinline__ double full_cost(const ProbDev& P, const double* xcol, int B, int n, int d, double xd_new) {
    if (COST >= kBranin) {
        return appendix_cost<COST>(n, ColX{xcol, B, d, xd_new}, P.table, P.table_rows);
    } else if (COST == kSchwefel) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = s + h64_schwefel(i == d ? xd_new : xcol[i * B]);
        return -(s / (double)n);
    } else if (COST == kRastrigin) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = s + g64_rastrigin(i == d ? xd_new : xcol[i * B]);
        return 10.0 * (double)n + s;
    } else if (COST == kAckley) {
        double s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < n; ++i) {
            const double x = i == d ? xd_new : xcol[i * B];
            s1 = s1 + x * x;
            s2 = s2 + cos(6.283185307179586 * x);
        }
        return ackley64(n, s1, s2);
    } else {
        double s = 0.0;
        for (int i = 0; i + 1 < n; ++i)
            s = s + rosen64(i == d ? xd_new : xcol[i * B], (i + 1) == d ? xd_new : xcol[(i + 1) * B]);
        return s;
    }
}

// Griewank's and Michalewicz's per-coordinate factors (cos(x_i / sqrt i) and
// sin(x_i) sin(i x_i^2 / pi)^20): each chain keeps them beside its state, so a
// step evaluates one new factor and redoes the sum and the product in index
// order from the kept ones -- the same operations on the same values as the
// full evaluation, at a fraction of its transcendental work.
template <int COST>
constexpr bool kKeepsTerms = COST == kGriewank || COST == kMichalewicz;

template <int COST>
__device__ __forceinline__ double term64(int i, double t) {
    if (COST == kGriewank) return cos(t / sqrt((double)(i + 1)));
    return sin(t) * pow(sin((double)(i + 1) * t * t / CUDART_PI), 20.0);
}

// f from the kept factors, with coordinate d's value and factor replaced (d < 0: none).
template <int COST>
__device__ __forceinline__ double kept_cost(const double* xcol, const double* tcol, int B, int n, int d, double xd,
                                            double td) {
    if (COST == kGriewank) {
        double q = 0.0, p = 1.0;
        for (int i = 0; i < n; ++i) {
            const double v = i == d ? xd : xcol[i * B];
            q += v * v;
            p *= i == d ? td : tcol[i * B];
        }
        return 1.0 + q / 4000.0 - p;
    }
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += i == d ? td : tcol[i * B];
    return -s;
}

template <int COST>
__device__ void sweep_tile(const SweepArgs& A, const ProbDev& P, const WorkItem& it, int level, double* xs,
                           unsigned long long* red) {
    const int t = threadIdx.x, B = blockDim.x, n = P.n;
    const bool active = t < it.count;
    const int64_t c = it.c0 + t;
    const int64_t gc = P.chain_base + c;
    const double T = A.T_tab[level];
    const double sl = A.s_tab[level];
    double* xcol = xs + t;

    if (level == 0) {
        if (active) {
            for (int k = 0; k < n; k += 4) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)(k >> 2), 0u, (uint32_t)c + P.cid0, P.pid), A.ikey0, A.ikey1);
                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (k + j < n) xcol[(k + j) * B] = P.lo[k + j] + u23d(ww[j]) * (P.hi[k + j] - P.lo[k + j]);
            }
        }
    } else if (own_start(A, level)) {  // the chain's own state (no exchange before this level)
        if (active)
            for (int k = 0; k < n; ++k) xcol[k * B] = A.X64[P.x_base + (size_t)k * (size_t)P.chains + (size_t)c];
    } else {
        for (int k = 0; k < n; ++k) xcol[k * B] = P.x_best64[k];
    }

    const bool tracing = (A.bits != nullptr) && level < A.trace_levels;
    uint32_t* mybits = tracing ? A.bits + ((size_t)level * (size_t)A.total_chains + (size_t)gc) * (size_t)A.words : nullptr;
    uint32_t nacc = 0;
    double* tcol = xs + (size_t)n * B + t;  // kept factors (kKeepsTerms costs only)
    if (active) {
        double F;
        if (kKeepsTerms<COST>) {
            for (int k = 0; k < n; ++k) tcol[k * B] = term64<COST>(k, xcol[k * B]);
            F = kept_cost<COST>(xcol, tcol, B, n, -1, 0.0, 0.0);
        } else {
            F = full_cost<COST>(P, xcol, B, n, -1, 0.0);
        }
        uint32_t bw = 0;
        for (int s = 0; s < A.L; ++s) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)level, (uint32_t)c + P.cid0, P.pid), A.key0, A.key1);
            const int d = coord_of(w.x, n);
            const double u1 = u23d(w.y), u2 = u23d(w.z), u3 = u23d(w.w);
            const double xd = xcol[d * B];
            const double lo = P.lo[d], hi = P.hi[d];
            double xp;
            if (A.proposal == 1) {  // uniform redraw of the coordinate
                xp = lo + u2 * (hi - lo);
            } else {
                const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
                xp = xd + P.sig[d] * sl * z;
            }
            if (A.boundary == 0) {
                if (xp < lo) xp = 2.0 * lo - xp;
                else if (xp > hi) xp = 2.0 * hi - xp;
            }
            if (xp < lo) xp = lo;
            if (xp > hi) xp = hi;
            double td = 0.0, Fp;
            if (kKeepsTerms<COST>) {
                td = term64<COST>(d, xp);
                Fp = kept_cost<COST>(xcol, tcol, B, n, d, xp, td);
            } else {
                Fp = full_cost<COST>(P, xcol, B, n, d, xp);
            }
            const double dF = Fp - F;
            const bool acc = (dF <= 0.0) || (u3 < exp(-dF / T));
            if (acc) {
                xcol[d * B] = xp;
                if (kKeepsTerms<COST>) tcol[d * B] = td;
                F = Fp;
                ++nacc;
            }
            if (tracing) {
                bw |= (acc ? 1u : 0u) << (s & 31);
                if ((s & 31) == 31 || s == A.L - 1) { mybits[s >> 5] = bw; bw = 0; }
            }
        }
        A.F[gc] = isfinite(F) ? F : CUDART_NAN;
        double* dst = A.X64 + P.x_base + c;
        for (int k = 0; k < n; ++k) dst[(size_t)k * (size_t)P.chains] = xcol[k * B];
    }
    // accepted-move count of the tile
    unsigned long long a = nacc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((t & 31) == 0) red[t >> 5] = a;
    __syncthreads();
    if (t == 0) {
        unsigned long long sum = 0;
        for (int i = 0; i < (B + 31) / 32; ++i) sum += red[i];
        atomicAdd(P.accepts, sum);
    }
}

__global__ void __launch_bounds__(kMaxBlock) sweep_f64_kernel(SweepArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const WorkItem it = A.items[blockIdx.x];
    const ProbDev P = A.probs[it.problem];
    const int level = A.run->level;
    unsigned long long* red = reinterpret_cast<unsigned long long*>(smem_raw);
    double* xs = reinterpret_cast<double*>(smem_raw + 32 * sizeof(unsigned long long));
    switch (P.cost) {
    case kSchwefel: sweep_tile<kSchwefel>(A, P, it, level, xs, red); break;
    case kRastrigin: sweep_tile<kRastrigin>(A, P, it, level, xs, red); break;
    case kAckley: sweep_tile<kAckley>(A, P, it, level, xs, red); break;
    case kRosenbrock: sweep_tile<kRosenbrock>(A, P, it, level, xs, red); break;
    case kBranin: sweep_tile<kBranin>(A, P, it, level, xs, red); break;
    case kCosineMixture: sweep_tile<kCosineMixture>(A, P, it, level, xs, red); break;
    case kDekkersAarts: sweep_tile<kDekkersAarts>(A, P, it, level, xs, red); break;
    case kEasom: sweep_tile<kEasom>(A, P, it, level, xs, red); break;
    case kExponential: sweep_tile<kExponential>(A, P, it, level, xs, red); break;
    case kGoldsteinPrice: sweep_tile<kGoldsteinPrice>(A, P, it, level, xs, red); break;
    case kGriewank: sweep_tile<kGriewank>(A, P, it, level, xs, red); break;
    case kHimmelblau: sweep_tile<kHimmelblau>(A, P, it, level, xs, red); break;
    case kLevyMontalvo: sweep_tile<kLevyMontalvo>(A, P, it, level, xs, red); break;
    case kLangerman: sweep_tile<kLangerman>(A, P, it, level, xs, red); break;
    case kMichalewicz: sweep_tile<kMichalewicz>(A, P, it, level, xs, red); break;
    case kSalomon: sweep_tile<kSalomon>(A, P, it, level, xs, red); break;
    case kSixHumpCamel: sweep_tile<kSixHumpCamel>(A, P, it, level, xs, red); break;
    case kShubert: sweep_tile<kShubert>(A, P, it, level, xs, red); break;
    case kShekel: sweep_tile<kShekel>(A, P, it, level, xs, red); break;
    case kFoxholes: sweep_tile<kFoxholes>(A, P, it, level, xs, red); break;
    default: if (threadIdx.x == 0) A.run->status = 1; break;
    }
}

}  // namespace

size_t sweep_f64_smem_bytes(int n, int block, bool keeps_terms) {
    return 32 * sizeof(unsigned long long) + (size_t)n * block * sizeof(double) * (keeps_terms ? 2 : 1);
}

bool sweep_f64_keeps_terms(int cost) { return cost == kGriewank || cost == kMichalewicz; }

cudaError_t sweep_f64_set_smem(size_t bytes) {
    // The limit only grows, so a later handle never invalidates an earlier handle's graphs.
    static size_t current = 0;
    if (bytes <= current) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(sweep_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) current = bytes;
    return e;
}

cudaError_t launch_sweep_f64(const SweepArgs& a, int num_items, int block, size_t smem, cudaStream_t s) {
    if (block > kMaxBlock) return cudaErrorInvalidValue;
    sweep_f64_kernel<<<num_items, block, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sa
