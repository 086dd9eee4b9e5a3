// polish.cu -- local minimisers of the hybrid SA, in FP64, one warp per start
// point: box-projected gradient descent with Armijo backtracking, and the
// paper's Nelder-Mead (nm_kernel below).
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
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cooperative_groups.h>
#include <math_constants.h>

#include "appendix.cuh"
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

// Nelder-Mead (the paper's local minimiser, Sec. 4.2 / Table 10) in the standard
// form of Lagarias, Reeds, Wright & Wright (1998): reflection 1, expansion 2,
// contraction 1/2, shrink 1/2, every trial point clipped into the box.  The
// simplex starts at x0 and x0 +- step_frac (u_k - l_k) e_k (minus if plus leaves
// the box); vertices are ranked by (f, slot): best = lowest f then lowest slot,
// worst and second worst = highest f then highest slot.  Stops when the f spread
// is <= ftol max(1, |f_best|) and every vertex lies within xtol (u_i - l_i) of the
// best, or after max_iter iterations.
//
// One block per start, threads over coordinates.  The simplex [(n+1) x n] lives
// in global memory (a vertex per row, so a block reads and writes it coalesced);
// f of the vertices, the vertex sum S, the centroid, the reflected and the trial
// point live in shared memory.  Up to kNmExactN coordinates the centroid of all
// vertices but the worst is summed in slot order every iteration, as written;
// above, it is (S - v_h) / n, with S updated by each replacement and summed
// afresh in slot order after a shrink and every n+1 iterations, so an iteration
// costs O(n) plus its one or two evaluations of f instead of O(n^2).  Rotated
// costs evaluate y_i = sum_j Q_ij x_j per thread from Q^T (coalesced columns).
constexpr int kNmMaxN = 4096;
constexpr int kNmExactN = 64;

// Trial-point coefficients: reflection c + r (c - v_h), expansion c + e (c - v_h),
// outside contraction c + o (c - v_h), inside contraction c - i (c - v_h), shrink
// v_l + s (v - v_l).  Standard: r = 1, e = 2, o = i = s = 1/2; adaptive (Gao & Han):
// e = 1 + 2/n, o = i = 3/4 - 1/(2n), s = 1 - 1/n.
struct NmCoef {
    double r, e, o, i, s;
};

__device__ __forceinline__ double clipd(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

// (f, slot) order: true when (fa, a) ranks below (fb, b)
__device__ __forceinline__ bool rank_less(double fa, int a, double fb, int b) { return fa < fb || (fa == fb && a < b); }

// Sum over the block (every thread gets it): butterflies per warp, then the warps' sums
// in warp order.  red: 32 doubles of shared scratch.
__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();  // red is reused by the next call
    return s;
}

// Product over the block (every thread gets it), like block_sum.
__device__ double block_prod(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(kFull, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double p = 1.0;
    for (int w = 0; w < nw; ++w) p *= red[w];
    __syncthreads();
    return p;
}

struct VecX {
    const double* v;
    __device__ __forceinline__ double operator()(int i) const { return v[i]; }
};

// The Appendix's other tests at x (shared memory): the n-dimensional sums and
// products are reduced over the block; the two-variable and table costs are
// evaluated by thread 0 and shared through block_sum (the others add zeros).
__device__ double bcost_appendix(int cost, int n, const double* x, const double* __restrict__ table, int rows,
                                 double* red) {
    constexpr double pi = CUDART_PI;
    const int t = threadIdx.x, B = blockDim.x;
    if (cost == kCosineMixture || cost == kExponential || cost == kSalomon || cost == kMichalewicz) {
        double a = 0.0, b = 0.0;
        for (int i = t; i < n; i += B) {
            const double v = x[i];
            if (cost == kMichalewicz) {
                a += sin(v) * pow(sin((double)(i + 1) * v * v / pi), 20.0);
            } else {
                a += v * v;
                if (cost == kCosineMixture) b += cos(5.0 * pi * v);
            }
        }
        a = block_sum(a, red);
        if (cost == kCosineMixture) return a - 0.1 * block_sum(b, red);
        if (cost == kExponential) return -exp(-0.5 * a);
        if (cost == kMichalewicz) return -a;
        const double r = sqrt(a);
        return 1.0 - cos(2.0 * pi * r) + 0.1 * r;
    }
    if (cost == kGriewank || cost == kShubert) {
        double q = 0.0, p = 1.0;
        for (int i = t; i < n; i += B) {
            const double v = x[i];
            if (cost == kGriewank) {
                q += v * v;
                p *= cos(v / sqrt((double)(i + 1)));
            } else {
                double s = 0.0;
                for (int j = 1; j <= 5; ++j) s += (double)j * cos((double)(j + 1) * v + (double)j);
                p *= s;
            }
        }
        p = block_prod(p, red);
        if (cost == kShubert) return p;
        return 1.0 + block_sum(q, red) / 4000.0 - p;
    }
    if (cost == kLevyMontalvo) {
        double s = 0.0;
        for (int i = t; i + 1 < n; i += B) {
            const double yi = 1.0 + (x[i] + 1.0) / 4.0, yn = 1.0 + (x[i + 1] + 1.0) / 4.0;
            const double sn = sin(pi * yn);
            s += (yi - 1.0) * (yi - 1.0) * (1.0 + 10.0 * sn * sn);
        }
        s = block_sum(s, red);
        const double y0 = 1.0 + (x[0] + 1.0) / 4.0, yl = 1.0 + (x[n - 1] + 1.0) / 4.0;
        const double s0 = sin(pi * y0);
        return pi / (double)n * (10.0 * s0 * s0 + s + (yl - 1.0) * (yl - 1.0));
    }
    const double v = t == 0 ? appendix_cost_any(cost, n, VecX{x}, table, rows) : 0.0;
    return block_sum(v, red);
}

// f at x (shared memory, visible to the block); every thread gets the value.
__device__ double bcost(int cost, int n, const double* x, const double* __restrict__ QT, const double* __restrict__ table,
                        int rows, double* red) {
    if (cost >= kBranin) return bcost_appendix(cost, n, x, table, rows, red);
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (cost == kRotRastrigin || cost == kRotSchwefel) {
            double y = 0.0;
            for (int j = 0; j < n; ++j) y = fma(QT[(size_t)j * n + i], x[j], y);
            s1 += rot_term(cost, y);
        } else {
            const double t = x[i];
            if (cost == kSchwefel) s1 += h64_schwefel(t);
            else if (cost == kRastrigin) s1 += g64_rastrigin(t);
            else if (cost == kAckley) { s1 += t * t; s2 += cos(6.283185307179586 * t); }
            else if (i + 1 < n) s1 += rosen64(t, x[i + 1]);
        }
    }
    s1 = block_sum(s1, red);
    if (cost == kAckley) s2 = block_sum(s2, red);
    if (cost == kSchwefel) return -(s1 / (double)n);
    if (cost == kRastrigin) return 10.0 * (double)n + s1;
    if (cost == kAckley) return ackley64(n, s1, s2);
    if (cost == kRotRastrigin) return 10.0 * (double)n + s1;
    if (cost == kRotSchwefel) return -(s1 / (double)n);
    return s1;
}

// Lowest (f, slot) of F[0..m) (best = true) or highest (best = false) among the slots
// other than `skip`; (f, slot) is a strict order, so the result does not depend on
// the reduction's order.  fr/jr: 32 doubles / ints of shared scratch.
__device__ int nm_pick(const double* F, int m, bool best, int skip, double* fr, int* jr, double* f_out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double fb = best ? CUDART_INF : -CUDART_INF;
    int jb = best ? m : -1;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        if (j == skip) continue;
        const double f = F[j];
        if (best ? rank_less(f, j, fb, jb) : rank_less(fb, jb, f, j)) { fb = f; jb = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double f = __shfl_xor_sync(kFull, fb, o);
        const int j = __shfl_xor_sync(kFull, jb, o);
        if (best ? rank_less(f, j, fb, jb) : rank_less(fb, jb, f, j)) { fb = f; jb = j; }
    }
    if (lane == 0) { fr[wid] = fb; jr[wid] = jb; }
    __syncthreads();
    for (int w = 0; w < nw; ++w)
        if (best ? rank_less(fr[w], jr[w], fb, jb) : rank_less(fb, jb, fr[w], jr[w])) { fb = fr[w]; jb = jr[w]; }
    __syncthreads();
    *f_out = fb;
    return jb;
}

__global__ void __launch_bounds__(1024) nm_kernel(int cost, int n, const double* __restrict__ lo,
                                                  const double* __restrict__ hi, const double* __restrict__ QT,
                                                  const double* __restrict__ table, int rows,
                                                  const double* __restrict__ x0, double* __restrict__ x_out,
                                                  double* __restrict__ f_out, int* __restrict__ it_out,
                                                  double step_frac, int max_iter, double ftol, double xtol,
                                                  double* __restrict__ ws, NmCoef K) {
    extern __shared__ __align__(16) double nsm[];
    const int t = threadIdx.x, B = blockDim.x, w = blockIdx.x, m = n + 1;
    double* F = nsm;
    double* S = F + m;
    double* xc = S + n;
    double* xr = xc + n;
    double* xt = xr + n;
    double* red = xt + n;                      // 32 doubles
    int* jred = reinterpret_cast<int*>(red + 32);  // 32 ints
    double* V = ws + (size_t)w * (size_t)m * (size_t)n;

    for (int i = t; i < n; i += B) {
        const double v0 = clipd(x0[(size_t)w * n + i], lo[i], hi[i]);
        for (int j = 0; j < m; ++j) {
            double v = v0;
            if (i == j - 1) {
                const double d = step_frac * (hi[i] - lo[i]);
                v = clipd(v + d <= hi[i] ? v + d : v - d, lo[i], hi[i]);
            }
            V[(size_t)j * n + i] = v;
        }
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        for (int i = t; i < n; i += B) xt[i] = V[(size_t)j * n + i];
        __syncthreads();
        const double f = bcost(cost, n, xt, QT, table, rows, red);
        if (t == 0) F[j] = f;
    }
    auto resum = [&]() {
        for (int i = t; i < n; i += B) {
            double a = 0.0;
            for (int j = 0; j < m; ++j) a += V[(size_t)j * n + i];
            S[i] = a;
        }
    };
    resum();
    __syncthreads();

    int it = 0;
    for (; it < max_iter; ++it) {
        double fl, fh, fs;
        const int l = nm_pick(F, m, true, -1, red, jred, &fl);
        const int h = nm_pick(F, m, false, -1, red, jred, &fh);
        const int sw = nm_pick(F, m, false, h, red, jred, &fs);
        if (l >= m || h < 0 || sw < 0) break;  // only if f is NaN at every vertex (never on a finite box)
        if (fh - fl <= ftol * fmax(1.0, fabs(fl))) {
            int small = 1;
            for (int j = 0; j < m; ++j)
                for (int i = t; i < n; i += B)
                    if (fabs(V[(size_t)j * n + i] - V[(size_t)l * n + i]) > xtol * (hi[i] - lo[i])) small = 0;
            if (__syncthreads_and(small)) break;
        }
        const double* vh = V + (size_t)h * n;
        for (int i = t; i < n; i += B) {
            double a;
            if (n <= kNmExactN) {
                a = 0.0;
                for (int j = 0; j < m; ++j)
                    if (j != h) a += V[(size_t)j * n + i];
            } else {
                a = S[i] - vh[i];
            }
            xc[i] = a / (double)n;
            xr[i] = clipd(xc[i] + K.r * (xc[i] - vh[i]), lo[i], hi[i]);
        }
        __syncthreads();
        const double fr = bcost(cost, n, xr, QT, table, rows, red);
        bool accept = false, trial = false;
        double fa = fr;
        if (fr < fl) {  // expansion
            for (int i = t; i < n; i += B) xt[i] = clipd(xc[i] + K.e * (xc[i] - vh[i]), lo[i], hi[i]);
            __syncthreads();
            const double fe = bcost(cost, n, xt, QT, table, rows, red);
            accept = true;
            if (fe < fr) { fa = fe; trial = true; }
        } else if (fr < fs) {
            accept = true;
        } else if (fr < fh) {  // outside contraction
            for (int i = t; i < n; i += B) xt[i] = clipd(xc[i] + K.o * (xc[i] - vh[i]), lo[i], hi[i]);
            __syncthreads();
            const double fo = bcost(cost, n, xt, QT, table, rows, red);
            if (fo <= fr) { accept = true; fa = fo; trial = true; }
        } else {  // inside contraction
            for (int i = t; i < n; i += B) xt[i] = clipd(xc[i] - K.i * (xc[i] - vh[i]), lo[i], hi[i]);
            __syncthreads();
            const double fi = bcost(cost, n, xt, QT, table, rows, red);
            if (fi < fh) { accept = true; fa = fi; trial = true; }
        }
        if (accept) {
            double* dst = V + (size_t)h * n;
            for (int i = t; i < n; i += B) {
                const double a = trial ? xt[i] : xr[i];
                S[i] += a - dst[i];
                dst[i] = a;
            }
            if (t == 0) F[h] = fa;
            __syncthreads();
            if ((it + 1) % m == 0) resum();  // bound the drift of the running sum
        } else {  // shrink towards the best vertex
            const double* vl = V + (size_t)l * n;
            for (int j = 0; j < m; ++j) {
                if (j == l) continue;
                double* v = V + (size_t)j * n;
                for (int i = t; i < n; i += B) {
                    const double a = clipd(vl[i] + K.s * (v[i] - vl[i]), lo[i], hi[i]);
                    v[i] = a;
                    xt[i] = a;
                }
                __syncthreads();
                const double f = bcost(cost, n, xt, QT, table, rows, red);
                if (t == 0) F[j] = f;
            }
            resum();
        }
        __syncthreads();
    }
    double fl;
    int l = nm_pick(F, m, true, -1, red, jred, &fl);
    if (l >= m) l = 0;
    for (int i = t; i < n; i += B) x_out[(size_t)w * n + i] = V[(size_t)l * n + i];
    if (t == 0) {
        f_out[w] = fl;
        if (it_out) it_out[w] = it;
    }
}

// ---- Nelder-Mead on a thread-block cluster (separable costs, many coordinates) ----
//
// The same method and order of operations as nm_kernel (above), for costs that
// are sums or products of one-coordinate terms.  One start runs on a cluster of
// G CTAs (G <= 8, one SM each, so G times the FP64 rate of one SM): CTA r owns the
// coordinates [r c, (r + 1) c), c = ceil(n / G), of every vertex and of the
// centroid, reflected and trial points, and keeps its own replica of the vertex
// values F.  An evaluation of f forms each CTA's partial sum (or product) over its
// coordinates, writes it into slot r of every CTA's exchange buffer through
// distributed shared memory, and crosses one cluster barrier; every CTA then
// combines the G partials in rank order, so all of them hold the same f bit for
// bit and take the same decisions.  The exchange buffer alternates between two
// halves, so a CTA that is one evaluation ahead never overwrites a partial a
// slower CTA has still to read (it cannot pass the next barrier before them).
namespace cg = cooperative_groups;

constexpr int kNmClusterMax = 8;

__device__ __forceinline__ bool nm_separable(int cost) {
    return cost == kSchwefel || cost == kRastrigin || cost == kAckley || cost == kCosineMixture ||
           cost == kExponential || cost == kMichalewicz || cost == kSalomon || cost == kGriewank || cost == kShubert;
}
__device__ __forceinline__ bool nm_second_is_product(int cost) { return cost == kGriewank || cost == kShubert; }

// One coordinate's contribution to the cost's two running quantities (a: a sum;
// b: a second sum, or a product for Griewank and Shubert).
__device__ __forceinline__ void nm_term(int cost, int i, double x, double& a, double& b) {
    constexpr double pi = CUDART_PI;
    switch (cost) {
    case kSchwefel: a += h64_schwefel(x); break;
    case kRastrigin: a += g64_rastrigin(x); break;
    case kAckley: a += x * x; b += cos(6.283185307179586 * x); break;
    case kCosineMixture: a += x * x; b += cos(5.0 * pi * x); break;
    case kExponential: case kSalomon: a += x * x; break;
    case kMichalewicz: a += sin(x) * pow(sin((double)(i + 1) * x * x / pi), 20.0); break;
    case kGriewank: a += x * x; b *= cos(x / sqrt((double)(i + 1))); break;
    default: {  // kShubert
        double s = 0.0;
        for (int j = 1; j <= 5; ++j) s += (double)j * cos((double)(j + 1) * x + (double)j);
        b *= s;
    }
    }
}

__device__ __forceinline__ double nm_finish(int cost, int n, double a, double b) {
    constexpr double pi = CUDART_PI;
    switch (cost) {
    case kSchwefel: return -(a / (double)n);
    case kRastrigin: return 10.0 * (double)n + a;
    case kAckley: return ackley64(n, a, b);
    case kCosineMixture: return a - 0.1 * b;
    case kExponential: return -exp(-0.5 * a);
    case kMichalewicz: return -a;
    case kSalomon: { const double r = sqrt(a); return 1.0 - cos(2.0 * pi * r) + 0.1 * r; }
    case kGriewank: return 1.0 + a / 4000.0 - b;
    default: return b;  // kShubert
    }
}

// The cluster-wide pair (sum of a, sum or product of b) of every CTA's (a, b);
// pbuf: 2 halves x kNmClusterMax slots x 2 doubles of shared memory; half: the
// half this exchange uses (alternates).
__device__ void nm_cluster_reduce(cg::cluster_group& cl, int G, bool prod, double a, double b, double* pbuf,
                                  int& half, double& A, double& Bv) {
    double* mine = pbuf + half * 2 * kNmClusterMax;
    if (threadIdx.x == 0) {
        const int r = (int)cl.block_rank();
        for (int q = 0; q < G; ++q) {
            double* dst = cl.map_shared_rank(mine, q);
            dst[2 * r] = a;
            dst[2 * r + 1] = b;
        }
    }
    cl.sync();
    A = 0.0;
    Bv = prod ? 1.0 : 0.0;
    for (int q = 0; q < G; ++q) {
        A += mine[2 * q];
        Bv = prod ? Bv * mine[2 * q + 1] : Bv + mine[2 * q + 1];
    }
    half ^= 1;
}

// f at the point whose slice [i0, i0 + cnt) this CTA holds in xs (shared memory).
__device__ double nm_cluster_cost(cg::cluster_group& cl, int G, int cost, int n, const double* xs, int i0, int cnt,
                                  double* red, double* pbuf, int& half) {
    const bool prod = nm_second_is_product(cost);
    double a = 0.0, b = prod ? 1.0 : 0.0;
    for (int li = threadIdx.x; li < cnt; li += blockDim.x) nm_term(cost, i0 + li, xs[li], a, b);
    a = block_sum(a, red);
    b = prod ? block_prod(b, red) : block_sum(b, red);
    double A, Bv;
    nm_cluster_reduce(cl, G, prod, a, b, pbuf, half, A, Bv);
    return nm_finish(cost, n, A, Bv);
}

__global__ void __launch_bounds__(256, 1) nm_cluster_kernel(int cost, int n, const double* __restrict__ lo,
                                                         const double* __restrict__ hi, const double* __restrict__ x0,
                                                         double* __restrict__ x_out, double* __restrict__ f_out,
                                                         int* __restrict__ it_out, double step_frac, int max_iter,
                                                         double ftol, double xtol, double* __restrict__ ws, int G,
                                                         NmCoef K) {
    extern __shared__ __align__(16) double csm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int w = blockIdx.x / G;  // the start this cluster runs
    const int t = threadIdx.x, B = blockDim.x, m = n + 1;
    const int chunk = (n + G - 1) / G;
    const int i0 = rank * chunk;
    const int cnt = max(0, min(n, i0 + chunk) - i0);
    double* F = csm;
    double* S = F + m;
    double* xc = S + chunk;
    double* xr = xc + chunk;
    double* xt = xr + chunk;
    double* pbuf = xt + chunk;                 // 2 x kNmClusterMax x 2
    double* red = pbuf + 4 * kNmClusterMax;   // 32 doubles
    int* jred = reinterpret_cast<int*>(red + 32);
    double* V = ws + (size_t)w * (size_t)m * (size_t)n;
    int half = 0;

    for (int li = t; li < cnt; li += B) {
        const int i = i0 + li;
        const double v0 = clipd(x0[(size_t)w * n + i], lo[i], hi[i]);
        for (int j = 0; j < m; ++j) {
            double v = v0;
            if (i == j - 1) {
                const double d = step_frac * (hi[i] - lo[i]);
                v = clipd(v + d <= hi[i] ? v + d : v - d, lo[i], hi[i]);
            }
            V[(size_t)j * n + i] = v;
        }
    }
    for (int j = 0; j < m; ++j) {
        for (int li = t; li < cnt; li += B) xt[li] = V[(size_t)j * n + i0 + li];
        __syncthreads();
        const double f = nm_cluster_cost(cl, G, cost, n, xt, i0, cnt, red, pbuf, half);
        if (t == 0) F[j] = f;
    }
    auto resum = [&]() {
        for (int li = t; li < cnt; li += B) {
            double a = 0.0;
            for (int j = 0; j < m; ++j) a += V[(size_t)j * n + i0 + li];
            S[li] = a;
        }
    };
    resum();
    __syncthreads();

    int it = 0;
    for (; it < max_iter; ++it) {
        double fl, fh, fs;
        const int l = nm_pick(F, m, true, -1, red, jred, &fl);
        const int h = nm_pick(F, m, false, -1, red, jred, &fh);
        const int sw = nm_pick(F, m, false, h, red, jred, &fs);
        if (l >= m || h < 0 || sw < 0) break;  // only if f is NaN at every vertex
        if (fh - fl <= ftol * fmax(1.0, fabs(fl))) {
            double big = 0.0;
            for (int j = 0; j < m; ++j)
                for (int li = t; li < cnt; li += B) {
                    const int i = i0 + li;
                    if (fabs(V[(size_t)j * n + i] - V[(size_t)l * n + i]) > xtol * (hi[i] - lo[i])) big = 1.0;
                }
            big = block_sum(big, red);
            double A, Bv;
            nm_cluster_reduce(cl, G, false, big, 0.0, pbuf, half, A, Bv);
            if (A == 0.0) break;
        }
        const double* vh = V + (size_t)h * n + i0;
        for (int li = t; li < cnt; li += B) {
            xc[li] = (S[li] - vh[li]) / (double)n;
            const int i = i0 + li;
            xr[li] = clipd(xc[li] + K.r * (xc[li] - vh[li]), lo[i], hi[i]);
        }
        __syncthreads();
        const double fr = nm_cluster_cost(cl, G, cost, n, xr, i0, cnt, red, pbuf, half);
        bool accept = false, trial = false;
        double fa = fr;
        if (fr < fl) {  // expansion
            for (int li = t; li < cnt; li += B) xt[li] = clipd(xc[li] + K.e * (xc[li] - vh[li]), lo[i0 + li], hi[i0 + li]);
            __syncthreads();
            const double fe = nm_cluster_cost(cl, G, cost, n, xt, i0, cnt, red, pbuf, half);
            accept = true;
            if (fe < fr) { fa = fe; trial = true; }
        } else if (fr < fs) {
            accept = true;
        } else if (fr < fh) {  // outside contraction
            for (int li = t; li < cnt; li += B) xt[li] = clipd(xc[li] + K.o * (xc[li] - vh[li]), lo[i0 + li], hi[i0 + li]);
            __syncthreads();
            const double fo = nm_cluster_cost(cl, G, cost, n, xt, i0, cnt, red, pbuf, half);
            if (fo <= fr) { accept = true; fa = fo; trial = true; }
        } else {  // inside contraction
            for (int li = t; li < cnt; li += B) xt[li] = clipd(xc[li] - K.i * (xc[li] - vh[li]), lo[i0 + li], hi[i0 + li]);
            __syncthreads();
            const double fi = nm_cluster_cost(cl, G, cost, n, xt, i0, cnt, red, pbuf, half);
            if (fi < fh) { accept = true; fa = fi; trial = true; }
        }
        if (accept) {
            double* dst = V + (size_t)h * n + i0;
            for (int li = t; li < cnt; li += B) {
                const double a = trial ? xt[li] : xr[li];
                S[li] += a - dst[li];
                dst[li] = a;
            }
            if (t == 0) F[h] = fa;
            __syncthreads();
            if ((it + 1) % m == 0) resum();
        } else {  // shrink towards the best vertex
            const double* vl = V + (size_t)l * n + i0;
            for (int j = 0; j < m; ++j) {
                if (j == l) continue;
                double* v = V + (size_t)j * n + i0;
                for (int li = t; li < cnt; li += B) {
                    const double a = clipd(vl[li] + K.s * (v[li] - vl[li]), lo[i0 + li], hi[i0 + li]);
                    v[li] = a;
                    xt[li] = a;
                }
                __syncthreads();
                const double f = nm_cluster_cost(cl, G, cost, n, xt, i0, cnt, red, pbuf, half);
                if (t == 0) F[j] = f;
            }
            resum();
        }
        __syncthreads();
    }
    double fl;
    int l = nm_pick(F, m, true, -1, red, jred, &fl);
    if (l >= m) l = 0;
    for (int li = t; li < cnt; li += B) x_out[(size_t)w * n + i0 + li] = V[(size_t)l * n + i0 + li];
    if (rank == 0 && t == 0) {
        f_out[w] = fl;
        if (it_out) it_out[w] = it;
    }
    cl.sync();  // no CTA leaves while a peer may still address its shared memory
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

size_t nm_ws_doubles(int n) { return (size_t)(n + 1) * (size_t)n; }

int nm_max_n() { return kNmMaxN; }

// Costs of one-coordinate terms with at least 128 coordinates run on a cluster of
// G = min(8, n / 64) CTAs (rounded down to a power of two).
static int nm_cluster_size(int cost, int n) {
    const bool sep = cost == kSchwefel || cost == kRastrigin || cost == kAckley || cost == kCosineMixture ||
                     cost == kExponential || cost == kMichalewicz || cost == kSalomon || cost == kGriewank ||
                     cost == kShubert;
    if (!sep || n < 128) return 1;
    int G = 2;
    while (G * 2 <= kNmClusterMax && G * 2 * 64 <= n) G *= 2;
    return G;
}

cudaError_t launch_nm(int cost, int n, const double* lo, const double* hi, const double* QT, const double* table,
                      int table_rows, int k, const double* x0, double* x_out, double* f_out, int* it_out,
                      double step_frac, int max_iter, double ftol, double xtol, bool adaptive, double* ws,
                      cudaStream_t s) {
    if (n < 1 || n > kNmMaxN) return cudaErrorInvalidValue;
    NmCoef K;
    const double dn = (double)n;
    K.r = 1.0;
    K.e = adaptive ? 1.0 + 2.0 / dn : 2.0;
    K.o = adaptive ? 0.75 - 1.0 / (2.0 * dn) : 0.5;
    K.i = K.o;
    K.s = adaptive ? 1.0 - 1.0 / dn : 0.5;
    const int G = nm_cluster_size(cost, n);
    if (G > 1) {
        const int chunk = (n + G - 1) / G;
        const int block = std::min(256, std::max(32, (chunk + 31) / 32 * 32));
        const size_t smem = ((size_t)(n + 1) + 4 * (size_t)chunk + 4 * kNmClusterMax + 32) * sizeof(double) +
                            32 * sizeof(int);
        static size_t current_c = 0;  // the limit only grows
        if (smem > current_c) {
            const cudaError_t e =
                cudaFuncSetAttribute(nm_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            current_c = smem;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(k * G));
        cfg.blockDim = dim3((unsigned)block);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)G;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, nm_cluster_kernel, cost, n, lo, hi, x0, x_out, f_out, it_out, step_frac,
                                  max_iter, ftol, xtol, ws, G, K);
    }
    const int block = std::min(1024, std::max(32, (n + 31) / 32 * 32));
    const size_t smem = ((size_t)(n + 1) + 4 * (size_t)n + 32) * sizeof(double) + 32 * sizeof(int);
    static size_t current = 0;  // the limit only grows
    if (smem > current) {
        const cudaError_t e = cudaFuncSetAttribute(nm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        current = smem;
    }
    nm_kernel<<<k, block, smem, s>>>(cost, n, lo, hi, QT, table, table_rows, x0, x_out, f_out, it_out, step_frac,
                                     max_iter, ftol, xtol, ws, K);
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
