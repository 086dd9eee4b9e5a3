// appendix.cuh -- the paper's other Appendix test functions in FP64 (Tests 2-12
// and 15-19), evaluated in full from an accessor x(i), i = 0 .. n-1 (the
// paper's x_1 is x(0)).  Sums and products run in index order.  Tests 11, 18
// and 19 read a table of rows (a_i1 .. a_in, c_i), rows x (n + 1) doubles.
//
// Two formulas are taken in their standard form where the printed one is
// garbled: the cosine mixture as sum x_i^2 - 0.1 sum cos(5 pi x_i) (the printed
// signs put the minimum at the corners, against the printed f* = -0.1 n at 0)
// and Griewank with its product outside the sum.
#pragma once
#include <cmath>
#include <math_constants.h>

#include "sa_device.cuh"

namespace sa {

__device__ __forceinline__ bool is_appendix(int cost) { return cost >= kBranin && cost <= kFoxholes; }

template <int COST, class X>
__device__ __forceinline__ double appendix_cost(int n, const X& x, const double* __restrict__ table, int rows) {
    constexpr double pi = CUDART_PI;
    if (COST == kBranin) {  // Test 2
        const double a = x(1) - 5.1 * x(0) * x(0) / (4.0 * pi * pi) + 5.0 * x(0) / pi - 6.0;
        return a * a + 10.0 * (1.0 - 1.0 / (8.0 * pi)) * cos(x(0)) + 10.0;
    } else if (COST == kCosineMixture) {  // Test 3
        double c = 0.0, q = 0.0;
        for (int i = 0; i < n; ++i) {
            const double t = x(i);
            c += cos(5.0 * pi * t);
            q += t * t;
        }
        return q - 0.1 * c;
    } else if (COST == kDekkersAarts) {  // Test 4
        const double a = x(0) * x(0), b = x(1) * x(1), r = a + b;
        return 1e5 * a + b - r * r + 1e-5 * (r * r) * (r * r);
    } else if (COST == kEasom) {  // Test 5
        const double u = x(0) - pi, v = x(1) - pi;
        return -cos(x(0)) * cos(x(1)) * exp(-u * u - v * v);
    } else if (COST == kExponential) {  // Test 6
        double q = 0.0;
        for (int i = 0; i < n; ++i) q += x(i) * x(i);
        return -exp(-0.5 * q);
    } else if (COST == kGoldsteinPrice) {  // Test 7
        const double a = x(0), b = x(1);
        const double s = a + b + 1.0, t = 2.0 * a - 3.0 * b;
        const double p = 1.0 + s * s * (19.0 - 14.0 * a + 3.0 * a * a - 14.0 * b + 6.0 * a * b + 3.0 * b * b);
        const double q = 30.0 + t * t * (18.0 - 32.0 * a + 12.0 * a * a + 48.0 * b - 36.0 * a * b + 27.0 * b * b);
        return p * q;
    } else if (COST == kGriewank) {  // Test 8
        double q = 0.0, p = 1.0;
        for (int i = 0; i < n; ++i) {
            const double t = x(i);
            q += t * t;
            p *= cos(t / sqrt((double)(i + 1)));
        }
        return 1.0 + q / 4000.0 - p;
    } else if (COST == kHimmelblau) {  // Test 9
        const double a = x(0) * x(0) + x(1) - 11.0, b = x(0) + x(1) * x(1) - 7.0;
        return a * a + b * b;
    } else if (COST == kLevyMontalvo) {  // Test 10, y_i = 1 + (x_i + 1) / 4
        const double y0 = 1.0 + (x(0) + 1.0) / 4.0;
        const double s0 = sin(pi * y0);
        double s = 10.0 * s0 * s0;
        for (int i = 0; i + 1 < n; ++i) {
            const double yi = 1.0 + (x(i) + 1.0) / 4.0, yn = 1.0 + (x(i + 1) + 1.0) / 4.0;
            const double sn = sin(pi * yn);
            s += (yi - 1.0) * (yi - 1.0) * (1.0 + 10.0 * sn * sn);
        }
        const double yl = 1.0 + (x(n - 1) + 1.0) / 4.0;
        s += (yl - 1.0) * (yl - 1.0);
        return pi / (double)n * s;
    } else if (COST == kLangerman || COST == kShekel || COST == kFoxholes) {  // Tests 11, 18, 19
        double s = 0.0;
        for (int r = 0; r < rows; ++r) {
            const double* row = table + (size_t)r * (size_t)(n + 1);
            double d = 0.0;
            for (int j = 0; j < n; ++j) d += (x(j) - row[j]) * (x(j) - row[j]);
            if (COST == kLangerman) s += row[n] * exp(-d / pi) * cos(pi * d);
            else s += 1.0 / (d + row[n]);
        }
        return -s;
    } else if (COST == kMichalewicz) {  // Test 12, m = 10
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const double t = x(i);
            s += sin(t) * pow(sin((double)(i + 1) * t * t / pi), 20.0);
        }
        return -s;
    } else if (COST == kSalomon) {  // Test 15
        double q = 0.0;
        for (int i = 0; i < n; ++i) q += x(i) * x(i);
        const double r = sqrt(q);
        return 1.0 - cos(2.0 * pi * r) + 0.1 * r;
    } else if (COST == kSixHumpCamel) {  // Test 16
        const double a = x(0) * x(0), b = x(1) * x(1);
        return (4.0 - 2.1 * a + a * a / 3.0) * a + x(0) * x(1) + (-4.0 + 4.0 * b) * b;
    } else {  // kShubert, Test 17
        double p = 1.0;
        for (int i = 0; i < n; ++i) {
            const double t = x(i);
            double s = 0.0;
            for (int j = 1; j <= 5; ++j) s += (double)j * cos((double)(j + 1) * t + (double)j);
            p *= s;
        }
        return p;
    }
}

// Dispatch on a run-time cost id (sizes and tables as above); NaN for an unknown id.
template <class X>
__device__ double appendix_cost_any(int cost, int n, const X& x, const double* __restrict__ table, int rows) {
    switch (cost) {
    case kBranin: return appendix_cost<kBranin>(n, x, table, rows);
    case kCosineMixture: return appendix_cost<kCosineMixture>(n, x, table, rows);
    case kDekkersAarts: return appendix_cost<kDekkersAarts>(n, x, table, rows);
    case kEasom: return appendix_cost<kEasom>(n, x, table, rows);
    case kExponential: return appendix_cost<kExponential>(n, x, table, rows);
    case kGoldsteinPrice: return appendix_cost<kGoldsteinPrice>(n, x, table, rows);
    case kGriewank: return appendix_cost<kGriewank>(n, x, table, rows);
    case kHimmelblau: return appendix_cost<kHimmelblau>(n, x, table, rows);
    case kLevyMontalvo: return appendix_cost<kLevyMontalvo>(n, x, table, rows);
    case kLangerman: return appendix_cost<kLangerman>(n, x, table, rows);
    case kMichalewicz: return appendix_cost<kMichalewicz>(n, x, table, rows);
    case kSalomon: return appendix_cost<kSalomon>(n, x, table, rows);
    case kSixHumpCamel: return appendix_cost<kSixHumpCamel>(n, x, table, rows);
    case kShubert: return appendix_cost<kShubert>(n, x, table, rows);
    case kShekel: return appendix_cost<kShekel>(n, x, table, rows);
    case kFoxholes: return appendix_cost<kFoxholes>(n, x, table, rows);
    default: return CUDART_NAN;
    }
}

}  // namespace sa
