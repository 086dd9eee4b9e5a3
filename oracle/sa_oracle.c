/*
 * sa_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU reference of synchronous parallel simulated annealing
 * (Ferreiro, Garcia, Lopez-Salas, Vazquez: "An efficient implementation of
 * parallel simulated annealing algorithm in GPUs").  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load this file's
 * library.  It shares no code, header or constant table with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   - the box-constrained problem  min_{x in I} f(x),  I = prod [l_k, u_k]   (Eq. 1)
 *   - per chain and per temperature level, N (here: L) Metropolis steps:
 *     pick a coordinate, perturb it, evaluate f, accept by the Boltzmann rule
 *     (Sec. 2.1 Steps 2-3, Eq. "proba", k_b = 1)
 *   - at the end of every level a reduction picks the chain with the lowest
 *     final f; all chains restart from it and T is cooled geometrically
 *     T <- rho T  (Sec. 2.2.2 synchronous approach; Listings 3-4; Sec. 2.1 Step 5)
 *
 * Readings where the paper is silent (each one is also a pinned test):
 *   - randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), one
 *     128-bit block per (step, level, chain, problem); key = (seed_lo,
 *     seed_hi ^ tag).  Uniforms u(w) = ((w >> 9) + 0.5) * 2^-23, in (0,1).
 *   - neighbour: coordinate d = (w0 * n) >> 32, Gaussian step via the cosine
 *     branch of Box-Muller, sigma = sigma_frac * (u_d - l_d) * sqrt(T / T0).
 *   - box: reflect once then clip (or clip only).
 *   - acceptance: dF <= 0 or u3 < exp(-dF / T).
 *   - tie-break of the reduction: lowest chain index.
 *   - the answer returned is the incumbent: the best level minimum seen.
 *   - local minimisers of the hybrid SA (Sec. 4.2, Table 10): the paper's
 *     Nelder-Mead in the standard form (coefficients 1, 2, 1/2, 1/2; trial
 *     points clipped into the box), and box-projected gradient descent.
 *
 * Compiled with -ffp-contract=off so that every product and sum is rounded
 * exactly as written, on every host architecture.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SAO_TAG_SWEEP 0u
#define SAO_TAG_INIT 1u
#define SAO_TAG_DA 3u
#define SAO_TAG_XO 5u

enum { SAO_SCHWEFEL = 0, SAO_RASTRIGIN = 1, SAO_ACKLEY = 2, SAO_ROSENBROCK = 3,
       SAO_ROT_RASTRIGIN = 4, SAO_ROT_SCHWEFEL = 5,
       /* the rest of the Appendix's test suite */
       SAO_BRANIN = 6, SAO_COSINE_MIXTURE = 7, SAO_DEKKERS_AARTS = 8, SAO_EASOM = 9, SAO_EXPONENTIAL = 10,
       SAO_GOLDSTEIN_PRICE = 11, SAO_GRIEWANK = 12, SAO_HIMMELBLAU = 13, SAO_LEVY_MONTALVO = 14,
       SAO_LANGERMAN = 15, SAO_MICHALEWICZ = 16, SAO_SALOMON = 17, SAO_SIX_HUMP_CAMEL = 18, SAO_SHUBERT = 19,
       SAO_SHEKEL = 20, SAO_FOXHOLES = 21, SAO_NUM_COSTS = 22 };

static int is_rot(int32_t cost) { return cost == SAO_ROT_RASTRIGIN || cost == SAO_ROT_SCHWEFEL; }
/* Costs with a table of rows (a_i, c_i): Tests 11, 18 and 19. */
static int is_table(int32_t cost) { return cost == SAO_LANGERMAN || cost == SAO_SHEKEL || cost == SAO_FOXHOLES; }
/* Costs defined for n = 2 only. */
static int is_2d(int32_t cost) {
    return cost == SAO_BRANIN || cost == SAO_DEKKERS_AARTS || cost == SAO_EASOM || cost == SAO_GOLDSTEIN_PRICE ||
           cost == SAO_HIMMELBLAU || cost == SAO_SIX_HUMP_CAMEL;
}
/* Costs with a local energy difference in mode 1 (the others recompute f in full). */
static int has_local(int32_t cost) { return cost <= SAO_ROT_SCHWEFEL; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its definition (Salmon et al. 2011, Sec. 4):   */
/* each round multiplies counter words 0 and 2 by two fixed odd constants,     */
/* swaps the halves and xors in the key; the key is bumped by two Weyl        */
/* constants between rounds.                                                   */
/* ------------------------------------------------------------------------ */
void sao_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static inline void sao_block(uint64_t seed, uint32_t tag, uint32_t c0, uint32_t c1,
                             uint32_t c2, uint32_t c3, uint32_t w[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ tag};
    sao_philox4x32_10(ctr, key, w);
}

/* Uniform in (0,1) from the top 23 bits of a word: exact in FP32 and FP64. */
double sao_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

uint32_t sao_coord(uint32_t w, int32_t n) { return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32); }

/* ------------------------------------------------------------------------ */
/* Cost functions, each written as the formula the paper prints (Appendix    */
/* and Sec. 4.1), summed in index order.                                      */
/* ------------------------------------------------------------------------ */
static double h_schwefel(double t) { return t * sin(sqrt(fabs(t))); }
static double g_rastrigin(double t) { return t * t - 10.0 * cos(2.0 * M_PI * t); }

/* Normalised Schwefel (Sec. 4.1): f = -(1/n) sum x_i sin(sqrt|x_i|). */
static double f_schwefel(int n, const double* x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += h_schwefel(x[i]);
    return -(s / (double)n);
}
/* Rastrigin (Appendix, Test 13): 10 n + sum (x_i^2 - 10 cos 2 pi x_i). */
static double f_rastrigin(int n, const double* x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += g_rastrigin(x[i]);
    return 10.0 * (double)n + s;
}
static double ackley_from_sums(int n, double s1, double s2) {
    return -20.0 * exp(-0.2 * sqrt(s1 / (double)n)) - exp(s2 / (double)n) + 20.0 + M_E;
}
/* Ackley (Appendix, Test 1). */
static double f_ackley(int n, const double* x) {
    double s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) { s1 += x[i] * x[i]; s2 += cos(2.0 * M_PI * x[i]); }
    return ackley_from_sums(n, s1, s2);
}
/* Generalised Rosenbrock (Appendix, Test 14), standard form
 * sum_{i<n-1} 100 (x_{i+1} - x_i^2)^2 + (1 - x_i)^2 (the printed x_i is read as x_i^2). */
static double rosen_term(double a, double b) {
    double t = b - a * a, u = 1.0 - a;
    return 100.0 * t * t + u * u;
}
static double f_rosenbrock(int n, const double* x) {
    double s = 0.0;
    for (int i = 0; i + 1 < n; ++i) s += rosen_term(x[i], x[i + 1]);
    return s;
}
/* y = Q x for a row-major n x n Q, each row summed in index order. */
static void rotate(int n, const double* Q, const double* x, double* y) {
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        const double* q = Q + (size_t)i * n;
        for (int j = 0; j < n; ++j) s += q[j] * x[j];
        y[i] = s;
    }
}

/* y = Q x (the rotated costs' transform), exposed for the tests of the GPU's batched transform. */
void sao_rotate(int32_t n, const double* Q, const double* x, double* y) { rotate(n, Q, x, y); }

/* ---- the rest of the Appendix (Tests 2-12 and 15-19), x[0] is the paper's x_1 ---- */

/* Test 2, Branin: (x2 - 5.1 x1^2 / (4 pi^2) + 5 x1 / pi - 6)^2 + 10 (1 - 1/(8 pi)) cos x1 + 10. */
static double f_branin(const double* x) {
    const double a = x[1] - 5.1 * x[0] * x[0] / (4.0 * M_PI * M_PI) + 5.0 * x[0] / M_PI - 6.0;
    return a * a + 10.0 * (1.0 - 1.0 / (8.0 * M_PI)) * cos(x[0]) + 10.0;
}
/* Test 3, cosine mixture, read as sum x_i^2 - 0.1 sum cos(5 pi x_i): the printed
 * signs give a minimum of -0.9 n at the corners, not the printed -0.1 n at 0. */
static double f_cosine_mixture(int n, const double* x) {
    double c = 0.0, q = 0.0;
    for (int i = 0; i < n; ++i) { c += cos(5.0 * M_PI * x[i]); q += x[i] * x[i]; }
    return q - 0.1 * c;
}
/* Test 4, Dekkers and Aarts: 1e5 x1^2 + x2^2 - (x1^2 + x2^2)^2 + 1e-5 (x1^2 + x2^2)^4. */
static double f_dekkers_aarts(const double* x) {
    const double a = x[0] * x[0], b = x[1] * x[1], r = a + b;
    return 1e5 * a + b - r * r + 1e-5 * (r * r) * (r * r);
}
/* Test 5, Easom: -cos x1 cos x2 exp(-(x1 - pi)^2 - (x2 - pi)^2). */
static double f_easom(const double* x) {
    const double u = x[0] - M_PI, v = x[1] - M_PI;
    return -cos(x[0]) * cos(x[1]) * exp(-u * u - v * v);
}
/* Test 6, exponential: -exp(-0.5 sum x_i^2). */
static double f_exponential(int n, const double* x) {
    double q = 0.0;
    for (int i = 0; i < n; ++i) q += x[i] * x[i];
    return -exp(-0.5 * q);
}
/* Test 7, Goldstein and Price. */
static double f_goldstein_price(const double* x) {
    const double a = x[0], b = x[1];
    const double s = a + b + 1.0, t = 2.0 * a - 3.0 * b;
    const double p = 1.0 + s * s * (19.0 - 14.0 * a + 3.0 * a * a - 14.0 * b + 6.0 * a * b + 3.0 * b * b);
    const double q = 30.0 + t * t * (18.0 - 32.0 * a + 12.0 * a * a + 48.0 * b - 36.0 * a * b + 27.0 * b * b);
    return p * q;
}
/* Test 8, Griewank, read in its standard form 1 + sum x_i^2 / 4000 - prod cos(x_i / sqrt i)
 * (the paper prints the product inside the sum), i = 1..n. */
static double f_griewank(int n, const double* x) {
    double q = 0.0, p = 1.0;
    for (int i = 0; i < n; ++i) {
        q += x[i] * x[i];
        p *= cos(x[i] / sqrt((double)(i + 1)));
    }
    return 1.0 + q / 4000.0 - p;
}
/* Test 9, Himmelblau: (x1^2 + x2 - 11)^2 + (x1 + x2^2 - 7)^2. */
static double f_himmelblau(const double* x) {
    const double a = x[0] * x[0] + x[1] - 11.0, b = x[0] + x[1] * x[1] - 7.0;
    return a * a + b * b;
}
/* Test 10, Levy and Montalvo: (pi/n) (10 sin^2(pi y_1) + sum_{i<n} (y_i - 1)^2 (1 + 10 sin^2(pi y_{i+1}))
 * + (y_n - 1)^2), y_i = 1 + (x_i + 1) / 4. */
static double f_levy_montalvo(int n, const double* x) {
    double y0 = 1.0 + (x[0] + 1.0) / 4.0;
    const double s0 = sin(M_PI * y0);
    double s = 10.0 * s0 * s0;
    for (int i = 0; i + 1 < n; ++i) {
        const double yi = 1.0 + (x[i] + 1.0) / 4.0, yn = 1.0 + (x[i + 1] + 1.0) / 4.0;
        const double sn = sin(M_PI * yn);
        s += (yi - 1.0) * (yi - 1.0) * (1.0 + 10.0 * sn * sn);
    }
    const double yl = 1.0 + (x[n - 1] + 1.0) / 4.0;
    s += (yl - 1.0) * (yl - 1.0);
    return M_PI / (double)n * s;
}
/* Squared distance of x to row i of a table of rows (a_i1 .. a_in, c_i). */
static double row_dist2(int n, const double* x, const double* row) {
    double d = 0.0;
    for (int j = 0; j < n; ++j) d += (x[j] - row[j]) * (x[j] - row[j]);
    return d;
}
/* Test 11, modified Langerman: -sum_i c_i exp(-D_i / pi) cos(pi D_i), D_i = |x - a_i|^2. */
static double f_langerman(int n, const double* x, const double* table, int rows) {
    double s = 0.0;
    for (int i = 0; i < rows; ++i) {
        const double* r = table + (size_t)i * (size_t)(n + 1);
        const double d = row_dist2(n, x, r);
        s += r[n] * exp(-d / M_PI) * cos(M_PI * d);
    }
    return -s;
}
/* Test 12, Michalewicz with m = 10: -sum_i sin(x_i) sin(i x_i^2 / pi)^20, i = 1..n. */
static double f_michalewicz(int n, const double* x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += sin(x[i]) * pow(sin((double)(i + 1) * x[i] * x[i] / M_PI), 20.0);
    return -s;
}
/* Test 15, Salomon: 1 - cos(2 pi |x|) + 0.1 |x|. */
static double f_salomon(int n, const double* x) {
    double q = 0.0;
    for (int i = 0; i < n; ++i) q += x[i] * x[i];
    const double r = sqrt(q);
    return 1.0 - cos(2.0 * M_PI * r) + 0.1 * r;
}
/* Test 16, six-hump camel back: (4 - 2.1 x1^2 + x1^4 / 3) x1^2 + x1 x2 + (-4 + 4 x2^2) x2^2. */
static double f_six_hump_camel(const double* x) {
    const double a = x[0] * x[0], b = x[1] * x[1];
    return (4.0 - 2.1 * a + a * a / 3.0) * a + x[0] * x[1] + (-4.0 + 4.0 * b) * b;
}
/* Test 17, Shubert: prod_i sum_{j=1..5} j cos((j + 1) x_i + j). */
static double f_shubert(int n, const double* x) {
    double p = 1.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 1; j <= 5; ++j) s += (double)j * cos((double)(j + 1) * x[i] + (double)j);
        p *= s;
    }
    return p;
}
/* Tests 18 and 19, Shekel and modified Shekel foxholes: -sum_i 1 / (D_i + c_i). */
static double f_shekel(int n, const double* x, const double* table, int rows) {
    double s = 0.0;
    for (int i = 0; i < rows; ++i) {
        const double* r = table + (size_t)i * (size_t)(n + 1);
        s += 1.0 / (row_dist2(n, x, r) + r[n]);
    }
    return -s;
}

/* Full definition of f at x.  Q: rotated costs' n x n matrix; table: rows x (n + 1)
 * (a_i, c_i) of Tests 11, 18, 19; ywork: n doubles of scratch for rotated costs. */
double sao_cost_tab(int32_t cost, int32_t n, const double* x, const double* Q, const double* table, int32_t rows,
                    double* ywork) {
    switch (cost) {
    case SAO_SCHWEFEL: return f_schwefel(n, x);
    case SAO_RASTRIGIN: return f_rastrigin(n, x);
    case SAO_ACKLEY: return f_ackley(n, x);
    case SAO_ROSENBROCK: return f_rosenbrock(n, x);
    case SAO_ROT_RASTRIGIN: rotate(n, Q, x, ywork); return f_rastrigin(n, ywork);
    case SAO_ROT_SCHWEFEL: rotate(n, Q, x, ywork); return f_schwefel(n, ywork);
    case SAO_BRANIN: return f_branin(x);
    case SAO_COSINE_MIXTURE: return f_cosine_mixture(n, x);
    case SAO_DEKKERS_AARTS: return f_dekkers_aarts(x);
    case SAO_EASOM: return f_easom(x);
    case SAO_EXPONENTIAL: return f_exponential(n, x);
    case SAO_GOLDSTEIN_PRICE: return f_goldstein_price(x);
    case SAO_GRIEWANK: return f_griewank(n, x);
    case SAO_HIMMELBLAU: return f_himmelblau(x);
    case SAO_LEVY_MONTALVO: return f_levy_montalvo(n, x);
    case SAO_LANGERMAN: return f_langerman(n, x, table, rows);
    case SAO_MICHALEWICZ: return f_michalewicz(n, x);
    case SAO_SALOMON: return f_salomon(n, x);
    case SAO_SIX_HUMP_CAMEL: return f_six_hump_camel(x);
    case SAO_SHUBERT: return f_shubert(n, x);
    case SAO_SHEKEL: case SAO_FOXHOLES: return f_shekel(n, x, table, rows);
    default: return NAN;
    }
}
double sao_cost_ws(int32_t cost, int32_t n, const double* x, const double* Q, double* ywork) {
    return sao_cost_tab(cost, n, x, Q, NULL, 0, ywork);
}
double sao_cost(int32_t cost, int32_t n, const double* x, const double* Q, const double* table, int32_t rows) {
    double* y = is_rot(cost) ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
    double f = sao_cost_tab(cost, n, x, Q, table, rows, y);
    free(y);
    return f;
}

/* Gradient of f (used by the box-projected local minimiser). */
static double dh_schwefel(double t) {
    double r = sqrt(fabs(t));
    return sin(r) + 0.5 * r * cos(r);
}
static double dg_rastrigin(double t) { return 2.0 * t + 20.0 * M_PI * sin(2.0 * M_PI * t); }
void sao_grad(int32_t cost, int32_t n, const double* x, const double* Q, double* g) {
    if (cost == SAO_SCHWEFEL) {
        for (int i = 0; i < n; ++i) g[i] = -dh_schwefel(x[i]) / (double)n;
    } else if (cost == SAO_RASTRIGIN) {
        for (int i = 0; i < n; ++i) g[i] = dg_rastrigin(x[i]);
    } else if (cost == SAO_ACKLEY) {
        double s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < n; ++i) { s1 += x[i] * x[i]; s2 += cos(2.0 * M_PI * x[i]); }
        double r = sqrt(s1 / (double)n);
        double e1 = exp(-0.2 * r), e2 = exp(s2 / (double)n);
        for (int i = 0; i < n; ++i) {
            double a = (r > 0.0) ? 4.0 * e1 * x[i] / ((double)n * r) : 0.0;
            g[i] = a + 2.0 * M_PI * sin(2.0 * M_PI * x[i]) * e2 / (double)n;
        }
    } else if (cost == SAO_ROSENBROCK) {
        for (int i = 0; i < n; ++i) {
            double gi = 0.0;
            if (i + 1 < n) gi += -400.0 * x[i] * (x[i + 1] - x[i] * x[i]) - 2.0 * (1.0 - x[i]);
            if (i > 0) gi += 200.0 * (x[i] - x[i - 1] * x[i - 1]);
            g[i] = gi;
        }
    } else { /* rotated: grad_x = Q^T g'(y) */
        double* y = (double*)malloc(sizeof(double) * (size_t)n);
        double* gy = (double*)malloc(sizeof(double) * (size_t)n);
        rotate(n, Q, x, y);
        for (int i = 0; i < n; ++i)
            gy[i] = (cost == SAO_ROT_RASTRIGIN) ? dg_rastrigin(y[i]) : -dh_schwefel(y[i]) / (double)n;
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += Q[(size_t)i * n + j] * gy[i];
            g[j] = s;
        }
        free(y);
        free(gy);
    }
}

/* ------------------------------------------------------------------------ */
/* Synchronous parallel SA                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t cost;
    int32_t n;
    int64_t chains;
    int32_t L;        /* Metropolis steps per chain and level (the paper's N) */
    int32_t K;        /* levels to run in this call */
    int32_t level0;   /* absolute index of the first level (resume) */
    int32_t boundary; /* 0: reflect once then clip; 1: clip */
    int32_t mode;     /* 0: full recompute of f(x'); 1: local difference */
    int32_t threads;  /* OpenMP threads, 0 = runtime default */
    uint32_t problem; /* counter word 3 (problem index in a batch) */
    uint64_t seed;
    double T0, rho, sigma_frac;
    const double* lo;
    const double* hi;
    const double* Q; /* row-major n x n, rotated costs only */
    int32_t independent; /* 0: synchronous (Sec. 2.2.2: every level restarts all chains from
                            the best one); 1: asynchronous (Sec. 2.2.1: no exchange, each chain
                            continues from its own state; the levels' minima still give the
                            incumbent).  Independent runs start at level 0. */
    int32_t exchange_every; /* > 1: the exchange (restart from the best) only after levels
                               m-1, 2m-1, ...; chains continue their own states in between */
    const double* table; /* Tests 11, 18, 19: rows x (n + 1), row i = (a_i1 .. a_in, c_i) */
    int32_t table_rows;
    int32_t proposal;    /* 0: Gaussian step sigma_frac (u_d - l_d) sqrt(T / T0) z (Box-Muller);
                            1: the coordinate redrawn uniformly, x_d' = l_d + u2 (u_d - l_d) */
    int32_t crossover;   /* 0: every exchange restarts all chains from the minimum; 1: stochastic
                            crossover (Boltzmann selection, see crossover_sources) */
} sao_cfg;

typedef struct {
    double* x_best;      /* [n] in: restart point when level0 > 0; out: restart point after the last level */
    double* f_best;      /* [1] F(x_best), in/out */
    double* x_inc;       /* [n] incumbent, in/out */
    double* f_inc;       /* [1] incumbent value, in/out (+inf before the first level) */
    int64_t* argmin;     /* [K] p* per level, or NULL */
    double* f_level;     /* [K] F_{p*} per level, or NULL */
    int64_t* accepts;    /* [K] accepted moves per level, or NULL */
    uint32_t* bits;      /* [trace_levels][chains][ceil(L/32)] accept bits, or NULL */
    int32_t trace_levels;
    double* F_final;     /* [chains] F at the end of the last level, or NULL */
    double* X_final;     /* [chains * n] states at the end of the last level, or NULL */
    int64_t* xo_src;     /* [K][chains] crossover: the chain each chain restarts from after
                            level k (-1 where no exchange follows), or NULL */
} sao_out;

/* T_l = T0 rho^l by repeated multiplication (the host loop of Listing 3). */
double sao_temperature(double T0, double rho, int32_t level) {
    double T = T0;
    for (int l = 0; l < level; ++l) T = T * rho;
    return T;
}

/* Number of levels of the do-while of Listing 3: run, cool, stop once T <= T_min. */
int32_t sao_levels_for(double T0, double rho, double T_min) {
    double T = T0;
    int32_t k = 0;
    do { ++k; T = T * rho; } while (T > T_min && k < 100000000);
    return k;
}

static double apply_box(double xp, double l, double u, int32_t boundary) {
    if (boundary == 0) {
        if (xp < l) xp = 2.0 * l - xp;
        else if (xp > u) xp = 2.0 * u - xp;
    }
    if (xp < l) xp = l;
    if (xp > u) xp = u;
    return xp;
}

/* Initial point of a chain at level 0: x_k = l_k + u (u_k - l_k), coordinate
 * k taking word k mod 4 of Philox block (k/4, 0, chain, problem), tag INIT. */
void sao_init_point(const sao_cfg* cfg, int64_t c, double* x) {
    for (int k = 0; k < cfg->n; k += 4) {
        uint32_t w[4];
        sao_block(cfg->seed, SAO_TAG_INIT, (uint32_t)(k / 4), 0u, (uint32_t)c, cfg->problem, w);
        for (int j = 0; j < 4 && k + j < cfg->n; ++j)
            x[k + j] = cfg->lo[k + j] + sao_uniform(w[j]) * (cfg->hi[k + j] - cfg->lo[k + j]);
    }
}

/* Sum of g over the rotated coordinates y (rotated costs, mode 1). */
static double gsum(int32_t cost, int n, const double* y) {
    double s = 0.0;
    if (cost == SAO_ROT_RASTRIGIN) for (int i = 0; i < n; ++i) s += g_rastrigin(y[i]);
    else for (int i = 0; i < n; ++i) s += h_schwefel(y[i]);
    return s;
}
static double f_from_gsum(int32_t cost, int n, double s) {
    return (cost == SAO_ROT_RASTRIGIN) ? 10.0 * (double)n + s : -(s / (double)n);
}

/*
 * One chain for one level: L Metropolis steps at temperature T starting from
 * x (level 0: its own random point; later: the common restart point).
 * On return x holds the final state and the function returns f(x) recomputed
 * from the definition.  bits (may be NULL) receives the accept decisions.
 */
/*
 * Delayed acceptance (Christen & Fox 2005; not in the paper): when ft_prop is
 * given, ft_prop[s] is the surrogate's value at step s's proposal and ft0 its
 * value at the level's start state.  Stage 1 passes with probability
 * min(1, exp(-dFs / T)), dFs = ft(x') - ft(x), drawn with word 0 of the Philox
 * block (s, level, chain, problem) of stream tag 3; only then is the true dF
 * evaluated, and the move is accepted with probability
 * min(1, exp(-(dF - dFs) / T)) drawn with the sweep stream's u3.
 * n_true (may be NULL) counts the true evaluations.
 */
typedef struct {
    int kind;              /* 0: none; 1: table (ft0, ft_prop); 2: a f(x) + b sum_i sin(x_i) */
    double ft0;
    const double* ft_prop;
    double a, b;
    int plant;             /* 0; tests of the parity checks only: 1 = stage 2 with the sign of
                              the surrogate difference flipped (a planted mistake) */
} sao_da;

static double chain_level_da(const sao_cfg* cfg, int32_t level, int64_t c, double* x,
                             uint32_t* bits, int64_t* n_accept, double* dF_out, double* tau_out,
                             const sao_da* da, int64_t* n_true);

static double chain_level(const sao_cfg* cfg, int32_t level, int64_t c, double* x,
                          uint32_t* bits, int64_t* n_accept, double* dF_out, double* tau_out) {
    return chain_level_da(cfg, level, c, x, bits, n_accept, dF_out, tau_out, NULL, NULL);
}

/* The analytic test surrogate a f(x) + b sum_i sin(x_i), in full. */
static double da_fn(const sao_cfg* cfg, const sao_da* da, const double* x, double* ywork) {
    double s = 0.0;
    for (int i = 0; i < cfg->n; ++i) s += sin(x[i]);
    return da->a * sao_cost_ws(cfg->cost, cfg->n, x, cfg->Q, ywork) + da->b * s;
}

/* Step 2 of Sec. 2.1 for chain c at step s of a level: the Philox block of
 * (s, level, c, problem) picks the coordinate d (word 0) and moves it -- a Gaussian
 * step (Box-Muller, cosine branch, words 1 and 2) scaled by sqrt(T / T0), or a
 * uniform redraw of the coordinate (word 2) -- reflected/clipped into the box.
 * Returns x'_d; *d_out = d, u3_out (may be NULL) = the uniform of word 3. */
static double propose(const sao_cfg* cfg, int32_t level, int64_t c, int s, double s_l, const double* x, int* d_out,
                      double* u3_out) {
    uint32_t w[4];
    sao_block(cfg->seed, SAO_TAG_SWEEP, (uint32_t)s, (uint32_t)level, (uint32_t)c, cfg->problem, w);
    const int d = (int)sao_coord(w[0], cfg->n);
    const double u1 = sao_uniform(w[1]), u2 = sao_uniform(w[2]);
    const double xd = x[d];
    double xp;
    if (cfg->proposal == 1) {
        xp = apply_box(cfg->lo[d] + u2 * (cfg->hi[d] - cfg->lo[d]), cfg->lo[d], cfg->hi[d], cfg->boundary);
    } else {
        const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
        const double sigma = cfg->sigma_frac * (cfg->hi[d] - cfg->lo[d]) * s_l;
        xp = apply_box(xd + sigma * z, cfg->lo[d], cfg->hi[d], cfg->boundary);
    }
    *d_out = d;
    if (u3_out) *u3_out = sao_uniform(w[3]);
    return xp;
}

/* The proposal (d, x'_d) that chain c at state x makes at step s of a level. */
void sao_proposal(const sao_cfg* cfg, int32_t level, int64_t c, int32_t s, const double* x, int32_t* d_out,
                  double* xp_out) {
    const double T = sao_temperature(cfg->T0, cfg->rho, level);
    int d = 0;
    *xp_out = propose(cfg, level, c, s, sqrt(T / cfg->T0), x, &d, NULL);
    *d_out = d;
}

static double chain_level_da(const sao_cfg* cfg, int32_t level, int64_t c, double* x,
                             uint32_t* bits, int64_t* n_accept, double* dF_out, double* tau_out,
                             const sao_da* da, int64_t* n_true) {
    double* ywork = is_rot(cfg->cost) ? (double*)malloc(sizeof(double) * (size_t)cfg->n) : NULL;
    const int n = cfg->n;
    const double T = sao_temperature(cfg->T0, cfg->rho, level);
    const double s_l = sqrt(T / cfg->T0);
    const int rot = is_rot(cfg->cost);
    double* y = rot ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
    double* yp = rot ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
    double F = sao_cost_tab(cfg->cost, n, x, cfg->Q, cfg->table, cfg->table_rows, y);
    double S1 = 0.0, S2 = 0.0, G = 0.0;
    if (cfg->mode == 1 && cfg->cost == SAO_ACKLEY)
        for (int i = 0; i < n; ++i) { S1 += x[i] * x[i]; S2 += cos(2.0 * M_PI * x[i]); }
    if (cfg->mode == 1 && rot) G = gsum(cfg->cost, n, y); /* y = Q x from the call above */
    int64_t acc = 0, evals = 0;
    const int use_da = da && da->kind != 0;
    double ft_cur = !use_da ? 0.0 : (da->kind == 1 ? da->ft0 : da_fn(cfg, da, x, ywork));
    double ft_new = 0.0;
    const int words = (cfg->L + 31) / 32;
    if (bits) memset(bits, 0, sizeof(uint32_t) * (size_t)words);

    for (int s = 0; s < cfg->L; ++s) {
        /* Step 2: move coordinate d -- a Gaussian step (Box-Muller, cosine branch), or a
         * uniform redraw of the coordinate in [l_d, u_d] with the second uniform. */
        int d = 0;
        double u3 = 0.0;
        const double xp = propose(cfg, level, c, s, s_l, x, &d, &u3);
        const double xd = x[d];

        /* Delayed acceptance, stage 1 (surrogate only). */
        double dFs = 0.0;
        if (use_da) {
            uint32_t wd[4];
            sao_block(cfg->seed, SAO_TAG_DA, (uint32_t)s, (uint32_t)level, (uint32_t)c, cfg->problem, wd);
            if (da->kind == 1) {
                ft_new = da->ft_prop[s];
            } else {
                x[d] = xp;
                ft_new = da_fn(cfg, da, x, ywork);
                x[d] = xd;
            }
            dFs = ft_new - ft_cur;
            if (!(dFs <= 0.0 || sao_uniform(wd[0]) < exp(-dFs / T))) {
                if (dF_out) dF_out[s] = NAN;
                if (tau_out) tau_out[s] = NAN;
                continue;
            }
        }
        ++evals;

        /* Step 3: energy difference. */
        double dF, Fp = 0.0, S1p = 0.0, S2p = 0.0, Gp = 0.0;
        if (cfg->mode == 0) {
            x[d] = xp;
            Fp = sao_cost_tab(cfg->cost, n, x, cfg->Q, cfg->table, cfg->table_rows, y);
            x[d] = xd;
            dF = Fp - F;
        } else if (cfg->cost == SAO_SCHWEFEL) {
            dF = -((h_schwefel(xp) - h_schwefel(xd)) / (double)n);
        } else if (cfg->cost == SAO_RASTRIGIN) {
            dF = g_rastrigin(xp) - g_rastrigin(xd);
        } else if (cfg->cost == SAO_ACKLEY) {
            S1p = S1 - xd * xd + xp * xp;
            S2p = S2 - cos(2.0 * M_PI * xd) + cos(2.0 * M_PI * xp);
            dF = ackley_from_sums(n, S1p, S2p) - ackley_from_sums(n, S1, S2);
        } else if (cfg->cost == SAO_ROSENBROCK) {
            double before = 0.0, after = 0.0;
            if (d > 0) { before += rosen_term(x[d - 1], xd); after += rosen_term(x[d - 1], xp); }
            if (d + 1 < n) { before += rosen_term(xd, x[d + 1]); after += rosen_term(xp, x[d + 1]); }
            dF = after - before;
        } else { /* rotated: y' = y + (x'_d - x_d) Q[:, d] */
            const double delta = xp - xd;
            for (int i = 0; i < n; ++i) yp[i] = y[i] + delta * cfg->Q[(size_t)i * n + d];
            Gp = gsum(cfg->cost, n, yp);
            dF = f_from_gsum(cfg->cost, n, Gp) - f_from_gsum(cfg->cost, n, G);
        }

        /* Metropolis criterion, Eq. "proba" with k_b = 1 (stage 2 of delayed
         * acceptance: the same test on dF - dFs). */
        const double dFa = (use_da && da->plant == 1) ? dF + dFs : dF - dFs;
        const int accept = (dFa <= 0.0) || (u3 < exp(-dFa / T));
        if (dF_out) dF_out[s] = dF;
        if (tau_out) tau_out[s] = -T * log(u3); /* the same test written as dF < tau */
        if (accept) {
            x[d] = xp;
            ++acc;
            if (use_da) ft_cur = ft_new;
            if (bits) bits[s >> 5] |= 1u << (s & 31);
            if (cfg->mode == 0) {
                F = Fp;
            } else {
                F = F + dF;
                if (cfg->cost == SAO_ACKLEY) { S1 = S1p; S2 = S2p; }
                if (rot) { double* t = y; y = yp; yp = t; G = Gp; }
            }
        }
    }
    double Fend = sao_cost_tab(cfg->cost, n, x, cfg->Q, cfg->table, cfg->table_rows, yp ? yp : y);
    free(y);
    free(yp);
    free(ywork);
    if (n_accept) *n_accept = acc;
    if (n_true) *n_true = evals;
    return Fend;
}

/* One chain, one level of delayed acceptance with the surrogate values given. */
double sao_da_chain_level(const sao_cfg* cfg, int32_t level, int64_t c, double* x, double ft0,
                          const double* ft_prop, uint32_t* bits, int64_t* n_accept, int64_t* n_true) {
    const sao_da da = {1, ft0, ft_prop, 0.0, 0.0, 0};
    return chain_level_da(cfg, level, c, x, bits, n_accept, NULL, NULL, &da, n_true);
}

/* The same, also returning each step's true difference dF_out[s] (NaN where
 * stage 1 rejected the move and f was not evaluated). */
double sao_da_chain_level_steps(const sao_cfg* cfg, int32_t level, int64_t c, double* x, double ft0,
                                const double* ft_prop, uint32_t* bits, int64_t* n_accept, int64_t* n_true,
                                double* dF_out) {
    const sao_da da = {1, ft0, ft_prop, 0.0, 0.0, 0};
    return chain_level_da(cfg, level, c, x, bits, n_accept, dF_out, NULL, &da, n_true);
}

/* The same, also returning each step's threshold tau_out[s] = -T ln u3 (NaN where
 * stage 1 rejected the move); plant != 0 only in the tests that show a parity
 * check catches a planted mistake (see sao_da). */
double sao_da_chain_level_trace(const sao_cfg* cfg, int32_t level, int64_t c, double* x, double ft0,
                                const double* ft_prop, uint32_t* bits, int64_t* n_accept, int64_t* n_true,
                                double* dF_out, double* tau_out, int32_t plant) {
    const sao_da da = {1, ft0, ft_prop, 0.0, 0.0, plant};
    return chain_level_da(cfg, level, c, x, bits, n_accept, dF_out, tau_out, &da, n_true);
}

/* The same with the analytic test surrogate a f(x) + b sum_i sin(x_i). */
double sao_da_chain_level_fn(const sao_cfg* cfg, int32_t level, int64_t c, double* x, double a, double b,
                             uint32_t* bits, int64_t* n_accept, int64_t* n_true) {
    const sao_da da = {2, 0.0, NULL, a, b, 0};
    return chain_level_da(cfg, level, c, x, bits, n_accept, NULL, NULL, &da, n_true);
}

double sao_chain_level(const sao_cfg* cfg, int32_t level, int64_t c, double* x,
                       uint32_t* bits, int64_t* n_accept) {
    return chain_level(cfg, level, c, x, bits, n_accept, NULL, NULL);
}

/* The same, also returning every step's dF and threshold tau = -T ln u3
 * (diagnostics for judging near-ties of reduced-precision decisions). */
double sao_chain_level_steps(const sao_cfg* cfg, int32_t level, int64_t c, double* x,
                             uint32_t* bits, int64_t* n_accept, double* dF_out, double* tau_out) {
    return chain_level(cfg, level, c, x, bits, n_accept, dF_out, tau_out);
}

/* The cost's own requirements: Q for rotated costs, a table for Tests 11, 18, 19,
 * n = 2 for the two-variable tests, mode 0 where no local difference is written. */
static int cost_ok(const sao_cfg* cfg) {
    if (cfg->cost < 0 || cfg->cost >= SAO_NUM_COSTS || (is_rot(cfg->cost) && !cfg->Q)) return 0;
    if (is_table(cfg->cost) && (!cfg->table || cfg->table_rows < 1)) return 0;
    if ((is_2d(cfg->cost) && cfg->n != 2) || (cfg->mode == 1 && !has_local(cfg->cost))) return 0;
    return 1;
}

/*
 * Stochastic crossover (a reading of the SOS scheme the paper cites in Sec. 2.2:
 * an exchange operator that is random instead of the minimum): at an exchange,
 * chain c restarts from the final state of chain j, drawn with probability
 * w_j / sum_k w_k, w_j = exp(-(F_j - F_min) / T) at the level's temperature T
 * (0 for a non-finite F_j).  The draw inverts the running sum S_j = w_0 + ... + w_j
 * at t = u_c S_{C-1}: j = min{ j : S_j > t }, u_c from word 0 of the Philox block
 * (0, level, c, problem) of stream tag 5.  As T -> 0 every chain draws the minimum.
 */
static void crossover_sources(const sao_cfg* cfg, int32_t level, const double* F, int64_t C, double Fmin,
                              int64_t* src, double* S) {
    const double T = sao_temperature(cfg->T0, cfg->rho, level);
    double acc = 0.0;
    for (int64_t j = 0; j < C; ++j) {
        acc += isfinite(F[j]) ? exp(-(F[j] - Fmin) / T) : 0.0;
        S[j] = acc;
    }
    for (int64_t c = 0; c < C; ++c) {
        uint32_t w[4];
        sao_block(cfg->seed, SAO_TAG_XO, 0u, (uint32_t)level, (uint32_t)c, cfg->problem, w);
        const double t = sao_uniform(w[0]) * acc;
        int64_t a = 0, b = C - 1;
        while (a < b) {
            const int64_t m = a + (b - a) / 2;
            if (S[m] > t) b = m;
            else a = m + 1;
        }
        src[c] = a;
    }
}

/* The crossover's draw for given final values (exposed for tests). */
int sao_crossover_sources(const sao_cfg* cfg, int32_t level, const double* F, int64_t C, int64_t* src) {
    if (!cfg || !F || !src || C < 1) return -1;
    int64_t p = 0;
    for (int64_t c = 1; c < C; ++c)
        if (F[c] < F[p]) p = c;
    double* S = (double*)malloc(sizeof(double) * (size_t)C);
    if (!S) return -2;
    crossover_sources(cfg, level, F, C, F[p], src, S);
    free(S);
    return 0;
}

/*
 * Run levels level0 .. level0+K-1 of synchronous parallel SA (Listings 3-4).
 * Returns 0 on success, -1 on a bad argument, -2 on allocation failure.
 */
int sao_run(const sao_cfg* cfg, sao_out* out) {
    if (!cfg || !out || cfg->n < 1 || cfg->chains < 1 || cfg->L < 0 || cfg->K < 0 ||
        !cfg->lo || !cfg->hi || !out->x_best || !out->f_best || !out->x_inc || !out->f_inc)
        return -1;
    if (!cost_ok(cfg)) return -1;
    const int periodic = cfg->exchange_every > 1;
    if ((cfg->independent || periodic || cfg->crossover) && cfg->level0 != 0) return -1;
    if (cfg->crossover && cfg->independent) return -1;
    const int n = cfg->n;
    const int64_t C = cfg->chains;
    const int words = (cfg->L + 31) / 32;
    double* X = (double*)malloc(sizeof(double) * (size_t)C * (size_t)n);
    double* F = (double*)malloc(sizeof(double) * (size_t)C);
    int64_t* A = (int64_t*)malloc(sizeof(int64_t) * (size_t)C);
    double* Xn = cfg->crossover ? (double*)malloc(sizeof(double) * (size_t)C * (size_t)n) : NULL;
    double* S = cfg->crossover ? (double*)malloc(sizeof(double) * (size_t)C) : NULL;
    int64_t* src = cfg->crossover ? (int64_t*)malloc(sizeof(int64_t) * (size_t)C) : NULL;
    if (!X || !F || !A || (cfg->crossover && (!Xn || !S || !src))) {
        free(X); free(F); free(A); free(Xn); free(S); free(src);
        return -2;
    }
#ifdef _OPENMP
    int nthreads = cfg->threads > 0 ? cfg->threads : omp_get_max_threads();
#endif
    for (int k = 0; k < cfg->K; ++k) {
        const int32_t level = cfg->level0 + k;
        uint32_t* bits = (out->bits && k < out->trace_levels)
                             ? out->bits + (size_t)k * (size_t)C * (size_t)words : NULL;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
        for (int64_t c = 0; c < C; ++c) {
            double* x = X + (size_t)c * n;
            /* crossover: x already holds the state the chain drew at the exchange */
            const int own = cfg->independent || cfg->crossover || (periodic && level % cfg->exchange_every != 0);
            if (level == 0) sao_init_point(cfg, c, x);
            else if (!own) memcpy(x, out->x_best, sizeof(double) * (size_t)n);
            /* own start: x is the chain's own state after the previous level */
            F[c] = sao_chain_level(cfg, level, c, x, bits ? bits + (size_t)c * words : NULL, &A[c]);
        }
        /* Reduction over the chains' final values, lowest index on ties (Sec. 2.2.2). */
        int64_t p = 0;
        int64_t acc = 0;
        for (int64_t c = 0; c < C; ++c) {
            if (F[c] < F[p]) p = c;
            acc += A[c];
        }
        memcpy(out->x_best, X + (size_t)p * n, sizeof(double) * (size_t)n);
        out->f_best[0] = F[p];
        if (F[p] < out->f_inc[0]) {
            out->f_inc[0] = F[p];
            memcpy(out->x_inc, X + (size_t)p * n, sizeof(double) * (size_t)n);
        }
        if (out->argmin) out->argmin[k] = p;
        if (out->f_level) out->f_level[k] = F[p];
        if (out->accepts) out->accepts[k] = acc;
        if (k == cfg->K - 1) {
            if (out->F_final) memcpy(out->F_final, F, sizeof(double) * (size_t)C);
            if (out->X_final) memcpy(out->X_final, X, sizeof(double) * (size_t)C * (size_t)n);
        }
        /* Stochastic crossover before the next level when it starts with an exchange. */
        const int32_t nxt = level + 1;
        const int exchange_next = !(periodic && nxt % cfg->exchange_every != 0);
        if (out->xo_src) for (int64_t c = 0; c < C; ++c) out->xo_src[(size_t)k * (size_t)C + (size_t)c] = -1;
        if (cfg->crossover && exchange_next && k + 1 < cfg->K) {
            crossover_sources(cfg, level, F, C, F[p], src, S);
            for (int64_t c = 0; c < C; ++c)
                memcpy(Xn + (size_t)c * n, X + (size_t)src[c] * n, sizeof(double) * (size_t)n);
            double* t = X; X = Xn; Xn = t;
            if (out->xo_src) memcpy(out->xo_src + (size_t)k * (size_t)C, src, sizeof(int64_t) * (size_t)C);
        }
    }
    free(X);
    free(F);
    free(A);
    free(Xn);
    free(S);
    free(src);
    return 0;
}

/*
 * One level for a subset of chains [c0, c1): used to check single chains of a
 * large run one by one.  x_start = NULL means level 0 (own random start).
 */
int sao_level_chains(const sao_cfg* cfg, int32_t level, const double* x_start, int64_t c0,
                     int64_t c1, double* F_out, double* X_out, uint32_t* bits_out,
                     int64_t* acc_out) {
    if (!cfg || c1 < c0 || (level > 0 && !x_start) || !cost_ok(cfg)) return -1;
    const int n = cfg->n;
    const int words = (cfg->L + 31) / 32;
#ifdef _OPENMP
    int nthreads = cfg->threads > 0 ? cfg->threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int64_t c = c0; c < c1; ++c) {
        double* x = (double*)malloc(sizeof(double) * (size_t)n);
        if (x_start) memcpy(x, x_start, sizeof(double) * (size_t)n);
        else sao_init_point(cfg, c, x);
        int64_t a = 0;
        double Fc = sao_chain_level(cfg, level, c, x, bits_out ? bits_out + (size_t)(c - c0) * words : NULL, &a);
        if (F_out) F_out[c - c0] = Fc;
        if (X_out) memcpy(X_out + (size_t)(c - c0) * n, x, sizeof(double) * (size_t)n);
        if (acc_out) acc_out[c - c0] = a;
        free(x);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Box-projected gradient descent with Armijo backtracking: the local       */
/* minimiser of the hybrid SA (the paper hands the SA point to Nelder-Mead, */
/* Sec. 4.2 / Table 10; here a projected gradient method takes that role).  */
/* The first search starts at alpha = 1, every later one at twice the last  */
/* accepted step (capped at 1e12), halving at most max_halvings times.       */
/* ------------------------------------------------------------------------ */
int sao_pgd(int32_t cost, int32_t n, const double* lo, const double* hi, const double* Q,
            double* x, int32_t max_iter, double tol, double armijo_c, int32_t max_halvings,
            double* f_out, int32_t* iters_out) {
    if (!has_local(cost)) return -1; /* gradients are written for Sec. 4.1's and the rotated costs only */
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* xn = (double*)malloc(sizeof(double) * (size_t)n);
    double* yw = (double*)malloc(sizeof(double) * (size_t)n);
    if (!g || !xn || !yw) { free(g); free(xn); free(yw); return -2; }
    for (int i = 0; i < n; ++i) x[i] = fmin(fmax(x[i], lo[i]), hi[i]);
    double f = sao_cost_ws(cost, n, x, Q, yw);
    double alpha_next = 1.0;
    int it = 0;
    for (; it < max_iter; ++it) {
        sao_grad(cost, n, x, Q, g);
        double pg = 0.0; /* infinity norm of the projected gradient P(x - g) - x */
        for (int i = 0; i < n; ++i) {
            double v = fmin(fmax(x[i] - g[i], lo[i]), hi[i]) - x[i];
            if (fabs(v) > pg) pg = fabs(v);
        }
        if (pg < tol) break;
        double alpha = alpha_next;
        int ok = 0;
        double fn = f;
        for (int h = 0; h < max_halvings; ++h) {
            double slope = 0.0;
            for (int i = 0; i < n; ++i) {
                xn[i] = fmin(fmax(x[i] - alpha * g[i], lo[i]), hi[i]);
                slope += g[i] * (xn[i] - x[i]);
            }
            fn = sao_cost_ws(cost, n, xn, Q, yw);
            if (fn <= f + armijo_c * slope) { ok = 1; break; }
            alpha = 0.5 * alpha;
        }
        if (!ok) break;
        memcpy(x, xn, sizeof(double) * (size_t)n);
        f = fn;
        alpha_next = fmin(2.0 * alpha, 1e12);
    }
    free(g);
    free(xn);
    free(yw);
    if (f_out) *f_out = f;
    if (iters_out) *iters_out = it;
    return 0;
}


/* ------------------------------------------------------------------------ */
/* Nelder-Mead (the paper's local minimiser of the hybrid SA, Sec. 4.2 and    */
/* Table 10), in the standard form of Lagarias, Reeds, Wright & Wright (SIAM  */
/* J. Optim. 1998): reflection rho = 1, expansion chi = 2, contraction        */
/* psi = 1/2, shrink sigma = 1/2; every trial point is formed from the        */
/* centroid c and the worst vertex v_h (c + rho (c - v_h), c + rho chi        */
/* (c - v_h), c + psi rho (c - v_h), c - psi (c - v_h)).  adaptive: the       */
/* dimension-dependent coefficients of Gao & Han (Comput. Optim. Appl. 2012),  */
/* chi = 1 + 2/n, psi = 3/4 - 1/(2n), sigma = 1 - 1/n.                         */
/* Box constraints: every trial point is clipped into the box.  Vertices are */
/* ordered by (f, slot); the initial simplex is x0 and x0 + delta_k e_k,     */
/* delta_k = step_frac (u_k - l_k) (or minus, if that leaves the box).       */
/* Stops when both f_worst - f_best <= ftol max(1, |f_best|) and every       */
/* vertex is within xtol (u_i - l_i) of the best in every coordinate i, or   */
/* after max_iter iterations.  x: in start point, out best vertex.           */
/* ------------------------------------------------------------------------ */
static void nm_clip(int n, const double* lo, const double* hi, double* x) {
    for (int i = 0; i < n; ++i) x[i] = fmin(fmax(x[i], lo[i]), hi[i]);
}

int sao_nelder_mead(int32_t cost, int32_t n, const double* lo, const double* hi, const double* Q,
                    const double* table, int32_t rows, double* x, double step_frac, int32_t max_iter, double ftol,
                    double xtol, int32_t adaptive, double* f_out, int32_t* iters_out) {
    const int m = n + 1;
    const double rho = 1.0;
    const double chi = adaptive ? 1.0 + 2.0 / (double)n : 2.0;
    const double psi = adaptive ? 0.75 - 1.0 / (2.0 * (double)n) : 0.5;
    const double sig = adaptive ? 1.0 - 1.0 / (double)n : 0.5;
    double* V = (double*)malloc(sizeof(double) * (size_t)m * n);
    double* F = (double*)malloc(sizeof(double) * (size_t)m);
    double* xc = (double*)malloc(sizeof(double) * (size_t)n);
    double* xr = (double*)malloc(sizeof(double) * (size_t)n);
    double* xt = (double*)malloc(sizeof(double) * (size_t)n);
    double* yw = (double*)malloc(sizeof(double) * (size_t)n);
    if (!V || !F || !xc || !xr || !xt || !yw) {
        free(V); free(F); free(xc); free(xr); free(xt); free(yw);
        return -2;
    }
    nm_clip(n, lo, hi, x);
    for (int j = 0; j < m; ++j) {
        double* v = V + (size_t)j * n;
        memcpy(v, x, sizeof(double) * (size_t)n);
        if (j > 0) {
            const int k = j - 1;
            const double d = step_frac * (hi[k] - lo[k]);
            v[k] = (v[k] + d <= hi[k]) ? v[k] + d : v[k] - d;
            nm_clip(n, lo, hi, v);
        }
        F[j] = sao_cost_tab(cost, n, v, Q, table, rows, yw);
    }
    int it = 0;
    for (; it < max_iter; ++it) {
        /* best l, worst h, second worst s in the order (f, slot) */
        int l = 0, h = 0;
        for (int j = 1; j < m; ++j) {
            if (F[j] < F[l]) l = j;
            if (F[j] >= F[h]) h = j;
        }
        int sw = (h == 0) ? 1 : 0;
        for (int j = 0; j < m; ++j)
            if (j != h && F[j] >= F[sw]) sw = j;
        if (F[h] - F[l] <= ftol * fmax(1.0, fabs(F[l]))) {
            int small = 1;
            for (int j = 0; j < m && small; ++j)
                for (int i = 0; i < n; ++i)
                    if (fabs(V[(size_t)j * n + i] - V[(size_t)l * n + i]) > xtol * (hi[i] - lo[i])) { small = 0; break; }
            if (small) break;
        }
        /* centroid of every vertex but the worst, summed in slot order */
        for (int i = 0; i < n; ++i) {
            double a = 0.0;
            for (int j = 0; j < m; ++j)
                if (j != h) a += V[(size_t)j * n + i];
            xc[i] = a / (double)n;
        }
        const double* vh = V + (size_t)h * n;
        for (int i = 0; i < n; ++i) xr[i] = xc[i] + rho * (xc[i] - vh[i]);
        nm_clip(n, lo, hi, xr);
        const double fr = sao_cost_tab(cost, n, xr, Q, table, rows, yw);
        int accept = 0;
        double fa = fr;
        const double* xa = xr;
        if (fr < F[l]) {
            for (int i = 0; i < n; ++i) xt[i] = xc[i] + rho * chi * (xc[i] - vh[i]);
            nm_clip(n, lo, hi, xt);
            const double fe = sao_cost_tab(cost, n, xt, Q, table, rows, yw);
            accept = 1;
            if (fe < fr) { fa = fe; xa = xt; }
        } else if (fr < F[sw]) {
            accept = 1;
        } else if (fr < F[h]) {
            for (int i = 0; i < n; ++i) xt[i] = xc[i] + psi * rho * (xc[i] - vh[i]);
            nm_clip(n, lo, hi, xt);
            const double fo = sao_cost_tab(cost, n, xt, Q, table, rows, yw);
            if (fo <= fr) { accept = 1; fa = fo; xa = xt; }
        } else {
            for (int i = 0; i < n; ++i) xt[i] = xc[i] - psi * (xc[i] - vh[i]);
            nm_clip(n, lo, hi, xt);
            const double fi = sao_cost_tab(cost, n, xt, Q, table, rows, yw);
            if (fi < F[h]) { accept = 1; fa = fi; xa = xt; }
        }
        if (accept) {
            memcpy(V + (size_t)h * n, xa, sizeof(double) * (size_t)n);
            F[h] = fa;
        } else { /* shrink towards the best vertex */
            const double* vl = V + (size_t)l * n;
            for (int j = 0; j < m; ++j) {
                if (j == l) continue;
                double* v = V + (size_t)j * n;
                for (int i = 0; i < n; ++i) v[i] = vl[i] + sig * (v[i] - vl[i]);
                nm_clip(n, lo, hi, v);
                F[j] = sao_cost_tab(cost, n, v, Q, table, rows, yw);
            }
        }
    }
    int l = 0;
    for (int j = 1; j < m; ++j)
        if (F[j] < F[l]) l = j;
    memcpy(x, V + (size_t)l * n, sizeof(double) * (size_t)n);
    if (f_out) *f_out = F[l];
    if (iters_out) *iters_out = it;
    free(V); free(F); free(xc); free(xr); free(xt); free(yw);
    return 0;
}
