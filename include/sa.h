/*
 * sa.h -- C ABI of a GB300 (sm_103a) library for synchronous parallel
 * simulated annealing (Ferreiro, Garcia, Lopez-Salas, Vazquez, "An efficient
 * implementation of parallel simulated annealing algorithm in GPUs").
 *
 * The problem (Eq. 1):  minimise f(x) over the box I = prod_k [l_k, u_k].
 * The method (Sec. 2.2.2, Listings 3-4): C Markov chains each run L
 * Metropolis steps at the temperature of the current level; a reduction then
 * finds the chain with the lowest f, every chain restarts from it, and the
 * temperature is cooled geometrically, T <- rho T (Sec. 2.1, Step 5).
 *
 * Conventions for every entry point below
 *   - Host pointers are plain host memory owned by the caller; the library
 *     copies what it needs before returning (or, for outputs, writes into them
 *     before returning).  Device pointers are named d_* and are caller-owned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a handle is enqueued on its stream.
 *   - Every call returns sa_status.  After SA_ECUDA, SA_ETIMEOUT or
 *     SA_ENUMERIC a handle only accepts sa_destroy (further calls give
 *     SA_ESTATE).  Handles are not thread-safe.
 *   - Layouts: vectors of length n are contiguous doubles; matrices are
 *     row-major.
 */
#ifndef SA_GB300_H
#define SA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SA_OK = 0,
    SA_EINVAL = 1,   /* an argument is out of range (see each call) */
    SA_ENOMEM = 2,   /* a device or host allocation failed */
    SA_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    SA_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    SA_ENUMERIC = 5, /* the best state of a level is not finite */
    SA_ESTATE = 6    /* the handle is in an error state or the call is out of order */
} sa_status;

/* Cost functions.  Schwefel is the paper's normalised form (Sec. 4.1,
 * f = -(1/n) sum x_i sin sqrt|x_i|); Ackley, Rastrigin and Rosenbrock are the
 * Appendix tests 1, 13 and 14 (Rosenbrock in its standard x_{i+1} - x_i^2
 * form).  The rotated variants evaluate the same formula at y = Q x for an
 * orthogonal Q (an extension: the paper has no rotated costs).  SA_BRANIN ..
 * SA_FOXHOLES are the Appendix's Tests 2-12 and 15-19, evaluated in full in
 * FP64 at every step (SA_FP64 only; no local difference, no gradient).  The
 * cosine mixture (Test 3) is sum x_i^2 - 0.1 sum cos(5 pi x_i) and Griewank
 * (Test 8) 1 + sum x_i^2 / 4000 - prod cos(x_i / sqrt i): their standard forms,
 * which the printed minima fit.  Branin, Dekkers-Aarts, Easom, Goldstein-Price,
 * Himmelblau and the six-hump camel need n = 2; modified Langerman, Shekel and
 * the modified Shekel foxholes (Tests 11, 18, 19) take their A and c as a
 * table (sa_problem.table). */
typedef enum {
    SA_SCHWEFEL = 0,
    SA_RASTRIGIN = 1,
    SA_ACKLEY = 2,
    SA_ROSENBROCK = 3,
    SA_ROT_RASTRIGIN = 4,
    SA_ROT_SCHWEFEL = 5,
    SA_BRANIN = 6,          /* Test 2 */
    SA_COSINE_MIXTURE = 7,  /* Test 3 */
    SA_DEKKERS_AARTS = 8,   /* Test 4 */
    SA_EASOM = 9,           /* Test 5 */
    SA_EXPONENTIAL = 10,    /* Test 6: -exp(-sum x_i^2 / 2) */
    SA_GOLDSTEIN_PRICE = 11, /* Test 7 */
    SA_GRIEWANK = 12,       /* Test 8 */
    SA_HIMMELBLAU = 13,     /* Test 9 */
    SA_LEVY_MONTALVO = 14,  /* Test 10 */
    SA_LANGERMAN = 15,      /* Test 11: -sum_i c_i exp(-D_i / pi) cos(pi D_i), D_i = |x - a_i|^2 */
    SA_MICHALEWICZ = 16,    /* Test 12, m = 10 */
    SA_SALOMON = 17,        /* Test 15 */
    SA_SIX_HUMP_CAMEL = 18, /* Test 16 */
    SA_SHUBERT = 19,        /* Test 17 */
    SA_SHEKEL = 20,         /* Test 18: -sum_i 1 / (D_i + c_i) */
    SA_FOXHOLES = 21        /* Test 19: the same sum over the foxholes table */
} sa_cost;

enum { SA_REFLECT = 0, SA_CLIP = 1 };                 /* box handling of a move */
enum { SA_FP64 = 0, SA_FP32 = 1, SA_MIXED_BF16 = 2 }; /* arithmetic of the sweep */
/* local minimiser of the hybrid SA (the adaptive Nelder-Mead: Gao & Han's coefficients) */
enum { SA_POLISH_PGD = 0, SA_POLISH_NELDER_MEAD = 1, SA_POLISH_NELDER_MEAD_ADAPTIVE = 2 };
/* Move of the selected coordinate (Sec. 2.1 Step 2: "a random number to modify the selected
 * coordinate"): a Gaussian step sigma_frac (u_d - l_d) sqrt(T / T0) z (Box-Muller, cosine
 * branch, then the box rule), or a uniform redraw x_d' = l_d + u2 (u_d - l_d) with the
 * block's second uniform. */
enum { SA_PROPOSAL_GAUSSIAN = 0, SA_PROPOSAL_UNIFORM = 1 };

typedef struct {
    int32_t cost;        /* sa_cost */
    const double* Q;     /* host, n x n row-major, orthogonal; NULL unless rotated */
    const double* table; /* host, table_rows x (n + 1): row i = (a_i1 .. a_in, c_i); NULL unless
                            SA_LANGERMAN, SA_SHEKEL or SA_FOXHOLES */
    int32_t table_rows;  /* 1 .. 4096 for those costs, else 0 */
} sa_problem;

typedef struct {
    const double* lo; /* host, [n]: l_k */
    const double* hi; /* host, [n]: u_k, hi[k] >= lo[k] */
} sa_box;

/* Annealing schedule (Sec. 2.1 Step 5; Listing 3 host loop). */
typedef struct {
    double T0;          /* initial temperature, > 0 */
    double rho;         /* cooling factor, 0 < rho < 1 */
    double T_min;       /* stop temperature (used when levels == 0), 0 < T_min < T0 */
    int32_t levels;     /* > 0: run exactly this many levels; 0: the do-while of Listing 3 */
    double sigma_frac;  /* Gaussian step sigma = sigma_frac (u_d - l_d) sqrt(T / T0), > 0 */
    int32_t boundary;   /* SA_REFLECT (reflect once, then clip) or SA_CLIP */
    int32_t precision;  /* SA_FP64 or SA_FP32 (state in FP32, argmin in FP64) */
    int32_t surrogate;  /* 0: Metropolis; 1: delayed acceptance with the learned surrogate
                           (rotated costs, SA_FP32, sa_create only; see sa_da_trace) */
    int32_t polish_k;   /* hybrid SA: after the last level, polish the polish_k best final
                           states (0..1024) with the method polish_method names; the best
                           polished point becomes the incumbent if it is lower (0 = off) */
    int32_t trace_levels; /* record accept bits of the first trace_levels levels (0 = off) */
    int32_t cost_repeat;  /* rotated costs: evaluate each energy difference this many times
                             (0 or 1 = once; more only to emulate a costlier f, results unchanged) */
    int32_t independent;  /* 0: synchronous (Sec. 2.2.2: every level restarts all chains from the
                             best one); 1: asynchronous (Sec. 2.2.1: no exchange, every chain
                             continues from its own state; the levels' minima still give the
                             incumbent).  One chain is the sequential algorithm (Sec. 2.1). */
    int32_t exchange_every; /* m > 1: synchronous exchange only after levels m-1, 2m-1, ...; the
                               chains continue their own states in between (0 or 1: every level) */
    int32_t polish_method;  /* SA_POLISH_PGD: sa_polish (max_iter 1000, tol 1e-10);
                               SA_POLISH_NELDER_MEAD(_ADAPTIVE): sa_nelder_mead with step_frac = sigma_frac
                               sqrt(T_last / T0) (the last level's step scale), max_iter
                               200 (n + 1), ftol 1e-12, xtol 1e-10 (n <= 4096) */
    int32_t proposal;       /* SA_PROPOSAL_GAUSSIAN (the default) or SA_PROPOSAL_UNIFORM (not with
                               the surrogate) */
    int32_t crossover;      /* 0: an exchange restarts every chain from the minimum (Sec. 2.2.2);
                               1: stochastic crossover (a reading of the SOS scheme cited in Sec. 2.2):
                               chain c restarts from chain j's final state, j drawn with probability
                               exp(-(F_j - F_min) / T) / Z at the finished level's temperature
                               (Philox stream tag 5).  Every chain's F is then exact in FP64 at
                               every level.  Not with the surrogate, independent chains or
                               sa_set_chain_offset */
} sa_schedule;

typedef struct {
    int64_t steps;        /* Metropolis steps run so far: chains * L * levels_done */
    int64_t accepts;      /* accepted moves so far */
    int32_t levels_done;  /* levels completed */
    int32_t levels_total; /* levels of the schedule */
    double f_level;       /* F of the restart point chosen by the last level */
    int64_t argmin;       /* chain index p* chosen by the last level */
    int64_t h2d_bytes;    /* bytes this handle copied host -> device so far */
    int64_t d2h_bytes;    /* bytes this handle copied device -> host so far */
    int64_t t_start_ns;   /* device clock (ns) when level 0 of the current run started */
    int64_t rechecks;     /* rotated costs: decisions re-taken in FP64 so far (0 otherwise) */
    int64_t true_evals;   /* energy differences of f evaluated (= steps unless delayed acceptance) */
} sa_stats;

typedef struct sa_handle sa_handle;

/* Fill *s with the defaults: T0 = 100, rho = 0.9, T_min = 0, levels = 50,
 * sigma_frac = 0.1, SA_REFLECT, SA_FP64, no tracing. */
void sa_default_schedule(sa_schedule* s);

/* Levels run by the do-while of Listing 3: the smallest K >= 1 with
 * T0 rho^K <= T_min (temperatures by repeated multiplication).  Returns -1 on
 * a bad argument.  T0 = 1000, rho = 0.99, T_min = 0.01 gives 1146 (Table 1). */
int32_t sa_levels_for(double T0, double rho, double T_min);

/*
 * Create a solver for one problem (Eq. 1) with `chains` Markov chains of `L`
 * steps per level.  Copies box, Q and the schedule to device memory that the
 * handle owns (stream-ordered allocation on `stream`).  Launches nothing.
 * Rotated costs (SA_ROT_*) need precision SA_FP32: each chain keeps y = Q x
 * as an FP32 pair (hi + lo), updates it by rank-1 corrections on accepted
 * moves, decides in FP32 with a rigorous error bound and re-takes in FP64
 * every decision that falls inside the bound (sa_stats.rechecks counts them);
 * level 0 transforms the initial points as one FP64 product X0 Q^T.  They
 * hold 12 chains n bytes of level-0 buffers and 24 n^2 bytes of copies of Q.
 * Errors: SA_EINVAL if n < 1, chains < 1, L < 1, lo[k] > hi[k] or not finite,
 * T0 <= 0, rho not in (0,1), levels < 0, levels == 0 and T_min not in
 * (0, T0), sigma_frac <= 0, unknown cost/boundary/precision, a rotated cost
 * without Q, with a non-finite Q entry, with n^2 > 2^28 or with precision other
 * than SA_FP32, surrogate not 0 or 1 (1: rotated costs only), independent not 0
 * or 1, exchange_every < 0, a surrogate with independent or exchange_every > 1,
 * or chains > 2^31 - 1;
 * SA_ENOMEM / SA_ECUDA on allocation or copy failure.  *out is NULL on error.
 */
sa_status sa_create(const sa_problem* problem, const sa_box* box, int32_t n, int64_t chains,
                    int32_t L, const sa_schedule* schedule, uint64_t seed, void* stream,
                    sa_handle** out);

/*
 * Create one solver for num_problems independent problems that share L and
 * the schedule (each problem p has its own cost, box, n[p] and chains[p]).
 * Every level runs all problems' sweeps in one graph launch (problems are
 * grouped by dimension; the groups' kernels run concurrently) followed by one
 * argmin/restart launch over all problems.  Problem p draws its randomness
 * from Philox counter word 3 = p, so its result equals a single-problem run
 * with that problem index.  Arguments are arrays of length num_problems with
 * the meaning and checks of sa_create.  Errors: as sa_create, plus SA_EINVAL
 * if num_problems < 1.
 */
sa_status sa_create_batch(const sa_problem* problems, const sa_box* boxes, const int32_t* n,
                          const int64_t* chains, int32_t num_problems, int32_t L,
                          const sa_schedule* schedule, uint64_t seed, void* stream,
                          sa_handle** out);

/*
 * Pick the block shape (chains per block) and the number of steps evaluated
 * together per chain for each dimension group by timing the level-0 sweep of
 * that group with each candidate (results do not depend on the choice).
 * Leaves the handle rewound to level 0 and re-captures its graphs; *ms_out
 * (may be NULL) receives the sum of the chosen level-0 sweep times.
 * Synchronises.  Errors: SA_ESTATE on a failed handle, SA_ECUDA.
 */
sa_status sa_autotune(sa_handle* h, double* ms_out);

/*
 * Describe the launch groups of a handle as a JSON array (kind, problems,
 * n_max, block, smem, unroll, work items) into buf (NUL-terminated, truncated
 * to len).  Returns the full length of the description, or -1 on NULL h.
 */
int32_t sa_describe(const sa_handle* h, char* buf, size_t len);

/*
 * Run up to `levels` further temperature levels (-1 = all remaining).  Each
 * level is: Metropolis sweep of every chain (Listing 4), reduction to the
 * lowest-f chain with lowest-index tie-break, restart and cooling (Listing 3).
 * Asynchronous: the work is enqueued on the handle's stream and the call
 * returns; errors raised on the device surface at the next sa_best.
 * Errors: SA_ESTATE on a failed handle or when no level remains,
 * SA_EINVAL if levels == 0 or < -1, SA_ECUDA on a launch failure.
 */
sa_status sa_run(sa_handle* h, int32_t levels);

/*
 * Rewind the handle to level 0 (same problem, schedule and seed), so that the
 * next sa_run repeats the run from its random initial points.  Asynchronous
 * (stream-ordered device writes only).  Errors: SA_ESTATE on a failed handle.
 */
sa_status sa_reset(sa_handle* h);

/*
 * Run up to `levels` further levels like sa_run, but launch the kernels one
 * by one (no graph) with CUDA events around them on the handle's stream, and
 * return per level the sweep kernel's time (sweep_ms[l]) and the whole level's
 * time (level_ms[l]) in milliseconds; arrays host [levels], may be NULL.  When
 * the call starts at level 0, level_ms[0] also holds the run's start-up work
 * (the initial states, their costs and, for rotated costs, the transform
 * Y0 = X0 Q^T).  Synchronises.  Errors as sa_run.
 */
sa_status sa_profile(sa_handle* h, int32_t levels, double* sweep_ms, double* level_ms);

/*
 * Synchronise the handle's stream and return the incumbent: the best restart
 * point over all levels run so far (x_out: host [n], f_out: host scalar, both
 * may be NULL) and statistics (st may be NULL).  f is evaluated in FP64.
 * `problem` must be 0 for a single-problem handle.
 * Errors: SA_ESTATE before the first level or on a failed handle, SA_EINVAL
 * on a bad problem index, SA_ECUDA / SA_ETIMEOUT / SA_ENUMERIC from the device.
 */
sa_status sa_best(sa_handle* h, int32_t problem, double* x_out, double* f_out, sa_stats* st);

/*
 * Per-level log of one problem (synchronises): for each completed level l <
 * cap, argmin[l] = p*, f_level[l] = F(x_{p*}) in FP64, f_inc[l] = the
 * incumbent after level l, t_ns[l] = device clock (ns) when level l ended.
 * Any output may be NULL.  *count = levels written.
 */
sa_status sa_level_log(sa_handle* h, int32_t problem, int64_t* argmin, double* f_level,
                       double* f_inc, int64_t* t_ns, int32_t cap, int32_t* count);

/*
 * Accept bits recorded for traced level `level` (< trace_levels, completed):
 * bits_out[c * words + s / 32] bit (s % 32) = 1 iff step s of chain c was
 * accepted, words = ceil(L / 32).  `nwords` must be >= chains * words.
 */
sa_status sa_trace(sa_handle* h, int32_t level, uint32_t* bits_out, size_t nwords);

/*
 * Final states of the last completed traced level (synchronises): X_out
 * host [chains * n] (chain-major), F_out host [chains] f in FP64.  Only
 * available when that level was traced.
 */
sa_status sa_trace_states(sa_handle* h, int32_t level, double* X_out, double* F_out);

/*
 * Delayed acceptance (schedule.surrogate == 1; an extension, the paper has no
 * surrogate).  Each step, every chain's proposal x' first passes stage 1 with
 * probability min(1, exp(-(f~(x') - f~(x)) / T)) on the surrogate f~ (Christen
 * & Fox 2005), drawn from word 0 of the Philox block (step, level, chain,
 * problem) of stream tag 3; only survivors have their true difference dF
 * evaluated, and are accepted with probability min(1, exp(-(dF - (f~(x') -
 * f~(x))) / T)) using the sweep's u3.  f~ = mu + sigma MLP((x - mid) / half),
 * the network of sa_mlp_*, is re-initialised at level 0 of every run (seed of
 * the handle), trained before each later level by 128 Adam steps (batches of
 * 4096, half drawn from a ring buffer of the last ~2^20 chain states -- taken 4
 * times per level, evenly spaced -- and half from the previous level's states,
 * with their values; targets standardised by the buffer's mean and deviation)
 * and frozen
 * during the level.  sa_da_trace returns, for a traced completed level, the
 * surrogate's value at every chain's start state (ft0_out: host [chains]) and
 * at every proposal (ftp_out: host [L * chains], step-major); either may be
 * NULL.  Checkpoints are not available for such handles (SA_EINVAL).
 */
sa_status sa_da_trace(sa_handle* h, int32_t level, float* ft0_out, float* ftp_out);

/*
 * The surrogate network of the last completed level of a delayed-acceptance
 * handle (the one that level used: training for the next level runs at its
 * start), so a test can recompute f~ = mu + sigma MLP(bf16((x - mid) / half))
 * on its own.  All outputs are host buffers and may be NULL:
 *   params_out    [sa_mlp_param_count(n)] FP32 parameters (layout of sa_mlp_*)
 *   ms_out        [2] mu and sigma, the standardisation of the targets
 *   mid_out       [n] mid-points of the box, inv_half_out [n] 1 / half-widths
 * Errors: SA_EINVAL if h is not a surrogate handle or no level has run;
 * SA_ESTATE after an earlier error; SA_ECUDA.
 */
sa_status sa_da_network(sa_handle* h, float* params_out, float* ms_out, float* mid_out, float* inv_half_out);

/*
 * Chains sharded over several solvers (e.g. one per GPU), with the exchange of
 * Sec. 2.2.2 done by the caller between levels:
 *   sa_set_chain_offset  before the first level: this handle's chains are the
 *                        global chains offset .. offset + chains - 1 (Philox
 *                        counter word 2 = global index), so a sharded run
 *                        draws exactly the numbers of the unsharded one.
 *                        Single-problem handles; offset + chains <= 2^32.
 *   sa_restart_point     after a level: this shard's restart point (the
 *                        lowest-F chain of the shard, x_out host [n], may be
 *                        NULL) and its FP64 value.
 *   sa_set_restart       after the exchange: make (x, f) -- the lowest f over
 *                        all shards, lowest global index `argmin` on ties --
 *                        the restart point of the next level, update the
 *                        incumbent and the level log.  x must lie in the box.
 * With these, running the shards level by level and exchanging the (f, index)
 * minimum gives the unsharded run's levels bit for bit.  All three
 * synchronise the handle's stream.  Errors: SA_EINVAL on a bad argument,
 * SA_ESTATE before the first level (restart calls) or after it (offset).
 */
sa_status sa_set_chain_offset(sa_handle* h, int64_t offset);
sa_status sa_restart_point(sa_handle* h, int32_t problem, double* x_out, double* f_out);
sa_status sa_set_restart(sa_handle* h, int32_t problem, const double* x, double f, int64_t argmin);

/*
 * Serialise the state between levels (restart point, incumbent, level index,
 * counters) into buf.  With buf == NULL, *len receives the size needed.
 * Errors: SA_EINVAL if *len is too small, or for handles whose chains carry
 * their own state across levels (independent, exchange_every > 1) or that use
 * the surrogate.
 * Synchronises.
 */
sa_status sa_checkpoint(sa_handle* h, void* buf, size_t* len);

/* Restore a checkpoint taken from a handle created with identical arguments.
 * Continuing reproduces the uninterrupted run bit for bit (the random streams
 * are counter-based on (step, level, chain)).  Errors: SA_EINVAL on a size,
 * version or fingerprint mismatch. */
sa_status sa_restore(sa_handle* h, const void* buf, size_t len);

/* Release the handle and its device memory (stream-ordered).  NULL is a no-op. */
void sa_destroy(sa_handle* h);

const char* sa_strerror(sa_status s);

/*
 * Local minimiser of the hybrid SA (the paper polishes SA points with
 * Nelder-Mead, Sec. 4.2 / Table 10; this library uses box-projected gradient
 * descent): from each of k start points x0[j*n .. j*n+n) (host), iterate
 * x <- P_I(x - alpha grad f(x)) in FP64 with alpha halved from 1 (at most 30
 * times) until f(x_new) <= f(x) + 1e-4 grad f . (x_new - x); stop when the
 * projected gradient's infinity norm is below tol, when no step decreases
 * f, or after max_iter iterations.  Writes the final points to x_out (host
 * [k*n]), their values to f_out (host [k]) and the iteration counts to
 * iters_out (host [k], may be NULL).  Rotated costs take Q (host, n x n
 * row-major) and use grad f = Q^T g'(Q x); separable costs need Q == NULL.
 * Allocates its device buffers stream-ordered; synchronises `stream`.
 * Errors: SA_EINVAL on n < 1, k not in [1, 1024], a bad box, max_iter < 0,
 * tol < 0, a NULL array, Q missing for a rotated cost (or given for a
 * separable one), a non-finite Q entry or n^2 > 2^28; SA_ENOMEM; SA_ECUDA.
 */
sa_status sa_polish(int32_t cost, int32_t n, const double* lo, const double* hi, const double* Q, int32_t k,
                    const double* x0, int32_t max_iter, double tol, double* x_out, double* f_out,
                    int32_t* iters_out, void* stream);

/*
 * Nelder-Mead, the local minimiser of the paper's hybrid SA (Sec. 4.2, Table
 * 10), in the standard form (Lagarias, Reeds, Wright & Wright, SIAM J. Optim.
 * 1998): reflection 1, expansion 2, outside and inside contraction 1/2,
 * shrink 1/2 towards the best vertex -- or, with adaptive = 1, Gao & Han's
 * dimension-dependent coefficients (expansion 1 + 2/n, contractions
 * 3/4 - 1/(2n), shrink 1 - 1/n).  Every trial point is c + a (c - v_h) for the
 * centroid c and the worst vertex v_h, clipped into the box.  From each of k start points x0[j*n .. j*n+n) (host) the simplex is
 * x0 and x0 + delta_i e_i, delta_i = step_frac (u_i - l_i) (minus that if plus
 * leaves the box); vertices rank by (f, slot) -- best = lowest f, then lowest
 * slot; worst and second worst = highest f, then highest slot.  Stops when
 * f_worst - f_best <= ftol max(1, |f_best|) and every vertex is within
 * xtol (u_i - l_i) of the best in every coordinate i, or after max_iter
 * iterations.  FP64.  Writes the best vertices to x_out (host [k*n]), their
 * values to f_out (host [k]) and the iteration counts to iters_out (host [k],
 * may be NULL).  Rotated costs take Q (host, n x n row-major), the others
 * Q == NULL; the table costs take table (host, table_rows x (n + 1), as in
 * sa_problem), the others table == NULL.  Every cost of sa_cost is accepted.  Device workspace ((n+1) n doubles per start: the simplex)
 * is allocated stream-ordered; synchronises `stream`.  Above 64 coordinates
 * the centroid comes from a running vertex sum (summed afresh after a shrink
 * and every n+1 iterations), so results differ from a sequential
 * implementation by rounding there as well as in f.
 * Errors: SA_EINVAL on n < 1 or n > 4096, k not in [1, 1024], a bad box,
 * step_frac not in (0, 1], max_iter < 0, ftol or xtol negative or NaN, a NULL
 * array, adaptive not 0 or 1, Q or the table missing where the cost needs it (or given where it
 * does not), a non-finite Q or table entry, n != 2 for a two-variable test, or
 * a workspace above 4 GiB; SA_ENOMEM; SA_ECUDA.
 */
sa_status sa_nelder_mead(int32_t cost, int32_t n, const double* lo, const double* hi, const double* Q,
                         const double* table, int32_t table_rows, int32_t k, const double* x0, double step_frac,
                         int32_t max_iter, double ftol, double xtol, int32_t adaptive, double* x_out,
                         double* f_out, int32_t* iters_out, void* stream);

/*
 * Kernel-level entry point: tensor-core GEMM D = A . B^T with A [M x K] and
 * B [N x K] row-major BF16 (K contiguous; leading dimensions lda, ldb in
 * elements, rows 16-byte aligned) and D [M x N] row-major FP32 (leading
 * dimension ldd), FP32 accumulation (tcgen05 on sm_103a).  Used by the
 * rotated-cost transform and the surrogate network; exposed for testing.
 * M must be a multiple of 128, N of 64, K of 64, ldd of 4.  d_status (device
 * int, may be NULL) receives SA_ETIMEOUT if a bounded wait inside the kernel
 * expires.  Asynchronous.  Errors: SA_EINVAL on shapes, alignment or NULL.
 */
sa_status sa_gemm_bf16(const void* d_A, int32_t lda, const void* d_B, int32_t ldb, float* d_D, int32_t ldd,
                       int32_t M, int32_t N, int32_t K, int32_t* d_status, void* stream);

/*
 * The learned surrogate of the delayed-acceptance sweep (an extension: the
 * paper has no surrogate):  f~(x) = w3 . g(W2 g(W1 x + b1) + b2) + b3 with
 * g(z) = z Phi(z) (erf-form GELU) and hidden widths 512 and 512, fitted to
 * the mean squared error (1/2B) sum_b (f~(x_b) - t_b)^2 with Adam (Kingma & Ba,
 * ICLR 2015).  Parameters are one FP32 device vector of sa_mlp_param_count(n)
 * elements laid out W1 [512 x n] (row-major), b1 [512], W2 [512 x 512],
 * b2 [512], w3 [512], b3 [1].  The matrix products run on the tensor cores
 * (BF16 operands, FP32 accumulation); everything else in FP32.  erf in g is
 * Hastings' rational approximation (Abramowitz and Stegun 7.1.26, |error| <=
 * 1.5e-7).  sa_mlp_forward runs both layers and the head in one kernel for
 * n <= 128 (the hidden layer never leaves the chip) and as two GEMMs above.
 *   sa_mlp_param_count  number of parameters (-1 if n < 1)
 *   sa_mlp_init         He-normal weights from Philox (stream tag 2 of seed), zero biases
 *   sa_mlp_forward      d_y[b] = f~(d_X[b]) for B rows of d_X [B x n] (FP32, device)
 *   sa_mlp_loss_grad    d_grad = dL/dparams, *d_loss = L (FP32 device scalar, may be NULL)
 *   sa_mlp_adam         one Adam step at step >= 1: moments d_m, d_v (device, count each) updated
 * All are asynchronous on `stream`; forward and loss_grad allocate their
 * workspace stream-ordered.  Errors: SA_EINVAL on NULL pointers, n not in
 * [1, 4096], B < 1, count < 1, step < 1 or hyper-parameters out of range;
 * SA_ENOMEM; SA_ECUDA.
 */
int64_t sa_mlp_param_count(int32_t n);
sa_status sa_mlp_init(float* d_params, int32_t n, uint64_t seed, void* stream);
sa_status sa_mlp_forward(const float* d_params, int32_t n, const float* d_X, int32_t B, float* d_y, void* stream);
sa_status sa_mlp_loss_grad(const float* d_params, int32_t n, const float* d_X, const float* d_t, int32_t B,
                           float* d_grad, float* d_loss, void* stream);
sa_status sa_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int64_t count, int32_t step,
                      float lr, float beta1, float beta2, float eps, void* stream);

/*
 * Kernel-level entry point: the rotated costs' level-0 transform (the candidate
 * transform y = Q x of the mixed-precision path, for rotated costs f(x) = F(Q x))
 * on the tensor cores, for a batch of states at once: Y = X Q^T, each element
 * as a double-float pair.  Every row of X and of Q is split into six slices of
 * integers of magnitude <= 128 on a common power-of-two scale per row, held
 * exactly in BF16; each product of two slices accumulates exactly in FP32 (its
 * partial sums are integers below 2^24), and the 21 slice pairs of order <= 7
 * are summed into the pairs.  Against the exact product each element errs by at
 * most 7.1 n 2^(E + F - 48) (the dropped slice pairs and the slices'
 * remainders), 2^E > max |x| of its row and 2^F > max |q| of its coordinate,
 * plus the pairs' rounding, 2^-42 sum_j |x_j q_j|, while 2^(E + F) >= 2^-72:
 * smaller scales fall below the FP32 range of the pairs and are flushed.
 *   d_X   device, FP32 [rows x n], row-major (the states)
 *   d_Q   device, FP64 [n x n], row-major
 *   d_Y   device, FP32 [rows x n x 2]: element (r, i) as (hi, lo), hi + lo ~ (X Q^T)[r][i]
 *   d_status  device int (may be NULL): SA_ETIMEOUT if a bounded wait of the GEMMs ran out
 * Shapes: n a multiple of 64, n <= 1024, rows a multiple of 128.  Allocates its
 * workspace stream-ordered.  Errors: SA_EINVAL (NULL pointer, other shapes),
 * SA_ENOMEM, SA_ECUDA.
 */
sa_status sa_rotate_rows(const float* d_X, int64_t rows, int32_t n, const double* d_Q, float* d_Y,
                         int32_t* d_status, void* stream);

/*
 * Kernel-level entry point: Philox4x32-10 (Salmon et al., SC'11) blocks for
 * counters (c0 + i, c1, c2, c3), i = 0..count-1, with key (key0, key1);
 * block i goes to d_out[4 i .. 4 i + 3].  d_out: device, >= 4 count uint32.
 * Errors: SA_EINVAL if count < 0 or d_out == NULL with count > 0.
 */
sa_status sa_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t key0,
                         uint32_t key1, int64_t count, uint32_t* d_out, void* stream);

/*
 * Kernel-level entry point: the reduction of Sec. 2.2.2 on its own.  Finds
 * p = argmin_c d_F[c] over c < count (lowest index among equal values; NaN
 * never wins) and writes it to *d_index and d_F[p] to *d_value (device).
 * d_scratch: device, >= sa_argmin_scratch_bytes(count) bytes, caller-owned.
 * Errors: SA_EINVAL if count < 1 or a pointer is NULL.
 */
size_t sa_argmin_scratch_bytes(int64_t count);
sa_status sa_argmin_f64(const double* d_F, int64_t count, int64_t* d_index, double* d_value,
                        void* d_scratch, void* stream);

/*
 * sa_argmin_f64 for callers that cannot allocate device memory (the paper has
 * no counterpart: this is a library convenience).  Some callers cannot hand
 * over a scratch buffer -- code inside a host framework whose allocator owns
 * the device's memory, latency-critical loops where cudaMalloc would
 * synchronise the device, or code that must not run out of memory mid-run.
 * This call allocates nothing: its scratch is a fixed array of
 * SA_ARGMIN_STATIC_MAX_COUNT / 2048 * 16 bytes (1 MiB) inside the library,
 * held by every GPU that loads the library until the process exits.
 * Same inputs, outputs and result as sa_argmin_f64.
 *   - count must be <= SA_ARGMIN_STATIC_MAX_COUNT; larger gives SA_EINVAL.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.
 *   - A device reset (cudaDeviceReset) destroys the array and the looked-up
 *     address goes stale: a process that resets a device does not call this
 *     function on that device again.
 *   - All calls share the array: calls whose kernels overlap on the GPU
 *     (other streams, other host threads) race and may return wrong results.
 *     Order such calls on one stream.
 * Errors: SA_EINVAL on count < 1, count too large or a NULL pointer;
 * SA_ECUDA if the address lookup or a launch fails.
 */
#define SA_ARGMIN_STATIC_MAX_COUNT ((int64_t)1 << 27)

/*
 * Measurement entry point (the paper has no counterpart): the throughput of
 * one arithmetic pipe of the current GPU, for the roofline of the sweep
 * (the minimum over pipes of rate / algorithmic operations per step).  One
 * kernel per operation runs a full wave of blocks of 256 threads, each
 * thread eight independent chains of `op` for iters x 4 rounds, timed with
 * CUDA events; the SM clock it ran at is read from one block (SM cycles over
 * global-timer nanoseconds).
 *   op                    one of sa_pipe_op: the SFU approximations the sweep
 *                         uses, 32x32->64-bit products (IMAD_WIDE), their high
 *                         and low halves, 3-input logic, FP32 and FP64
 *                         fused multiply-adds, and whole Philox4x32-10 blocks
 *   iters                 1 .. 2^20 (a few thousand give stable rates)
 *   *ops_per_clock_per_sm operations (Philox: blocks) per SM clock cycle, per SM
 *   *ops_per_second       the same per second of the whole GPU, from CUDA
 *                         events around the launch (may be NULL)
 * Synchronous: returns after the measurement; allocates a small stream-ordered
 * scratch.  Errors: SA_EINVAL on a bad op or iters or a NULL output;
 * SA_ENOMEM; SA_ECUDA.
 */
typedef enum {
    SA_PIPE_SIN = 0, SA_PIPE_COS = 1, SA_PIPE_LG2 = 2, SA_PIPE_EX2 = 3, SA_PIPE_SQRT = 4, SA_PIPE_RSQRT = 5,
    SA_PIPE_IMAD_WIDE = 6, SA_PIPE_IMAD_HI = 7, SA_PIPE_IMAD_LO = 8, SA_PIPE_LOP3 = 9, SA_PIPE_FFMA = 10,
    SA_PIPE_DFMA = 11, SA_PIPE_PHILOX = 12, SA_PIPE_COUNT = 13
} sa_pipe_op;
sa_status sa_pipe_rate(int32_t op, int32_t iters, void* stream, double* ops_per_clock_per_sm,
                       double* ops_per_second);
sa_status sa_argmin_f64_static(const double* d_F, int64_t count, int64_t* d_index, double* d_value,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SA_GB300_H */
