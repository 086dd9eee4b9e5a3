// sa_internal.h -- descriptors shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sa {

// Philox stream tags: key = (seed_lo, seed_hi ^ tag).
constexpr uint32_t kTagSweep = 0u;
constexpr uint32_t kTagInit = 1u;
constexpr uint32_t kTagCrossover = 5u;

// Scalars kept per problem in device memory.
enum ScalarSlot : int {
    kFBest = 0,   // F(x_best) in FP64 (restart point of the next level)
    kFInc = 1,    // incumbent value
    kS1 = 2,      // Ackley: sum x_best^2 (FP64)
    kS2 = 3,      // Ackley: sum cos(2 pi x_best) (FP64)
    kFRot = 4,    // rotated costs: F at the pair Q x_best (restart value of the next level)
    kNumScalars = 8
};

// One problem of a (possibly batched) run; lives in device memory.
struct ProbDev {
    int32_t cost, n;
    int64_t chains;
    int64_t chain_base;   // offset of this problem's chains in per-chain arrays
    int64_t x_base;       // offset (elements) of this problem's [n][chains] state block
    uint32_t pid;         // Philox counter word 3
    uint32_t cid0;        // global id of chain 0 (Philox counter word 2 = cid0 + chain; a shard's offset)
    int32_t nblk_argmin;  // blocks of the argmin kernel for this problem
    int32_t uniform;      // 1: every coordinate has the same [lo, hi] (scalars below are used)
    int32_t unroll;       // steps evaluated together per chain in the FP32 sweep (1, 2 or 4)
    int32_t rand_batch;   // FP32 chain-per-thread sweep: steps whose randomness is drawn as one batch (1 or 16)
    int32_t warp_mode;    // FP32 sweep: 0 = one chain per thread, 1 = one chain per warp
    float kappa;          // warp mode: bound on the FP32 error of one accepted step's dF
    float lo_u, hi_u, sig_u;  // the uniform box and sigma_frac (hi - lo) in FP32
    const double* lo;     // [n]
    const double* hi;     // [n]
    const double* sig;    // [n] sigma_frac (hi - lo)
    const float* lo32;    // [n] lo rounded up to FP32
    const float* hi32;    // [n] hi rounded down to FP32
    const float* sig32;   // [n]
    double* x_best64;     // [n] restart point (FP64 path)
    float* x_best32;      // [n] restart point (FP32 path)
    double* x_inc;        // [n] incumbent
    double* scal;         // [kNumScalars]
    unsigned long long* level_min;  // candidate threshold of the current level (ordered key)
    unsigned int* done;   // last-block-done counter of the argmin
    double* part_val;     // [max(nblk_argmin, items)] partial minima
    int64_t* part_idx;    // [max(nblk_argmin, items)]
    int32_t items;        // batched level kernel: the problem's tiles in the launch
    int64_t* log_argmin;  // [levels]
    double* log_f;        // [levels]
    double* log_finc;     // [levels]
    long long* log_t;     // [levels] device clock (ns) at the end of the level
    unsigned long long* accepts;  // running count of accepted moves
    // Tests 11, 18, 19: rows (a_i1 .. a_in, c_i) (NULL otherwise)
    const double* table;  // [table_rows][n + 1]
    int32_t table_rows;
    // rotated costs f(x) = F(Q x) (NULL otherwise)
    const double* q64;    // [n][n] Q row-major (FP64)
    const double* qt64;   // [n][n] Q transposed: qt64[d * n + i] = Q[i][d]
    const float* qt_hi;   // [n][n] FP32 part of qt64
    const float* qt_lo;   // [n][n] FP32 remainder: qt64 - qt_hi rounded to FP32
    float* ybest_hi;      // [n] Q x_best as a double-float pair (hi + lo)
    float* ybest_lo;      // [n]
    const float* x0;      // [chains][n] level-0 states (FP32)
    const float2* y0;     // [chains][n] Q x0 as (hi, lo) pairs
    unsigned long long* rechecks;  // running count of FP64 re-checked decisions
    unsigned int* rot_done;  // last-block-done counter of the restart transform
    double* rot_part;     // [ceil(n / 128)] its partial sums
    float qmax;           // max |Q_ij| rounded up to FP32
    float ymax;           // bound on |(Q x)_i| over the box: max_i sum_j |Q_ij| max(|l_j|, |u_j|)
};

// Device-resident run state shared by all problems of a handle.
struct RunDev {
    int32_t level;   // level index the next sweep runs
    int32_t status;  // sa_status raised on the device (0 = ok)
    long long t_start;  // device clock (ns) when the current run's level 0 started
    int32_t probs_done;  // batched level kernel: problems whose level has ended in the current launch
    int32_t pad;
};

struct WorkItem {
    int32_t problem;
    int32_t count;   // chains in this tile
    int64_t c0;      // first chain (problem-local index)
    int32_t lanes;   // batched level kernel: lanes per chain (2, 4, 8), or 0 for one chain per thread
    int32_t slot;    // batched level kernel: the tile's index among its problem's tiles
};

struct SweepArgs {
    const ProbDev* probs;
    const WorkItem* items;
    RunDev* run;
    const double* T_tab;   // [levels] temperature of each level (repeated multiplication)
    const double* s_tab;   // [levels] sqrt(T_l / T0)
    double* F;             // [total chains] FP64 value of each chain's final state (+inf: not a candidate)
    float* X32;            // state blocks, [n][chains] per problem (FP32 path)
    double* X64;           // state blocks, [n][chains] per problem (FP64 path)
    uint32_t* bits;        // [trace_levels][total chains][words] accept bits, or NULL
    int64_t total_chains;
    int32_t L;
    int32_t words;         // ceil(L / 32)
    int32_t trace_levels;
    int32_t full_level;    // level whose every chain is re-evaluated in FP64 and stored (-1: none)
    int32_t boundary;      // 0 reflect then clip, 1 clip
    int32_t cost_repeat;   // rotated costs: evaluations of each energy difference (1; more only to emulate costlier f)
    int32_t independent;   // 1: asynchronous chains (no restart from the best; each continues its own state)
    int32_t exchange_every;  // > 1: restart from the best only after every exchange_every-th level
    int32_t proposal;        // 0: Gaussian step; 1: uniform redraw of the coordinate in its interval
    int32_t crossover;       // 1: stochastic crossover at each exchange (every level > 0 starts from X)
    int32_t levels_total;    // levels of the schedule (the crossover skips the last level)
    uint32_t key0, key1;   // Philox key of the sweep stream
    uint32_t ikey0, ikey1; // Philox key of the initial-point stream
    uint32_t rk[20];       // sweep key of each Philox round r: (rk[2r], rk[2r+1]) (kernel-parameter operands)
};

// Does level `level` start each chain from its own state (rather than from the
// best state of the previous level)?  Asynchronous chains never exchange; with a
// period m > 1 the exchange follows levels m-1, 2m-1, ... (Sec. 2.2.1-2.2.2).
// With the stochastic crossover every level > 0 starts from X, which the crossover
// has refilled with the drawn states when an exchange preceded the level.
__host__ __device__ inline bool own_start(const SweepArgs& a, int level) {
    return level > 0 && (a.independent || a.crossover || (a.exchange_every > 1 && level % a.exchange_every != 0));
}
// Must every chain keep its state at the end of a level (for the next level's own start)?
__host__ __device__ inline bool keep_states(const SweepArgs& a) {
    return a.independent || a.crossover || a.exchange_every > 1;
}
// Is the level after `level` an exchange level (the synchronous restart or the crossover)?
__host__ __device__ inline bool exchange_after(const SweepArgs& a, int level) {
    const int next = level + 1;
    return !a.independent && next < a.levels_total && !(a.exchange_every > 1 && next % a.exchange_every != 0);
}

// Launch wrappers (one per translation unit).
cudaError_t launch_sweep_f32(const SweepArgs& a, int num_items, int block, size_t smem, cudaStream_t s);
cudaError_t launch_sweep_f64(const SweepArgs& a, int num_items, int block, size_t smem, cudaStream_t s);
cudaError_t launch_argmin_restart(const SweepArgs& a, const ProbDev* probs, int num_probs, int max_blocks,
                                  int precision, cudaStream_t s);
cudaError_t launch_level_end(RunDev* run, cudaStream_t s);
// Stochastic crossover of one problem before the current level (device-side no-op unless
// an exchange follows the previous level): Boltzmann weights of the previous level's F,
// their running sum, one draw per chain, and the drawn states gathered into the
// problem's start states.
struct CrossoverWork {
    double* w;        // [max chains] weights
    double* S;        // [max chains] running sums
    double* bsum;     // [max blocks] block sums, then their exclusive prefix
    int64_t* src;     // [max chains] drawn source chain
    void* xtmp;       // gather buffer: max over problems of n * chains * 12 bytes
};
cudaError_t launch_crossover(const SweepArgs& a, const ProbDev* dprob, const ProbDev& hprob, int precision, bool rot,
                             uint32_t xkey0, uint32_t xkey1, const CrossoverWork& w, cudaStream_t s);
size_t crossover_blocks(int64_t chains);
cudaError_t launch_reset(ProbDev* probs, int num_probs, RunDev* run, cudaStream_t s);
cudaError_t launch_stamp_start(RunDev* run, cudaStream_t s);
cudaError_t sweep_f32_set_smem(size_t bytes);
// Group layout of the FP32 sweep: `lanes` (G) lanes run one chain, `cache` keeps the
// separable terms beside the state; the built (G, cache) pairs are (32, on), (8, on/off),
// (4, on/off) and (2, off).  block: threads per block (a multiple of 32, <= 256).
bool sweep_f32w_layout_ok(int lanes, bool cache);
cudaError_t launch_sweep_f32w(const SweepArgs& a, int num_items, int lanes, bool cache, int block, size_t smem,
                              cudaStream_t s);
size_t sweep_f32w_smem_bytes(int n, int lanes, bool cache, int block);
cudaError_t sweep_f32w_set_smem(int lanes, bool cache, size_t bytes);
int sweep_f32w_chains_per_block(int lanes, int block);
size_t sweep_f32w_static_bytes(int lanes);
// One launch per level for a batch of FP32 problems: every tile of every problem
// (item.lanes: 2, 4 or 8 lanes per chain, or 0 for one chain per thread with
// item.count <= the tile's capacity), then each problem's last tile to finish
// ends the problem's level (argmin, restart point, incumbent) and the last
// problem advances the level.  256 threads per block.
constexpr int kBatchThreads = 256;
int batch_tile_capacity(int cost, int n, int* lanes);
size_t batch_smem_bytes(int cost, int n);
cudaError_t batch_set_smem(size_t bytes);
cudaError_t launch_batch_level(const SweepArgs& a, int num_items, int num_probs, size_t smem, cudaStream_t s);
cudaError_t sweep_f64_set_smem(size_t bytes);
cudaError_t launch_pgd(int cost, int n, const double* lo, const double* hi, const double* Q, int k, const double* x0,
                       double* x_out, double* f_out, int* it_out, int max_iter, double tol, cudaStream_t s);
// Nelder-Mead from k starts (one block each); ws: k * nm_ws_doubles(n) doubles; rotated
// costs take QT = Q^T (row-major, i.e. Q column-major); n <= nm_max_n().
size_t nm_ws_doubles(int n);
int nm_max_n();
cudaError_t launch_nm(int cost, int n, const double* lo, const double* hi, const double* QT, const double* table,
                      int table_rows, int k, const double* x0, double* x_out, double* f_out, int* it_out,
                      double step_frac, int max_iter, double ftol, double xtol, bool adaptive, double* ws,
                      cudaStream_t s);
cudaError_t launch_topk(double* F, int64_t count, int k, int64_t* idx, cudaStream_t s);
cudaError_t launch_gemm_bf16_f32(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K,
                                 int* status, cudaStream_t s);
int* gemm_status_ptr();
// Y (double-float pairs, [M x N], leading dimension ldy) += (A . B^T) 2^(er[row] + fq[col] - shift),
// for BF16 integer slices of magnitude <= 128 and K <= 1024 (the exact split product of rot_tc.cu).
cudaError_t launch_gemm_accum_pair(const void* A, int lda, const void* B, int ldb, float2* Y, int ldy, int M, int N,
                                   int K, const int* er, const int* fq, int shift, int* status, cudaStream_t s);
cudaError_t launch_gemm_accum_pair2(const void* A, int lda, const void* B, int ldb, int b_rows, int b_row1, int b_row2,
                                    float2* Y, int ldy, int M, int N, int K, const int* er, const int* fq, int shift1,
                                    int shift2, int* status, cudaStream_t s);
// The rotated costs' level-0 transform on the tensor cores (rot_tc.cu): Y [C x n] pairs =
// X [C x n] (FP32) . Q^T (Q FP64 [n x n] row-major), exactly split; shapes with n % 64 == 0,
// n <= 1024 and C % 128 == 0; work: rot_tc_work_bytes(C, n) bytes of device memory.
size_t rot_tc_work_bytes(int64_t C, int n);
bool rot_tc_shape_ok(int64_t C, int n);
cudaError_t launch_rot_tc(const float* X, int64_t C, int n, const double* Q, float2* Y, void* work, int* status,
                          cudaStream_t s);
// Surrogate layers on the tensor-core GEMM: out = gelu(A B^T + bias) as BF16 (Z = the
// pre-activation, FP32, optional); and part[row][t] = sum over the 128 columns of tile t
// of gelu(A B^T + bias) w (N a multiple of 128).
cudaError_t launch_gemm_bias_gelu(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const float* bias,
                                  void* out_bf16, int ldo, float* Z, int ldz, int* status, cudaStream_t s);
cudaError_t launch_gemm_bias_gelu_dot(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                                      const float* bias, const float* w, float* part, float* Z, int ldz, int* status,
                                      cudaStream_t s);
cudaError_t launch_gather(const float* X32, const double* X64, int64_t x_base, int64_t chains, int n, const int64_t* idx,
                          int k, double* out, cudaStream_t s);
cudaError_t launch_polish_update(ProbDev* probs, int problem, const double* xs, const double* fs, int k, cudaStream_t s);

// costs: bit 0 rotated Rastrigin, bit 1 rotated Schwefel among the launch's problems
cudaError_t launch_sweep_rot(const SweepArgs& a, int num_items, size_t smem, int costs, cudaStream_t s);
size_t sweep_rot_smem_bytes(int n);
cudaError_t sweep_rot_set_smem(size_t bytes);
int sweep_rot_chains_per_block();
cudaError_t launch_rot_restart(const ProbDev* d_prob, int n, cudaStream_t s);
int rot_restart_blocks(int n);
// tc_work: the tensor-core transform's workspace (rot_tc_work_bytes), or NULL for the FP64 GEMM.
cudaError_t launch_rot_level0(const ProbDev* d_prob, const ProbDev& host_prob, const SweepArgs& a, float* x0, float2* y0,
                              void* tc_work, int* status, cudaStream_t s);

// ---- the learned surrogate (mlp.cu) ----------------------------------------
constexpr int kMlpHidden = 512;

// Offsets (elements) of the blocks of the flat FP32 parameter vector.
struct MlpOffsets {
    int64_t W1, b1, W2, b2, w3, b3, total;
};
__host__ __device__ inline MlpOffsets mlp_offsets(int n) {
    MlpOffsets o;
    o.W1 = 0;
    o.b1 = (int64_t)kMlpHidden * n;
    o.W2 = o.b1 + kMlpHidden;
    o.b2 = o.W2 + (int64_t)kMlpHidden * kMlpHidden;
    o.w3 = o.b2 + kMlpHidden;
    o.b3 = o.w3 + kMlpHidden;
    o.total = o.b3 + 1;
    return o;
}

struct MlpDev {
    int n, np;        // input dimension and its padding to a multiple of 64
    float* p;         // FP32 parameters
    __nv_bfloat16* W1b;        // BF16 [512 x np]
    __nv_bfloat16* W2b;        // BF16 [512 x 512]
    __nv_bfloat16* W2tb;       // BF16 W2^T [512 x 512]
};

// Per-batch workspace (rows padded to Bp, a multiple of 128).
struct MlpWork {
    __nv_bfloat16* Xb; // BF16 [Bp x np] inputs
    __nv_bfloat16* XT; // BF16 [np x Bp]
    float* Z1;        // [Bp x 512] first pre-activation (nullptr: not stored)
    __nv_bfloat16* A1; // BF16 [Bp x 512]
    __nv_bfloat16* A1T; // BF16 [512 x Bp]
    float* Z2;        // [Bp x 512] second pre-activation (nullptr: not stored)
    __nv_bfloat16* dZ2b; // BF16 [Bp x 512]
    __nv_bfloat16* dZ2T; // BF16 [512 x Bp]
    float* dA1;       // [Bp x 512]
    __nv_bfloat16* dZ1b; // BF16 [Bp x 512]
    __nv_bfloat16* dZ1T; // BF16 [512 x Bp]
    float* y;         // [Bp]
    float* dy;        // [Bp]
    float* part;      // [Bp x 4] partial output sums
    float* dW1;       // [512 x np]
    float* colpart;   // [ceil(Bp / 64) x 2 x 512] partial column sums
};

cudaError_t mlp_cast(const MlpDev& m, cudaStream_t s);
cudaError_t mlp_init(float* p, int n, uint64_t seed, cudaStream_t s);
cudaError_t mlp_forward(const MlpDev& m, const void* Xb, int Bp, MlpWork& w, float* part, int* status, cudaStream_t s);
// Inference: part [Bp x 4] of the head for the BF16 inputs Xb [Bp x np], by the fused
// one-kernel forward pass (mlp_fused.cu) where it applies (np = 64 or 128; not when
// SA_MLP_FUSED=0), else by the two GEMMs with A1 [Bp x 512] as their workspace.
cudaError_t mlp_infer(const MlpDev& m, const void* Xb, int Bp, __nv_bfloat16* A1, float* part, int* status,
                      cudaStream_t s);
bool mlp_fused_ok(int np, int rows);
bool mlp_use_fused(int np, int Bp);
cudaError_t launch_mlp_fused(const void* X, int np, int rows, const void* W1, const void* W2, const float* b1,
                             const float* b2, const float* w3, float* part, int* status, cudaStream_t s);
cudaError_t mlp_finish_y(const MlpDev& m, const float* part, int B, float* y, cudaStream_t s);
cudaError_t mlp_loss_grad(const MlpDev& m, const void* Xb, int B, int Bp, const float* t, MlpWork& w, float* grad,
                          float* loss, int* status, cudaStream_t s);
cudaError_t mlp_adam(float* p, const float* g, float* mo, float* vo, int64_t count, int step, float lr, float b1, float b2,
                     float eps, cudaStream_t s);
cudaError_t mlp_pack(const float* X, int B, int n, int Bp, int np, void* Xb, cudaStream_t s);
size_t mlp_work_bytes(int Bp, int np);
void mlp_work_carve(void* base, int Bp, int np, MlpWork& w);

// ---- delayed acceptance with the surrogate (da.cu) -----------------------------
struct DaDev {
    int problem;             // index of the (rotated) problem in the handle
    int np, Cp;              // padded input width and chain count (multiples of 64 / 128)
    int step_blocks;         // grid of the step kernel (set by da_prepare)
    int64_t cap;             // ring buffer rows (a multiple of the chain count)
    int batch;               // training batch rows
    float* xf;               // [C][n] current states
    float* yh;               // [C][n] Q x as pairs
    float* yl;
    __nv_bfloat16* xs;       // [Cp][np] standardised states, the network's input rows
    double* Fa;              // [C] F of the current state (tracked)
    double* Ea;              // [C] bound on the error of Fa
    float* fts;              // [C] f~ of the current state
    float* part;             // [Cp][4] the output head's partial sums
    __nv_bfloat16* A1;       // [Cp][512] hidden activations of the inference GEMMs
    float* ms;               // [2] mean and standard deviation of the targets (frozen per level)
    float* mid;              // [n] input standardisation (x - mid) / half
    float* inv_half;         // [n]
    const float* b3;         // the output bias inside the parameters
    float* trace_ft0;        // [trace_levels][C] f~ at the level's start states (or NULL)
    float* trace_ftp;        // [trace_levels][L][C] f~ at every proposal (or NULL)
    unsigned long long* evals;  // true energy differences evaluated (stage-1 survivors)
    float* rx;               // [cap][n] ring buffer of states
    float* rf;               // [cap] and of their values
    float* bt;               // [batch] standardised training targets
    float* grad;             // [params] gradient of the training loss
    float* m;                // [params] Adam moments
    float* v;
    int* adam_step;          // Adam steps taken (device)
    int* train_on;           // 1 once the buffer holds pairs (device)
    uint32_t dkey0, dkey1;   // Philox key of stream tag 3 (stage-1 uniforms)
    uint32_t tkey0, tkey1;   // Philox key of stream tag 4 (training batches)
    MlpDev mlp;
    MlpWork work;            // training workspace (batch rows)
};

cudaError_t da_prepare(DaDev& D, int64_t chains);
cudaError_t da_run_start(const DaDev& D, uint64_t seed, cudaStream_t s);
cudaError_t launch_da_level(const SweepArgs& A, const DaDev& D, int64_t chains, int L, int train_steps, float lr,
                            int* status, cudaStream_t s);

constexpr int kArgminThreads = 256;
constexpr int kArgminPerThread = 8;

}  // namespace sa
