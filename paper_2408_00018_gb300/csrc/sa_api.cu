// sa_api.cu -- the C ABI of include/sa.h: handle life cycle, level loop
// (captured once as CUDA graphs and replayed), results, log, checkpoints.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sa.h"
#include "sa_internal.h"

namespace sa {
size_t sweep_f32_smem_bytes(int n, int block);
size_t sweep_f64_smem_bytes(int n, int block, bool keeps_terms);
bool sweep_f64_keeps_terms(int cost);
cudaError_t launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                               int64_t count, uint32_t* out, cudaStream_t s);
int64_t argmin_num_parts(int64_t count);
cudaError_t launch_argmin_f64(const double* F, int64_t count, int64_t* idx, double* val, void* scratch, cudaStream_t s);
}  // namespace sa

using namespace sa;

namespace {

constexpr uint32_t kCkptMagic = 0x42475341u;  // "ASGB"
constexpr uint32_t kCkptVersion = 1u;
constexpr int kGraphLevels = 8;

struct HostProb {
    int32_t cost, n;
    int64_t chains, chain_base, x_base;
    std::vector<double> lo, hi, Q;
    std::vector<double> table;  // Tests 11, 18, 19: table_rows x (n + 1)
    int32_t table_rows = 0;
    ProbDev dev;  // with device pointers
    void* tc_work = nullptr;  // rotated costs: workspace of the tensor-core level-0 transform (or NULL)
};

// Problems whose sweep runs as one kernel launch with one block shape.  A
// batch of problems of uneven dimension is split by n into groups; within a
// level the groups' sweeps run concurrently on forked streams.
enum GroupKind { kSweepF64 = 0, kSweepF32 = 1, kSweepF32Warp = 2, kSweepRot = 3, kSweepDA = 4, kSweepBatch = 5 };

// Delayed acceptance: training per level and buffer sizes.
constexpr int kDaTrainSteps = 128;
constexpr int kDaBatch = 4096;
constexpr float kDaLr = 1e-3f;
constexpr int64_t kDaBufferRows = (int64_t)1 << 20;
constexpr uint32_t kTagDa = 3u, kTagTrain = 4u;

bool is_rot(int cost) { return cost == SA_ROT_RASTRIGIN || cost == SA_ROT_SCHWEFEL; }
// The Appendix's Tests 2-12 and 15-19: FP64 full evaluation only.
bool is_appendix(int cost) { return cost >= SA_BRANIN && cost <= SA_FOXHOLES; }
bool is_table(int cost) { return cost == SA_LANGERMAN || cost == SA_SHEKEL || cost == SA_FOXHOLES; }
bool is_2d(int cost) {
    return cost == SA_BRANIN || cost == SA_DEKKERS_AARTS || cost == SA_EASOM || cost == SA_GOLDSTEIN_PRICE ||
           cost == SA_HIMMELBLAU || cost == SA_SIX_HUMP_CAMEL;
}
constexpr int kMaxTableRows = 4096;
// A cost's own requirements on n, Q and the table (shared by the solver and sa_nelder_mead).
bool cost_args_ok(int cost, int n, const double* Q, const double* table, int rows) {
    if (cost < SA_SCHWEFEL || cost > SA_FOXHOLES || n < 1) return false;
    if (is_rot(cost) != (Q != nullptr)) return false;
    if (is_rot(cost) && (int64_t)n * n > ((int64_t)1 << 28)) return false;
    if (is_2d(cost) && n != 2) return false;
    if (is_table(cost) != (table != nullptr)) return false;
    if (is_table(cost)) {
        if (rows < 1 || rows > kMaxTableRows || (int64_t)rows * (n + 1) > ((int64_t)1 << 24)) return false;
        for (size_t e = 0; e < (size_t)rows * (size_t)(n + 1); ++e)
            if (!std::isfinite(table[e])) return false;
    } else if (rows != 0) {
        return false;
    }
    if (Q)
        for (size_t e = 0; e < (size_t)n * n; ++e)
            if (!std::isfinite(Q[e])) return false;
    return true;
}
struct Group {
    int kind = kSweepF32;
    int n_max = 1;
    bool f64_terms = false;  // FP64 group: a problem keeps per-coordinate factors (twice the state)
    int block = 32;        // threads per block
    int lanes = 32;        // group layout (kSweepF32Warp): lanes per chain
    bool cache = true;     // group layout: separable terms cached beside the state
    size_t smem = 0;       // dynamic shared memory per block
    std::vector<int> probs;
    std::vector<WorkItem> items;
    WorkItem* d_items = nullptr;  // capacity: items at the smallest block shape
    size_t items_cap = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct sa_handle {
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    sa_schedule sch{};
    uint64_t seed = 0;
    int32_t L = 0;
    int32_t levels_total = 0;
    int32_t levels_done = 0;
    int32_t words = 0;
    int precision = 0;
    int64_t total_chains = 0;
    int64_t total_x = 0;
    std::vector<HostProb> probs;
    std::vector<Group> groups;
    cudaEvent_t fork_ev = nullptr;
    int max_argmin_blocks = 0;
    uint64_t fingerprint = 0;
    sa_status failed = SA_OK;
    int64_t h2d_bytes = 0, d2h_bytes = 0;
    // device
    std::vector<void*> allocs;
    ProbDev* d_probs = nullptr;
    std::vector<ProbDev> pd;  // host copy of the descriptors
    RunDev* d_run = nullptr;
    double* d_T = nullptr;
    double* d_s = nullptr;
    double* d_F = nullptr;
    float* d_X32 = nullptr;
    double* d_X64 = nullptr;
    uint32_t* d_bits = nullptr;
    // hybrid polish buffers (polish_k > 0)
    double* d_Fcopy = nullptr;
    int64_t* d_topk = nullptr;
    double *d_px0 = nullptr, *d_px = nullptr, *d_pf = nullptr;
    int* d_pit = nullptr;
    double* d_nmws = nullptr;  // Nelder-Mead workspace (polish_method == SA_POLISH_NELDER_MEAD)
    CrossoverWork xo{};        // stochastic crossover scratch (schedule.crossover)
    uint32_t xkey0 = 0, xkey1 = 0;
    double nm_step = 0.0;      // its initial simplex size, as a fraction of the box
    SweepArgs args{};
    cudaGraphExec_t g1 = nullptr, gN = nullptr;
    // delayed acceptance with the surrogate (schedule.surrogate == 1)
    bool da = false;
    DaDev dd{};
};

namespace {

sa_status fail(sa_handle* h, sa_status s) {
    if (h && h->failed == SA_OK) h->failed = s;
    return s;
}

template <class T>
sa_status dalloc(sa_handle* h, T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    if (cudaMallocAsync(&q, count * sizeof(T), h->stream) != cudaSuccess) {
        cudaGetLastError();
        return SA_ENOMEM;
    }
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return SA_OK;
}

template <class T>
sa_status h2d(sa_handle* h, T* dst, const T* src, size_t count) {
    if (count == 0) return SA_OK;
    h->h2d_bytes += (int64_t)(count * sizeof(T));
    return cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, h->stream) == cudaSuccess ? SA_OK : SA_ECUDA;
}

bool batch_level_ok(const sa_handle* h) {
    if (const char* e = std::getenv("SA_BATCH_LEVEL"))
        if (e[0] == '0') return false;
    if (h->precision == SA_FP64 || h->sch.surrogate || h->probs.size() < 2) return false;
    for (const HostProb& p : h->probs) {
        if (!(p.cost == SA_SCHWEFEL || p.cost == SA_RASTRIGIN || p.cost == SA_ACKLEY || p.cost == SA_ROSENBROCK))
            return false;
        if (batch_smem_bytes(p.cost, p.n) > 200 * 1024) return false;
    }
    return true;
}

uint64_t fnv(uint64_t h, const void* p, size_t len) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < len; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}

float round_up_f(double v) {
    float f = (float)v;
    if ((double)f < v) f = std::nextafterf(f, INFINITY);
    return f;
}
float round_down_f(double v) {
    float f = (float)v;
    if ((double)f > v) f = std::nextafterf(f, -INFINITY);
    return f;
}

sa_status check_schedule(const sa_schedule* s) {
    if (!s) return SA_EINVAL;
    if (!(s->T0 > 0.0) || !std::isfinite(s->T0)) return SA_EINVAL;
    if (!(s->rho > 0.0 && s->rho < 1.0)) return SA_EINVAL;
    if (s->levels < 0) return SA_EINVAL;
    if (s->levels == 0 && !(s->T_min > 0.0 && s->T_min < s->T0)) return SA_EINVAL;
    if (!(s->sigma_frac > 0.0) || !std::isfinite(s->sigma_frac)) return SA_EINVAL;
    if (s->boundary != SA_REFLECT && s->boundary != SA_CLIP) return SA_EINVAL;
    if (s->precision != SA_FP64 && s->precision != SA_FP32) return SA_EINVAL;
    if ((s->surrogate != 0 && s->surrogate != 1) || s->polish_k < 0 || s->polish_k > 1024) return SA_EINVAL;
    if (s->polish_method != SA_POLISH_PGD && s->polish_method != SA_POLISH_NELDER_MEAD &&
        s->polish_method != SA_POLISH_NELDER_MEAD_ADAPTIVE)
        return SA_EINVAL;
    if ((s->proposal != SA_PROPOSAL_GAUSSIAN && s->proposal != SA_PROPOSAL_UNIFORM) ||
        (s->proposal == SA_PROPOSAL_UNIFORM && s->surrogate))
        return SA_EINVAL;
    if ((s->crossover != 0 && s->crossover != 1) || (s->crossover && (s->surrogate || s->independent)))
        return SA_EINVAL;
    if (s->cost_repeat < 0 || s->cost_repeat > 4096) return SA_EINVAL;
    if ((s->independent != 0 && s->independent != 1) || (s->independent && s->surrogate)) return SA_EINVAL;
    if (s->exchange_every < 0 || (s->exchange_every > 1 && s->surrogate)) return SA_EINVAL;
    if (s->trace_levels < 0) return SA_EINVAL;
    return SA_OK;
}

// Checks of one problem shared by sa_create and sa_create_batch.
sa_status check_problem(const sa_problem& pr, const sa_box& box, int32_t n, int64_t chains, const sa_schedule& sch) {
    if (n < 1 || chains < 1 || chains > 2147483647LL || !box.lo || !box.hi) return SA_EINVAL;
    if (!cost_args_ok(pr.cost, n, pr.Q, pr.table, pr.table_rows)) return SA_EINVAL;
    if (sch.surrogate && (!is_rot(pr.cost) || n > 4096)) return SA_EINVAL;
    // rotated costs run the FP32 rank-1 sweep; the Appendix's other tests the FP64 sweep
    if (is_rot(pr.cost) && sch.precision != SA_FP32) return SA_EINVAL;
    if (is_appendix(pr.cost) && sch.precision != SA_FP64) return SA_EINVAL;
    // no gradient is written for the Appendix's other tests: they polish with Nelder-Mead
    if (is_appendix(pr.cost) && sch.polish_k > 0 && sch.polish_method == SA_POLISH_PGD) return SA_EINVAL;
    if (sch.polish_k > 0 && sch.polish_method != SA_POLISH_PGD && n > nm_max_n()) return SA_EINVAL;
    for (int k = 0; k < n; ++k)
        if (!std::isfinite(box.lo[k]) || !std::isfinite(box.hi[k]) || box.lo[k] > box.hi[k]) return SA_EINVAL;
    return SA_OK;
}

int pick_block(int precision, int n_max) {
    // FP64 arithmetic is a small fraction of the FP32 rate on this GPU, so the
    // FP64 sweep uses one warp per block: chains spread over as many SMs as
    // possible.
    if (precision == SA_FP64) return 32;
    // ~64 KB of chain state per block: several blocks per SM, so that one
    // block's end-of-level work overlaps the others' sweeps.  SA_BLOCK_BYTES
    // overrides the per-block state budget for tuning runs.
    const int bytes = 4;
    int budget = 65536;
    if (const char* e = std::getenv("SA_BLOCK_BYTES")) {
        const int v = std::atoi(e);
        if (v >= 4096 && v <= 220 * 1024) budget = v;
    }
    int b = budget / (bytes * n_max);
    b = (b / 32) * 32;
    if (b > 256) b = 256;
    if (b < 32) b = 32;
    return b;
}

// Steps evaluated together per chain in the FP32 sweep: speculation pays when
// two steps of a group rarely touch the same coordinate.  SA_UNROLL overrides
// (1, 2 or 4) for tuning runs; the result is the same for every choice.
int pick_unroll(int cost, int n) {
    if (const char* e = std::getenv("SA_UNROLL")) {
        const int u = std::atoi(e);
        if (u == 1 || u == 2 || u == 4) return u;
    }
    if (cost == SA_ACKLEY) return 1;
    if (n >= 16) return 2;  // measured at n = 256: U = 2 1.84 ms, U = 4 1.88 ms, U = 1 2.22 ms per level
    return 1;
}

// Steps whose randomness the chain-per-thread FP32 sweep draws as one batch
// (16, or 1 for one group of U steps at a time).  SA_RAND_BATCH overrides it
// for tuning runs; the decisions are the same for every choice.
int pick_rand_batch() {
    if (const char* e = std::getenv("SA_RAND_BATCH")) {
        const int r = std::atoi(e);
        if (r == 1 || r == 16) return r;
    }
    return 16;
}

// FP32 sweep layout: one chain per warp (32 consecutive steps per group)
// pays when a group rarely touches a coordinate twice and the cost has no
// global running sums.  SA_WARP_MODE=0/1 overrides for tuning runs.
bool warp_eligible(int cost) { return cost == SA_SCHWEFEL || cost == SA_RASTRIGIN || cost == SA_ROSENBROCK; }

bool pick_warp_mode(int cost, int n) {
    if (!warp_eligible(cost)) return false;
    if (const char* e = std::getenv("SA_WARP_MODE")) {
        if (e[0] == '0') return false;
        if (e[0] == '1') return true;
    }
    // Default before autotuning, from measured levels of 262144 chains on this
    // GPU: the chain-per-thread layout up to n = 128 (Schwefel n = 128: 1.43 ms
    // per level against 1.60 ms with 4 lanes per chain); above it its shared
    // memory per chain leaves too few warps per SM (n = 256: 1.83 ms against
    // 1.55 ms with 4 lanes per chain; n = 512, 131072 chains: 1.53 ms against
    // 0.91 ms with 8).
    return n > 128;
}

// Group layout of the FP32 sweep for a dimension bucket: lanes per chain,
// cached terms, threads per block.  The block size maximises the chains an
// SM holds (its shared memory, 1 KiB reserved per block, 2048 threads and the
// kernel's register budget of 80 per thread), larger blocks on ties, at least
// 8 chains per block.  SA_CHAIN_LANES (2, 4, 8, 32), SA_TERM_CACHE (0/1) and
// SA_GROUP_BLOCK (threads) override it for tuning runs; every choice gives the
// same decisions.
struct GroupLayout { int lanes; bool cache; int block; };
GroupLayout pick_group_layout(int n) {
    GroupLayout g{n > 256 ? 8 : 4, false, 0};
    if (const char* e = std::getenv("SA_CHAIN_LANES")) {
        const int v = std::atoi(e);
        if (v == 2 || v == 4 || v == 8 || v == 32) g.lanes = v;
    }
    if (const char* e = std::getenv("SA_TERM_CACHE")) g.cache = e[0] == '1';
    if (g.lanes == 32) g.cache = true;
    if (g.lanes == 2) g.cache = false;
    constexpr size_t kSmemPerSm = 228 * 1024, kReserved = 1024;
    int best_b = 8 * g.lanes < 32 ? 32 : 8 * g.lanes;
    long best_chains = -1;
    for (int b = best_b; b <= 256; b += 32) {
        const size_t smem = sweep_f32w_smem_bytes(n, g.lanes, g.cache, b) + sweep_f32w_static_bytes(g.lanes);
        if (smem > 227 * 1024) break;
        const long by_smem = (long)(kSmemPerSm / (smem + kReserved));
        const long by_threads = 2048 / b, by_regs = 65536 / (80L * b);
        const long blocks = std::min(by_smem, std::min(by_threads, by_regs));
        const long chains = blocks * (b / g.lanes);
        if (chains >= best_chains) { best_chains = chains; best_b = b; }
    }
    g.block = best_b;
    if (const char* e = std::getenv("SA_GROUP_BLOCK")) {
        const int v = (std::atoi(e) / 32) * 32;
        if (v >= 32 && v <= 256 && v >= 8 * g.lanes) g.block = v;
    }
    return g;
}

// Does a handle run its FP32 levels as one launch each (the batched level
// kernel)?  Batches of more than one problem of the separable costs, whose
// largest tile fits a block.  SA_BATCH_LEVEL=0 keeps the launch per dimension
// group instead (tuning runs and the tests that compare the two).
bool batch_level_ok(const sa_handle* h);

// Bound on the FP32 error of one accepted step's dF over the whole box (the
// per-step bounds of sa_device.cuh at their largest), used by the warp layout.
float step_kappa(int cost, int n, const std::vector<float>& lo32, const std::vector<float>& hi32) {
    double B = 0.0;
    for (size_t k = 0; k < lo32.size(); ++k) B = std::fmax(B, std::fmax(std::fabs((double)lo32[k]), std::fabs((double)hi32[k])));
    double kap = 0.0;
    if (cost == SA_SCHWEFEL) kap = (2.0 * B * (std::sqrt(B) * 4.8e-7 + 2.6e-6) + 2.0 * B * 2.4e-7) / n;
    else if (cost == SA_RASTRIGIN) kap = 4.8e-5 + 4.0 * (B * B + 10.0) * 1.2e-7;
    return (float)(kap * 1.01);
}

cudaError_t launch_group(sa_handle* h, const Group& g, cudaStream_t s) {
    SweepArgs a = h->args;
    a.items = g.d_items;
    const int num = (int)g.items.size();
    if (num == 0) return cudaSuccess;
    if (g.kind == kSweepF64) return launch_sweep_f64(a, num, g.block, g.smem, s);
    if (g.kind == kSweepF32Warp) return launch_sweep_f32w(a, num, g.lanes, g.cache, g.block, g.smem, s);
    if (g.kind == kSweepRot) {
        int costs = 0;
        for (int p : g.probs) costs |= h->probs[p].cost == SA_ROT_RASTRIGIN ? 1 : 2;
        return launch_sweep_rot(a, num, g.smem, costs, s);
    }
    if (g.kind == kSweepBatch) return launch_batch_level(a, num, (int)h->probs.size(), g.smem, s);
    if (g.kind == kSweepDA)
        // the GEMMs report a timeout in the run's own status word, which every sa_run reads
        return launch_da_level(a, h->dd, h->probs[h->dd.problem].chains, h->L, kDaTrainSteps, kDaLr,
                               &h->d_run->status, s);
    return launch_sweep_f32(a, num, g.block, g.smem, s);
}

// The sweep of one level: one launch per group; several groups run
// concurrently on forked streams (also inside a captured graph).
cudaError_t launch_sweep(sa_handle* h, cudaStream_t s) {
    // stochastic crossover: this level's start states drawn from the previous level's final
    // states (a no-op on the device unless an exchange precedes this level); the previous
    // level's states stay readable until here (sa_trace_states)
    if (h->sch.crossover)
        for (size_t p = 0; p < h->probs.size(); ++p) {
            const cudaError_t e = launch_crossover(h->args, h->d_probs + p, h->probs[p].dev, h->precision,
                                                   is_rot(h->probs[p].cost), h->xkey0, h->xkey1, h->xo, s);
            if (e != cudaSuccess) return e;
        }
    if (h->groups.size() == 1) return launch_group(h, h->groups[0], s);
    cudaError_t e = cudaEventRecord(h->fork_ev, s);
    for (Group& g : h->groups) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g.stream, h->fork_ev, 0);
        if (e == cudaSuccess) e = launch_group(h, g, g.stream);
        if (e == cudaSuccess) e = cudaEventRecord(g.done, g.stream);
    }
    for (Group& g : h->groups)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g.done, 0);
    return e;
}

// Work items of a group for its current block shape (tiles of one problem's
// chains), largest problems first; uploaded on the handle's stream.
sa_status set_group_items(sa_handle* h, Group& g) {
    if (g.kind == kSweepBatch) {
        // every tile of every problem in one launch, largest problems first; each
        // problem's tiles take its own layout and capacity (batch_tile_capacity)
        std::vector<int> order = g.probs;
        std::sort(order.begin(), order.end(), [h](int a, int b) { return h->probs[a].chains > h->probs[b].chains; });
        g.items.clear();
        for (int p : order) {
            int lanes = 0;
            const int cap = batch_tile_capacity(h->probs[p].cost, h->probs[p].n, &lanes);
            int32_t slot = 0;
            for (int64_t c0 = 0; c0 < h->probs[p].chains; c0 += cap, ++slot) {
                const int64_t cnt = h->probs[p].chains - c0 < cap ? h->probs[p].chains - c0 : cap;
                g.items.push_back(WorkItem{p, (int32_t)cnt, c0, lanes, slot});
            }
            h->pd[p].items = slot;
        }
        if (g.items.size() > g.items_cap) return SA_EINVAL;
        h->h2d_bytes += (int64_t)(g.items.size() * sizeof(WorkItem));
        return cudaMemcpyAsync(g.d_items, g.items.data(), g.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                               h->stream) == cudaSuccess ? SA_OK : SA_ECUDA;
    }
    const int per_item = g.kind == kSweepF32Warp ? sweep_f32w_chains_per_block(g.lanes, g.block)
                         : (g.kind == kSweepRot || g.kind == kSweepDA) ? sweep_rot_chains_per_block()
                                                                       : g.block;
    std::vector<int> order = g.probs;
    std::sort(order.begin(), order.end(), [h](int a, int b) { return h->probs[a].chains > h->probs[b].chains; });
    g.items.clear();
    for (int p : order)
        for (int64_t c0 = 0; c0 < h->probs[p].chains; c0 += per_item) {
            const int64_t cnt = h->probs[p].chains - c0 < per_item ? h->probs[p].chains - c0 : per_item;
            g.items.push_back(WorkItem{p, (int32_t)cnt, c0, 0, 0});
        }
    if (g.items.size() > g.items_cap) return SA_EINVAL;
    if (g.items.empty()) return SA_OK;
    h->h2d_bytes += (int64_t)(g.items.size() * sizeof(WorkItem));
    return cudaMemcpyAsync(g.d_items, g.items.data(), g.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                           h->stream) == cudaSuccess ? SA_OK : SA_ECUDA;
}

size_t group_smem(const Group& g) {
    if (g.kind == kSweepBatch) return g.smem;  // the largest tile of the batch (set at creation)
    if (g.kind == kSweepF32Warp) return sweep_f32w_smem_bytes(g.n_max, g.lanes, g.cache, g.block);
    if (g.kind == kSweepRot) return sweep_rot_smem_bytes(g.n_max);
    if (g.kind == kSweepF64) return sweep_f64_smem_bytes(g.n_max, g.block, g.f64_terms);
    return sweep_f32_smem_bytes(g.n_max, g.block);
}

cudaError_t group_set_smem(const Group& g) {
    if (g.kind == kSweepBatch) return batch_set_smem(g.smem);
    if (g.kind == kSweepF32Warp) return sweep_f32w_set_smem(g.lanes, g.cache, g.smem);
    if (g.kind == kSweepRot) return sweep_rot_set_smem(g.smem);
    if (g.kind == kSweepF64) return sweep_f64_set_smem(g.smem);
    return sweep_f32_set_smem(g.smem);
}

// FP32 dimension buckets: problems with n in (bound[i-1], bound[i]] share a group.
constexpr int kBucketBounds[] = {16, 32, 64, 128, 256, 512, 1 << 30};

cudaError_t launch_level_tail(sa_handle* h, cudaStream_t s) {
    // the batched level kernel ends every problem's level and cools by itself
    if (h->groups.size() == 1 && h->groups[0].kind == kSweepBatch) return cudaSuccess;
    cudaError_t e = launch_argmin_restart(h->args, h->d_probs, (int)h->probs.size(), h->max_argmin_blocks,
                                          h->precision == SA_FP64 ? 0 : 1, s);
    // rotated costs: y_best = Q x_best and F(y_best) for the next level
    for (size_t p = 0; p < h->probs.size() && e == cudaSuccess; ++p)
        if (is_rot(h->probs[p].cost)) e = launch_rot_restart(h->d_probs + p, h->probs[p].n, s);
    if (e == cudaSuccess) e = launch_level_end(h->d_run, s);
    return e;
}

// Work that precedes level 0 of a run: the start stamp and, for rotated
// costs, the initial points X0 and their transform Y0 = X0 Q^T.
cudaError_t launch_level0_prep(sa_handle* h, cudaStream_t s);

sa_status capture_levels(sa_handle* h, int levels, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SA_ECUDA;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < levels && e == cudaSuccess; ++k) {
        e = launch_sweep(h, h->cap_stream);
        if (e == cudaSuccess) e = launch_level_tail(h, h->cap_stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return SA_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? SA_OK : SA_ECUDA;
}

sa_status device_status(sa_handle* h) {
    int32_t st = 0;
    if (cudaMemcpyAsync(&st, &h->d_run->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return fail(h, SA_ECUDA);
    if (st == 5) return fail(h, SA_ENUMERIC);
    if (st == 4) return fail(h, SA_ETIMEOUT);
    if (st != 0) return fail(h, SA_ECUDA);
    return SA_OK;
}

// Hybrid SA (after the last level): the polish_k best final states of each
// problem, by FP64 value with lowest index on ties, are polished by
// box-projected gradient descent or by Nelder-Mead (Sec. 4.2, Table 10); the
// best polished point replaces the incumbent if it is lower.
sa_status run_polish(sa_handle* h) {
    if (h->sch.polish_k <= 0) return SA_OK;
    for (size_t p = 0; p < h->probs.size(); ++p) {
        const HostProb& hp = h->probs[p];
        const int k = (int)std::min<int64_t>(h->sch.polish_k, hp.chains);
        if (cudaMemcpyAsync(h->d_Fcopy, h->d_F + hp.chain_base, hp.chains * sizeof(double), cudaMemcpyDeviceToDevice,
                            h->stream) != cudaSuccess ||
            launch_topk(h->d_Fcopy, hp.chains, k, h->d_topk, h->stream) != cudaSuccess ||
            launch_gather(h->d_X32, h->d_X64, hp.x_base, hp.chains, hp.n, h->d_topk, k, h->d_px0, h->stream) !=
                cudaSuccess ||
            (h->sch.polish_method != SA_POLISH_PGD
                 ? launch_nm(hp.cost, hp.n, hp.dev.lo, hp.dev.hi, hp.dev.qt64, hp.dev.table, hp.dev.table_rows, k,
                             h->d_px0, h->d_px, h->d_pf, h->d_pit, h->nm_step, 200 * (hp.n + 1), 1e-12, 1e-10,
                             h->sch.polish_method == SA_POLISH_NELDER_MEAD_ADAPTIVE, h->d_nmws, h->stream)
                 : launch_pgd(hp.cost, hp.n, hp.dev.lo, hp.dev.hi, hp.dev.q64, k, h->d_px0, h->d_px, h->d_pf,
                              h->d_pit, 1000, 1e-10, h->stream)) != cudaSuccess ||
            launch_polish_update(h->d_probs, (int)p, h->d_px, h->d_pf, k, h->stream) != cudaSuccess)
            return fail(h, SA_ECUDA);
    }
    return SA_OK;
}

// Device copies of Q for a rotated cost (row-major FP64; transposed FP64 and
// its FP32 hi + lo split for the sweep's column reads), the restart pair and
// the level-0 buffers X0 [chains][n] and Y0 [chains][n] (pairs).
sa_status setup_rot(sa_handle* h, HostProb& hp, ProbDev& d) {
    const int n = hp.n;
    const size_t nn = (size_t)n * n;
    std::vector<double> qt(nn);
    std::vector<float> qh(nn), ql(nn);
    double qmax = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double q = hp.Q[(size_t)i * n + j];
            qt[(size_t)j * n + i] = q;
            qmax = std::fmax(qmax, std::fabs(q));
        }
    for (size_t k = 0; k < nn; ++k) {
        qh[k] = (float)qt[k];
        ql[k] = (float)(qt[k] - (double)qh[k]);
    }
    double *q64, *qt64, *rpart;
    float *qth, *qtl, *ybh, *ybl, *x0;
    float2* y0;
    unsigned long long* rech;
    unsigned int* rdone;
    sa_status st;
    const size_t cn = (size_t)hp.chains * n;
    if ((st = dalloc(h, &q64, nn)) || (st = dalloc(h, &qt64, nn)) || (st = dalloc(h, &qth, nn)) ||
        (st = dalloc(h, &qtl, nn)) || (st = dalloc(h, &ybh, n)) || (st = dalloc(h, &ybl, n)) ||
        (st = dalloc(h, &x0, cn)) || (st = dalloc(h, &y0, cn)) || (st = dalloc(h, &rech, 1)) ||
        (st = dalloc(h, &rdone, 1)) || (st = dalloc(h, &rpart, rot_restart_blocks(n))))
        return st;
    const unsigned long long z64 = 0;
    const unsigned int z32 = 0;
    if ((st = h2d(h, q64, hp.Q.data(), nn)) || (st = h2d(h, qt64, qt.data(), nn)) || (st = h2d(h, qth, qh.data(), nn)) ||
        (st = h2d(h, qtl, ql.data(), nn)) || (st = h2d(h, rech, &z64, 1)) || (st = h2d(h, rdone, &z32, 1)))
        return st;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SA_ECUDA;  // host temporaries die here
    d.q64 = q64; d.qt64 = qt64; d.qt_hi = qth; d.qt_lo = qtl; d.ybest_hi = ybh; d.ybest_lo = ybl;
    d.x0 = x0; d.y0 = y0; d.rechecks = rech; d.rot_done = rdone; d.rot_part = rpart;
    // the level-0 transform on the tensor cores where the shape allows (SA_ROT_TC=0: the FP64 GEMM)
    const char* tc_env = std::getenv("SA_ROT_TC");
    if (rot_tc_shape_ok(hp.chains, n) && !(tc_env && tc_env[0] == '0')) {
        unsigned char* w;
        if ((st = dalloc(h, &w, rot_tc_work_bytes(hp.chains, n)))) return st;
        hp.tc_work = w;
    }
    float qm = (float)qmax;
    if ((double)qm < qmax) qm = std::nextafterf(qm, INFINITY);
    d.qmax = qm;
    double ymax = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += std::fabs(hp.Q[(size_t)i * n + j]) * std::fmax(std::fabs(hp.lo[j]), std::fabs(hp.hi[j]));
        ymax = std::fmax(ymax, r);
    }
    d.ymax = (float)(ymax * 1.001);
    return SA_OK;
}

// Buffers of the delayed-acceptance sweep and of the surrogate's training.
sa_status setup_da(sa_handle* h) {
    const HostProb& hp = h->probs[0];
    DaDev& D = h->dd;
    const int n = hp.n;
    const int64_t C = hp.chains;
    D.problem = 0;
    D.np = (n + 63) / 64 * 64;
    D.Cp = (int)((C + 127) / 128 * 128);
    D.cap = std::max<int64_t>(1, kDaBufferRows / C) * C;  // a multiple of C: one insertion never wraps onto itself
    D.batch = kDaBatch;
    const int64_t P = mlp_offsets(n).total;
    const int tl = h->args.trace_levels;
    sa_status st;
    float *mid, *ih;
    if ((st = dalloc(h, &D.xf, (size_t)C * n)) || (st = dalloc(h, &D.yh, (size_t)C * n)) ||
        (st = dalloc(h, &D.yl, (size_t)C * n)) || (st = dalloc(h, &D.xs, (size_t)D.Cp * D.np)) ||
        (st = dalloc(h, &D.Fa, C)) || (st = dalloc(h, &D.Ea, C)) || (st = dalloc(h, &D.fts, C)) ||
        (st = dalloc(h, &D.part, (size_t)D.Cp * 4)) || (st = dalloc(h, &D.A1, (size_t)D.Cp * kMlpHidden)) ||
        (st = dalloc(h, &D.ms, 2)) || (st = dalloc(h, &mid, n)) || (st = dalloc(h, &ih, n)) ||
        (st = dalloc(h, &D.evals, 1)) || (st = dalloc(h, &D.rx, (size_t)D.cap * n)) || (st = dalloc(h, &D.rf, D.cap)) ||
        (st = dalloc(h, &D.bt, D.batch)) || (st = dalloc(h, &D.grad, P)) || (st = dalloc(h, &D.m, P)) ||
        (st = dalloc(h, &D.v, P)) || (st = dalloc(h, &D.adam_step, 1)) || (st = dalloc(h, &D.train_on, 1)) ||
        (st = dalloc(h, &D.mlp.p, P)) || (st = dalloc(h, &D.mlp.W1b, (size_t)kMlpHidden * D.np)) ||
        (st = dalloc(h, &D.mlp.W2b, (size_t)kMlpHidden * kMlpHidden)) ||
        (st = dalloc(h, &D.mlp.W2tb, (size_t)kMlpHidden * kMlpHidden)))
        return st;
    if (tl > 0 && ((st = dalloc(h, &D.trace_ft0, (size_t)tl * C)) || (st = dalloc(h, &D.trace_ftp, (size_t)tl * h->L * C))))
        return st;
    unsigned char* wbase;
    if ((st = dalloc(h, &wbase, mlp_work_bytes(D.batch, D.np) + 1024))) return st;
    mlp_work_carve(reinterpret_cast<void*>(((uintptr_t)wbase + 1023) & ~(uintptr_t)1023), D.batch, D.np, D.work);
    D.mid = mid;
    D.inv_half = ih;
    D.mlp.n = n;
    D.mlp.np = D.np;
    D.b3 = D.mlp.p + mlp_offsets(n).b3;
    if (da_prepare(D, C) != cudaSuccess) return SA_ECUDA;
    D.dkey0 = (uint32_t)h->seed;
    D.dkey1 = (uint32_t)(h->seed >> 32) ^ kTagDa;
    D.tkey0 = (uint32_t)h->seed;
    D.tkey1 = (uint32_t)(h->seed >> 32) ^ kTagTrain;
    std::vector<float> m(n), ihv(n);
    for (int k = 0; k < n; ++k) {
        m[k] = (float)(0.5 * (hp.lo[k] + hp.hi[k]));
        const double half = 0.5 * (hp.hi[k] - hp.lo[k]);
        ihv[k] = (float)(half > 0.0 ? 1.0 / half : 0.0);
    }
    // zero the padded rows of the input matrix once (the kernels write only real rows)
    if (cudaMemsetAsync(D.xs, 0, (size_t)D.Cp * D.np * sizeof(__nv_bfloat16), h->stream) != cudaSuccess ||
        cudaMemsetAsync(D.part, 0, (size_t)D.Cp * 4 * sizeof(float), h->stream) != cudaSuccess)
        return SA_ECUDA;
    if ((st = h2d(h, mid, m.data(), n)) || (st = h2d(h, ih, ihv.data(), n))) return st;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SA_ECUDA;
    h->da = true;
    return SA_OK;
}

sa_status build(sa_handle* h, const sa_problem* problems, const sa_box* boxes, const int32_t* ns,
                const int64_t* chains, int32_t num) {
    sa_status st;
    const int P = num;
    int n_max = 1;
    h->total_chains = 0;
    h->total_x = 0;
    h->probs.resize(P);
    for (int p = 0; p < P; ++p) {
        HostProb& hp = h->probs[p];
        hp.cost = problems[p].cost;
        hp.n = ns[p];
        hp.chains = chains[p];
        hp.chain_base = h->total_chains;
        hp.x_base = h->total_x;
        h->total_chains += hp.chains;
        h->total_x += (int64_t)hp.n * hp.chains;
        hp.lo.assign(boxes[p].lo, boxes[p].lo + hp.n);
        hp.hi.assign(boxes[p].hi, boxes[p].hi + hp.n);
        if (is_rot(hp.cost)) hp.Q.assign(problems[p].Q, problems[p].Q + (size_t)hp.n * hp.n);
        if (is_table(hp.cost)) {
            hp.table_rows = problems[p].table_rows;
            hp.table.assign(problems[p].table, problems[p].table + (size_t)hp.table_rows * (hp.n + 1));
        }
        if (hp.n > n_max) n_max = hp.n;
    }
    h->words = (h->L + 31) / 32;
    h->levels_total = h->sch.levels > 0 ? h->sch.levels : sa_levels_for(h->sch.T0, h->sch.rho, h->sch.T_min);
    if (h->levels_total < 1) return SA_EINVAL;

    // launch groups: FP64 -> one group; FP32 -> one group per dimension bucket
    (void)n_max;
    if (h->sch.surrogate) {
        h->groups.resize(1);
        h->groups[0].kind = kSweepDA;
        h->groups[0].probs.push_back(0);
    } else if (h->precision == SA_FP64) {
        h->groups.resize(1);
        h->groups[0].kind = kSweepF64;
        for (int p = 0; p < P; ++p) {
            h->groups[0].probs.push_back(p);
            if (sweep_f64_keeps_terms(h->probs[p].cost)) h->groups[0].f64_terms = true;
        }
    } else if (batch_level_ok(h)) {
        h->groups.resize(1);
        Group& g = h->groups[0];
        g.kind = kSweepBatch;
        for (int p = 0; p < P; ++p) {
            g.probs.push_back(p);
            g.smem = std::max(g.smem, batch_smem_bytes(h->probs[p].cost, h->probs[p].n));
        }
    } else {
        // one group per (dimension bucket, class) pair: class 0 = thread
        // layout only, 1 = costs the chain-per-warp layout serves (no global
        // running sums), 2 = rotated costs (chain-per-warp rank-1 sweep)
        const int nb = (int)(sizeof(kBucketBounds) / sizeof(int));
        std::vector<Group> b(3 * nb);
        for (int p = 0; p < P; ++p) {
            int i = 0;
            while (h->probs[p].n > kBucketBounds[i]) ++i;
            const int cls = is_rot(h->probs[p].cost) ? 2 : (warp_eligible(h->probs[p].cost) ? 1 : 0);
            b[3 * i + cls].probs.push_back(p);
        }
        for (int i = 0; i < 3 * nb; ++i) {
            Group& g = b[i];
            if (g.probs.empty()) continue;
            int nmax = 1;
            for (int p : g.probs) nmax = std::max(nmax, h->probs[p].n);
            const int cls = i % 3;
            g.kind = cls == 2 ? kSweepRot
                     : (cls == 1 && pick_warp_mode(h->probs[g.probs[0]].cost, nmax)) ? kSweepF32Warp
                                                                                     : kSweepF32;
            h->groups.push_back(g);
        }
    }
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (Group& g : h->groups) {
        for (int p : g.probs) g.n_max = std::max(g.n_max, h->probs[p].n);
        if (g.kind == kSweepF32Warp) {
            const GroupLayout gl = pick_group_layout(g.n_max);
            g.lanes = gl.lanes;
            g.cache = gl.cache;
        }
        g.block = g.kind == kSweepF32Warp ? pick_group_layout(g.n_max).block
                  : g.kind == kSweepRot   ? 32 * sweep_rot_chains_per_block()
                  : g.kind == kSweepBatch ? kBatchThreads
                                          : pick_block(h->precision, g.n_max);
        g.smem = g.kind == kSweepDA ? 0 : group_smem(g);
        if ((int)g.smem > max_optin) return SA_EINVAL;  // n too large for on-chip state
        if (g.kind != kSweepDA && group_set_smem(g) != cudaSuccess) return SA_ECUDA;
        const int64_t tile = (g.kind == kSweepRot || g.kind == kSweepDA) ? sweep_rot_chains_per_block() : 8;  // smallest tile
        for (int p : g.probs) {
            int64_t t = tile;
            if (g.kind == kSweepBatch) {  // each problem's own tile capacity
                int lanes = 0;
                t = std::min<int64_t>(t, batch_tile_capacity(h->probs[p].cost, h->probs[p].n, &lanes));
            }
            g.items_cap += (size_t)((h->probs[p].chains + t - 1) / t);
        }
        if ((st = dalloc(h, &g.d_items, g.items_cap))) return st;
        if (h->groups.size() > 1 &&
            (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess))
            return SA_ECUDA;
    }
    if (h->groups.size() > 1 && cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess)
        return SA_ECUDA;
    h->max_argmin_blocks = 1;

    // device memory
    if ((st = dalloc(h, &h->d_probs, P)) ||
        (st = dalloc(h, &h->d_run, 1)) || (st = dalloc(h, &h->d_T, h->levels_total)) ||
        (st = dalloc(h, &h->d_s, h->levels_total)) || (st = dalloc(h, &h->d_F, h->total_chains)))
        return st;
    if (h->precision == SA_FP64) { if ((st = dalloc(h, &h->d_X64, h->total_x))) return st; }
    else if ((st = dalloc(h, &h->d_X32, h->total_x))) return st;
    const int tl = h->sch.trace_levels < h->levels_total ? h->sch.trace_levels : h->levels_total;
    if (tl > 0 && (st = dalloc(h, &h->d_bits, (size_t)tl * h->total_chains * h->words))) return st;

    std::vector<ProbDev>& pd = h->pd;
    pd.resize(P);
    for (int p = 0; p < P; ++p) {
        HostProb& hp = h->probs[p];
        const int n = hp.n;
        ProbDev d{};
        d.cost = hp.cost;
        d.n = n;
        d.chains = hp.chains;
        d.chain_base = hp.chain_base;
        d.x_base = hp.x_base;
        d.pid = (uint32_t)p;
        const int64_t span = (int64_t)kArgminThreads * kArgminPerThread;
        d.nblk_argmin = (int32_t)((hp.chains + span - 1) / span);
        if (d.nblk_argmin > h->max_argmin_blocks) h->max_argmin_blocks = d.nblk_argmin;
        std::vector<double> sig(n);
        std::vector<float> lo32(n), hi32(n), sig32(n);
        bool uniform = true;
        for (int k = 0; k < n; ++k) {
            sig[k] = h->sch.sigma_frac * (hp.hi[k] - hp.lo[k]);
            lo32[k] = round_up_f(hp.lo[k]);
            hi32[k] = round_down_f(hp.hi[k]);
            if (lo32[k] > hi32[k]) lo32[k] = hi32[k] = (float)hp.lo[k];
            sig32[k] = (float)sig[k];
            uniform = uniform && hp.lo[k] == hp.lo[0] && hp.hi[k] == hp.hi[0];
        }
        d.uniform = uniform ? 1 : 0;
        d.lo_u = lo32[0];
        d.hi_u = hi32[0];
        d.sig_u = sig32[0];
        d.unroll = pick_unroll(hp.cost, n);
        d.rand_batch = pick_rand_batch();
        d.warp_mode = 0;
        d.kappa = step_kappa(hp.cost, n, lo32, hi32);
        double *dlo, *dhi, *dsig, *xb64, *xinc, *scal, *pval, *lf, *lfi;
        float *dlo32, *dhi32, *dsig32, *xb32;
        unsigned long long *lmin, *acc;
        unsigned int* done;
        // partial argmins: one per argmin block, per 32-chain tile, and per batch tile
        int blanes = 0;
        const int64_t bcap = std::max(1, batch_tile_capacity(hp.cost, hp.n, &blanes));
        const int64_t nparts = std::max<int64_t>(std::max<int64_t>(d.nblk_argmin, (hp.chains + 31) / 32),
                                                 (hp.chains + bcap - 1) / bcap);
        int64_t *pidx, *la;
        long long* lt;
        if ((st = dalloc(h, &dlo, n)) || (st = dalloc(h, &dhi, n)) || (st = dalloc(h, &dsig, n)) ||
            (st = dalloc(h, &dlo32, n)) || (st = dalloc(h, &dhi32, n)) || (st = dalloc(h, &dsig32, n)) ||
            (st = dalloc(h, &xb64, n)) || (st = dalloc(h, &xb32, n)) || (st = dalloc(h, &xinc, n)) ||
            (st = dalloc(h, &scal, kNumScalars)) || (st = dalloc(h, &lmin, 1)) || (st = dalloc(h, &done, 1)) ||
            (st = dalloc(h, &pval, nparts)) || (st = dalloc(h, &pidx, nparts)) ||
            (st = dalloc(h, &la, h->levels_total)) || (st = dalloc(h, &lf, h->levels_total)) ||
            (st = dalloc(h, &lfi, h->levels_total)) || (st = dalloc(h, &lt, h->levels_total)) ||
            (st = dalloc(h, &acc, 1)))
            return st;
        d.lo = dlo; d.hi = dhi; d.sig = dsig; d.lo32 = dlo32; d.hi32 = dhi32; d.sig32 = dsig32;
        d.x_best64 = xb64; d.x_best32 = xb32; d.x_inc = xinc; d.scal = scal; d.level_min = lmin; d.done = done;
        d.part_val = pval; d.part_idx = pidx; d.log_argmin = la; d.log_f = lf; d.log_finc = lfi; d.log_t = lt;
        d.accepts = acc;
        if (is_rot(hp.cost) && (st = setup_rot(h, hp, d))) return st;
        if (is_table(hp.cost)) {
            double* dt;
            if ((st = dalloc(h, &dt, hp.table.size())) || (st = h2d(h, dt, hp.table.data(), hp.table.size()))) return st;
            d.table = dt;
            d.table_rows = hp.table_rows;
        }
        hp.dev = d;
        pd[p] = d;
        std::vector<double> sc(kNumScalars, 0.0);
        sc[kFBest] = INFINITY;
        sc[kFInc] = INFINITY;
        const unsigned long long inf_key = 0xFFF0000000000000ull;
        const unsigned int zero = 0;
        const unsigned long long zero64 = 0;
        std::vector<double> zeros(n, 0.0);
        std::vector<float> zf(n, 0.0f);
        if ((st = h2d(h, dlo, hp.lo.data(), n)) || (st = h2d(h, dhi, hp.hi.data(), n)) ||
            (st = h2d(h, dsig, sig.data(), n)) || (st = h2d(h, dlo32, lo32.data(), n)) ||
            (st = h2d(h, dhi32, hi32.data(), n)) || (st = h2d(h, dsig32, sig32.data(), n)) ||
            (st = h2d(h, scal, sc.data(), kNumScalars)) || (st = h2d(h, lmin, &inf_key, 1)) ||
            (st = h2d(h, done, &zero, 1)) || (st = h2d(h, acc, &zero64, 1)) || (st = h2d(h, xinc, zeros.data(), n)) ||
            (st = h2d(h, xb64, zeros.data(), n)) || (st = h2d(h, xb32, zf.data(), n)))
            return st;
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SA_ECUDA;  // host temporaries die here
    }
    std::vector<double> T(h->levels_total), s(h->levels_total);
    double Tl = h->sch.T0;
    for (int l = 0; l < h->levels_total; ++l) {
        T[l] = Tl;
        s[l] = std::sqrt(Tl / h->sch.T0);
        Tl = Tl * h->sch.rho;
    }
    RunDev run{0, 0, 0};
    for (Group& g : h->groups) {
        for (int p : g.probs) pd[p].warp_mode = g.kind == kSweepF32Warp ? 1 : 0;
        if ((st = set_group_items(h, g))) return st;
    }
    if ((st = h2d(h, h->d_probs, pd.data(), P)) ||
        (st = h2d(h, h->d_run, &run, 1)) || (st = h2d(h, h->d_T, T.data(), T.size())) ||
        (st = h2d(h, h->d_s, s.data(), s.size())))
        return st;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SA_ECUDA;

    SweepArgs& a = h->args;
    a.probs = h->d_probs;
    a.items = nullptr;  // per group at launch
    a.run = h->d_run;
    a.T_tab = h->d_T;
    a.s_tab = h->d_s;
    a.F = h->d_F;
    a.X32 = h->d_X32;
    a.X64 = h->d_X64;
    a.bits = h->d_bits;
    a.total_chains = h->total_chains;
    a.L = h->L;
    a.words = h->words;
    a.trace_levels = tl;
    a.full_level = h->sch.polish_k > 0 ? h->levels_total - 1 : -1;
    if (h->sch.polish_k > 0) {
        int n_max = 1;
        for (auto& hp : h->probs) n_max = std::max(n_max, hp.n);
        const size_t k = (size_t)h->sch.polish_k;
        if ((st = dalloc(h, &h->d_Fcopy, h->total_chains)) || (st = dalloc(h, &h->d_topk, k)) ||
            (st = dalloc(h, &h->d_px0, k * n_max)) || (st = dalloc(h, &h->d_px, k * n_max)) ||
            (st = dalloc(h, &h->d_pf, k)) || (st = dalloc(h, &h->d_pit, k)))
            return st;
        if (h->sch.polish_method != SA_POLISH_PGD) {
            if (n_max > nm_max_n() || k * nm_ws_doubles(n_max) * sizeof(double) > ((size_t)1 << 32)) return SA_EINVAL;
            if ((st = dalloc(h, &h->d_nmws, k * nm_ws_doubles(n_max)))) return st;
            h->nm_step = std::min(1.0, h->sch.sigma_frac * s.back());  // s[l] = sqrt(T_l / T0)
        }
    }
    a.boundary = h->sch.boundary;
    a.proposal = h->sch.proposal;
    a.crossover = h->sch.crossover;
    a.levels_total = h->levels_total;
    if (h->sch.crossover) {
        int64_t cmax = 1;
        size_t xbytes = 16;
        for (auto& hp : h->probs) {
            cmax = std::max(cmax, hp.chains);
            const size_t total = (size_t)hp.chains * (size_t)hp.n;
            xbytes = std::max(xbytes, total * (is_rot(hp.cost) ? 12 : (h->precision == SA_FP64 ? 8 : 4)) + 16);
        }
        unsigned char* xt;
        if ((st = dalloc(h, &h->xo.w, (size_t)cmax)) || (st = dalloc(h, &h->xo.S, (size_t)cmax)) ||
            (st = dalloc(h, &h->xo.bsum, crossover_blocks(cmax) + 1)) || (st = dalloc(h, &h->xo.src, (size_t)cmax)) ||
            (st = dalloc(h, &xt, xbytes)))
            return st;
        h->xo.xtmp = xt;
        h->xkey0 = (uint32_t)h->seed;
        h->xkey1 = (uint32_t)(h->seed >> 32) ^ kTagCrossover;
    }
    a.key0 = (uint32_t)h->seed;
    a.key1 = (uint32_t)(h->seed >> 32) ^ kTagSweep;
    a.ikey0 = (uint32_t)h->seed;
    a.ikey1 = (uint32_t)(h->seed >> 32) ^ kTagInit;
    for (int r = 0; r < 10; ++r) {  // Philox key schedule k + r (W0, W1)
        a.rk[2 * r] = a.key0 + (uint32_t)r * 0x9E3779B9u;
        a.rk[2 * r + 1] = a.key1 + (uint32_t)r * 0xBB67AE85u;
    }

    a.cost_repeat = h->sch.cost_repeat > 1 ? h->sch.cost_repeat : 1;
    a.independent = h->sch.independent;
    a.exchange_every = h->sch.exchange_every > 1 ? h->sch.exchange_every : 1;
    if (h->sch.surrogate && (st = setup_da(h))) return st;

    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return SA_ECUDA;
    if ((st = capture_levels(h, 1, &h->g1))) return st;
    if (h->levels_total >= kGraphLevels && !h->da && (st = capture_levels(h, kGraphLevels, &h->gN))) return st;

    uint64_t fp = 1469598103934665603ull;
    fp = fnv(fp, &h->sch, sizeof(h->sch));
    fp = fnv(fp, &h->seed, sizeof(h->seed));
    fp = fnv(fp, &h->L, sizeof(h->L));
    for (auto& hp : h->probs) {
        fp = fnv(fp, hp.Q.data(), hp.Q.size() * sizeof(double));
        fp = fnv(fp, hp.table.data(), hp.table.size() * sizeof(double));
        fp = fnv(fp, &hp.cost, sizeof(hp.cost));
        fp = fnv(fp, &hp.n, sizeof(hp.n));
        fp = fnv(fp, &hp.chains, sizeof(hp.chains));
        fp = fnv(fp, hp.lo.data(), hp.lo.size() * sizeof(double));
        fp = fnv(fp, hp.hi.data(), hp.hi.size() * sizeof(double));
    }
    h->fingerprint = fp;
    return SA_OK;
}

cudaError_t launch_level0_prep(sa_handle* h, cudaStream_t s) {
    cudaError_t e = launch_stamp_start(h->d_run, s);
    if (e == cudaSuccess && h->da) e = da_run_start(h->dd, h->seed, s);
    for (size_t p = 0; p < h->probs.size() && e == cudaSuccess; ++p) {
        const HostProb& hp = h->probs[p];
        if (is_rot(hp.cost))
            e = launch_rot_level0(h->d_probs + p, hp.dev, h->args, const_cast<float*>(hp.dev.x0),
                                  const_cast<float2*>(hp.dev.y0), hp.tc_work, &h->d_run->status, s);
    }
    return e;
}

}  // namespace

extern "C" {

void sa_default_schedule(sa_schedule* s) {
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
    s->T0 = 100.0;
    s->rho = 0.9;
    s->T_min = 0.0;
    s->levels = 50;
    s->sigma_frac = 0.1;
    s->boundary = SA_REFLECT;
    s->precision = SA_FP64;
}

int32_t sa_levels_for(double T0, double rho, double T_min) {
    if (!(T0 > 0.0) || !(rho > 0.0 && rho < 1.0) || !(T_min > 0.0)) return -1;
    double T = T0;
    int32_t k = 0;
    do {
        ++k;
        T = T * rho;
    } while (T > T_min && k < 100000000);
    return k;
}

const char* sa_strerror(sa_status s) {
    switch (s) {
    case SA_OK: return "ok";
    case SA_EINVAL: return "invalid argument";
    case SA_ENOMEM: return "out of memory";
    case SA_ECUDA: return "CUDA error";
    case SA_ETIMEOUT: return "bounded device wait timed out";
    case SA_ENUMERIC: return "non-finite best state";
    case SA_ESTATE: return "handle in error state or call out of order";
    }
    return "unknown status";
}

sa_status sa_create(const sa_problem* problem, const sa_box* box, int32_t n, int64_t chains, int32_t L,
                    const sa_schedule* schedule, uint64_t seed, void* stream, sa_handle** out) {
    if (out) *out = nullptr;
    if (!problem || !box || !out || L < 1) return SA_EINVAL;
    if (check_schedule(schedule) != SA_OK) return SA_EINVAL;
    if (check_problem(*problem, *box, n, chains, *schedule) != SA_OK) return SA_EINVAL;
    sa_handle* h = new (std::nothrow) sa_handle();
    if (!h) return SA_ENOMEM;
    h->stream = static_cast<cudaStream_t>(stream);
    h->sch = *schedule;
    h->seed = seed;
    h->L = L;
    h->precision = schedule->precision;
    sa_status st = build(h, problem, box, &n, &chains, 1);
    if (st != SA_OK) {
        sa_destroy(h);
        return st;
    }
    *out = h;
    return SA_OK;
}

sa_status sa_run(sa_handle* h, int32_t levels) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (levels == 0 || levels < -1) return SA_EINVAL;
    const int remaining = h->levels_total - h->levels_done;
    if (remaining <= 0) return SA_ESTATE;
    int k = (levels == -1 || levels > remaining) ? remaining : levels;
    if (h->levels_done == 0 && launch_level0_prep(h, h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    while (k > 0) {
        cudaError_t e;
        int step;
        if (h->gN && k >= kGraphLevels) { e = cudaGraphLaunch(h->gN, h->stream); step = kGraphLevels; }
        else { e = cudaGraphLaunch(h->g1, h->stream); step = 1; }
        if (e != cudaSuccess) return fail(h, SA_ECUDA);
        h->levels_done += step;
        k -= step;
    }
    if (h->levels_done == h->levels_total) return run_polish(h);
    return SA_OK;
}

sa_status sa_reset(sa_handle* h) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (launch_reset(h->d_probs, (int)h->probs.size(), h->d_run, h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    h->levels_done = 0;
    return SA_OK;
}

sa_status sa_profile(sa_handle* h, int32_t levels, double* sweep_ms, double* level_ms) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (levels == 0 || levels < -1) return SA_EINVAL;
    const int remaining = h->levels_total - h->levels_done;
    if (remaining <= 0) return SA_ESTATE;
    const int k = (levels == -1 || levels > remaining) ? remaining : levels;
    std::vector<cudaEvent_t> ev(3 * (size_t)k + 1, nullptr);  // the last one: before the start-up work
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (auto& f : ev) if (f) cudaEventDestroy(f);
            return fail(h, SA_ECUDA);
        }
    sa_status st = SA_OK;
    const bool from0 = h->levels_done == 0;
    if (cudaEventRecord(ev[3 * (size_t)k], h->stream) != cudaSuccess ||
        (from0 && launch_level0_prep(h, h->stream) != cudaSuccess))
        st = SA_ECUDA;
    for (int l = 0; l < k && st == SA_OK; ++l) {
        if (cudaEventRecord(ev[3 * l], h->stream) != cudaSuccess || launch_sweep(h, h->stream) != cudaSuccess ||
            cudaEventRecord(ev[3 * l + 1], h->stream) != cudaSuccess || launch_level_tail(h, h->stream) != cudaSuccess ||
            cudaEventRecord(ev[3 * l + 2], h->stream) != cudaSuccess)
            st = SA_ECUDA;
        else
            h->levels_done += 1;
    }
    if (st == SA_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = SA_ECUDA;
    for (int l = 0; l < k && st == SA_OK; ++l) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, ev[3 * l], ev[3 * l + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&b, ev[(l == 0 && from0) ? 3 * (size_t)k : 3 * l], ev[3 * l + 2]) != cudaSuccess) {
            st = SA_ECUDA;
            break;
        }
        if (sweep_ms) sweep_ms[l] = a;
        if (level_ms) level_ms[l] = b;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (st == SA_OK && h->levels_done == h->levels_total) return run_polish(h);
    return st == SA_OK ? SA_OK : fail(h, st);
}

sa_status sa_gemm_bf16(const void* d_A, int32_t lda, const void* d_B, int32_t ldb, float* d_D, int32_t ldd, int32_t M,
                       int32_t N, int32_t K, int32_t* d_status, void* stream) {
    if (!d_A || !d_B || !d_D || M <= 0 || N <= 0 || K <= 0 || lda < K || ldb < K || ldd < N) return SA_EINVAL;
    if (M % 128 || N % 64 || K % 64 || ldd % 4) return SA_EINVAL;
    int* st = d_status ? d_status : gemm_status_ptr();
    const cudaError_t e = launch_gemm_bf16_f32(d_A, lda, d_B, ldb, d_D, ldd, M, N, K, st, static_cast<cudaStream_t>(stream));
    if (e == cudaErrorInvalidValue) { cudaGetLastError(); return SA_EINVAL; }
    return e == cudaSuccess ? SA_OK : SA_ECUDA;
}

sa_status sa_rotate_rows(const float* d_X, int64_t rows, int32_t n, const double* d_Q, float* d_Y, int32_t* d_status,
                         void* stream) {
    if (!d_X || !d_Q || !d_Y || rows < 1 || n < 1) return SA_EINVAL;
    if (!rot_tc_shape_ok(rows, n)) return SA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* w = nullptr;
    if (cudaMallocAsync(&w, rot_tc_work_bytes(rows, n), s) != cudaSuccess) {
        cudaGetLastError();
        return SA_ENOMEM;
    }
    int* st = d_status ? d_status : gemm_status_ptr();
    const cudaError_t e = launch_rot_tc(d_X, rows, n, d_Q, reinterpret_cast<float2*>(d_Y), w, st, s);
    cudaFreeAsync(w, s);
    return e == cudaSuccess ? SA_OK : SA_ECUDA;
}

sa_status sa_polish(int32_t cost, int32_t n, const double* lo, const double* hi, const double* Q, int32_t k,
                    const double* x0, int32_t max_iter, double tol, double* x_out, double* f_out, int32_t* iters_out,
                    void* stream) {
    if (n < 1 || k < 1 || k > 1024 || !lo || !hi || !x0 || !x_out || !f_out || max_iter < 0 || !(tol >= 0.0))
        return SA_EINVAL;
    if (cost < SA_SCHWEFEL || cost > SA_ROT_SCHWEFEL) return SA_EINVAL;
    const bool rot = is_rot(cost);
    if (rot != (Q != nullptr) || (rot && (int64_t)n * n > ((int64_t)1 << 28))) return SA_EINVAL;
    for (int d = 0; d < n; ++d)
        if (!std::isfinite(lo[d]) || !std::isfinite(hi[d]) || lo[d] > hi[d]) return SA_EINVAL;
    if (rot)
        for (size_t e = 0; e < (size_t)n * n; ++e)
            if (!std::isfinite(Q[e])) return SA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *dlo = nullptr, *dhi = nullptr, *dx0 = nullptr, *dx = nullptr, *df = nullptr, *dq = nullptr;
    int* dit = nullptr;
    const size_t kn = (size_t)k * n;
    sa_status st = SA_OK;
    if ((rot && cudaMallocAsync(&dq, (size_t)n * n * sizeof(double), s)) ||
        cudaMallocAsync(&dlo, n * sizeof(double), s) || cudaMallocAsync(&dhi, n * sizeof(double), s) ||
        cudaMallocAsync(&dx0, kn * sizeof(double), s) || cudaMallocAsync(&dx, kn * sizeof(double), s) ||
        cudaMallocAsync(&df, k * sizeof(double), s) || cudaMallocAsync(&dit, k * sizeof(int), s))
        st = SA_ENOMEM;
    if (st == SA_OK &&
        ((rot && cudaMemcpyAsync(dq, Q, (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice, s)) ||
         cudaMemcpyAsync(dlo, lo, n * sizeof(double), cudaMemcpyHostToDevice, s) ||
         cudaMemcpyAsync(dhi, hi, n * sizeof(double), cudaMemcpyHostToDevice, s) ||
         cudaMemcpyAsync(dx0, x0, kn * sizeof(double), cudaMemcpyHostToDevice, s) ||
         launch_pgd(cost, n, dlo, dhi, dq, k, dx0, dx, df, dit, max_iter, tol, s) ||
         cudaMemcpyAsync(x_out, dx, kn * sizeof(double), cudaMemcpyDeviceToHost, s) ||
         cudaMemcpyAsync(f_out, df, k * sizeof(double), cudaMemcpyDeviceToHost, s) ||
         (iters_out && cudaMemcpyAsync(iters_out, dit, k * sizeof(int), cudaMemcpyDeviceToHost, s)) ||
         cudaStreamSynchronize(s)))
        st = SA_ECUDA;
    for (void* p : {(void*)dlo, (void*)dhi, (void*)dx0, (void*)dx, (void*)df, (void*)dit, (void*)dq})
        if (p) cudaFreeAsync(p, s);
    cudaGetLastError();
    return st;
}

sa_status sa_nelder_mead(int32_t cost, int32_t n, const double* lo, const double* hi, const double* Q,
                         const double* table, int32_t table_rows, int32_t k, const double* x0, double step_frac,
                         int32_t max_iter, double ftol, double xtol, int32_t adaptive, double* x_out,
                         double* f_out, int32_t* iters_out, void* stream) {
    if (adaptive != 0 && adaptive != 1) return SA_EINVAL;
    if (n < 1 || k < 1 || k > 1024 || !lo || !hi || !x0 || !x_out || !f_out || max_iter < 0 || !(ftol >= 0.0) ||
        !(xtol >= 0.0) || !(step_frac > 0.0 && step_frac <= 1.0))
        return SA_EINVAL;
    if (!cost_args_ok(cost, n, Q, table, table_rows) || n > nm_max_n()) return SA_EINVAL;
    const bool rot = is_rot(cost);
    const size_t ws = (size_t)k * nm_ws_doubles(n);
    if (ws * sizeof(double) > ((size_t)1 << 32)) return SA_EINVAL;
    for (int d = 0; d < n; ++d)
        if (!std::isfinite(lo[d]) || !std::isfinite(hi[d]) || lo[d] > hi[d]) return SA_EINVAL;
    std::vector<double> qt;
    if (rot) {
        qt.resize((size_t)n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) qt[(size_t)j * n + i] = Q[(size_t)i * n + j];
    }
    const size_t tn = table ? (size_t)table_rows * (size_t)(n + 1) : 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *dlo = nullptr, *dhi = nullptr, *dx0 = nullptr, *dx = nullptr, *df = nullptr, *dq = nullptr, *dws = nullptr;
    double* dtab = nullptr;
    int* dit = nullptr;
    const size_t kn = (size_t)k * n;
    sa_status st = SA_OK;
    if ((rot && cudaMallocAsync(&dq, (size_t)n * n * sizeof(double), s)) ||
        cudaMallocAsync(&dlo, n * sizeof(double), s) || cudaMallocAsync(&dhi, n * sizeof(double), s) ||
        cudaMallocAsync(&dx0, kn * sizeof(double), s) || cudaMallocAsync(&dx, kn * sizeof(double), s) ||
        cudaMallocAsync(&df, k * sizeof(double), s) || cudaMallocAsync(&dit, k * sizeof(int), s) ||
        cudaMallocAsync(&dws, ws * sizeof(double), s) || (tn && cudaMallocAsync(&dtab, tn * sizeof(double), s)))
        st = SA_ENOMEM;
    if (st == SA_OK &&
        ((rot && cudaMemcpyAsync(dq, qt.data(), (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice, s)) ||
         cudaMemcpyAsync(dlo, lo, n * sizeof(double), cudaMemcpyHostToDevice, s) ||
         cudaMemcpyAsync(dhi, hi, n * sizeof(double), cudaMemcpyHostToDevice, s) ||
         cudaMemcpyAsync(dx0, x0, kn * sizeof(double), cudaMemcpyHostToDevice, s) ||
         (tn && cudaMemcpyAsync(dtab, table, tn * sizeof(double), cudaMemcpyHostToDevice, s)) ||
         launch_nm(cost, n, dlo, dhi, dq, dtab, table_rows, k, dx0, dx, df, dit, step_frac, max_iter, ftol, xtol,
                   adaptive != 0, dws, s) ||
         cudaMemcpyAsync(x_out, dx, kn * sizeof(double), cudaMemcpyDeviceToHost, s) ||
         cudaMemcpyAsync(f_out, df, k * sizeof(double), cudaMemcpyDeviceToHost, s) ||
         (iters_out && cudaMemcpyAsync(iters_out, dit, k * sizeof(int), cudaMemcpyDeviceToHost, s)) ||
         cudaStreamSynchronize(s)))
        st = SA_ECUDA;
    for (void* p : {(void*)dlo, (void*)dhi, (void*)dx0, (void*)dx, (void*)df, (void*)dit, (void*)dq, (void*)dws,
                    (void*)dtab})
        if (p) cudaFreeAsync(p, s);
    cudaGetLastError();
    return st;
}

sa_status sa_best(sa_handle* h, int32_t problem, double* x_out, double* f_out, sa_stats* stt) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (problem < 0 || problem >= (int)h->probs.size()) return SA_EINVAL;
    if (h->levels_done == 0) return SA_ESTATE;
    sa_status st = device_status(h);
    if (st != SA_OK) return st;
    const HostProb& hp = h->probs[problem];
    std::vector<double> sc(kNumScalars);
    unsigned long long acc = 0, rech = 0, evals = 0;
    int64_t am = -1;
    long long t0 = 0;
    h->d2h_bytes += (int64_t)(sizeof(double) * kNumScalars + sizeof(acc) + sizeof(am) + sizeof(t0) +
                              (x_out ? sizeof(double) * hp.n : 0));
    if (cudaMemcpyAsync(sc.data(), hp.dev.scal, sizeof(double) * kNumScalars, cudaMemcpyDeviceToHost, h->stream) ||
        cudaMemcpyAsync(&t0, &h->d_run->t_start, sizeof(t0), cudaMemcpyDeviceToHost, h->stream) ||
        cudaMemcpyAsync(&acc, hp.dev.accepts, sizeof(acc), cudaMemcpyDeviceToHost, h->stream) ||
        (hp.dev.rechecks && cudaMemcpyAsync(&rech, hp.dev.rechecks, sizeof(rech), cudaMemcpyDeviceToHost, h->stream)) ||
        (h->da && cudaMemcpyAsync(&evals, h->dd.evals, sizeof(evals), cudaMemcpyDeviceToHost, h->stream)) ||
        cudaMemcpyAsync(&am, hp.dev.log_argmin + (h->levels_done - 1), sizeof(am), cudaMemcpyDeviceToHost, h->stream) ||
        (x_out && cudaMemcpyAsync(x_out, hp.dev.x_inc, sizeof(double) * hp.n, cudaMemcpyDeviceToHost, h->stream)) ||
        cudaStreamSynchronize(h->stream))
        return fail(h, SA_ECUDA);
    if (f_out) *f_out = sc[kFInc];
    if (stt) {
        stt->steps = hp.chains * (int64_t)h->L * h->levels_done;
        stt->accepts = (int64_t)acc;
        stt->levels_done = h->levels_done;
        stt->levels_total = h->levels_total;
        stt->f_level = sc[kFBest];
        stt->argmin = am;
        stt->h2d_bytes = h->h2d_bytes;
        stt->d2h_bytes = h->d2h_bytes;
        stt->t_start_ns = t0;
        stt->rechecks = (int64_t)rech;
        stt->true_evals = h->da ? (int64_t)evals : stt->steps;
    }
    return SA_OK;
}

sa_status sa_set_chain_offset(sa_handle* h, int64_t offset) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (h->probs.size() != 1 || offset < 0 || offset + h->probs[0].chains > ((int64_t)1 << 32)) return SA_EINVAL;
    if (h->sch.crossover) return SA_EINVAL;  // the crossover draws among one handle's chains
    if (h->levels_done != 0) return SA_ESTATE;
    h->pd[0].cid0 = (uint32_t)offset;
    h->probs[0].dev.cid0 = (uint32_t)offset;
    if (h2d(h, h->d_probs, h->pd.data(), h->pd.size()) != SA_OK || cudaStreamSynchronize(h->stream) != cudaSuccess)
        return fail(h, SA_ECUDA);
    return SA_OK;
}

sa_status sa_restart_point(sa_handle* h, int32_t problem, double* x_out, double* f_out) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (problem < 0 || problem >= (int)h->probs.size()) return SA_EINVAL;
    if (h->levels_done == 0) return SA_ESTATE;
    sa_status st = device_status(h);
    if (st != SA_OK) return st;
    const HostProb& hp = h->probs[problem];
    if (x_out) {
        if (h->precision == SA_FP64) {
            if (cudaMemcpy(x_out, hp.dev.x_best64, sizeof(double) * hp.n, cudaMemcpyDeviceToHost)) return fail(h, SA_ECUDA);
        } else {
            std::vector<float> xf(hp.n);
            if (cudaMemcpy(xf.data(), hp.dev.x_best32, sizeof(float) * hp.n, cudaMemcpyDeviceToHost)) return fail(h, SA_ECUDA);
            for (int k = 0; k < hp.n; ++k) x_out[k] = xf[k];
        }
        h->d2h_bytes += (int64_t)(sizeof(double) * hp.n);
    }
    if (f_out && cudaMemcpy(f_out, hp.dev.scal + kFBest, sizeof(double), cudaMemcpyDeviceToHost)) return fail(h, SA_ECUDA);
    return SA_OK;
}

sa_status sa_set_restart(sa_handle* h, int32_t problem, const double* x, double f, int64_t argmin) {
    if (!h || !x) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (problem < 0 || problem >= (int)h->probs.size() || !std::isfinite(f)) return SA_EINVAL;
    if (h->levels_done == 0) return SA_ESTATE;
    HostProb& hp = h->probs[problem];
    for (int k = 0; k < hp.n; ++k)
        if (!(x[k] >= hp.lo[k] && x[k] <= hp.hi[k])) return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    const ProbDev& d = hp.dev;
    double finc = 0.0;
    if (cudaMemcpy(&finc, d.scal + kFInc, sizeof(double), cudaMemcpyDeviceToHost)) return fail(h, SA_ECUDA);
    std::vector<float> xf(hp.n);
    for (int k = 0; k < hp.n; ++k) xf[k] = (float)x[k];
    const int l = h->levels_done - 1;
    const double fi = f < finc ? f : finc;
    if (cudaMemcpy(d.x_best64, x, sizeof(double) * hp.n, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d.x_best32, xf.data(), sizeof(float) * hp.n, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d.scal + kFBest, &f, sizeof(double), cudaMemcpyHostToDevice) ||
        (f < finc && (cudaMemcpy(d.x_inc, x, sizeof(double) * hp.n, cudaMemcpyHostToDevice) ||
                      cudaMemcpy(d.scal + kFInc, &f, sizeof(double), cudaMemcpyHostToDevice))) ||
        cudaMemcpy(d.log_argmin + l, &argmin, sizeof(int64_t), cudaMemcpyHostToDevice) ||
        cudaMemcpy(d.log_f + l, &f, sizeof(double), cudaMemcpyHostToDevice) ||
        cudaMemcpy(d.log_finc + l, &fi, sizeof(double), cudaMemcpyHostToDevice))
        return fail(h, SA_ECUDA);
    h->h2d_bytes += (int64_t)(sizeof(double) * hp.n * 2 + sizeof(float) * hp.n);
    // rotated costs: the next level starts from y_best = Q x_best
    if (is_rot(hp.cost) && (launch_rot_restart(h->d_probs + problem, hp.n, h->stream) != cudaSuccess ||
                            cudaStreamSynchronize(h->stream) != cudaSuccess))
        return fail(h, SA_ECUDA);
    return SA_OK;
}

sa_status sa_da_trace(sa_handle* h, int32_t level, float* ft0_out, float* ftp_out) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (!h->da || level < 0 || level >= h->args.trace_levels || level >= h->levels_done) return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    const int64_t C = h->probs[0].chains;
    if ((ft0_out && cudaMemcpy(ft0_out, h->dd.trace_ft0 + (size_t)level * C, sizeof(float) * C, cudaMemcpyDeviceToHost)) ||
        (ftp_out && cudaMemcpy(ftp_out, h->dd.trace_ftp + (size_t)level * h->L * C, sizeof(float) * h->L * C,
                               cudaMemcpyDeviceToHost)))
        return fail(h, SA_ECUDA);
    return SA_OK;
}

sa_status sa_da_network(sa_handle* h, float* params_out, float* ms_out, float* mid_out, float* inv_half_out) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (!h->da || h->levels_done < 1) return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    const int n = h->probs[h->dd.problem].n;
    const int64_t P = mlp_offsets(n).total;
    if ((params_out && cudaMemcpy(params_out, h->dd.mlp.p, sizeof(float) * P, cudaMemcpyDeviceToHost)) ||
        (ms_out && cudaMemcpy(ms_out, h->dd.ms, sizeof(float) * 2, cudaMemcpyDeviceToHost)) ||
        (mid_out && cudaMemcpy(mid_out, h->dd.mid, sizeof(float) * n, cudaMemcpyDeviceToHost)) ||
        (inv_half_out && cudaMemcpy(inv_half_out, h->dd.inv_half, sizeof(float) * n, cudaMemcpyDeviceToHost)))
        return fail(h, SA_ECUDA);
    return SA_OK;
}

sa_status sa_level_log(sa_handle* h, int32_t problem, int64_t* argmin, double* f_level, double* f_inc, int64_t* t_ns,
                       int32_t cap, int32_t* count) {
    if (!h || cap < 0) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (problem < 0 || problem >= (int)h->probs.size()) return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    const ProbDev& d = h->probs[problem].dev;
    const int m = cap < h->levels_done ? cap : h->levels_done;
    if (m > 0) {
        if ((argmin && cudaMemcpy(argmin, d.log_argmin, sizeof(int64_t) * m, cudaMemcpyDeviceToHost)) ||
            (f_level && cudaMemcpy(f_level, d.log_f, sizeof(double) * m, cudaMemcpyDeviceToHost)) ||
            (f_inc && cudaMemcpy(f_inc, d.log_finc, sizeof(double) * m, cudaMemcpyDeviceToHost)) ||
            (t_ns && cudaMemcpy(t_ns, d.log_t, sizeof(int64_t) * m, cudaMemcpyDeviceToHost)))
            return fail(h, SA_ECUDA);
    }
    if (count) *count = m;
    return SA_OK;
}

sa_status sa_trace(sa_handle* h, int32_t level, uint32_t* bits_out, size_t nwords) {
    if (!h || !bits_out) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (level < 0 || level >= h->args.trace_levels || level >= h->levels_done) return SA_EINVAL;
    const size_t need = (size_t)h->total_chains * h->words;
    if (nwords < need) return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    if (cudaMemcpy(bits_out, h->d_bits + (size_t)level * need, need * sizeof(uint32_t), cudaMemcpyDeviceToHost))
        return fail(h, SA_ECUDA);
    return SA_OK;
}

sa_status sa_trace_states(sa_handle* h, int32_t level, double* X_out, double* F_out) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (level < 0 || level != h->levels_done - 1 || level >= h->args.trace_levels) return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    if (F_out && cudaMemcpy(F_out, h->d_F, sizeof(double) * h->total_chains, cudaMemcpyDeviceToHost))
        return fail(h, SA_ECUDA);
    if (X_out) {
        for (const HostProb& hp : h->probs) {
            const size_t cnt = (size_t)hp.n * hp.chains;
            std::vector<double> tmp(cnt);
            if (h->precision == SA_FP64) {
                if (cudaMemcpy(tmp.data(), h->d_X64 + hp.x_base, cnt * sizeof(double), cudaMemcpyDeviceToHost))
                    return fail(h, SA_ECUDA);
            } else {
                std::vector<float> tf(cnt);
                if (cudaMemcpy(tf.data(), h->d_X32 + hp.x_base, cnt * sizeof(float), cudaMemcpyDeviceToHost))
                    return fail(h, SA_ECUDA);
                for (size_t i = 0; i < cnt; ++i) tmp[i] = tf[i];
            }
            double* dst = X_out + hp.x_base;
            for (int64_t c = 0; c < hp.chains; ++c)
                for (int k = 0; k < hp.n; ++k) dst[(size_t)c * hp.n + k] = tmp[(size_t)k * hp.chains + c];
        }
    }
    return SA_OK;
}

sa_status sa_checkpoint(sa_handle* h, void* buf, size_t* len) {
    if (!h || !len) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (h->da || keep_states(h->args)) return SA_EINVAL;  // the surrogate's and the chains' states are not part of a checkpoint
    size_t need = 4 * sizeof(uint32_t) + sizeof(uint64_t) + sizeof(int32_t) * 2;
    for (const HostProb& hp : h->probs)
        need += sizeof(double) * (kNumScalars + 2 * (size_t)hp.n) + sizeof(uint64_t) +
                (size_t)h->levels_done * (sizeof(int64_t) * 2 + sizeof(double) * 2);
    if (!buf) { *len = need; return SA_OK; }
    if (*len < need) return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    unsigned char* p = static_cast<unsigned char*>(buf);
    auto put = [&p](const void* src, size_t n) { std::memcpy(p, src, n); p += n; };
    const uint32_t hdr[4] = {kCkptMagic, kCkptVersion, (uint32_t)h->probs.size(), (uint32_t)h->precision};
    put(hdr, sizeof(hdr));
    put(&h->fingerprint, sizeof(uint64_t));
    put(&h->levels_done, sizeof(int32_t));
    put(&h->levels_total, sizeof(int32_t));
    for (const HostProb& hp : h->probs) {
        const ProbDev& d = hp.dev;
        std::vector<double> sc(kNumScalars), xb(hp.n), xi(hp.n);
        unsigned long long acc = 0;
        const int m = h->levels_done;
        std::vector<int64_t> la(m), lt(m);
        std::vector<double> lf(m), lfi(m);
        if (cudaMemcpy(sc.data(), d.scal, sizeof(double) * kNumScalars, cudaMemcpyDeviceToHost) ||
            cudaMemcpy(xi.data(), d.x_inc, sizeof(double) * hp.n, cudaMemcpyDeviceToHost) ||
            cudaMemcpy(&acc, d.accepts, sizeof(acc), cudaMemcpyDeviceToHost))
            return fail(h, SA_ECUDA);
        if (h->precision == SA_FP64) {
            if (cudaMemcpy(xb.data(), d.x_best64, sizeof(double) * hp.n, cudaMemcpyDeviceToHost)) return fail(h, SA_ECUDA);
        } else {
            std::vector<float> xf(hp.n);
            if (cudaMemcpy(xf.data(), d.x_best32, sizeof(float) * hp.n, cudaMemcpyDeviceToHost)) return fail(h, SA_ECUDA);
            for (int k = 0; k < hp.n; ++k) xb[k] = xf[k];
        }
        if (m > 0 && (cudaMemcpy(la.data(), d.log_argmin, sizeof(int64_t) * m, cudaMemcpyDeviceToHost) ||
                      cudaMemcpy(lf.data(), d.log_f, sizeof(double) * m, cudaMemcpyDeviceToHost) ||
                      cudaMemcpy(lfi.data(), d.log_finc, sizeof(double) * m, cudaMemcpyDeviceToHost) ||
                      cudaMemcpy(lt.data(), d.log_t, sizeof(int64_t) * m, cudaMemcpyDeviceToHost)))
            return fail(h, SA_ECUDA);
        put(sc.data(), sizeof(double) * kNumScalars);
        put(xb.data(), sizeof(double) * hp.n);
        put(xi.data(), sizeof(double) * hp.n);
        put(&acc, sizeof(uint64_t));
        put(la.data(), sizeof(int64_t) * m);
        put(lf.data(), sizeof(double) * m);
        put(lfi.data(), sizeof(double) * m);
        put(lt.data(), sizeof(int64_t) * m);
    }
    *len = need;
    return SA_OK;
}

sa_status sa_restore(sa_handle* h, const void* buf, size_t len) {
    if (!h || !buf) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (h->da || keep_states(h->args)) return SA_EINVAL;
    const unsigned char* p = static_cast<const unsigned char*>(buf);
    const unsigned char* end = p + len;
    auto get = [&p, end](void* dst, size_t n) {
        if ((size_t)(end - p) < n) return false;
        std::memcpy(dst, p, n);
        p += n;
        return true;
    };
    uint32_t hdr[4];
    uint64_t fp;
    int32_t done, total;
    if (!get(hdr, sizeof(hdr)) || !get(&fp, sizeof(fp)) || !get(&done, sizeof(done)) || !get(&total, sizeof(total)))
        return SA_EINVAL;
    if (hdr[0] != kCkptMagic || hdr[1] != kCkptVersion || hdr[2] != h->probs.size() || hdr[3] != (uint32_t)h->precision ||
        fp != h->fingerprint || total != h->levels_total || done < 0 || done > total)
        return SA_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    for (const HostProb& hp : h->probs) {
        const ProbDev& d = hp.dev;
        std::vector<double> sc(kNumScalars), xb(hp.n), xi(hp.n);
        uint64_t acc;
        std::vector<int64_t> la(done), lt(done);
        std::vector<double> lf(done), lfi(done);
        if (!get(sc.data(), sizeof(double) * kNumScalars) || !get(xb.data(), sizeof(double) * hp.n) ||
            !get(xi.data(), sizeof(double) * hp.n) || !get(&acc, sizeof(acc)) || !get(la.data(), sizeof(int64_t) * done) ||
            !get(lf.data(), sizeof(double) * done) || !get(lfi.data(), sizeof(double) * done) ||
            !get(lt.data(), sizeof(int64_t) * done))
            return SA_EINVAL;
        std::vector<float> xf(hp.n);
        for (int k = 0; k < hp.n; ++k) xf[k] = (float)xb[k];
        if (cudaMemcpy(d.scal, sc.data(), sizeof(double) * kNumScalars, cudaMemcpyHostToDevice) ||
            cudaMemcpy(d.x_inc, xi.data(), sizeof(double) * hp.n, cudaMemcpyHostToDevice) ||
            cudaMemcpy(d.x_best64, xb.data(), sizeof(double) * hp.n, cudaMemcpyHostToDevice) ||
            cudaMemcpy(d.x_best32, xf.data(), sizeof(float) * hp.n, cudaMemcpyHostToDevice) ||
            cudaMemcpy(d.accepts, &acc, sizeof(acc), cudaMemcpyHostToDevice))
            return fail(h, SA_ECUDA);
        if (done > 0 && (cudaMemcpy(d.log_argmin, la.data(), sizeof(int64_t) * done, cudaMemcpyHostToDevice) ||
                         cudaMemcpy(d.log_f, lf.data(), sizeof(double) * done, cudaMemcpyHostToDevice) ||
                         cudaMemcpy(d.log_finc, lfi.data(), sizeof(double) * done, cudaMemcpyHostToDevice) ||
                         cudaMemcpy(d.log_t, lt.data(), sizeof(int64_t) * done, cudaMemcpyHostToDevice)))
            return fail(h, SA_ECUDA);
    }
    RunDev run{done, 0};
    if (cudaMemcpy(h->d_run, &run, sizeof(run), cudaMemcpyHostToDevice)) return fail(h, SA_ECUDA);
    // rotated costs: the next level starts from y_best = Q x_best
    for (size_t p = 0; p < h->probs.size() && done > 0; ++p)
        if (is_rot(h->probs[p].cost) &&
            (launch_rot_restart(h->d_probs + p, h->probs[p].n, h->stream) != cudaSuccess ||
             cudaStreamSynchronize(h->stream) != cudaSuccess))
            return fail(h, SA_ECUDA);
    h->levels_done = done;
    return SA_OK;
}

void sa_destroy(sa_handle* h) {
    if (!h) return;
    if (h->g1) cudaGraphExecDestroy(h->g1);
    if (h->gN) cudaGraphExecDestroy(h->gN);
    for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (Group& g : h->groups) {
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    cudaGetLastError();
    delete h;
}

sa_status sa_create_batch(const sa_problem* problems, const sa_box* boxes, const int32_t* n, const int64_t* chains,
                          int32_t num_problems, int32_t L, const sa_schedule* schedule, uint64_t seed, void* stream,
                          sa_handle** out) {
    if (out) *out = nullptr;
    if (!problems || !boxes || !n || !chains || !out || num_problems < 1 || L < 1) return SA_EINVAL;
    if (check_schedule(schedule) != SA_OK || schedule->surrogate) return SA_EINVAL;
    for (int p = 0; p < num_problems; ++p)
        if (check_problem(problems[p], boxes[p], n[p], chains[p], *schedule) != SA_OK) return SA_EINVAL;
    sa_handle* h = new (std::nothrow) sa_handle();
    if (!h) return SA_ENOMEM;
    h->stream = static_cast<cudaStream_t>(stream);
    h->sch = *schedule;
    h->seed = seed;
    h->L = L;
    h->precision = schedule->precision;
    sa_status st = build(h, problems, boxes, n, chains, num_problems);
    if (st != SA_OK) {
        sa_destroy(h);
        return st;
    }
    *out = h;
    return SA_OK;
}

sa_status sa_autotune(sa_handle* h, double* ms_out) {
    if (!h) return SA_EINVAL;
    if (h->failed != SA_OK) return SA_ESTATE;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(h, SA_ECUDA);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(h, SA_ECUDA);
    sa_status st = SA_OK;
    double total = 0.0;
    static const int kBudgets[] = {16384, 32768, 65536, 114688};
    static const int kUnrolls[] = {1, 2, 4};
    struct Shape { int kind, block, unroll, lanes; bool cache; };
    // Apply a launch shape to a group (block, shared memory, work items, per-problem unroll).
    auto apply = [h](Group& g, const Shape& c) -> sa_status {
        g.kind = c.kind;
        g.block = c.block;
        g.lanes = c.lanes;
        g.cache = c.cache;
        g.smem = group_smem(g);
        if (group_set_smem(g) != cudaSuccess) return SA_ECUDA;
        sa_status s2 = set_group_items(h, g);
        if (s2) return s2;
        for (int p : g.probs) {
            h->pd[p].unroll = (h->probs[p].cost == SA_ACKLEY) ? 1 : c.unroll;
            h->pd[p].warp_mode = c.kind == kSweepF32Warp ? 1 : 0;
        }
        return h2d(h, h->d_probs, h->pd.data(), h->pd.size());
    };
    for (Group& g : h->groups) {
        if (g.kind == kSweepF64 || g.kind == kSweepRot) continue;  // one shape only
        if (g.kind == kSweepBatch) {  // one shape (each problem's layout is fixed): time one level
            float ms = 0.f;
            if (launch_reset(h->d_probs, (int)h->probs.size(), h->d_run, h->stream) != cudaSuccess ||
                cudaEventRecord(e0, h->stream) != cudaSuccess || launch_group(h, g, h->stream) != cudaSuccess ||
                cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = SA_ECUDA;
                break;
            }
            total += ms;
            continue;
        }
        std::vector<Shape> cands;
        int last_block = -1;
        for (int budget : kBudgets) {
            int b = budget / (4 * g.n_max);
            b = std::min(256, std::max(32, (b / 32) * 32));
            if (b == last_block) continue;
            last_block = b;
            for (int u : kUnrolls) cands.push_back(Shape{kSweepF32, b, u, 32, true});
        }
        bool eligible = true;
        for (int p : g.probs) eligible = eligible && warp_eligible(h->probs[p].cost);
        if (eligible) {
            // group layouts: lanes per chain x cached terms, ~64 KiB of state per block
            static const int kLanes[] = {2, 4, 8, 32};
            for (int ln : kLanes)
                for (int ch = 0; ch < 2; ++ch) {
                    if (!sweep_f32w_layout_ok(ln, ch == 1)) continue;
                    const int per_chain = (ch ? 2 : 1) * 4 * (g.n_max + 1);
                    int b = ((65536 / per_chain) * ln / 32) * 32;
                    b = std::min(256, std::max(b, std::max(32, 8 * ln)));
                    if ((int)sweep_f32w_smem_bytes(g.n_max, ln, ch == 1, b) > 227 * 1024) continue;
                    cands.push_back(Shape{kSweepF32Warp, b, 1, ln, ch == 1});
                }
        }
        double best = 1e30;
        Shape best_shape = cands[0];
        for (const Shape& c : cands) {
            if ((st = apply(g, c))) break;
            float ms = 0.f;
            if (launch_reset(h->d_probs, (int)h->probs.size(), h->d_run, h->stream) != cudaSuccess ||
                cudaEventRecord(e0, h->stream) != cudaSuccess || launch_group(h, g, h->stream) != cudaSuccess ||
                cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = SA_ECUDA;
                break;
            }
            if (ms < best) { best = ms; best_shape = c; }
        }
        if (st != SA_OK) break;
        if ((st = apply(g, best_shape))) break;
        total += best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == SA_OK) st = h2d(h, h->d_probs, h->pd.data(), h->pd.size());
    if (st == SA_OK && launch_reset(h->d_probs, (int)h->probs.size(), h->d_run, h->stream) != cudaSuccess) st = SA_ECUDA;
    if (st == SA_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = SA_ECUDA;
    if (st != SA_OK) return fail(h, st);
    h->levels_done = 0;
    // the graphs hold the old launch shapes: capture again
    if (h->g1) { cudaGraphExecDestroy(h->g1); h->g1 = nullptr; }
    if (h->gN) { cudaGraphExecDestroy(h->gN); h->gN = nullptr; }
    if ((st = capture_levels(h, 1, &h->g1))) return fail(h, st);
    if (h->levels_total >= kGraphLevels && (st = capture_levels(h, kGraphLevels, &h->gN))) return fail(h, st);
    if (ms_out) *ms_out = total;
    return SA_OK;
}

int32_t sa_describe(const sa_handle* h, char* buf, size_t len) {
    if (!h) return -1;
    std::string s = "[";
    for (size_t i = 0; i < h->groups.size(); ++i) {
        const Group& g = h->groups[i];
        int u = g.probs.empty() ? 1 : h->pd[g.probs[0]].unroll;
        char tmp[256];
        std::snprintf(tmp, sizeof(tmp), "%s{\"kind\":\"%s\",\"problems\":%zu,\"n_max\":%d,\"block\":%d,\"smem\":%zu,\"unroll\":%d,\"items\":%zu,\"lanes\":%d,\"cache\":%d}",
                      i ? "," : "", g.kind == kSweepF64 ? "fp64" : g.kind == kSweepF32Warp ? "fp32_warp" : g.kind == kSweepRot ? "rot_warp" : g.kind == kSweepBatch ? "fp32_batch_level" : "fp32_thread",
                      g.probs.size(), g.n_max, g.block, g.smem, u, g.items.size(),
                      g.kind == kSweepF32Warp ? g.lanes : (g.kind == kSweepF32 ? 1 : 32), g.cache ? 1 : 0);
        s += tmp;
    }
    s += "]";
    if (buf && len > 0) {
        std::strncpy(buf, s.c_str(), len - 1);
        buf[len - 1] = '\0';
    }
    return (int32_t)s.size();
}

sa_status sa_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t key0, uint32_t key1, int64_t count,
                         uint32_t* d_out, void* stream) {
    if (count < 0 || (count > 0 && !d_out)) return SA_EINVAL;
    return launch_philox_fill(c0, c1, c2, c3, key0, key1, count, d_out, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SA_OK : SA_ECUDA;
}

size_t sa_argmin_scratch_bytes(int64_t count) {
    if (count < 1) return 0;
    return (size_t)argmin_num_parts(count) * 16;
}

sa_status sa_argmin_f64(const double* d_F, int64_t count, int64_t* d_index, double* d_value, void* d_scratch,
                        void* stream) {
    if (count < 1 || !d_F || !d_index || !d_value || !d_scratch) return SA_EINVAL;
    if (argmin_num_parts(count) > 2147483647LL) return SA_EINVAL;
    return launch_argmin_f64(d_F, count, d_index, d_value, d_scratch, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SA_OK : SA_ECUDA;
}

}  // extern "C"
