// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <cstdint>
#include <cstdio>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "rs.h"

namespace rs {

// ------------------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
rs_status cuda_fail(cudaError_t e, const char *what);

#define RS_CUDA(call)                                                         \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::rs::cuda_fail(e_, #call);             \
    } while (0)

// Host-side fault injection (tests): rs_inject_alloc_failures(skip, count) lets the next `skip`
// per-call device allocations of the evaluation paths succeed and makes the `count` after them
// fail as if the device were out of memory.
bool take_injected_alloc_failure();
inline cudaError_t dev_alloc_async(void **p, size_t bytes, cudaStream_t stream)
{
    if (take_injected_alloc_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMallocAsync(p, bytes, stream);
}
template <typename T>
inline cudaError_t dev_alloc_async(T **p, size_t bytes, cudaStream_t stream)
{
    return dev_alloc_async(reinterpret_cast<void **>(p), bytes, stream);
}
template <typename T>
inline cudaError_t dev_alloc_pool_async(T **p, size_t bytes, cudaMemPool_t pool, cudaStream_t stream)
{
    if (take_injected_alloc_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMallocFromPoolAsync(reinterpret_cast<void **>(p), bytes, pool, stream);
}

// Device status word bits (set with atomicOr by kernels that find a problem).
enum : uint32_t {
    ST_BAD_OFFSETS = 1u << 0,
    ST_BAD_CLASS = 1u << 1,
    ST_BAD_FEATURE = 1u << 2,
    ST_BAD_OP = 1u << 3,
    ST_BAD_LABEL = 1u << 4,
    ST_TOO_LARGE = 1u << 5,
    ST_WAIT_TIMEOUT = 1u << 8,
    ST_QUEUE_TIMEOUT = 1u << 9,
};
std::string status_text(uint32_t st);

// ------------------------------------------------------------------------------ records

// One condition packed for the evaluator (16 bytes, read as one 128-bit broadcast load).
// Threshold conditions are rewritten into a single compare of the raw feature value against an
// exact float32 cut (see pack.cu); '<' pair conditions are rewritten as '>' with the two sides
// swapped. Both rewrites are exact for every input including NaN, infinities and subnormals.
enum : uint32_t {
    KIND_GT = 0,     // x[f] > v0
    KIND_LT = 1,     // x[f] < v0
    KIND_PAIR = 2,   // fl(v0 * x[f]) > fl(v1 * x[g])
    KIND_MGT = 3,    // fl(v0 * x[f]) > v1  (coefficient 0 / inf: kept as the plain product)
    KIND_MLT = 4,    // fl(v0 * x[f]) < v1
    KIND_NEVER = 5,  // never true
    KIND_IN = 6,     // x[f] an integer category code k in 0..63 with bit k of (v1 bits : v0 bits)
};

// Record format v2 (rule-at-a-time evaluator): w0 = [0,18) feature row offset in 16-byte units |
// [18] pair | [19,31) rule length; w1 = [0,18) second feature row offset | [18,30) rule class;
// then v0, v1 with the test fl(v0*x[f]) > v1 (LIN) or fl(v0*x[f]) > fl(v1*x[g]) (pair).
constexpr uint32_t OFF_MASK = 0x3FFFFu;
constexpr uint32_t PAIR_BIT = 1u << 18;
constexpr int LEN_SHIFT = 19;
constexpr int CLS_SHIFT = 18;
// v4 only: a threshold condition that is not a +-1 cut (zero or infinite coefficient, never true)
constexpr uint32_t GENERAL_BIT = 1u << 31;

// Record format v5 (rank-coded evaluator): per rule its threshold cuts, its pair conditions and
// its remaining product conditions, one record per condition (same positions as the conditions).
// w0 = tag << 29 | end-of-rule << 28 | rule class << 16 (last record of a rule) | feature.
//   cut:     x[f] > w2 (R5_CUT_GT) or x[f] <= w2 (R5_CUT_LT: x[f] < c stored as w2 = nextdown(c))
//   pair:    fl(w2 * x[f]) > fl(w3 * x[w1])
//   product: fl(w2 * x[f]) > w3
//   set:     x[f] an integer category code k in 0..63 with bit k of the 64-bit set (w3 : w2)
enum : uint32_t { R5_NONE = 0, R5_CUT_GT = 2, R5_CUT_LT = 3, R5_PAIR = 4, R5_GEN = 5, R5_SET = 6 };
constexpr int R5_TAG_SHIFT = 29;
constexpr uint32_t R5_END_BIT = 1u << 28;
constexpr int R5_CLS_SHIFT = 16;
constexpr uint32_t R5_F_MASK = 0xFFFFu;

struct __align__(16) Rec {
    uint32_t meta;   // [0,3) kind | [3] last condition of its rule | [4,16) rule class | [16,32) skip
    uint16_t f, g;
    float v0, v1;
};
__host__ __device__ inline uint32_t rec_kind(uint32_t m) { return m & 7u; }
__host__ __device__ inline bool rec_last(uint32_t m) { return (m >> 3) & 1u; }
__host__ __device__ inline int rec_cls(uint32_t m) { return (int)((m >> 4) & 0xFFFu); }
__host__ __device__ inline int rec_skip(uint32_t m) { return (int)(m >> 16); }

// Per-set table written by the packer.
struct __align__(16) SetInfo {
    int32_t rec_begin, rec_end;  // records [rec_begin, rec_end) (truncated after an empty rule)
    int32_t deflt;               // effective default (the class of a leading empty rule, if any)
    int32_t cost;                // rec_end - rec_begin
};

// Device-side view of a batch (device pointers). When dR / dC are set, the rule and condition
// counts are read on the device (batches built on the device); R and C then hold capacities that
// size the packing grids.
struct BatchDev {
    int32_t P, R, C;
    const int32_t *dR = nullptr, *dC = nullptr;
    const int32_t *set_rule_off, *rule_cond_off, *rule_class, *set_default;
    const int32_t *cond_f, *cond_g;
    const int8_t *cond_op;
    const float *cond_a, *cond_b, *cond_t;
    const uint64_t *cond_set = nullptr;   // category sets (membership conditions), or null
};

// Membership of one value in a 64-bit category set: an integer code 0..63 whose bit is set
// (false for fractions, negatives, codes above 63, NaN and infinities).
__host__ __device__ __forceinline__ bool category_member(float x, uint32_t lo, uint32_t hi)
{
    if (!(x >= 0.f && x <= 63.f)) return false;
    const int k = (int)x;
    if ((float)k != x) return false;
    return ((k < 32 ? lo : hi) >> (k & 31)) & 1u;
}

// ------------------------------------------------------------------------------ datasets

struct Dataset {
    int64_t N = 0, n_pad = 0;
    int32_t F = 0, K = 0;
    bool finite = false;          // no NaN or infinity in X
    float *Xt = nullptr;          // [F][n_pad], samples grouped by label (stable), zero padded
    int32_t *y = nullptr;         // [n_pad] labels in that order, -1 for padding
    int32_t *perm = nullptr;      // [N] caller index of sorted position
    int32_t *inv = nullptr;       // [N] sorted position of caller index
    std::vector<int64_t> class_count;
    std::map<int, CUtensorMap> tmaps;   // keyed by samples per tile
    // Rank table (finite datasets with F <= RANK_MAX_F), per 128-sample tile and feature f:
    // Rk[f][n] = the position of x[f][n] in the tile's column f in ascending order, equal values in
    // sample order (0..127).
    uint8_t *Rk = nullptr;
    bool ranked = false;
    // Contexts with a dataset budget (rs_set_dataset_budget): the caller's data kept on the host
    // (row-major X, labels) so that the device copy can be evicted and rebuilt; whether the device
    // copy exists, its bytes, and the registry tick of its last use.
    std::vector<float> hX;
    std::vector<int32_t> hy;
    bool resident = true;
    size_t dev_bytes = 0;
    uint64_t last_use = 0;
    // Under a budget: an event recorded on each call's stream when the call returns (the call's
    // device work on the dataset is done once it completes), and whether some call's work could
    // not be marked so (a stream being captured, or no event to spare): evicting it then waits for
    // the device. Under the context's mu.
    std::vector<cudaEvent_t> inflight;
    bool unmarked_use = false;
    bool rmap_ok = false;
    CUtensorMap rmap;
    std::mutex mu;
};

// ------------------------------------------------------------------------------ tile configs

struct TileConfig {
    int id;
    int V;       // samples per lane
    int W;       // warps per CTA
    int ver;     // 1: condition-at-a-time evaluator, 2: rule-at-a-time (record v2),
                 // 3: rule-at-a-time with the margin-minimum conjunction,
                 // 4: sign-mask conjunction for finite datasets (falls back to 3 otherwise)
                 // 5: rank-coded cuts for ranked datasets (falls back to 4, then 3)
    bool gmem = false;   // form 1 reading features from global memory (no shared tile: any F)
    int S() const { return 32 * V; }
};
constexpr int RANK_TILE = 128;    // samples per rank tile (ranks fit in 7 bits)
constexpr int RANK_MAX_F = 160;   // widest dataset given rank tables
int tile_config_count();
const TileConfig &tile_config(int id);
// Largest F a configuration can stage (its x tile must fit in shared memory).
bool tile_config_fits(const TileConfig &tc, int F);

// ------------------------------------------------------------------------------ context

struct GraphEntry;

// Kernel launch counting and optional CUDA-event timing of the evaluator kernels.
enum TimedKind { TK_HARD = 0, TK_SOFT = 1 };
struct Profiler {
    std::atomic<int64_t> launches{0};
    std::mutex mu;
    struct Pending { cudaEvent_t e0, e1; int kind; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int64_t n[2] = {0, 0};
    double ms[2] = {0, 0};
};

struct Ctx {
    int device = 0;
    uint32_t flags = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    uint64_t budget = 0;
    std::string autotune_path;
    std::mutex mu;
    std::map<uint64_t, std::shared_ptr<Dataset>> datasets;
    uint64_t next_ds = 1;
    uint64_t ds_budget = 0;                  // device bytes of resident datasets (0: no limit)
    size_t ds_resident = 0;                  // device bytes of the resident datasets
    uint64_t ds_tick = 0;                    // dataset use counter (least recently used order)
    int64_t ds_evictions = 0, ds_rebuilds = 0;
    std::vector<cudaEvent_t> ds_events;      // spare events for the datasets' in-flight marks
    int forced_tile = -1;
    std::map<std::string, int> tune_table;   // key -> tile config id
    std::map<std::string, std::shared_ptr<GraphEntry>> graphs;
    uint32_t *d_sticky = nullptr;            // async-mode sticky device status
    unsigned char *static_scratch = nullptr; // device address of rs_eval_hard_static's fixed array
    unsigned long long *d_walked = nullptr;  // [4] walked-work counters (RS_CTX_COUNT_WORK contexts)
    Profiler prof;
    struct Server *server = nullptr;
};

std::shared_ptr<Dataset> find_dataset(Ctx *ctx, uint64_t ds);
// The dataset with its device copy present (rebuilt from the host copy if it was evicted, after
// evicting others to make room), marked as the most recently used; errors: RS_ERR_NOT_FOUND, or
// the rebuild's error.
rs_status use_dataset(Ctx *ctx, uint64_t ds, std::shared_ptr<Dataset> *out);
rs_status set_dataset_budget(Ctx *ctx, uint64_t bytes);
// Under a dataset budget: mark the device work a call enqueued on `stream` for dataset ds, so that
// an eviction waits for that work only (no-op without a budget). `may_create`: the call may create
// an event when none is spare (not the allocation-free entry).
void mark_dataset_use(Ctx *ctx, Dataset *ds, cudaStream_t stream, bool may_create = true);
// Records the mark when the call's scope ends (after its work is enqueued).
struct DatasetUseMark {
    Ctx *ctx;
    Dataset *ds;
    cudaStream_t stream;
    bool may_create = true;
    ~DatasetUseMark() { if (ds) mark_dataset_use(ctx, ds, stream, may_create); }
};
// Free the context's spare events and every dataset's marks (context teardown).
void release_dataset_events(Ctx *ctx);

// Count `n` kernel launches of the library.
inline void count_launch(Ctx *ctx, int n = 1) { ctx->prof.launches += n; }
// Begin / end a timed region around one kernel launch on `stream` (no-ops unless RS_CTX_PROFILE).
struct TimedLaunch {
    Ctx *ctx;
    int kind;
    cudaStream_t stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TimedLaunch(Ctx *c, int k, cudaStream_t s);
    ~TimedLaunch();
};
rs_status device_guard(Ctx *ctx);

// Pinned per-thread status slot used by synchronous calls to read back the device status word.
uint32_t *host_status_slot();

// ------------------------------------------------------------------------------ kernels / launchers

// Sets of at most LAST_END_MAX_K classes also get, per class k, the end (relative to the set's
// first record) after which no record can change the count of a tile whose samples all have label
// k: for a class other than the set's default, the end of its last rule of class k (later rules
// only take samples of that tile away from a correct prediction or leave them to the default);
// for the default class, the end of its last rule of any other class (every rule after it names
// the default class, so every sample still unclaimed there is predicted correctly).
constexpr int LAST_END_MAX_K = 64;

struct PackOut {
    Rec *recs = nullptr;          // [C]
    SetInfo *sets = nullptr;      // [P]
    int32_t *order = nullptr;     // [P] set ids, most expensive first
    uint32_t *status = nullptr;   // device status word
    int32_t *last_end = nullptr;  // [P*K] or null
    int32_t *correct = nullptr;   // [P] zeroed by the packing when given
    int32_t *per_class = nullptr; // [P*K] zeroed by the packing when given
};

// Validate + pack (+ order) a device batch, zeroing the count outputs named in `o`. Enqueued on
// `stream`.
// Returns the number of kernels launched.
int launch_pack(const BatchDev &b, int F, int K, int S, int ver, const PackOut &o, cudaStream_t stream);

// Per-call scratch of a hard evaluation.
struct Scratch {
    Rec *recs = nullptr;
    SetInfo *sets = nullptr;
    int32_t *order = nullptr;
    uint32_t *status = nullptr;
    int32_t *out_dev = nullptr;   // device outputs when the caller's are host memory
    int32_t *last_end = nullptr;  // [P*K] (K <= LAST_END_MAX_K) or null
};

struct HardArgs {
    const Rec *recs;
    const SetInfo *sets;
    const int32_t *order;
    int32_t P;
    const int32_t *y;        // sorted labels [n_pad], -1 padding
    const int32_t *perm;     // [N]
    int64_t N, n_pad;
    int32_t F, K;
    int32_t *correct;        // [P]  (zeroed by the launcher)
    int32_t *per_class;      // [P*K] or null
    int32_t *preds;          // [P*N] or null
    int32_t groups;          // set groups (grid.y)
    uint32_t *status;
    const int32_t *last_end; // [P*K] or null (see PackOut)
    const float *Xt;         // [F][n_pad] (read directly by the global-memory configuration)
    bool cat;                // the records may hold membership tests
    unsigned long long *walked;  // [4] or null: records, rows, rule ends, (set, tile) walks summed
                                 // over the rank-coded evaluator's walks (work-counting contexts)
};
// Zero outputs and run the evaluator with tile configuration `tc`.
rs_status launch_hard(Ctx *ctx, Dataset *ds, const TileConfig &tc, const HardArgs &a,
                      cudaStream_t stream);
int choose_groups(Ctx *ctx, const Dataset *ds, const TileConfig &tc, int P);
rs_status launch_hard2(Ctx *ctx, Dataset *ds, int V, int W, bool mm, const HardArgs &a,
                       cudaStream_t stream);
rs_status launch_hard4(Ctx *ctx, Dataset *ds, int V, int W, const HardArgs &a, cudaStream_t stream);
rs_status launch_hard5(Ctx *ctx, Dataset *ds, int W, const HardArgs &a, cudaStream_t stream);
// Shared memory of the v5 evaluator for F features and W warps.
size_t hard5_smem_bytes(int F, int W);
// The evaluator version a configuration runs as for this dataset and output choice.
int effective_version(const TileConfig &tc, const Dataset &ds, bool preds);
const TileConfig &categorical_config(const TileConfig &tc, const Dataset &ds, bool preds);
// Enqueue packing + evaluation of a device batch with the given scratch.
rs_status enqueue_hard(Ctx *ctx, Dataset *ds, const TileConfig &tc, const BatchDev &bd,
                       const Scratch &s, int32_t *correct, int32_t *per_class, int32_t *preds,
                       cudaStream_t stream);
// The built-in tile choice for a dataset (no autotuned entry).
int heuristic_tile_for(const Dataset &ds);
const CUtensorMap *dataset_tmap(Dataset *ds, int S);
const CUtensorMap *dataset_rank_tmap(Dataset *ds);

struct SoftArgs {
    BatchDev b;
    const float *Xt;
    const int32_t *y;
    const int32_t *perm;
    int64_t N, n_pad;
    int32_t F, K;
    float tau;
    float *loss;        // [P]
    float *probs;       // [P*N*K] or null
    const float *dloss; // [P] or null (forward only)
    float *grad_a, *grad_b, *grad_t;
    uint32_t *status;
};
// Validate (one host readback of the batch's largest set) and run.
rs_status launch_soft(Ctx *ctx, const SoftArgs &a, cudaStream_t stream);
// Run with known bounds on rules and conditions per set, no host synchronisation; the kernels
// skip all work if the status word is non-zero.
rs_status soft_step_known(Ctx *ctx, const SoftArgs &a, int maxR, int maxC, cudaStream_t stream);
// Hard evaluation of a device-built batch whose R and C are known only on the device.
rs_status enqueue_hard_dev_sizes(Ctx *ctx, Dataset *ds, const TileConfig &tc, BatchDev bd,
                                 const int32_t *dR, const int32_t *dC, const Scratch &s,
                                 int32_t *correct, int32_t *per_class, int32_t *preds,
                                 cudaStream_t stream);

}  // namespace rs

struct rs_ctx : public rs::Ctx {};
