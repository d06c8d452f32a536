/*
 * rs.h -- C ABI of the GB300 (sm_103a) rule-set evaluation library (librs.so).
 *
 * The library evaluates whole populations of ordered rule sets against a tabular dataset, the
 * evaluation step of accelerated evolutionary rule-based learning (Shahrzad & Miikkulainen,
 * "GPU-Accelerated Rule Evaluation and Evolution", GECCO'25 Companion; Sec. 3 and Fig. 1).
 *
 *   condition  a*x[f] op t           (threshold)       Sec. 3 / Fig. 1a rows with one weight
 *              a*x[f] op b*x[g]      (feature pair)    Sec. 3 / Fig. 1a row [0, 1.0, -0.38, ...]
 *              op is '>' or '<'; each product is one correctly rounded float32 multiply and the
 *              compare is strict and IEEE-ordered (NaN compares false, a zero margin is false:
 *              the hard activation of Sec. 3 maps negative margins to false, positive to true).
 *   rule       conjunction of its conditions naming one class (Fig. 1b "&" and "->"); an empty
 *              rule fires.
 *   rule set   ordered list of rules (Sec. 1, list-based grammar): the first rule that fires gives
 *              the class, otherwise the set's default class.
 *   fitness    classification accuracy (Sec. 1), returned as exact int32 correct counts.
 *   soft path  sigmoid relaxation for back-propagation fine-tuning of coefficients and thresholds
 *              with the rule structure kept (Sec. 3, Fig. 1c).
 *
 * Conventions
 *   - Every function returns rs_status (0 = RS_OK, < 0 = error). No exception crosses the ABI.
 *     rs_last_error() returns a thread-local message for the last failing call of the thread.
 *   - Pointers are plain host or device addresses as stated per argument. The caller owns every
 *     buffer; synchronous calls borrow them until the call returns (default contexts) or until
 *     the work enqueued on `stream` completes (RS_CTX_ASYNC contexts).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - A context is bound to one CUDA device; calls on one context are thread-safe.
 *   - The library never reads memory outside the sizes given; malformed batches are rejected
 *     with RS_ERR_INVALID before any count is produced.
 */
#ifndef RS_H
#define RS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rs_status;

#define RS_OK               0
#define RS_PENDING          1    /* rs_poll: the request has not finished yet */
#define RS_ERR_INVALID     -1    /* bad argument, index, class or offset array */
#define RS_ERR_TOO_LARGE   -2    /* a request larger than the whole memory budget or a limit */
#define RS_ERR_OOM         -3    /* device allocation failed */
#define RS_ERR_TIMEOUT     -4    /* a bounded device or host wait gave up */
#define RS_ERR_DEVICE      -5    /* a CUDA error; sticky for the context */
#define RS_ERR_UNSUPPORTED -6    /* device is not sm_103 / feature not available */
#define RS_ERR_NOT_FOUND   -7    /* unknown dataset handle or ticket */
#define RS_ERR_CANCELLED   -8    /* request cancelled before it ran */

/* Limits enforced by the library. */
#define RS_MAX_FEATURES  4096
#define RS_MAX_CLASSES   4096

typedef struct rs_ctx rs_ctx;

#define RS_CTX_ASYNC        1u   /* eval calls return after enqueue; device-side errors are
                                    reported by rs_check (sticky until read) */
#define RS_CTX_NO_GRAPH     2u   /* launch kernels directly instead of replaying captured graphs */
#define RS_CTX_NO_AUTOTUNE  4u   /* use the built-in tile heuristic, never time candidates */
#define RS_CTX_PROFILE      8u   /* bracket the evaluator kernels with CUDA events (read with
                                    rs_profile_read); implies RS_CTX_NO_GRAPH */
#define RS_CTX_COUNT_WORK  16u   /* the rank-coded hard evaluator counts the work it does
                                    (rs_profile_read: records, rows and rule ends walked) */

typedef struct {
    int32_t device;              /* CUDA device ordinal */
    uint32_t flags;              /* RS_CTX_* */
    uint64_t mem_budget_bytes;   /* serving admission budget; 0 = 40 GiB */
    const char *autotune_cache;  /* JSON file the autotuner reads at create and writes on update;
                                    NULL = in-memory only */
} rs_config;

/* Create a context on cfg->device (cfg may be NULL: device 0, default flags). */
rs_status rs_create(const rs_config *cfg, rs_ctx **out);
/* Destroy a context: waits for its serving work, frees every dataset and cached graph. */
rs_status rs_destroy(rs_ctx *ctx);
/* Thread-local description of the last error of the calling thread ("" if none). */
const char *rs_last_error(void);
/* Library version string. */
const char *rs_version(void);
/* Synchronize `stream` and return (and clear) the first device-side error recorded by calls of
 * an RS_CTX_ASYNC context; RS_OK if none. */
rs_status rs_check(rs_ctx *ctx, void *stream);

/* ------------------------------------------------------------------------------ datasets */

#define RS_MEM_HOST   0          /* arrays are host memory (pageable or pinned) */
#define RS_MEM_DEVICE 1          /* arrays are device memory of the context's device */

/*
 * Register a dataset (Sec. 3: the candidates are evaluated on the GPU against data loaded there;
 * here the data stays resident while any number of populations is evaluated against it).
 *   X      float32, row-major N x F (sample n, feature f at X[n*F + f]); host or device per `mem`
 *   y      int32[N], labels in 0..K-1
 *   N >= 1, 1 <= F <= RS_MAX_FEATURES, 1 <= K <= RS_MAX_CLASSES
 * The library keeps its own copy (feature-major, samples grouped by label); the caller may free X
 * and y when the call returns. Device memory held: 4 bytes per value and 12 per sample (labels,
 * order), N rounded up to 256, plus for finite data with F <= 160 one byte per value (the rank of
 * each value within its 128-sample tile, for the rank-coded evaluator).
 * Errors: RS_ERR_INVALID (sizes, a label out of range), RS_ERR_OOM.
 * On success *ds_out receives a non-zero handle.
 */
rs_status rs_dataset_create(rs_ctx *ctx, const float *X, const int32_t *y, int64_t N, int32_t F,
                            int32_t K, int32_t mem, void *stream, uint64_t *ds_out);
/*
 * Unregister a dataset and free its device copy (and its host copy under a dataset budget). The
 * device's queued work completes first, so no call enqueued earlier on any stream still reads it.
 * Errors: RS_ERR_NOT_FOUND (unknown handle); RS_ERR_INVALID while the dataset is in use: a call on
 * it is running in another thread, or a serving request on it has not been polled yet (queued,
 * running, completed or cancelled: poll it first). The handle stays valid after an error.
 */
rs_status rs_dataset_destroy(rs_ctx *ctx, uint64_t ds);
/* Shape of a dataset; class_count (host, int64[K]) may be NULL. */
rs_status rs_dataset_info(rs_ctx *ctx, uint64_t ds, int64_t *N, int32_t *F, int32_t *K,
                          int64_t *class_count);

/*
 * Device-memory budget of the context's registered datasets, for a server that keeps the datasets
 * of many clients resident (no counterpart in the paper): 0 (the default) means no limit. With a
 * budget, rs_dataset_create also keeps a host copy of X and y, and whenever registering or using a
 * dataset would take the resident datasets beyond `bytes`, the least recently used datasets that
 * nothing is using (no call running on them, no serving request queued or running on them, not
 * yet polled) are evicted: their device copies are freed, and the next call that names one
 * rebuilds it from its host copy (the registration's work again). Datasets registered before a
 * budget was set have no host copy and stay resident. If too little can be evicted the budget is
 * exceeded rather than a call refused. Each call marks the device work it enqueued on a dataset
 * (an event on its stream); a dataset whose marked work is still pending (calls of asynchronous
 * contexts) is not chosen, and only work no mark covers (calls on a stream being captured) makes
 * an eviction wait for the whole device. rs_eval_hard_static, which allocates nothing, returns
 * RS_ERR_INVALID on an evicted dataset. Lowering the budget evicts at once.
 */
rs_status rs_set_dataset_budget(rs_ctx *ctx, uint64_t bytes);

typedef struct {
    int64_t datasets;          /* registered */
    int64_t resident;          /* with their device copy present */
    uint64_t resident_bytes;   /* device bytes of those */
    int64_t evictions;         /* device copies freed under the budget so far */
    int64_t rebuilds;          /* evicted datasets made resident again so far */
} rs_dataset_stats;
rs_status rs_dataset_stats_read(rs_ctx *ctx, rs_dataset_stats *out);

/* --------------------------------------------------------------------------- rule sets */

/*
 * A population of P ordered rule sets in CSR form (Sec. 3 / Fig. 1a, one record per condition
 * instead of a dense row). All arrays live in host or device memory according to `mem`.
 *   set_rule_off  int32[P+1]  rules of set p: [set_rule_off[p], set_rule_off[p+1]); [0]=0, [P]=R
 *   rule_cond_off int32[R+1]  conditions of rule r: [rule_cond_off[r], rule_cond_off[r+1]);
 *                             [0]=0, [R]=C; non-decreasing
 *   rule_class    int32[R]    class named by rule r, 0..K-1
 *   set_default   int32[P]    class of set p when no rule fires, 0..K-1
 *   cond_f        int32[C]    feature of the left-hand product, 0..F-1
 *   cond_g        int32[C]    -1: threshold condition a*x[f] op t; else 0..F-1: a*x[f] op b*x[g]
 *   cond_op       int8[C]     RS_OP_GT '>', RS_OP_LT '<', RS_OP_IN category membership
 *   cond_a, cond_b, cond_t  float32[C]   (b unused for thresholds, t unused for pairs; all
 *                             three unused by membership conditions)
 *   cond_set      uint64[C]   category set of each RS_OP_IN condition (bit k: code k), read only
 *                             for those; NULL when no condition has op RS_OP_IN
 * A membership condition (categorical features, the future work of Sec. 5) has cond_g = -1 and is
 * true iff x[f] is an integer category code k, 0 <= k <= 63, whose bit is set in cond_set[c]
 * (fractions, negatives, codes above 63, NaN and infinities are in no set). The soft path keeps it
 * as its exact 0/1 indicator (no gradient). Evolution (rs_evolve) works on inequalities only.
 * P >= 0, R >= 0, C >= 0; P, R, C < 2^31 - 1; a rule has at most 4095 conditions.
 */
#define RS_OP_GT 0
#define RS_OP_LT 1
#define RS_OP_IN 2

typedef struct {
    int32_t P, R, C;
    int32_t mem;
    const int32_t *set_rule_off;
    const int32_t *rule_cond_off;
    const int32_t *rule_class;
    const int32_t *set_default;
    const int32_t *cond_f;
    const int32_t *cond_g;
    const int8_t *cond_op;
    const float *cond_a;
    const float *cond_b;
    const float *cond_t;
    const uint64_t *cond_set;
} rs_batch;

/* ------------------------------------------------------------------------ hard evaluation */

/*
 * Exact first-fire evaluation of every set of `batch` on every sample of dataset `ds`
 * (Sec. 3 inequalities + hard activation, Fig. 1b conjunction and rule order, Sec. 1 fitness).
 *   correct    int32[P]     #{n : pred_p(n) = y_n}
 *   per_class  int32[P*K]   #{n : pred_p(n) = y_n = k} at [p*K + k]; may be NULL
 *   preds      int32[P*N]   pred_p(n) at [p*N + n] in the caller's sample order; may be NULL
 * Outputs live in the memory space given by batch->mem (host buffers: the library copies).
 * Results are bit-identical to the plain definition (no FMA, no flush-to-zero).
 * Launch: on a stream the caller created, packing and evaluation run as one CUDA graph cached per
 * (dataset, tile configuration, stream, output kinds). A call whose sizes and device pointers
 * repeat the previous call's on that stream is captured, and later calls with them launch the
 * graph as it is, reading the arrays' current contents; a shape seen for the first time runs
 * directly. Staging and scratch memory of the graph belong to it and are kept until the dataset
 * or the context is destroyed. On the legacy default stream (NULL), on a stream the caller is
 * capturing, and in RS_CTX_NO_GRAPH / RS_CTX_PROFILE contexts the kernels are enqueued directly
 * with per-call scratch from the stream-ordered pool. Calls from several host threads are safe,
 * on one stream or on several.
 * Errors: RS_ERR_INVALID (malformed batch: nothing is counted, outputs undefined),
 *         RS_ERR_TOO_LARGE (a rule of more than 4095 conditions; outputs undefined),
 *         RS_ERR_NOT_FOUND (ds), RS_ERR_OOM, RS_ERR_DEVICE.
 */
rs_status rs_eval_hard(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t *correct,
                       int32_t *per_class, int32_t *preds, void *stream);

/* ------------------------------------------------------------------------- soft evaluation */

/*
 * Sigmoid-relaxed forward (Sec. 3: a sigmoid replaces the hard activation to make evaluation
 * differentiable).
 * Per condition u = s*(a*x[f] - rhs)/tau with s = +1 for '>' and -1 for '<', rhs = t or b*x[g];
 * rule firing probability q_r = prod_c sigmoid(u_c); rule r decides with probability
 * q_r * prod_{j<r} (1 - q_j); the default class takes prod_j (1 - q_j);
 *   loss[p] = (1/N) sum_n -log p_p(y_n | x_n)      float32[P]
 *   probs   float32[P*N*K] class probabilities at [(p*N + n)*K + k] (caller's sample order);
 *           may be NULL
 * Computed in float32 in the log domain. tau > 0.
 */
rs_status rs_eval_soft_fwd(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float tau,
                           float *loss, float *probs, void *stream);

/*
 * Adjoint of rs_eval_soft_fwd (Sec. 3 back-propagation; Fig. 1c shows coefficients and thresholds
 * moving). Given dloss float32[P] (dObjective/dloss[p]) it writes, for every condition c,
 *   grad_a[c] = sum_p dloss[p] * dloss[p]/da_c,  grad_b[c] (pairs; 0 for thresholds),
 *   grad_t[c] (thresholds; 0 for pairs)          float32[C] each
 * and, if loss != NULL, the forward loss float32[P]. The forward is recomputed in the same pass.
 * Reductions over samples use a fixed order: repeated calls give bit-identical results.
 */
rs_status rs_eval_soft_bwd(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float tau,
                           const float *dloss, float *grad_a, float *grad_b, float *grad_t,
                           float *loss, void *stream);

/*
 * rs_eval_hard without any device allocation. The paper has no counterpart: this entry point
 * exists for callers that must not call cudaMalloc or any allocating routine while they evaluate
 * -- a host whose device memory is owned by another allocator or is fully reserved in advance, or
 * a real-time loop that may not block in an allocator. It computes exactly what rs_eval_hard
 * computes, with the per-call scratch taken from one fixed array of RS_STATIC_SCRATCH_BYTES that
 * lives in the library's device image (every GPU that loads the library holds it until exit).
 *   batch   device arrays only (batch->mem must be RS_MEM_DEVICE)
 *   outputs correct, per_class, preds: device memory of the context's device (or managed memory);
 *           anything else is RS_ERR_INVALID with a message and nothing is launched
 *   limit   16*C + 20*P + 768 bytes, plus 4*P*K when the dataset has K <= 64 classes (each part
 *           rounded up to 256 B), must fit in the array, otherwise RS_ERR_TOO_LARGE with a
 *           message; nothing is launched then
 *   set-up  rs_create looks up the array's device address (cudaGetSymbolAddress, with the
 *           context's device current) and keeps it in the context; the first call for a dataset
 *           builds its tile descriptor on the host, so make that first call before any stream
 *           capture
 *   sharing every call uses the same array: calls whose GPU work overlaps (different streams,
 *           host threads or contexts on one device) race on it and must be serialised by the
 *           caller. Each call clears the status word it needs; the rest is rewritten before use.
 * The dataset itself is registered beforehand with rs_dataset_create. Like rs_eval_hard, the call
 * stops a tile of one label k where no later record can change its count (K <= 64): after the
 * set's last rule of class k, or, when the set defaults to k, after its last rule of another class.
 */
#define RS_STATIC_SCRATCH_BYTES (8u << 20)
rs_status rs_eval_hard_static(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t *correct,
                              int32_t *per_class, int32_t *preds, void *stream);

/* ------------------------------------------------------------------------------- serving */

#define RS_KIND_HARD 0
#define RS_KIND_SOFT 1

/*
 * Continuous batching of fitness-evaluation requests (hard evaluation). rs_submit copies the batch
 * (host or device arrays per batch->mem) into pinned staging -- the caller may free it on return --
 * and queues the request. Requests are admitted in arrival order while the context's memory budget
 * (rs_config.mem_budget_bytes) and the request slots allow; admitted requests share one persistent
 * kernel: a 128-sample tile of a request's dataset times a group of its sets is a work unit, and
 * CTAs claim units from the request with the fewest unclaimed units (the oldest among equals), so
 * units of requests admitted while others run interleave with theirs on the device. Results equal
 * rs_eval_hard's exactly.
 *   kind    RS_KIND_HARD (soft requests carry a temperature: rs_submit_soft)
 *   errors  RS_ERR_TOO_LARGE if the request alone exceeds the budget; RS_ERR_UNSUPPORTED for
 *           datasets with more than 256 features, and for batches with category sets (membership
 *           tests) unless the dataset is finite with at most 128 features; RS_ERR_NOT_FOUND (ds)
 * Request memory comes from a pool of the scheduler's own that keeps what it has mapped, up to the
 * budget, until the context is destroyed.
 * Thread-safe. *ticket receives a non-zero id.
 */
rs_status rs_submit(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t kind, uint64_t *ticket);

typedef struct {
    int64_t submit_ns, admit_ns, done_ns;   /* host steady-clock times of the request */
} rs_ticket_info;

/*
 * Wait up to timeout_us (0 = do not wait) for a request. Returns RS_PENDING while it runs; on
 * completion writes correct (host int32[P]) and per_class (host int32[P*K], may be NULL) and the
 * request's times (info, may be NULL), releases the ticket and returns its status (RS_OK,
 * RS_ERR_INVALID for a malformed batch, RS_ERR_CANCELLED).
 */
rs_status rs_poll(rs_ctx *ctx, uint64_t ticket, int64_t timeout_us, int32_t *correct,
                  int32_t *per_class, rs_ticket_info *info);
/*
 * Soft-loss requests (Sec. 3 sigmoid relaxation, the forward of rs_eval_soft_fwd at temperature
 * tau > 0): queued, admitted under the same budget and run as their own kernels next to the
 * persistent kernel. rs_poll_soft writes loss (host float[P], may be NULL) and the times, releases
 * the ticket and returns its status (RS_ERR_INVALID for a malformed batch or a hard ticket).
 * Losses equal rs_eval_soft_fwd's bit for bit.
 */
rs_status rs_submit_soft(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float tau, uint64_t *ticket);
rs_status rs_poll_soft(rs_ctx *ctx, uint64_t ticket, int64_t timeout_us, float *loss, rs_ticket_info *info);
/* Cancel a request that has not been admitted yet (RS_ERR_INVALID once it runs). */
rs_status rs_cancel(rs_ctx *ctx, uint64_t ticket);

typedef struct {
    int64_t queued, active;          /* requests waiting for admission / admitted */
    uint64_t device_bytes_in_use;    /* charged against the budget */
    uint64_t units_published;        /* work units published since start */
    int64_t kernel_launches;         /* persistent-kernel launches since start */
} rs_serving_stats;
rs_status rs_serving_stats_read(rs_ctx *ctx, rs_serving_stats *out);

/* ------------------------------------------------------------------------------ evolution */

/*
 * A population in fixed slots (host arrays): set p has nrule[p] rules; rule r of set p sits at
 * [p*RMAX + r] and has ncond[...] conditions; condition k of that rule at [(p*RMAX + r)*CMAX + k]
 * (cond_g = -1 marks a threshold). Slots past nrule / ncond are carried along and never read.
 */
typedef struct {
    int32_t *nrule;    /* [P] 1..RMAX */
    int32_t *deflt;    /* [P] default class */
    int32_t *rcls;     /* [P*RMAX] */
    int32_t *ncond;    /* [P*RMAX] 1..CMAX */
    int32_t *cf, *cg;  /* [P*RMAX*CMAX] */
    int8_t *cop;
    float *ca, *cb, *ct;
    int32_t *fitness;  /* [P] out: correct counts of the returned population; may be NULL */
} rs_population;

typedef struct {
    int32_t P, RMAX, CMAX;    /* population shape; RMAX <= 32, CMAX <= 64 */
    int32_t generations;
    int32_t elite;            /* best individuals copied unchanged each generation */
    int32_t tune_every;       /* fine-tune every this many generations (0 = never) */
    int32_t tune_top;         /* the best tune_top sets are fine-tuned */
    int32_t tune_steps;       /* full-batch Adam steps per fine-tuning (lr, 0.9, 0.999, 1e-8) */
    float tau, lr;            /* sigmoid temperature, Adam learning rate */
    int32_t lamarckian;       /* 0: the tuned fitness (the better of before / after tuning)
                                 ranks the individual, its genome is kept (Baldwin effect, Sec. 3);
                                 1: tuned coefficients that improved it are written back */
    uint64_t seed;
    int32_t first_generation; /* index of the first generation of this call (0 for a new run): a
                                 run resumed from a saved population with the same seed and
                                 first_generation = generations done so far continues exactly as
                                 an uninterrupted run (random counters and the tuning schedule
                                 use the absolute index) */
} rs_evolve_config;

/*
 * Run `generations` generations of evolution on the device (Sec. 3: tournament selection,
 * offspring with randomized coefficients, back-propagation fine-tuning guiding evolution through
 * the Baldwin effect). Each generation: evaluate every set exactly (rs_eval_hard semantics), rank
 * by (correct desc, index asc), copy the `elite` best, fill the rest with children of two binary
 * tournaments (uniform rule-list crossover with probability 1/2, one mutation with probability
 * 9/10: new random coefficients, new feature, flipped comparison, add/delete a condition,
 * add/delete a rule, new class). Random numbers: Philox4x64-10, counter (i/4, child, generation,
 * 0), key (seed, 0x65766f6c).
 * `pop` holds the initial population on entry and the final one (after `generations` steps) on
 * return. best / mean (host, may be NULL): best and mean correct count of each evaluated
 * generation, generations + 1 entries.
 * Launch: a generation is captured once as a CUDA graph per (parity of the generation, fine-tuning
 * or not) and replayed (RS_CTX_NO_GRAPH / RS_CTX_PROFILE: launched kernel by kernel, with the same
 * results). Device memory for the run is allocated at entry and released at return.
 * Errors: RS_ERR_INVALID for a bad configuration, a NULL population array or a set whose rule
 * count is outside 0..RMAX or a live rule's condition count outside 0..CMAX (checked on the host
 * before anything runs); features, classes and operators out of range are reported by the
 * device validation at the end of the run.
 */
rs_status rs_evolve(rs_ctx *ctx, uint64_t ds, const rs_evolve_config *cfg, rs_population *pop,
                    int32_t *best, double *mean, void *stream);

/*
 * Full-batch fine-tuning of one population's coefficients and thresholds (Sec. 3 back-propagation;
 * Fig. 1c): `steps` Adam steps (lr, beta 0.9 / 0.999, eps 1e-8) on the summed soft loss of all sets,
 * gradients from rs_eval_soft_bwd. The structure comes from `batch` (device arrays; its cond_a,
 * cond_b, cond_t are not read); the parameters a, b, t (device float32[C]) are updated in place
 * (b only for pairs, t only for thresholds). loss_trace (host float32[steps*P], may be NULL)
 * receives the per-set loss before each step. The batch is validated once, before the first step
 * (RS_ERR_INVALID / RS_ERR_TOO_LARGE as rs_eval_soft_fwd gives them, nothing updated); the steps
 * then run without waiting for the host, which reads the trace and the status at the end.
 */
rs_status rs_finetune(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float *a, float *b, float *t,
                      float tau, float lr, int32_t steps, float *loss_trace, void *stream);

/* ---------------------------------------------------------------------------- tile tuning */

/* Number of compiled tile configurations of the hard evaluator. */
int32_t rs_tile_config_count(void);
/* Describe configuration `id`: samples per CTA tile, warps per CTA, samples per lane. */
rs_status rs_tile_config_info(int32_t id, int32_t *samples_per_tile, int32_t *warps,
                              int32_t *samples_per_lane);
/* Evaluator form of configuration `id`: 1 condition at a time; 2 rule at a time; 3 rule at a
 * time with the margin minimum; 4 sign-mask conjunction (finite datasets, else runs as 3);
 * 5 rank-coded cuts (datasets with rank tables: finite and at most 160 features; else runs as
 * 4, then 3). Forms 4 and 5 produce counts only: a call that asks for predictions runs as 3.
 * The other configurations stage a feature tile in shared memory and need F small enough for
 * it; configuration 23 (form 1) reads the features from global memory and takes any F. */
rs_status rs_tile_config_form(int32_t id, int32_t *form);
/* Force configuration `id` for every following hard evaluation of the context, those of
 * rs_evolve included (-1 = automatic: autotuned table, else heuristic; rs_evolve then takes the
 * heuristic). */
rs_status rs_set_tile_config(rs_ctx *ctx, int32_t id);
/* The configuration the next rs_eval_hard of `batch` on `ds` would use: the forced one
 * (rs_set_tile_config), else the tuned one for the batch's shape key (feature count, class count,
 * mean conditions per rule, log2 N, membership tests), else the built-in heuristic. */
rs_status rs_tile_config_pick(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t *id);
/* Time every configuration on this dataset and batch (device pointers), record the fastest in the
 * context's table (and its JSON cache file) and return its id in *best. The cache file is read at
 * rs_create; a file that does not parse as a whole, or that names a configuration this library
 * does not have, is ignored (the heuristic applies until the tuner writes it again). */
rs_status rs_autotune(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, void *stream,
                      int32_t *best);

/* ------------------------------------------------------------------------------- profile */

typedef struct {
    int64_t launches;        /* kernels the library launched since the last reset */
    int64_t hard_launches;   /* evaluator (hard) kernel launches timed */
    double hard_ms;          /* their summed CUDA-event durations (RS_CTX_PROFILE contexts) */
    int64_t soft_launches;   /* soft forward/adjoint kernel launches timed */
    double soft_ms;
    /* Work the rank-coded hard evaluator actually did (RS_CTX_COUNT_WORK contexts), summed over its
     * walks of one rule set over one 128-sample tile: records (conditions) walked before the
     * all-claimed exit or the class-tail stop, pair / product / membership rows among them, rule
     * ends among them, and the number of (set, tile) walks. */
    int64_t hard_records_walked;
    int64_t hard_rows_walked;
    int64_t hard_rule_ends_walked;
    int64_t hard_set_tiles;
} rs_profile;

/* Read the counters of `ctx` (waits for the timed launches to finish); reset them if `reset`. */
rs_status rs_profile_read(rs_ctx *ctx, rs_profile *out, int32_t reset);

/*
 * Measured issue rates of the context's GPU, in lane operations per second, for the kernels'
 * rooflines (no paper counterpart; a measurement helper): a stream of independent FP32 fused
 * multiply-adds, FP32 multiplies, three-input logic operations, population counts, base-2
 * exponentials of the special-function unit, and float compares writing a register, each over
 * 2048 threads per SM. Takes a few milliseconds; allocates and frees a small device buffer.
 */
typedef struct {
    double ffma, fmul, lop3, popc, ex2, fset;
} rs_pipe_rates;
rs_status rs_measure_pipe_rates(rs_ctx *ctx, rs_pipe_rates *out);

/* ---------------------------------------------------------------------------- test hooks */

/*
 * Self-check of the exact threshold rewrite used by the hard evaluator: for each (a[i], t[i],
 * op[i]) (host arrays, n entries) and every one of the 2^32 float32 bit patterns x, compare
 * fl(a*x) op t against the rewritten single compare. *mismatches (host) receives the total count.
 */
rs_status rs_selftest_threshold_rewrite(rs_ctx *ctx, const float *a, const float *t,
                                        const int8_t *op, int32_t n, uint64_t *mismatches);

/*
 * Self-check of the soft path's log(1 + e) for 0 <= e <= 1 (the term of every log-sigmoid and
 * log-sum-exp of Sec. 3's sigmoid relaxation): out[i] = the kernels' log1p(e[i]) for host arrays
 * e, out of n entries, evaluated on the context's device.
 */
rs_status rs_selftest_log1p_unit(rs_ctx *ctx, const float *e, int32_t n, float *out);

/*
 * Self-check of the soft forward's log(1 - q) from log q (the log-probability that a rule does not
 * fire, Sec. 3's soft first-fire product): out[i] = the kernels' log(1 - e^s[i]) for host arrays s
 * (s <= 0; 0 gives -inf, -inf gives 0), n entries, evaluated on the context's device.
 */
rs_status rs_selftest_log1m_exp(rs_ctx *ctx, const float *s, int32_t n, float *out);

/*
 * Fault injection on the host: of the per-call device allocations of the evaluation paths
 * (rs_eval_hard, rs_eval_soft_fwd/bwd, serving admission), the next `skip` succeed and the `count`
 * after them fail as if the device were out of memory (process-wide; count 0 disarms). A call
 * whose allocation fails returns RS_ERR_OOM having released whatever it had taken; serving keeps
 * the request queued and admits it once allocations succeed again.
 */
rs_status rs_inject_alloc_failures(int32_t skip, int32_t count);

/*
 * Bounded device wait: runs the bounded mbarrier wait that guards every asynchronous copy of the
 * evaluators on a barrier that nothing completes, with a limit of limit_ns (clamped to 1 ms ..
 * 2 s). The wait gives up, the kernel records a timeout in its status word and returns, and the
 * call returns RS_ERR_TIMEOUT; the context stays usable.
 */
rs_status rs_selftest_bounded_wait(rs_ctx *ctx, int64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RS_H */
