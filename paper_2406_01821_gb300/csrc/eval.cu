// Orchestration of one evaluation call: argument checks, host staging, scratch, packing, tile
// configuration choice (autotuned table or heuristic), optional CUDA-graph replay, status check.
#include <algorithm>
#include <cctype>
#include <chrono>
#include <cmath>
#include <fstream>
#include <sstream>

#include "rs_internal.cuh"
#include "graph_util.cuh"

namespace rs {

rs_status selftest_rewrite(const float *a_h, const float *t_h, const int8_t *op_h, int n,
                           uint64_t *mismatches, int sm_count);

// ------------------------------------------------------------------------ batch checks / staging

static rs_status check_batch(const rs_batch *b)
{
    if (!b) { set_error("batch is NULL"); return RS_ERR_INVALID; }
    if (b->P < 0 || b->R < 0 || b->C < 0 || b->P == INT32_MAX || b->R == INT32_MAX || b->C == INT32_MAX) {
        set_error("negative batch sizes (P=%d R=%d C=%d)", b->P, b->R, b->C);
        return RS_ERR_INVALID;
    }
    if (b->mem != RS_MEM_HOST && b->mem != RS_MEM_DEVICE) { set_error("bad batch mem kind"); return RS_ERR_INVALID; }
    if (!b->set_rule_off || !b->rule_cond_off) { set_error("offset arrays are NULL"); return RS_ERR_INVALID; }
    if (b->P > 0 && !b->set_default) { set_error("set_default is NULL"); return RS_ERR_INVALID; }
    if (b->R > 0 && !b->rule_class) { set_error("rule_class is NULL"); return RS_ERR_INVALID; }
    if (b->C > 0 && (!b->cond_f || !b->cond_g || !b->cond_op || !b->cond_a || !b->cond_b || !b->cond_t)) {
        set_error("condition arrays are NULL");
        return RS_ERR_INVALID;
    }
    return RS_OK;
}

// Device copy of a batch: either the caller's device pointers or a staged copy of host arrays.
struct StagedBatch {
    BatchDev d{};
    void *buf = nullptr;
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte offsets of the eleven arrays of a host batch inside one staging buffer; returns its size.
static size_t staging_layout(const rs_batch *b, size_t off[11], size_t sz[11])
{
    const size_t P = b->P, R = b->R, C = b->C;
    const size_t cs = b->cond_set ? 8 * C : 0;
    const size_t s[11] = {4 * (P + 1), 4 * (R + 1), 4 * R, 4 * P, 4 * C, 4 * C, C, 4 * C, 4 * C, 4 * C, cs};
    size_t total = 0;
    for (int i = 0; i < 11; ++i) { sz[i] = s[i]; off[i] = total; total = align_up(total + s[i], 256); }
    return std::max<size_t>(total, 256);
}

// Copy a host batch into a staging buffer laid out by staging_layout (stream-ordered).
static rs_status stage_into(const rs_batch *b, char *base, cudaStream_t stream, BatchDev &d)
{
    size_t off[11], sz[11];
    staging_layout(b, off, sz);
    const void *src[11] = {b->set_rule_off, b->rule_cond_off, b->rule_class, b->set_default,
                           b->cond_f, b->cond_g, b->cond_op, b->cond_a, b->cond_b, b->cond_t, b->cond_set};
    for (int i = 0; i < 11; ++i)
        if (sz[i]) RS_CUDA(cudaMemcpyAsync(base + off[i], src[i], sz[i], cudaMemcpyHostToDevice, stream));
    d.P = b->P; d.R = b->R; d.C = b->C;
    d.set_rule_off = (const int32_t *)(base + off[0]);
    d.rule_cond_off = (const int32_t *)(base + off[1]);
    d.rule_class = (const int32_t *)(base + off[2]);
    d.set_default = (const int32_t *)(base + off[3]);
    d.cond_f = (const int32_t *)(base + off[4]);
    d.cond_g = (const int32_t *)(base + off[5]);
    d.cond_op = (const int8_t *)(base + off[6]);
    d.cond_a = (const float *)(base + off[7]);
    d.cond_b = (const float *)(base + off[8]);
    d.cond_t = (const float *)(base + off[9]);
    d.cond_set = b->cond_set ? (const uint64_t *)(base + off[10]) : nullptr;
    return RS_OK;
}

// The caller's device arrays, unchanged.
static BatchDev device_view(const rs_batch *b)
{
    BatchDev d{};
    d.P = b->P; d.R = b->R; d.C = b->C;
    d.set_rule_off = b->set_rule_off; d.rule_cond_off = b->rule_cond_off;
    d.rule_class = b->rule_class; d.set_default = b->set_default;
    d.cond_f = b->cond_f; d.cond_g = b->cond_g; d.cond_op = b->cond_op;
    d.cond_a = b->cond_a; d.cond_b = b->cond_b; d.cond_t = b->cond_t;
    d.cond_set = b->cond_set;
    return d;
}

static rs_status stage_batch(const rs_batch *b, cudaStream_t stream, StagedBatch &out)
{
    if (b->mem == RS_MEM_DEVICE) { out.d = device_view(b); return RS_OK; }
    size_t off[11], sz[11];
    const size_t total = staging_layout(b, off, sz);
    RS_CUDA(dev_alloc_async(&out.buf, total, stream));
    return stage_into(b, static_cast<char *>(out.buf), stream, out.d);
}

// ------------------------------------------------------------------------ tile configuration

static std::string tune_key(const Dataset &ds, const rs_batch *b)
{
    const double meanC = b->R > 0 ? (double)b->C / b->R : 0.0;
    const int cb = (int)std::lround(std::min(meanC, 16.0) * 2);   // half-condition buckets
    const int nb = (int)std::floor(std::log2((double)ds.N));
    std::ostringstream k;
    k << "F" << ds.F << "|K" << ds.K << "|C" << cb << "|N" << nb << (b->cond_set ? "|cat" : "");
    return k.str();
}

static int heuristic_tile(const Dataset &ds)
{
    // The rank-coded evaluator with 32 warps (it runs as the sign-mask form on datasets without
    // rank tables and as the margin-minimum form on non-finite data), then smaller tiles for wide
    // data, and for data too wide for any shared tile the configuration reading global memory.
    static const int prefs[] = {22, 21, 18, 16, 20, 3, 5, 23};
    for (int id : prefs)
        if (tile_config_fits(tile_config(id), ds.F)) return id;
    return 5;
}

int heuristic_tile_for(const Dataset &ds) { return heuristic_tile(ds); }

static int pick_tile(Ctx *ctx, const Dataset &ds, const rs_batch *b)
{
    if (ctx->forced_tile >= 0 && tile_config_fits(tile_config(ctx->forced_tile), ds.F))
        return ctx->forced_tile;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->tune_table.find(tune_key(ds, b));
        if (it != ctx->tune_table.end() && tile_config_fits(tile_config(it->second), ds.F))
            return it->second;
    }
    return heuristic_tile(ds);
}

// Strict reader of the cache file written by save_tune_table: {"key": id, ...} with ids of
// compiled configurations. A file that does not parse as a whole (truncated, edited, another
// format) or names an unknown configuration is ignored, never partly applied: the context then
// uses the heuristic until the tuner writes the file again.
static bool parse_tune_table(const std::string &s, std::map<std::string, int> &out)
{
    size_t i = 0;
    auto ws = [&] { while (i < s.size() && std::isspace((unsigned char)s[i])) ++i; };
    ws();
    if (i >= s.size() || s[i++] != '{') return false;
    ws();
    if (i < s.size() && s[i] == '}') { ++i; ws(); return i == s.size(); }
    while (true) {
        ws();
        if (i >= s.size() || s[i++] != '"') return false;
        const size_t k0 = i;
        while (i < s.size() && s[i] != '"' && s[i] != '\\' && (unsigned char)s[i] >= 0x20) ++i;
        if (i >= s.size() || s[i] != '"' || i == k0) return false;
        const std::string key = s.substr(k0, i - k0);
        ++i;
        ws();
        if (i >= s.size() || s[i++] != ':') return false;
        ws();
        const size_t d0 = i;
        while (i < s.size() && i - d0 < 6 && std::isdigit((unsigned char)s[i])) ++i;
        if (i == d0 || (i < s.size() && std::isdigit((unsigned char)s[i]))) return false;
        const int id = std::atoi(s.c_str() + d0);
        if (id < 0 || id >= tile_config_count()) return false;
        out[key] = id;
        ws();
        if (i >= s.size()) return false;
        if (s[i] == ',') { ++i; continue; }
        if (s[i] != '}') return false;
        ++i;
        ws();
        return i == s.size();
    }
}

void load_tune_table(Ctx *ctx)
{
    if (ctx->autotune_path.empty()) return;
    std::ifstream in(ctx->autotune_path, std::ios::binary);
    if (!in) return;
    std::string s((std::istreambuf_iterator<char>(in)), std::istreambuf_iterator<char>());
    if (s.size() > (1u << 20)) return;                 // not a file this library wrote
    std::map<std::string, int> table;
    if (parse_tune_table(s, table)) ctx->tune_table = std::move(table);
}

static void save_tune_table(Ctx *ctx)
{
    if (ctx->autotune_path.empty()) return;
    std::ofstream out(ctx->autotune_path + ".tmp");
    out << "{";
    bool first = true;
    for (auto &kv : ctx->tune_table) {
        out << (first ? "" : ",") << "\n  \"" << kv.first << "\": " << kv.second;
        first = false;
    }
    out << "\n}\n";
    out.close();
    std::rename((ctx->autotune_path + ".tmp").c_str(), ctx->autotune_path.c_str());
}

// ------------------------------------------------------------------------ the call

// Scratch of one call in one buffer: packed records, set descriptors, evaluation order, the
// status word, per-(set, class) last rule ends (K <= LAST_END_MAX_K) and, for host outputs,
// the device copies of the outputs. scratch_layout returns the size; with a base it also
// fills in the pointers.
static size_t scratch_layout(const BatchDev &b, bool host_out, int K, int64_t N, bool per_class,
                             bool preds, char *base, Scratch *s)
{
    const size_t rec_b = align_up(sizeof(Rec) * std::max(b.C, 1), 256);
    const size_t set_b = align_up(sizeof(SetInfo) * std::max(b.P, 1), 256);
    const size_t ord_b = align_up(sizeof(int32_t) * std::max(b.P, 1), 256);
    const size_t st_b = 256;
    const size_t le_b = K <= LAST_END_MAX_K ? align_up(sizeof(int32_t) * std::max(b.P, 1) * (size_t)K, 256) : 0;
    size_t out_b = 0;
    if (host_out) {
        out_b = align_up(sizeof(int32_t) * b.P, 256);
        if (per_class) out_b += align_up(sizeof(int32_t) * (size_t)b.P * K, 256);
        if (preds) out_b += align_up(sizeof(int32_t) * (size_t)b.P * N, 256);
    }
    if (base && s) {
        s->recs = (Rec *)base;
        s->sets = (SetInfo *)(base + rec_b);
        s->order = (int32_t *)(base + rec_b + set_b);
        s->status = (uint32_t *)(base + rec_b + set_b + ord_b);
        s->last_end = le_b ? (int32_t *)(base + rec_b + set_b + ord_b + st_b) : nullptr;
        s->out_dev = host_out ? (int32_t *)(base + rec_b + set_b + ord_b + st_b + le_b) : nullptr;
    }
    return rec_b + set_b + ord_b + st_b + le_b + out_b;
}

static rs_status alloc_scratch(const BatchDev &b, bool host_out, int K, int64_t N, bool per_class,
                               bool preds, cudaStream_t stream, Scratch &s)
{
    char *base = nullptr;
    const size_t bytes = scratch_layout(b, host_out, K, N, per_class, preds, nullptr, nullptr);
    RS_CUDA(dev_alloc_async(&base, bytes, stream));
    scratch_layout(b, host_out, K, N, per_class, preds, base, &s);
    RS_CUDA(cudaMemsetAsync(s.status, 0, sizeof(uint32_t), stream));
    return RS_OK;
}

// Enqueue pack + evaluation (the part a graph captures).
rs_status enqueue_hard(Ctx *ctx, Dataset *ds, const TileConfig &tc_in, const BatchDev &bd,
                              const Scratch &s, int32_t *correct, int32_t *per_class,
                              int32_t *preds, cudaStream_t stream)
{
    PackOut po;
    po.recs = s.recs; po.sets = s.sets; po.order = s.order; po.status = s.status;
    po.last_end = ds->K <= LAST_END_MAX_K ? s.last_end : nullptr;
    po.correct = correct;
    po.per_class = per_class;
    // batches with membership conditions run the forms that evaluate them (rank-coded or v1)
    const TileConfig &tc = bd.cond_set ? categorical_config(tc_in, *ds, preds != nullptr) : tc_in;
    const int ver = effective_version(tc, *ds, preds != nullptr);
    const int pack_ver = ver == 5 ? 5 : (ver == 4 ? 4 : (ver >= 2 ? 2 : 1));
    count_launch(ctx, launch_pack(bd, ds->F, ds->K, tc.S(), pack_ver, po, stream));
    RS_CUDA(cudaGetLastError());
    HardArgs a{};
    a.recs = s.recs;
    a.sets = s.sets;
    a.order = s.order;
    a.P = bd.P;
    a.y = ds->y;
    a.perm = ds->perm;
    a.N = ds->N;
    a.n_pad = ds->n_pad;
    a.F = ds->F;
    a.K = ds->K;
    a.correct = correct;
    a.per_class = per_class;
    a.preds = preds;
    a.groups = choose_groups(ctx, ds, tc, bd.P);
    a.status = s.status;
    a.last_end = po.last_end;
    a.Xt = ds->Xt;
    a.cat = bd.cond_set != nullptr;
    a.walked = (ctx->flags & RS_CTX_COUNT_WORK) ? ctx->d_walked : nullptr;
    return launch_hard(ctx, ds, tc, a, stream);
}

rs_status enqueue_hard_dev_sizes(Ctx *ctx, Dataset *ds, const TileConfig &tc, BatchDev bd,
                                 const int32_t *dR, const int32_t *dC, const Scratch &s,
                                 int32_t *correct, int32_t *per_class, int32_t *preds,
                                 cudaStream_t stream)
{
    // R and C are capacities here (packing grids); the kernels read the real counts from dR / dC
    bd.dR = dR;
    bd.dC = dC;
    return enqueue_hard(ctx, ds, tc, bd, s, correct, per_class, preds, stream);
}

// A cached executable graph for one call shape (dataset, tile, stream, output kinds) with the
// staging and scratch buffers it was captured against. A call whose pointers and sizes equal
// those of the last capture launches it as it is; any other call captures again and updates
// the executable in place (same topology) or instantiates it anew. The buffers only grow and
// are released with the entry (dataset destroyed or context closed). One call at a time runs
// on an entry (its mutex), so calls on one stream from several host threads stay correct. The
// capture runs on a stream of the entry's own, never on the caller's: a stream in capture mode
// would take in whatever another host thread enqueues on it meanwhile.
// What a call passes that a captured graph bakes in, apart from the entry's own buffers: sizes,
// and the caller's device pointers (device batches and device outputs; host arrays are staged
// through the entry's buffers, so only their sizes count).
struct CallShape {
    int32_t P = 0, R = 0, C = 0;
    bool host = false;
    const void *arrays[11] = {};
    const void *outputs[3] = {};
    bool operator==(const CallShape &o) const
    {
        if (P != o.P || R != o.R || C != o.C || host != o.host) return false;
        for (int i = 0; i < 11; ++i)
            if (arrays[i] != o.arrays[i]) return false;
        for (int i = 0; i < 3; ++i)
            if (outputs[i] != o.outputs[i]) return false;
        return true;
    }
};

static CallShape call_shape(const rs_batch *b, const int32_t *correct, const int32_t *per_class,
                            const int32_t *preds)
{
    CallShape c;
    c.P = b->P; c.R = b->R; c.C = b->C;
    c.host = b->mem == RS_MEM_HOST;
    if (!c.host) {
        const void *a[11] = {b->set_rule_off, b->rule_cond_off, b->rule_class, b->set_default, b->cond_f,
                             b->cond_g, b->cond_op, b->cond_a, b->cond_b, b->cond_t, b->cond_set};
        for (int i = 0; i < 11; ++i) c.arrays[i] = a[i];
        c.outputs[0] = correct; c.outputs[1] = per_class; c.outputs[2] = preds;
    }
    return c;
}

struct GraphEntry {
    std::mutex mu;
    CallShape last{};                // the previous call's shape on this entry
    bool has_last = false;
    CallShape captured{};            // the shape the executable holds
    bool has_captured = false;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;                 // kernel nodes of the executable (launch accounting on replay)
    char *stage = nullptr;           // host batches: device copy of the eleven arrays
    size_t stage_cap = 0;
    char *scratch = nullptr;
    size_t scratch_cap = 0;
    uint32_t *status_host = nullptr; // synchronous contexts: pinned copy of the status word
    // the arguments the executable was captured with
    BatchDev bd{};
    const int32_t *correct = nullptr, *per_class = nullptr, *preds = nullptr;
    const char *scratch_at = nullptr;
    ~GraphEntry()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (capture) cudaStreamDestroy(capture);
        if (stage) cudaFree(stage);
        if (scratch) cudaFree(scratch);
        if (status_host) cudaFreeHost(status_host);
    }
};

static bool same_batch(const BatchDev &a, const BatchDev &b)
{
    return a.P == b.P && a.R == b.R && a.C == b.C && a.dR == b.dR && a.dC == b.dC &&
           a.set_rule_off == b.set_rule_off && a.rule_cond_off == b.rule_cond_off &&
           a.rule_class == b.rule_class && a.set_default == b.set_default && a.cond_f == b.cond_f &&
           a.cond_g == b.cond_g && a.cond_op == b.cond_op && a.cond_a == b.cond_a &&
           a.cond_b == b.cond_b && a.cond_t == b.cond_t && a.cond_set == b.cond_set;
}

// Grow a buffer owned by a graph entry to at least `need` bytes. cudaFree of the old buffer
// waits for the device, so work still reading it (asynchronous contexts) has finished.
static rs_status grow_buffer(char *&p, size_t &cap, size_t need)
{
    if (need <= cap) return RS_OK;
    if (p) { RS_CUDA(cudaFree(p)); p = nullptr; cap = 0; }
    need = align_up(need + need / 8, 4096);   // headroom: a slowly growing batch does not re-allocate every call
    if (take_injected_alloc_failure()) return cuda_fail(cudaErrorMemoryAllocation, "cudaMalloc");
    RS_CUDA(cudaMalloc(&p, need));
    cap = need;
    return RS_OK;
}

rs_status finish_status(Ctx *ctx, const uint32_t *d_status, cudaStream_t stream);
rs_status report_status(uint32_t h);

__global__ void k_merge_status(const uint32_t *src, uint32_t *dst)
{
    if (*src) atomicOr(dst, *src);
}

static rs_status copy_outputs_to_host(const rs_batch *b, const Dataset &ds, int32_t *correct,
                                      int32_t *per_class, int32_t *preds, const int32_t *d_correct,
                                      const int32_t *d_pc, const int32_t *d_preds, cudaStream_t stream)
{
    RS_CUDA(cudaMemcpyAsync(correct, d_correct, sizeof(int32_t) * b->P, cudaMemcpyDeviceToHost, stream));
    if (per_class)
        RS_CUDA(cudaMemcpyAsync(per_class, d_pc, sizeof(int32_t) * (size_t)b->P * ds.K,
                                cudaMemcpyDeviceToHost, stream));
    if (preds)
        RS_CUDA(cudaMemcpyAsync(preds, d_preds, sizeof(int32_t) * (size_t)b->P * ds.N,
                                cudaMemcpyDeviceToHost, stream));
    return RS_OK;
}

// Device output pointers of a call: the caller's, or (host outputs) the scratch copies.
static void device_outputs(const Scratch &s, const rs_batch *b, const Dataset &ds, bool host,
                           int32_t *&d_correct, int32_t *&d_pc, int32_t *&d_preds)
{
    if (!host) return;
    d_correct = s.out_dev;
    char *p = (char *)(s.out_dev) + align_up(sizeof(int32_t) * b->P, 256);
    if (d_pc) { d_pc = (int32_t *)p; p += align_up(sizeof(int32_t) * (size_t)b->P * ds.K, 256); }
    if (d_preds) d_preds = (int32_t *)p;
}

// Kernels enqueued directly on the caller's stream, staging and scratch from the stream-ordered
// pool for this call only.
static rs_status eval_hard_direct(Ctx *ctx, Dataset *ds, int tid, const rs_batch *b, int32_t *correct,
                                  int32_t *per_class, int32_t *preds, cudaStream_t stream)
{
    rs_status rc;
    const bool host = b->mem == RS_MEM_HOST;
    StagedBatch sb;
    if ((rc = stage_batch(b, stream, sb))) return rc;
    Scratch s;
    if ((rc = alloc_scratch(sb.d, host, ds->K, ds->N, per_class != nullptr, preds != nullptr, stream, s))) {
        if (sb.buf) cudaFreeAsync(sb.buf, stream);
        return rc;
    }
    int32_t *d_correct = correct, *d_pc = per_class, *d_preds = preds;
    device_outputs(s, b, *ds, host, d_correct, d_pc, d_preds);
    rc = enqueue_hard(ctx, ds, tile_config(tid), sb.d, s, d_correct, d_pc, d_preds, stream);
    if (!rc && host) rc = copy_outputs_to_host(b, *ds, correct, per_class, preds, d_correct, d_pc, d_preds, stream);
    if (!rc) rc = finish_status(ctx, s.status, stream);
    cudaFreeAsync(s.recs, stream);
    if (sb.buf) cudaFreeAsync(sb.buf, stream);
    return rc;
}

// The graph path of eval_hard: staging and scratch live in the cached entry, and a call with
// the same arguments as the last capture is a single graph launch.
static rs_status eval_hard_graph(Ctx *ctx, uint64_t ds_h, Dataset *ds, int tid, const rs_batch *b,
                                 int32_t *correct, int32_t *per_class, int32_t *preds,
                                 cudaStream_t stream)
{
    const bool host = b->mem == RS_MEM_HOST;
    std::ostringstream key;
    key << "ds" << ds_h << "|t" << tid << "|s" << (uintptr_t)stream << "|pc" << (per_class != nullptr)
        << "|pr" << (preds != nullptr) << "|P" << (b->P > 0) << "|R" << (b->R > 0)
        << "|cat" << (b->cond_set != nullptr) << "|h" << host;
    std::shared_ptr<GraphEntry> ge;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto &slot = ctx->graphs[key.str()];
        if (!slot) slot = std::make_shared<GraphEntry>();
        ge = slot;
    }
    std::lock_guard<std::mutex> call(ge->mu);
    // A shape seen for the first time (not the captured one, not the previous call's) runs
    // directly; it is captured when the next call repeats it. Callers whose shapes change from
    // call to call so never pay for a capture.
    const CallShape shape = call_shape(b, correct, per_class, preds);
    const bool known = ge->exec && ge->has_captured && ge->captured == shape;
    const bool repeated = ge->has_last && ge->last == shape;
    ge->last = shape;
    ge->has_last = true;
    if (!known && !repeated) return eval_hard_direct(ctx, ds, tid, b, correct, per_class, preds, stream);
    rs_status rc;
    BatchDev bd;
    if (host) {
        size_t off[11], sz[11];
        if ((rc = grow_buffer(ge->stage, ge->stage_cap, staging_layout(b, off, sz)))) return rc;
        if ((rc = stage_into(b, ge->stage, stream, bd))) return rc;
    } else {
        bd = device_view(b);
    }
    const bool pc = per_class != nullptr, pr = preds != nullptr;
    if ((rc = grow_buffer(ge->scratch, ge->scratch_cap, scratch_layout(bd, host, ds->K, ds->N, pc, pr, nullptr, nullptr))))
        return rc;
    const bool async = ctx->flags & RS_CTX_ASYNC;
    if (!async && !ge->status_host) RS_CUDA(cudaHostAlloc(&ge->status_host, sizeof(uint32_t), cudaHostAllocDefault));
    Scratch s;
    scratch_layout(bd, host, ds->K, ds->N, pc, pr, ge->scratch, &s);
    int32_t *d_correct = correct, *d_pc = per_class, *d_preds = preds;
    device_outputs(s, b, *ds, host, d_correct, d_pc, d_preds);

    const bool same = ge->exec && same_batch(ge->bd, bd) && ge->correct == d_correct &&
                      ge->per_class == d_pc && ge->preds == d_preds && ge->scratch_at == ge->scratch;
    if (same) {
        RS_CUDA(cudaGraphLaunch(ge->exec, stream));
        count_launch(ctx, ge->kernels);
    } else {
        // The graph resets the status word, evaluates, and hands the status on: into the
        // context's sticky word (asynchronous contexts) or into the entry's pinned word.
        if (!ge->capture) RS_CUDA(cudaStreamCreateWithFlags(&ge->capture, cudaStreamNonBlocking));
        cudaStream_t cs = ge->capture;
        cudaGraph_t g = nullptr;
        RS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        rs_status erc = RS_OK;
        cudaError_t me = cudaMemsetAsync(s.status, 0, sizeof(uint32_t), cs);
        if (me != cudaSuccess) erc = cuda_fail(me, "cudaMemsetAsync");
        if (!erc) erc = enqueue_hard(ctx, ds, tile_config(tid), bd, s, d_correct, d_pc, d_preds, cs);
        if (!erc && async) {
            k_merge_status<<<1, 1, 0, cs>>>(s.status, ctx->d_sticky);
            me = cudaGetLastError();
            if (me != cudaSuccess) erc = cuda_fail(me, "k_merge_status");
            else count_launch(ctx);
        } else if (!erc) {
            me = cudaMemcpyAsync(ge->status_host, s.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs);
            if (me != cudaSuccess) erc = cuda_fail(me, "cudaMemcpyAsync");
        }
        cudaError_t ce = cudaStreamEndCapture(cs, &g);
        if (erc) { if (g) cudaGraphDestroy(g); return erc; }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        bool ok = false;
        if (ge->exec) {
            cudaGraphExecUpdateResultInfo info;
            ok = cudaGraphExecUpdate(ge->exec, g, &info) == cudaSuccess;
            if (!ok) cudaGetLastError();
        }
        if (!ok) {
            if (ge->exec) { cudaGraphExecDestroy(ge->exec); ge->exec = nullptr; }
            cudaError_t ie = cudaGraphInstantiate(&ge->exec, g, 0);
            if (ie != cudaSuccess) { ge->exec = nullptr; cudaGraphDestroy(g); return cuda_fail(ie, "cudaGraphInstantiate"); }
        }
        ge->kernels = graph_kernel_nodes(g);
        cudaGraphDestroy(g);
        // remember the arguments only once the executable holds them
        ge->bd = bd;
        ge->correct = d_correct; ge->per_class = d_pc; ge->preds = d_preds;
        ge->scratch_at = ge->scratch;
        ge->captured = shape;
        ge->has_captured = true;
        RS_CUDA(cudaGraphLaunch(ge->exec, stream));
    }
    if (host && (rc = copy_outputs_to_host(b, *ds, correct, per_class, preds, d_correct, d_pc, d_preds, stream)))
        return rc;
    if (async) return RS_OK;
    RS_CUDA(cudaStreamSynchronize(stream));
    return report_status(*ge->status_host);
}

rs_status eval_hard(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t *correct,
                    int32_t *per_class, int32_t *preds, cudaStream_t stream, int tile_override)
{
    rs_status rc = check_batch(b);
    if (rc) return rc;
    if (!correct && b->P > 0) { set_error("correct is NULL"); return RS_ERR_INVALID; }
    std::shared_ptr<Dataset> ds;
    if ((rc = use_dataset(ctx, ds_h, &ds))) return rc;
    if ((rc = device_guard(ctx))) return rc;
    DatasetUseMark use_mark{ctx, ds.get(), stream};
    if (b->R > 0 && ds->K > 4096) return RS_ERR_UNSUPPORTED;

    const int tid = tile_override >= 0 ? tile_override : pick_tile(ctx, *ds, b);
    // The cached graph (captured on a stream of its own, launched on the caller's) on streams the
    // caller created. Calls on the legacy default stream launch directly with scratch from the
    // stream-ordered pool: callers that use it for one-off calls of ever-changing shapes would pay
    // a capture per call and hold per-dataset buffers. A stream the caller is capturing also gets
    // the direct launches, which then join the caller's graph.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (stream) RS_CUDA(cudaStreamIsCapturing(stream, &cap));
    const bool use_graph = !(ctx->flags & (RS_CTX_NO_GRAPH | RS_CTX_PROFILE)) && tile_override < 0 &&
                           stream != nullptr && cap == cudaStreamCaptureStatusNone;
    if (use_graph) return eval_hard_graph(ctx, ds_h, ds.get(), tid, b, correct, per_class, preds, stream);

    return eval_hard_direct(ctx, ds.get(), tid, b, correct, per_class, preds, stream);
}

// Synchronous contexts: wait and report the device status word of this call. Asynchronous
// contexts: fold it into the context's sticky word (read by rs_check) and return immediately.
rs_status finish_status(Ctx *ctx, const uint32_t *d_status, cudaStream_t stream)
{
    if (ctx->flags & RS_CTX_ASYNC) {
        k_merge_status<<<1, 1, 0, stream>>>(d_status, ctx->d_sticky);
        RS_CUDA(cudaGetLastError());
        count_launch(ctx);
        return RS_OK;
    }
    uint32_t *hs = host_status_slot();
    if (!hs) return RS_ERR_OOM;
    RS_CUDA(cudaMemcpyAsync(hs, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    RS_CUDA(cudaStreamSynchronize(stream));
    return report_status(*hs);
}

// The call's result from its device status word (0: accepted).
rs_status report_status(uint32_t h)
{
    if (!h) return RS_OK;
    set_error("batch rejected: %s", status_text(h).c_str());
    if (h & (ST_WAIT_TIMEOUT | ST_QUEUE_TIMEOUT)) return RS_ERR_TIMEOUT;
    return (h & ST_TOO_LARGE) ? RS_ERR_TOO_LARGE : RS_ERR_INVALID;
}

rs_status check_async(Ctx *ctx, cudaStream_t stream)
{
    RS_CUDA(cudaStreamSynchronize(stream));
    uint32_t h = 0;
    RS_CUDA(cudaMemcpy(&h, ctx->d_sticky, sizeof(h), cudaMemcpyDeviceToHost));
    RS_CUDA(cudaMemset(ctx->d_sticky, 0, sizeof(uint32_t)));
    if (h) {
        set_error("device reported: %s", status_text(h).c_str());
        return (h & (ST_WAIT_TIMEOUT | ST_QUEUE_TIMEOUT)) ? RS_ERR_TIMEOUT : RS_ERR_INVALID;
    }
    return RS_OK;
}

// ------------------------------------------------------------------------ autotuner

rs_status autotune(Ctx *ctx, uint64_t ds_h, const rs_batch *b, cudaStream_t stream, int32_t *best)
{
    rs_status rc = check_batch(b);
    if (rc) return rc;
    if (b->mem != RS_MEM_DEVICE) { set_error("rs_autotune takes a device batch"); return RS_ERR_INVALID; }
    std::shared_ptr<Dataset> ds;
    if ((rc = use_dataset(ctx, ds_h, &ds))) return rc;
    if ((rc = device_guard(ctx))) return rc;
    DatasetUseMark use_mark{ctx, ds.get(), stream};
    int32_t *correct = nullptr;
    RS_CUDA(cudaMalloc(&correct, sizeof(int32_t) * std::max(1, b->P)));
    cudaEvent_t e0, e1;
    RS_CUDA(cudaEventCreate(&e0));
    RS_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best_id = -1;
    for (int id = 0; id < tile_config_count(); ++id) {
        if (!tile_config_fits(tile_config(id), ds->F)) continue;
        // one warm-up, then the best of two timed runs
        if ((rc = eval_hard(ctx, ds_h, b, correct, nullptr, nullptr, stream, id))) break;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, stream);
            if ((rc = eval_hard(ctx, ds_h, b, correct, nullptr, nullptr, stream, id))) break;
            cudaEventRecord(e1, stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_min = std::min(ms_min, ms);
        }
        if (rc) break;
        if (ms_min < best_ms) { best_ms = ms_min; best_id = id; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(correct);
    if (rc) return rc;
    if (best_id < 0) { set_error("no tile configuration fits F=%d", ds->F); return RS_ERR_UNSUPPORTED; }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->tune_table[tune_key(*ds, b)] = best_id;
        save_tune_table(ctx);
    }
    if (best) *best = best_id;
    return RS_OK;
}

// The configuration the next rs_eval_hard of this batch on this dataset would use.
rs_status tile_pick(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t *id)
{
    rs_status rc = check_batch(b);
    if (rc) return rc;
    if (!id) { set_error("id is NULL"); return RS_ERR_INVALID; }
    auto ds = find_dataset(ctx, ds_h);
    if (!ds) { set_error("unknown dataset %llu", (unsigned long long)ds_h); return RS_ERR_NOT_FOUND; }
    *id = pick_tile(ctx, *ds, b);
    return RS_OK;
}

// ------------------------------------------------------------------------ soft

rs_status eval_soft(Ctx *ctx, uint64_t ds_h, const rs_batch *b, float tau, float *loss,
                    float *probs, const float *dloss, float *ga, float *gb, float *gt,
                    cudaStream_t stream)
{
    rs_status rc = check_batch(b);
    if (rc) return rc;
    if (!(tau > 0.f) || !std::isfinite(tau)) { set_error("tau must be finite and > 0"); return RS_ERR_INVALID; }
    std::shared_ptr<Dataset> ds;
    if ((rc = use_dataset(ctx, ds_h, &ds))) return rc;
    if ((rc = device_guard(ctx))) return rc;
    DatasetUseMark use_mark{ctx, ds.get(), stream};
    const bool host = b->mem == RS_MEM_HOST;
    const bool bwd = dloss != nullptr;
    if (bwd && b->C > 0 && (!ga || !gb || !gt)) { set_error("gradient outputs are NULL"); return RS_ERR_INVALID; }
    StagedBatch sb;
    if ((rc = stage_batch(b, stream, sb))) return rc;
    // device-side outputs (+ staged dloss)
    const size_t P = b->P, C = b->C;
    float *d_loss = loss, *d_probs = probs, *d_ga = ga, *d_gb = gb, *d_gt = gt;
    const float *d_dloss = dloss;
    char *obuf = nullptr;
    uint32_t *d_status = nullptr;
    {
        size_t need = 256;   // status word
        if (host) {
            need += align_up(4 * std::max<size_t>(P, 1), 256) * 2;
            if (probs) need += align_up(4 * P * ds->N * ds->K, 256);
            if (bwd) need += align_up(4 * std::max<size_t>(C, 1), 256) * 3;
        }
        const cudaError_t ae = dev_alloc_async(&obuf, need, stream);
        if (ae != cudaSuccess) {
            if (sb.buf) cudaFreeAsync(sb.buf, stream);
            return cuda_fail(ae, "soft outputs");
        }
        d_status = (uint32_t *)obuf;
        char *p = obuf + 256;
        if (host) {
            d_loss = (float *)p; p += align_up(4 * std::max<size_t>(P, 1), 256);
            float *dl = (float *)p; p += align_up(4 * std::max<size_t>(P, 1), 256);
            if (probs) { d_probs = (float *)p; p += align_up(4 * P * ds->N * ds->K, 256); }
            if (bwd) {
                d_ga = (float *)p; p += align_up(4 * std::max<size_t>(C, 1), 256);
                d_gb = (float *)p; p += align_up(4 * std::max<size_t>(C, 1), 256);
                d_gt = (float *)p; p += align_up(4 * std::max<size_t>(C, 1), 256);
                RS_CUDA(cudaMemcpyAsync(dl, dloss, 4 * P, cudaMemcpyHostToDevice, stream));
                d_dloss = dl;
            }
        }
        RS_CUDA(cudaMemsetAsync(d_status, 0, 4, stream));
    }
    float *tmp_loss = nullptr;
    if (!d_loss) {   // the backward call may omit the loss output
        const cudaError_t ae = dev_alloc_async(&tmp_loss, 4 * std::max<size_t>(P, 1), stream);
        if (ae != cudaSuccess) {
            cudaFreeAsync(obuf, stream);
            if (sb.buf) cudaFreeAsync(sb.buf, stream);
            return cuda_fail(ae, "soft loss scratch");
        }
        d_loss = tmp_loss;
    }
    SoftArgs a{};
    a.b = sb.d;
    a.Xt = ds->Xt;
    a.y = ds->y;
    a.perm = ds->perm;
    a.N = ds->N;
    a.n_pad = ds->n_pad;
    a.F = ds->F;
    a.K = ds->K;
    a.tau = tau;
    a.loss = d_loss;
    a.probs = d_probs;
    a.dloss = d_dloss;
    a.grad_a = d_ga;
    a.grad_b = d_gb;
    a.grad_t = d_gt;
    a.status = d_status;
    rc = launch_soft(ctx, a, stream);
    if (rc == RS_OK && host) {
        if (loss) RS_CUDA(cudaMemcpyAsync(loss, d_loss, 4 * P, cudaMemcpyDeviceToHost, stream));
        if (probs) RS_CUDA(cudaMemcpyAsync(probs, d_probs, 4 * P * ds->N * ds->K, cudaMemcpyDeviceToHost, stream));
        if (bwd && C) {
            RS_CUDA(cudaMemcpyAsync(ga, d_ga, 4 * C, cudaMemcpyDeviceToHost, stream));
            RS_CUDA(cudaMemcpyAsync(gb, d_gb, 4 * C, cudaMemcpyDeviceToHost, stream));
            RS_CUDA(cudaMemcpyAsync(gt, d_gt, 4 * C, cudaMemcpyDeviceToHost, stream));
        }
    }
    if (rc == RS_OK) rc = finish_status(ctx, d_status, stream);
    cudaFreeAsync(obuf, stream);
    if (tmp_loss) cudaFreeAsync(tmp_loss, stream);
    if (sb.buf) cudaFreeAsync(sb.buf, stream);
    if (host && rc == RS_OK) RS_CUDA(cudaStreamSynchronize(stream));
    return rc;
}

}  // namespace rs
