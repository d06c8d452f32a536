// extern "C" entry points declared in include/rs.h. Every function converts exceptions and CUDA
// errors into rs_status and never lets a C++ exception cross the boundary.
#include <nvtx3/nvToolsExt.h>
#include <new>

#include "rs_internal.cuh"

namespace rs {
const char *last_error();
rs_status dataset_create(Ctx *ctx, const float *X, const int32_t *y, int64_t N, int32_t F,
                         int32_t K, int32_t mem, cudaStream_t stream, uint64_t *out);
rs_status dataset_destroy(Ctx *ctx, uint64_t h, bool force);
rs_status eval_hard(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t *correct,
                    int32_t *per_class, int32_t *preds, cudaStream_t stream, int tile_override);
rs_status eval_soft(Ctx *ctx, uint64_t ds_h, const rs_batch *b, float tau, float *loss,
                    float *probs, const float *dloss, float *ga, float *gb, float *gt,
                    cudaStream_t stream);
rs_status autotune(Ctx *ctx, uint64_t ds_h, const rs_batch *b, cudaStream_t stream, int32_t *best);
rs_status check_async(Ctx *ctx, cudaStream_t stream);
rs_status selftest_rewrite(const float *a_h, const float *t_h, const int8_t *op_h, int n,
                           uint64_t *mismatches, int sm_count);
void load_tune_table(Ctx *ctx);
void server_shutdown(Ctx *ctx);
rs_status profile_read(Ctx *ctx, rs_profile *out, int reset);
rs_status submit(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t kind, uint64_t *ticket);
rs_status poll(Ctx *ctx, uint64_t ticket, int64_t timeout_us, int32_t *correct, int32_t *per_class,
               rs_ticket_info *info);
rs_status cancel(Ctx *ctx, uint64_t ticket);
rs_status submit_soft(Ctx *ctx, uint64_t ds_h, const rs_batch *b, float tau, uint64_t *ticket);
rs_status poll_soft(Ctx *ctx, uint64_t ticket, int64_t timeout_us, float *loss, rs_ticket_info *info);
rs_status server_stats(Ctx *ctx, rs_serving_stats *out);
rs_status evolve_run(Ctx *ctx, uint64_t ds_h, const rs_evolve_config *cfg, rs_population *hp,
                     int32_t *best_out, double *mean_out, cudaStream_t s);
rs_status finetune_run(Ctx *ctx, uint64_t ds_h, const rs_batch *b, float *pa, float *pb, float *pt,
                       float tau, float lr, int steps, float *loss_trace, cudaStream_t s);
void set_injected_alloc_failures(int32_t skip, int32_t count);
void preload_hard_kernels();
void preload_hard2_kernels();
void preload_hard4_kernels();
void preload_hard5_kernels();
void preload_pack_kernels();
void preload_soft_kernels();
void preload_serve_kernels();
void preload_dataset_kernels();
rs_status selftest_bounded_wait(Ctx *ctx, int64_t limit_ns, cudaStream_t stream);
rs_status eval_hard_static(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t *correct,
                           int32_t *per_class, int32_t *preds, cudaStream_t stream);
rs_status static_scratch_lookup(unsigned char **out);
rs_status tile_pick(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t *id);
rs_status selftest_soft_math(int which, const float *e_h, int n, float *out_h, cudaStream_t stream);
rs_status measure_pipe_rates(Ctx *ctx, rs_pipe_rates *out);
}  // namespace rs

using namespace rs;

// Every entry point is an NVTX range named after it (no cost unless a profiler attaches).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Every entry point leaves the calling thread's current device as it found it: the library makes
// its context's device current for its own work and restores the caller's on return.
struct CurrentDeviceRestore {
    int prev = -1;
    CurrentDeviceRestore()
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
    }
    ~CurrentDeviceRestore()
    {
        int cur = -1;
        if (prev < 0) return;
        if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return; }
        if (cur != prev && cudaSetDevice(prev) != cudaSuccess) cudaGetLastError();
    }
};

#define RS_GUARD(...)                                                    \
    try {                                                                \
        CurrentDeviceRestore device_restore_;                            \
        NvtxRange nvtx_range_(__func__);                                 \
        __VA_ARGS__                                                      \
    } catch (const std::bad_alloc &) {                                   \
        set_error("host allocation failed");                             \
        return RS_ERR_OOM;                                               \
    } catch (...) {                                                      \
        set_error("internal error");                                     \
        return RS_ERR_DEVICE;                                            \
    }

static cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char *rs_last_error(void) { return rs::last_error(); }
const char *rs_version(void) { return "rulesgpu 0.1 (sm_103a)"; }

rs_status rs_create(const rs_config *cfg, rs_ctx **out)
{
    RS_GUARD({
        if (!out) { set_error("out is NULL"); return RS_ERR_INVALID; }
        *out = nullptr;
        rs_config c{0, 0, 0, nullptr};
        if (cfg) c = *cfg;
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            set_error("no CUDA device available");
            return RS_ERR_UNSUPPORTED;
        }
        if (c.device < 0 || c.device >= ndev) { set_error("bad device %d", c.device); return RS_ERR_INVALID; }
        RS_CUDA(cudaSetDevice(c.device));
        cudaDeviceProp prop;
        RS_CUDA(cudaGetDeviceProperties(&prop, c.device));
        if (!(prop.major == 10 && prop.minor == 3)) {
            set_error("device %d is sm_%d%d; this library is built for sm_103a", c.device, prop.major, prop.minor);
            return RS_ERR_UNSUPPORTED;
        }
        auto *ctx = new rs_ctx();
        ctx->device = c.device;
        ctx->flags = c.flags;
        ctx->sm_count = prop.multiProcessorCount;
        ctx->smem_optin = prop.sharedMemPerBlockOptin;
        ctx->budget = c.mem_budget_bytes ? c.mem_budget_bytes : (40ull << 30);
        if (c.autotune_cache) ctx->autotune_path = c.autotune_cache;
        if (cudaMalloc(&ctx->d_sticky, sizeof(uint32_t)) != cudaSuccess ||
            cudaMemset(ctx->d_sticky, 0, sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            set_error("cannot allocate the context status word");
            return RS_ERR_OOM;
        }
        if (cudaMalloc(&ctx->d_walked, 4 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMemset(ctx->d_walked, 0, 4 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ctx->d_sticky);
            delete ctx;
            set_error("cannot allocate the context's counters");
            return RS_ERR_OOM;
        }
        // device address of rs_eval_hard_static's fixed scratch array, with this device current
        if (rs_status rc = static_scratch_lookup(&ctx->static_scratch)) {
            cudaFree(ctx->d_sticky);
            cudaFree(ctx->d_walked);
            delete ctx;
            return rc;
        }
        // keep freed stream-ordered scratch in the pool instead of returning it to the OS
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
        // load every kernel now rather than at the first launch that needs it (lazy loading would
        // put that cost on the first requests)
        preload_dataset_kernels();
        preload_pack_kernels();
        preload_hard_kernels();
        preload_hard2_kernels();
        preload_hard4_kernels();
        preload_hard5_kernels();
        preload_soft_kernels();
        preload_serve_kernels();
        cudaGetLastError();
        if (!(ctx->flags & RS_CTX_NO_AUTOTUNE)) load_tune_table(ctx);
        *out = ctx;
        return RS_OK;
    })
}

rs_status rs_destroy(rs_ctx *ctx)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        cudaSetDevice(ctx->device);
        server_shutdown(ctx);
        cudaDeviceSynchronize();
        std::vector<uint64_t> ids;
        for (auto &kv : ctx->datasets) ids.push_back(kv.first);
        for (auto id : ids) dataset_destroy(ctx, id, true);   // serving is shut down: nothing reads them
        release_dataset_events(ctx);
        ctx->graphs.clear();
        cudaFree(ctx->d_sticky);
        cudaFree(ctx->d_walked);
        delete ctx;
        return RS_OK;
    })
}

rs_status rs_check(rs_ctx *ctx, void *stream)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return check_async(ctx, S(stream));
    })
}

rs_status rs_dataset_create(rs_ctx *ctx, const float *X, const int32_t *y, int64_t N, int32_t F,
                            int32_t K, int32_t mem, void *stream, uint64_t *ds_out)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return dataset_create(ctx, X, y, N, F, K, mem, S(stream), ds_out);
    })
}

rs_status rs_set_dataset_budget(rs_ctx *ctx, uint64_t bytes)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return set_dataset_budget(ctx, bytes);
    })
}

rs_status rs_dataset_stats_read(rs_ctx *ctx, rs_dataset_stats *out)
{
    RS_GUARD({
        if (!ctx || !out) return RS_ERR_INVALID;
        std::lock_guard<std::mutex> lk(ctx->mu);
        *out = rs_dataset_stats{};
        for (auto &kv : ctx->datasets) {
            ++out->datasets;
            if (kv.second->resident) ++out->resident;
        }
        out->resident_bytes = ctx->ds_resident;
        out->evictions = ctx->ds_evictions;
        out->rebuilds = ctx->ds_rebuilds;
        return RS_OK;
    })
}

rs_status rs_dataset_destroy(rs_ctx *ctx, uint64_t ds)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return dataset_destroy(ctx, ds, false);
    })
}

rs_status rs_dataset_info(rs_ctx *ctx, uint64_t ds, int64_t *N, int32_t *F, int32_t *K,
                          int64_t *class_count)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        auto d = find_dataset(ctx, ds);
        if (!d) { set_error("unknown dataset"); return RS_ERR_NOT_FOUND; }
        if (N) *N = d->N;
        if (F) *F = d->F;
        if (K) *K = d->K;
        if (class_count)
            for (int k = 0; k < d->K; ++k) class_count[k] = d->class_count[k];
        return RS_OK;
    })
}

rs_status rs_eval_hard(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t *correct,
                       int32_t *per_class, int32_t *preds, void *stream)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return eval_hard(ctx, ds, batch, correct, per_class, preds, S(stream), -1);
    })
}

rs_status rs_eval_hard_static(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t *correct,
                              int32_t *per_class, int32_t *preds, void *stream)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return eval_hard_static(ctx, ds, batch, correct, per_class, preds, S(stream));
    })
}

rs_status rs_eval_soft_fwd(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float tau,
                           float *loss, float *probs, void *stream)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        if (!loss) { set_error("loss is NULL"); return RS_ERR_INVALID; }
        return eval_soft(ctx, ds, batch, tau, loss, probs, nullptr, nullptr, nullptr, nullptr,
                         S(stream));
    })
}

rs_status rs_eval_soft_bwd(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float tau,
                           const float *dloss, float *grad_a, float *grad_b, float *grad_t,
                           float *loss, void *stream)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        if (!dloss) { set_error("dloss is NULL"); return RS_ERR_INVALID; }
        return eval_soft(ctx, ds, batch, tau, loss, nullptr, dloss, grad_a, grad_b, grad_t,
                         S(stream));
    })
}

rs_status rs_profile_read(rs_ctx *ctx, rs_profile *out, int32_t reset)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return profile_read(ctx, out, reset);
    })
}

rs_status rs_evolve(rs_ctx *ctx, uint64_t ds, const rs_evolve_config *cfg, rs_population *pop,
                    int32_t *best, double *mean, void *stream)
{
    RS_GUARD({
        if (!ctx || !cfg || !pop) return RS_ERR_INVALID;
        return evolve_run(ctx, ds, cfg, pop, best, mean, S(stream));
    })
}

rs_status rs_finetune(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float *a, float *b, float *t,
                      float tau, float lr, int32_t steps, float *loss_trace, void *stream)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return finetune_run(ctx, ds, batch, a, b, t, tau, lr, steps, loss_trace, S(stream));
    })
}

rs_status rs_submit(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t kind, uint64_t *ticket)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return submit(ctx, ds, batch, kind, ticket);
    })
}

rs_status rs_poll(rs_ctx *ctx, uint64_t ticket, int64_t timeout_us, int32_t *correct,
                  int32_t *per_class, rs_ticket_info *info)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return poll(ctx, ticket, timeout_us, correct, per_class, info);
    })
}

rs_status rs_submit_soft(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, float tau, uint64_t *ticket)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return submit_soft(ctx, ds, batch, tau, ticket);
    })
}

rs_status rs_poll_soft(rs_ctx *ctx, uint64_t ticket, int64_t timeout_us, float *loss, rs_ticket_info *info)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return poll_soft(ctx, ticket, timeout_us, loss, info);
    })
}

rs_status rs_cancel(rs_ctx *ctx, uint64_t ticket)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return cancel(ctx, ticket);
    })
}

rs_status rs_serving_stats_read(rs_ctx *ctx, rs_serving_stats *out)
{
    RS_GUARD({
        if (!ctx || !out) return RS_ERR_INVALID;
        return server_stats(ctx, out);
    })
}

int32_t rs_tile_config_count(void) { return tile_config_count(); }

rs_status rs_tile_config_info(int32_t id, int32_t *samples_per_tile, int32_t *warps,
                              int32_t *samples_per_lane)
{
    if (id < 0 || id >= tile_config_count()) { set_error("bad tile config %d", id); return RS_ERR_INVALID; }
    const TileConfig &t = tile_config(id);
    if (samples_per_tile) *samples_per_tile = t.S();
    if (warps) *warps = t.W;
    if (samples_per_lane) *samples_per_lane = t.V;
    return RS_OK;
}

rs_status rs_tile_config_form(int32_t id, int32_t *form)
{
    if (id < 0 || id >= tile_config_count() || !form) { set_error("bad tile config %d", id); return RS_ERR_INVALID; }
    *form = tile_config(id).ver;
    return RS_OK;
}

rs_status rs_set_tile_config(rs_ctx *ctx, int32_t id)
{
    if (!ctx) return RS_ERR_INVALID;
    if (id < -1 || id >= tile_config_count()) { set_error("bad tile config %d", id); return RS_ERR_INVALID; }
    ctx->forced_tile = id;
    return RS_OK;
}

rs_status rs_tile_config_pick(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, int32_t *id)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return tile_pick(ctx, ds, batch, id);
    })
}

rs_status rs_autotune(rs_ctx *ctx, uint64_t ds, const rs_batch *batch, void *stream, int32_t *best)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        return autotune(ctx, ds, batch, S(stream), best);
    })
}

rs_status rs_measure_pipe_rates(rs_ctx *ctx, rs_pipe_rates *out)
{
    RS_GUARD({
        if (!ctx || !out) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return measure_pipe_rates(ctx, out);
    })
}

rs_status rs_selftest_log1p_unit(rs_ctx *ctx, const float *e, int32_t n, float *out)
{
    RS_GUARD({
        if (!ctx || !e || !out || n < 1) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return selftest_soft_math(0, e, n, out, nullptr);
    })
}

rs_status rs_selftest_log1m_exp(rs_ctx *ctx, const float *s, int32_t n, float *out)
{
    RS_GUARD({
        if (!ctx || !s || !out || n < 1) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return selftest_soft_math(1, s, n, out, nullptr);
    })
}

rs_status rs_selftest_threshold_rewrite(rs_ctx *ctx, const float *a, const float *t,
                                        const int8_t *op, int32_t n, uint64_t *mismatches)
{
    RS_GUARD({
        if (!ctx || !a || !t || !op || !mismatches || n < 1) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return selftest_rewrite(a, t, op, n, mismatches, ctx->sm_count);
    })
}

rs_status rs_inject_alloc_failures(int32_t skip, int32_t count)
{
    RS_GUARD({
        if (skip < 0 || count < 0) return RS_ERR_INVALID;
        set_injected_alloc_failures(skip, count);
        return RS_OK;
    })
}

rs_status rs_selftest_bounded_wait(rs_ctx *ctx, int64_t limit_ns, void *stream)
{
    RS_GUARD({
        if (!ctx) return RS_ERR_INVALID;
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        return selftest_bounded_wait(ctx, limit_ns, S(stream));
    })
}

}  // extern "C"
