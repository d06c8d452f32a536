// Hard evaluation for callers that cannot allocate device memory.
//
// rs_eval_hard_static runs the same packing and evaluator kernels as rs_eval_hard, but every
// piece of per-call scratch (condition records, per-set table, schedule order, status word and,
// for datasets of at most LAST_END_MAX_K classes, the per-class last-rule ends that let a tile of
// one label stop early) lives in one file-scope device array of fixed size instead of
// stream-ordered allocations. The array is part of the loaded module: every GPU that loads this
// library holds it until the process exits.
//
// Host code must not use the array's name as a device address (in host code it names a host-side
// stand-in). The device address is looked up with cudaGetSymbolAddress when a context is created,
// with the context's device current, and kept in the context: a context never outlives the
// primary context it was created in, so the address cannot go stale (a cudaDeviceReset while an
// rs context is alive invalidates that rs context as a whole).
#include "rs_internal.cuh"

namespace rs {

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[RS_STATIC_SCRATCH_BYTES];

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

__global__ void k_fold_status(const uint32_t *src, uint32_t *dst)
{
    if (*src) atomicOr(dst, *src);
}

// An output the kernels write must be device memory of the context's device (or managed memory):
// host memory handed here by mistake is rejected instead of being written by a kernel.
rs_status check_output(const void *p, int device, const char *name)
{
    if (!p) return RS_OK;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); at.type = cudaMemoryTypeUnregistered; }
    const bool ok = at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == device);
    if (!ok) {
        set_error("rs_eval_hard_static: %s is not device memory of device %d (use rs_eval_hard for host outputs)",
                  name, device);
        return RS_ERR_INVALID;
    }
    return RS_OK;
}

}  // namespace

// Called by rs_create with the context's device current.
rs_status static_scratch_lookup(unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    *out = static_cast<unsigned char *>(p);
    return RS_OK;
}

size_t static_scratch_need(int64_t P, int64_t C, int64_t K)
{
    const int64_t P1 = std::max<int64_t>(P, 1);
    return up256(sizeof(Rec) * (size_t)std::max<int64_t>(C, 1)) + up256(sizeof(SetInfo) * (size_t)P1) +
           up256(sizeof(int32_t) * (size_t)P1) + 256 +
           (K <= LAST_END_MAX_K ? up256(sizeof(int32_t) * (size_t)P1 * (size_t)std::max<int64_t>(K, 1)) : 0);
}

rs_status eval_hard_static(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t *correct,
                           int32_t *per_class, int32_t *preds, cudaStream_t stream)
{
    if (!b) { set_error("batch is NULL"); return RS_ERR_INVALID; }
    if (b->mem != RS_MEM_DEVICE) {
        set_error("rs_eval_hard_static takes device arrays only (batch->mem = RS_MEM_DEVICE)");
        return RS_ERR_INVALID;
    }
    if (b->P < 0 || b->R < 0 || b->C < 0) { set_error("negative batch sizes"); return RS_ERR_INVALID; }
    if (!b->set_rule_off || !b->rule_cond_off || (b->P > 0 && (!b->set_default || !correct)) ||
        (b->R > 0 && !b->rule_class) ||
        (b->C > 0 && (!b->cond_f || !b->cond_g || !b->cond_op || !b->cond_a || !b->cond_b || !b->cond_t))) {
        set_error("NULL batch or output array");
        return RS_ERR_INVALID;
    }
    auto ds = find_dataset(ctx, ds_h);
    if (!ds) { set_error("unknown dataset %llu", (unsigned long long)ds_h); return RS_ERR_NOT_FOUND; }
    if (!ds->resident) {   // rebuilding it would allocate: an allocating call makes it resident
        set_error("dataset %llu was evicted under the context's dataset budget; any allocating call on it "
                  "rebuilds it", (unsigned long long)ds_h);
        return RS_ERR_INVALID;
    }
    DatasetUseMark use_mark{ctx, ds.get(), stream, false};
    const size_t need = static_scratch_need(b->P, b->C, ds->K);
    if (need > RS_STATIC_SCRATCH_BYTES) {
        set_error("batch needs %zu bytes of scratch (P=%d, C=%d, K=%d); rs_eval_hard_static holds %zu "
                  "(16 B per condition + 20 B per set + 4 B per set and class when K <= %d + 768 B); "
                  "use rs_eval_hard",
                  need, b->P, b->C, ds->K, (size_t)RS_STATIC_SCRATCH_BYTES, LAST_END_MAX_K);
        return RS_ERR_TOO_LARGE;
    }
    rs_status rc = device_guard(ctx);
    if (rc) return rc;
    if ((rc = check_output(correct, ctx->device, "correct")) || (rc = check_output(per_class, ctx->device, "per_class")) ||
        (rc = check_output(preds, ctx->device, "preds")))
        return rc;
    unsigned char *base = ctx->static_scratch;
    if (!base) { set_error("static scratch address unknown"); return RS_ERR_DEVICE; }

    Scratch s;
    s.recs = reinterpret_cast<Rec *>(base);
    s.sets = reinterpret_cast<SetInfo *>(base + up256(sizeof(Rec) * (size_t)std::max(b->C, 1)));
    s.order = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(s.sets) +
                                          up256(sizeof(SetInfo) * (size_t)std::max(b->P, 1)));
    s.status = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(s.order) +
                                            up256(sizeof(int32_t) * (size_t)std::max(b->P, 1)));
    if (ds->K <= LAST_END_MAX_K) s.last_end = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(s.status) + 256);
    // The array keeps the previous call's contents: the status word must start at zero. Records,
    // the set table, the order and the per-class last-rule ends are fully rewritten by the packer
    // before they are read.
    RS_CUDA(cudaMemsetAsync(s.status, 0, sizeof(uint32_t), stream));

    BatchDev bd{};
    bd.P = b->P; bd.R = b->R; bd.C = b->C;
    bd.set_rule_off = b->set_rule_off; bd.rule_cond_off = b->rule_cond_off;
    bd.rule_class = b->rule_class; bd.set_default = b->set_default;
    bd.cond_f = b->cond_f; bd.cond_g = b->cond_g; bd.cond_op = b->cond_op;
    bd.cond_a = b->cond_a; bd.cond_b = b->cond_b; bd.cond_t = b->cond_t;
    bd.cond_set = b->cond_set;

    const int tid = ctx->forced_tile >= 0 && tile_config_fits(tile_config(ctx->forced_tile), ds->F)
                        ? ctx->forced_tile
                        : heuristic_tile_for(*ds);
    if ((rc = enqueue_hard(ctx, ds.get(), tile_config(tid), bd, s, correct, per_class, preds, stream)))
        return rc;

    if (ctx->flags & RS_CTX_ASYNC) {
        k_fold_status<<<1, 1, 0, stream>>>(s.status, ctx->d_sticky);
        RS_CUDA(cudaGetLastError());
        count_launch(ctx);
        return RS_OK;
    }
    uint32_t st = 0;
    RS_CUDA(cudaMemcpyAsync(&st, s.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    RS_CUDA(cudaStreamSynchronize(stream));
    if (st) {
        set_error("batch rejected: %s", status_text(st).c_str());
        return (st & (ST_WAIT_TIMEOUT | ST_QUEUE_TIMEOUT)) ? RS_ERR_TIMEOUT : RS_ERR_INVALID;
    }
    return RS_OK;
}

}  // namespace rs
