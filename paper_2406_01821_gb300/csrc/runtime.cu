// Runtime: errors, contexts, dataset registration (feature-major, label-grouped, on device).
#include <cstdarg>
#include <cstring>
#include <cudaTypedefs.h>

#include "rs_internal.cuh"
#include "dataset_lru.h"
#include "tma.cuh"

namespace rs {

// ------------------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

const char *last_error() { return g_last_error.c_str(); }

static std::mutex g_inject_mu;
static int32_t g_inject_skip = 0, g_inject_fail = 0;
static std::atomic<bool> g_inject_armed{false};

void set_injected_alloc_failures(int32_t skip, int32_t count)
{
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_skip = skip;
    g_inject_fail = count;
    g_inject_armed.store(count > 0);
}

bool take_injected_alloc_failure()
{
    if (!g_inject_armed.load(std::memory_order_relaxed)) return false;
    std::lock_guard<std::mutex> lk(g_inject_mu);
    if (g_inject_skip > 0) { --g_inject_skip; return false; }
    if (g_inject_fail > 0) {
        if (--g_inject_fail == 0) g_inject_armed.store(false);
        return true;
    }
    return false;
}

// A bounded wait on an mbarrier that nothing completes: the wait must give up within limit_ns.
__global__ void k_bounded_wait_selftest(uint64_t limit_ns, uint32_t *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool landed = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!__syncthreads_and(landed) && threadIdx.x == 0) atomicOr(status, ST_WAIT_TIMEOUT);
}

rs_status selftest_bounded_wait(Ctx *ctx, int64_t limit_ns, cudaStream_t stream)
{
    const uint64_t lim = (uint64_t)std::min<int64_t>(std::max<int64_t>(limit_ns, 1000000), 2000000000);
    uint32_t *d = nullptr;
    RS_CUDA(cudaMallocAsync(&d, sizeof(uint32_t), stream));
    RS_CUDA(cudaMemsetAsync(d, 0, sizeof(uint32_t), stream));
    k_bounded_wait_selftest<<<1, 32, 0, stream>>>(lim, d);
    count_launch(ctx);
    uint32_t h = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    cudaFreeAsync(d, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    if (h & ST_WAIT_TIMEOUT) {
        set_error("device wait gave up after %.1f ms (self-test)", (double)lim / 1e6);
        return RS_ERR_TIMEOUT;
    }
    return RS_OK;
}

rs_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RS_ERR_OOM;
    }
    return RS_ERR_DEVICE;
}

std::string status_text(uint32_t st)
{
    std::string s;
    auto add = [&](uint32_t bit, const char *t) {
        if (st & bit) { if (!s.empty()) s += ", "; s += t; }
    };
    add(ST_BAD_OFFSETS, "malformed offset arrays");
    add(ST_BAD_CLASS, "class id out of range");
    add(ST_BAD_FEATURE, "feature index out of range");
    add(ST_BAD_OP, "comparison op not 0 ('>') or 1 ('<')");
    add(ST_BAD_LABEL, "label out of range");
    add(ST_TOO_LARGE, "a set exceeds the soft path's rule or condition limit");
    add(ST_WAIT_TIMEOUT, "device wait limit reached");
    add(ST_QUEUE_TIMEOUT, "work queue wait limit reached");
    return s;
}

uint32_t *host_status_slot()
{
    // one pinned word per host thread, allocated on first use and kept for the thread's life
    struct Slot {
        uint32_t *p = nullptr;
        ~Slot() { if (p) cudaFreeHost(p); }
    };
    static thread_local Slot slot;
    if (!slot.p) {
        if (cudaHostAlloc(&slot.p, 64, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            slot.p = nullptr;
        }
    }
    return slot.p;
}

rs_status device_guard(Ctx *ctx)
{
    int cur = -1;
    RS_CUDA(cudaGetDevice(&cur));
    if (cur != ctx->device) RS_CUDA(cudaSetDevice(ctx->device));
    return RS_OK;
}

std::shared_ptr<Dataset> find_dataset(Ctx *ctx, uint64_t ds)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(ds);
    if (it == ctx->datasets.end()) return nullptr;
    return it->second;
}

// ------------------------------------------------------------------------------ profiling

static cudaEvent_t take_event(Profiler &p)
{
    if (!p.pool.empty()) { cudaEvent_t e = p.pool.back(); p.pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

TimedLaunch::TimedLaunch(Ctx *c, int k, cudaStream_t s) : ctx(c), kind(k), stream(s)
{
    if (!(ctx->flags & RS_CTX_PROFILE)) return;
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    e0 = take_event(ctx->prof);
    e1 = take_event(ctx->prof);
    if (e0) cudaEventRecord(e0, stream);
}

TimedLaunch::~TimedLaunch()
{
    if (!e0 || !e1) return;
    cudaEventRecord(e1, stream);
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    ctx->prof.pending.push_back({e0, e1, kind});
}

rs_status profile_read(Ctx *ctx, rs_profile *out, int reset)
{
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    for (auto &p : ctx->prof.pending) {
        RS_CUDA(cudaEventSynchronize(p.e1));
        float ms = 0.f;
        RS_CUDA(cudaEventElapsedTime(&ms, p.e0, p.e1));
        ctx->prof.n[p.kind] += 1;
        ctx->prof.ms[p.kind] += ms;
        ctx->prof.pool.push_back(p.e0);
        ctx->prof.pool.push_back(p.e1);
    }
    ctx->prof.pending.clear();
    unsigned long long w[4] = {0, 0, 0, 0};
    const bool walked = ctx->d_walked && (ctx->flags & RS_CTX_COUNT_WORK);
    if (walked) {
        RS_CUDA(cudaDeviceSynchronize());
        RS_CUDA(cudaMemcpy(w, ctx->d_walked, sizeof(w), cudaMemcpyDeviceToHost));
    }
    if (out) {
        out->launches = ctx->prof.launches.load();
        out->hard_launches = ctx->prof.n[TK_HARD];
        out->hard_ms = ctx->prof.ms[TK_HARD];
        out->soft_launches = ctx->prof.n[TK_SOFT];
        out->soft_ms = ctx->prof.ms[TK_SOFT];
        out->hard_records_walked = (int64_t)w[0];
        out->hard_rows_walked = (int64_t)w[1];
        out->hard_rule_ends_walked = (int64_t)w[2];
        out->hard_set_tiles = (int64_t)w[3];
    }
    if (reset) {
        ctx->prof.launches = 0;
        ctx->prof.n[0] = ctx->prof.n[1] = 0;
        ctx->prof.ms[0] = ctx->prof.ms[1] = 0;
        if (walked) RS_CUDA(cudaMemset(ctx->d_walked, 0, sizeof(w)));
    }
    return RS_OK;
}

// ------------------------------------------------------------------------------ registration

namespace {

constexpr int REG_BLOCK = 1024;

// Per block of REG_BLOCK samples: label histogram and each sample's rank among earlier samples
// of the same label in the block (a stable order within the block).
__global__ void k_label_rank(const int32_t *y, int64_t N, int K, int32_t *blk_count,
                             int32_t *rank, uint32_t *status)
{
    extern __shared__ int32_t sh[];
    int32_t *ys = sh;                 // [REG_BLOCK]
    int32_t *hist = sh + REG_BLOCK;   // [K]
    const int64_t n = (int64_t)blockIdx.x * REG_BLOCK + threadIdx.x;
    for (int k = threadIdx.x; k < K; k += blockDim.x) hist[k] = 0;
    int lab = -1;
    if (n < N) {
        lab = y[n];
        if (lab < 0 || lab >= K) { atomicOr(status, ST_BAD_LABEL); lab = -1; }
    }
    ys[threadIdx.x] = lab;
    __syncthreads();
    if (lab >= 0) atomicAdd(&hist[lab], 1);
    int r = 0;
    for (int i = 0; i < (int)threadIdx.x; ++i) r += (ys[i] == lab);
    if (n < N) rank[n] = r;
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        blk_count[(int64_t)blockIdx.x * K + k] = hist[k];
}

// One thread per label: exclusive offsets of every block within the label-grouped order.
__global__ void k_label_offsets(int32_t *blk_count, int64_t nblk, int K, int64_t *class_total)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int64_t run = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        int32_t c = blk_count[b * K + k];
        blk_count[b * K + k] = (int32_t)run;
        run += c;
    }
    class_total[k] = run;
}

__global__ void k_class_start(const int64_t *class_total, int K, int64_t *class_start)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t run = 0;
        for (int k = 0; k < K; ++k) { class_start[k] = run; run += class_total[k]; }
    }
}

__global__ void k_label_scatter(const int32_t *y, int64_t N, int K, const int32_t *blk_off,
                                const int64_t *class_start, const int32_t *rank, int32_t *perm,
                                int32_t *inv, int32_t *y_sorted)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int lab = y[n];
    if (lab < 0 || lab >= K) return;
    const int64_t blk = n / REG_BLOCK;
    const int64_t pos = class_start[lab] + blk_off[blk * K + lab] + rank[n];
    perm[pos] = (int32_t)n;
    inv[n] = (int32_t)pos;
    y_sorted[pos] = lab;
}

// Xt[f][m] = X[perm[m]][f] for m < N, 0 for the padding; 32x32 tiles through shared memory.
__global__ void k_transpose_gather(const float *X, int64_t N, int F, int64_t n_pad,
                                   const int32_t *perm, float *Xt)
{
    __shared__ float tile[32][33];
    const int64_t m0 = (int64_t)blockIdx.x * 32;
    const int f0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int64_t m = m0 + j;
        const int f = f0 + tx;
        float v = 0.f;
        if (m < N && f < F) v = X[(int64_t)perm[m] * F + f];
        tile[j][tx] = v;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int f = f0 + j;
        const int64_t m = m0 + tx;
        if (f < F && m < n_pad) Xt[(int64_t)f * n_pad + m] = tile[tx][j];
    }
}

__global__ void k_nonfinite(const float *x, int64_t n, uint32_t *flag)
{
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Rank table of one 128-sample tile and feature per warp: the position of each value in the
// tile's ascending order, equal values in sample order (-0 before +0: any order within a group of
// equal values keeps the group contiguous, which is all the cut tests need). The evaluators
// rebuild the sorted column from it in shared memory (one scatter), so it is the only table kept
// beside the features. The warp sorts the keys (value order, then sample) with a bitonic network,
// lane l holding elements 4l .. 4l+3, and scatters each element's final place back to its sample.
__global__ void k_rank_tiles(const float *Xt, int64_t n_pad, int F, uint8_t *Rk)
{
    __shared__ uint8_t pos_of[8][RANK_TILE];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int f = blockIdx.y * (blockDim.x >> 5) + wib;
    if (f >= F) return;
    const int64_t t = blockIdx.x;
    const float4 x4 = *reinterpret_cast<const float4 *>(Xt + (int64_t)f * n_pad + t * RANK_TILE + 4 * lane);
    const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
    unsigned long long a[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const uint32_t u = __float_as_uint(xv[v]);
        const uint32_t key = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // float order (finite data)
        a[v] = ((unsigned long long)key << 32) | (uint32_t)(4 * lane + v);
    }
#pragma unroll
    for (int k = 2; k <= RANK_TILE; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 4) {                            // partners in lane ^ (j / 4), same slot
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int e = 4 * lane + v;
                    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, a[v], j >> 2);
                    const bool take_min = ((e & j) == 0) == ((e & k) == 0);
                    a[v] = take_min ? (o < a[v] ? o : a[v]) : (o > a[v] ? o : a[v]);
                }
            } else {                                 // partners within the lane
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    if (v & j) continue;
                    const int w = v | j;
                    const bool asc = ((4 * lane + v) & k) == 0;
                    const unsigned long long lo = a[v] < a[w] ? a[v] : a[w], hi = a[v] < a[w] ? a[w] : a[v];
                    a[v] = asc ? lo : hi;
                    a[w] = asc ? hi : lo;
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) pos_of[wib][(uint32_t)a[v]] = (uint8_t)(4 * lane + v);
    __syncwarp();
    const uint32_t w = *reinterpret_cast<const uint32_t *>(&pos_of[wib][4 * lane]);
    reinterpret_cast<uint32_t *>(Rk + (int64_t)f * n_pad + t * RANK_TILE)[lane] = w;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

const CUtensorMap *dataset_rank_tmap(Dataset *ds)
{
    std::lock_guard<std::mutex> lk(ds->mu);
    if (ds->rmap_ok) return &ds->rmap;
    if (!ds->Rk) { set_error("dataset has no rank tables"); return nullptr; }
    auto enc = get_encode();
    if (!enc) { set_error("cuTensorMapEncodeTiled not available"); return nullptr; }
    cuuint64_t dims[2] = {(cuuint64_t)ds->n_pad, (cuuint64_t)ds->F};
    cuuint64_t strides[1] = {(cuuint64_t)ds->n_pad};
    cuuint32_t box[2] = {(cuuint32_t)RANK_TILE, (cuuint32_t)(ds->F < 256 ? ds->F : 256)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&ds->rmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ds->Rk, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for the rank table, F=%d", (int)r, ds->F);
        return nullptr;
    }
    ds->rmap_ok = true;
    return &ds->rmap;
}

const CUtensorMap *dataset_tmap(Dataset *ds, int S)
{
    std::lock_guard<std::mutex> lk(ds->mu);
    auto it = ds->tmaps.find(S);
    if (it != ds->tmaps.end()) return &it->second;
    auto enc = get_encode();
    if (!enc) { set_error("cuTensorMapEncodeTiled not available"); return nullptr; }
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)ds->n_pad, (cuuint64_t)ds->F};
    cuuint64_t strides[1] = {(cuuint64_t)ds->n_pad * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)S, (cuuint32_t)(ds->F < 256 ? ds->F : 256)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ds->Xt, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for S=%d F=%d", (int)r, S, ds->F);
        return nullptr;
    }
    auto res = ds->tmaps.emplace(S, m);
    return &res.first->second;
}

// Build the device copy of dataset d (N, F, K and n_pad set) from X and y (host or device per
// `mem`): feature-major Xt grouped by label, labels, permutation and inverse, class counts, the
// finite flag and, for finite data of at most RANK_MAX_F features, the rank table.
static rs_status build_device(Dataset &d, const float *X, const int32_t *y, int32_t mem, cudaStream_t stream)
{
    const int64_t N = d.N;
    const int32_t F = d.F, K = d.K;
    const int64_t nblk = (N + REG_BLOCK - 1) / REG_BLOCK;

    float *Xd = nullptr;
    int32_t *yd = nullptr, *blk = nullptr, *rank = nullptr;
    int64_t *ctot = nullptr, *cstart = nullptr;
    uint32_t *st = nullptr;
    rs_status rc = RS_OK;
    auto cleanup = [&] {
        if (mem == RS_MEM_HOST) { cudaFree(Xd); cudaFree(yd); }
        cudaFree(blk); cudaFree(rank); cudaFree(ctot); cudaFree(cstart); cudaFree(st);
    };
    auto release = [&] {              // the dataset's own arrays, after a failure
        cudaFree(d.Xt); cudaFree(d.y); cudaFree(d.perm); cudaFree(d.inv); cudaFree(d.Rk);
        d.Xt = nullptr; d.y = nullptr; d.perm = nullptr; d.inv = nullptr; d.Rk = nullptr;
    };
#define REG_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            rc = cuda_fail(e_, #call);                      \
            cleanup();                                      \
            release();                                      \
            return rc;                                      \
        }                                                   \
    } while (0)

    if (mem == RS_MEM_HOST) {
        REG_CUDA(cudaMalloc(&Xd, sizeof(float) * N * F));
        REG_CUDA(cudaMalloc(&yd, sizeof(int32_t) * N));
        REG_CUDA(cudaMemcpyAsync(Xd, X, sizeof(float) * N * F, cudaMemcpyHostToDevice, stream));
        REG_CUDA(cudaMemcpyAsync(yd, y, sizeof(int32_t) * N, cudaMemcpyHostToDevice, stream));
    } else {
        Xd = const_cast<float *>(X);
        yd = const_cast<int32_t *>(y);
    }
    REG_CUDA(cudaMalloc(&d.Xt, sizeof(float) * d.n_pad * F));
    REG_CUDA(cudaMalloc(&d.y, sizeof(int32_t) * d.n_pad));
    REG_CUDA(cudaMalloc(&d.perm, sizeof(int32_t) * N));
    REG_CUDA(cudaMalloc(&d.inv, sizeof(int32_t) * N));
    REG_CUDA(cudaMalloc(&blk, sizeof(int32_t) * nblk * K));
    REG_CUDA(cudaMalloc(&rank, sizeof(int32_t) * N));
    REG_CUDA(cudaMalloc(&ctot, sizeof(int64_t) * K));
    REG_CUDA(cudaMalloc(&cstart, sizeof(int64_t) * K));
    REG_CUDA(cudaMalloc(&st, sizeof(uint32_t)));
    REG_CUDA(cudaMemsetAsync(st, 0, sizeof(uint32_t), stream));
    k_fill_i32<<<(unsigned)((d.n_pad + 255) / 256), 256, 0, stream>>>(d.y, d.n_pad, -1);
    k_label_rank<<<(unsigned)nblk, REG_BLOCK, sizeof(int32_t) * (REG_BLOCK + K), stream>>>(
        yd, N, K, blk, rank, st);
    REG_CUDA(cudaGetLastError());
    uint32_t hst = 0;
    // labels must be valid before they are used as scatter positions
    REG_CUDA(cudaMemcpyAsync(&hst, st, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    REG_CUDA(cudaStreamSynchronize(stream));
    if (hst) {
        cleanup();
        set_error("dataset rejected: %s", status_text(hst).c_str());
        release();
        return RS_ERR_INVALID;
    }
    k_label_offsets<<<(K + 127) / 128, 128, 0, stream>>>(blk, nblk, K, ctot);
    k_class_start<<<1, 32, 0, stream>>>(ctot, K, cstart);
    k_label_scatter<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(yd, N, K, blk, cstart, rank,
                                                                      d.perm, d.inv, d.y);
    dim3 tg((unsigned)(d.n_pad / 32), (unsigned)((F + 31) / 32));
    k_transpose_gather<<<tg, dim3(32, 8), 0, stream>>>(Xd, N, F, d.n_pad, d.perm, d.Xt);
    REG_CUDA(cudaGetLastError());
    REG_CUDA(cudaMemsetAsync(st, 0, sizeof(uint32_t), stream));
    k_nonfinite<<<1024, 256, 0, stream>>>(d.Xt, d.n_pad * F, st);
    REG_CUDA(cudaGetLastError());
    uint32_t nonfinite = 0;
    REG_CUDA(cudaMemcpyAsync(&nonfinite, st, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    d.class_count.resize(K);
    REG_CUDA(cudaMemcpyAsync(d.class_count.data(), ctot, sizeof(int64_t) * K,
                             cudaMemcpyDeviceToHost, stream));
    REG_CUDA(cudaStreamSynchronize(stream));
    d.finite = nonfinite == 0;
    if (d.finite && F <= RANK_MAX_F) {
        // rank table for the rank-coded evaluator (1 byte per value)
        REG_CUDA(cudaMalloc(&d.Rk, (size_t)d.n_pad * F));
        dim3 rg((unsigned)(d.n_pad / RANK_TILE), (unsigned)((F + 7) / 8));
        k_rank_tiles<<<rg, 256, 0, stream>>>(d.Xt, d.n_pad, F, d.Rk);
        REG_CUDA(cudaGetLastError());
        REG_CUDA(cudaStreamSynchronize(stream));
        d.ranked = true;
    }
    cleanup();
#undef REG_CUDA
    return RS_OK;
}

static size_t dataset_device_bytes(const Dataset &d)
{
    return sizeof(float) * (size_t)d.n_pad * d.F + sizeof(int32_t) * ((size_t)d.n_pad + 2 * (size_t)d.N) +
           (d.Rk ? (size_t)d.n_pad * d.F : 0);
}

static void free_device(Dataset &d)
{
    cudaFree(d.Xt);
    cudaFree(d.y);
    cudaFree(d.perm);
    cudaFree(d.inv);
    cudaFree(d.Rk);
    d.Xt = nullptr; d.y = nullptr; d.perm = nullptr; d.inv = nullptr; d.Rk = nullptr;
    std::lock_guard<std::mutex> lk(d.mu);
    d.tmaps.clear();                 // tensor maps hold the device addresses
    d.rmap_ok = false;
}

// With ctx->mu held: drop the cached graphs that reference dataset h.
static void drop_graphs(Ctx *ctx, uint64_t h)
{
    const std::string key = "ds" + std::to_string(h) + "|";
    for (auto g = ctx->graphs.begin(); g != ctx->graphs.end();) {
        if (g->first.rfind(key, 0) == 0) g = ctx->graphs.erase(g);
        else ++g;
    }
}

// With ctx->mu held: return the dataset's completed in-flight marks to the spare events; true if
// none is left (no call's device work on it is pending, as far as the marks tell).
static bool reap_marks(Ctx *ctx, Dataset &d)
{
    auto &v = d.inflight;
    for (size_t i = 0; i < v.size();) {
        const cudaError_t q = cudaEventQuery(v[i]);
        if (q == cudaErrorNotReady) { ++i; continue; }
        cudaGetLastError();
        ctx->ds_events.push_back(v[i]);
        v[i] = v.back();
        v.pop_back();
    }
    return v.empty();
}

void mark_dataset_use(Ctx *ctx, Dataset *ds, cudaStream_t stream, bool may_create)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->ds_budget) return;
    reap_marks(ctx, *ds);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) { cudaGetLastError(); cap = cudaStreamCaptureStatusActive; }
    cudaEvent_t ev = nullptr;
    if (cap == cudaStreamCaptureStatusNone) {
        if (!ctx->ds_events.empty()) {
            ev = ctx->ds_events.back();
            ctx->ds_events.pop_back();
        } else if (!may_create || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ev = nullptr;
        }
    }
    if (ev && cudaEventRecord(ev, stream) == cudaSuccess) {
        ds->inflight.push_back(ev);
        return;
    }
    cudaGetLastError();
    if (ev) ctx->ds_events.push_back(ev);
    ds->unmarked_use = true;         // its eviction waits for the whole device
}

void release_dataset_events(Ctx *ctx)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto &kv : ctx->datasets) {
        for (cudaEvent_t e : kv.second->inflight) cudaEventDestroy(e);
        kv.second->inflight.clear();
    }
    for (cudaEvent_t e : ctx->ds_events) cudaEventDestroy(e);
    ctx->ds_events.clear();
}

// With ctx->mu held: evict least recently used datasets so that `need` more device bytes fit the
// budget (dataset_lru.h), `keep` excepted.
static void make_room(Ctx *ctx, size_t need, uint64_t keep)
{
    if (!ctx->ds_budget) return;
    std::vector<lru::Entry> entries;
    for (auto &kv : ctx->datasets) {
        Dataset &d = *kv.second;
        // the registry's own reference is the only one (no call or request holds the dataset), and
        // the device work of the calls that used it has completed, or is unknown (then waited for)
        const bool idle = kv.second.use_count() == 1 && (!d.resident || reap_marks(ctx, d));
        entries.push_back({kv.first, d.dev_bytes, d.last_use, d.resident, !d.hy.empty() && idle});
    }
    const std::vector<uint64_t> v = lru::victims(entries, ctx->ds_resident, need, ctx->ds_budget, keep);
    if (v.empty()) return;
    bool unmarked = false;
    for (uint64_t h : v) unmarked |= ctx->datasets[h]->unmarked_use;
    if (unmarked) cudaDeviceSynchronize();   // work that no mark covers finishes first
    for (uint64_t h : v) {
        Dataset &d = *ctx->datasets[h];
        drop_graphs(ctx, h);
        free_device(d);
        d.resident = false;
        d.unmarked_use = false;
        ctx->ds_resident -= std::min(ctx->ds_resident, d.dev_bytes);
        ++ctx->ds_evictions;
    }
}

rs_status dataset_create(Ctx *ctx, const float *X, const int32_t *y, int64_t N, int32_t F,
                         int32_t K, int32_t mem, cudaStream_t stream, uint64_t *out)
{
    if (!X || !y || !out) { set_error("null pointer"); return RS_ERR_INVALID; }
    if (N < 1 || N > (int64_t)INT32_MAX - 1024 || F < 1 || F > RS_MAX_FEATURES || K < 1 ||
        K > RS_MAX_CLASSES) {
        set_error("dataset shape out of range (N=%lld F=%d K=%d)", (long long)N, F, K);
        return RS_ERR_INVALID;
    }
    if (mem != RS_MEM_HOST && mem != RS_MEM_DEVICE) { set_error("bad mem kind"); return RS_ERR_INVALID; }
    auto ds = std::make_shared<Dataset>();
    ds->N = N;
    ds->F = F;
    ds->K = K;
    ds->n_pad = (N + 255) / 256 * 256;
    bool budget = false;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        budget = ctx->ds_budget != 0;
        if (budget) {                 // room for the largest form it can take (with a rank table)
            const size_t upper = sizeof(float) * (size_t)ds->n_pad * F + sizeof(int32_t) * ((size_t)ds->n_pad + 2 * (size_t)N) +
                                 (F <= RANK_MAX_F ? (size_t)ds->n_pad * F : 0);
            make_room(ctx, upper, 0);
        }
    }
    if (budget) {                     // the host copy an eviction rebuilds from
        ds->hX.resize((size_t)N * F);
        ds->hy.resize((size_t)N);
        const cudaMemcpyKind kind = mem == RS_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
        cudaError_t e = cudaMemcpy(ds->hX.data(), X, sizeof(float) * (size_t)N * F, kind);
        if (e == cudaSuccess) e = cudaMemcpy(ds->hy.data(), y, sizeof(int32_t) * (size_t)N, kind);
        if (e != cudaSuccess) return cuda_fail(e, "dataset host copy");
    }
    const rs_status rc = build_device(*ds, X, y, mem, stream);
    if (rc) return rc;
    ds->dev_bytes = dataset_device_bytes(*ds);
    std::lock_guard<std::mutex> lk(ctx->mu);
    const uint64_t h = ctx->next_ds++;
    ds->last_use = ++ctx->ds_tick;
    ctx->ds_resident += ds->dev_bytes;
    ctx->datasets[h] = ds;
    *out = h;
    return RS_OK;
}

rs_status use_dataset(Ctx *ctx, uint64_t h, std::shared_ptr<Dataset> *out)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->datasets.find(h);
    if (it == ctx->datasets.end()) {
        set_error("unknown dataset %llu", (unsigned long long)h);
        return RS_ERR_NOT_FOUND;
    }
    Dataset &d = *it->second;
    d.last_use = ++ctx->ds_tick;
    if (!d.resident) {                // evicted: rebuild it from the host copy
        rs_status rc = device_guard(ctx);
        if (rc) return rc;
        make_room(ctx, d.dev_bytes, h);
        if ((rc = build_device(d, d.hX.data(), d.hy.data(), RS_MEM_HOST, nullptr))) return rc;
        d.resident = true;
        ctx->ds_resident += d.dev_bytes;
        ++ctx->ds_rebuilds;
    }
    *out = it->second;
    return RS_OK;
}

rs_status set_dataset_budget(Ctx *ctx, uint64_t bytes)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->ds_budget = bytes;
    // spare marks, so that calls that may not create one (the allocation-free entry) find one
    while (bytes && ctx->ds_events.size() < 32) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); break; }
        ctx->ds_events.push_back(e);
    }
    make_room(ctx, 0, 0);
    return RS_OK;
}

rs_status dataset_destroy(Ctx *ctx, uint64_t h, bool force)
{
    std::shared_ptr<Dataset> ds;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->datasets.find(h);
        if (it == ctx->datasets.end()) { set_error("unknown dataset %llu", (unsigned long long)h); return RS_ERR_NOT_FOUND; }
        // another reference than the registry's: a call running on the dataset, or a serving
        // request on it (queued, running or not yet polled) whose kernels would read the freed copy
        if (!force && it->second.use_count() > 1) {
            set_error("dataset %llu is in use: a call on it is running, or a serving request on it has not "
                      "been polled", (unsigned long long)h);
            return RS_ERR_INVALID;
        }
        ds = it->second;
        ctx->datasets.erase(it);
        drop_graphs(ctx, h);          // cached graphs that reference this dataset
        if (ds->resident) ctx->ds_resident -= std::min(ctx->ds_resident, ds->dev_bytes);
        for (cudaEvent_t e : ds->inflight) ctx->ds_events.push_back(e);   // the device wait below covers them
        ds->inflight.clear();
    }
    RS_CUDA(cudaDeviceSynchronize());
    free_device(*ds);
    return RS_OK;
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_dataset_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_label_rank);
    cudaFuncGetAttributes(&fa, k_label_offsets);
    cudaFuncGetAttributes(&fa, k_class_start);
    cudaFuncGetAttributes(&fa, k_label_scatter);
    cudaFuncGetAttributes(&fa, k_transpose_gather);
    cudaFuncGetAttributes(&fa, k_nonfinite);
    cudaFuncGetAttributes(&fa, k_rank_tiles);
    cudaFuncGetAttributes(&fa, k_fill_i32);
}

}  // namespace rs
