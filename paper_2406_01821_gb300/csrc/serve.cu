// Serving: continuous batching of fitness-evaluation requests from many concurrent evolution runs.
//
// rs_submit copies a request's population into pinned host staging and queues it. A scheduler
// thread admits queued requests in arrival order while the memory budget and the request slots
// allow, uploads and packs each one, writes its descriptor into a device table and publishes it in
// the device list of active requests with a claim word (epoch | next unit | units). One persistent
// kernel, kept alive while work arrives, lets each CTA claim a unit -- a 128-sample tile of the
// request's dataset times a group of up to 128 of its sets -- from the active requests in
// round-robin order (processor sharing: a small request does not wait behind a large one), load
// the tile into shared memory, evaluate those sets on it and add exact counts. The CTA finishing
// a request's last unit raises the request's flag in mapped host memory; the scheduler then copies
// the counts back on its own stream and frees the slot and its memory. Requests admitted while
// others run join the rotation at once, so their work overlaps on the device.
//
// Claims are compare-and-swap on the 64-bit claim word, so a CTA holding a stale view of the
// active list can only claim real, unclaimed units. Waits are bounded: an idle persistent kernel
// exits after a short idle limit (the scheduler relaunches it when work is published).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>

#include "eval_core.cuh"
#include "eval_rank.cuh"
#include "rs_internal.cuh"
#include "serve_sched.h"

namespace rs {

namespace {

constexpr int SV = 4;                 // samples per lane
constexpr int SW = 32;                // warps per CTA: one CTA per SM on all but SPARE_SMS SMs
constexpr int SS = 32 * SV;           // samples per tile (unit)
constexpr int SERVE_MAX_F = 256;      // shared x tile [F][128]: 128 KB
constexpr int SERVE_RANK_MAX_F = 128; // rank-coded units: x, ranks, reversed ranks, sorted [F][128]
constexpr int SVS = 8;                // pass-row slots per warp of rank-coded units
constexpr size_t TILE_BYTES = (size_t)SERVE_MAX_F * SS * 4 > (size_t)SERVE_RANK_MAX_F * SS * 10
                                  ? (size_t)SERVE_MAX_F * SS * 4
                                  : (size_t)SERVE_RANK_MAX_F * SS * 10;
constexpr size_t ONES_BYTES = (size_t)SS * 4;   // a row of 1.0: the right side of product conditions
constexpr size_t SERVE_SMEM = TILE_BYTES + (size_t)SW * 64 * 16 + (size_t)SW * SVS * 32 * 4 + ONES_BYTES;
constexpr int MAX_SLOTS = 2048;
constexpr int GROUP_SETS = 128;       // sets per unit: four per warp
constexpr int GROUP_SETS_RANKED = 256;  // rank-coded units: their tile staging is heavier
constexpr int SERVE_RANK_MIN_P = 64;    // smaller requests keep the sign-mask units
constexpr int SPARE_SMS = 4;          // left to the packing kernels of new requests
constexpr uint64_t IDLE_NS = 20000000ull;   // persistent kernel idle limit: 20 ms
// claim word: epoch (24 bits) | next unit (20 bits) | units (20 bits)
constexpr int CW_NEXT = 20, CW_EPOCH = 40;
constexpr unsigned long long CW_MASK = (1ull << 20) - 1;

struct __align__(16) ReqDesc {
    const float *Xt;
    const int32_t *y;
    int64_t N, n_pad;
    int32_t F, K;
    const uint4 *recs;
    const SetInfo *sets;
    const int32_t *order;
    int32_t P, tiles, groups, finite;
    int32_t *correct, *per_class;
    uint64_t epoch;
    const uint8_t *Rk;                  // rank tables (rank-coded units), or null
    const int32_t *last_end;            // [P*K] per-class last rule ends, or null
    int32_t ranked, gsets;              // gsets: sets per unit
    int32_t cat;                        // the records may hold membership tests
};

struct ServeArgs {
    const ReqDesc *table;
    unsigned long long *claims;             // [MAX_SLOTS] claim words
    const volatile int32_t *active;         // [MAX_SLOTS] active slots (a hint; claims decide)
    const volatile int32_t *nactive;
    unsigned int *rr;                       // round-robin cursor
    int32_t *done;                          // [MAX_SLOTS] units finished per slot
    volatile unsigned long long *host_flag; // mapped host memory [MAX_SLOTS]: finished epoch
    const volatile int32_t *stop;           // mapped host memory
};

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// One unit on a dataset with rank tables: stage the tile's x and ranks, build its reversed ranks
// and sorted columns, then walk sets [set0, set1) with the rank-coded evaluator.
__device__ __forceinline__ void serve_unit_ranked(const ReqDesc &d, int tile, int set0, int set1,
                                                  unsigned char *smem, uint4 *st, uint32_t *vr, uint32_t ones_off,
                                                  int *s_next)
{
    using namespace rank;
    const int F = d.F, lane = threadIdx.x & 31;
    unsigned char *xs = smem;                                  // float [F][T]
    unsigned char *rs = xs + (size_t)F * T * 4;                // u8 [F][T], reversed after it
    float *us = reinterpret_cast<float *>(rs + (size_t)F * T * 2);
    const int64_t col0 = (int64_t)tile * T;
    for (int i = threadIdx.x; i < F * (T / 4); i += blockDim.x) {
        const int f = i / (T / 4), c4 = i % (T / 4);
        reinterpret_cast<float4 *>(xs)[i] = *reinterpret_cast<const float4 *>(d.Xt + (int64_t)f * d.n_pad + col0 + 4 * c4);
    }
    for (int i = threadIdx.x; i < F * (T / 16); i += blockDim.x) {
        const int f = i / (T / 16), c16 = i % (T / 16);
        reinterpret_cast<uint4 *>(rs)[i] = *reinterpret_cast<const uint4 *>(d.Rk + (int64_t)f * d.n_pad + col0 + 16 * c16);
    }
    __syncthreads();
    build_tile_tables(reinterpret_cast<const float *>(xs), rs, (uint32_t)F * T, us, F, F);
    const int32_t *yl = d.y + col0 + lane * 4;
    const int64_t t_last = min(col0 + T, d.N) - 1;
    const int kmin = d.y[col0], kmax = d.y[t_last];
    const bool uniform = kmin == kmax;
    const uint32_t claimed0 = class_bytes(yl, -1);
    const uint32_t rev_off = (uint32_t)F * T;
    const uint32_t vr_off = (uint32_t)(reinterpret_cast<unsigned char *>(vr) - rs);
    const unsigned char *rl = rs + lane * 4, *xl = xs + lane * 16;
    __syncthreads();
    while (true) {
        int m = 0;
        if (lane == 0) m = atomicAdd(s_next, 1);
        m = __shfl_sync(FULL, m, 0);
        if (set0 + m >= set1) break;
        const int p = __ldcg(d.order + set0 + m);
        const int4 t = __ldcg(reinterpret_cast<const int4 *>(d.sets + p));
        const int rb = t.x, deflt = t.z;
        // one label k in the tile: records after the set's last rule of class k (default of another
        // class) or of any other class (default k) cannot change its count
        const int nrec = (uniform && d.last_end)
                             ? min(__ldcg(d.last_end + (int64_t)p * d.K + kmin), t.y - t.x)
                             : t.y - t.x;
        uint32_t hit;
        rank::WalkCount wc;                 // not reported by the serving kernel
        if (d.cat)
            hit = uniform ? walk_set<true, SVS, true>(st, vr, vr_off, lane, d.recs, rb, nrec, us, rev_off, F, kmin,
                                                      rl, xl, ones_off, yl, claimed0, deflt, wc)
                          : walk_set<false, SVS, true>(st, vr, vr_off, lane, d.recs, rb, nrec, us, rev_off, F, -2,
                                                       rl, xl, ones_off, yl, claimed0, deflt, wc);
        else
            hit = uniform ? walk_set<true, SVS, false>(st, vr, vr_off, lane, d.recs, rb, nrec, us, rev_off, F, kmin,
                                                       rl, xl, ones_off, yl, claimed0, deflt, wc)
                          : walk_set<false, SVS, false>(st, vr, vr_off, lane, d.recs, rb, nrec, us, rev_off, F, -2,
                                                        rl, xl, ones_off, yl, claimed0, deflt, wc);
        const int hits = __reduce_add_sync(FULL, __popc(hit));
        if (lane == 0 && hits) atomicAdd(&d.correct[p], hits);
        if (d.per_class) {
            if (uniform) {
                if (lane == 0 && hits) atomicAdd(&d.per_class[(int64_t)p * d.K + kmin], hits);
            } else {
                for (int k = kmin; k <= kmax; ++k) {
                    const int c = __reduce_add_sync(FULL, __popc(hit & class_bytes(yl, k)));
                    if (lane == 0 && c) atomicAdd(&d.per_class[(int64_t)p * d.K + k], c);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(SW * 32, 1) k_serve(ServeArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *xs = reinterpret_cast<float *>(smem);                                   // [F][SS]
    uint4 *stage_all = reinterpret_cast<uint4 *>(smem + TILE_BYTES);
    uint32_t *vrows = reinterpret_cast<uint32_t *>(stage_all + SW * 64);            // [SW][SVS][32]
    float *ones = reinterpret_cast<float *>(vrows + SW * SVS * 32);                  // [SS] of 1.0
    const uint32_t ones_off = (uint32_t)(reinterpret_cast<unsigned char *>(ones) - smem);
    if (threadIdx.x < SS) ones[threadIdx.x] = 1.f;                                   // read after a barrier
    __shared__ int s_slot, s_unit, s_next;
    __shared__ ReqDesc sd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *st = stage_all + warp * 64;

    while (true) {
        if (warp == 0) {
            // Warp 0 claims the next unit from the active request with the fewest unclaimed
            // units (the oldest among equals): shortest remaining work first, so a small request
            // is not held behind a large one. The lanes read 32 claim words at a time; the chosen
            // request is taken by compare-and-swap (a lost race rescans).
            int slot = -1, unit = -1;
            uint64_t idle0 = 0;
            while (true) {
                // host-written words: lane 0 reads them, so every lane takes the same branches
                if (__shfl_sync(core::FULL, lane == 0 ? *a.stop : 0, 0)) break;
                const int n = __shfl_sync(core::FULL, lane == 0 ? *a.nactive : 0, 0);
                // best = (remaining units << 11) | list index, minimised over the active list
                uint32_t best = 0xFFFFFFFFu;
                for (int base = 0; base < n; base += 32) {
                    const int i = base + lane;
                    const int sl = i < n ? a.active[i] : -1;
                    uint32_t key = 0xFFFFFFFFu;
                    if (sl >= 0 && sl < MAX_SLOTS) {
                        const unsigned long long w = *reinterpret_cast<volatile unsigned long long *>(a.claims + sl);
                        const uint32_t next = (uint32_t)((w >> CW_NEXT) & CW_MASK), units = (uint32_t)(w & CW_MASK);
                        if (next < units) key = ((units - next) << 11) | (uint32_t)i;
                    }
                    best = min(best, __reduce_min_sync(core::FULL, key));
                }
                if (best != 0xFFFFFFFFu) {
                    const int i = (int)(best & 0x7FFu);
                    int got = -1, sl = -1;
                    if (lane == 0) {
                        sl = a.active[i];
                        if (sl >= 0 && sl < MAX_SLOTS) {
                            unsigned long long w = *reinterpret_cast<volatile unsigned long long *>(a.claims + sl);
                            while (((w >> CW_NEXT) & CW_MASK) < (w & CW_MASK)) {
                                const unsigned long long old = atomicCAS(a.claims + sl, w, w + (1ull << CW_NEXT));
                                if (old == w) { got = (int)((w >> CW_NEXT) & CW_MASK); break; }
                                w = old;
                            }
                        }
                    }
                    got = __shfl_sync(core::FULL, got, 0);
                    if (got >= 0) { slot = __shfl_sync(core::FULL, sl, 0); unit = got; break; }
                    continue;                   // the request filled up meanwhile: rescan
                }
                const uint64_t tn = __shfl_sync(core::FULL, now_ns(), 0);
                if (idle0 == 0) idle0 = tn;
                else if (tn - idle0 > IDLE_NS) break;
                __nanosleep(2000);
            }
            if (lane == 0) {
                s_slot = slot;
                s_unit = unit;
                s_next = 0;
            }
        }
        __syncthreads();
        const int slot = s_slot, unit = s_unit;
        if (slot < 0) return;
        __threadfence();
        // Descriptors and per-request buffers are reused while this kernel lives: read them
        // through L2 (.cg), never from a possibly stale L1 line.
        if (threadIdx.x < (int)(sizeof(ReqDesc) / 16))
            reinterpret_cast<int4 *>(&sd)[threadIdx.x] =
                __ldcg(reinterpret_cast<const int4 *>(a.table + slot) + threadIdx.x);
        __syncthreads();
        const ReqDesc &d = sd;       // shared: keeps the descriptor out of registers
        const int tile = unit / d.groups, grp = unit % d.groups;
        const int set0 = grp * d.gsets, set1 = min(d.P, set0 + d.gsets);
        if (d.ranked) {
            serve_unit_ranked(d, tile, set0, set1, smem, st, vrows + warp * SVS * 32, ones_off, &s_next);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const int fin = atomicAdd(&a.done[slot], 1) + 1;
                if (fin == d.tiles * d.groups) {
                    __threadfence_system();
                    a.host_flag[slot] = d.epoch;
                }
            }
            __syncthreads();
            continue;
        }
        // stage the tile x[0..F)[tile*SS .. +SS) (n_pad is a multiple of 256)
        const int64_t col0 = (int64_t)tile * SS;
        const int nvec = d.F * (SS / 4);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
            const int f = i / (SS / 4), c4 = i % (SS / 4);
            reinterpret_cast<float4 *>(xs)[i] =
                *reinterpret_cast<const float4 *>(d.Xt + (int64_t)f * d.n_pad + col0 + 4 * c4);
        }
        const int64_t n0 = col0 + lane * SV;
        int y[SV];
        bool valid[SV];
#pragma unroll
        for (int v = 0; v < SV; ++v) {
            y[v] = d.y[n0 + v];
            valid[v] = y[v] >= 0;
        }
        const int64_t t_last = min(col0 + SS, d.N) - 1;
        const int kmin = d.y[col0], kmax = d.y[t_last];
        const bool uniform = kmin == kmax;
        __syncthreads();
        const float *xl = xs + lane * SV;
        while (true) {
            int m = 0;
            if (lane == 0) m = atomicAdd(&s_next, 1);
            m = __shfl_sync(core::FULL, m, 0);
            if (set0 + m >= set1) break;
            const int p = __ldcg(d.order + set0 + m);
            SetInfo si;
            {
                const int4 t = __ldcg(reinterpret_cast<const int4 *>(d.sets + p));
                si.rec_begin = t.x; si.rec_end = t.y; si.deflt = t.z; si.cost = t.w;
            }
            bool hit[SV];
            if (d.finite) {
                uint32_t h[SV];
                core::eval_set_sign<SV>(d.recs, si.rec_begin, si.rec_end, st, xl, lane, si.deflt, y,
                                        uniform, kmin, h);
#pragma unroll
                for (int v = 0; v < SV; ++v) hit[v] = h[v] != 0u;
            } else {
                int pred[SV];
                core::eval_set<SV>(d.recs, si.rec_begin, si.rec_end, st, xl, lane, si.deflt, valid, pred);
#pragma unroll
                for (int v = 0; v < SV; ++v) hit[v] = pred[v] == y[v];
            }
            int hits = 0;
#pragma unroll
            for (int v = 0; v < SV; ++v) hits += __popc(__ballot_sync(core::FULL, hit[v]));
            if (lane == 0 && hits) atomicAdd(&d.correct[p], hits);
            if (d.per_class) {
                if (uniform) {
                    if (lane == 0 && hits) atomicAdd(&d.per_class[(int64_t)p * d.K + kmin], hits);
                } else {
                    for (int k = kmin; k <= kmax; ++k) {
                        int c = 0;
#pragma unroll
                        for (int v = 0; v < SV; ++v) c += __popc(__ballot_sync(core::FULL, hit[v] && y[v] == k));
                        if (lane == 0 && c) atomicAdd(&d.per_class[(int64_t)p * d.K + k], c);
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int fin = atomicAdd(&a.done[slot], 1) + 1;
            if (fin == d.tiles * d.groups) {
                __threadfence_system();
                a.host_flag[slot] = d.epoch;
            }
        }
        __syncthreads();
    }
}

__global__ void k_set_claim(unsigned long long *claims, int slot, unsigned long long word)
{
    __threadfence();
    atomicExch(claims + slot, word);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Requests on datasets with rank tables use the rank-coded evaluator when they have enough sets
// to amortise its tile staging (x, ranks and sorted columns, and one search per cut and tile).
// Requests with membership conditions always take them (the sign-mask units have no membership
// test).
bool serve_ranked(const Dataset &ds, int P, bool cat)
{
    return ds.ranked && ds.F <= SERVE_RANK_MAX_F && (P >= SERVE_RANK_MIN_P || cat);
}
int64_t serve_groups(const Dataset &ds, int P, bool cat)
{
    const int g = serve_ranked(ds, P, cat) ? GROUP_SETS_RANKED : GROUP_SETS;
    return std::max<int64_t>(1, (P + g - 1) / g);
}

}  // namespace

// ------------------------------------------------------------------------------ host side

struct Request : sched::Core {
    std::shared_ptr<Dataset> ds;
    int32_t P = 0, R = 0, C = 0, K = 0;
    int32_t kind = 0;                     // RS_KIND_HARD or RS_KIND_SOFT
    float tau = 0.f;                      // soft requests: temperature
    int32_t maxR = 0, maxC = 0;           // soft requests: largest set (rules, conditions)
    void *h_stage = nullptr;              // pinned copy of a host batch's arrays
    void *d_stage = nullptr;              // device copy of a device batch's arrays (same layout)
    size_t stage_bytes = 0, stage_cap = 0, result_cap = 0;   // pinned buffer capacities
    size_t off[11] = {};
    bool cat = false;                     // the batch carries category sets
    void *d_buf = nullptr;
    cudaEvent_t ev = nullptr;
    int32_t *h_correct = nullptr, *h_pc = nullptr;   // pinned results
    int32_t *d_correct = nullptr, *d_pc = nullptr;
    uint32_t *d_status = nullptr;
    uint32_t *h_status = nullptr;
    std::chrono::steady_clock::time_point t_submit, t_admit, t_done;
};

struct Server;

// The device side of the scheduler (serve_sched.h) on CUDA.
struct CudaBackend {
    Server *s = nullptr;
    bool admit(Request &r);
    bool kernel_live();
    void launch_kernel();
    bool units_done(Request &r);
    void start_copy_out(Request &r);
    int copies_done(Request &r);
    void release(Request &r);
};

struct Server {
    Ctx *ctx = nullptr;
    std::mutex mu;                         // scheduler state (held by the scheduler thread while it works)
    std::condition_variable cv_work, cv_done;
    sched::Scheduler<Request, CudaBackend> sch;   // queue, admission, budget, slots (under mu)
    CudaBackend dev;
    std::thread thread;
    bool quit = false;
    // Submissions go through an inbox under their own lock, so rs_submit never waits for the
    // scheduler's device work; the scheduler moves them to `queued`. Lock order: mu, then in_mu.
    std::mutex in_mu;
    std::condition_variable in_cv;
    std::vector<std::shared_ptr<Request>> inbox;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;   // under in_mu
    uint64_t next_ticket = 1;                                       // under in_mu
    std::atomic<bool> quit_flag{false};
    std::atomic<int> fatal_flag{0};
    cudaStream_t sstream = nullptr, kstream = nullptr;
    // request memory: a pool of the server's own that keeps what it has mapped (up to the budget),
    // so that admissions do not wait for the CUDA driver to map memory again
    cudaMemPool_t pool = nullptr;
    cudaEvent_t kevent = nullptr;
    bool kernel_live = false;
    ReqDesc *d_table = nullptr;
    unsigned long long *d_claims = nullptr;
    int32_t *d_active = nullptr;           // [MAX_SLOTS + 1]: list, then its length
    unsigned int *d_rr = nullptr;
    std::vector<int32_t> h_active;         // host copy of the active list
    cudaStream_t cstream = nullptr;        // completion copies
    int32_t *d_done = nullptr;
    unsigned long long *h_flag = nullptr;
    int32_t *h_stop = nullptr;
    unsigned long long published = 0;
    rs_status fatal = RS_OK;
    int grid = 0;
    size_t smem = 0;
    // pinned host buffers of finished requests, reused by new ones (pinning memory is slow and
    // can stall other CUDA calls): capacity -> buffer
    std::mutex pool_mu;
    std::multimap<size_t, void *> pinned_free;
    cudaStream_t ustream = nullptr;            // copies of device batches at submission
    std::mutex up_mu;
    std::vector<cudaEvent_t> event_pool;       // completion events of finished requests, for reuse
    char *arena = nullptr;                     // pinned staging arena (PINNED_ARENA_BYTES)
    std::map<size_t, size_t> arena_free;       // free blocks of the arena: offset -> bytes
};

static rs_status server_start(Ctx *ctx, Server **out);
// Pinned staging pool -------------------------------------------------------------------------

// Staging comes first from one pinned arena allocated when the server starts, carved first-fit in
// 4 KiB units with a coalescing free list, so that rs_submit does not pin memory (pinning takes
// milliseconds and holds up other CUDA calls); a request that does not fit falls back to pinned
// buffers of its own, pooled by size.
constexpr size_t PINNED_ARENA_BYTES = 256ull << 20, PINNED_UNIT = 4096;

static void *arena_get(Server *s, size_t bytes, size_t *cap)
{
    const size_t need = (bytes + PINNED_UNIT - 1) / PINNED_UNIT * PINNED_UNIT;
    for (auto it = s->arena_free.begin(); it != s->arena_free.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, left = it->second - need;
        s->arena_free.erase(it);
        if (left) s->arena_free.emplace(off + need, left);
        *cap = need;
        return s->arena + off;
    }
    return nullptr;
}

static bool arena_put(Server *s, void *p, size_t cap)
{
    if (!s->arena || (char *)p < s->arena || (char *)p >= s->arena + PINNED_ARENA_BYTES) return false;
    size_t off = (size_t)((char *)p - s->arena), len = cap;
    auto next = s->arena_free.lower_bound(off);
    if (next != s->arena_free.end() && next->first == off + len) {     // merge with the block after
        len += next->second;
        next = s->arena_free.erase(next);
    }
    if (next != s->arena_free.begin()) {                                 // and with the one before
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            off = prev->first;
            len += prev->second;
            s->arena_free.erase(prev);
        }
    }
    s->arena_free.emplace(off, len);
    return true;
}

static void *pinned_get(Server *s, size_t bytes, size_t *cap)
{
    {
        std::lock_guard<std::mutex> lk(s->pool_mu);
        if (s->arena)
            if (void *p = arena_get(s, bytes, cap)) return p;
        auto it = s->pinned_free.lower_bound(bytes);
        if (it != s->pinned_free.end() && it->first <= 4 * bytes + 65536) {
            void *p = it->second;
            *cap = it->first;
            s->pinned_free.erase(it);
            return p;
        }
    }
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    void *p = nullptr;
    if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    *cap = c;
    return p;
}

static void pinned_put(Server *s, void *p, size_t cap)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(s->pool_mu);
    if (arena_put(s, p, cap)) return;
    s->pinned_free.emplace(cap, p);
}

static void server_loop(Server *s);

static rs_status server_get(Ctx *ctx, Server **out)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->server) {
        rs_status rc = server_start(ctx, &ctx->server);
        if (rc) return rc;
    }
    *out = ctx->server;
    return RS_OK;
}

static rs_status server_start(Ctx *ctx, Server **out)
{
    auto *s = new Server();
    s->ctx = ctx;
    auto fail = [&](cudaError_t e, const char *w) {
        rs_status rc = cuda_fail(e, w);
        delete s;
        return rc;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s->sstream, cudaStreamNonBlocking))) return fail(e, "stream");
    if ((e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking))) return fail(e, "stream");
    if ((e = cudaEventCreateWithFlags(&s->kevent, cudaEventDisableTiming))) return fail(e, "event");
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        if ((e = cudaMemPoolCreate(&s->pool, &props))) return fail(e, "memory pool");
        uint64_t keep = ctx->budget;
        if ((e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep)))
            return fail(e, "pool attribute");
    }
    if ((e = cudaMalloc(&s->d_table, sizeof(ReqDesc) * MAX_SLOTS))) return fail(e, "table");
    if ((e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking))) return fail(e, "stream");
    if ((e = cudaStreamCreateWithFlags(&s->ustream, cudaStreamNonBlocking))) return fail(e, "stream");
    if ((e = cudaMalloc(&s->d_claims, sizeof(unsigned long long) * MAX_SLOTS))) return fail(e, "claims");
    if ((e = cudaMemset(s->d_claims, 0, sizeof(unsigned long long) * MAX_SLOTS))) return fail(e, "claims");
    if ((e = cudaMalloc(&s->d_active, sizeof(int32_t) * (MAX_SLOTS + 1)))) return fail(e, "active");
    if ((e = cudaMemset(s->d_active, 0, sizeof(int32_t) * (MAX_SLOTS + 1)))) return fail(e, "active");
    if ((e = cudaMalloc(&s->d_rr, sizeof(unsigned int)))) return fail(e, "rr");
    if ((e = cudaMemset(s->d_rr, 0, sizeof(unsigned int)))) return fail(e, "rr");
    if ((e = cudaMalloc(&s->d_done, sizeof(int32_t) * MAX_SLOTS))) return fail(e, "done");
    if ((e = cudaHostAlloc(&s->h_flag, sizeof(unsigned long long) * MAX_SLOTS, cudaHostAllocMapped))) return fail(e, "flags");
    if ((e = cudaHostAlloc(&s->h_stop, sizeof(int32_t), cudaHostAllocMapped))) return fail(e, "stop");
    // the staging arena (without it, staging falls back to buffers of their own)
    if (cudaHostAlloc(&s->arena, PINNED_ARENA_BYTES, cudaHostAllocDefault) == cudaSuccess)
        s->arena_free.emplace(0, PINNED_ARENA_BYTES);
    else {
        cudaGetLastError();
        s->arena = nullptr;
    }
    memset(s->h_flag, 0, sizeof(unsigned long long) * MAX_SLOTS);
    *s->h_stop = 0;
    s->sch.init(ctx->budget, MAX_SLOTS);
    s->dev.s = s;
    s->smem = SERVE_SMEM;
    if ((e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem)))
        return fail(e, "k_serve attribute");
    // one CTA per SM: the rest of each SM stays available to the packing kernels of new requests
    s->grid = std::max(1, ctx->sm_count - SPARE_SMS);
    s->thread = std::thread(server_loop, s);
    *out = s;
    return RS_OK;
}

void server_shutdown(Ctx *ctx)
{
    Server *s = ctx->server;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->quit = true;
    }
    s->quit_flag = true;
    {
        std::lock_guard<std::mutex> il(s->in_mu);
    }
    s->in_cv.notify_all();
    s->cv_work.notify_all();
    if (s->thread.joinable()) s->thread.join();
    *(volatile int32_t *)s->h_stop = 1;
    cudaStreamSynchronize(s->kstream);
    cudaStreamSynchronize(s->sstream);
    cudaStreamSynchronize(s->cstream);
    cudaStreamSynchronize(s->ustream);
    for (auto &kv : s->all) {
        Request &r = *kv.second;
        if (r.d_stage) cudaFree(r.d_stage);
        r.d_stage = nullptr;
        if (r.h_stage) cudaFreeHost(r.h_stage);
        if (r.h_correct) cudaFreeHost(r.h_correct);
        r.h_stage = nullptr;
        r.h_correct = nullptr;
        if (r.d_buf) cudaFree(r.d_buf);
        if (r.ev) cudaEventDestroy(r.ev);
    }
    cudaFree(s->d_table);
    cudaFree(s->d_claims);
    cudaFree(s->d_active);
    cudaFree(s->d_rr);
    cudaFree(s->d_done);
    for (auto &kv : s->pinned_free) cudaFreeHost(kv.second);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    if (s->arena) cudaFreeHost(s->arena);
    cudaFreeHost(s->h_flag);
    cudaFreeHost(s->h_stop);
    cudaEventDestroy(s->kevent);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    cudaStreamDestroy(s->sstream);
    cudaStreamDestroy(s->kstream);
    cudaStreamDestroy(s->cstream);
    cudaStreamDestroy(s->ustream);
    delete s;
    ctx->server = nullptr;
}

static size_t request_device_bytes(int64_t P, int64_t R, int64_t C, int64_t K, bool cat)
{
    size_t b = 0;
    b += align256(4 * (P + 1)) + align256(4 * (R + 1)) + align256(4 * R) + align256(4 * P);
    b += 3 * align256(4 * C) + align256(C) + 3 * align256(4 * C);       // condition arrays
    if (cat) b += align256(8 * C);                                       // category sets
    b += align256(16 * std::max<int64_t>(C, 1)) + align256(16 * std::max<int64_t>(P, 1)) +
         align256(4 * std::max<int64_t>(P, 1));                          // records, sets, order
    b += align256(4 * P) + align256(4 * P * K) + 256;                   // outputs, status
    if (K <= LAST_END_MAX_K) b += align256(4 * P * K);                  // per-class last rule ends
    return b;
}

rs_status submit_impl(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t kind, float tau, uint64_t *ticket)
{
    if (!b || !ticket) { set_error("NULL batch or ticket"); return RS_ERR_INVALID; }
    if (kind != RS_KIND_HARD && kind != RS_KIND_SOFT) { set_error("unknown request kind %d", kind); return RS_ERR_INVALID; }
    if (kind == RS_KIND_SOFT && !(tau > 0.f)) { set_error("tau must be positive"); return RS_ERR_INVALID; }
    if (b->P < 0 || b->R < 0 || b->C < 0 || (b->mem != RS_MEM_HOST && b->mem != RS_MEM_DEVICE)) {
        set_error("bad batch");
        return RS_ERR_INVALID;
    }
    std::shared_ptr<Dataset> ds;
    if (rs_status urc = use_dataset(ctx, ds_h, &ds)) return urc;
    if (kind == RS_KIND_HARD && ds->F > SERVE_MAX_F) {
        set_error("hard requests are served on datasets of at most %d features", SERVE_MAX_F);
        return RS_ERR_UNSUPPORTED;
    }
    const bool cat = b->cond_set != nullptr;
    if (kind == RS_KIND_HARD && cat && !serve_ranked(*ds, b->P, true)) {
        set_error("hard requests with membership conditions are served on finite datasets of at most %d "
                  "features", SERVE_RANK_MAX_F);
        return RS_ERR_UNSUPPORTED;
    }
    rs_status rc = device_guard(ctx);
    if (rc) return rc;
    Server *s = nullptr;
    if ((rc = server_get(ctx, &s))) return rc;
    auto r = std::make_shared<Request>();
    r->ds = ds;
    r->P = b->P; r->R = b->R; r->C = b->C; r->K = ds->K; r->kind = kind; r->tau = tau; r->cat = cat;
    r->needs_slot = kind == RS_KIND_HARD;     // soft requests run as their own kernels
    r->device_bytes = request_device_bytes(b->P, b->R, b->C, ds->K, cat);
    if (r->device_bytes > ctx->budget) {
        set_error("request needs %zu bytes of device memory; the budget is %llu", r->device_bytes,
                  (unsigned long long)ctx->budget);
        return RS_ERR_TOO_LARGE;
    }
    const int64_t units = ((ds->N + SS - 1) / SS) * serve_groups(*ds, b->P, cat);
    if (kind == RS_KIND_HARD && units > (int64_t)CW_MASK) {
        set_error("request too large to serve (%lld work units)", (long long)units);
        return RS_ERR_TOO_LARGE;
    }
    // copy the batch into pinned staging: the caller may free its arrays on return
    const size_t P = b->P, R = b->R, C = b->C;
    const size_t sz[11] = {4 * (P + 1), 4 * (R + 1), 4 * R, 4 * P, 4 * C, 4 * C, C, 4 * C, 4 * C, 4 * C,
                           cat ? 8 * C : 0};
    const void *src[11] = {b->set_rule_off, b->rule_cond_off, b->rule_class, b->set_default,
                           b->cond_f, b->cond_g, b->cond_op, b->cond_a, b->cond_b, b->cond_t, b->cond_set};
    size_t tot = 0;
    for (int i = 0; i < 11; ++i) { r->off[i] = tot; tot = align256(tot + sz[i]); }
    r->stage_bytes = tot;
    for (int i = 0; i < 11; ++i)
        if (sz[i] && !src[i]) { set_error("NULL batch array"); return RS_ERR_INVALID; }
    if (b->mem == RS_MEM_HOST) {
        // a host batch: copied into pinned staging, uploaded at admission
        r->h_stage = pinned_get(s, std::max<size_t>(tot, 256), &r->stage_cap);
        if (!r->h_stage) { set_error("pinned host memory exhausted"); return RS_ERR_OOM; }
        for (int i = 0; i < 11; ++i)
            if (sz[i]) memcpy((char *)r->h_stage + r->off[i], src[i], sz[i]);
    } else {
        // a device batch: copied device to device into staging of its own (no host round trip),
        // finished before rs_submit returns so that the caller may free its arrays
        std::lock_guard<std::mutex> ul(s->up_mu);
        cudaError_t e = dev_alloc_async(&r->d_stage, std::max<size_t>(tot, 256), s->ustream);
        for (int i = 0; i < 11 && e == cudaSuccess; ++i)
            if (sz[i]) e = cudaMemcpyAsync((char *)r->d_stage + r->off[i], src[i], sz[i], cudaMemcpyDeviceToDevice,
                                           s->ustream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->ustream);
        if (e != cudaSuccess) {
            if (r->d_stage) { cudaFreeAsync(r->d_stage, s->ustream); cudaStreamSynchronize(s->ustream); }
            r->d_stage = nullptr;
            return cuda_fail(e, "rs_submit copy");
        }
    }
    if (kind == RS_KIND_SOFT) {
        // the largest set bounds the soft kernels' shared memory; malformed offsets are left to
        // the device checks, which see the same arrays
        std::vector<int32_t> offs;
        const int32_t *sro, *rco;
        if (r->h_stage) {
            sro = (const int32_t *)((char *)r->h_stage + r->off[0]);
            rco = (const int32_t *)((char *)r->h_stage + r->off[1]);
        } else {
            offs.resize(P + 1 + R + 1);
            const cudaError_t e1 = cudaMemcpy(offs.data(), b->set_rule_off, 4 * (P + 1), cudaMemcpyDeviceToHost);
            const cudaError_t e2 = cudaMemcpy(offs.data() + P + 1, b->rule_cond_off, 4 * (R + 1),
                                              cudaMemcpyDeviceToHost);
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                cudaFree(r->d_stage);
                r->d_stage = nullptr;
                return cuda_fail(e1 != cudaSuccess ? e1 : e2, "rs_submit_soft offsets");
            }
            sro = offs.data();
            rco = offs.data() + P + 1;
        }
        int32_t mr = 1, mc = 1;
        for (size_t p = 0; p < P; ++p) {
            const int32_t rb = sro[p], re = sro[p + 1];
            if (rb < 0 || re < rb || (size_t)re > R) continue;
            mr = std::max(mr, re - rb);
            const int32_t cb = rco[rb], ce = rco[re];
            if (cb >= 0 && ce >= cb && (size_t)ce <= C) mc = std::max(mc, ce - cb);
        }
        r->maxR = mr;
        r->maxC = mc;
    }
    r->h_correct = (int32_t *)pinned_get(
        s, align256(4 * std::max<size_t>(P, 1)) + 4 * std::max<size_t>(P * r->K, 1) + 256, &r->result_cap);
    auto release_stage = [&] {
        pinned_put(s, r->h_stage, r->stage_cap);
        r->h_stage = nullptr;
        if (r->d_stage) cudaFree(r->d_stage);
        r->d_stage = nullptr;
    };
    if (!r->h_correct) {
        release_stage();
        set_error("pinned host memory exhausted");
        return RS_ERR_OOM;
    }
    r->h_pc = (int32_t *)((char *)r->h_correct + align256(4 * std::max<size_t>(P, 1)));
    r->h_status = (uint32_t *)((char *)r->h_pc + 4 * std::max<size_t>(P * r->K, 1));
    *r->h_status = 0;
    {   // a pooled event: rs_submit makes no CUDA call for host batches once the pool is warm
        std::lock_guard<std::mutex> lk(s->pool_mu);
        if (!s->event_pool.empty()) {
            r->ev = s->event_pool.back();
            s->event_pool.pop_back();
        }
    }
    if (cudaError_t e = r->ev ? cudaSuccess : cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming)) {
        release_stage();
        pinned_put(s, r->h_correct, r->result_cap);
        r->h_correct = nullptr;
        return cuda_fail(e, "cudaEventCreate");
    }
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> il(s->in_mu);
        if (s->fatal_flag.load()) {
            release_stage();
            pinned_put(s, r->h_correct, r->result_cap);
            r->h_correct = nullptr;
            cudaEventDestroy(r->ev);
            r->ev = nullptr;
            set_error("serving stopped after a device error");
            return (rs_status)s->fatal_flag.load();
        }
        r->ticket = s->next_ticket++;
        s->inbox.push_back(r);
        s->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    s->in_cv.notify_one();
    return RS_OK;
}

// Scheduler-thread helpers (called with s->mu held) ------------------------------------------

static void push_active(Server *s)
{
    // list, then its length, in one copy (pageable source: staged before the call returns)
    std::vector<int32_t> buf(s->h_active);
    buf.resize(MAX_SLOTS + 1, -1);
    buf[MAX_SLOTS] = (int32_t)s->h_active.size();
    cudaMemcpyAsync(s->d_active, buf.data(), sizeof(int32_t) * (MAX_SLOTS + 1), cudaMemcpyHostToDevice,
                    s->sstream);
}

// The batch arrays into the request's device memory: from pinned staging (host batches, one copy
// per array) or in one device-to-device copy from the device staging (device batches), which is
// then released.
static void upload_batch(Server *s, Request &r, char *base)
{
    if (r.d_stage) {
        cudaMemcpyAsync(base, r.d_stage, r.stage_bytes, cudaMemcpyDeviceToDevice, s->sstream);
        cudaFreeAsync(r.d_stage, s->sstream);
        r.d_stage = nullptr;
        return;
    }
    for (int i = 0; i < 11; ++i)
        if ((i + 1 < 11 ? r.off[i + 1] : r.stage_bytes) > r.off[i])
            cudaMemcpyAsync(base + r.off[i], (char *)r.h_stage + r.off[i],
                            (i + 1 < 11 ? r.off[i + 1] : r.stage_bytes) - r.off[i], cudaMemcpyHostToDevice,
                            s->sstream);
}

// A soft-loss request runs as its own kernels on the staging stream (next to the persistent
// kernel): upload, the soft forward, and the copy of the per-set losses and the status word.
static bool admit_soft(Server *s, Request &r)
{
    char *base = nullptr;
    if (dev_alloc_pool_async(&base, r.device_bytes, s->pool, s->sstream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    r.d_buf = base;
    r.t_admit = std::chrono::steady_clock::now();
    upload_batch(s, r, base);
    char *p = base + r.stage_bytes;
    SoftArgs a{};
    a.b.P = r.P; a.b.R = r.R; a.b.C = r.C;
    a.b.set_rule_off = (int32_t *)(base + r.off[0]); a.b.rule_cond_off = (int32_t *)(base + r.off[1]);
    a.b.rule_class = (int32_t *)(base + r.off[2]); a.b.set_default = (int32_t *)(base + r.off[3]);
    a.b.cond_f = (int32_t *)(base + r.off[4]); a.b.cond_g = (int32_t *)(base + r.off[5]);
    a.b.cond_op = (int8_t *)(base + r.off[6]); a.b.cond_a = (float *)(base + r.off[7]);
    a.b.cond_b = (float *)(base + r.off[8]); a.b.cond_t = (float *)(base + r.off[9]);
    a.b.cond_set = r.cat ? (uint64_t *)(base + r.off[10]) : nullptr;
    float *d_loss = (float *)p; p += align256(4 * std::max<size_t>(r.P, 1));
    r.d_status = (uint32_t *)p;
    a.Xt = r.ds->Xt; a.y = r.ds->y; a.perm = r.ds->perm; a.N = r.ds->N; a.n_pad = r.ds->n_pad;
    a.F = r.ds->F; a.K = r.K; a.tau = r.tau; a.loss = d_loss; a.status = r.d_status;
    cudaMemsetAsync(r.d_status, 0, 4, s->sstream);
    if (r.P > 0) soft_step_known(s->ctx, a, r.maxR, r.maxC, s->sstream);
    cudaGetLastError();
    if (r.P > 0) cudaMemcpyAsync(r.h_correct, d_loss, 4 * (size_t)r.P, cudaMemcpyDeviceToHost, s->sstream);
    cudaMemcpyAsync(r.h_status, r.d_status, 4, cudaMemcpyDeviceToHost, s->sstream);
    cudaEventRecord(r.ev, s->sstream);
    r.state = sched::COPYING;
    return true;
}

// Admission of a request the scheduler let through (budget and, for hard requests, a slot already
// checked; r.slot set): device memory, upload, packing, descriptor and claim word.
bool CudaBackend::admit(Request &r)
{
    if (r.kind == RS_KIND_SOFT) return admit_soft(s, r);
    const int64_t tiles = (r.ds->N + SS - 1) / SS;
    const int64_t groups = serve_groups(*r.ds, r.P, r.cat);
    char *base = nullptr;
    if (dev_alloc_pool_async(&base, r.device_bytes, s->pool, s->sstream) != cudaSuccess) {
        cudaGetLastError();
        return false;                      // retry later, when memory is back
    }
    r.d_buf = base;
    r.t_admit = std::chrono::steady_clock::now();
    // batch arrays
    upload_batch(s, r, base);
    char *p = base + r.stage_bytes;
    BatchDev bd{};
    bd.P = r.P; bd.R = r.R; bd.C = r.C;
    bd.set_rule_off = (int32_t *)(base + r.off[0]); bd.rule_cond_off = (int32_t *)(base + r.off[1]);
    bd.rule_class = (int32_t *)(base + r.off[2]); bd.set_default = (int32_t *)(base + r.off[3]);
    bd.cond_f = (int32_t *)(base + r.off[4]); bd.cond_g = (int32_t *)(base + r.off[5]);
    bd.cond_op = (int8_t *)(base + r.off[6]); bd.cond_a = (float *)(base + r.off[7]);
    bd.cond_b = (float *)(base + r.off[8]); bd.cond_t = (float *)(base + r.off[9]);
    bd.cond_set = r.cat ? (uint64_t *)(base + r.off[10]) : nullptr;
    PackOut po;
    po.recs = (Rec *)p; p += align256(16 * std::max(r.C, 1));
    po.sets = (SetInfo *)p; p += align256(16 * std::max(r.P, 1));
    po.order = (int32_t *)p; p += align256(4 * std::max(r.P, 1));
    r.d_correct = (int32_t *)p; p += align256(4 * r.P);
    r.d_pc = (int32_t *)p; p += align256(4 * (size_t)r.P * r.K);
    r.d_status = (uint32_t *)p;
    p += 256;
    po.status = r.d_status;
    if (r.K <= LAST_END_MAX_K) po.last_end = (int32_t *)p;
    po.correct = r.d_correct;     // zeroed by the packing
    po.per_class = r.d_pc;
    cudaMemsetAsync(r.d_status, 0, 4, s->sstream);
    const bool finite = r.ds->finite;
    const bool ranked = serve_ranked(*r.ds, r.P, r.cat);
    count_launch(s->ctx, launch_pack(bd, r.ds->F, r.K, SS, ranked ? 5 : (finite ? 4 : 2), po, s->sstream));
    ReqDesc d{};
    d.Xt = r.ds->Xt; d.y = r.ds->y; d.N = r.ds->N; d.n_pad = r.ds->n_pad; d.F = r.ds->F; d.K = r.K;
    d.recs = reinterpret_cast<const uint4 *>(po.recs); d.sets = po.sets; d.order = po.order;
    d.P = r.P; d.tiles = (int32_t)tiles; d.groups = (int32_t)groups; d.finite = finite ? 1 : 0;
    d.correct = r.d_correct; d.per_class = r.d_pc;
    d.epoch = r.ticket & 0xFFFFFFull;
    d.Rk = ranked ? r.ds->Rk : nullptr;
    d.ranked = ranked ? 1 : 0;
    d.gsets = ranked ? GROUP_SETS_RANKED : GROUP_SETS;
    d.last_end = po.last_end;
    d.cat = r.cat ? 1 : 0;
    // a copy from pageable memory is staged before the call returns, so `d` may go out of scope
    cudaMemcpyAsync(&s->d_table[r.slot], &d, sizeof(d), cudaMemcpyHostToDevice, s->sstream);
    cudaMemsetAsync(&s->d_done[r.slot], 0, 4, s->sstream);
    const unsigned long long units = (unsigned long long)(tiles * groups);
    if (units > 0 && r.P > 0) {
        // the descriptor is in place before the claim word opens the request to the kernel
        const unsigned long long word = (d.epoch << CW_EPOCH) | units;
        k_set_claim<<<1, 1, 0, s->sstream>>>(s->d_claims, r.slot, word);
        count_launch(s->ctx);
        s->h_active.push_back(r.slot);
        push_active(s);
        s->published += units;
        r.state = sched::RUNNING;
    } else {                   // nothing to evaluate: results are the zeros just written
        cudaMemcpyAsync(r.h_correct, r.d_correct, 4 * (size_t)r.P, cudaMemcpyDeviceToHost, s->sstream);
        cudaMemcpyAsync(r.h_status, r.d_status, 4, cudaMemcpyDeviceToHost, s->sstream);
        r.state = sched::COPYING;
    }
    cudaEventRecord(r.ev, s->sstream);
    return true;
}

bool CudaBackend::kernel_live()
{
    if (!s->kernel_live) return false;
    if (cudaEventQuery(s->kevent) == cudaSuccess) s->kernel_live = false;    // it left after its idle limit
    else cudaGetLastError();
    return s->kernel_live;
}

void CudaBackend::launch_kernel()
{
    // the descriptors and ring entries must be in place before the kernel starts
    cudaStreamWaitEvent(s->kstream, s->sch.active.back()->ev, 0);
    ServeArgs a{s->d_table, s->d_claims, s->d_active, s->d_active + MAX_SLOTS, s->d_rr, s->d_done,
                (volatile unsigned long long *)s->h_flag, (volatile int32_t *)s->h_stop};
    k_serve<<<s->grid, SW * 32, s->smem, s->kstream>>>(a);
    cudaEventRecord(s->kevent, s->kstream);
    count_launch(s->ctx);
    s->kernel_live = true;
}

bool CudaBackend::units_done(Request &r)
{
    return ((volatile unsigned long long *)s->h_flag)[r.slot] == (r.ticket & 0xFFFFFFull);
}

void CudaBackend::start_copy_out(Request &r)
{
    cudaMemcpyAsync(r.h_correct, r.d_correct, 4 * (size_t)r.P, cudaMemcpyDeviceToHost, s->cstream);
    cudaMemcpyAsync(r.h_pc, r.d_pc, 4 * (size_t)r.P * r.K, cudaMemcpyDeviceToHost, s->cstream);
    cudaMemcpyAsync(r.h_status, r.d_status, 4, cudaMemcpyDeviceToHost, s->cstream);
    cudaEventRecord(r.ev, s->cstream);
    s->h_active.erase(std::remove(s->h_active.begin(), s->h_active.end(), r.slot), s->h_active.end());
    push_active(s);
}

int CudaBackend::copies_done(Request &r)
{
    const cudaError_t q = cudaEventQuery(r.ev);
    if (q == cudaSuccess) return 1;
    if (q == cudaErrorNotReady) return 0;
    s->fatal = cuda_fail(q, "serving");
    s->fatal_flag = (int)s->fatal;
    return (int)s->fatal;
}

void CudaBackend::release(Request &r)
{
    r.t_done = std::chrono::steady_clock::now();
    r.status = *r.h_status ? RS_ERR_INVALID : RS_OK;
    cudaFreeAsync(r.d_buf, s->sstream);   // the copies out have completed
    r.d_buf = nullptr;
    // the batch's pinned staging went to the device before the request's work ran (stream order):
    // it returns to the pool now, not at the poll, so that requests whose results wait to be
    // polled do not hold the staging arena
    pinned_put(s, r.h_stage, r.stage_cap);
    r.h_stage = nullptr;
}

static void server_loop(Server *s)
{
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        {
            std::lock_guard<std::mutex> il(s->in_mu);
            for (auto &r : s->inbox) s->sch.queued.push_back(r);
            s->inbox.clear();
        }
        if (s->quit && s->sch.idle()) break;
        const bool progress = s->sch.step(s->dev);
        if (progress) s->cv_done.notify_all();
        if (!progress) {
            if (s->sch.idle()) {
                if (s->quit) break;
                lk.unlock();
                {
                    std::unique_lock<std::mutex> il(s->in_mu);
                    s->in_cv.wait_for(il, std::chrono::milliseconds(50),
                                      [&] { return !s->inbox.empty() || s->quit_flag.load(); });
                }
                lk.lock();
            } else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            }
        }
    }
}

rs_status poll_impl(Ctx *ctx, uint64_t ticket, int64_t timeout_us, int32_t kind, int32_t *correct,
                    int32_t *per_class, float *loss, rs_ticket_info *info)
{
    Server *s = ctx->server;
    if (!s) { set_error("no request was submitted"); return RS_ERR_NOT_FOUND; }
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> il(s->in_mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return RS_ERR_NOT_FOUND; }
        r = it->second;
    }
    if (r->kind != kind) {
        set_error("ticket %llu is a %s request", (unsigned long long)ticket, r->kind == RS_KIND_SOFT ? "soft" : "hard");
        return RS_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] { return r->state >= sched::DONE; };
    if (!done()) {
        if (timeout_us <= 0) return RS_PENDING;
        if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) return RS_PENDING;
    }
    if (info) {
        info->submit_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_submit.time_since_epoch()).count();
        info->admit_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_admit.time_since_epoch()).count();
        info->done_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_done.time_since_epoch()).count();
    }
    rs_status rc = r->status;
    if (rc == RS_OK) {
        if (correct) memcpy(correct, r->h_correct, 4 * (size_t)r->P);
        if (per_class) memcpy(per_class, r->h_pc, 4 * (size_t)r->P * r->K);
        if (loss) memcpy(loss, r->h_correct, 4 * (size_t)r->P);
    } else if (rc == RS_ERR_CANCELLED) {
        set_error("request cancelled");
    } else {
        set_error("request rejected by the device checks (malformed batch)");
    }
    if (r->state == sched::RELEASED) {   // another poll took the results first
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return RS_ERR_NOT_FOUND;
    }
    // results are released at the first successful poll
    if (r->d_stage) {                // cancelled before admission
        cudaFree(r->d_stage);
        r->d_stage = nullptr;
    }
    pinned_put(s, r->h_stage, r->stage_cap);
    pinned_put(s, r->h_correct, r->result_cap);
    if (r->ev) {
        std::lock_guard<std::mutex> pl(s->pool_mu);
        s->event_pool.push_back(r->ev);
    }
    r->h_stage = nullptr; r->h_correct = nullptr; r->ev = nullptr;
    r->state = sched::RELEASED;
    lk.unlock();
    {
        std::lock_guard<std::mutex> il(s->in_mu);
        s->all.erase(ticket);
    }
    return rc;
}

rs_status cancel(Ctx *ctx, uint64_t ticket)
{
    Server *s = ctx->server;
    if (!s) return RS_ERR_NOT_FOUND;
    std::shared_ptr<Request> rp;
    {
        std::lock_guard<std::mutex> il(s->in_mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return RS_ERR_NOT_FOUND;
        rp = it->second;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Request &r = *rp;
    if (!s->sch.cancel(r, RS_ERR_CANCELLED)) { set_error("request already admitted"); return RS_ERR_INVALID; }
    r.t_done = std::chrono::steady_clock::now();
    s->cv_done.notify_all();
    return RS_OK;
}

rs_status server_stats(Ctx *ctx, rs_serving_stats *out)
{
    Server *s = ctx->server;
    memset(out, 0, sizeof(*out));
    if (!s) return RS_OK;
    std::lock_guard<std::mutex> lk(s->mu);
    std::lock_guard<std::mutex> il(s->in_mu);
    out->queued = (int64_t)(s->sch.queued.size() + s->inbox.size());
    out->active = (int64_t)s->sch.active.size();
    out->device_bytes_in_use = s->sch.used;
    out->units_published = s->published;
    out->kernel_launches = s->sch.launches;
    return RS_OK;
}

rs_status submit(Ctx *ctx, uint64_t ds_h, const rs_batch *b, int32_t kind, uint64_t *ticket)
{
    if (kind == RS_KIND_SOFT) {
        set_error("soft requests carry a temperature: use rs_submit_soft");
        return RS_ERR_INVALID;
    }
    return submit_impl(ctx, ds_h, b, kind, 0.f, ticket);
}
rs_status submit_soft(Ctx *ctx, uint64_t ds_h, const rs_batch *b, float tau, uint64_t *ticket)
{
    return submit_impl(ctx, ds_h, b, RS_KIND_SOFT, tau, ticket);
}
rs_status poll(Ctx *ctx, uint64_t ticket, int64_t timeout_us, int32_t *correct, int32_t *per_class,
               rs_ticket_info *info)
{
    return poll_impl(ctx, ticket, timeout_us, RS_KIND_HARD, correct, per_class, nullptr, info);
}
rs_status poll_soft(Ctx *ctx, uint64_t ticket, int64_t timeout_us, float *loss, rs_ticket_info *info)
{
    return poll_impl(ctx, ticket, timeout_us, RS_KIND_SOFT, nullptr, nullptr, loss, info);
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_serve_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_serve);
    cudaFuncGetAttributes(&fa, k_set_claim);
}

}  // namespace rs
