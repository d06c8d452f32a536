// The hard evaluator: exact first-fire evaluation of a population of ordered rule sets.
//
// Grid: (sample tile, set group). A CTA stages the feature-major tile x[0..F)[S samples] of the
// label-grouped dataset into shared memory with one 2-D TMA load per 256 features, then its
// warps pull sets of the group from a shared counter (most expensive first). A warp evaluates a
// whole set on the tile: lane l owns samples l*V .. l*V+V-1 and keeps, per sample, a "rule still
// alive" flag (AND of the rule's conditions so far, seeded with "not yet claimed") and the
// predicted class. Condition records stream through a per-warp shared-memory stage (32 records,
// next chunk prefetched into registers) and are read as warp-uniform broadcasts. A rule whose
// alive flags are all false across the warp skips its remaining conditions; a set whose samples
// are all claimed stops early. At the end of a set the per-sample hits are bit-sliced with
// __ballot_sync, popc-reduced and added to the set's int32 counters with one atomic per warp.
//
// Compiled without FMA contraction; every product is an explicit round-to-nearest multiply and
// every compare is an IEEE ordered compare, so results equal the plain definition bit for bit.
#include "rs_internal.cuh"
#include "tma.cuh"

namespace rs {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint64_t TMA_WAIT_LIMIT_NS = 2000000000ull;   // 2 s

template <int V>
__device__ __forceinline__ void load_v(const float *p, float (&x)[V])
{
    if constexpr (V == 1) {
        x[0] = p[0];
    } else if constexpr (V == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        x[0] = t.x; x[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < V; k += 4) {
            float4 t = *reinterpret_cast<const float4 *>(p + k);
            x[k] = t.x; x[k + 1] = t.y; x[k + 2] = t.z; x[k + 3] = t.w;
        }
    }
}

__device__ __forceinline__ uint4 ldg_rec(const Rec *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// GM: features are read from global memory (x[f][n] at Xt[f * n_pad + n]) instead of a staged
// shared tile, for datasets too wide for any tile.
template <int V, int W, bool GM = false>
__global__ void __launch_bounds__(W * 32) k_hard(const __grid_constant__ CUtensorMap tmap, HardArgs a)
{
    constexpr int S = 32 * V;
    extern __shared__ __align__(128) unsigned char smem[];
    const int F = a.F;
    const int Fb = F < 256 ? F : 256;
    const int nbox = (F + Fb - 1) / Fb;
    const int Frows = GM ? 0 : nbox * Fb;
    float *xs = reinterpret_cast<float *>(smem);
    Rec *stage = reinterpret_cast<Rec *>(smem + (size_t)Frows * S * sizeof(float));
    uint64_t *bar = reinterpret_cast<uint64_t *>(stage + W * 32);
    int *next = reinterpret_cast<int *>(bar + 1);

    const int tile = blockIdx.x, group = blockIdx.y, G = gridDim.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *next = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (!GM && threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(Frows * S * sizeof(float)));
        for (int b = 0; b < nbox; ++b) tma_load_2d(xs + (size_t)b * Fb * S, &tmap, tile * S, b * Fb, bar);
    }

    // Per-lane samples (label-grouped order); padding samples carry label -1 and never count.
    const int64_t n0 = (int64_t)tile * S + lane * V;
    int y[V];
#pragma unroll
    for (int v = 0; v < V; ++v) y[v] = a.y[n0 + v];
    int perm[V];
    if (a.preds) {
#pragma unroll
        for (int v = 0; v < V; ++v) perm[v] = (n0 + v < a.N) ? a.perm[n0 + v] : 0;
    }
    const int64_t t_first = (int64_t)tile * S;
    const int64_t t_last = min((int64_t)tile * S + S, a.N) - 1;
    const int kmin = a.y[t_first], kmax = a.y[t_last];   // labels are sorted within the dataset

    if (!GM && !mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS)) {
        if (threadIdx.x == 0) atomicOr(a.status, ST_WAIT_TIMEOUT);
        mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS);   // let copies in flight land before exit
        return;
    }

    const int count = (a.P - group + G - 1) / G;
    Rec *st = stage + warp * 32;
    const float *xl = GM ? a.Xt + n0 : xs + lane * V;     // x[f] of the lane's samples at xl + f * xstride
    const int64_t xstride = GM ? a.n_pad : S;

    while (true) {
        int m = 0;
        if (lane == 0) m = atomicAdd(next, 1);
        m = __shfl_sync(FULL, m, 0);
        if (m >= count) break;
        const int p = a.order[group + m * G];
        const SetInfo si = a.sets[p];

        int pred[V];
        bool unc[V], al[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pred[v] = si.deflt;
            unc[v] = y[v] >= 0;
            al[v] = unc[v];
        }
        int i = si.rec_begin;
        const int re = si.rec_end;
        int base = i;
        uint4 pf = make_uint4(0, 0, 0, 0);
        if (i < re) {
            if (base + lane < re) reinterpret_cast<uint4 *>(st)[lane] = ldg_rec(a.recs + base + lane);
            __syncwarp();
            if (base + 32 + lane < re) pf = ldg_rec(a.recs + base + 32 + lane);
        }
        while (i < re) {
            if (i >= base + 32) {
                __syncwarp();
                if (i < base + 64) {
                    base += 32;
                    reinterpret_cast<uint4 *>(st)[lane] = pf;
                } else {
                    base = i;
                    if (base + lane < re) reinterpret_cast<uint4 *>(st)[lane] = ldg_rec(a.recs + base + lane);
                }
                __syncwarp();
                pf = make_uint4(0, 0, 0, 0);
                if (base + 32 + lane < re) pf = ldg_rec(a.recs + base + 32 + lane);
            }
            const uint4 raw = reinterpret_cast<const uint4 *>(st)[i - base];
            const uint32_t meta = raw.x;
            const int f = (int)(raw.y & 0xFFFFu), g = (int)(raw.y >> 16);
            const float v0 = __uint_as_float(raw.z), v1 = __uint_as_float(raw.w);
            const uint32_t kind = rec_kind(meta);
            float x[V];
            load_v<V>(xl + f * xstride, x);
            if (kind == KIND_GT) {
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = al[v] && (x[v] > v0);
            } else if (kind == KIND_LT) {
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = al[v] && (x[v] < v0);
            } else if (kind == KIND_PAIR) {
                float z[V];
                load_v<V>(xl + g * xstride, z);
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = al[v] && (__fmul_rn(v0, x[v]) > __fmul_rn(v1, z[v]));
            } else if (kind == KIND_MGT) {
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = al[v] && (__fmul_rn(v0, x[v]) > v1);
            } else if (kind == KIND_MLT) {
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = al[v] && (__fmul_rn(v0, x[v]) < v1);
            } else if (kind == KIND_IN) {
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = al[v] && category_member(x[v], raw.z, raw.w);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = false;
            }
            if (rec_last(meta)) {
                const int cls = rec_cls(meta);
                bool any_unc = false;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (al[v]) { pred[v] = cls; unc[v] = false; }
                    any_unc |= unc[v];
                }
                if (!__any_sync(FULL, any_unc)) break;
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = unc[v];
                ++i;
            } else {
                bool any_al = false;
#pragma unroll
                for (int v = 0; v < V; ++v) any_al |= al[v];
                if (!__any_sync(FULL, any_al)) {
                    i += rec_skip(meta) + 1;          // rule cannot fire: jump past it
#pragma unroll
                    for (int v = 0; v < V; ++v) al[v] = unc[v];
                } else {
                    ++i;
                }
            }
        }
        __syncwarp();

        // Counts: hit = prediction equals the label (padding has label -1).
        int hits = 0;
        bool hit[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            hit[v] = pred[v] == y[v];
            hits += __popc(__ballot_sync(FULL, hit[v]));
        }
        if (lane == 0 && hits) atomicAdd(&a.correct[p], hits);
        if (a.per_class) {
            if (kmin == kmax) {
                if (lane == 0 && hits) atomicAdd(&a.per_class[(int64_t)p * a.K + kmin], hits);
            } else {
                for (int k = kmin; k <= kmax; ++k) {
                    int ck = 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) ck += __popc(__ballot_sync(FULL, hit[v] && y[v] == k));
                    if (lane == 0 && ck) atomicAdd(&a.per_class[(int64_t)p * a.K + k], ck);
                }
            }
        }
        if (a.preds) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (y[v] >= 0) a.preds[(int64_t)p * a.N + perm[v]] = pred[v];
        }
    }
}

template <int V, int W, bool GM = false>
size_t smem_bytes(int F)
{
    if (GM) return (size_t)W * 32 * sizeof(Rec) + 16;
    const int Fb = F < 256 ? F : 256;
    const int Frows = ((F + Fb - 1) / Fb) * Fb;
    return (size_t)Frows * 32 * V * sizeof(float) + (size_t)W * 32 * sizeof(Rec) + 16;
}

template <int V, int W, bool GM = false>
rs_status launch_t(Ctx *ctx, Dataset *ds, const HardArgs &a, cudaStream_t stream)
{
    const size_t smem = smem_bytes<V, W, GM>(a.F);
    if (smem > ctx->smem_optin) return RS_ERR_TOO_LARGE;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(k_hard<V, W, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ctx->smem_optin);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(k_hard)");
    CUtensorMap none{};
    const CUtensorMap *tm = GM ? &none : dataset_tmap(ds, 32 * V);
    if (!tm) return RS_ERR_DEVICE;
    const int tiles = (int)((a.N + 32 * V - 1) / (32 * V));
    dim3 grid(tiles, a.groups);
    {
        TimedLaunch tl(ctx, TK_HARD, stream);
        k_hard<V, W, GM><<<grid, W * 32, smem, stream>>>(*tm, a);
    }
    RS_CUDA(cudaGetLastError());
    count_launch(ctx);
    return RS_OK;
}

// Compiled configurations: (samples per lane, warps per CTA).
const TileConfig kConfigs[] = {
    {0, 4, 8, 1}, {1, 4, 4, 1}, {2, 4, 16, 1}, {3, 2, 8, 1}, {4, 2, 16, 1}, {5, 1, 16, 1},
    {6, 8, 8, 1}, {7, 8, 4, 1},
    {8, 4, 8, 2}, {9, 4, 16, 2}, {10, 2, 16, 2},
    {11, 4, 8, 3}, {12, 4, 16, 3}, {13, 2, 16, 3}, {14, 2, 32, 3}, {15, 4, 32, 3},
    {16, 4, 8, 4}, {17, 4, 16, 4}, {18, 4, 32, 4}, {19, 2, 16, 4}, {20, 2, 32, 4},
    {21, 4, 16, 5}, {22, 4, 32, 5},
    {23, 4, 8, 1, true},
};
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

}  // namespace

int tile_config_count() { return kNumConfigs; }

int effective_version(const TileConfig &tc, const Dataset &ds, bool preds)
{
    if (tc.ver >= 4 && (preds || !ds.finite)) return 3;   // same V and W exist for version 3
    if (tc.ver == 5 && (!ds.ranked || hard5_smem_bytes(ds.F, tc.W) > 227 * 1024)) return 4;
    return tc.ver;
}

const TileConfig &tile_config(int id) { return kConfigs[id]; }

// Membership conditions are evaluated by the rank-coded form and by v1; a configuration of
// another form is replaced by the first v1 configuration that fits the dataset.
const TileConfig &categorical_config(const TileConfig &tc, const Dataset &ds, bool preds)
{
    if (tc.ver == 1 || effective_version(tc, ds, preds) == 5) return tc;
    for (int id : {0, 5, 23})
        if (tile_config_fits(kConfigs[id], ds.F)) return kConfigs[id];
    return kConfigs[23];
}

bool tile_config_fits(const TileConfig &tc, int F)
{
    if (tc.gmem) return true;
    const int Fb = F < 256 ? F : 256;
    const int Frows = ((F + Fb - 1) / Fb) * Fb;
    const size_t stage = (size_t)tc.W * (tc.ver >= 2 ? 64 : 32) * sizeof(Rec);
    const size_t smem = (size_t)Frows * tc.S() * sizeof(float) + stage + 16;
    return smem <= 227 * 1024 && (tc.ver == 1 || (size_t)F * tc.S() / 4 < (1u << 18));
}

rs_status launch_hard(Ctx *ctx, Dataset *ds, const TileConfig &tc, const HardArgs &a,
                      cudaStream_t stream)
{
    // correct and per_class were zeroed by the packing (k_pack_sets), which every call runs first
    if (a.P == 0) return RS_OK;
    const int ver = effective_version(tc, *ds, a.preds != nullptr);
    if (ver == 5) return launch_hard5(ctx, ds, tc.W, a, stream);
    if (ver == 4) return launch_hard4(ctx, ds, tc.V, tc.W, a, stream);
    if (ver >= 2) return launch_hard2(ctx, ds, tc.V, tc.W, ver == 3, a, stream);
    switch (tc.id) {
    case 0: return launch_t<4, 8>(ctx, ds, a, stream);
    case 1: return launch_t<4, 4>(ctx, ds, a, stream);
    case 2: return launch_t<4, 16>(ctx, ds, a, stream);
    case 3: return launch_t<2, 8>(ctx, ds, a, stream);
    case 4: return launch_t<2, 16>(ctx, ds, a, stream);
    case 5: return launch_t<1, 16>(ctx, ds, a, stream);
    case 6: return launch_t<8, 8>(ctx, ds, a, stream);
    case 7: return launch_t<8, 4>(ctx, ds, a, stream);
    case 23: return launch_t<4, 8, true>(ctx, ds, a, stream);
    default: return RS_ERR_INVALID;
    }
}

int choose_groups(Ctx *ctx, const Dataset *ds, const TileConfig &tc, int P)
{
    const int64_t tiles = (ds->N + tc.S() - 1) / tc.S();
    // aim for at least ~4 CTAs per SM in total so that warps of late tiles overlap early ones
    const int64_t want = (int64_t)ctx->sm_count * 4;
    int64_t g = (want + tiles - 1) / tiles;
    if (g < 1) g = 1;
    // keep >= 2 sets per warp in a group so the dynamic counter can balance within the CTA, unless
    // that leaves SMs idle (small launches): then down to one set per warp
    int64_t gmax = std::max<int64_t>(1, P / (2 * tc.W));
    if (tiles * gmax < ctx->sm_count) gmax = std::max<int64_t>(1, (P + tc.W - 1) / tc.W);
    if (g > gmax) g = gmax;
    // a launch of a few waves loses its last wave's idle SMs: among g .. 4g groups take the count
    // whose last wave is fullest (one resident CTA per SM, as for the 32-warp evaluators)
    const int64_t slots = ctx->sm_count;
    if (tiles * g < 16 * slots) {
        auto fill = [&](int64_t c) {
            const int64_t ctas = tiles * c;
            return (double)ctas / (double)(((ctas + slots - 1) / slots) * slots);
        };
        int64_t best = g;
        for (int64_t c = g + 1; c <= std::min(gmax, 4 * g); ++c)
            if (fill(c) > fill(best) + 1e-9) best = c;
        g = best;
    }
    if (g > 65535) g = 65535;
    return (int)g;
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_hard_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_hard<4, 8>);
    cudaFuncGetAttributes(&fa, k_hard<4, 4>);
    cudaFuncGetAttributes(&fa, k_hard<4, 16>);
    cudaFuncGetAttributes(&fa, k_hard<2, 8>);
    cudaFuncGetAttributes(&fa, k_hard<2, 16>);
    cudaFuncGetAttributes(&fa, k_hard<1, 16>);
    cudaFuncGetAttributes(&fa, k_hard<8, 8>);
    cudaFuncGetAttributes(&fa, k_hard<8, 4>);
    cudaFuncGetAttributes(&fa, k_hard<4, 8, true>);
}

}  // namespace rs
