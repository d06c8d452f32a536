// Rule-at-a-time variant of the hard evaluator (record format v2).
//
// Differences from k_hard: every condition is one of two forms -- LIN: fl(v0*x[f]) > v1, or
// PAIR: fl(v0*x[f]) > fl(v1*x[g]) -- so threshold '>' / '<' cuts, zero/infinite coefficients and
// never-true conditions share one code path (a '<' becomes '>' on exactly negated operands; the
// multiply by +-1 runs on the FMA pipe, the compare on the ALU pipe). Records carry their feature
// rows as shared-memory offsets for the launch's tile width, and the first record of a rule carries
// the rule length, so a rule is evaluated as one counted loop with the claim and the "all claimed"
// vote once per rule. Records stream through a two-chunk linear stage per warp.
#include "rs_internal.cuh"
#include "tma.cuh"

namespace rs {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint64_t TMA_WAIT_LIMIT_NS = 2000000000ull;

template <int V>
__device__ __forceinline__ void load_v2(const float *p, float (&x)[V])
{
    if constexpr (V == 2) {
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

__device__ __forceinline__ float min_nan(float a, float b)
{
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Margin form: the condition holds iff m = fl(fl(v0*x) - rhs) > 0 (exact for every input: the
// difference of two floats is positive iff the first is larger under gradual underflow, and
// inf - inf and NaN operands give NaN, which is not > 0). A rule fires iff the NaN-propagating
// minimum of its margins is > 0.
template <int V>
__device__ __forceinline__ void eval_rec_m(const uint4 r, const float *xl, float (&mn)[V])
{
    float x[V];
    load_v2<V>(xl + (r.x & OFF_MASK) * 4, x);
    const float v0 = __uint_as_float(r.z), v1 = __uint_as_float(r.w);
    if (r.x & PAIR_BIT) {
        float z[V];
        load_v2<V>(xl + (r.y & OFF_MASK) * 4, z);
#pragma unroll
        for (int v = 0; v < V; ++v)
            mn[v] = min_nan(mn[v], __fsub_rn(__fmul_rn(v0, x[v]), __fmul_rn(v1, z[v])));
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) mn[v] = min_nan(mn[v], __fsub_rn(__fmul_rn(v0, x[v]), v1));
    }
}

template <int V>
__device__ __forceinline__ void eval_rec(const uint4 r, const float *xl, bool (&al)[V])
{
    float x[V];
    load_v2<V>(xl + (r.x & OFF_MASK) * 4, x);
    const float v0 = __uint_as_float(r.z), v1 = __uint_as_float(r.w);
    if (r.x & PAIR_BIT) {
        float z[V];
        load_v2<V>(xl + (r.y & OFF_MASK) * 4, z);
#pragma unroll
        for (int v = 0; v < V; ++v) al[v] = al[v] && (__fmul_rn(v0, x[v]) > __fmul_rn(v1, z[v]));
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) al[v] = al[v] && (__fmul_rn(v0, x[v]) > v1);
    }
}

template <int V, int W, bool MM>
__global__ void __launch_bounds__(W * 32) k_hard2(const __grid_constant__ CUtensorMap tmap, HardArgs a)
{
    constexpr int S = 32 * V;
    extern __shared__ __align__(128) unsigned char smem[];
    const int F = a.F;
    const int Fb = F < 256 ? F : 256;
    const int nbox = (F + Fb - 1) / Fb;
    const int Frows = nbox * Fb;
    float *xs = reinterpret_cast<float *>(smem);
    uint4 *stage_all = reinterpret_cast<uint4 *>(smem + (size_t)Frows * S * sizeof(float));
    uint64_t *bar = reinterpret_cast<uint64_t *>(stage_all + W * 64);
    int *next = reinterpret_cast<int *>(bar + 1);
    const uint4 *recs = reinterpret_cast<const uint4 *>(a.recs);

    const int tile = blockIdx.x, group = blockIdx.y, G = gridDim.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *next = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(Frows * S * sizeof(float)));
        for (int b = 0; b < nbox; ++b) tma_load_2d(xs + (size_t)b * Fb * S, &tmap, tile * S, b * Fb, bar);
    }
    const int64_t n0 = (int64_t)tile * S + lane * V;
    int y[V];
#pragma unroll
    for (int v = 0; v < V; ++v) y[v] = a.y[n0 + v];
    int perm[V];
    if (a.preds) {
#pragma unroll
        for (int v = 0; v < V; ++v) perm[v] = (n0 + v < a.N) ? a.perm[n0 + v] : 0;
    }
    const int64_t t_last = min((int64_t)tile * S + S, a.N) - 1;
    const int kmin = a.y[(int64_t)tile * S], kmax = a.y[t_last];

    if (!mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS)) {
        if (threadIdx.x == 0) atomicOr(a.status, ST_WAIT_TIMEOUT);
        mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS);
        return;
    }

    const int count = (a.P - group + G - 1) / G;
    uint4 *st = stage_all + warp * 64;
    const float *xl = xs + lane * V;
    const uint4 zero4 = make_uint4(0, 0, 0, 0);

    while (true) {
        int m = 0;
        if (lane == 0) m = atomicAdd(next, 1);
        m = __shfl_sync(FULL, m, 0);
        if (m >= count) break;
        const int p = a.order[group + m * G];
        const SetInfo si = a.sets[p];
        const int rb = si.rec_begin, re = si.rec_end;

        int pred[V];
        bool unc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pred[v] = si.deflt;
            unc[v] = y[v] >= 0;
        }
        // stage holds records [rb + 32*ck, rb + 32*ck + 64)
        int ck = 0;
        uint4 pf = zero4;
        if (rb < re) {
            __syncwarp();
            st[lane] = (rb + lane < re) ? __ldg(recs + rb + lane) : zero4;
            st[32 + lane] = (rb + 32 + lane < re) ? __ldg(recs + rb + 32 + lane) : zero4;
            pf = (rb + 64 + lane < re) ? __ldg(recs + rb + 64 + lane) : zero4;
            __syncwarp();
        }
        int rel = 0;
        const int nrec = re - rb;
        while (rel < nrec) {
            while ((rel >> 5) > ck) {       // slide the stage by one chunk
                const uint4 keep = st[32 + lane];
                __syncwarp();
                st[lane] = keep;
                st[32 + lane] = pf;
                __syncwarp();
                ++ck;
                const int nx = rb + 32 * (ck + 2) + lane;
                pf = (nx < re) ? __ldg(recs + nx) : zero4;
            }
            const uint4 *rp = st + (rel - 32 * ck);
            const uint4 r0 = rp[0];
            const int nc = max(1, (int)((r0.x >> LEN_SHIFT) & 0xFFFu));   // >= 1: progress
            const int cls = (int)(r0.y >> CLS_SHIFT);
            bool al[V];
            if constexpr (MM) {
                float mn[V];
#pragma unroll
                for (int v = 0; v < V; ++v) mn[v] = unc[v] ? __uint_as_float(0x7F800000u) : -1.f;
                if (nc <= 33) {
                    eval_rec_m<V>(r0, xl, mn);
#pragma unroll 2
                    for (int k = 1; k < nc; ++k) eval_rec_m<V>(rp[k], xl, mn);
                } else {
                    eval_rec_m<V>(r0, xl, mn);
                    for (int k = 1; k < nc; ++k) eval_rec_m<V>(__ldg(recs + rb + rel + k), xl, mn);
                }
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = mn[v] > 0.f;
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) al[v] = unc[v];
                if (nc <= 33) {
                    eval_rec<V>(r0, xl, al);
#pragma unroll 2
                    for (int k = 1; k < nc; ++k) eval_rec<V>(rp[k], xl, al);
                } else {
                    // long rule: read its records straight from global memory
                    eval_rec<V>(r0, xl, al);
                    for (int k = 1; k < nc; ++k) eval_rec<V>(__ldg(recs + rb + rel + k), xl, al);
                }
            }
            bool any_unc = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (al[v]) { pred[v] = cls; unc[v] = false; }
                any_unc |= unc[v];
            }
            if (!__any_sync(FULL, any_unc)) break;
            rel += nc;
        }
        __syncwarp();

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
                    int ckc = 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) ckc += __popc(__ballot_sync(FULL, hit[v] && y[v] == k));
                    if (lane == 0 && ckc) atomicAdd(&a.per_class[(int64_t)p * a.K + k], ckc);
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

}  // namespace

template <int V, int W>
static size_t smem_bytes2(int F)
{
    const int Fb = F < 256 ? F : 256;
    const int Frows = ((F + Fb - 1) / Fb) * Fb;
    return (size_t)Frows * 32 * V * sizeof(float) + (size_t)W * 64 * 16 + 16;
}

template <int V, int W, bool MM>
rs_status launch2_t(Ctx *ctx, Dataset *ds, const HardArgs &a, cudaStream_t stream)
{
    const size_t smem = smem_bytes2<V, W>(a.F);
    if (smem > ctx->smem_optin) return RS_ERR_TOO_LARGE;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(k_hard2<V, W, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ctx->smem_optin);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(k_hard2)");
    const CUtensorMap *tm = dataset_tmap(ds, 32 * V);
    if (!tm) return RS_ERR_DEVICE;
    const int tiles = (int)((a.N + 32 * V - 1) / (32 * V));
    dim3 grid(tiles, a.groups);
    {
        TimedLaunch tl(ctx, TK_HARD, stream);
        k_hard2<V, W, MM><<<grid, W * 32, smem, stream>>>(*tm, a);
    }
    RS_CUDA(cudaGetLastError());
    count_launch(ctx);
    return RS_OK;
}

rs_status launch_hard2(Ctx *ctx, Dataset *ds, int V, int W, bool mm, const HardArgs &a,
                       cudaStream_t stream)
{
    if (a.P == 0) return RS_OK;
    if (!mm) {
        if (V == 4 && W == 8) return launch2_t<4, 8, false>(ctx, ds, a, stream);
        if (V == 4 && W == 16) return launch2_t<4, 16, false>(ctx, ds, a, stream);
        if (V == 2 && W == 16) return launch2_t<2, 16, false>(ctx, ds, a, stream);
    } else {
        if (V == 4 && W == 8) return launch2_t<4, 8, true>(ctx, ds, a, stream);
        if (V == 4 && W == 16) return launch2_t<4, 16, true>(ctx, ds, a, stream);
        if (V == 2 && W == 16) return launch2_t<2, 16, true>(ctx, ds, a, stream);
        if (V == 2 && W == 32) return launch2_t<2, 32, true>(ctx, ds, a, stream);
        if (V == 4 && W == 32) return launch2_t<4, 32, true>(ctx, ds, a, stream);
    }
    return RS_ERR_INVALID;
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_hard2_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_hard2<4, 8, false>);
    cudaFuncGetAttributes(&fa, k_hard2<4, 16, false>);
    cudaFuncGetAttributes(&fa, k_hard2<2, 16, false>);
    cudaFuncGetAttributes(&fa, k_hard2<4, 8, true>);
    cudaFuncGetAttributes(&fa, k_hard2<4, 16, true>);
    cudaFuncGetAttributes(&fa, k_hard2<2, 16, true>);
    cudaFuncGetAttributes(&fa, k_hard2<2, 32, true>);
    cudaFuncGetAttributes(&fa, k_hard2<4, 32, true>);
}

}  // namespace rs
