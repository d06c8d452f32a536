// Sign-mask evaluator for datasets with only finite values (record format v4).
//
// A threshold condition x > c holds exactly when x >= c' with c' = nextup(c), i.e. when
// m = fl(x - c') has a clear sign bit: for finite x and c' != +0 the difference is +0 only for
// x = c', positive above and negative below (gradual underflow), and x - c' never produces -0 or
// NaN. A '<' cut is the same test on -x. Since the product by +-1 is exact, m is one fused
// multiply-add, computed for two samples at a time with the packed f32x2 FMA; a rule's
// conjunction is the OR of its conditions' margin bit patterns (fires iff the sign stays clear),
// seeded with the "already claimed" sign of each sample. Feature-pair and general-product
// conditions take an ordinary compare and contribute a sign mask.
//
// Per-class counting uses the label grouping of the dataset: in a tile holding one label k, only
// rules of class k (and the default, if it is k) can add hits, decided once per rule for the whole
// warp. Predictions are not produced here (the caller then uses the general evaluator).
#include "rs_internal.cuh"
#include "eval_core.cuh"
#include "tma.cuh"

namespace rs {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint64_t TMA_WAIT_LIMIT_NS = 2000000000ull;

template <int V, int W>
__global__ void __launch_bounds__(W * 32) k_hard4(const __grid_constant__ CUtensorMap tmap, HardArgs a)
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
    const int64_t t_last = min((int64_t)tile * S + S, a.N) - 1;
    const int kmin = a.y[(int64_t)tile * S], kmax = a.y[t_last];
    const bool uniform = kmin == kmax;

    if (!mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS)) {
        if (threadIdx.x == 0) atomicOr(a.status, ST_WAIT_TIMEOUT);
        mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS);
        return;
    }

    const int count = (a.P - group + G - 1) / G;
    uint4 *st = stage_all + warp * 64;
    const float *xl = xs + lane * V;

    while (true) {
        int m = 0;
        if (lane == 0) m = atomicAdd(next, 1);
        m = __shfl_sync(FULL, m, 0);
        if (m >= count) break;
        const int p = a.order[group + m * G];
        const SetInfo si = a.sets[p];
        const int rb = si.rec_begin, re = si.rec_end;

        uint32_t hit[V];
        core::eval_set_sign<V>(recs, rb, re, st, xl, lane, si.deflt, y, uniform, kmin, hit);
        int hits = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) hits += __popc(__ballot_sync(FULL, hit[v] != 0u));
        if (lane == 0 && hits) atomicAdd(&a.correct[p], hits);
        if (a.per_class) {
            if (uniform) {
                if (lane == 0 && hits) atomicAdd(&a.per_class[(int64_t)p * a.K + kmin], hits);
            } else {
                for (int k = kmin; k <= kmax; ++k) {
                    int ckc = 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) ckc += __popc(__ballot_sync(FULL, hit[v] != 0u && y[v] == k));
                    if (lane == 0 && ckc) atomicAdd(&a.per_class[(int64_t)p * a.K + k], ckc);
                }
            }
        }
    }
}

}  // namespace

template <int V, int W>
rs_status launch4_t(Ctx *ctx, Dataset *ds, const HardArgs &a, cudaStream_t stream)
{
    const int Fb = a.F < 256 ? a.F : 256;
    const int Frows = ((a.F + Fb - 1) / Fb) * Fb;
    const size_t smem = (size_t)Frows * 32 * V * sizeof(float) + (size_t)W * 64 * 16 + 16;
    if (smem > ctx->smem_optin) return RS_ERR_TOO_LARGE;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(k_hard4<V, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ctx->smem_optin);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(k_hard4)");
    const CUtensorMap *tm = dataset_tmap(ds, 32 * V);
    if (!tm) return RS_ERR_DEVICE;
    const int tiles = (int)((a.N + 32 * V - 1) / (32 * V));
    dim3 grid(tiles, a.groups);
    {
        TimedLaunch tl(ctx, TK_HARD, stream);
        k_hard4<V, W><<<grid, W * 32, smem, stream>>>(*tm, a);
    }
    RS_CUDA(cudaGetLastError());
    count_launch(ctx);
    return RS_OK;
}

rs_status launch_hard4(Ctx *ctx, Dataset *ds, int V, int W, const HardArgs &a, cudaStream_t stream)
{
    if (a.P == 0) return RS_OK;
    if (V == 4 && W == 8) return launch4_t<4, 8>(ctx, ds, a, stream);
    if (V == 4 && W == 16) return launch4_t<4, 16>(ctx, ds, a, stream);
    if (V == 4 && W == 32) return launch4_t<4, 32>(ctx, ds, a, stream);
    if (V == 2 && W == 16) return launch4_t<2, 16>(ctx, ds, a, stream);
    if (V == 2 && W == 32) return launch4_t<2, 32>(ctx, ds, a, stream);
    return RS_ERR_INVALID;
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_hard4_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_hard4<4, 8>);
    cudaFuncGetAttributes(&fa, k_hard4<4, 16>);
    cudaFuncGetAttributes(&fa, k_hard4<4, 32>);
    cudaFuncGetAttributes(&fa, k_hard4<2, 16>);
    cudaFuncGetAttributes(&fa, k_hard4<2, 32>);
}

}  // namespace rs
