// Rank-coded batch evaluator (record format v5); the method and the device code are described in
// eval_rank.cuh.
#include "rs_internal.cuh"
#include "eval_rank.cuh"
#include "tma.cuh"

namespace rs {

namespace {

using namespace rank;
constexpr uint64_t TMA_WAIT_LIMIT_NS = 2000000000ull;

template <int W, bool CAT>
__global__ void __launch_bounds__(W * 32, 1) k_hard5(const __grid_constant__ CUtensorMap tmx,
                                                  const __grid_constant__ CUtensorMap tmr, HardArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int F = a.F;
    const int Fb = F < 256 ? F : 256;
    const int nbox = (F + Fb - 1) / Fb;
    const int Frows = nbox * Fb;
    unsigned char *xs = smem;                                         // float [Frows][T]
    unsigned char *rs = xs + (size_t)Frows * T * 4;                   // u8 [Frows][T], then reversed
    float *us = reinterpret_cast<float *>(rs + (size_t)Frows * T * 2);  // float [F][T] sorted (built here)
    uint4 *stage_all = reinterpret_cast<uint4 *>(us + (size_t)Frows * T);
    constexpr int VS = vslots<W>();
    uint32_t *vrows = reinterpret_cast<uint32_t *>(stage_all + W * 32);     // [W][VS][32]
    float *ones = reinterpret_cast<float *>(vrows + W * VS * 32);             // [T] of 1.0 (products)
    uint64_t *bar = reinterpret_cast<uint64_t *>(ones + T);
    int *next = reinterpret_cast<int *>(bar + 1);
    uint32_t *walked = reinterpret_cast<uint32_t *>(bar + 2);        // [W][4] work counters (counting)
    const uint4 *recs = reinterpret_cast<const uint4 *>(a.recs);

    const int tile = blockIdx.x, group = blockIdx.y, G = gridDim.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *next = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 4 * W) walked[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)Frows * T * 5u);
        for (int b = 0; b < nbox; ++b) {
            tma_load_2d(xs + (size_t)b * Fb * T * 4, &tmx, tile * T, b * Fb, bar);
            tma_load_2d(rs + (size_t)b * Fb * T, &tmr, tile * T, b * Fb, bar);
        }
    }
    const int32_t *yl = a.y + (int64_t)tile * T + lane * 4;   // n_pad is a multiple of T
    const int64_t t_last = min((int64_t)tile * T + T, a.N) - 1;
    const int kmin = a.y[(int64_t)tile * T], kmax = a.y[t_last];
    const bool uniform = kmin == kmax;
    const uint32_t claimed0 = class_bytes(yl, -1);                 // padding samples

    const bool landed = mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS);
    if (!__syncthreads_and(landed)) {
        if (threadIdx.x == 0) atomicOr(a.status, ST_WAIT_TIMEOUT);
        mbar_wait_bounded(bar, 0, TMA_WAIT_LIMIT_NS);   // copies still in flight land first
        return;
    }
    const uint32_t rev_off = (uint32_t)Frows * T;
    build_tile_tables(reinterpret_cast<const float *>(xs), rs, rev_off, us, F, Frows);
    if (threadIdx.x < T) ones[threadIdx.x] = 1.f;
    __syncthreads();

    const unsigned char *rl = rs + lane * 4;       // this lane's four rank bytes of row 0
    const unsigned char *xl = xs + lane * 16;      // this lane's four floats of row 0
    const uint32_t ones_off = (uint32_t)(reinterpret_cast<unsigned char *>(ones) - xs);
    const int count = (a.P - group + G - 1) / G;
    uint4 *st = stage_all + warp * 32;

    while (true) {
        int m = 0;
        if (lane == 0) m = atomicAdd(next, 1);
        m = __shfl_sync(FULL, m, 0);
        if (m >= count) break;
        const int p = a.order[group + m * G];
        const SetInfo si = a.sets[p];
        const int rb = si.rec_begin;
        // one label k in the tile: records after the set's last rule of class k (default of another
        // class) or of any other class (default k) cannot change its count
        const int nrec = (uniform && a.last_end)
                             ? min(a.last_end[(int64_t)p * a.K + kmin], si.rec_end - si.rec_begin)
                             : si.rec_end - si.rec_begin;

        uint32_t *vr = vrows + warp * VS * 32;
        const uint32_t vr_off = (uint32_t)(reinterpret_cast<unsigned char *>(vr) - rs);
        WalkCount wc;
        const uint32_t hit =
            uniform ? walk_set<true, VS, CAT>(st, vr, vr_off, lane, recs, rb, nrec, us, rev_off, F, kmin, rl, xl,
                                              ones_off, yl, claimed0, si.deflt, wc)
                    : walk_set<false, VS, CAT>(st, vr, vr_off, lane, recs, rb, nrec, us, rev_off, F, -2, rl, xl,
                                               ones_off, yl, claimed0, si.deflt, wc);
        if (a.walked && lane == 0) {           // the warp's own slots: no atomics
            uint32_t *wk = walked + 4 * warp;
            wk[0] += wc.records;
            wk[1] += wc.rows;
            wk[2] += wc.ends;
            wk[3] += 1;
        }
        const int hits = __reduce_add_sync(FULL, __popc(hit));
        if (lane == 0 && hits) atomicAdd(&a.correct[p], hits);
        if (a.per_class) {
            if (uniform) {
                if (lane == 0 && hits) atomicAdd(&a.per_class[(int64_t)p * a.K + kmin], hits);
            } else {
                for (int k = kmin; k <= kmax; ++k) {
                    const int ckc = __reduce_add_sync(FULL, __popc(hit & class_bytes(yl, k)));
                    if (lane == 0 && ckc) atomicAdd(&a.per_class[(int64_t)p * a.K + k], ckc);
                }
            }
        }
    }
    if (a.walked && lane < 4) atomicAdd(&a.walked[lane], (unsigned long long)walked[4 * warp + lane]);
}

}  // namespace

size_t hard5_smem_bytes(int F, int W)
{
    const int Fb = F < 256 ? F : 256;
    const size_t Frows = (size_t)((F + Fb - 1) / Fb) * Fb;
    const size_t vs = W >= 32 ? vslots<32>() : vslots<16>();
    return Frows * T * (4 + 2 + 4) + (size_t)W * 32 * 16 + (size_t)W * vs * 32 * 4 + T * 4 + 16 + (size_t)W * 16;
}

template <int W, bool CAT>
static rs_status launch5_t(Ctx *ctx, Dataset *ds, const HardArgs &a, cudaStream_t stream)
{
    const size_t smem = hard5_smem_bytes(a.F, W);
    if (smem > ctx->smem_optin || !ds->ranked) return RS_ERR_TOO_LARGE;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(k_hard5<W, CAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)ctx->smem_optin);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute(k_hard5)");
    const CUtensorMap *tmx = dataset_tmap(ds, T);
    const CUtensorMap *tmr = dataset_rank_tmap(ds);
    if (!tmx || !tmr) return RS_ERR_DEVICE;
    const int tiles = (int)((a.N + T - 1) / T);
    dim3 grid(tiles, a.groups);
    {
        TimedLaunch tl(ctx, TK_HARD, stream);
        k_hard5<W, CAT><<<grid, W * 32, smem, stream>>>(*tmx, *tmr, a);
    }
    RS_CUDA(cudaGetLastError());
    count_launch(ctx);
    return RS_OK;
}

rs_status launch_hard5(Ctx *ctx, Dataset *ds, int W, const HardArgs &a, cudaStream_t stream)
{
    if (a.P == 0) return RS_OK;
    if (W == 16) return a.cat ? launch5_t<16, true>(ctx, ds, a, stream) : launch5_t<16, false>(ctx, ds, a, stream);
    if (W == 32) return a.cat ? launch5_t<32, true>(ctx, ds, a, stream) : launch5_t<32, false>(ctx, ds, a, stream);
    return RS_ERR_INVALID;
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_hard5_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_hard5<16, false>);
    cudaFuncGetAttributes(&fa, k_hard5<16, true>);
    cudaFuncGetAttributes(&fa, k_hard5<32, false>);
    cudaFuncGetAttributes(&fa, k_hard5<32, true>);
}

}  // namespace rs
