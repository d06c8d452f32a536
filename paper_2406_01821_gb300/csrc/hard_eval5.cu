// Rank-coded evaluator for datasets with rank tables (record format v5).
//
// A threshold condition has been rewritten exactly as x > c or x < c (pack.cu). Within one
// 128-sample tile, let rank(x) be the number of the tile's values (same feature) strictly below
// x. Because x is itself one of the tile's values,
//     x >  c  <=>  rank(x) >= L,   L = #{tile values <= c}
//     x <= c  <=>  rank(x) <  L
// (a '<' cut x < c arrives as x <= nextdown(c)). L is counted once per tile and condition, by a
// binary search over the tile's sorted values, when the condition's record is staged. The test
// of a lane's four samples is then one 32-bit subtraction on four rank bytes (0..127), with the
// failure in bit 7 of each byte:
//     '>':  byte (L + 127) - rank          >= 128  <=>  rank <  L   (fails)
//     '<=': byte (255 - L) - (127 - rank)  >= 128  <=>  rank >= L   (fails)
// Each byte difference lies in [0, 255], so no borrow crosses a byte. The second form reads a
// table of reversed ranks (127 - rank), built in shared memory from the first, so that both
// forms are "constant minus table word". A rule's failures are ORed into one word per lane; pair
// and product conditions are compared on the float tile and packed into the same byte layout.
// Claims, per-class hits and the all-claimed exit work on these words (bit 7 of byte v belongs
// to the lane's sample v). A set's records are one flat stream (each rule's conditions, the last
// one flagged) walked 32 records at a time. Predictions are not produced here.
#include "rs_internal.cuh"
#include "tma.cuh"

namespace rs {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t HIGH = 0x80808080u;          // bit 7 of every byte
constexpr uint32_t ONES = 0x01010101u;
constexpr uint64_t TMA_WAIT_LIMIT_NS = 2000000000ull;
constexpr int T = RANK_TILE;                     // samples per tile (= one warp, four per lane)

// #{j : row[j] <= c} (or < c) over the 128 ascending values of a row stored at j ^ sw.
template <bool LE>
__device__ __forceinline__ int count_below(const float *row, int sw, float c)
{
    int pos = 0;
#pragma unroll
    for (int step = 64; step >= 1; step >>= 1) {
        const float u = row[(pos + step - 1) ^ sw];
        if (LE ? (u <= c) : (u < c)) pos += step;
    }
    const float u = row[pos ^ sw];               // pos <= 127: one more for a full count
    if (LE ? (u <= c) : (u < c)) pos += 1;
    return pos;
}

// pass rows per warp for pair / product conditions of one chunk
template <int W> __host__ __device__ constexpr int vslots() { return W >= 32 ? 12 : 16; }
constexpr uint32_t NOOP_K = 127u * ONES;     // constant - rank never has bit 7 set: never fails

// The staged form of a cut for this tile: {rank-table byte offset of the row, per-byte constant}.
__device__ __forceinline__ uint2 stage_cut(uint4 r, const float *us, uint32_t rev_off, int F)
{
    const uint32_t f = min(r.x & R5_F_MASK, (uint32_t)(F - 1));
    const bool le = (r.x >> R5_TAG_SHIFT) == R5_CUT_LT;
    const int L = count_below<true>(us + f * T, (int)(f & 31u), __uint_as_float(r.z));
    return make_uint2((le ? rev_off : 0u) + f * T, (uint32_t)(le ? 255 - L : L + 127) * ONES);
}

// 0xFF in byte v where p[v] > q[v] (IEEE compare: false with NaN), 0 elsewhere.
__device__ __forceinline__ uint32_t gt_bytes(const float (&p)[4], const float (&q)[4])
{
    uint32_t s[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) asm("set.gt.u32.f32 %0, %1, %2;" : "=r"(s[v]) : "f"(p[v]), "f"(q[v]));
    return __byte_perm(__byte_perm(s[0], s[1], 0x0040), __byte_perm(s[2], s[3], 0x0040), 0x5410);
}

// Bit 7 of byte v where the lane's sample v (labels yl[0..3]) has label k. Only tiles that hold
// more than one label need it, so the labels are read again instead of kept in registers.
__device__ __forceinline__ uint32_t class_bytes(const int32_t *yl, int k)
{
    const int4 y = __ldg(reinterpret_cast<const int4 *>(yl));
    return ((y.x == k) ? 0x80u : 0u) | ((y.y == k) ? 0x8000u : 0u) | ((y.z == k) ? 0x800000u : 0u) |
           ((y.w == k) ? 0x80000000u : 0u);
}

// Pass bits (0x80 in byte v where the condition holds for the lane's sample v) of a pair
// condition fl(a * x[f]) > fl(b * x[g]) or a product condition fl(a * x[f]) > b. The products are
// separately rounded (packed two-lane multiplies).
__device__ __forceinline__ uint32_t pass_bytes(uint4 r, const unsigned char *xl, int F)
{
    const uint32_t f = min(r.x & R5_F_MASK, (uint32_t)(F - 1));
    const float4 x = *reinterpret_cast<const float4 *>(xl + f * T * 4u);
    const float a = __uint_as_float(r.z), b = __uint_as_float(r.w);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    const float2 p01 = __fmul2_rn(make_float2(x.x, x.y), a2), p23 = __fmul2_rn(make_float2(x.z, x.w), a2);
    float2 q01 = b2, q23 = b2;
    if ((r.x >> R5_TAG_SHIFT) == R5_PAIR) {
        const uint32_t g = min(r.y, (uint32_t)(F - 1));
        const float4 z = *reinterpret_cast<const float4 *>(xl + g * T * 4u);
        q01 = __fmul2_rn(make_float2(z.x, z.y), b2);
        q23 = __fmul2_rn(make_float2(z.z, z.w), b2);
    }
    const float p[4] = {p01.x, p01.y, p23.x, p23.y}, q[4] = {q01.x, q01.y, q23.x, q23.y};
    return gt_bytes(p, q) & HIGH;
}

// One group of four staged records with end-of-rule flags M (bit u: record u ends its rule).
template <uint32_t M, bool UNI>
__device__ __forceinline__ void group4(const uint32_t (&e)[4], const uint32_t *sw, const int32_t *yl,
                                       uint32_t &fail, uint32_t &claimed, uint32_t &hit)
{
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        fail |= e[u];
        if (M & (1u << u)) {
            const uint32_t w = sw[u];
            const uint32_t newly = ~fail & HIGH;
            if (UNI) hit |= newly & w;
            else hit |= newly & class_bytes(yl, (int)w);
            claimed |= newly;
            fail = claimed;
        }
    }
}

// Walk the rules of one set (records [rb, rb + nrec)) over the lane's four samples; returns the
// hit bits (bit 7 of byte v: sample v predicted correctly, default included). UNI: the tile holds
// one label (kmine) and end records carry the class mask.
//
// The set is walked in chunks of up to 32 records. Staging turns every record of a chunk into the
// same form {byte offset from the lane's rank word, per-byte constant}: a cut points at its rank
// row; a pair or product condition is first evaluated by the whole warp into a pass row
// (0x80 / 0x00 per sample, constant 0x80808080) in the warp's `vrow` slots; padding records are
// no-ops. The chunk is then one straight run of identical steps, with the first-fire claim
// applied after each rule's last record (a warp vote gives their positions).
template <bool UNI, int VS>
__device__ __forceinline__ uint32_t walk_set(uint4 *st, uint32_t *vrow, uint32_t vrow_off, int lane,
                                             const uint4 *recs, int rb, int nrec, const float *us,
                                             uint32_t rev_off, int F, int kmine, const unsigned char *rl,
                                             const unsigned char *xl, const int32_t *yl, uint32_t claimed,
                                             int deflt)
{
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    uint2 *s8 = reinterpret_cast<uint2 *>(st);            // staged {offset, constant}, 32 entries
    uint32_t *sw = reinterpret_cast<uint32_t *>(st) + 64;  // end-of-rule class mask / class
    uint4 pf = lane < nrec ? __ldcg(recs + rb + lane) : zero4;
    uint32_t hit = 0, fail = claimed;
    bool done = false;
    int c0 = 0;
    while (c0 < nrec && !done) {
        const uint4 raw = pf;
        const uint32_t tag = raw.x >> R5_TAG_SHIFT;
        int cnt = min(32, nrec - c0);
        uint32_t pm = __ballot_sync(FULL, lane < cnt && (tag == R5_PAIR || tag == R5_GEN));
        if (__popc(pm) > VS) {              // end the chunk before the pair that finds no slot
            uint32_t m = pm;
            for (int k = 0; k < VS; ++k) m &= m - 1u;
            cnt = __ffs(m) - 1;
            pm &= (1u << cnt) - 1u;
        }
        const uint32_t ends = __ballot_sync(FULL, lane < cnt && (raw.x & R5_END_BIT) != 0u);
        pf = (c0 + cnt + lane < nrec) ? __ldcg(recs + rb + c0 + cnt + lane) : zero4;

        __syncwarp();
        st[lane] = raw;                     // raw records, read back by the pass-row loop
        // every lane runs the cut search (branch-free staging); other records then take their form
        const uint32_t cls = (raw.x >> R5_CLS_SHIFT) & 0xFFFu;
        const uint32_t ew = UNI ? ((int)cls == kmine ? 0xFFFFFFFFu : 0u) : cls;
        uint2 sr = stage_cut(raw, us, rev_off, F);
        if ((pm >> lane) & 1u) sr = make_uint2(vrow_off + 128u * (uint32_t)__popc(pm & ((1u << lane) - 1u)), HIGH);
        else if (lane >= cnt || tag == R5_NONE) sr = make_uint2(0u, NOOP_K);
        __syncwarp();
        {                                             // pass rows, one warp-wide evaluation each
            uint32_t m = pm;
            uint32_t *vr = vrow + lane;
            while (m) {
                const uint4 p0 = st[__ffs(m) - 1];
                m &= m - 1u;
                if (m) {
                    const uint4 p1 = st[__ffs(m) - 1];
                    m &= m - 1u;
                    const uint32_t v0 = pass_bytes(p0, xl, F), v1 = pass_bytes(p1, xl, F);
                    vr[0] = v0;
                    vr[32] = v1;
                    vr += 64;
                } else {
                    vr[0] = pass_bytes(p0, xl, F);
                }
            }
        }
        __syncwarp();
        s8[lane] = sr;
        sw[lane] = ew;
        __syncwarp();

        for (int g = 0; g < cnt; g += 4) {
            const uint4 ra = *reinterpret_cast<const uint4 *>(s8 + g);
            const uint4 rc = *reinterpret_cast<const uint4 *>(s8 + g + 2);
            const uint32_t e0 = ra.y - *reinterpret_cast<const uint32_t *>(rl + ra.x);
            const uint32_t e1 = ra.w - *reinterpret_cast<const uint32_t *>(rl + ra.z);
            const uint32_t e2 = rc.y - *reinterpret_cast<const uint32_t *>(rl + rc.x);
            const uint32_t e3 = rc.w - *reinterpret_cast<const uint32_t *>(rl + rc.z);
            const uint32_t e[4] = {e0, e1, e2, e3};
            const uint32_t *swg = sw + g;
            switch ((ends >> g) & 0xFu) {
#define RS_GROUP4(M) case M: group4<M, UNI>(e, swg, yl, fail, claimed, hit); break;
            RS_GROUP4(0) RS_GROUP4(1) RS_GROUP4(2) RS_GROUP4(3) RS_GROUP4(4) RS_GROUP4(5) RS_GROUP4(6)
            RS_GROUP4(7) RS_GROUP4(8) RS_GROUP4(9) RS_GROUP4(10) RS_GROUP4(11) RS_GROUP4(12)
            RS_GROUP4(13) RS_GROUP4(14) RS_GROUP4(15)
#undef RS_GROUP4
            }
            if (((ends >> g) & 0xFu) && __all_sync(FULL, claimed == HIGH)) { done = true; break; }
        }
        c0 += cnt;
    }
    const uint32_t left = ~claimed & HIGH;
    if (UNI) hit |= (deflt == kmine) ? left : 0u;
    else hit |= left & class_bytes(yl, deflt);
    return hit;
}

template <int W>
__global__ void __launch_bounds__(W * 32, 1) k_hard5(const __grid_constant__ CUtensorMap tmx,
                                                  const __grid_constant__ CUtensorMap tmr, HardArgs a,
                                                  const float *__restrict__ Us)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int F = a.F;
    const int Fb = F < 256 ? F : 256;
    const int nbox = (F + Fb - 1) / Fb;
    const int Frows = nbox * Fb;
    unsigned char *xs = smem;                                         // float [Frows][T]
    unsigned char *rs = xs + (size_t)Frows * T * 4;                   // u8 [Frows][T], then reversed
    float *us = reinterpret_cast<float *>(rs + (size_t)Frows * T * 2);  // float [F][T] sorted
    uint4 *stage_all = reinterpret_cast<uint4 *>(us + (size_t)Frows * T);
    constexpr int VS = vslots<W>();
    uint32_t *vrows = reinterpret_cast<uint32_t *>(stage_all + W * 32);     // [W][VS][32]
    uint64_t *bar = reinterpret_cast<uint64_t *>(vrows + W * VS * 32);
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
        const uint32_t ubytes = (uint32_t)F * T * 4u;
        mbar_arrive_expect_tx(bar, (uint32_t)Frows * T * 5u + ubytes);
        for (int b = 0; b < nbox; ++b) {
            tma_load_2d(xs + (size_t)b * Fb * T * 4, &tmx, tile * T, b * Fb, bar);
            tma_load_2d(rs + (size_t)b * Fb * T, &tmr, tile * T, b * Fb, bar);
        }
        bulk_load(us, Us + (size_t)tile * F * T, ubytes, bar);
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
    {
        const uint32_t *r32 = reinterpret_cast<const uint32_t *>(rs);
        uint32_t *rr32 = reinterpret_cast<uint32_t *>(rs + rev_off);
        for (int i = threadIdx.x; i < Frows * T / 4; i += W * 32) rr32[i] = r32[i] ^ 0x7F7F7F7Fu;
    }
    __syncthreads();

    const unsigned char *rl = rs + lane * 4;       // this lane's four rank bytes of row 0
    const unsigned char *xl = xs + lane * 16;      // this lane's four floats of row 0
    const int count = (a.P - group + G - 1) / G;
    uint4 *st = stage_all + warp * 32;

    while (true) {
        int m = 0;
        if (lane == 0) m = atomicAdd(next, 1);
        m = __shfl_sync(FULL, m, 0);
        if (m >= count) break;
        const int p = a.order[group + m * G];
        const SetInfo si = a.sets[p];
        const int rb = si.rec_begin, nrec = si.rec_end - si.rec_begin;

        uint32_t *vr = vrows + warp * VS * 32;
        const uint32_t vr_off = (uint32_t)(reinterpret_cast<unsigned char *>(vr) - rs);
        const uint32_t hit =
            uniform ? walk_set<true, VS>(st, vr, vr_off, lane, recs, rb, nrec, us, rev_off, F, kmin, rl, xl, yl,
                                     claimed0, si.deflt)
                    : walk_set<false, VS>(st, vr, vr_off, lane, recs, rb, nrec, us, rev_off, F, -2, rl, xl, yl,
                                      claimed0, si.deflt);
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
}

}  // namespace

size_t hard5_smem_bytes(int F, int W)
{
    const int Fb = F < 256 ? F : 256;
    const size_t Frows = (size_t)((F + Fb - 1) / Fb) * Fb;
    const size_t vs = W >= 32 ? vslots<32>() : vslots<16>();
    return Frows * T * (4 + 2 + 4) + (size_t)W * 32 * 16 + (size_t)W * vs * 32 * 4 + 16;
}

template <int W>
static rs_status launch5_t(Ctx *ctx, Dataset *ds, const HardArgs &a, cudaStream_t stream)
{
    const size_t smem = hard5_smem_bytes(a.F, W);
    if (smem > ctx->smem_optin || !ds->ranked) return RS_ERR_TOO_LARGE;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(k_hard5<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
        k_hard5<W><<<grid, W * 32, smem, stream>>>(*tmx, *tmr, a, ds->Us);
    }
    RS_CUDA(cudaGetLastError());
    count_launch(ctx);
    return RS_OK;
}

rs_status launch_hard5(Ctx *ctx, Dataset *ds, int W, const HardArgs &a, cudaStream_t stream)
{
    if (a.P > 0) RS_CUDA(cudaMemsetAsync(a.correct, 0, sizeof(int32_t) * a.P, stream));
    if (a.P > 0 && a.per_class)
        RS_CUDA(cudaMemsetAsync(a.per_class, 0, sizeof(int32_t) * (size_t)a.P * a.K, stream));
    if (a.P == 0) return RS_OK;
    if (W == 16) return launch5_t<16>(ctx, ds, a, stream);
    if (W == 32) return launch5_t<32>(ctx, ds, a, stream);
    return RS_ERR_INVALID;
}

}  // namespace rs
