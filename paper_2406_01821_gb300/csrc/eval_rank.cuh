// Device code of the rank-coded evaluator (record format v5), shared by the batch evaluator and
// the serving kernel.
//
// A threshold condition has been rewritten exactly as x > c or x < c (pack.cu). Within one
// 128-sample tile, let rank(x) be the position of x in the tile's values (same feature) in
// ascending order, equal values in sample order: #{values below x} + #{equal values before it}.
// Because x is itself one of the tile's values, and a group of equal values is either wholly
// <= c or wholly > c,
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
#pragma once
#include "rs_internal.cuh"

namespace rs {
namespace rank {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t HIGH = 0x80808080u;          // bit 7 of every byte
constexpr uint32_t ONES = 0x01010101u;
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

// The per-tile tables built in shared memory by the whole block once the tile's features xs
// [F][T] and rank bytes rs [Frows][T] have landed: the reversed ranks (127 - rank) at rs + rev_off
// and each feature's sorted column us[f][pos ^ (f & 31)] = x[f][n] with pos the rank of x[f][n]
// (its position in the tile's stable ascending order: a permutation, so every slot is written).
__device__ __forceinline__ void build_tile_tables(const float *xs, unsigned char *rs, uint32_t rev_off, float *us,
                                                  int F, int Frows)
{
    const uint32_t *r32 = reinterpret_cast<const uint32_t *>(rs);
    uint32_t *rr32 = reinterpret_cast<uint32_t *>(rs + rev_off);
    for (int i = threadIdx.x; i < Frows * T / 4; i += blockDim.x) rr32[i] = r32[i] ^ 0x7F7F7F7Fu;
    for (int i = threadIdx.x; i < F * T; i += blockDim.x) {
        const int f = i / T;
        us[f * T + (rs[i] ^ (f & 31))] = xs[i];
    }
}

// The staged form of a cut for this tile: {rank-table byte offset of the row, per-byte constant}.
__device__ __forceinline__ uint2 stage_cut(uint4 r, const float *us, uint32_t rev_off, int F)
{
    const uint32_t f = min(r.x & R5_F_MASK, (uint32_t)(F - 1));
    const bool le = (r.x >> R5_TAG_SHIFT) == R5_CUT_LT;
    const int L = count_below<true>(us + f * T, (int)(f & 31u), __uint_as_float(r.z));
    return make_uint2((le ? rev_off : 0u) + f * T, (uint32_t)(le ? 255 - L : L + 127) * ONES);
}

// Bit 7 of byte v where the lane's sample v (labels yl[0..3]) has label k. Only tiles that hold
// more than one label need it, so the labels are read again instead of kept in registers.
__device__ __forceinline__ uint32_t class_bytes(const int32_t *yl, int k)
{
    const int4 y = __ldg(reinterpret_cast<const int4 *>(yl));
    return ((y.x == k) ? 0x80u : 0u) | ((y.y == k) ? 0x8000u : 0u) | ((y.z == k) ? 0x800000u : 0u) |
           ((y.w == k) ? 0x80000000u : 0u);
}

// Pass row of a pair condition fl(a * x[f]) > fl(b * x[g]) or a product condition
// fl(a * x[f]) > b, staged as {byte offset of row f, byte offset of row g (a row of 1.0 for a
// product: fl(b * 1) = b), a, b}: bit 7 of byte v is set exactly where the condition holds for the
// lane's sample v (bits 0..6 carry no meaning; the walk's constant 0xFFFFFFFF minus the word puts
// the failure in bit 7 without a borrow). The products p, q are separately rounded (packed
// two-lane multiplies); p > q is read as the sign of d = fl(fl(q - p) + 0): for p, q finite or
// infinite, fl(q - p) is negative exactly when p > q (gradual underflow keeps the sign of a tiny
// difference; equal values give +0) except q = -0, p = +0, whose -0 the added +0 turns into +0;
// a NaN operand or inf - inf gives the canonical NaN, whose sign bit is clear (false, as the
// IEEE compare). Used on finite datasets only (rank tables), where the products are finite or
// +-inf.
__device__ __forceinline__ uint32_t pass_row(uint4 q, const unsigned char *xl)
{
    const float4 x = *reinterpret_cast<const float4 *>(xl + q.x);
    const float4 z = *reinterpret_cast<const float4 *>(xl + q.y);
    const float2 a2 = make_float2(__uint_as_float(q.z), __uint_as_float(q.z));
    const float2 b2 = make_float2(__uint_as_float(q.w), __uint_as_float(q.w));
    const float2 m1 = make_float2(-1.f, -1.f), z2 = make_float2(0.f, 0.f);
    const float2 p01 = __fmul2_rn(make_float2(x.x, x.y), a2), p23 = __fmul2_rn(make_float2(x.z, x.w), a2);
    const float2 q01 = __fmul2_rn(make_float2(z.x, z.y), b2), q23 = __fmul2_rn(make_float2(z.z, z.w), b2);
    const float2 d01 = __fadd2_rn(__ffma2_rn(p01, m1, q01), z2);      // fl(q - p) + 0, exactly rounded
    const float2 d23 = __fadd2_rn(__ffma2_rn(p23, m1, q23), z2);
    const uint32_t s01 = __byte_perm(__float_as_uint(d01.x), __float_as_uint(d01.y), 0x0073);
    const uint32_t s23 = __byte_perm(__float_as_uint(d23.x), __float_as_uint(d23.y), 0x0073);
    return __byte_perm(s01, s23, 0x5410);
}

// Pass row of a membership condition, staged as {byte offset of row f, -, set bits 0..31, set
// bits 32..63}: 0xFF in byte v where the lane's sample v holds a category code in the set.
__device__ __forceinline__ uint32_t set_row(uint4 q, const unsigned char *xl)
{
    const float4 x = *reinterpret_cast<const float4 *>(xl + q.x);
    return (category_member(x.x, q.z, q.w) ? 0x000000FFu : 0u) | (category_member(x.y, q.z, q.w) ? 0x0000FF00u : 0u) |
           (category_member(x.z, q.z, q.w) ? 0x00FF0000u : 0u) | (category_member(x.w, q.z, q.w) ? 0xFF000000u : 0u);
}

// One group of four staged records with end-of-rule flags M (bit u: record u ends its rule).
template <uint32_t M, bool UNI>
__device__ __forceinline__ void group4(const uint32_t (&e)[4], const uint32_t *sw, const int32_t *yl,
                                       uint32_t &fail, uint32_t &claimed, uint32_t &hit)
{
    uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
    if (M) w4 = *reinterpret_cast<const uint4 *>(sw);       // the group's four class words at once
    const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        fail |= e[u];
        if (M & (1u << u)) {
            const uint32_t w = ws[u];
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
// one label (kmine) and end records carry the class mask. CAT: the records may hold membership
// tests (without it, a membership record is never packed: the packer rejects op 2 without sets).
//
// The set is walked in chunks of up to 32 records. Staging turns every record of a chunk into the
// same form {byte offset from the lane's rank word, per-byte constant}: a cut points at its rank
// row; a pair or product condition is first evaluated by the whole warp into a pass row
// (0xFF / 0x00 per sample, constant 0xFFFFFFFF) in the warp's `vrow` slots, from a table of the
// chunk's pairs that the lanes build in parallel; padding records are no-ops. The chunk is then one
// straight run of identical steps, with the first-fire claim applied after each rule's last record
// (a warp vote gives their positions); the all-claimed exit is tested once per chunk.
// Work a walk did: records, pair / product / membership rows and rule ends (profiling counters).
struct WalkCount {
    uint32_t records = 0, rows = 0, ends = 0;
};

template <bool UNI, int VS, bool CAT>
__device__ __forceinline__ uint32_t walk_set(uint4 *st, uint32_t *vrow, uint32_t vrow_off, int lane,
                                             const uint4 *recs, int rb, int nrec, const float *us,
                                             uint32_t rev_off, int F, int kmine, const unsigned char *rl,
                                             const unsigned char *xl, uint32_t ones_off, const int32_t *yl,
                                             uint32_t claimed, int deflt, WalkCount &wc)
{
    static_assert(VS <= 16, "pair table and staged records share the warp's 512-byte stage");
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
        uint32_t sm = CAT ? __ballot_sync(FULL, lane < cnt && tag == R5_SET) : 0u;   // membership tests
        if (__popc(pm | sm) > VS) {         // end the chunk before the pass row that finds no slot
            uint32_t m = pm | sm;
            for (int k = 0; k < VS; ++k) m &= m - 1u;
            cnt = __ffs(m) - 1;
            pm &= (1u << cnt) - 1u;
            sm &= (1u << cnt) - 1u;
        }
        const uint32_t ends = __ballot_sync(FULL, lane < cnt && (raw.x & R5_END_BIT) != 0u);
        pf = (c0 + cnt + lane < nrec) ? __ldcg(recs + rb + c0 + cnt + lane) : zero4;

        __syncwarp();                       // the previous chunk's readers of the stage are done
        // every lane runs the cut search (branch-free staging); other records then take their form.
        // A pair or product condition gets a pass-row slot and a pair-table entry.
        const uint32_t cls = (raw.x >> R5_CLS_SHIFT) & 0xFFFu;
        const uint32_t ew = UNI ? ((int)cls == kmine ? 0xFFFFFFFFu : 0u) : cls;
        uint2 sr = stage_cut(raw, us, rev_off, F);
        const int np = __popc(pm);
        if ((pm >> lane) & 1u) {
            const uint32_t slot = __popc(pm & ((1u << lane) - 1u));
            const uint32_t f = min(raw.x & R5_F_MASK, (uint32_t)(F - 1));
            const uint32_t g = min(raw.y, (uint32_t)(F - 1));
            st[slot] = make_uint4(f * (T * 4u), tag == R5_PAIR ? g * (T * 4u) : ones_off, raw.z, raw.w);
            sr = make_uint2(vrow_off + 128u * slot, FULL);
        } else if (CAT && ((sm >> lane) & 1u)) {
            const uint32_t slot = np + __popc(sm & ((1u << lane) - 1u));
            const uint32_t f = min(raw.x & R5_F_MASK, (uint32_t)(F - 1));
            st[slot] = make_uint4(f * (T * 4u), 0u, raw.z, raw.w);
            sr = make_uint2(vrow_off + 128u * slot, FULL);
        } else if (lane >= cnt || tag == R5_NONE) {
            sr = make_uint2(0u, NOOP_K);
        }
        __syncwarp();
        {                                             // pass rows, one warp-wide evaluation each
            uint32_t *vr = vrow + lane;
            for (int j = 0; j < np; j += 2) {
                const uint32_t v0 = pass_row(st[j], xl);
                if (j + 1 < np) vr[32] = pass_row(st[j + 1], xl);
                vr[0] = v0;
                vr += 64;
            }
            if (CAT)
                for (int j = np; j < np + __popc(sm); ++j) vrow[j * 32 + lane] = set_row(st[j], xl);
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
        }
        done = __all_sync(FULL, claimed == HIGH);     // all 128 samples claimed: the set is decided
        c0 += cnt;
        wc.rows += __popc(pm | sm);
        wc.ends += __popc(ends);
    }
    wc.records += c0;
    const uint32_t left = ~claimed & HIGH;
    if (UNI) hit |= (deflt == kmine) ? left : 0u;
    else hit |= left & class_bytes(yl, deflt);
    return hit;
}

}  // namespace rank
}  // namespace rs
