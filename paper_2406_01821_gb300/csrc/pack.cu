// Batch validation and packing: CSR rule sets -> 16-byte condition records + per-set table, and
// the cost order used to schedule sets (largest first).
//
// The exact threshold rewrite. For a finite non-zero coefficient a, the rounded product
// fl(a*x) is a monotone function of x (non-decreasing for a > 0, non-increasing for a < 0):
// the exact product is monotone and round-to-nearest is monotone, including in the subnormal
// and overflow ranges. Hence the set {x : fl(a*x) op t} is an up-set or a down-set of the
// ordered float32 line and equals {x > c} or {x < c} for one float32 c (NaN x is false in both
// forms). c is where the condition's truth changes: looked for first within a few floats of the
// quotient t / a, else by binary search over the 2^32 ordered bit patterns, in both cases by
// evaluating the condition itself with a correctly rounded multiply, so the rewrite is exact by
// construction (and checked exhaustively by rs_selftest_threshold_rewrite).
#include "rs_internal.cuh"

namespace rs {

// Order-preserving map of non-NaN floats to uint32 (-0 and +0 are adjacent).
__device__ inline uint32_t fkey(float x)
{
    uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline float keyf(uint32_t k)
{
    uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(u);
}

__device__ inline bool thr_true(float a, float x, float t, int op)
{
    float p = __fmul_rn(a, x);
    return op == 0 ? (p > t) : (p < t);
}

// The transition of the condition's truth over the ordered float line, searched near the
// correctly rounded quotient t / a: where products are normal numbers it lies within a float or
// two of it. up: false below, true above (returns the last false key); else true below, false
// above (returns the first false key). At most six steps, never past +-inf; a transition is only
// returned once both of its sides were evaluated, and the predicate is monotone with a single
// transition, so the result is the one the binary search finds. false: not found nearby.
__device__ bool transition_near_quotient(float a, float t, int op, bool up, uint32_t &out)
{
    const float q = __fdiv_rn(t, a);
    if (!(fabsf(q) <= 3.0e38f)) return false;
    const uint32_t kmin = fkey(__uint_as_float(0xFF800000u)), kmax = fkey(__uint_as_float(0x7F800000u));
    uint32_t k = fkey(q);
    const auto on = [&](uint32_t kk) { return thr_true(a, keyf(kk), t, op); };
    const bool here = on(k);
    for (int i = 0; i < 6; ++i) {
        if (up == here) {            // on the side the transition is below: step down
            if (k <= kmin) return false;
            if (on(k - 1) != here) { out = up ? k - 1 : k; return true; }
            --k;
        } else {                     // step up
            if (k >= kmax) return false;
            if (on(k + 1) != here) { out = up ? k : k + 1; return true; }
            ++k;
        }
    }
    return false;
}

// Rewrite  fl(a*x) op t  into (kind, v0, v1).
__device__ void rewrite_threshold(float a, float t, int op, uint32_t &kind, float &v0, float &v1)
{
    const float ninf = __uint_as_float(0xFF800000u), pinf = __uint_as_float(0x7F800000u);
    if (isnan(a) || isnan(t)) { kind = KIND_NEVER; v0 = 0.f; v1 = 0.f; return; }
    if (a == 0.f || isinf(a)) { kind = op == 0 ? KIND_MGT : KIND_MLT; v0 = a; v1 = t; return; }
    const bool up = (a > 0.f) == (op == 0);     // condition set is {x > c}
    uint32_t lo = fkey(ninf), hi = fkey(pinf);
    if (up) {
        // false at -inf always; true somewhere iff true at +inf
        if (!thr_true(a, pinf, t, op)) { kind = KIND_NEVER; v0 = 0.f; v1 = 0.f; return; }
        uint32_t k;
        if (transition_near_quotient(a, t, op, true, k)) { kind = KIND_GT; v0 = keyf(k); v1 = 0.f; return; }
        while (hi - lo > 1u) {        // invariant: false at lo, true at hi
            uint32_t mid = lo + (hi - lo) / 2u;
            if (thr_true(a, keyf(mid), t, op)) hi = mid; else lo = mid;
        }
        kind = KIND_GT; v0 = keyf(lo); v1 = 0.f;
    } else {
        // false at +inf always; true somewhere iff true at -inf
        if (!thr_true(a, ninf, t, op)) { kind = KIND_NEVER; v0 = 0.f; v1 = 0.f; return; }
        uint32_t k;
        if (transition_near_quotient(a, t, op, false, k)) { kind = KIND_LT; v0 = keyf(k); v1 = 0.f; return; }
        while (hi - lo > 1u) {        // invariant: true at lo, false at hi
            uint32_t mid = lo + (hi - lo) / 2u;
            if (thr_true(a, keyf(mid), t, op)) lo = mid; else hi = mid;
        }
        kind = KIND_LT; v0 = keyf(hi); v1 = 0.f;
    }
}

__device__ inline bool rec_eval_scalar(uint32_t kind, float v0, float v1, float x)
{
    switch (kind) {
    case KIND_GT: return x > v0;
    case KIND_LT: return x < v0;
    case KIND_MGT: return __fmul_rn(v0, x) > v1;
    case KIND_MLT: return __fmul_rn(v0, x) < v1;
    default: return false;
    }
}

// The v2 form of a threshold condition: fl(v0 * x) > v1 with the same truth value for every x.
// A '<' cut c becomes -x > -c and a '<' product becomes fl(-a * x) > -t (negation is exact).
__device__ void rewrite_lin(float a, float t, int op, float &v0, float &v1)
{
    uint32_t kind;
    float c0, c1;
    rewrite_threshold(a, t, op, kind, c0, c1);
    switch (kind) {
    case KIND_GT: v0 = 1.f; v1 = c0; break;
    case KIND_LT: v0 = -1.f; v1 = -c0; break;
    case KIND_MGT: v0 = c0; v1 = c1; break;
    case KIND_MLT: v0 = -c0; v1 = -c1; break;
    default: v0 = 0.f; v1 = __uint_as_float(0x7F800000u); break;   // never true
    }
}

// Pack v2 records: one thread per rule.
__global__ void k_pack_rules2(BatchDev b, int F, int K, int S, int form, Rec *recs_out, uint32_t *status)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (b.dR) { b.R = *b.dR; b.C = *b.dC; }
    if (r >= b.R) return;
    const int c0 = b.rule_cond_off[r], c1 = b.rule_cond_off[r + 1];
    if (c0 < 0 || c1 < c0 || c1 > b.C) { atomicOr(status, ST_BAD_OFFSETS); return; }
    if (c1 - c0 > 0xFFF) { atomicOr(status, ST_TOO_LARGE); return; }
    int cls = b.rule_class[r];
    if (cls < 0 || cls >= K) { atomicOr(status, ST_BAD_CLASS); cls = 0; }
    uint4 *out = reinterpret_cast<uint4 *>(recs_out);
    const uint32_t len = (uint32_t)(c1 - c0);
    const uint32_t row16 = (uint32_t)S / 4;   // 16-byte units per feature row
    for (int c = c0; c < c1; ++c) {
        const int f = b.cond_f[c], g = b.cond_g[c], op = b.cond_op[c];
        uint32_t w0 = len << LEN_SHIFT, w1 = (uint32_t)cls << CLS_SHIFT;
        float v0 = 0.f, v1 = __uint_as_float(0x7F800000u);   // never true
        if (f < 0 || f >= F || g < -1 || g >= F) {
            atomicOr(status, ST_BAD_FEATURE);
        } else if (op != 0 && op != 1) {
            atomicOr(status, ST_BAD_OP);
        } else if (g < 0 && form == 4) {
            // cut form: x > c  <=>  sign(fl(+-x - c')) clear with c' = nextup(+-c)
            uint32_t kind;
            float c0, c1;
            rewrite_threshold(b.cond_a[c], b.cond_t[c], op, kind, c0, c1);
            const float pinf = __uint_as_float(0x7F800000u);
            if (kind == KIND_GT) { v0 = 1.f; v1 = -nextafterf(c0, pinf); }
            else if (kind == KIND_LT) { v0 = -1.f; v1 = -nextafterf(-c0, pinf); }
            else { rewrite_lin(b.cond_a[c], b.cond_t[c], op, v0, v1); w0 |= GENERAL_BIT; }
            w0 |= (uint32_t)f * row16;
        } else if (g < 0) {
            rewrite_lin(b.cond_a[c], b.cond_t[c], op, v0, v1);
            w0 |= (uint32_t)f * row16;
        } else {
            const int lf = op == 0 ? f : g, rg = op == 0 ? g : f;
            v0 = op == 0 ? b.cond_a[c] : b.cond_b[c];
            v1 = op == 0 ? b.cond_b[c] : b.cond_a[c];
            w0 |= ((uint32_t)lf * row16) | PAIR_BIT;
            w1 |= (uint32_t)rg * row16;
        }
        out[c] = make_uint4(w0, w1, __float_as_uint(v0), __float_as_uint(v1));
    }
}


// Order buckets of the counting sort of sets by cost (k_order, and k_pack_sets for one-block batches).
constexpr int ORDER_BUCKETS = 1024;
__device__ __forceinline__ int order_bucket(int cost) { return ORDER_BUCKETS - 1 - min(cost, ORDER_BUCKETS - 1); }

// Exclusive prefix sum over the bucket counts in place, by the whole block (blockDim.x a multiple
// of 32 that divides ORDER_BUCKETS; every thread of the block calls it).
__device__ void scan_buckets(int *hist)
{
    __shared__ int warp_sums[32];
    const int per = ORDER_BUCKETS / blockDim.x;
    const int base = threadIdx.x * per;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int local = 0;
    for (int i = 0; i < per; ++i) local += hist[base + i];
    int x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    int run = x - local + (warp ? warp_sums[warp - 1] : 0);
    for (int i = 0; i < per; ++i) {
        const int h = hist[base + i];
        hist[base + i] = run;
        run += h;
    }
    __syncthreads();
}

// Offsets, default class and first empty rule of set p (an empty rule fires for every sample
// still unclaimed, so the set effectively ends there with that class as its default). Returns
// the set's cost (its record count).
__device__ int pack_one_set(const BatchDev &b, int K, int p, SetInfo *sets, int32_t *last_end, uint32_t *status)
{
    SetInfo si{0, 0, 0, 0};
    const int rb = b.set_rule_off[p], re = b.set_rule_off[p + 1];
    int d = b.set_default[p];
    if (d < 0 || d >= K) { atomicOr(status, ST_BAD_CLASS); d = 0; }
    si.deflt = d;
    if (rb < 0 || re < rb || re > b.R) {
        atomicOr(status, ST_BAD_OFFSETS);
        sets[p] = si;
        return 0;
    }
    int c_begin = 0, c_end = 0;
    bool ok = true;
    if (last_end)
        for (int k = 0; k < K; ++k) last_end[(int64_t)p * K + k] = 0;
    for (int r = rb; r < re; ++r) {
        const int c0 = b.rule_cond_off[r], c1 = b.rule_cond_off[r + 1];
        if (c0 < 0 || c1 < c0 || c1 > b.C) { ok = false; break; }
        if (c1 - c0 > 0xFFF) { atomicOr(status, ST_TOO_LARGE); ok = false; break; }
        if (r == rb) { c_begin = c0; c_end = c0; }
        const int cls = b.rule_class[r];
        if (cls < 0 || cls >= K) { atomicOr(status, ST_BAD_CLASS); ok = false; break; }
        if (c1 == c0) { si.deflt = cls; break; }   // empty rule: fires on everything left
        c_end = c1;
        if (last_end) last_end[(int64_t)p * K + cls] = c1 - c_begin;
    }
    if (!ok) {
        atomicOr(status, ST_BAD_OFFSETS);
        c_begin = c_end = 0;
        if (last_end)
            for (int k = 0; k < K; ++k) last_end[(int64_t)p * K + k] = 0;
    } else if (last_end) {
        // for the default class d: the end of the last rule of any other class (after it every rule
        // left names d, and so does the default: every sample still unclaimed counts for d)
        int m = 0;
        for (int k = 0; k < K; ++k)
            if (k != si.deflt) m = max(m, last_end[(int64_t)p * K + k]);
        last_end[(int64_t)p * K + si.deflt] = m;
    }
    si.rec_begin = c_begin;
    si.rec_end = c_end;
    si.cost = c_end - c_begin;
    sets[p] = si;
    return si.cost;
}

// One thread per set: the set's descriptor, and zeroed counts (correct[p], per_class[p][*]) when
// the output pointers are given. With `order_here` (a batch of at most one block) the block also
// sorts the sets by cost, which otherwise k_order does in a launch of its own.
__global__ void k_pack_sets(BatchDev b, int K, PackOut o, bool order_here)
{
    __shared__ int hist[ORDER_BUCKETS];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (b.dR) { b.R = *b.dR; b.C = *b.dC; }
    if (p == 0) {
        if (b.set_rule_off[0] != 0 || b.set_rule_off[b.P] != b.R ||
            b.rule_cond_off[0] != 0 || b.rule_cond_off[b.R] != b.C)
            atomicOr(o.status, ST_BAD_OFFSETS);
    }
    int cost = 0;
    if (p < b.P) {
        if (o.correct) o.correct[p] = 0;
        if (o.per_class)
            for (int k = 0; k < K; ++k) o.per_class[(int64_t)p * K + k] = 0;
        cost = pack_one_set(b, K, p, o.sets, o.last_end, o.status);
    }
    if (!order_here) return;   // uniform over the launch
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    if (p < b.P) atomicAdd(&hist[order_bucket(cost)], 1);
    __syncthreads();
    scan_buckets(hist);
    if (p < b.P) o.order[atomicAdd(&hist[order_bucket(cost)], 1)] = p;
}

// Kind of a condition in format v5, decided with the same tests as rewrite_threshold (without its
// search): R5_CUT_GT / R5_CUT_LT for a +-cut, R5_PAIR, R5_SET for a category membership test,
// or R5_GEN for everything else (zero or infinite coefficient, never-true conditions, invalid
// input).
__device__ uint32_t kind5(const BatchDev &b, int c, int F)
{
    const int f = b.cond_f[c], g = b.cond_g[c], op = b.cond_op[c];
    if (op == RS_OP_IN && b.cond_set && g == -1 && f >= 0 && f < F) return R5_SET;
    if (f < 0 || f >= F || g < -1 || g >= F || (op != 0 && op != 1)) return R5_GEN;
    if (g >= 0) return R5_PAIR;
    const float a = b.cond_a[c], t = b.cond_t[c];
    if (isnan(a) || isnan(t) || a == 0.f || isinf(a)) return R5_GEN;
    const bool up = (a > 0.f) == (op == 0);
    const float end = up ? __uint_as_float(0x7F800000u) : __uint_as_float(0xFF800000u);
    if (!thr_true(a, end, t, op)) return R5_GEN;
    return up ? R5_CUT_GT : R5_CUT_LT;
}

// Pack v5 records, one thread per rule: the cuts, the pairs and the remaining conditions (a
// conjunction does not depend on the order of its conditions); the rule's last record carries
// the end-of-rule flag and the rule class.
__global__ void k_pack_rules5(BatchDev b, int F, int K, Rec *recs_out, uint32_t *status)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (b.dR) { b.R = *b.dR; b.C = *b.dC; }
    if (r >= b.R) return;
    const int c0 = b.rule_cond_off[r], c1 = b.rule_cond_off[r + 1];
    if (c0 < 0 || c1 < c0 || c1 > b.C) { atomicOr(status, ST_BAD_OFFSETS); return; }
    if (c1 - c0 > 0xFFF) { atomicOr(status, ST_TOO_LARGE); return; }
    int cls = b.rule_class[r];
    if (cls < 0 || cls >= K) { atomicOr(status, ST_BAD_CLASS); cls = 0; }
    uint4 *out = reinterpret_cast<uint4 *>(recs_out);
    int ncut = 0, npair = 0;
    for (int c = c0; c < c1; ++c) {
        const uint32_t k = kind5(b, c, F);
        ncut += (k == R5_CUT_GT || k == R5_CUT_LT);
        npair += (k == R5_PAIR);
    }
    int qc = c0, qp = c0 + ncut, qg = c0 + ncut + npair;
    const float pinf = __uint_as_float(0x7F800000u);
    for (int c = c0; c < c1; ++c) {
        const uint32_t k = kind5(b, c, F);
        const int f = b.cond_f[c], g = b.cond_g[c], op = b.cond_op[c];
        int q;
        uint4 rec;
        if (k == R5_CUT_GT || k == R5_CUT_LT) {
            uint32_t kind;
            float cut, unused;
            rewrite_threshold(b.cond_a[c], b.cond_t[c], op, kind, cut, unused);
            // x < c  <=>  x <= nextdown(c) for non-NaN x: both cut kinds then count tile values <= w2
            if (k == R5_CUT_LT) cut = nextafterf(cut, __uint_as_float(0xFF800000u));
            rec = make_uint4((k << R5_TAG_SHIFT) | (uint32_t)f, 0u, __float_as_uint(cut), 0u);
            q = qc++;
        } else if (k == R5_PAIR) {
            const int lf = op == 0 ? f : g, rg = op == 0 ? g : f;
            const float a = op == 0 ? b.cond_a[c] : b.cond_b[c];
            const float bb = op == 0 ? b.cond_b[c] : b.cond_a[c];
            rec = make_uint4((R5_PAIR << R5_TAG_SHIFT) | (uint32_t)lf, (uint32_t)rg, __float_as_uint(a),
                             __float_as_uint(bb));
            q = qp++;
        } else if (k == R5_SET) {
            const uint64_t set = b.cond_set[c];
            rec = make_uint4((R5_SET << R5_TAG_SHIFT) | (uint32_t)f, 0u, (uint32_t)set, (uint32_t)(set >> 32));
            q = qg++;
        } else {
            float v0 = 0.f, v1 = pinf;   // never true
            uint32_t rf = 0;
            if (f < 0 || f >= F || g < -1 || g >= F) atomicOr(status, ST_BAD_FEATURE);
            else if (op != 0 && op != 1) atomicOr(status, ST_BAD_OP);
            else { rewrite_lin(b.cond_a[c], b.cond_t[c], op, v0, v1); rf = (uint32_t)f; }
            rec = make_uint4((R5_GEN << R5_TAG_SHIFT) | rf, 0u, __float_as_uint(v0), __float_as_uint(v1));
            q = qg++;
        }
        if (q == c1 - 1) rec.x |= R5_END_BIT | ((uint32_t)cls << R5_CLS_SHIFT);
        out[q] = rec;
    }
}

// One thread per rule: build the records of its conditions.
__global__ void k_pack_rules(BatchDev b, int F, int K, Rec *recs, uint32_t *status)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (b.dR) { b.R = *b.dR; b.C = *b.dC; }
    if (r >= b.R) return;
    const int c0 = b.rule_cond_off[r], c1 = b.rule_cond_off[r + 1];
    if (c0 < 0 || c1 < c0 || c1 > b.C) { atomicOr(status, ST_BAD_OFFSETS); return; }
    if (c1 - c0 > 0xFFF) { atomicOr(status, ST_TOO_LARGE); return; }    // rule length is 12 bits
    int cls = b.rule_class[r];
    if (cls < 0 || cls >= K) { atomicOr(status, ST_BAD_CLASS); cls = 0; }
    for (int c = c0; c < c1; ++c) {
        const int f = b.cond_f[c], g = b.cond_g[c], op = b.cond_op[c];
        Rec rec;
        uint32_t kind = KIND_NEVER;
        float v0 = 0.f, v1 = 0.f;
        int rf = 0, rg = 0;
        if (f < 0 || f >= F || g < -1 || g >= F) {
            atomicOr(status, ST_BAD_FEATURE);
        } else if (op == RS_OP_IN && b.cond_set && g == -1) {
            const uint64_t set = b.cond_set[c];
            kind = KIND_IN;
            v0 = __uint_as_float((uint32_t)set);
            v1 = __uint_as_float((uint32_t)(set >> 32));
            rf = f;
        } else if (op != 0 && op != 1) {
            atomicOr(status, ST_BAD_OP);
        } else if (g < 0) {
            rewrite_threshold(b.cond_a[c], b.cond_t[c], op, kind, v0, v1);
            rf = f;
        } else if (op == 0) {      // a*x[f] > b*x[g]
            kind = KIND_PAIR; rf = f; rg = g; v0 = b.cond_a[c]; v1 = b.cond_b[c];
        } else {                   // a*x[f] < b*x[g]  <=>  b*x[g] > a*x[f]
            kind = KIND_PAIR; rf = g; rg = f; v0 = b.cond_b[c]; v1 = b.cond_a[c];
        }
        const uint32_t last = (c == c1 - 1) ? 1u : 0u;
        const uint32_t skip = (uint32_t)min(c1 - 1 - c, 0xFFFF);
        rec.meta = kind | (last << 3) | ((uint32_t)cls << 4) | (skip << 16);
        rec.f = (uint16_t)rf;
        rec.g = (uint16_t)rg;
        rec.v0 = v0;
        rec.v1 = v1;
        recs[c] = rec;
    }
}

// Single-CTA counting sort of sets by cost, most expensive first (bucketed; the order only
// schedules work, results do not depend on it).
__global__ void k_order(const SetInfo *sets, int P, int32_t *order)
{
    __shared__ int hist[ORDER_BUCKETS];
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) atomicAdd(&hist[order_bucket(sets[p].cost)], 1);
    __syncthreads();
    scan_buckets(hist);
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        int pos = atomicAdd(&hist[order_bucket(sets[p].cost)], 1);
        order[pos] = p;
    }
}

int launch_pack(const BatchDev &b, int F, int K, int S, int ver, const PackOut &o, cudaStream_t stream)
{
    int n = 0;
    constexpr int SET_BLOCK = 256;
    const bool order_here = o.order && b.P <= SET_BLOCK;
    if (b.P > 0) { k_pack_sets<<<(b.P + SET_BLOCK - 1) / SET_BLOCK, SET_BLOCK, 0, stream>>>(b, K, o, order_here); ++n; }
    if (b.R > 0 && ver == 5) {
        k_pack_rules5<<<(b.R + 127) / 128, 128, 0, stream>>>(b, F, K, o.recs, o.status);
        ++n;
    } else if (b.R > 0 && ver >= 2) {
        k_pack_rules2<<<(b.R + 127) / 128, 128, 0, stream>>>(b, F, K, S, ver == 4 ? 4 : 2, o.recs, o.status);
        ++n;
    } else if (b.R > 0) {
        k_pack_rules<<<(b.R + 127) / 128, 128, 0, stream>>>(b, F, K, o.recs, o.status);
        ++n;
    }
    if (b.P > 0 && o.order && !order_here) { k_order<<<1, 1024, 0, stream>>>(o.sets, b.P, o.order); ++n; }
    return n;
}

// --------------------------------------------------------------- exhaustive rewrite self-check

// Rewrite once per entry, then sweep x.
__global__ void k_rewrite_table(const float *a, const float *t, const int8_t *op, int n,
                                uint32_t *kind, float *v0, float *v1)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) rewrite_threshold(a[j], t[j], op[j], kind[j], v0[j], v1[j]);
}

__global__ void k_sweep(const float *a, const float *t, const int8_t *op, const uint32_t *kind,
                        const float *v0, const float *v1, int j, unsigned long long *mismatches)
{
    uint64_t local = 0;
    const float aj = a[j], tj = t[j];
    const int oj = op[j];
    const uint32_t kj = kind[j];
    const float c0 = v0[j], c1 = v1[j];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32);
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float x = __uint_as_float((uint32_t)i);
        local += (thr_true(aj, x, tj, oj) != rec_eval_scalar(kj, c0, c1, x));
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(mismatches, (unsigned long long)local);
}

rs_status selftest_rewrite(const float *a_h, const float *t_h, const int8_t *op_h, int n,
                           uint64_t *mismatches, int sm_count)
{
    float *a = nullptr, *t = nullptr, *v0 = nullptr, *v1 = nullptr;
    int8_t *op = nullptr;
    uint32_t *kind = nullptr;
    unsigned long long *mm = nullptr;
    RS_CUDA(cudaMalloc(&a, sizeof(float) * n));
    RS_CUDA(cudaMalloc(&t, sizeof(float) * n));
    RS_CUDA(cudaMalloc(&v0, sizeof(float) * n));
    RS_CUDA(cudaMalloc(&v1, sizeof(float) * n));
    RS_CUDA(cudaMalloc(&op, n));
    RS_CUDA(cudaMalloc(&kind, sizeof(uint32_t) * n));
    RS_CUDA(cudaMalloc(&mm, sizeof(unsigned long long)));
    RS_CUDA(cudaMemcpy(a, a_h, sizeof(float) * n, cudaMemcpyHostToDevice));
    RS_CUDA(cudaMemcpy(t, t_h, sizeof(float) * n, cudaMemcpyHostToDevice));
    RS_CUDA(cudaMemcpy(op, op_h, n, cudaMemcpyHostToDevice));
    RS_CUDA(cudaMemset(mm, 0, sizeof(unsigned long long)));
    k_rewrite_table<<<(n + 127) / 128, 128>>>(a, t, op, n, kind, v0, v1);
    for (int j = 0; j < n; ++j) k_sweep<<<sm_count * 8, 256>>>(a, t, op, kind, v0, v1, j, mm);
    unsigned long long h = 0;
    RS_CUDA(cudaMemcpy(&h, mm, sizeof(h), cudaMemcpyDeviceToHost));
    cudaFree(a); cudaFree(t); cudaFree(v0); cudaFree(v1); cudaFree(op); cudaFree(kind); cudaFree(mm);
    *mismatches = h;
    return RS_OK;
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_pack_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_pack_rules);
    cudaFuncGetAttributes(&fa, k_pack_rules2);
    cudaFuncGetAttributes(&fa, k_pack_rules5);
    cudaFuncGetAttributes(&fa, k_pack_sets);
    cudaFuncGetAttributes(&fa, k_order);
}

}  // namespace rs
