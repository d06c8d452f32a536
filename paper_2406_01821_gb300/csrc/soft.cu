// The soft path: sigmoid-relaxed first-fire evaluation (forward) and its hand-written adjoint.
//
// Per condition  u = s*(a*x[f] - rhs)/tau  (s = +1 for '>', -1 for '<'; rhs = t or b*x[g]).
// Per rule       lq_r = sum_c log sigmoid(u_c)      (log of the firing probability q_r)
//                l1q_r = log(1 - q_r) = log(-expm1(lq_r))
//                lu_r = sum_{j<r} l1q_j             (log probability that no earlier rule fired)
// Class k        log p_k = logsumexp over rules of class k of (lq_r + lu_r), plus lu_R for the
//                default class.  Loss  L_p = (1/N) sum_n -log p_{y_n}.
// Adjoint        S_r = P(outcome y | evaluation starts at rule r), T_r = 1 - S_r, both kept as logs
//                and both sums of positive terms:
//                  lS_R = 0 if default = y else -inf;  lS_r = logsumexp([cls_r = y] lq_r, l1q_r + lS_{r+1})
//                  lT_R = 0 if default != y else -inf; lT_r = logsumexp([cls_r != y] lq_r, l1q_r + lT_{r+1})
//                dl/dlq_r = exp(lq_r + lu_r - lp) * (S_{r+1} - [cls_r = y])
//                         =  exp(lq_r + lu_r + lS_{r+1} - lp)   if cls_r != y
//                         = -exp(lq_r + lu_r + lT_{r+1} - lp)   if cls_r  = y
//                (the second form avoids the cancellation of S_{r+1} - 1 when S_{r+1} is near 1)
//                dl/du_c  = dl/dlq_r * sigmoid(-u_c);  du/da = s x_f / tau, du/dt = -s / tau,
//                du/db = -s x_g / tau.
// Everything is evaluated in float32 in the log domain, which keeps 1 - q_r and the products of
// many sigmoids representable where the linear form underflows. A float32 log-probability of
// magnitude L is only known to about L * 2^-24, and at large margins (fine-tuned coefficients)
// L reaches thousands while the probabilities that make up the gradient are ratios of such
// values: a 64-sample group in which some sample's log p_y exceeds SOFT_FF_LIMIT in magnitude
// (or is not finite) is evaluated again in float-float arithmetic (about 48 significant bits),
// with the margins formed exactly, 1 - q_r taken as a log-sum-exp of -u_c when q_r rounds to 1,
// and each d ell / d u_c formed in the exponent (soft_group_ff). Other groups keep the float path.
//
// Work: one warp owns a (rule set, sample chunk) pair and walks the chunk 64 samples at a time
// (two per lane), so each partial sum has a fixed summation order. The forward keeps lu_r per
// rule and sample; the adjoint computes lq_r again from the conditions. Chunks are a function of N
// only; partial losses and gradients per chunk are reduced in a second kernel in a fixed order,
// which makes results bit-reproducible run to run and independent of scheduling.
#include "rs_internal.cuh"
#include "soft_step.cuh"
#include "block_scan.cuh"

namespace rs {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int SOFT_W = 4;                 // warps per CTA
constexpr int SOFT_MAX_RULES = 64;        // rules per set held in shared memory
constexpr int SOFT_MAX_CONDS = 512;       // conditions per set accumulated in shared memory
constexpr int SOFT_MAX_CHUNKS = 128;
constexpr int SOFT_V = 2;                 // samples per lane; a group is 32 * SOFT_V samples
constexpr int SOFT_G = 32 * SOFT_V;

// Floats of a warp's shared arrays: lu [maxR + 1][G], acc [maxC][4], and lq [maxR][G] when the
// class probabilities are written.
__host__ __device__ constexpr size_t soft_per_warp(int maxR, int maxC, bool with_lq)
{
    return (size_t)(maxR + 1) * SOFT_G + (size_t)maxC * 4 + (with_lq ? (size_t)maxR * SOFT_G : 0);
}

struct __align__(16) SoftRec {
    uint32_t meta;    // bit 0: pair condition, bit 1: '<', bit 2: category membership
    uint16_t f, g;
    float a, bt;      // bt = threshold t, or the pair coefficient b; a membership test holds the
                      // bits of its category set (0..31 in a, 32..63 in bt)
};

__global__ void k_pack_soft(BatchDev b, int F, int K, SoftRec *recs, uint32_t *status, int32_t *work_counter)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) *work_counter = 0;            // the soft kernel's task counter
    if (b.dR) { b.R = *b.dR; b.C = *b.dC; }
    if (c >= b.C) return;
    const int f = b.cond_f[c], g = b.cond_g[c], op = b.cond_op[c];
    SoftRec r{0, 0, 0, 0.f, 0.f};
    if (f < 0 || f >= F || g < -1 || g >= F) atomicOr(status, ST_BAD_FEATURE);
    else if (op == RS_OP_IN && b.cond_set && g == -1) {
        const uint64_t set = b.cond_set[c];
        r.meta = 4u;
        r.f = (uint16_t)f;
        r.a = __uint_as_float((uint32_t)set);
        r.bt = __uint_as_float((uint32_t)(set >> 32));
    } else if (op != 0 && op != 1) atomicOr(status, ST_BAD_OP);
    else {
        r.meta = (g >= 0 ? 1u : 0u) | (op == 1 ? 2u : 0u);
        r.f = (uint16_t)f;
        r.g = (uint16_t)(g >= 0 ? g : 0);
        r.a = b.cond_a[c];
        r.bt = g >= 0 ? b.cond_b[c] : b.cond_t[c];
    }
    recs[c] = r;
}

// Validation of the set/rule structure (one thread per set).
// Single-CTA counting sort of the sets by size (rules + conditions, most first), so that the
// warps of one CTA group walk sets of similar length. Malformed offsets count as size 0 (the
// check kernel rejects the batch).
constexpr int SOFT_ORDER_BUCKETS = 1024;
__global__ void k_soft_order(BatchDev b, int32_t *order)
{
    __shared__ int hist[SOFT_ORDER_BUCKETS];
    const int R = b.dR ? *b.dR : b.R, C = b.dC ? *b.dC : b.C;
    for (int i = threadIdx.x; i < SOFT_ORDER_BUCKETS; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    auto bucket = [&](int p) {
        const int rb = b.set_rule_off[p], re = b.set_rule_off[p + 1];
        int cost = 0;
        if (rb >= 0 && re >= rb && re <= R) {
            const int cb = b.rule_cond_off[rb], ce = b.rule_cond_off[re];
            if (cb >= 0 && ce >= cb && ce <= C) cost = (re - rb) + (ce - cb);
        }
        return SOFT_ORDER_BUCKETS - 1 - min(cost, SOFT_ORDER_BUCKETS - 1);
    };
    for (int p = threadIdx.x; p < b.P; p += blockDim.x) atomicAdd(&hist[bucket(p)], 1);
    __syncthreads();
    block_exclusive_scan_array(hist, SOFT_ORDER_BUCKETS);
    for (int p = threadIdx.x; p < b.P; p += blockDim.x) order[atomicAdd(&hist[bucket(p)], 1)] = p;
}

__global__ void k_check_sets_soft(BatchDev b, int K, uint32_t *status, int32_t *maxima, int maxR,
                                  int maxC)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (b.dR) { b.R = *b.dR; b.C = *b.dC; }
    if (p == 0) {
        if (b.set_rule_off[0] != 0 || b.set_rule_off[b.P] != b.R ||
            b.rule_cond_off[0] != 0 || b.rule_cond_off[b.R] != b.C)
            atomicOr(status, ST_BAD_OFFSETS);
    }
    if (p >= b.P) return;
    const int rb = b.set_rule_off[p], re = b.set_rule_off[p + 1];
    const int d = b.set_default[p];
    if (d < 0 || d >= K) atomicOr(status, ST_BAD_CLASS);
    if (rb < 0 || re < rb || re > b.R) { atomicOr(status, ST_BAD_OFFSETS); return; }
    if (re - rb > SOFT_MAX_RULES) { atomicOr(status, ST_TOO_LARGE); return; }
    for (int r = rb; r < re; ++r) {
        const int c0 = b.rule_cond_off[r], c1 = b.rule_cond_off[r + 1];
        if (c0 < 0 || c1 < c0 || c1 > b.C) { atomicOr(status, ST_BAD_OFFSETS); return; }
        const int cls = b.rule_class[r];
        if (cls < 0 || cls >= K) atomicOr(status, ST_BAD_CLASS);
    }
    const int nc = re > rb ? b.rule_cond_off[re] - b.rule_cond_off[rb] : 0;
    if (nc > SOFT_MAX_CONDS || re - rb > maxR || nc > maxC) atomicOr(status, ST_TOO_LARGE);
    atomicMax(&maxima[0], re - rb);
    atomicMax(&maxima[1], nc);
}

// log(1 + e) for 0 <= e <= 1 as e p(e), with p the polynomial of degree 8 of least maximum
// relative error against log1p(e) / e on [0, 1] (Remez exchange, 3.0e-8 before its coefficients
// were rounded to float32), evaluated by Horner's rule in fused multiply-adds: within 2 ulp of
// log1p over the interval, and e p(e) keeps the relative accuracy of log1p(e) = e (1 - e/2 + ...)
// as e goes to 0. No division and no special case.
__device__ __forceinline__ float log1p_unit(float e)
{
    float p = 5.232694093e-03f;
    p = fmaf(p, e, -2.950523794e-02f);
    p = fmaf(p, e, 7.822595537e-02f);
    p = fmaf(p, e, -1.366324574e-01f);
    p = fmaf(p, e, 1.910600662e-01f);
    p = fmaf(p, e, -2.484298199e-01f);
    p = fmaf(p, e, 3.331909776e-01f);
    p = fmaf(p, e, -4.999949336e-01f);
    p = fmaf(p, e, 9.999999404e-01f);
    return e * p;
}

// The float path's exponentials of non-positive arguments use the hardware approximation
// (__expf: ex2.approx of x log2(e)); for the arguments that occur here (|x| up to about 100,
// beyond which the float-float pass takes over for the terms that matter) its relative error
// stays below a few 1e-6, within the soft tolerance. Logarithms stay accurate (the hardware lg2
// has an absolute error near 1 that is too large relative to log1p of small arguments); the
// float-float pass keeps expf.
__device__ __forceinline__ float exp_np(float x) { return __expf(x); }

// log(1 - e^s) for s <= 0: the log-probability that a rule whose conditions hold with
// probability q = e^s does not fire. Both pieces are evaluated and one is selected (a warp's
// samples fall on both sides):
// * q <= e^(-1/2): log1p(-q) = -q a(q), a the degree-10 polynomial of least maximum relative
//   error against -log1p(-q) / q on [0, e^(-1/2)] (Remez exchange; within 2 ulp given q). q comes
//   from the hardware exponential, whose relative error (a few 1e-6 at most for the arguments
//   that matter) becomes that of the result: an absolute error below 1e-7 in the log domain.
// * t = -s < 1/2: log t + t b(t), b the degree-3 polynomial of least maximum relative error
//   against log((1 - e^-t) / t) / t on [0, 1/2]; log t = k ln 2 + log m for t = m 2^k, 1 <= m < 2,
//   with log m from the hardware logarithm, whose error on [1, 2] is at most 2^-21.41 absolute,
//   whatever k: as t goes to 0 the absolute error stays at that level instead of growing with
//   |log t| (lu, a sum of these terms, is an absolute quantity in the log domain).
// s = 0 gives -inf (the rule fires for certain), s = -inf gives -0.
__device__ __forceinline__ float log1m_exp(float s)
{
    const float t = -s;
    const float q = exp_np(s);
    float pa = 5.805101871e+00f;
    pa = fmaf(pa, q, -1.336368465e+01f);
    pa = fmaf(pa, q, 1.424522972e+01f);
    pa = fmaf(pa, q, -8.279889107e+00f);
    pa = fmaf(pa, q, 3.204409838e+00f);
    pa = fmaf(pa, q, -5.293834209e-01f);
    pa = fmaf(pa, q, 2.968223989e-01f);
    pa = fmaf(pa, q, 2.422454804e-01f);
    pa = fmaf(pa, q, 3.336488008e-01f);
    pa = fmaf(pa, q, 4.999950230e-01f);
    pa = fmaf(pa, q, 1.000000000e+00f);
    const float ra = -q * pa;
    float pb = -3.432709782e-04f;
    pb = fmaf(pb, t, -1.679248726e-06f);
    pb = fmaf(pb, t, 4.166686162e-02f);
    pb = fmaf(pb, t, -5.000000000e-01f);
    const bool sub = t < 0x1p-126f;                  // subnormal t: scaled by 2^24 first
    const int it = __float_as_int(sub ? t * 0x1p24f : t);
    const float k = (float)((it >> 23) - (sub ? 127 + 24 : 127));
    const float m = __int_as_float((it & 0x007FFFFF) | 0x3F800000);
    const float lt = fmaf(k, 6.931471825e-01f, fmaf(k, -1.904654212e-09f, __logf(m)));   // ln 2 as hi + lo
    const float rb = t == 0.f ? -INFINITY : fmaf(t, pb, lt);
    return t >= 0.5f ? ra : rb;
}

// The soft kernels' elementary functions evaluated on the device (test hooks): 0 = log1p_unit,
// 1 = log1m_exp.
__global__ void k_selftest_soft_math(const float *in, int n, float *out, int which)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = which == 0 ? log1p_unit(in[i]) : log1m_exp(in[i]);
}

__device__ __forceinline__ float log_sigmoid(float u)
{
    // log(1/(1+e^-u)) = -(max(-u,0) + log1p(e^-|u|))
    const float e = exp_np(-fabsf(u));
    return -(fmaxf(-u, 0.f) + log1p_unit(e));
}

__device__ __forceinline__ float sigmoid_neg(float u)     // 1/(1+e^u)
{
    const float e = exp_np(-fabsf(u));
    return __fdividef(u >= 0.f ? e : 1.f, 1.f + e);
}

__device__ __forceinline__ float log_add(float a, float b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    const float m = fmaxf(a, b);
    return m + log1p_unit(exp_np(-fabsf(a - b)));
}

// Kahan-compensated accumulation.
__device__ __forceinline__ void kadd(float &s, float &c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// The same for the loss, whose terms may be +inf (a label no path reaches): an infinite sum stays
// infinite rather than turning NaN.
__device__ __forceinline__ void kadd_loss(float &s, float &c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = isinf(t) ? 0.f : (t - s) - y;
    s = t;
}

struct SoftKArgs {
    const SoftRec *recs;
    const int32_t *set_rule_off, *rule_cond_off, *rule_class, *set_default;
    int32_t P;
    const float *Xt;
    const int32_t *y;
    const int32_t *perm;
    int64_t N, n_pad;
    int32_t K;
    float inv_tau;
    float inv_tau_lo;                // 1/tau - inv_tau (float-float path)
    int32_t nchunks, chunk;          // chunk = samples per chunk (multiple of 32)
    float *part_loss;                // [nchunks][P]
    float *part_ga, *part_gbt;       // [nchunks][C]
    float *probs;                    // [P*N*K] or null
    int32_t backward;
    int32_t *next;                   // work counter
    int32_t maxR, maxC;              // shared-memory capacity per warp (rules, conditions)
    int64_t Ccap;                    // row stride of the gradient partials
    const uint32_t *status;          // no work if non-zero (malformed batch)
    const int32_t *order;            // sets by decreasing size (schedule only; results do not depend on it)
    uint8_t *ffmark;                 // [nchunks][P]: the task left groups to the float-float pass
    uint32_t *ffbits;                // [nchunks][P][ff_wpt]: bit g of a task: its group g is one of them
    int32_t ff_wpt;                  // words per task (groups per chunk / 32, rounded up)
};

// Feature access for one group of 64 samples: the lane's first sample column either in global
// memory (x[f] at col[f * stride]) or in a staged shared-memory tile [F][64] (stride 64); its
// second sample is 32 columns further.
struct XView {
    const float *col;
    int64_t stride;
    // x[f] of the lane's sample v (32 v samples after its first)
    __device__ __forceinline__ float operator()(int f, int v) const { return col[(int64_t)f * stride + 32 * v]; }
};

// The lane's sample v: (d ell / d a, d ell / d b or d t) of condition rc, given d ell / d log q of
// its rule.
__device__ __forceinline__ float2 cond_grad(const SoftKArgs &a, const SoftRec &rc, const XView &x, int v, float gq)
{
    const float xf = x(rc.f, v);
    const bool pair = rc.meta & 1u;
    const float xg = pair ? x(rc.g, v) : 0.f;
    const float lhs = rc.a * xf;
    const float rhs = pair ? rc.bt * xg : rc.bt;
    const float sg = (rc.meta & 2u) ? -1.f : 1.f;
    const float u = sg * (lhs - rhs) * a.inv_tau;
    const float du = gq * sigmoid_neg(u) * sg * a.inv_tau;
    return make_float2(du * xf, pair ? -du * xg : -du);
}

// log q of one rule (its conditions [c0, c1)) for the lane's V samples: the sum of the
// conditions' log-sigmoids (membership tests: 0 or -inf). The forward and the adjoint both call it.
template <bool CAT, int V>
__device__ __forceinline__ void rule_logq(const SoftKArgs &a, int c0, int c1, const XView &x, float (&s)[V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) s[v] = 0.f;
#pragma unroll 2
    for (int c = c0; c < c1; ++c) {
        const SoftRec rc = a.recs[c];
        if (CAT && (rc.meta & 4u)) {   // membership: its exact indicator, a factor 1 or 0 of q_r
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (!category_member(x(rc.f, v), __float_as_uint(rc.a), __float_as_uint(rc.bt))) s[v] = -INFINITY;
            continue;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float lhs = rc.a * x(rc.f, v);
            const float rhs = (rc.meta & 1u) ? rc.bt * x(rc.g, v) : rc.bt;
            float u = (lhs - rhs) * a.inv_tau;
            if (rc.meta & 2u) u = -u;
            s[v] += log_sigmoid(u);
        }
    }
}

// rule_logq for the adjoint, which also keeps u and e^-|u| of the rule's first SOFT_CACHE
// conditions (same arithmetic and order, so the same log q) for their gradients.
constexpr int SOFT_CACHE = 4;
template <bool CAT, int V>
__device__ __forceinline__ void rule_logq_cached(const SoftKArgs &a, int c0, int c1, const XView &x, float (&s)[V],
                                                 float (&cu)[SOFT_CACHE][V], float (&ce)[SOFT_CACHE][V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) s[v] = 0.f;
#pragma unroll
    for (int k = 0; k < SOFT_CACHE; ++k) {
        if (c0 + k >= c1) break;
        const SoftRec rc = a.recs[c0 + k];
        if (CAT && (rc.meta & 4u)) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (!category_member(x(rc.f, v), __float_as_uint(rc.a), __float_as_uint(rc.bt))) s[v] = -INFINITY;
            continue;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float lhs = rc.a * x(rc.f, v);
            const float rhs = (rc.meta & 1u) ? rc.bt * x(rc.g, v) : rc.bt;
            float u = (lhs - rhs) * a.inv_tau;
            if (rc.meta & 2u) u = -u;
            const float e = exp_np(-fabsf(u));
            cu[k][v] = u;
            ce[k][v] = e;
            s[v] += -(fmaxf(-u, 0.f) + log1p_unit(e));
        }
    }
#pragma unroll 2
    for (int c = c0 + SOFT_CACHE; c < c1; ++c) {
        const SoftRec rc = a.recs[c];
        if (CAT && (rc.meta & 4u)) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (!category_member(x(rc.f, v), __float_as_uint(rc.a), __float_as_uint(rc.bt))) s[v] = -INFINITY;
            continue;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float lhs = rc.a * x(rc.f, v);
            const float rhs = (rc.meta & 1u) ? rc.bt * x(rc.g, v) : rc.bt;
            float u = (lhs - rhs) * a.inv_tau;
            if (rc.meta & 2u) u = -u;
            s[v] += log_sigmoid(u);
        }
    }
}

// cond_grad from the condition's u (already signed) and e = e^-|u|.
__device__ __forceinline__ float2 cond_grad_cached(const SoftKArgs &a, const SoftRec &rc, const XView &x, int v,
                                                   float gq, float u, float e)
{
    const float xf = x(rc.f, v);
    const bool pair = rc.meta & 1u;
    const float sg = (rc.meta & 2u) ? -1.f : 1.f;
    const float du = gq * __fdividef(u >= 0.f ? e : 1.f, 1.f + e) * sg * a.inv_tau;
    return make_float2(du * xf, pair ? -du * x(rc.g, v) : -du);
}

// ------------------------------------------------------------------ float-float arithmetic
// A value held as the unevaluated sum hi + lo of two floats (Dekker, "A floating-point technique
// for extending the available precision", 1971; Knuth's TwoSum): about 48 significant bits. The
// transformations below are written with explicitly rounded operations so that no contraction
// or reassociation can change them. Non-finite values carry lo = 0 and bypass the
// transformations (which would turn an infinity into NaN).
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ ff ff_fast_sum(float a, float b)     // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ float ff_f(ff x) { return __fadd_rn(x.hi, x.lo); }
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    if (!isfinite(x.hi) || !isfinite(y.hi)) return {__fadd_rn(x.hi, y.hi), 0.f};
    const ff s = ff_two_sum(x.hi, y.hi);
    return ff_fast_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ff ff_add_f(ff x, float y) { return ff_add(x, ff{y, 0.f}); }

__device__ __forceinline__ ff ff_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    if (!isfinite(p)) return {p, 0.f};
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    if (!isfinite(p)) return {p, 0.f};
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fadd_rn(e, __fadd_rn(__fmul_rn(x.hi, y.lo), __fmul_rn(x.lo, y.hi)));
    return ff_fast_sum(p, e);
}

__device__ __forceinline__ bool ff_less(ff x, ff y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

// log(e^a + e^b): the larger term plus log1p of the exponential of the (float) difference
__device__ __forceinline__ ff ff_log_add(ff a, ff b)
{
    if (a.hi == -INFINITY) return b;
    if (b.hi == -INFINITY) return a;
    const bool ab = ff_less(b, a);
    const ff m = ab ? a : b, o = ab ? b : a;
    return ff_add_f(m, log1p_unit(expf(ff_f(ff_add(o, ff_neg(m))))));
}

// log y for 0 < y <= 1 in float-float: y = m 2^k with m in [sqrt(1/2), sqrt(2)), log y = k ln 2 +
// log m; ln 2 split into a head of 15 significant bits (k * head is exact for |k| < 512) and a tail.
__device__ __forceinline__ ff ff_log_unit(float y)
{
    int k;
    float m = frexpf(y, &k);
    if (m < 0.70710678f) { m = __fmul_rn(m, 2.f); --k; }
    constexpr float LN2_HI = 0.693145751953125f, LN2_LO = 1.42860682030941723e-6f;
    const ff kl = ff_fast_sum(__fmul_rn((float)k, LN2_HI), __fmul_rn((float)k, LN2_LO));
    return ff_add_f(kl, logf(m));
}

// The signed scaled margin u = s * (a * x[f] - rhs) / tau of condition rc for the lane's sample
// v, in float-float: the products are exact (a float times a float), 1/tau is a float-float.
__device__ __forceinline__ ff margin_ff(const SoftKArgs &a, const SoftRec &rc, const XView &x, int v)
{
    const ff lhs = ff_two_prod(rc.a, x(rc.f, v));
    const ff rhs = (rc.meta & 1u) ? ff_two_prod(rc.bt, x(rc.g, v)) : ff{rc.bt, 0.f};
    ff u = ff_mul(ff_add(lhs, ff_neg(rhs)), ff{a.inv_tau, a.inv_tau_lo});
    if (rc.meta & 2u) u = ff_neg(u);
    return u;
}

// log sigmoid(u) = min(u, 0) - log1p(e^-|u|); l1pe returns log1p(e^-|u|), which log sigmoid(-u) =
// -max(u, 0) - log1p(e^-|u|) shares.
__device__ __forceinline__ ff log_sigmoid_ff(ff u, float &l1pe)
{
    l1pe = log1p_unit(expf(-fabsf(ff_f(u))));
    return u.hi < 0.f ? ff_add_f(u, -l1pe) : ff{-l1pe, 0.f};
}

// log q of one rule for the lane's sample v in float-float (membership tests: 0 or -inf).
template <bool CAT>
__device__ ff rule_logq_ff(const SoftKArgs &a, int c0, int c1, const XView &x, int v)
{
    ff s{0.f, 0.f};
    for (int c = c0; c < c1; ++c) {
        const SoftRec rc = a.recs[c];
        if (CAT && (rc.meta & 4u)) {
            if (!category_member(x(rc.f, v), __float_as_uint(rc.a), __float_as_uint(rc.bt))) s = {-INFINITY, 0.f};
            continue;
        }
        float l1pe;
        s = ff_add(s, log_sigmoid_ff(margin_ff(a, rc, x, v), l1pe));
    }
    return s;
}

// log(1 - q) of one rule from its log q (float-float). Where q <= 1/2 the float value is exact to
// its last bit's scale; below that, 1 - q = -expm1(log q) and its log is taken in float-float;
// where log q is within 2^-24 of 0, every condition's margin exceeds ~16.6 tau and
// 1 - q = sum_c softplus(-u_c) = sum_c e^{-u_c} to float precision, whose log is the
// log-sum-exp of -u_c with the largest term factored out. A rule of holding membership tests
// only has q = 1 exactly and log(1 - q) = -inf.
template <bool CAT>
__device__ ff rule_log1mq_ff(const SoftKArgs &a, int c0, int c1, const XView &x, int v, ff lq)
{
    if (lq.hi == -INFINITY) return {0.f, 0.f};
    const float lqf = ff_f(lq);
    if (isnan(lqf)) return {lqf, 0.f};
    if (lqf < -0.69314718f) return {log1pf(-expf(lqf)), 0.f};
    if (lqf < -0x1p-24f) return ff_log_unit(-expm1f(lqf));
    ff m{INFINITY, 0.f};
    for (int c = c0; c < c1; ++c) {
        const SoftRec rc = a.recs[c];
        if (CAT && (rc.meta & 4u)) continue;
        const ff u = margin_ff(a, rc, x, v);
        if (ff_less(u, m)) m = u;
    }
    if (m.hi == INFINITY) return {-INFINITY, 0.f};
    float acc = 0.f;
    for (int c = c0; c < c1; ++c) {
        const SoftRec rc = a.recs[c];
        if (CAT && (rc.meta & 4u)) continue;
        acc += expf(ff_f(ff_add(m, ff_neg(margin_ff(a, rc, x, v)))));
    }
    return ff_add_f(ff_neg(m), logf(acc));
}

// The four gradient sums of conditions c and c + 1 (g0, g1: this lane's d/da, d/db-or-dt) reduced
// over the warp in one butterfly and added to the warp's accumulators.
__device__ __forceinline__ void reduce_pair(float2 g0, float2 g1, int ci0, bool has1, float (*acc)[4], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8;
    // lanes 0..15 gather the first condition's two sums, lanes 16..31 the second's
    float k0 = b4 ? g1.x : g0.x, k1 = b4 ? g1.y : g0.y;
    k0 += __shfl_xor_sync(FULL, b4 ? g0.x : g1.x, 16);
    k1 += __shfl_xor_sync(FULL, b4 ? g0.y : g1.y, 16);
    // then lanes with bit 3 clear the d/da sum, set the other
    float t = (b3 ? k1 : k0) + __shfl_xor_sync(FULL, b3 ? k0 : k1, 8);
    t += __shfl_xor_sync(FULL, t, 4);
    t += __shfl_xor_sync(FULL, t, 2);
    t += __shfl_xor_sync(FULL, t, 1);
    // lanes 0, 8, 16, 24 hold the totals; each condition's sums always land in the same lanes
    if ((lane & 7) == 0 && (!b4 || has1)) {
        const int ci = ci0 + (b4 ? 1 : 0), k = b3 ? 2 : 0;
        kadd(acc[ci][k], acc[ci][k + 1], t);
    }
}

// Class probabilities of the sample in slot `sl` (lane + 32 v) of the group from its per-rule log q
// and log "no earlier rule fired" (lq, lu; lu[R] for the default).
template <int V>
__device__ __forceinline__ void write_probs(const SoftKArgs &a, int p, int rb, int R, int deflt, int64_t n0, int sl,
                                            float (*lq)[32 * V], float (*lu)[32 * V])
{
    const int64_t orig = a.perm[n0 + sl];
    for (int k = 0; k < a.K; ++k) {
        float lpk = (deflt == k) ? lu[R][sl] : -INFINITY;
        for (int j = 0; j < R; ++j)
            if (a.rule_class[rb + j] == k) lpk = log_add(lpk, lq[j][sl] + lu[j][sl]);
        a.probs[((int64_t)p * a.N + orig) * a.K + k] = expf(lpk);
    }
}

constexpr float SOFT_FF_LIMIT = 32.f;    // |log p_y| beyond which a group is evaluated in float-float

// soft_group in float-float arithmetic, one sample of each lane at a time (all lanes walk the same
// rules and conditions, so the gradient butterflies stay warp-wide). Forward: log q_r and
// log(1 - q_r) of every rule, lu and log p_y accumulated in float-float. Adjoint: lu_r recovered
// backwards as lu_{r+1} - log(1 - q_r) (exact to float-float precision; from the saved value at
// the first rule with q_r = 1, after which lu is -inf), the S and T recursions in float-float, and
// d ell / d u_c = -+exp(lq_r + lu_r + lT_{r+1} or lS_{r+1} - lp_y + log sigmoid(-u_c)) formed in the
// exponent. Per-set sums keep the float path's fixed order: the loss in the caller's Kahan sum,
// the gradients through the same butterfly and lanes.
template <bool BWD, bool CAT, int V>
__device__ __forceinline__ void soft_group_ff(const SoftKArgs &a, int p, int rb, int R, int cb, int deflt, int64_t n0,
                                           uint32_t valid, const XView &x, float (*lq)[32 * V],
                                           float (*lu)[32 * V], float (*acc)[4], int lane, float &loss_s,
                                           float &loss_c)
{
    for (int v = 0; v < V; ++v) {
        const bool ok = (valid >> v) & 1u;
        const int yv = ok ? a.y[n0 + lane + 32 * v] : -1;
        const int sl = lane + 32 * v;
        // ---------------- forward
        ff lur{0.f, 0.f}, lpy{-INFINITY, 0.f}, lu_fin{0.f, 0.f};
        int jinf = R;                          // first rule with q = 1 (log(1 - q) = -inf)
        for (int j = 0; j < R; ++j) {
            const int r = rb + j;
            const int c0 = a.rule_cond_off[r], c1 = a.rule_cond_off[r + 1];
            const ff lqj = rule_logq_ff<CAT>(a, c0, c1, x, v);
            const ff l1q = rule_log1mq_ff<CAT>(a, c0, c1, x, v, lqj);
            if (a.rule_class[r] == yv) lpy = ff_log_add(lpy, ff_add(lqj, lur));
            if (lq) lq[j][sl] = lqj.hi;
            lu[j][sl] = lur.hi;
            if (l1q.hi == -INFINITY && jinf == R) { jinf = j; lu_fin = lur; }
            lur = ff_add(lur, l1q);
        }
        lu[R][sl] = lur.hi;
        if (deflt == yv) lpy = ff_log_add(lpy, lur);
        if (ok) kadd_loss(loss_s, loss_c, -ff_f(lpy));
        if (a.probs && ok) write_probs<V>(a, p, rb, R, deflt, n0, sl, lq, lu);   // this lane's own slot
        if (!BWD) continue;
        // ---------------- adjoint
        ff lS = deflt == yv ? ff{0.f, 0.f} : ff{-INFINITY, 0.f};
        ff lT = deflt == yv ? ff{-INFINITY, 0.f} : ff{0.f, 0.f};
        ff lu_next = lur;
        for (int j = R - 1; j >= 0; --j) {
            const int r = rb + j;
            const int cls = a.rule_class[r];
            const int c0 = a.rule_cond_off[r], c1 = a.rule_cond_off[r + 1];
            const ff lqj = rule_logq_ff<CAT>(a, c0, c1, x, v);
            const ff l1q = rule_log1mq_ff<CAT>(a, c0, c1, x, v, lqj);
            const ff luj = j > jinf ? ff{-INFINITY, 0.f} : (j == jinf ? lu_fin : ff_add(lu_next, ff_neg(l1q)));
            lu_next = luj;
            const bool same = cls == yv;
            const ff lw = same ? lT : lS;
            const bool zero = !ok || lw.hi == -INFINITY || lqj.hi == -INFINITY || luj.hi == -INFINITY;
            const ff G = ff_add(ff_add(ff_add(lqj, luj), lw), ff_neg(lpy));
            const float sign = same ? -1.f : 1.f;
            lS = ff_log_add(same ? lqj : ff{-INFINITY, 0.f}, ff_add(l1q, lS));
            lT = ff_log_add(same ? ff{-INFINITY, 0.f} : lqj, ff_add(l1q, lT));
            for (int c = c0; c < c1; c += 2) {
                const bool has1 = c + 1 < c1;
                float2 g[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    if (i == 1 && !has1) break;
                    const SoftRec rc = a.recs[c + i];
                    if ((CAT && (rc.meta & 4u)) || zero) continue;
                    const ff u = margin_ff(a, rc, x, v);
                    float l1pe;
                    log_sigmoid_ff(u, l1pe);
                    const ff lsn = u.hi > 0.f ? ff_add_f(ff_neg(u), -l1pe) : ff{-l1pe, 0.f};   // log sigmoid(-u)
                    const float sg = (rc.meta & 2u) ? -1.f : 1.f;
                    const float du = sign * expf(ff_f(ff_add(G, lsn))) * sg * a.inv_tau;
                    g[i] = make_float2(du * x(rc.f, v), (rc.meta & 1u) ? -du * x(rc.g, v) : -du);
                }
                reduce_pair(g[0], g[1], c - cb, has1, acc, lane);
            }
        }
    }
}

// Forward of set p over one group of 32 * V samples (lane l holds samples n0 + l + 32 v; bit v
// of valid: the sample exists): the rules' log "no earlier rule fired" into lu (and log q into
// lq when class probabilities are written), the labels yn and log p_y. Returns true when some
// sample's log p_y is beyond SOFT_FF_LIMIT in magnitude or not finite (warp-uniform).
template <bool CAT, int V>
__device__ __forceinline__ bool soft_forward(const SoftKArgs &a, int rb, int R, int deflt, int64_t n0, uint32_t valid,
                                             const XView &x, float (*lq)[32 * V], float (*lu)[32 * V], int lane,
                                             int (&yn)[V], float (&lpy)[V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) yn[v] = ((valid >> v) & 1u) ? a.y[n0 + lane + 32 * v] : -1;
    float lu_r[V];
#pragma unroll
    for (int v = 0; v < V; ++v) { lu_r[v] = 0.f; lpy[v] = -INFINITY; }
    for (int j = 0; j < R; ++j) {
        const int r = rb + j;
        const int c0 = a.rule_cond_off[r], c1 = a.rule_cond_off[r + 1];
        float s[V];
        rule_logq<CAT, V>(a, c0, c1, x, s);
        const int cls = a.rule_class[r];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (lq) lq[j][lane + 32 * v] = s[v];      // kept only for the class probabilities
            lu[j][lane + 32 * v] = lu_r[v];
            if (cls == yn[v]) lpy[v] = log_add(lpy[v], s[v] + lu_r[v]);
            lu_r[v] += log1m_exp(s[v]);
        }
    }
    bool big = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        lu[R][lane + 32 * v] = lu_r[v];
        if (deflt == yn[v]) lpy[v] = log_add(lpy[v], lu_r[v]);
        if (((valid >> v) & 1u) && !(fabsf(lpy[v]) <= SOFT_FF_LIMIT)) big = true;
    }
    return __any_sync(FULL, big);
}

// Forward (and adjoint) of set p over one group of 32 * V samples: lane l holds samples
// n0 + l + 32 v (v < V; bit v of valid: the sample exists), whose independent chains interleave.
// lu: the warp's per-rule log-probabilities that no earlier rule fired [rule][32 V]; lq: the
// rules' log q, kept only when class probabilities are written (null otherwise: the adjoint
// computes them again); acc: the per-condition gradient sums.
// CAT: the batch may hold membership conditions. Returns true, having added nothing, when some
// sample's log p_y is beyond SOFT_FF_LIMIT: the task is then marked, and k_soft_ff evaluates the
// group in float-float after this kernel.
template <bool BWD, bool CAT, int V>
__device__ __forceinline__ bool soft_group(const SoftKArgs &a, int p, int rb, int R, int cb, int deflt,
                                           int64_t n0, uint32_t valid, const XView &x,
                                           float (*lq)[32 * V], float (*lu)[32 * V], float (*acc)[4], int lane,
                                           float &loss_s, float &loss_c)
{
    int yn[V];
    float lpy[V];
    if (soft_forward<CAT, V>(a, rb, R, deflt, n0, valid, x, lq, lu, lane, yn, lpy)) return true;
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (((valid >> v) & 1u)) kadd_loss(loss_s, loss_c, -lpy[v]);
    if (a.probs) {
#pragma unroll
        for (int v = 0; v < V; ++v)
            if ((valid >> v) & 1u) write_probs<V>(a, p, rb, R, deflt, n0, lane + 32 * v, lq, lu);
    }
    if (!BWD) return false;
    // ---------------- adjoint
    float lS[V], lT[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        lS[v] = (deflt == yn[v]) ? 0.f : -INFINITY;
        lT[v] = (deflt == yn[v]) ? -INFINITY : 0.f;
    }
    for (int j = R - 1; j >= 0; --j) {
        const int r = rb + j;
        const int cls = a.rule_class[r];
        const int c0 = a.rule_cond_off[r], c1 = a.rule_cond_off[r + 1];
        float lqr[V], cu[SOFT_CACHE][V], ce[SOFT_CACHE][V];
        rule_logq_cached<CAT, V>(a, c0, c1, x, lqr, cu, ce);   // log q again: cheaper than keeping it
        float gq[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float lqj = lqr[v], luj = lu[j][lane + 32 * v];
            const bool same = cls == yn[v];
            const float g = exp_np(lqj + luj + (same ? lT[v] : lS[v]) - lpy[v]);
            gq[v] = ((valid >> v) & 1u) ? (same ? -g : g) : 0.f;
            // log(1 - q_j): the forward's step from lu_j to lu_{j+1}. Where lu_j is -inf (an earlier
            // rule certainly fired) the value does not matter (every later term is multiplied by
            // exp(lu) = 0 and lS, lT only meet it through lu): any finite value keeps them finite.
            const float lun = lu[j + 1][lane + 32 * v];
            const float l1q = luj == -INFINITY ? 0.f : lun - luj;
            // one of the two recursions adds q_j (the one of the sample's label class or not), the
            // other only carries the factor 1 - q_j
            const float grow = log_add(lqj, l1q + (same ? lS[v] : lT[v]));
            const float carry = l1q + (same ? lT[v] : lS[v]);
            lS[v] = same ? grow : carry;
            lT[v] = same ? carry : grow;
        }
        // conditions two at a time: the four sums (d/da, d/db-or-dt of both, over all 32 V samples)
        // share one butterfly; the first SOFT_CACHE conditions reuse u and e^-|u| from above
#pragma unroll
        for (int k = 0; k < SOFT_CACHE; k += 2) {
            const int c = c0 + k;
            if (c >= c1) break;
            const bool has1 = c + 1 < c1;
            const SoftRec r0 = a.recs[c];
            const SoftRec r1 = a.recs[has1 ? c + 1 : c];
            const bool use0 = !(CAT && (r0.meta & 4u)), use1 = has1 && !(CAT && (r1.meta & 4u));
            float2 g0 = make_float2(0.f, 0.f), g1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (use0) {
                    const float2 t = cond_grad_cached(a, r0, x, v, gq[v], cu[k][v], ce[k][v]);
                    g0.x += t.x; g0.y += t.y;
                }
                if (use1) {
                    const float2 t = cond_grad_cached(a, r1, x, v, gq[v], cu[k + 1][v], ce[k + 1][v]);
                    g1.x += t.x; g1.y += t.y;
                }
            }
            reduce_pair(g0, g1, c - cb, has1, acc, lane);
        }
#pragma unroll 2
        for (int c = c0 + SOFT_CACHE; c < c1; c += 2) {
            const bool has1 = c + 1 < c1;
            const SoftRec r0 = a.recs[c];
            const SoftRec r1 = a.recs[has1 ? c + 1 : c];
            const bool use0 = !(CAT && (r0.meta & 4u)), use1 = has1 && !(CAT && (r1.meta & 4u));
            float2 g0 = make_float2(0.f, 0.f), g1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (use0) { const float2 t = cond_grad(a, r0, x, v, gq[v]); g0.x += t.x; g0.y += t.y; }
                if (use1) { const float2 t = cond_grad(a, r1, x, v, gq[v]); g1.x += t.x; g1.y += t.y; }
            }
            reduce_pair(g0, g1, c - cb, has1, acc, lane);
        }
    }
    return false;
}

// Write a task's chunk partials (loss; gradient sums when BWD).
template <bool BWD>
__device__ __forceinline__ void soft_flush(const SoftKArgs &a, int p, int ch, int cb, int ce, float loss_s,
                                           float (*acc)[4], int lane)
{
    float ls = loss_s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(FULL, ls, o);
    if (lane == 0) a.part_loss[(int64_t)ch * a.P + p] = ls;
    if (BWD) {
        __syncwarp();
        for (int i = lane; i < (ce - cb); i += 32) {
            a.part_ga[(int64_t)ch * a.Ccap + cb + i] = acc[i][0];
            a.part_gbt[(int64_t)ch * a.Ccap + cb + i] = acc[i][2];
        }
        __syncwarp();
    }
}

template <bool BWD, bool CAT>
__global__ void __maxnreg__(96) k_soft(SoftKArgs a)     // launched with SOFT_W warps
{
    // per warp: lu[maxR+1][G], acc[maxC][4] (ga sum/comp, gbt sum/comp), lq[maxR][G] (probabilities)
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t tasks = (int64_t)a.P * a.nchunks;
    const size_t per_warp = soft_per_warp(a.maxR, a.maxC, a.probs != nullptr);
    float *base_w = sm + per_warp * w;
    float(*lu)[SOFT_G] = reinterpret_cast<float(*)[SOFT_G]>(base_w);
    float(*acc)[4] = reinterpret_cast<float(*)[4]>(base_w + (size_t)(a.maxR + 1) * SOFT_G);
    float(*lq)[SOFT_G] = a.probs ? reinterpret_cast<float(*)[SOFT_G]>(base_w + (size_t)(a.maxR + 1) * SOFT_G +
                                                                    (size_t)a.maxC * 4)
                                 : nullptr;
    if (*a.status) return;

    while (true) {
        int64_t task = 0;
        if (lane == 0) task = atomicAdd(a.next, 1);
        task = __shfl_sync(FULL, task, 0);
        if (task >= tasks) break;
        const int p = a.order[task / a.nchunks];
        const int ch = (int)(task % a.nchunks);
        const int rb = a.set_rule_off[p], re = a.set_rule_off[p + 1];
        const int cb = a.rule_cond_off[rb], ce = a.rule_cond_off[re];
        if (BWD) {
            for (int i = lane; i < (ce - cb); i += 32) {
                acc[i][0] = 0.f; acc[i][1] = 0.f; acc[i][2] = 0.f; acc[i][3] = 0.f;
            }
            __syncwarp();
        }
        float loss_s = 0.f, loss_c = 0.f;
        const int64_t s0 = (int64_t)ch * a.chunk;
        const int64_t s1 = min(s0 + a.chunk, a.N);
        uint32_t *fbits = a.ffbits + ((int64_t)ch * a.P + p) * a.ff_wpt;
        uint32_t fw = 0, ff = 0;
        int gi = 0;
        for (int64_t nb = s0; nb < s1; nb += SOFT_G, ++gi) {
            uint32_t valid = 0;
#pragma unroll
            for (int v = 0; v < SOFT_V; ++v) valid |= (nb + lane + 32 * v < s1 ? 1u : 0u) << v;
            // the dataset is padded to a multiple of 128 samples: every read stays inside it
            const XView x{a.Xt + nb + lane, a.n_pad};
            if (soft_group<BWD, CAT, SOFT_V>(a, p, rb, re - rb, cb, a.set_default[p], nb, valid, x, lq, lu, acc,
                                             lane, loss_s, loss_c))
                fw |= 1u << (gi & 31);
            if ((gi & 31) == 31 || nb + SOFT_G >= s1) {
                if (lane == 0) fbits[gi >> 5] = fw;
                ff |= fw;
                fw = 0;
            }
        }
        soft_flush<BWD>(a, p, ch, cb, ce, loss_s, acc, lane);
        if (lane == 0) a.ffmark[(int64_t)ch * a.P + p] = ff != 0;
    }
}

// The same evaluation with the warps of a CTA on as many neighbouring sets (in size order) over
// the same chunk: the features of each 64-sample group are staged once per CTA in shared memory
// (double-buffered asynchronous copies), so condition loads are shared-memory reads. Per-set
// results are identical to k_soft (same per-sample arithmetic and summation order).
constexpr int SOFT_TW_MIN = 4, SOFT_TW_MAX = 24;   // warps (sets) per CTA of the staged-tile kernel
constexpr int SOFT_TILE_STATIC = 256;   // bytes kept for the kernel's static shared memory

__device__ __forceinline__ void stage_group(float *dst, const float *Xt, int64_t n_pad, int F, int64_t nb)
{
    // F rows x G samples, 16-byte pieces
    constexpr int PR = SOFT_G / 4;   // pieces per row
    for (int i = threadIdx.x; i < F * PR; i += blockDim.x) {
        const int f = i / PR, q = i % PR;
        const float *src = Xt + (int64_t)f * n_pad + nb + 4 * q;
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + f * SOFT_G + 4 * q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Launched with at most SOFT_TW_MAX warps: 96 registers per thread keep the two samples' chains
// of the adjoint in registers and fit 512 threads (a launch bound of 512 capped it at 64 and spilled).
template <bool BWD, bool CAT>
__global__ void __maxnreg__(96) k_soft_tile(SoftKArgs a, int F)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ int64_t s_task;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int TW = blockDim.x >> 5;                   // sets per CTA group
    const int64_t set_groups = (a.P + TW - 1) / TW;
    const int64_t tasks = set_groups * a.nchunks;
    const size_t per_warp = soft_per_warp(a.maxR, a.maxC, a.probs != nullptr);
    float *base_w = sm + per_warp * w;
    float(*lu)[SOFT_G] = reinterpret_cast<float(*)[SOFT_G]>(base_w);
    float(*acc)[4] = reinterpret_cast<float(*)[4]>(base_w + (size_t)(a.maxR + 1) * SOFT_G);
    float(*lq)[SOFT_G] = a.probs ? reinterpret_cast<float(*)[SOFT_G]>(base_w + (size_t)(a.maxR + 1) * SOFT_G +
                                                                    (size_t)a.maxC * 4)
                                 : nullptr;
    float *xbuf = sm + per_warp * TW;                 // [2][F][G]
    if (*a.status) return;

    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_task = atomicAdd(a.next, 1);
        __syncthreads();
        const int64_t task = s_task;
        if (task >= tasks) break;
        const int g = (int)(task / a.nchunks);
        const int ch = (int)(task % a.nchunks);
        // the CTA's warps move through the chunk in step: sets of one group have similar sizes
        const bool active = g * TW + w < a.P;
        const int p = active ? a.order[g * TW + w] : 0;
        int rb = 0, R = 0, cb = 0, ce = 0, deflt = 0;
        if (active) {
            rb = a.set_rule_off[p];
            const int re = a.set_rule_off[p + 1];
            R = re - rb;
            cb = a.rule_cond_off[rb];
            ce = a.rule_cond_off[re];
            deflt = a.set_default[p];
            if (BWD) {
                for (int i = lane; i < (ce - cb); i += 32) {
                    acc[i][0] = 0.f; acc[i][1] = 0.f; acc[i][2] = 0.f; acc[i][3] = 0.f;
                }
                __syncwarp();
            }
        }
        float loss_s = 0.f, loss_c = 0.f;
        uint32_t fw = 0, ff = 0;
        const int64_t s0 = (int64_t)ch * a.chunk;
        const int64_t s1 = min(s0 + a.chunk, a.N);
        const int ngroups = (int)((s1 - s0 + SOFT_G - 1) / SOFT_G);
        uint32_t *fbits = a.ffbits + ((int64_t)ch * a.P + p) * a.ff_wpt;
        stage_group(xbuf, a.Xt, a.n_pad, F, s0);
        for (int gi = 0; gi < ngroups; ++gi) {
            const int64_t nb = s0 + SOFT_G * (int64_t)gi;
            if (gi + 1 < ngroups) {
                stage_group(xbuf + ((gi + 1) & 1) * F * SOFT_G, a.Xt, a.n_pad, F, nb + SOFT_G);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            if (active) {
                uint32_t valid = 0;
#pragma unroll
                for (int v = 0; v < SOFT_V; ++v) valid |= (nb + lane + 32 * v < s1 ? 1u : 0u) << v;
                const XView x{xbuf + (gi & 1) * F * SOFT_G + lane, SOFT_G};
                if (soft_group<BWD, CAT, SOFT_V>(a, p, rb, R, cb, deflt, nb, valid, x, lq, lu, acc, lane, loss_s,
                                                 loss_c))
                    fw |= 1u << (gi & 31);
                if ((gi & 31) == 31 || gi + 1 == ngroups) {
                    if (lane == 0) fbits[gi >> 5] = fw;
                    ff |= fw;
                    fw = 0;
                }
            }
            __syncthreads();              // the buffer is restaged two groups later
        }
        if (active) {
            soft_flush<BWD>(a, p, ch, cb, ce, loss_s, acc, lane);
            if (lane == 0) a.ffmark[(int64_t)ch * a.P + p] = ff != 0;
        }
    }
}

// The float-float pass: one warp per (set, chunk) task that the main kernel marked. The warp
// evaluates, in group order, the groups whose bits the main kernel set (those it left out) in
// float-float (soft_group_ff); their loss and gradient sums, Kahan-summed in group order, are
// added to the task's partials. Runs after the main kernel on the same stream; features are read
// from global memory.
template <bool BWD, bool CAT>
__global__ void __launch_bounds__(SOFT_W * 32) k_soft_ff(SoftKArgs a)
{
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t task = (int64_t)blockIdx.x * SOFT_W + w;
    if (*a.status || task >= (int64_t)a.P * a.nchunks) return;
    const int p = (int)(task % a.P);
    const int ch = (int)(task / a.P);
    if (!a.ffmark[(int64_t)ch * a.P + p]) return;
    const size_t per_warp = soft_per_warp(a.maxR, a.maxC, a.probs != nullptr);
    float *base_w = sm + per_warp * w;
    float(*lu)[SOFT_G] = reinterpret_cast<float(*)[SOFT_G]>(base_w);
    float(*acc)[4] = reinterpret_cast<float(*)[4]>(base_w + (size_t)(a.maxR + 1) * SOFT_G);
    float(*lq)[SOFT_G] = a.probs ? reinterpret_cast<float(*)[SOFT_G]>(base_w + (size_t)(a.maxR + 1) * SOFT_G +
                                                                    (size_t)a.maxC * 4)
                                 : nullptr;
    const int rb = a.set_rule_off[p], re = a.set_rule_off[p + 1];
    const int cb = a.rule_cond_off[rb], ce = a.rule_cond_off[re];
    const int deflt = a.set_default[p];
    if (BWD) {
        for (int i = lane; i < (ce - cb); i += 32) {
            acc[i][0] = 0.f; acc[i][1] = 0.f; acc[i][2] = 0.f; acc[i][3] = 0.f;
        }
        __syncwarp();
    }
    float loss_s = 0.f, loss_c = 0.f;
    const int64_t s0 = (int64_t)ch * a.chunk;
    const int64_t s1 = min(s0 + a.chunk, a.N);
    const uint32_t *fbits = a.ffbits + ((int64_t)ch * a.P + p) * a.ff_wpt;
    uint32_t fw = 0;
    int gi = 0;
    for (int64_t nb = s0; nb < s1; nb += SOFT_G, ++gi) {
        if ((gi & 31) == 0) fw = fbits[gi >> 5];
        if (!((fw >> (gi & 31)) & 1u)) continue;
        uint32_t valid = 0;
#pragma unroll
        for (int v = 0; v < SOFT_V; ++v) valid |= (nb + lane + 32 * v < s1 ? 1u : 0u) << v;
        const XView x{a.Xt + nb + lane, a.n_pad};
        soft_group_ff<BWD, CAT, SOFT_V>(a, p, rb, re - rb, cb, deflt, nb, valid, x, lq, lu, acc, lane, loss_s,
                                        loss_c);
    }
    float ls = loss_s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(FULL, ls, o);
    if (lane == 0) a.part_loss[(int64_t)ch * a.P + p] += ls;
    if (BWD) {
        __syncwarp();
        for (int i = lane; i < (ce - cb); i += 32) {
            a.part_ga[(int64_t)ch * a.Ccap + cb + i] += acc[i][0];
            a.part_gbt[(int64_t)ch * a.Ccap + cb + i] += acc[i][2];
        }
    }
}

__device__ __forceinline__ float tree_sum_strided(const float *base, int64_t stride, int n)
{
    // pairwise sum of base[0], base[stride], ... (n <= SOFT_MAX_CHUNKS) in a fixed order
    float v[SOFT_MAX_CHUNKS];
#pragma unroll
    for (int i = 0; i < SOFT_MAX_CHUNKS; ++i) v[i] = (i < n) ? base[(int64_t)i * stride] : 0.f;
#pragma unroll
    for (int w = 1; w < SOFT_MAX_CHUNKS; w <<= 1)
#pragma unroll
        for (int i = 0; i + w < SOFT_MAX_CHUNKS; i += 2 * w) v[i] += v[i + w];
    return v[0];
}

__global__ void k_soft_reduce_loss(const float *part_loss, int nchunks, int P, float inv_n, float *loss,
                                   const uint32_t *status)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || *status) return;
    loss[p] = tree_sum_strided(part_loss + p, P, nchunks) * inv_n;
}

// One Adam update of parameter *p with gradient g and moments *m, *v; every operation separately
// rounded, so that the result does not depend on the file's contraction setting.
__device__ __forceinline__ void adam_one(float *p, float g, float *m, float *v, float bc1, float bc2,
                                         const SoftAdam &ad)
{
    const float mk = __fadd_rn(__fmul_rn(ad.b1, *m), __fmul_rn(1.0f - ad.b1, g));
    const float vk = __fadd_rn(__fmul_rn(ad.b2, *v), __fmul_rn(__fmul_rn(1.0f - ad.b2, g), g));
    *m = mk;
    *v = vk;
    const float mh = __fdiv_rn(mk, bc1), vh = __fdiv_rn(vk, bc2);
    *p = __fsub_rn(*p, __fdiv_rn(__fmul_rn(ad.lr, mh), __fadd_rn(sqrtf(vh), ad.eps)));
}

// One CTA per set, its threads looping over the set's conditions (grads scaled by dloss[p] / N);
// thread 0 also writes the set's loss when `loss` is given; with adam.a the Adam update of the
// set's conditions follows at once.
__global__ void k_soft_reduce_grad(const float *part_ga, const float *part_gbt, const float *part_loss,
                                   int nchunks, const int32_t *set_rule_off, const int32_t *rule_cond_off,
                                   const SoftRec *recs, int P, int64_t C, const float *dloss,
                                   float inv_n, float *grad_a, float *grad_b, float *grad_t, float *loss,
                                   SoftAdam adam, const uint32_t *status)
{
    const int p = blockIdx.x;
    if (p >= P || *status) return;
    if (loss && threadIdx.x == 0) loss[p] = tree_sum_strided(part_loss + p, P, nchunks) * inv_n;
    const float bc1 = 1.0f - powf(adam.b1, (float)adam.step), bc2 = 1.0f - powf(adam.b2, (float)adam.step);
    const int cb = rule_cond_off[set_rule_off[p]], ce = rule_cond_off[set_rule_off[p + 1]];
    const float scale = dloss[p] * inv_n;
    for (int c = cb + threadIdx.x; c < ce; c += blockDim.x) {
        const float ga = tree_sum_strided(part_ga + c, C, nchunks) * scale;
        const float gbt = tree_sum_strided(part_gbt + c, C, nchunks) * scale;
        const bool pair = recs[c].meta & 1u;
        grad_a[c] = ga;
        grad_b[c] = pair ? gbt : 0.f;
        grad_t[c] = pair ? 0.f : gbt;
        if (adam.a) {
            adam_one(adam.a + c, ga, adam.m + 2 * c, adam.v + 2 * c, bc1, bc2, adam);
            adam_one((pair ? adam.b : adam.t) + c, gbt, adam.m + 2 * c + 1, adam.v + 2 * c + 1, bc1, bc2, adam);
        }
    }
}

}  // namespace

// Shared body of both entry points. `known` = bounds given by the caller (no host readback).
template <bool CAT>
static void set_soft_attributes(Ctx *ctx)
{
    cudaFuncSetAttribute(k_soft<true, CAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin);
    cudaFuncSetAttribute(k_soft<false, CAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin);
    // the staged-tile kernel has a little static shared memory of its own
    cudaFuncSetAttribute(k_soft_tile<true, CAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ctx->smem_optin - SOFT_TILE_STATIC);
    cudaFuncSetAttribute(k_soft_tile<false, CAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ctx->smem_optin - SOFT_TILE_STATIC);
    cudaFuncSetAttribute(k_soft_ff<true, CAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin);
    cudaFuncSetAttribute(k_soft_ff<false, CAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->smem_optin);
    cudaGetLastError();
}

// Resident CTAs per SM of the staged-tile kernel with tw warps and per-warp arrays of
// per_warp bytes (0 when it does not fit).
template <bool BWD, bool CAT>
static int soft_tile_per_sm(Ctx *ctx, int tw, size_t per_warp, int F)
{
    const size_t bytes = per_warp * tw + sizeof(float) * 2 * SOFT_G * (size_t)F;
    if (bytes + SOFT_TILE_STATIC > ctx->smem_optin) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_soft_tile<BWD, CAT>, tw * 32, bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

// Launch shape of the soft kernel: warps per CTA (staged-tile form) and resident CTAs per SM.
struct SoftShape {
    int tw = SOFT_TW_MIN;
    int per_sm = 1;
};

// The staged-tile form takes the number of warps per CTA that keeps the most warps resident for
// this batch's per-warp arrays (ties: fewer warps per CTA, so that a CTA's sets are closer in
// size); small populations keep at most P / 8 warps per CTA, since a CTA walks its sets in step
// and a wide CTA over few sets of uneven size waits for the longest.
template <bool CAT>
static SoftShape soft_shape(Ctx *ctx, bool tiled, bool bwd, int F, size_t smem, size_t per_warp, int P)
{
    SoftShape sh;
    if (tiled) {
        int best = 0;
        const int tw_max = std::max(SOFT_TW_MIN, std::min(SOFT_TW_MAX, P / 8));
        for (int t = SOFT_TW_MIN; t <= tw_max; ++t) {
            const int c = bwd ? soft_tile_per_sm<true, CAT>(ctx, t, per_warp, F)
                              : soft_tile_per_sm<false, CAT>(ctx, t, per_warp, F);
            if (c * t > best) { best = c * t; sh.tw = t; sh.per_sm = c; }
        }
    } else {
        if (bwd) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh.per_sm, k_soft<true, CAT>, SOFT_W * 32, smem);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh.per_sm, k_soft<false, CAT>, SOFT_W * 32, smem);
    }
    sh.per_sm = std::max(1, sh.per_sm);
    return sh;
}

// One persistent wave of the soft kernel: the staged-tile form or the per-warp form, forward only
// or forward + adjoint, with or without membership conditions (CAT).
template <bool CAT>
static void launch_soft_kernel(Ctx *ctx, const SoftKArgs &k, bool tiled, bool bwd, int F, size_t smem,
                               size_t per_warp, const SoftShape &sh, cudaStream_t stream)
{
    const int grid = ctx->sm_count * sh.per_sm;
    if (tiled) {
        const size_t smem_tile = per_warp * sh.tw + sizeof(float) * 2 * SOFT_G * (size_t)F;
        if (bwd) k_soft_tile<true, CAT><<<grid, sh.tw * 32, smem_tile, stream>>>(k, F);
        else k_soft_tile<false, CAT><<<grid, sh.tw * 32, smem_tile, stream>>>(k, F);
    } else {
        if (bwd) k_soft<true, CAT><<<grid, SOFT_W * 32, smem, stream>>>(k);
        else k_soft<false, CAT><<<grid, SOFT_W * 32, smem, stream>>>(k);
    }
}

// Words of the float-float group bits for P sets over N samples, for any chunking of at most
// SOFT_MAX_CHUNKS chunks: chunks x ceil(groups per chunk / 32) <= N / 2048 + 2 * SOFT_MAX_CHUNKS.
static size_t ff_words(int P, int64_t N)
{
    return (size_t)P * (size_t)(N / 2048 + 2 * SOFT_MAX_CHUNKS + 1);
}

// Scratch layout of one soft call: records [C], order [P], per-chunk losses [chunks][P], the work
// counter and maxima [4], per-chunk gradient sums [chunks][C] twice (adjoint only), the tasks'
// float-float marks [chunks][P] and group bits.
struct SoftScratchLayout {
    size_t recs, order, part_loss, next, part_ga, part_gbt, ffmark, ffbits, total;
};

static SoftScratchLayout soft_layout(int64_t C, int P, int nchunks, bool bwd, int64_t N)
{
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    SoftScratchLayout L{};
    size_t o = 0;
    L.recs = o; o += up(sizeof(SoftRec) * (size_t)C);
    L.order = o; o += up(sizeof(int32_t) * (size_t)P);
    L.part_loss = o; o += up(sizeof(float) * (size_t)nchunks * P);
    L.next = o; o += 256;
    L.part_ga = o; o += bwd ? up(sizeof(float) * (size_t)nchunks * C) : 0;
    L.part_gbt = o; o += bwd ? up(sizeof(float) * (size_t)nchunks * C) : 0;
    L.ffmark = o; o += up((size_t)nchunks * P);
    L.ffbits = o; o += up(sizeof(uint32_t) * ff_words(P, N));
    L.total = o;
    return L;
}

size_t soft_scratch_bytes(int64_t cap_c, int cap_p, int64_t N)
{
    return soft_layout(std::max<int64_t>(cap_c, 1), std::max(cap_p, 1), SOFT_MAX_CHUNKS, true, N).total;
}

// `repeat`: a later step on the caller's scratch over the same structure as the step before it
// (only coefficients and thresholds changed), whose validation and set order still stand.
static rs_status soft_run(Ctx *ctx, const SoftArgs &s, int known_maxR, int known_maxC, cudaStream_t stream,
                          char *pre = nullptr, bool repeat = false, const SoftAdam *adam = nullptr)
{
    const BatchDev &b = s.b;
    const int P = b.P;
    const int64_t Ccap = std::max<int64_t>(b.C, 1);     // capacity when sizes are device-side
    if (P == 0) return RS_OK;
    // Sample chunks: about 1024 samples each, and for small problems as many as it takes to give
    // every SM some 64 (set, chunk) items, down to one 64-sample group per chunk. The chunking is
    // a function of (N, P, SM count) only, so repeated calls sum in the same order.
    const int64_t groups = (s.N + SOFT_G - 1) / SOFT_G;
    const int64_t want = std::max<int64_t>((s.N + 1023) / 1024, ((int64_t)ctx->sm_count * 64 + P - 1) / P);
    int nchunks = (int)std::min<int64_t>(std::min<int64_t>(SOFT_MAX_CHUNKS, groups), want);
    if (nchunks < 1) nchunks = 1;
    int64_t chunk = (s.N + nchunks - 1) / nchunks;
    chunk = (chunk + SOFT_G - 1) / SOFT_G * SOFT_G;
    nchunks = (int)((s.N + chunk - 1) / chunk);

    SoftRec *recs = nullptr;
    float *part_loss = nullptr, *part_ga = nullptr, *part_gbt = nullptr;
    int32_t *next = nullptr;   // [0] work counter, [1..2] max rules / conditions per set
    int32_t *order = nullptr;
    uint8_t *ffmark = nullptr;
    uint32_t *ffbits = nullptr;
    const bool bwd = s.dloss != nullptr;
    cudaError_t ae = cudaSuccess;
    if (pre) {                       // the caller's scratch, laid out for at most SOFT_MAX_CHUNKS chunks
        const SoftScratchLayout L = soft_layout(Ccap, P, SOFT_MAX_CHUNKS, bwd, s.N);
        recs = reinterpret_cast<SoftRec *>(pre + L.recs);
        order = reinterpret_cast<int32_t *>(pre + L.order);
        part_loss = reinterpret_cast<float *>(pre + L.part_loss);
        next = reinterpret_cast<int32_t *>(pre + L.next);
        part_ga = bwd ? reinterpret_cast<float *>(pre + L.part_ga) : nullptr;
        part_gbt = bwd ? reinterpret_cast<float *>(pre + L.part_gbt) : nullptr;
        ffmark = reinterpret_cast<uint8_t *>(pre + L.ffmark);
        ffbits = reinterpret_cast<uint32_t *>(pre + L.ffbits);
    } else {
        ae = dev_alloc_async(&recs, sizeof(SoftRec) * Ccap, stream);
        if (ae == cudaSuccess) ae = dev_alloc_async(&order, sizeof(int32_t) * (size_t)P, stream);
        if (ae == cudaSuccess) ae = dev_alloc_async(&part_loss, sizeof(float) * (size_t)nchunks * P, stream);
        if (ae == cudaSuccess) ae = dev_alloc_async(&next, sizeof(int32_t) * 4, stream);
        if (ae == cudaSuccess && bwd) ae = dev_alloc_async(&part_ga, sizeof(float) * (size_t)nchunks * Ccap, stream);
        if (ae == cudaSuccess && bwd) ae = dev_alloc_async(&part_gbt, sizeof(float) * (size_t)nchunks * Ccap, stream);
        if (ae == cudaSuccess) ae = dev_alloc_async(&ffmark, (size_t)nchunks * P, stream);
        if (ae == cudaSuccess) ae = dev_alloc_async(&ffbits, sizeof(uint32_t) * ff_words(P, s.N), stream);
    }
    if (ae != cudaSuccess) {         // release what was taken before the failure
        for (void *q : {(void *)recs, (void *)order, (void *)part_loss, (void *)next, (void *)part_ga, (void *)part_gbt,
                        (void *)ffmark, (void *)ffbits})
            if (q) cudaFreeAsync(q, stream);
        return cuda_fail(ae, "soft scratch");
    }
    const bool known = known_maxR > 0;
    repeat = repeat && pre && known;
    if (!repeat) {
        RS_CUDA(cudaMemsetAsync(next, 0, sizeof(int32_t) * 4, stream));
        k_check_sets_soft<<<(P + 255) / 256, 256, 0, stream>>>(b, s.K, s.status, next + 1,
                                                               known ? known_maxR : SOFT_MAX_RULES,
                                                               known ? known_maxC : SOFT_MAX_CONDS);
        count_launch(ctx);
    }
    k_pack_soft<<<(unsigned)((Ccap + 255) / 256), 256, 0, stream>>>(b, s.F, s.K, recs, s.status, next);
    count_launch(ctx);
    if (!repeat) {
        k_soft_order<<<1, 1024, 0, stream>>>(b, order);
        count_launch(ctx);
    }
    SoftKArgs k{};
    k.recs = recs;
    k.set_rule_off = b.set_rule_off;
    k.rule_cond_off = b.rule_cond_off;
    k.rule_class = b.rule_class;
    k.set_default = b.set_default;
    k.P = P;
    k.Xt = s.Xt;
    k.y = s.y;
    k.perm = s.perm;
    k.N = s.N;
    k.n_pad = s.n_pad;
    k.K = s.K;
    k.inv_tau = 1.0f / s.tau;
    k.inv_tau_lo = (float)(1.0 / (double)s.tau - (double)k.inv_tau);
    k.nchunks = nchunks;
    k.chunk = (int32_t)chunk;
    k.part_loss = part_loss;
    k.part_ga = part_ga;
    k.part_gbt = part_gbt;
    k.order = order;
    k.ffmark = ffmark;
    k.ffbits = ffbits;
    k.probs = s.probs;
    k.backward = bwd;
    k.next = next;
    k.Ccap = Ccap;
    k.status = s.status;
    rs_status rc = RS_OK;
    if (known) {
        k.maxR = known_maxR;
        k.maxC = known_maxC;
    } else {
        // validation must finish before the launch is sized: read the status and the maxima
        uint32_t *hs = host_status_slot();
        if (!hs) return RS_ERR_OOM;
        RS_CUDA(cudaMemcpyAsync(hs, s.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
        RS_CUDA(cudaMemcpyAsync(hs + 1, next + 1, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, stream));
        RS_CUDA(cudaStreamSynchronize(stream));
        k.maxR = std::max<int32_t>(1, (int32_t)hs[1]);
        k.maxC = std::max<int32_t>(1, (int32_t)hs[2]);
        if (*hs) {
            rc = (*hs & ST_TOO_LARGE) ? RS_ERR_TOO_LARGE : RS_ERR_INVALID;
            set_error("soft evaluation rejected the batch: %s", status_text(*hs).c_str());
        }
    }
    const size_t per_warp = sizeof(float) * soft_per_warp(k.maxR, k.maxC, k.probs != nullptr);
    const size_t smem = per_warp * SOFT_W;
    // the staged-tile kernel when its per-CTA footprint (8 warps + two feature tiles) fits
    const size_t smem_tile = per_warp * SOFT_TW_MIN + sizeof(float) * 2 * SOFT_G * (size_t)s.F;
    const bool tiled = s.F <= 128 && smem_tile + SOFT_TILE_STATIC <= ctx->smem_optin;
    if (rc == RS_OK && smem > ctx->smem_optin) {
        rc = RS_ERR_TOO_LARGE;
        set_error("soft evaluation: sets too large for shared memory");
    }
    if (rc == RS_OK) {
        static std::once_flag once;
        std::call_once(once, [&] {
            set_soft_attributes<false>(ctx);
            set_soft_attributes<true>(ctx);
        });
        const SoftShape sh = b.cond_set ? soft_shape<true>(ctx, tiled, bwd, s.F, smem, per_warp, P)
                                        : soft_shape<false>(ctx, tiled, bwd, s.F, smem, per_warp, P);
        if (tiled) {
            // The staged-tile kernel's CTAs take (set group, chunk) tasks until none is left. When
            // the tasks make only a few rounds of the resident CTAs, the last round decides the
            // time: take the chunk count (at most the one chosen above, whose partial sums the
            // scratch holds) that minimises rounds x samples per chunk, preferring more chunks.
            const int64_t set_groups = (P + sh.tw - 1) / sh.tw;
            const int64_t workers = (int64_t)ctx->sm_count * sh.per_sm;
            int64_t best_cost = INT64_MAX;
            for (int n = 1; n <= k.nchunks; ++n) {
                int64_t ch = (s.N + n - 1) / n;
                ch = (ch + SOFT_G - 1) / SOFT_G * SOFT_G;
                const int64_t nc = (s.N + ch - 1) / ch;
                const int64_t cost = (set_groups * nc + workers - 1) / workers * ch;
                if (cost < best_cost || (cost == best_cost && nc > nchunks)) {
                    best_cost = cost;
                    nchunks = (int)nc;
                    chunk = ch;
                }
            }
            k.nchunks = nchunks;
            k.chunk = (int32_t)chunk;
        }
        k.ff_wpt = (int32_t)(((k.chunk + SOFT_G - 1) / SOFT_G + 31) / 32);
        {
            TimedLaunch tl(ctx, TK_SOFT, stream);
            if (b.cond_set) launch_soft_kernel<true>(ctx, k, tiled, bwd, s.F, smem, per_warp, sh, stream);
            else launch_soft_kernel<false>(ctx, k, tiled, bwd, s.F, smem, per_warp, sh, stream);
        }
        {   // groups beyond float32's resolution (usually none: the kernel's warps exit at once)
            const unsigned ffgrid = (unsigned)(((int64_t)P * k.nchunks + SOFT_W - 1) / SOFT_W);
            if (b.cond_set) {
                if (bwd) k_soft_ff<true, true><<<ffgrid, SOFT_W * 32, smem, stream>>>(k);
                else k_soft_ff<false, true><<<ffgrid, SOFT_W * 32, smem, stream>>>(k);
            } else {
                if (bwd) k_soft_ff<true, false><<<ffgrid, SOFT_W * 32, smem, stream>>>(k);
                else k_soft_ff<false, false><<<ffgrid, SOFT_W * 32, smem, stream>>>(k);
            }
            count_launch(ctx);
        }
        if (bwd)                      // the gradients and (when asked) the loss in one launch
            k_soft_reduce_grad<<<P, 128, 0, stream>>>(part_ga, part_gbt, part_loss, nchunks, b.set_rule_off,
                                                     b.rule_cond_off, recs, P, Ccap, s.dloss,
                                                     1.0f / (float)s.N, s.grad_a, s.grad_b, s.grad_t,
                                                     s.loss, adam ? *adam : SoftAdam{}, s.status);
        else
            k_soft_reduce_loss<<<(P + 255) / 256, 256, 0, stream>>>(part_loss, nchunks, P,
                                                                   1.0f / (float)s.N, s.loss, s.status);
        count_launch(ctx, 2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "soft kernels");
    }
    if (!pre) {
        cudaFreeAsync(recs, stream);
        cudaFreeAsync(order, stream);
        cudaFreeAsync(part_loss, stream);
        cudaFreeAsync(next, stream);
        if (bwd) { cudaFreeAsync(part_ga, stream); cudaFreeAsync(part_gbt, stream); }
        cudaFreeAsync(ffmark, stream);
        cudaFreeAsync(ffbits, stream);
    }
    return rc;
}

// The soft kernels' log1p on [0, 1] (which = 0) or log(1 - e^s) (which = 1) evaluated on the
// device for host inputs (a test hook).
rs_status selftest_soft_math(int which, const float *e_h, int n, float *out_h, cudaStream_t stream)
{
    float *d = nullptr;
    RS_CUDA(dev_alloc_async(&d, sizeof(float) * 2 * (size_t)n, stream));
    rs_status rc = RS_OK;
    cudaError_t e = cudaMemcpyAsync(d, e_h, sizeof(float) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        k_selftest_soft_math<<<std::min((n + 255) / 256, 4096), 256, 0, stream>>>(d, n, d + n, which);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_h, d + n, sizeof(float) * n, cudaMemcpyDeviceToHost, stream);
    cudaFreeAsync(d, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "soft math self-test");
    return rc;
}

rs_status launch_soft(Ctx *ctx, const SoftArgs &s, cudaStream_t stream)
{
    return soft_run(ctx, s, 0, 0, stream);
}

rs_status soft_step_known(Ctx *ctx, const SoftArgs &a, int maxR, int maxC, cudaStream_t stream)
{
    return soft_run(ctx, a, std::max(1, maxR), std::max(1, maxC), stream);
}

rs_status soft_validate(Ctx *ctx, const SoftArgs &a, int *maxR, int *maxC, cudaStream_t stream)
{
    const BatchDev &b = a.b;
    if (b.P == 0) { *maxR = *maxC = 1; return RS_OK; }
    int32_t *maxima = nullptr;
    RS_CUDA(dev_alloc_async(&maxima, sizeof(int32_t) * 4, stream));
    RS_CUDA(cudaMemsetAsync(maxima, 0, sizeof(int32_t) * 4, stream));
    k_check_sets_soft<<<(b.P + 255) / 256, 256, 0, stream>>>(b, a.K, a.status, maxima, SOFT_MAX_RULES, SOFT_MAX_CONDS);
    count_launch(ctx);
    uint32_t *hs = host_status_slot();
    if (!hs) { cudaFreeAsync(maxima, stream); return RS_ERR_OOM; }
    RS_CUDA(cudaMemcpyAsync(hs, a.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    RS_CUDA(cudaMemcpyAsync(hs + 1, maxima, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, stream));
    cudaFreeAsync(maxima, stream);
    RS_CUDA(cudaStreamSynchronize(stream));
    *maxR = std::max<int32_t>(1, (int32_t)hs[1]);
    *maxC = std::max<int32_t>(1, (int32_t)hs[2]);
    if (*hs) {
        set_error("soft evaluation rejected the batch: %s", status_text(*hs).c_str());
        return (*hs & ST_TOO_LARGE) ? RS_ERR_TOO_LARGE : RS_ERR_INVALID;
    }
    return RS_OK;
}

rs_status soft_step_scratch(Ctx *ctx, const SoftArgs &a, int maxR, int maxC, void *scratch, int64_t cap_c,
                            int cap_p, bool repeat, const SoftAdam *adam, cudaStream_t stream)
{
    if (adam && !a.dloss) {
        set_error("soft step: an Adam update needs the adjoint");
        return RS_ERR_INVALID;
    }
    if (!scratch || a.b.P > cap_p || std::max<int64_t>(a.b.C, 1) > std::max<int64_t>(cap_c, 1)) {
        set_error("soft step: scratch smaller than the batch");
        return RS_ERR_INVALID;
    }
    return soft_run(ctx, a, std::max(1, maxR), std::max(1, maxC), stream, static_cast<char *>(scratch), repeat,
                    adam);
}

// Load the kernels of this file now (CUDA loads a kernel lazily at its first launch, which would
// otherwise land on the first request that needs it).
void preload_soft_kernels()
{
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_soft<false, false>);
    cudaFuncGetAttributes(&fa, k_soft<true, false>);
    cudaFuncGetAttributes(&fa, k_soft<false, true>);
    cudaFuncGetAttributes(&fa, k_soft<true, true>);
    cudaFuncGetAttributes(&fa, k_soft_tile<false, false>);
    cudaFuncGetAttributes(&fa, k_soft_tile<true, false>);
    cudaFuncGetAttributes(&fa, k_soft_tile<false, true>);
    cudaFuncGetAttributes(&fa, k_soft_tile<true, true>);
    cudaFuncGetAttributes(&fa, k_soft_ff<false, false>);
    cudaFuncGetAttributes(&fa, k_soft_ff<true, false>);
    cudaFuncGetAttributes(&fa, k_soft_ff<false, true>);
    cudaFuncGetAttributes(&fa, k_soft_ff<true, true>);
    cudaFuncGetAttributes(&fa, k_check_sets_soft);
    cudaFuncGetAttributes(&fa, k_pack_soft);
    cudaFuncGetAttributes(&fa, k_soft_order);
    cudaFuncGetAttributes(&fa, k_soft_reduce_grad);
    cudaFuncGetAttributes(&fa, k_soft_reduce_loss);
}

}  // namespace rs
