// Device building blocks shared by evaluators that process one rule set at a time per warp on a
// shared-memory feature tile (record format v2, margin-minimum conjunction).
#pragma once
#include "rs_internal.cuh"

namespace rs {
namespace core {

constexpr uint32_t FULL = 0xFFFFFFFFu;

template <int V>
__device__ __forceinline__ void load_vec(const float *p, float (&x)[V])
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

__device__ __forceinline__ float min_nan(float a, float b)
{
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// mn[v] = min(mn[v], margin of this condition); the condition holds iff its margin is > 0.
template <int V>
__device__ __forceinline__ void margin_min(const uint4 r, const float *xl, float (&mn)[V])
{
    float x[V];
    load_vec<V>(xl + (r.x & OFF_MASK) * 4, x);
    const float v0 = __uint_as_float(r.z), v1 = __uint_as_float(r.w);
    if (r.x & PAIR_BIT) {
        float z[V];
        load_vec<V>(xl + (r.y & OFF_MASK) * 4, z);
#pragma unroll
        for (int v = 0; v < V; ++v)
            mn[v] = min_nan(mn[v], __fsub_rn(__fmul_rn(v0, x[v]), __fmul_rn(v1, z[v])));
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) mn[v] = min_nan(mn[v], __fsub_rn(__fmul_rn(v0, x[v]), v1));
    }
}

// Evaluate one set (records [rb, re)) for this lane's V samples: pred[v] receives the class of the
// first firing rule or `deflt`. Records are read through L2 (.cg): callers may reuse record memory
// within one launch. `valid[v]` false marks padding samples (never claimed). `st` is the
// warp's 64-record stage in shared memory. All lanes of the warp must call this together.
template <int V>
__device__ void eval_set(const uint4 *recs, int rb, int re, uint4 *st, const float *xl, int lane,
                         int deflt, const bool (&valid)[V], int (&pred)[V])
{
    const uint4 zero4 = make_uint4(0, 0, 0, 0);
    bool unc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        pred[v] = deflt;
        unc[v] = valid[v];
    }
    int ck = 0;
    uint4 pf = zero4;
    if (rb < re) {
        __syncwarp();
        st[lane] = (rb + lane < re) ? __ldcg(recs + rb + lane) : zero4;
        st[32 + lane] = (rb + 32 + lane < re) ? __ldcg(recs + rb + 32 + lane) : zero4;
        pf = (rb + 64 + lane < re) ? __ldcg(recs + rb + 64 + lane) : zero4;
        __syncwarp();
    }
    int rel = 0;
    const int nrec = re - rb;
    while (rel < nrec) {
        while ((rel >> 5) > ck) {
            const uint4 keep = st[32 + lane];
            __syncwarp();
            st[lane] = keep;
            st[32 + lane] = pf;
            __syncwarp();
            ++ck;
            const int nx = rb + 32 * (ck + 2) + lane;
            pf = (nx < re) ? __ldcg(recs + nx) : zero4;
        }
        const uint4 *rp = st + (rel - 32 * ck);
        const uint4 r0 = rp[0];
        const int nc = max(1, (int)((r0.x >> LEN_SHIFT) & 0xFFFu));   // >= 1: progress
        const int cls = (int)(r0.y >> CLS_SHIFT);
        float mn[V];
#pragma unroll
        for (int v = 0; v < V; ++v) mn[v] = unc[v] ? __uint_as_float(0x7F800000u) : -1.f;
        margin_min<V>(r0, xl, mn);
        if (nc <= 33) {
#pragma unroll 2
            for (int k = 1; k < nc; ++k) margin_min<V>(rp[k], xl, mn);
        } else {
            for (int k = 1; k < nc; ++k) margin_min<V>(__ldcg(recs + rb + rel + k), xl, mn);
        }
        bool any_unc = false;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (mn[v] > 0.f) { pred[v] = cls; unc[v] = false; }
            any_unc |= unc[v];
        }
        if (!__any_sync(FULL, any_unc)) break;
        rel += nc;
    }
    __syncwarp();
}


// ---------------------------------------------------------------- sign-mask form (finite data)

constexpr uint32_t SIGN = 0x80000000u;

// acc[v] |= sign-bearing margin of this condition (record format v4): the sign stays clear iff
// the condition holds. Cut conditions: m = fma(+-1, x, -c') exactly; others: an ordinary compare.
template <int V>
__device__ __forceinline__ void cond_mask(const uint4 r, const float *xl, uint32_t (&acc)[V])
{
    float x[V];
    load_vec<V>(xl + (r.x & OFF_MASK) * 4, x);
    const float v0 = __uint_as_float(r.z), v1 = __uint_as_float(r.w);
    if (!(r.x & (PAIR_BIT | GENERAL_BIT))) {
        const float2 s2 = make_float2(v0, v0), c2 = make_float2(v1, v1);
#pragma unroll
        for (int v = 0; v < V; v += 2) {
            const float2 m = __ffma2_rn(make_float2(x[v], x[v + 1]), s2, c2);
            acc[v] |= __float_as_uint(m.x);
            acc[v + 1] |= __float_as_uint(m.y);
        }
    } else if (r.x & PAIR_BIT) {
        float z[V];
        load_vec<V>(xl + (r.y & OFF_MASK) * 4, z);
#pragma unroll
        for (int v = 0; v < V; ++v)
            acc[v] |= (__fmul_rn(v0, x[v]) > __fmul_rn(v1, z[v])) ? 0u : SIGN;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] |= (__fmul_rn(v0, x[v]) > v1) ? 0u : SIGN;
    }
}

// Evaluate one set (records [rb, re), format v4) on this lane's V samples. hit[v] gets its sign
// bit set when the sample's prediction equals its label: in a tile of one label (`uniform`, label
// kmin) only rules of that class count; otherwise the per-sample label y[v] decides. y[v] < 0
// marks padding. All lanes of the warp call this together.
template <int V>
__device__ void eval_set_sign(const uint4 *recs, int rb, int re, uint4 *st, const float *xl, int lane,
                              int deflt, const int (&y)[V], bool uniform, int kmin, uint32_t (&hit)[V])
{
    const uint4 zero4 = make_uint4(0, 0, 0, 0);
    uint32_t claimed[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        claimed[v] = y[v] >= 0 ? 0u : SIGN;
        hit[v] = 0u;
    }
    int ck = 0;
    uint4 pf = zero4;
    if (rb < re) {
        __syncwarp();
        st[lane] = (rb + lane < re) ? __ldcg(recs + rb + lane) : zero4;
        st[32 + lane] = (rb + 32 + lane < re) ? __ldcg(recs + rb + 32 + lane) : zero4;
        pf = (rb + 64 + lane < re) ? __ldcg(recs + rb + 64 + lane) : zero4;
        __syncwarp();
    }
    int rel = 0;
    const int nrec = re - rb;
    while (rel < nrec) {
        while ((rel >> 5) > ck) {
            const uint4 keep = st[32 + lane];
            __syncwarp();
            st[lane] = keep;
            st[32 + lane] = pf;
            __syncwarp();
            ++ck;
            const int nx = rb + 32 * (ck + 2) + lane;
            pf = (nx < re) ? __ldcg(recs + nx) : zero4;
        }
        const uint4 *rp = st + (rel - 32 * ck);
        const uint4 r0 = rp[0];
        const int nc = max(1, (int)((r0.x >> LEN_SHIFT) & 0xFFFu));   // >= 1: progress
        const int cls = (int)(r0.y >> CLS_SHIFT);
        uint32_t acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = claimed[v];
        cond_mask<V>(r0, xl, acc);
        if (nc <= 33) {
#pragma unroll 2
            for (int k = 1; k < nc; ++k) cond_mask<V>(rp[k], xl, acc);
        } else {
            for (int k = 1; k < nc; ++k) cond_mask<V>(__ldcg(recs + rb + rel + k), xl, acc);
        }
        uint32_t all = SIGN;
        if (uniform) {
            const bool mine = cls == kmin;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint32_t fired = ~acc[v] & SIGN;
                claimed[v] |= fired;
                if (mine) hit[v] |= fired;
                all &= claimed[v];
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint32_t fired = ~acc[v] & SIGN;
                claimed[v] |= fired;
                hit[v] |= (y[v] == cls) ? fired : 0u;
                all &= claimed[v];
            }
        }
        if (__all_sync(FULL, all != 0u)) break;
        rel += nc;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t left = ~claimed[v] & SIGN;
        hit[v] |= (uniform ? (deflt == kmin) : (y[v] == deflt)) ? left : 0u;
    }
    __syncwarp();
}

}  // namespace core
}  // namespace rs
