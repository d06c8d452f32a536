// Device-resident evolution of a population of rule sets (tournament selection, uniform rule-list
// crossover, one mutation with randomized coefficients; Sec. 3), with periodic back-propagation
// fine-tuning of the best sets (Adam on a, b, t through the soft adjoint) used Baldwin-style: the
// tuned fitness (the better of before and after tuning) ranks the individual, its genome is kept
// unless write-back of improved coefficients is requested.
//
// The population lives in fixed slots on the device: rule r of set p at [p*RMAX + r], condition k
// at [(p*RMAX + r)*CMAX + k]. Per generation: slots -> CSR (two scans) -> packed hard evaluation
// -> ranking -> next generation into the second buffer. Nothing returns to the host until the run
// ends except the soft path's parameters, which stay on the device too.
//
// Random numbers: Philox4x64-10 (Salmon et al., SC'11), counter (i/4, child, generation, 0), key
// (seed, 0x65766f6c); draw i of a child is word i%4 of that block, exactly as the CPU reference.
#include <algorithm>
#include <vector>

#include "rs_internal.cuh"
#include "block_scan.cuh"
#include "graph_util.cuh"
#include "soft_step.cuh"

namespace rs {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;

struct PopDev {
    int32_t P, RMAX, CMAX;
    int32_t *nrule, *deflt, *rcls, *ncond, *cf, *cg;
    int8_t *cop;
    float *ca, *cb, *ct;
};

__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
        c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

struct Rng {
    uint64_t seed, gen, child, i;
    uint64_t blk[4];
    uint64_t cached = ~0ull;
    const uint64_t *pre = nullptr;   // blocks 0 .. npre-1 of this stream, computed ahead (4 words each)
    uint64_t npre = 0;
    __device__ uint64_t next()
    {
        const uint64_t b = i >> 2;
        if (b < npre) return pre[4 * b + (i++ & 3)];
        if (b != cached) {
            philox4x64_10(b, child, gen, 0, seed, 0x65766f6cull, blk);
            cached = b;
        }
        return blk[(i++) & 3];
    }
    __device__ int32_t uniform_int(int32_t n) { return (int32_t)(((next() >> 32) * (uint64_t)(uint32_t)n) >> 32); }
    __device__ float uniform01() { return __fmul_rn((float)(next() >> 40), 1.0f / 16777216.0f); }
    __device__ float coef() { return __fsub_rn(__fmul_rn(uniform01(), 2.0f), 1.0f); }
};

struct DataView {
    const float *Xt;      // [F][n_pad] label-grouped
    const int32_t *inv;   // caller index -> grouped position
    int64_t N, n_pad;
    int32_t F, K;
    __device__ float draw(Rng &r, int32_t f) const
    {
        const int64_t n = (int64_t)(((r.next() >> 32) * (uint64_t)N) >> 32);
        return Xt[(int64_t)f * n_pad + inv[n]];
    }
};

struct Cond { int32_t f, g; int8_t op; float a, b, t; };

__device__ void random_condition(Rng &r, const DataView &d, Cond &c)
{
    const bool pair = (r.uniform01() < 0.2f) && d.F > 1;
    c.f = r.uniform_int(d.F);
    c.g = -1;
    if (pair) {
        c.g = r.uniform_int(d.F - 1);
        if (c.g >= c.f) c.g += 1;
    }
    c.op = (int8_t)(r.next() & 1);
    c.a = r.coef();
    c.b = pair ? r.coef() : 0.0f;
    c.t = pair ? 0.0f : __fmul_rn(c.a, d.draw(r, c.f));
}

__device__ __forceinline__ bool better(const int32_t *fit, int i, int j)
{
    return fit[i] > fit[j] || (fit[i] == fit[j] && i < j);
}

// order[rank] = individual; rank = number of individuals ranked before it.
__global__ void k_rank(const int32_t *fit, int P, int32_t *order)
{
    __shared__ int32_t sf[1024];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int fi = i < P ? fit[i] : 0;
    int pos = 0;
    for (int base = 0; base < P; base += 1024) {
        __syncthreads();
        for (int j = threadIdx.x; j < 1024 && base + j < P; j += blockDim.x) sf[j] = fit[base + j];
        __syncthreads();
        const int lim = min(1024, P - base);
        if (i < P)
            for (int j = 0; j < lim; ++j) {
                const int fj = sf[j];
                pos += (fj > fi) || (fj == fi && base + j < i);
            }
    }
    if (i < P) order[pos] = i;
}

__device__ void copy_rule(const PopDev &src, int si, int sr, const PopDev &dst, int di, int dr, int lane, int nl)
{
    const int64_t s = (int64_t)si * src.RMAX + sr, d = (int64_t)di * dst.RMAX + dr;
    if (lane == 0) { dst.rcls[d] = src.rcls[s]; dst.ncond[d] = src.ncond[s]; }
    for (int k = lane; k < src.CMAX; k += nl) {
        const int64_t q = s * src.CMAX + k, w = d * dst.CMAX + k;
        dst.cf[w] = src.cf[q]; dst.cg[w] = src.cg[q]; dst.cop[w] = src.cop[q];
        dst.ca[w] = src.ca[q]; dst.cb[w] = src.cb[q]; dst.ct[w] = src.ct[q];
    }
}

__device__ void put_cond(const PopDev &p, int64_t rj, int k, const Cond &c)
{
    const int64_t q = rj * p.CMAX + k;
    p.cf[q] = c.f; p.cg[q] = c.g; p.cop[q] = c.op; p.ca[q] = c.a; p.cb[q] = c.b; p.ct[q] = c.t;
}

__device__ Cond get_cond(const PopDev &p, int64_t rj, int k)
{
    const int64_t q = rj * p.CMAX + k;
    return Cond{p.cf[q], p.cg[q], p.cop[q], p.ca[q], p.cb[q], p.ct[q]};
}

// Single-thread mutation of child c in `o` (same operator list and draw order as the reference).
__device__ void mutate(Rng &r, const PopDev &o, int c, const DataView &d)
{
    const int32_t type = r.uniform_int(8);
    const int64_t base = (int64_t)c * o.RMAX;
    int32_t nr = o.nrule[c];
    int32_t j, k;
    switch (type) {
    case 0: {
        j = r.uniform_int(nr); k = r.uniform_int(o.ncond[base + j]);
        Cond x = get_cond(o, base + j, k);
        x.a = r.coef();
        if (x.g >= 0) x.b = r.coef();
        else x.t = __fmul_rn(x.a, d.draw(r, x.f));
        put_cond(o, base + j, k, x);
        break;
    }
    case 1: {
        j = r.uniform_int(nr); k = r.uniform_int(o.ncond[base + j]);
        Cond x = get_cond(o, base + j, k);
        x.f = r.uniform_int(d.F);
        if (x.g >= 0) {
            x.g = r.uniform_int(d.F - 1);
            if (x.g >= x.f) x.g += 1;
        } else {
            x.t = __fmul_rn(x.a, d.draw(r, x.f));
        }
        put_cond(o, base + j, k, x);
        break;
    }
    case 2: {
        j = r.uniform_int(nr); k = r.uniform_int(o.ncond[base + j]);
        o.cop[(base + j) * o.CMAX + k] ^= 1;
        break;
    }
    case 3: {
        j = r.uniform_int(nr);
        const int32_t n = o.ncond[base + j];
        if (n < o.CMAX) {
            Cond x;
            random_condition(r, d, x);
            put_cond(o, base + j, n, x);
            o.ncond[base + j] = n + 1;
        }
        break;
    }
    case 4: {
        j = r.uniform_int(nr);
        const int32_t n = o.ncond[base + j];
        if (n > 1) {
            k = r.uniform_int(n);
            for (int q = k; q + 1 < n; ++q) put_cond(o, base + j, q, get_cond(o, base + j, q + 1));
            o.ncond[base + j] = n - 1;
        }
        break;
    }
    case 5: {
        if (nr < o.RMAX) {
            const int32_t pos = r.uniform_int(nr + 1);
            int32_t n = 1 + r.uniform_int(3);
            if (n > o.CMAX) n = o.CMAX;
            for (int q = nr; q > pos; --q) {
                o.rcls[base + q] = o.rcls[base + q - 1];
                o.ncond[base + q] = o.ncond[base + q - 1];
                for (int kk = 0; kk < o.CMAX; ++kk) put_cond(o, base + q, kk, get_cond(o, base + q - 1, kk));
            }
            o.ncond[base + pos] = n;
            for (int q = 0; q < n; ++q) {
                Cond x;
                random_condition(r, d, x);
                put_cond(o, base + pos, q, x);
            }
            o.rcls[base + pos] = r.uniform_int(d.K);
            o.nrule[c] = nr + 1;
        }
        break;
    }
    case 6: {
        if (nr > 1) {
            j = r.uniform_int(nr);
            for (int q = j; q + 1 < nr; ++q) {
                o.rcls[base + q] = o.rcls[base + q + 1];
                o.ncond[base + q] = o.ncond[base + q + 1];
                for (int kk = 0; kk < o.CMAX; ++kk) put_cond(o, base + q, kk, get_cond(o, base + q + 1, kk));
            }
            o.nrule[c] = nr - 1;
        }
        break;
    }
    default: {
        j = r.uniform_int(nr);
        o.rcls[base + j] = r.uniform_int(d.K);
        break;
    }
    }
}

// One warp per child: copies in parallel, random decisions on lane 0.
// gen = gen0 + *gidx: the generation index is read on the device, so that one captured graph
// serves every generation.
constexpr int NEXT_GEN_THREADS = 256;   // k_next_generation's block: 8 warps, one child each

__global__ void __launch_bounds__(NEXT_GEN_THREADS) k_next_generation(PopDev in, const int32_t *fit, const int32_t *order,
                                                                     PopDev out, uint64_t seed, uint64_t gen0,
                                                                     const int64_t *gidx, int elite, DataView d)
{
    __shared__ uint64_t pre_all[NEXT_GEN_THREADS / 32][32 * 4];
    const uint64_t gen = gen0 + (uint64_t)*gidx;
    const int lane = threadIdx.x & 31;
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= in.P) return;
    const int P = in.P;
    int A = 0, B = 0;
    uint32_t take_b = 0;
    // The child's draws are made by lane 0 one after another; the first 32 Philox blocks of its
    // stream (128 draws, more than a child usually takes) are computed ahead by the 32 lanes at
    // once. Same numbers, same order of use.
    uint64_t *pre = pre_all[threadIdx.x >> 5];
    {
        uint64_t blk[4];
        philox4x64_10((uint64_t)lane, (uint64_t)c, gen, 0, seed, 0x65766f6cull, blk);
#pragma unroll
        for (int k = 0; k < 4; ++k) pre[4 * lane + k] = blk[k];
    }
    __syncwarp();
    Rng r{seed, gen, (uint64_t)c, 0};
    r.pre = pre;
    r.npre = 32;
    if (c < elite) {
        A = order[c];
    } else if (lane == 0) {
        int i = r.uniform_int(P), j = r.uniform_int(P);
        A = better(fit, i, j) ? i : j;
        i = r.uniform_int(P); j = r.uniform_int(P);
        B = better(fit, i, j) ? i : j;
        if (r.uniform01() < 0.5f) {
            const int na = in.nrule[A], nb = in.nrule[B];
            for (int q = 0; q < na; ++q)
                if (q < nb && (r.next() & 1)) take_b |= 1u << q;
        }
    }
    A = __shfl_sync(FULL, A, 0);
    B = __shfl_sync(FULL, B, 0);
    take_b = __shfl_sync(FULL, take_b, 0);
    if (lane == 0) { out.nrule[c] = in.nrule[A]; out.deflt[c] = in.deflt[A]; }
    for (int q = 0; q < in.RMAX; ++q) {
        const bool fromb = (take_b >> q) & 1u;
        copy_rule(in, fromb ? B : A, q, out, c, q, lane, 32);
    }
    __syncwarp();
    if (c >= elite && lane == 0) {
        // continue the child's draw sequence (the warp-wide copy did not draw)
        if (r.uniform01() < 0.9f) mutate(r, out, c, d);
    }
}

// ---------------------------------------------------------------- slots -> CSR

__global__ void k_count_conds(PopDev p, int32_t *rule_len, int32_t *set_len)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // one thread per set
    if (i >= p.P) return;
    const int nr = p.nrule[i];
    int tot = 0;
    for (int j = 0; j < nr; ++j) tot += p.ncond[(int64_t)i * p.RMAX + j];
    set_len[i] = tot;
    rule_len[i] = nr;
}

// Exclusive scan of n ints with one CTA (n up to a few million: strided chunks).
__global__ void k_scan1(const int32_t *in, int n, int32_t *out /*n+1*/)
{
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += in[i];
    int total = 0;
    int run = block_exclusive_scan(s, &total);
    if (t == 0) out[n] = total;
    for (int i = lo; i < hi; ++i) { out[i] = run; run += in[i]; }
}

struct CsrDev {
    int32_t *set_rule_off, *rule_cond_off, *rule_class, *set_default, *cond_f, *cond_g;
    int8_t *cond_op;
    float *cond_a, *cond_b, *cond_t;
    int32_t *cond_slot;    // flat slot index of each CSR condition (for parameter write-back)
};

// Set w of the batch (slot subset[w], or w) written by one warp at its scanned offsets: lane j
// takes rule j (a set has at most 32 rules), the rules' condition offsets from a warp scan of
// their counts, so that no lane waits on another's loads. The whole warp calls it.
__device__ void scatter_set(const PopDev &p, const int32_t *set_first_rule, const int32_t *set_first_cond,
                            const int32_t *subset, int w, const CsrDev &o, int lane)
{
    const int i = subset ? subset[w] : w;
    const int nr = p.nrule[i];
    const int r0 = set_first_rule[w];
    if (lane == 0) {
        o.set_rule_off[w] = r0;
        o.set_default[w] = p.deflt[i];
    }
    const int64_t rj = (int64_t)i * p.RMAX + lane;
    const int nc = lane < nr ? p.ncond[rj] : 0;
    int x = nc;
    for (int s = 1; s < 32; s <<= 1) {
        const int y = __shfl_up_sync(FULL, x, s);
        if (lane >= s) x += y;
    }
    if (lane < nr) {
        const int c = set_first_cond[w] + x - nc;
        o.rule_cond_off[r0 + lane] = c;
        o.rule_class[r0 + lane] = p.rcls[rj];
        for (int k = 0; k < nc; ++k) {
            const int64_t q = rj * p.CMAX + k;
            o.cond_f[c + k] = p.cf[q]; o.cond_g[c + k] = p.cg[q]; o.cond_op[c + k] = p.cop[q];
            o.cond_a[c + k] = p.ca[q]; o.cond_b[c + k] = p.cb[q]; o.cond_t[c + k] = p.ct[q];
            if (o.cond_slot) o.cond_slot[c + k] = (int32_t)q;
        }
    }
}

// One warp per set: write its rules and conditions at the scanned offsets; the first thread also
// closes the offset arrays.
__global__ void k_scatter_csr(PopDev p, const int32_t *set_first_rule, const int32_t *set_first_cond,
                              const int32_t *subset, int nsub, CsrDev o)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        o.set_rule_off[nsub] = set_first_rule[nsub];
        o.rule_cond_off[set_first_rule[nsub]] = set_first_cond[nsub];
    }
    if (w < nsub) scatter_set(p, set_first_rule, set_first_cond, subset, w, o, threadIdx.x & 31);
}

// CSR offsets of at most 1024 sets in one CTA of 1024 threads: the rule and condition counts of
// set subset[i] (or i) scanned into first_rule / first_cond [nsub + 1] (and the closing offsets).
// Replaces the counting, gathering and the two scans of the general path for small populations;
// the sets themselves are written by k_scatter_csr, a warp each across the GPU (writing them with
// this one CTA's warps in turn was slower).
__global__ void k_csr_offsets_small(PopDev p, const int32_t *subset, int nsub, int32_t *first_rule,
                                    int32_t *first_cond)
{
    const int i = threadIdx.x;
    int nr = 0, nc = 0;
    if (i < nsub) {
        const int src = subset ? subset[i] : i;
        nr = p.nrule[src];
        for (int j = 0; j < nr; ++j) nc += p.ncond[(int64_t)src * p.RMAX + j];
    }
    int tr = 0, tc = 0;
    const int er = block_exclusive_scan(nr, &tr);
    const int ec = block_exclusive_scan(nc, &tc);
    if (i < nsub) {
        first_rule[i] = er;
        first_cond[i] = ec;
    }
    if (i == 0) {
        first_rule[nsub] = tr;
        first_cond[nsub] = tc;
    }
}

__global__ void k_gather_len(const int32_t *len, const int32_t *subset, int n, int32_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = len[subset ? subset[i] : i];
}

// ---------------------------------------------------------------- tuning


// Fine-tuning refines fitness and never lowers it: a tuned set keeps the better of its fitness
// before and after tuning; `improved` marks the sets whose tuned coefficients did better.
__global__ void k_scatter_fit(const int32_t *tuned, const int32_t *subset, int n, int32_t *fit,
                              int32_t *improved)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = subset[i];
    improved[i] = tuned[i] > fit[s];
    fit[s] = max(fit[s], tuned[i]);
}

// Write-back of improved tuned coefficients into the genome (one warp per tuned set).
__global__ void k_write_back(const float *a, const float *b, const float *t, const int32_t *slot,
                             const int32_t *first_cond, const int32_t *improved, int n, PopDev p)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n || !improved[i]) return;
    for (int c = first_cond[i] + lane; c < first_cond[i + 1]; c += 32) {
        const int q = slot[c];
        p.ca[q] = a[c]; p.cb[q] = b[c]; p.ct[q] = t[c];
    }
}

// best[g] and mean[g] for g = *gidx; writes g + 1 to *gnext when given (one CTA of 1024 threads).
__device__ void stats_block(const int32_t *fit, int P, int32_t *best, double *mean, const int64_t *gidx,
                            int64_t *gnext)
{
    __shared__ long long ssum[1024];
    __shared__ int smax[1024];
    long long s = 0;
    int mx = INT32_MIN;
    for (int i = threadIdx.x; i < P; i += blockDim.x) { s += fit[i]; mx = max(mx, fit[i]); }
    ssum[threadIdx.x] = s;
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ssum[threadIdx.x] += ssum[threadIdx.x + w];
            smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t gen = *gidx;
        best[gen] = smax[0];
        mean[gen] = (double)ssum[0] / (double)P;
        if (gnext) *gnext = gen + 1;
    }
}

__global__ void k_stats(const int32_t *fit, int P, int32_t *best, double *mean, const int64_t *gidx,
                        int64_t *gnext)
{
    stats_block(fit, P, best, mean, gidx, gnext);
}

// k_stats and k_rank in one CTA of 1024 threads, for P <= 1024: the same statistics and the same
// order (fitness descending, index ascending among equals).
__global__ void k_stats_rank_small(const int32_t *fit, int P, int32_t *best, double *mean, const int64_t *gidx,
                                   int64_t *gnext, int32_t *order)
{
    __shared__ int32_t sf[1024];
    const int i = threadIdx.x;
    if (i < P) sf[i] = fit[i];
    stats_block(fit, P, best, mean, gidx, gnext);      // synchronises the block
    if (i < P) {
        const int fi = sf[i];
        int pos = 0;
        for (int j = 0; j < P; ++j) {
            const int fj = sf[j];
            pos += (fj > fi) || (fj == fi && j < i);
        }
        order[pos] = i;
    }
}

}  // namespace

// ---------------------------------------------------------------- host orchestration

struct EvolveBuffers {
    std::vector<void *> allocs;
    template <class T> rs_status get(T **p, size_t n)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(evolution buffers)");
        allocs.push_back(q);
        *p = static_cast<T *>(q);
        return RS_OK;
    }
    ~EvolveBuffers() { for (void *q : allocs) cudaFree(q); }
};

static rs_status alloc_pop(EvolveBuffers &B, PopDev &p, int P, int RMAX, int CMAX)
{
    p.P = P; p.RMAX = RMAX; p.CMAX = CMAX;
    const size_t R = (size_t)P * RMAX, C = R * CMAX;
    rs_status rc;
    if ((rc = B.get(&p.nrule, P)) || (rc = B.get(&p.deflt, P)) || (rc = B.get(&p.rcls, R)) ||
        (rc = B.get(&p.ncond, R)) || (rc = B.get(&p.cf, C)) || (rc = B.get(&p.cg, C)) ||
        (rc = B.get(&p.cop, C)) || (rc = B.get(&p.ca, C)) || (rc = B.get(&p.cb, C)) ||
        (rc = B.get(&p.ct, C)))
        return rc;
    return RS_OK;
}

// CSR of a subset (or all) of the population into preallocated arrays (capacity: whole population).
struct CsrWork {
    CsrDev o;
    int32_t *rule_len, *cond_len, *sub_rule_len, *sub_cond_len, *first_rule, *first_cond;
};

// Slots -> CSR batch of nsub sets (subset[i], or the first nsub); returns the kernels launched.
static int build_csr(const PopDev &p, const int32_t *subset, int nsub, CsrWork &w, cudaStream_t s)
{
    int n = 1;
    if (nsub <= 1024) {
        k_csr_offsets_small<<<1, 1024, 0, s>>>(p, subset, nsub, w.first_rule, w.first_cond);
    } else {
        k_count_conds<<<(p.P + 255) / 256, 256, 0, s>>>(p, w.rule_len, w.cond_len);
        k_gather_len<<<(nsub + 255) / 256, 256, 0, s>>>(w.rule_len, subset, nsub, w.sub_rule_len);
        k_gather_len<<<(nsub + 255) / 256, 256, 0, s>>>(w.cond_len, subset, nsub, w.sub_cond_len);
        k_scan1<<<1, 1024, 0, s>>>(w.sub_rule_len, nsub, w.first_rule);
        k_scan1<<<1, 1024, 0, s>>>(w.sub_cond_len, nsub, w.first_cond);
        n = 5;
    }
    k_scatter_csr<<<std::max(1, (nsub * 32 + 255) / 256), 256, 0, s>>>(p, w.first_rule, w.first_cond, subset,
                                                                      nsub, w.o);
    return n + 1;
}

rs_status evolve_run(Ctx *ctx, uint64_t ds_h, const rs_evolve_config *cfg, rs_population *hp,
                     int32_t *best_out, double *mean_out, cudaStream_t s)
{
    std::shared_ptr<Dataset> dsp;
    if (rs_status urc = use_dataset(ctx, ds_h, &dsp)) return urc;
    DatasetUseMark use_mark{ctx, dsp.get(), s};
    Dataset &ds = *dsp;
    const int P = cfg->P, RMAX = cfg->RMAX, CMAX = cfg->CMAX;
    if (P < 2 || RMAX < 1 || RMAX > 32 || CMAX < 1 || CMAX > 64 || cfg->generations < 0 ||
        cfg->first_generation < 0 || cfg->elite < 0 || cfg->elite > P || cfg->tune_top < 0 || cfg->tune_top > P ||
        cfg->tune_steps < 0 || !(cfg->tau > 0.f) || !hp) {
        set_error("bad evolution configuration");
        return RS_ERR_INVALID;
    }
    rs_status rc = device_guard(ctx);
    if (rc) return rc;
    // the slot counts bound every read of the slot arrays: check them before anything runs (the
    // rest of a genome, features, classes and operators, is validated by the packing)
    if (!hp->nrule || !hp->deflt || !hp->rcls || !hp->ncond || !hp->cf || !hp->cg || !hp->cop || !hp->ca ||
        !hp->cb || !hp->ct) {
        set_error("evolution: a population array is NULL");
        return RS_ERR_INVALID;
    }
    for (int q = 0; q < P; ++q) {
        const int32_t nr = hp->nrule[q];
        bool ok = nr >= 0 && nr <= RMAX;
        for (int j = 0; ok && j < nr; ++j) {
            const int32_t nc = hp->ncond[(size_t)q * RMAX + j];
            ok = nc >= 0 && nc <= CMAX;
        }
        if (!ok) {
            set_error("evolution: set %d has a rule or condition count outside 0..RMAX / 0..CMAX", q);
            return RS_ERR_INVALID;
        }
    }
    EvolveBuffers B;
    PopDev pop[2];
    if ((rc = alloc_pop(B, pop[0], P, RMAX, CMAX)) || (rc = alloc_pop(B, pop[1], P, RMAX, CMAX))) return rc;
    const size_t R = (size_t)P * RMAX, C = R * CMAX;
    // upload the initial population
    RS_CUDA(cudaMemcpyAsync(pop[0].nrule, hp->nrule, 4 * P, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].deflt, hp->deflt, 4 * P, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].rcls, hp->rcls, 4 * R, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].ncond, hp->ncond, 4 * R, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].cf, hp->cf, 4 * C, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].cg, hp->cg, 4 * C, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].cop, hp->cop, C, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].ca, hp->ca, 4 * C, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].cb, hp->cb, 4 * C, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemcpyAsync(pop[0].ct, hp->ct, 4 * C, cudaMemcpyHostToDevice, s));

    // work arrays
    CsrWork w{};
    if ((rc = B.get(&w.o.set_rule_off, P + 1)) || (rc = B.get(&w.o.rule_cond_off, R + 1)) ||
        (rc = B.get(&w.o.rule_class, R)) || (rc = B.get(&w.o.set_default, P)) ||
        (rc = B.get(&w.o.cond_f, C)) || (rc = B.get(&w.o.cond_g, C)) || (rc = B.get(&w.o.cond_op, C)) ||
        (rc = B.get(&w.o.cond_a, C)) || (rc = B.get(&w.o.cond_b, C)) || (rc = B.get(&w.o.cond_t, C)) ||
        (rc = B.get(&w.o.cond_slot, C)) || (rc = B.get(&w.rule_len, P)) || (rc = B.get(&w.cond_len, P)) ||
        (rc = B.get(&w.sub_rule_len, P)) || (rc = B.get(&w.sub_cond_len, P)) ||
        (rc = B.get(&w.first_rule, P + 1)) || (rc = B.get(&w.first_cond, P + 1)))
        return rc;
    int32_t *fit = nullptr, *order = nullptr, *best = nullptr, *tuned_fit = nullptr, *improved = nullptr;
    double *mean = nullptr;
    Scratch sc;
    const int G = cfg->generations;
    if ((rc = B.get(&fit, P)) || (rc = B.get(&order, P)) || (rc = B.get(&best, G + 1)) ||
        (rc = B.get(&mean, G + 1)) || (rc = B.get(&tuned_fit, P)) || (rc = B.get(&improved, P)) ||
        (rc = B.get(&sc.recs, C)) ||
        (rc = B.get(&sc.sets, P)) || (rc = B.get(&sc.order, P)) || (rc = B.get(&sc.status, 64)))
        return rc;
    if (ds.K <= LAST_END_MAX_K && (rc = B.get(&sc.last_end, (size_t)P * ds.K))) return rc;
    // tuning buffers (a, b, t copies, grads, Adam moments, per-set loss / dloss)
    const int T = cfg->tune_top;
    const size_t TC = (size_t)std::max(1, T) * RMAX * CMAX;
    float *ta, *tb, *tt, *ga, *gb, *gt, *mo, *ve, *loss, *dl;
    if ((rc = B.get(&ta, TC)) || (rc = B.get(&tb, TC)) || (rc = B.get(&tt, TC)) || (rc = B.get(&ga, TC)) ||
        (rc = B.get(&gb, TC)) || (rc = B.get(&gt, TC)) || (rc = B.get(&mo, 2 * TC)) ||
        (rc = B.get(&ve, 2 * TC)) || (rc = B.get(&loss, std::max(1, T))) || (rc = B.get(&dl, std::max(1, T))))
        return rc;
    std::vector<float> ones(std::max(1, T), 1.0f);
    RS_CUDA(cudaMemcpyAsync(dl, ones.data(), 4 * ones.size(), cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemsetAsync(sc.status, 0, 4, s));

    DataView dv{ds.Xt, ds.inv, ds.N, ds.n_pad, ds.F, ds.K};
    // a configuration forced on the context (rs_set_tile_config) applies here too, else the heuristic
    const TileConfig &tc = tile_config(ctx->forced_tile >= 0 && tile_config_fits(tile_config(ctx->forced_tile), ds.F)
                                           ? ctx->forced_tile
                                           : heuristic_tile_for(ds));
    auto evaluate = [&](int nsub, int32_t *out_fit, cudaStream_t st) -> rs_status {
        BatchDev bd{};
        bd.P = nsub;
        bd.R = (int32_t)((size_t)nsub * RMAX);          // capacities; real sizes are on the device
        bd.C = (int32_t)((size_t)nsub * RMAX * CMAX);
        bd.set_rule_off = w.o.set_rule_off; bd.rule_cond_off = w.o.rule_cond_off;
        bd.rule_class = w.o.rule_class; bd.set_default = w.o.set_default;
        bd.cond_f = w.o.cond_f; bd.cond_g = w.o.cond_g; bd.cond_op = w.o.cond_op;
        bd.cond_a = w.o.cond_a; bd.cond_b = w.o.cond_b; bd.cond_t = w.o.cond_t;
        return enqueue_hard_dev_sizes(ctx, &ds, tc, bd, w.first_rule + nsub, w.first_cond + nsub, sc,
                                      out_fit, nullptr, nullptr, st);
    };

    // The generation index lives on the device: while generation g runs, slot g & 1 holds g and
    // k_stats writes g + 1 into the other slot. With the population buffers also alternating by
    // the parity of g, a generation's work depends on the host only through (parity, tuning), so
    // one captured graph per pair serves every generation.
    int64_t *gslot = nullptr;
    void *soft_scratch = nullptr;
    const int64_t soft_cap_c = (int64_t)TC;
    if ((rc = B.get(&gslot, 2)) ||
        (T > 0 && (rc = B.get(reinterpret_cast<char **>(&soft_scratch), soft_scratch_bytes(soft_cap_c, T, ds.N)))))
        return rc;
    RS_CUDA(cudaMemsetAsync(gslot, 0, 2 * sizeof(int64_t), s));

    auto generation = [&](int par, bool tune, bool last, cudaStream_t st) -> rs_status {
        PopDev &in = pop[par];
        rs_status grc;
        count_launch(ctx, build_csr(in, nullptr, P, w, st));
        if ((grc = evaluate(P, fit, st))) return grc;
        if (tune) {
            k_rank<<<(P + 255) / 256, 256, 0, st>>>(fit, P, order);
            count_launch(ctx, 1 + build_csr(in, order, T, w, st));   // the T best, in rank order
            RS_CUDA(cudaMemcpyAsync(ta, w.o.cond_a, 4 * TC, cudaMemcpyDeviceToDevice, st));
            RS_CUDA(cudaMemcpyAsync(tb, w.o.cond_b, 4 * TC, cudaMemcpyDeviceToDevice, st));
            RS_CUDA(cudaMemcpyAsync(tt, w.o.cond_t, 4 * TC, cudaMemcpyDeviceToDevice, st));
            RS_CUDA(cudaMemsetAsync(mo, 0, 8 * TC, st));
            RS_CUDA(cudaMemsetAsync(ve, 0, 8 * TC, st));
            SoftArgs sa{};
            sa.b.P = T;
            sa.b.R = (int32_t)((size_t)T * RMAX);
            sa.b.C = (int32_t)TC;
            sa.b.dR = w.first_rule + T;
            sa.b.dC = w.first_cond + T;
            sa.b.set_rule_off = w.o.set_rule_off; sa.b.rule_cond_off = w.o.rule_cond_off;
            sa.b.rule_class = w.o.rule_class; sa.b.set_default = w.o.set_default;
            sa.b.cond_f = w.o.cond_f; sa.b.cond_g = w.o.cond_g; sa.b.cond_op = w.o.cond_op;
            sa.b.cond_a = ta; sa.b.cond_b = tb; sa.b.cond_t = tt;
            sa.Xt = ds.Xt; sa.y = ds.y; sa.perm = ds.perm; sa.N = ds.N; sa.n_pad = ds.n_pad;
            sa.F = ds.F; sa.K = ds.K; sa.tau = cfg->tau; sa.loss = loss; sa.dloss = dl;
            sa.grad_a = ga; sa.grad_b = gb; sa.grad_t = gt; sa.status = sc.status;
            SoftAdam adam;                                      // applied by the gradient reduction
            adam.a = ta; adam.b = tb; adam.t = tt; adam.m = mo; adam.v = ve; adam.lr = cfg->lr;
            for (int step = 1; step <= cfg->tune_steps; ++step) {
                adam.step = step;
                if ((grc = soft_step_scratch(ctx, sa, RMAX, RMAX * CMAX, soft_scratch, soft_cap_c, T, step > 1,
                                             &adam, st)))
                    return grc;
            }
            // tuned fitness of the T sets (hard evaluation with the tuned coefficients)
            RS_CUDA(cudaMemcpyAsync(w.o.cond_a, ta, 4 * TC, cudaMemcpyDeviceToDevice, st));
            RS_CUDA(cudaMemcpyAsync(w.o.cond_b, tb, 4 * TC, cudaMemcpyDeviceToDevice, st));
            RS_CUDA(cudaMemcpyAsync(w.o.cond_t, tt, 4 * TC, cudaMemcpyDeviceToDevice, st));
            if ((grc = evaluate(T, tuned_fit, st))) return grc;
            k_scatter_fit<<<(T + 255) / 256, 256, 0, st>>>(tuned_fit, order, T, fit, improved);
            if (cfg->lamarckian)
                k_write_back<<<(T * 32 + 255) / 256, 256, 0, st>>>(ta, tb, tt, w.o.cond_slot, w.first_cond,
                                                                 improved, T, in);
            count_launch(ctx, 2 + (cfg->lamarckian ? 1 : 0));
        }
        if (!last && P <= 1024) {
            k_stats_rank_small<<<1, 1024, 0, st>>>(fit, P, best, mean, gslot + par, gslot + (par ^ 1), order);
            count_launch(ctx);
        } else {
            k_stats<<<1, 1024, 0, st>>>(fit, P, best, mean, gslot + par, last ? nullptr : gslot + (par ^ 1));
            count_launch(ctx);
            if (last) return RS_OK;
            k_rank<<<(P + 255) / 256, 256, 0, st>>>(fit, P, order);
            count_launch(ctx);
        }
        k_next_generation<<<(P * 32 + NEXT_GEN_THREADS - 1) / NEXT_GEN_THREADS, NEXT_GEN_THREADS, 0, st>>>(
            in, fit, order, pop[par ^ 1], cfg->seed, (uint64_t)cfg->first_generation, gslot + par, cfg->elite, dv);
        count_launch(ctx);
        RS_CUDA(cudaGetLastError());
        return RS_OK;
    };

    // Captured generations (on a stream of their own), unless the context launches directly.
    struct GenGraphs {
        cudaStream_t cs = nullptr;
        cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
        int kernels[2][2] = {{0, 0}, {0, 0}};
        ~GenGraphs()
        {
            for (auto &row : exec)
                for (auto e : row)
                    if (e) cudaGraphExecDestroy(e);
            if (cs) cudaStreamDestroy(cs);
        }
    } gg;
    const bool graphs = !(ctx->flags & (RS_CTX_NO_GRAPH | RS_CTX_PROFILE));
    for (int g = 0; g <= G; ++g) {
        const int par = g & 1;
        const bool last = g == G;
        const bool tune = cfg->tune_every > 0 && T > 0 && cfg->tune_steps > 0 && !last &&
                          ((cfg->first_generation + g) % cfg->tune_every) == cfg->tune_every - 1;
        if (!graphs || last) {
            if ((rc = generation(par, tune, last, s))) return rc;
            continue;
        }
        cudaGraphExec_t &ex = gg.exec[par][tune];
        if (!ex) {
            if (!gg.cs) RS_CUDA(cudaStreamCreateWithFlags(&gg.cs, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            RS_CUDA(cudaStreamBeginCapture(gg.cs, cudaStreamCaptureModeThreadLocal));
            const rs_status crc = generation(par, tune, false, gg.cs);
            const cudaError_t ce = cudaStreamEndCapture(gg.cs, &graph);
            if (crc) { if (graph) cudaGraphDestroy(graph); return crc; }
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture(generation)");
            const cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
            gg.kernels[par][tune] = graph_kernel_nodes(graph);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) { ex = nullptr; return cuda_fail(ie, "cudaGraphInstantiate(generation)"); }
        } else {
            count_launch(ctx, gg.kernels[par][tune]);
        }
        RS_CUDA(cudaGraphLaunch(ex, s));
    }
    const int cur = (G & 1);
    // results
    PopDev &fin = pop[cur];
    RS_CUDA(cudaMemcpyAsync(hp->nrule, fin.nrule, 4 * P, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->deflt, fin.deflt, 4 * P, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->rcls, fin.rcls, 4 * R, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->ncond, fin.ncond, 4 * R, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->cf, fin.cf, 4 * C, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->cg, fin.cg, 4 * C, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->cop, fin.cop, C, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->ca, fin.ca, 4 * C, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->cb, fin.cb, 4 * C, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(hp->ct, fin.ct, 4 * C, cudaMemcpyDeviceToHost, s));
    if (hp->fitness) RS_CUDA(cudaMemcpyAsync(hp->fitness, fit, 4 * P, cudaMemcpyDeviceToHost, s));
    if (best_out) RS_CUDA(cudaMemcpyAsync(best_out, best, 4 * (G + 1), cudaMemcpyDeviceToHost, s));
    if (mean_out) RS_CUDA(cudaMemcpyAsync(mean_out, mean, 8 * (G + 1), cudaMemcpyDeviceToHost, s));
    uint32_t st = 0;
    RS_CUDA(cudaMemcpyAsync(&st, sc.status, 4, cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaStreamSynchronize(s));
    if (st) {
        set_error("evolution: %s", status_text(st).c_str());
        return RS_ERR_INVALID;
    }
    return RS_OK;
}

// Full-batch Adam fine-tuning of the coefficients and thresholds of a device batch (Sec. 3: 50
// epochs of gradient updates in the paper's example), the same step the evolution loop uses.
rs_status finetune_run(Ctx *ctx, uint64_t ds_h, const rs_batch *b, float *pa, float *pb, float *pt,
                       float tau, float lr, int steps, float *loss_trace, cudaStream_t s)
{
    std::shared_ptr<Dataset> dsp;
    if (rs_status urc = use_dataset(ctx, ds_h, &dsp)) return urc;
    DatasetUseMark use_mark{ctx, dsp.get(), s};
    if (!b || b->mem != RS_MEM_DEVICE || b->P < 0 || b->R < 0 || b->C < 0 || steps < 0 ||
        !(tau > 0.f) || (b->C > 0 && (!pa || !pb || !pt))) {
        set_error("rs_finetune: bad arguments (device batch, parameters and steps >= 0 required)");
        return RS_ERR_INVALID;
    }
    rs_status rc = device_guard(ctx);
    if (rc) return rc;
    if (b->P == 0 || steps == 0) return RS_OK;
    Dataset &ds = *dsp;
    EvolveBuffers B;
    const size_t C = std::max(b->C, 1), P = b->P;
    float *ga = nullptr, *gb = nullptr, *gt = nullptr, *mo = nullptr, *ve = nullptr, *loss = nullptr,
          *dl = nullptr;
    uint32_t *status = nullptr;
    if ((rc = B.get(&ga, C)) || (rc = B.get(&gb, C)) || (rc = B.get(&gt, C)) || (rc = B.get(&mo, 2 * C)) ||
        (rc = B.get(&ve, 2 * C)) || (rc = B.get(&loss, P)) || (rc = B.get(&dl, P)) ||
        (rc = B.get(&status, 64)))
        return rc;
    std::vector<float> ones(P, 1.0f);
    RS_CUDA(cudaMemcpyAsync(dl, ones.data(), 4 * P, cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaMemsetAsync(mo, 0, 8 * C, s));
    RS_CUDA(cudaMemsetAsync(ve, 0, 8 * C, s));
    RS_CUDA(cudaMemsetAsync(status, 0, 4, s));
    SoftArgs sa{};
    sa.b.P = b->P; sa.b.R = b->R; sa.b.C = b->C;
    sa.b.set_rule_off = b->set_rule_off; sa.b.rule_cond_off = b->rule_cond_off;
    sa.b.rule_class = b->rule_class; sa.b.set_default = b->set_default;
    sa.b.cond_f = b->cond_f; sa.b.cond_g = b->cond_g; sa.b.cond_op = b->cond_op;
    sa.b.cond_a = pa; sa.b.cond_b = pb; sa.b.cond_t = pt;
    sa.b.cond_set = b->cond_set;          // membership tests: indicators, no gradient, unchanged
    sa.Xt = ds.Xt; sa.y = ds.y; sa.perm = ds.perm; sa.N = ds.N; sa.n_pad = ds.n_pad;
    sa.F = ds.F; sa.K = ds.K; sa.tau = tau; sa.loss = loss; sa.dloss = dl;
    sa.grad_a = ga; sa.grad_b = gb; sa.grad_t = gt; sa.status = status;
    // validate once (the structure does not change between steps), then run the steps back to back
    // on scratch allocated once, the per-step losses kept on the device until the end
    int maxR = 1, maxC = 1;
    if ((rc = soft_validate(ctx, sa, &maxR, &maxC, s))) return rc;
    void *scratch = nullptr;
    float *trace = nullptr;
    if ((rc = B.get(reinterpret_cast<char **>(&scratch), soft_scratch_bytes((int64_t)C, (int)P, ds.N))) ||
        (loss_trace && (rc = B.get(&trace, (size_t)steps * P))))
        return rc;
    SoftAdam adam;                                              // applied by the gradient reduction
    adam.a = pa; adam.b = pb; adam.t = pt; adam.m = mo; adam.v = ve; adam.lr = lr;
    for (int step = 1; step <= steps; ++step) {
        sa.loss = trace ? trace + (size_t)(step - 1) * P : loss;
        adam.step = step;
        if ((rc = soft_step_scratch(ctx, sa, maxR, maxC, scratch, (int64_t)C, (int)P, step > 1,
                                    b->C > 0 ? &adam : nullptr, s)))
            return rc;
    }
    if (trace) RS_CUDA(cudaMemcpyAsync(loss_trace, trace, sizeof(float) * (size_t)steps * P, cudaMemcpyDeviceToHost, s));
    uint32_t st = 0;
    RS_CUDA(cudaMemcpyAsync(&st, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaStreamSynchronize(s));
    if (st) {
        set_error("fine-tuning: %s", status_text(st).c_str());
        return (st & ST_TOO_LARGE) ? RS_ERR_TOO_LARGE : RS_ERR_INVALID;
    }
    return RS_OK;
}

}  // namespace rs
