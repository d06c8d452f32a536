/*
 * Plain CPU oracle for ordered rule-set evaluation (test infrastructure).
 *
 * This file is a slow, obviously-correct restatement of what the method computes. It is used
 * only by the test suite, the smoke check and the CPU baseline of the benchmark; the library
 * never links or calls it, and it shares no code with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC (no FMA contraction,
 * no flush-to-zero), so every float32 product below is one correctly rounded multiply.
 *
 * Semantics followed (paper: "GPU-Accelerated Rule Evaluation and Evolution", GECCO'25 Comp.):
 *  - Sec. 3 and Fig. 1a/1b: a condition is an inequality over one feature and a threshold, or
 *    over two features (the "0.38 x worst compactness" row); the activation maps a negative
 *    margin to false and a positive one to true. A zero margin is false (strict compare).
 *  - Fig. 1b: a rule is the conjunction ("&") of its conditions and names one class.
 *  - Sec. 1 / Sec. 3 (list-based grammar): a rule set is an ordered list; the first rule that
 *    fires gives the class; when none fires the set's default class applies.
 *  - Sec. 1: fitness is classification accuracy, here the exact correct counts.
 *  - Sec. 3: a sigmoid activation makes evaluation differentiable so that back-propagation can
 *    tune coefficients and thresholds with the structure kept (Fig. 1c).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - compare form lhs = fl32(a*x[f]), rhs = t or fl32(b*x[g]); true iff lhs > rhs (op '>') or
 *    lhs < rhs (op '<'), IEEE ordered, so NaN is false;
 *  - an empty rule fires; an empty set predicts its default;
 *  - soft relaxation: q_r = prod_c sigmoid(s*(lhs-rhs)/tau), first-fire probability
 *    q_r * prod_{j<r} (1-q_j), the default class takes prod_j (1-q_j), loss = mean_n -log p(y_n),
 *    all in float64 in the log domain.
 *  - categorical features (Sec. 5 names them as future work): a feature may hold integer category
 *    codes stored as floats; a membership condition (op 2) on feature f with category set S
 *    (a 64-bit mask, bit k = code k) is true iff x[f] is an integer k with 0 <= k <= 63 and k is
 *    in S, false otherwise (other values, NaN). It has no coefficient, so the soft relaxation
 *    keeps it as its exact indicator (a factor 1 or 0 of q_r) and it has no gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ORC_PLANT selects a deliberately wrong variant, built only by the test that checks that the
 * pins catch it (0 = the oracle as stated). */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

typedef struct {
    int32_t P;
    const int32_t *set_rule_off, *rule_cond_off, *rule_class, *set_default;
    const int32_t *cond_f, *cond_g;
    const int8_t *cond_op;
    const float *cond_a, *cond_b, *cond_t;
    const uint64_t *cond_set;    /* category sets of op-2 conditions; NULL if there are none */
} orc_batch;

int orc_num_threads(int requested)
{
#ifdef _OPENMP
    if (requested > 0) return requested;
    return omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

/* Membership of one value in a category set: an integer code 0..63 whose bit is set. */
static int in_set(float x, uint64_t set)
{
    if (!(x >= 0.0f && x <= 63.0f)) return 0;      /* also false for NaN */
    const int k = (int)x;
#if ORC_PLANT == 8
    (void)0;                                       /* planted: a fractional value keeps its code */
#else
    if ((float)k != x) return 0;                   /* not an integer code */
#endif
#if ORC_PLANT == 9
    return (int)((set >> (63 - k)) & 1u);          /* planted: bits read from the top */
#else
    return (int)((set >> k) & 1u);
#endif
}

/* One condition on one sample, exactly as defined: two rounded float32 products, one compare
 * (or, for op 2, the category membership of x[f]). */
static int cond_true(const orc_batch *b, int64_t c, const float *xrow)
{
    if (b->cond_op[c] == 2) return b->cond_set ? in_set(xrow[b->cond_f[c]], b->cond_set[c]) : 0;
    float lhs = b->cond_a[c] * xrow[b->cond_f[c]];
    float rhs = (b->cond_g[c] < 0) ? b->cond_t[c] : b->cond_b[c] * xrow[b->cond_g[c]];
#if ORC_PLANT == 1
    if (b->cond_op[c] == 0) return lhs >= rhs;     /* planted: zero margin counted as true */
#elif ORC_PLANT == 2
    if (b->cond_op[c] == 0) return lhs > rhs;
    return !(lhs > rhs);                          /* planted: '<' as a negated '>' */
#elif ORC_PLANT == 3
    if (b->cond_g[c] >= 0) rhs = b->cond_b[c] * xrow[b->cond_f[c]];   /* planted: wrong feature */
#endif
    if (b->cond_op[c] == 0) return lhs > rhs;
    return lhs < rhs;
}

/* Class predicted by set p for one sample: first rule whose conditions all hold. */
static int32_t predict(const orc_batch *b, int32_t p, const float *xrow)
{
#if ORC_PLANT == 4
    int32_t last = -1;
#endif
    for (int32_t r = b->set_rule_off[p]; r < b->set_rule_off[p + 1]; ++r) {
        int fires = 1;
        for (int32_t c = b->rule_cond_off[r]; c < b->rule_cond_off[r + 1]; ++c) {
            if (!cond_true(b, c, xrow)) { fires = 0; break; }
        }
#if ORC_PLANT == 4
        if (fires) last = b->rule_class[r];      /* planted: last firing rule wins */
#else
        if (fires) return b->rule_class[r];
#endif
    }
#if ORC_PLANT == 4
    if (last >= 0) return last;
#endif
    return b->set_default[p];
}

/*
 * Hard evaluation. X is row-major N x F float32, y int32[N] in 0..K-1.
 * Outputs: correct[P]; per_class[P*K] (optional: #{n : pred = y_n = k}); preds[P*N] (optional).
 */
int orc_eval_hard(const float *X, int64_t N, int32_t F, const int32_t *y, int32_t K,
                  const orc_batch *b, int32_t *correct, int32_t *per_class, int32_t *preds,
                  int nthreads)
{
    (void)F;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t p = 0; p < b->P; ++p) {
        int32_t cnt = 0;
        if (per_class) for (int32_t k = 0; k < K; ++k) per_class[(int64_t)p * K + k] = 0;
        for (int64_t n = 0; n < N; ++n) {
            int32_t pr = predict(b, p, X + n * (int64_t)F);
            if (preds) preds[(int64_t)p * N + n] = pr;
            if (pr == y[n]) {
                ++cnt;
                if (per_class) per_class[(int64_t)p * K + pr] += 1;
            }
        }
        correct[p] = cnt;
    }
    return 0;
}

/* ------------------------------------------------------------------ soft path, float64 */

static double log_sigmoid(double u)          /* log(1 / (1 + exp(-u))) */
{
    if (u >= 0) return -log1p(exp(-u));
    return u - log1p(exp(u));
}

static double log_add(double a, double b)    /* log(exp(a) + exp(b)) */
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double m = a > b ? a : b;
    return m + log1p(exp(-fabs(a - b)));
}

/* Signed scaled margin of condition c: u = s * (a*x[f] - rhs) / tau, s = +1 for '>' else -1. */
static double margin(const orc_batch *b, int64_t c, const float *xrow, double tau)
{
    double lhs = (double)b->cond_a[c] * (double)xrow[b->cond_f[c]];
    double rhs = (b->cond_g[c] < 0) ? (double)b->cond_t[c]
                                    : (double)b->cond_b[c] * (double)xrow[b->cond_g[c]];
    double s = (b->cond_op[c] == 0) ? 1.0 : -1.0;
    return s * (lhs - rhs) / tau;
}

/*
 * log(1 - q_r) of rule r, where s = log q_r. Directly, log(-expm1(s)). When every margin of the
 * rule is so large that s is within 1e-200 of 0 (every u_c above about 460), 1 - q_r no longer
 * follows from s: there 1 - q_r = sum_c softplus(-u_c) = sum_c e^{-u_c} to float64 precision
 * (the first-order term of 1 - prod_c (1 - e^{-u_c})), and its log is the log-sum-exp of the
 * -u_c. Membership tests that hold contribute nothing; a rule of such tests only has q_r = 1.
 */
static double log_one_minus_q(const orc_batch *b, int32_t r, const float *xrow, double tau, double s)
{
    if (s == -INFINITY) return 0.0;
#if ORC_PLANT == 12
    return log(-expm1(s));                       /* planted: 1 - q taken from s alone */
#endif
    if (s < -1e-200) return log(-expm1(s));
    double l = -INFINITY;
    for (int32_t c = b->rule_cond_off[r]; c < b->rule_cond_off[r + 1]; ++c)
        if (b->cond_op[c] != 2) l = log_add(l, -margin(b, c, xrow, tau));
    return l;
}

/*
 * Soft forward (and optionally the adjoint) of every set over all samples, float64.
 *   loss[p]       = (1/N) sum_n -log p_{y_n}(n)
 *   probs[(p*N+n)*K+k] (optional) = p_k(n)
 *   If dloss != NULL: grad_{a,b,t}[c] = dloss[p] * dloss_p/dtheta_c, and (optional) mag_{a,b,t}[c]
 *   = |dloss[p]| * (1/N) sum_n |d ell_n / d theta_c|, the scale against which float32 round-off of
 *   a cancelling sum over samples is measured.
 */
int orc_soft(const float *X, int64_t N, int32_t F, const int32_t *y, int32_t K,
             const orc_batch *b, double tau, double *loss, double *probs,
             const double *dloss, double *grad_a, double *grad_b, double *grad_t,
             double *mag_a, double *mag_b, double *mag_t, int nthreads)
{
    (void)F;
    int32_t Rmax = 0;
    for (int32_t p = 0; p < b->P; ++p) {
        int32_t R = b->set_rule_off[p + 1] - b->set_rule_off[p];
        if (R > Rmax) Rmax = R;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *lq = (double *)malloc(sizeof(double) * (size_t)(Rmax + 1));
        double *l1q = (double *)malloc(sizeof(double) * (size_t)(Rmax + 1));
        double *lu = (double *)malloc(sizeof(double) * (size_t)(Rmax + 2));
        double *lp = (double *)malloc(sizeof(double) * (size_t)K);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int32_t p = 0; p < b->P; ++p) {
            const int32_t r0 = b->set_rule_off[p], R = b->set_rule_off[p + 1] - r0;
            const int32_t c0 = b->rule_cond_off[r0], c1 = b->rule_cond_off[r0 + R];
            double acc = 0.0;
            if (dloss) {
                for (int32_t c = c0; c < c1; ++c) {
                    grad_a[c] = grad_b[c] = grad_t[c] = 0.0;
                    if (mag_a) mag_a[c] = mag_b[c] = mag_t[c] = 0.0;
                }
            }
            for (int64_t n = 0; n < N; ++n) {
                const float *xrow = X + n * (int64_t)F;
                /* forward: log q_r, log(1 - q_r), log of "no earlier rule fired" */
                for (int32_t j = 0; j < R; ++j) {
                    int32_t r = r0 + j;
                    double s = 0.0;
                    for (int32_t c = b->rule_cond_off[r]; c < b->rule_cond_off[r + 1]; ++c)
                        s += (b->cond_op[c] == 2) ? (cond_true(b, c, xrow) ? 0.0 : -INFINITY)
                                                  : log_sigmoid(margin(b, c, xrow, tau));
                    lq[j] = s;
                    l1q[j] = log_one_minus_q(b, r, xrow, tau, s);
                }
                for (int32_t k = 0; k < K; ++k) lp[k] = -INFINITY;
                lu[0] = 0.0;
                for (int32_t j = 0; j < R; ++j) {
                    int32_t k = b->rule_class[r0 + j];
                    lp[k] = log_add(lp[k], lq[j] + lu[j]);
#if ORC_PLANT == 5
                    lu[j + 1] = lu[j];                    /* planted: later rules not discounted */
#else
                    lu[j + 1] = lu[j] + l1q[j];
#endif
                }
                lp[b->set_default[p]] = log_add(lp[b->set_default[p]], lu[R]);
                const int32_t yn = y[n];
                acc += -lp[yn];
                if (probs)
                    for (int32_t k = 0; k < K; ++k) probs[((int64_t)p * N + n) * K + k] = exp(lp[k]);
                if (!dloss) continue;
                /* adjoint. S_j = P(outcome y | evaluation starts at rule j), T_j = 1 - S_j, both
                 * kept as logs of sums of positive terms. d ell / d lq_j = exp(lq_j + lu_j - lp_y)
                 * * (S_{j+1} - [cls_j = y]), written as +exp(.. + lS) or -exp(.. + lT). */
                const double scale = dloss[p] / (double)N;
                const double lpy = lp[yn];
                double lS = (b->set_default[p] == yn) ? 0.0 : -INFINITY;
                double lT = (b->set_default[p] == yn) ? -INFINITY : 0.0;
                for (int32_t j = R - 1; j >= 0; --j) {
                    const int32_t r = r0 + j;
                    const int same = (b->rule_class[r] == yn);
                    /* d ell / d lq_j = sign * exp(lg); kept as its log so that the product with
                     * sigmoid(-u_c) below is formed in the exponent (both factors may lie outside
                     * the float64 range at large margins while the product is moderate) */
                    const double sign = same ? -1.0 : 1.0;
#if ORC_PLANT == 7
                    const double lg = lq[j] + lu[j] + lS - lpy;           /* planted: S for 1-S */
#else
                    const double lg = lq[j] + lu[j] + (same ? lT : lS) - lpy;
#endif
                    lS = log_add(same ? lq[j] : -INFINITY, l1q[j] + lS);
                    lT = log_add(same ? -INFINITY : lq[j], l1q[j] + lT);
                    for (int32_t c = b->rule_cond_off[r]; c < b->rule_cond_off[r + 1]; ++c) {
                        if (b->cond_op[c] == 2) continue;           /* an indicator: no gradient */
                        const double u = margin(b, c, xrow, tau);
                        const double du = sign * exp(lg + log_sigmoid(-u));   /* d ell / d u */
                        const double s = (b->cond_op[c] == 0) ? 1.0 : -1.0;
                        const double da = du * s * (double)xrow[b->cond_f[c]] / tau;
                        grad_a[c] += scale * da;
                        if (mag_a) mag_a[c] += fabs(scale * da);
                        if (b->cond_g[c] < 0) {
#if ORC_PLANT == 6
                            const double dt = du * s / tau;       /* planted: threshold sign */
#else
                            const double dt = -du * s / tau;
#endif
                            grad_t[c] += scale * dt;
                            if (mag_t) mag_t[c] += fabs(scale * dt);
                        } else {
                            const double db = -du * s * (double)xrow[b->cond_g[c]] / tau;
                            grad_b[c] += scale * db;
                            if (mag_b) mag_b[c] += fabs(scale * db);
                        }
                    }
                }
            }
            loss[p] = acc / (double)N;
        }
        free(lq); free(l1q); free(lu); free(lp);
    }
    return 0;
}
