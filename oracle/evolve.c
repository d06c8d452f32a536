/*
 * Plain CPU oracle of one generation of rule-set evolution (test infrastructure).
 *
 * The paper (Sec. 3) evolves rule sets by tournament selection and offspring generation with
 * randomized coefficients; fitness is classification accuracy (Sec. 1). It gives no further
 * detail, so the operators below are this library's reading, written out step by step:
 *
 *   1. rank by (correct count descending, index ascending); the top E individuals are copied
 *      unchanged (elitism);
 *   2. every other child: parents A and B, each the better of two uniformly drawn individuals
 *      (binary tournament); the child starts as a copy of A; with probability 1/2 each rule
 *      position j that B also has takes B's rule with probability 1/2 (uniform rule-list
 *      crossover);
 *   3. with probability 9/10 one mutation, chosen uniformly among: new random coefficients of a
 *      condition (offspring with coefficients drawn at random, Sec. 3), a new feature for a condition, flipped
 *      comparison, add a condition, delete a condition, add a random rule, delete a rule, new class
 *      of a rule. A threshold is drawn as t = fl32(a * x[n][f]) for a uniformly drawn sample n
 *      (an empirical quantile of feature f); a new condition is a feature pair with probability
 *      1/5; coefficients are uniform in [-1, 1).
 *
 * Random numbers come from Philox4x64-10 (Salmon et al., "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11), counter (i/4, child, generation, 0), key (seed, 0x65766f6c); draw i of a child
 * is word i%4 of that block. The CUDA path implements the same generator from the same
 * definition; nothing else is shared.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ORC_PLANT selects a deliberately wrong variant, built only by the test that checks that the
 * pins catch it (0 = the oracle as stated). */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

typedef struct {
    int32_t P, RMAX, CMAX;
    int32_t *nrule;    /* [P] */
    int32_t *deflt;    /* [P] */
    int32_t *rcls;     /* [P*RMAX] */
    int32_t *ncond;    /* [P*RMAX] */
    int32_t *cf, *cg;  /* [P*RMAX*CMAX] */
    int8_t *cop;
    float *ca, *cb, *ct;
} orc_pop;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0, p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

typedef struct { uint64_t seed, gen, child, i; } rng_t;

static uint64_t next64(rng_t *r)
{
    uint64_t ctr[4] = {r->i >> 2, r->child, r->gen, 0}, key[2] = {r->seed, 0x65766f6cull}, out[4];
    orc_philox4x64_10(ctr, key, out);
    return out[(r->i++) & 3];
}

static int32_t uniform_int(rng_t *r, int32_t n)      /* 0 .. n-1 */
{
    return (int32_t)(((next64(r) >> 32) * (uint64_t)(uint32_t)n) >> 32);
}

static float uniform01(rng_t *r)                     /* k * 2^-24, k in 0 .. 2^24-1 (exact) */
{
    return (float)(next64(r) >> 40) * (1.0f / 16777216.0f);
}

static float coef(rng_t *r)                          /* uniform in [-1, 1), exact */
{
    float u = uniform01(r);
    return u * 2.0f - 1.0f;
}

typedef struct {
    const float *X;    /* row-major N x F, caller order */
    int64_t N;
    int32_t F, K;
} orc_data;

static float data_draw(rng_t *r, const orc_data *d, int32_t f)
{
    int64_t n = (int64_t)(((next64(r) >> 32) * (uint64_t)d->N) >> 32);
#if ORC_PLANT == 11
    f = (f + 1) % d->F;                      /* planted: threshold drawn from the wrong feature */
#endif
    return d->X[n * d->F + f];
}

typedef struct { int32_t f, g; int8_t op; float a, b, t; } cond_t;

static void random_condition(rng_t *r, const orc_data *d, cond_t *c)
{
    int pair = (uniform01(r) < 0.2f) && d->F > 1;
    c->f = uniform_int(r, d->F);
    c->g = -1;
    if (pair) {
        c->g = uniform_int(r, d->F - 1);
        if (c->g >= c->f) c->g += 1;
    }
    c->op = (int8_t)(next64(r) & 1);
    c->a = coef(r);
    c->b = pair ? coef(r) : 0.0f;
    c->t = pair ? 0.0f : c->a * data_draw(r, d, c->f);
}

/* ---------------------------------------------------------------- individual helpers */

typedef struct {
    int32_t nrule, deflt;
    int32_t rcls[64];
    int32_t ncond[64];
    cond_t c[64][16];
} indiv_t;                 /* RMAX <= 64, CMAX <= 16 */

static void load(const orc_pop *p, int32_t i, indiv_t *v)
{
    v->nrule = p->nrule[i];
    v->deflt = p->deflt[i];
    for (int32_t j = 0; j < p->RMAX; ++j) {
        int64_t rj = (int64_t)i * p->RMAX + j;
        v->rcls[j] = p->rcls[rj];
        v->ncond[j] = p->ncond[rj];
        for (int32_t k = 0; k < p->CMAX; ++k) {
            int64_t q = rj * p->CMAX + k;
            cond_t *c = &v->c[j][k];
            c->f = p->cf[q]; c->g = p->cg[q]; c->op = p->cop[q];
            c->a = p->ca[q]; c->b = p->cb[q]; c->t = p->ct[q];
        }
    }
}

static void store(orc_pop *p, int32_t i, const indiv_t *v)
{
    p->nrule[i] = v->nrule;
    p->deflt[i] = v->deflt;
    for (int32_t j = 0; j < p->RMAX; ++j) {
        int64_t rj = (int64_t)i * p->RMAX + j;
        p->rcls[rj] = v->rcls[j];
        p->ncond[rj] = v->ncond[j];
        for (int32_t k = 0; k < p->CMAX; ++k) {
            int64_t q = rj * p->CMAX + k;
            const cond_t *c = &v->c[j][k];
            p->cf[q] = c->f; p->cg[q] = c->g; p->cop[q] = c->op;
            p->ca[q] = c->a; p->cb[q] = c->b; p->ct[q] = c->t;
        }
    }
}

static int better(const int32_t *fit, int32_t i, int32_t j)   /* is i ranked before j */
{
    return fit[i] > fit[j] || (fit[i] == fit[j] && i < j);
}

static int32_t tournament(rng_t *r, const int32_t *fit, int32_t P)
{
    int32_t i = uniform_int(r, P), j = uniform_int(r, P);
    return better(fit, i, j) ? i : j;
}

static void mutate(rng_t *r, indiv_t *v, const orc_data *d, int32_t RMAX, int32_t CMAX)
{
    int32_t type = uniform_int(r, 8);
    int32_t j, k;
#if ORC_PLANT == 10
    if (type == 3) type = 4;                 /* planted: add-condition never chosen */
#endif
    cond_t *c;
    switch (type) {
    case 0:                                  /* randomized coefficients */
        j = uniform_int(r, v->nrule); k = uniform_int(r, v->ncond[j]); c = &v->c[j][k];
        c->a = coef(r);
        if (c->g >= 0) c->b = coef(r);
        else c->t = c->a * data_draw(r, d, c->f);
        break;
    case 1:                                  /* new feature */
        j = uniform_int(r, v->nrule); k = uniform_int(r, v->ncond[j]); c = &v->c[j][k];
        c->f = uniform_int(r, d->F);
        if (c->g >= 0) {
            c->g = uniform_int(r, d->F - 1);
            if (c->g >= c->f) c->g += 1;
        } else {
            c->t = c->a * data_draw(r, d, c->f);
        }
        break;
    case 2:                                  /* flipped comparison */
        j = uniform_int(r, v->nrule); k = uniform_int(r, v->ncond[j]);
        v->c[j][k].op ^= 1;
        break;
    case 3:                                  /* add a condition */
        j = uniform_int(r, v->nrule);
        if (v->ncond[j] < CMAX) {
            random_condition(r, d, &v->c[j][v->ncond[j]]);
            v->ncond[j] += 1;
        }
        break;
    case 4:                                  /* delete a condition */
        j = uniform_int(r, v->nrule);
        if (v->ncond[j] > 1) {
            k = uniform_int(r, v->ncond[j]);
            for (int32_t q = k; q + 1 < v->ncond[j]; ++q) v->c[j][q] = v->c[j][q + 1];
            v->ncond[j] -= 1;
        }
        break;
    case 5:                                  /* add a random rule */
        if (v->nrule < RMAX) {
            int32_t pos = uniform_int(r, v->nrule + 1);
            int32_t n = 1 + uniform_int(r, 3);
            if (n > CMAX) n = CMAX;
            for (int32_t q = v->nrule; q > pos; --q) {
                v->rcls[q] = v->rcls[q - 1];
                v->ncond[q] = v->ncond[q - 1];
                memcpy(v->c[q], v->c[q - 1], sizeof(v->c[q]));
            }
            v->ncond[pos] = n;
            for (int32_t q = 0; q < n; ++q) random_condition(r, d, &v->c[pos][q]);
            v->rcls[pos] = uniform_int(r, d->K);
            v->nrule += 1;
        }
        break;
    case 6:                                  /* delete a rule */
        if (v->nrule > 1) {
            j = uniform_int(r, v->nrule);
            for (int32_t q = j; q + 1 < v->nrule; ++q) {
                v->rcls[q] = v->rcls[q + 1];
                v->ncond[q] = v->ncond[q + 1];
                memcpy(v->c[q], v->c[q + 1], sizeof(v->c[q]));
            }
            v->nrule -= 1;
        }
        break;
    default:                                 /* new class of a rule */
        j = uniform_int(r, v->nrule);
        v->rcls[j] = uniform_int(r, d->K);
        break;
    }
}

/*
 * One generation: `in` with fitness `fit` -> `out` (same shape). Slots beyond nrule / ncond are
 * carried along unchanged from the copied parent (they are never read).
 * Returns 0, or -1 if RMAX > 64 or CMAX > 16.
 */
int orc_evolve_step(const orc_pop *in, const int32_t *fit, orc_pop *out, uint64_t seed,
                    uint64_t gen, int32_t elite, const float *X, int64_t N, int32_t F, int32_t K)
{
    if (in->RMAX > 64 || in->CMAX > 16) return -1;
    const int32_t P = in->P;
    orc_data d = {X, N, F, K};
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
    indiv_t *v = (indiv_t *)malloc(sizeof(indiv_t));
    indiv_t *w = (indiv_t *)malloc(sizeof(indiv_t));
    /* rank: position of i = number of individuals ranked before it */
    for (int32_t i = 0; i < P; ++i) {
        int32_t pos = 0;
        for (int32_t j = 0; j < P; ++j) pos += better(fit, j, i);
        order[pos] = i;
    }
    for (int32_t c = 0; c < P; ++c) {
        if (c < elite) {
            load(in, order[c], v);
            store(out, c, v);
            continue;
        }
        rng_t r = {seed, gen, (uint64_t)c, 0};
        int32_t A = tournament(&r, fit, P), B = tournament(&r, fit, P);
        load(in, A, v);
        if (uniform01(&r) < 0.5f) {
            load(in, B, w);
            for (int32_t j = 0; j < v->nrule; ++j) {
                if (j < w->nrule && (next64(&r) & 1)) {
                    v->rcls[j] = w->rcls[j];
                    v->ncond[j] = w->ncond[j];
                    memcpy(v->c[j], w->c[j], sizeof(v->c[j]));
                }
            }
        }
        if (uniform01(&r) < 0.9f) mutate(&r, v, &d, in->RMAX, in->CMAX);
        store(out, c, v);
    }
    free(order);
    free(v);
    free(w);
    return 0;
}
