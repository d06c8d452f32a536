/*
 * A C program that uses the library only through its C ABI (include/rs.h, librs.so): it reads a
 * dataset and a population from a binary file, registers the dataset from host memory, evaluates
 * every rule set with rs_eval_hard from host arrays (host outputs: the library copies), prints
 * the correct and per-class counts, then times repeated synchronous calls. The tests compile and
 * link it on any host (the header and the library must agree) and run it on a GPU against the
 * oracle.
 *
 * Input (little-endian): int64 N; int32 F, K, P, R, C; float32 X[N*F] (row-major);
 * int32 y[N]; int32 set_rule_off[P+1], rule_cond_off[R+1], rule_class[R], set_default[P],
 * cond_f[C], cond_g[C]; int8 cond_op[C]; float32 cond_a[C], cond_b[C], cond_t[C].
 * Output: "correct c_0 ... c_{P-1}", "per_class" followed by P*K counts, "us_per_call u"; on a
 * failure "error <status> <message>" and exit status 1.
 *
 *   abi_consumer <input file> [timed calls]
 */
#define _POSIX_C_SOURCE 199309L           /* clock_gettime under -std=c99 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <time.h>

#include "rs.h"

static int read_all(FILE *f, void *dst, size_t bytes)
{
    return fread(dst, 1, bytes, f) == bytes;
}

static void *take(FILE *f, size_t bytes)
{
    void *p = malloc(bytes ? bytes : 1);
    if (!p || !read_all(f, p, bytes)) {
        free(p);
        return NULL;
    }
    return p;
}

static int fail(rs_status rc)
{
    printf("error %d %s\n", (int)rc, rs_last_error());
    return 1;
}

int main(int argc, char **argv)
{
    if (argc < 2) {
        fprintf(stderr, "usage: %s <input file> [timed calls]\n", argv[0]);
        return 2;
    }
    const int calls = argc > 2 ? atoi(argv[2]) : 200;
    FILE *f = fopen(argv[1], "rb");
    if (!f) {
        fprintf(stderr, "cannot open %s\n", argv[1]);
        return 2;
    }
    int64_t N = 0;
    int32_t dims[5];                       /* F, K, P, R, C */
    if (!read_all(f, &N, sizeof N) || !read_all(f, dims, sizeof dims)) {
        fprintf(stderr, "short input\n");
        return 2;
    }
    const int32_t F = dims[0], K = dims[1], P = dims[2], R = dims[3], C = dims[4];
    float *X = take(f, sizeof(float) * (size_t)N * F);
    int32_t *y = take(f, sizeof(int32_t) * (size_t)N);
    int32_t *sro = take(f, sizeof(int32_t) * ((size_t)P + 1));
    int32_t *rco = take(f, sizeof(int32_t) * ((size_t)R + 1));
    int32_t *rcls = take(f, sizeof(int32_t) * (size_t)R);
    int32_t *sdef = take(f, sizeof(int32_t) * (size_t)P);
    int32_t *cf = take(f, sizeof(int32_t) * (size_t)C);
    int32_t *cg = take(f, sizeof(int32_t) * (size_t)C);
    int8_t *cop = take(f, sizeof(int8_t) * (size_t)C);
    float *ca = take(f, sizeof(float) * (size_t)C);
    float *cb = take(f, sizeof(float) * (size_t)C);
    float *ct = take(f, sizeof(float) * (size_t)C);
    fclose(f);
    if (!X || !y || !sro || !rco || !rcls || !sdef || !cf || !cg || !cop || !ca || !cb || !ct) {
        fprintf(stderr, "short input\n");
        return 2;
    }

    rs_ctx *ctx = NULL;
    rs_status rc = rs_create(NULL, &ctx);
    if (rc != RS_OK) return fail(rc);
    uint64_t ds = 0;
    rc = rs_dataset_create(ctx, X, y, N, F, K, RS_MEM_HOST, NULL, &ds);
    if (rc != RS_OK) return fail(rc);

    rs_batch b = {0};                       /* cond_set stays NULL: no membership conditions */
    b.P = P;
    b.R = R;
    b.C = C;
    b.mem = RS_MEM_HOST;
    b.set_rule_off = sro;
    b.rule_cond_off = rco;
    b.rule_class = rcls;
    b.set_default = sdef;
    b.cond_f = cf;
    b.cond_g = cg;
    b.cond_op = cop;
    b.cond_a = ca;
    b.cond_b = cb;
    b.cond_t = ct;

    int32_t *correct = malloc(sizeof(int32_t) * (size_t)(P ? P : 1));
    int32_t *per_class = malloc(sizeof(int32_t) * (size_t)(P ? P : 1) * (size_t)K);
    if (!correct || !per_class) return 2;
    rc = rs_eval_hard(ctx, ds, &b, correct, per_class, NULL, NULL);
    if (rc != RS_OK) return fail(rc);
    printf("correct");
    for (int32_t p = 0; p < P; ++p) printf(" %d", (int)correct[p]);
    printf("\nper_class");
    for (int64_t i = 0; i < (int64_t)P * K; ++i) printf(" %d", (int)per_class[i]);
    printf("\n");

    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    for (int i = 0; i < calls; ++i) {
        rc = rs_eval_hard(ctx, ds, &b, correct, per_class, NULL, NULL);
        if (rc != RS_OK) return fail(rc);
    }
    clock_gettime(CLOCK_MONOTONIC, &t1);
    const double us = ((double)(t1.tv_sec - t0.tv_sec) * 1e9 + (double)(t1.tv_nsec - t0.tv_nsec)) / 1e3;
    printf("us_per_call %.3f\n", calls > 0 ? us / calls : 0.0);

    rc = rs_dataset_destroy(ctx, ds);
    if (rc != RS_OK) return fail(rc);
    rc = rs_destroy(ctx);
    if (rc != RS_OK) return fail(rc);
    free(X); free(y); free(sro); free(rco); free(rcls); free(sdef);
    free(cf); free(cg); free(cop); free(ca); free(cb); free(ct);
    free(correct); free(per_class);
    return 0;
}
