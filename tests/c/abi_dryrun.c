/* Plain-C client of liboc.so: declares the 2-D heat chain (5-point LINCOMB, COPY, MAX
 * reduction, 10 steps on 256^2 with halo 1) in a dry-run context with a 1 MiB budget and
 * a forced tile height of 64, flushes it, and prints the plan's shape and the slow-axis
 * range of every loop in every tile, one line each. Uses only include/oc.h. */
#include <stdio.h>
#include <stdlib.h>

#include "oc.h"

#define CHECK(call)                                                            \
    do {                                                                       \
        int rc_ = (call);                                                      \
        if (rc_ != OC_OK) {                                                    \
            fprintf(stderr, "%s: %d %s\n", #call, rc_, oc_last_error());       \
            return 1;                                                          \
        }                                                                      \
    } while (0)

int main(void)
{
    const int n = 256, steps = 10;
    void* streams[3] = {NULL, NULL, NULL};
    CHECK(oc_init(1u << 20, NULL, 0, streams, OC_FLAG_DRYRUN, OC_PLAN_FIXED));
    int size[3] = {n, n, 1}, hlo[3] = {1, 1, 0}, hhi[3] = {1, 1, 0};
    int u, un;
    CHECK(oc_decl_dat(2, size, hlo, hhi, OC_F64, NULL, 0, &u));
    CHECK(oc_decl_dat(2, size, hlo, hhi, OC_F64, NULL, 0, &un));
    int lo[3] = {0, 0, 0}, hi[3] = {n, n, 1};
    const int five[10] = {0, 0, 1, 0, -1, 0, 0, 1, 0, -1};
    const int zero[2] = {0, 0};
    const double heat[6] = {0.0, 0.6, 0.1, 0.1, 0.1, 0.1};
    const double mode_abs[1] = {1.0};
    for (int s = 0; s < steps; ++s) {
        int red;
        CHECK(oc_decl_reduction(OC_MAX, &red));
        oc_arg a[2] = {{un, OC_WRITE, 1, zero}, {u, OC_READ, 5, five}};
        CHECK(oc_enqueue_loop(OC_K_LINCOMB, lo, hi, 2, a, heat, 6));
        oc_arg c[2] = {{u, OC_WRITE, 1, zero}, {un, OC_READ, 1, zero}};
        CHECK(oc_enqueue_loop(OC_K_COPY, lo, hi, 2, c, NULL, 0));
        oc_arg r[2] = {{u, OC_READ, 1, zero}, {red, OC_REDUCE, 0, NULL}};
        CHECK(oc_enqueue_loop(OC_K_REDUCE, lo, hi, 2, r, mode_abs, 1));
    }
    CHECK(oc_set_tiling(64, 3));
    CHECK(oc_flush());
    int T, L, D, h, depth, rows;
    CHECK(oc_plan_shape(&T, &L, &D, &h, &depth, &rows));
    printf("tiles %d loops %d datasets %d height %d depth %d rows %d\n", T, L, D, h, depth, rows);
    int* se = (int*)malloc(sizeof(int) * 2 * (size_t)T * (size_t)L);
    CHECK(oc_plan_ranges(se));
    for (int t = 0; t < T; ++t)
        for (int i = 0; i < L; ++i)
            printf("range %d %d %d %d\n", t, i, se[(t * L + i) * 2], se[(t * L + i) * 2 + 1]);
    free(se);
    double v;
    if (oc_reduce(0, &v) != OC_ERR_STATE) return 2;   /* a dry run holds no results */
    CHECK(oc_finalize());
    return 0;
}
