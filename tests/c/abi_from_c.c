/*
 * A plain C99 caller of the library, for the CPU test suite: it includes
 * kifmm.h as a C compiler sees it, links libkifmm.so, builds a host-only
 * plan (no GPU needed) and checks the answers the ABI documents.  Exit
 * status 0 on success; otherwise the first failed check is printed.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "kifmm.h"

#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            fprintf(stderr, "check failed: %s (line %d): %s\n", #cond, \
                    __LINE__, fmm_last_error());                      \
            return 1;                                                 \
        }                                                             \
    } while (0)

int main(void) {
    enum { G = 12, N = G * G * G };
    static double x[N * 3];
    int64_t i, v;
    fmm_options o;
    fmm_plan_t plan = NULL;
    double surf[3 * 56];
    int64_t need = 0;
    float q[N];
    double phi[N];

    /* a 12 x 12 x 12 grid in the unit cube */
    for (i = 0; i < N; ++i) {
        x[3 * i + 0] = (double)(i % G) / G;
        x[3 * i + 1] = (double)((i / G) % G) / G;
        x[3 * i + 2] = (double)(i / (G * G)) / G;
        q[i] = 1.0f;
    }
    fmm_options_init(&o);
    CHECK(o.alpha_inner == 1.05 && o.alpha_outer == 2.95 && o.balance == 1);
    o.host_only = 1;
    CHECK(fmm_plan_create_ex(x, NULL, N, 4, 32, &o, &plan) == FMM_OK && plan != NULL);

    CHECK(fmm_plan_info(plan, FMM_INFO_N, &v) == FMM_OK && v == N);
    CHECK(fmm_plan_info(plan, FMM_INFO_NSURF, &v) == FMM_OK && v == 6 * 3 * 3 + 2);
    CHECK(fmm_plan_info(plan, FMM_INFO_DEPTH, &v) == FMM_OK && v == 2);
    CHECK(fmm_plan_info(plan, FMM_INFO_LEAVES, &v) == FMM_OK && v == 64);
    CHECK(fmm_plan_info(plan, FMM_INFO_NODES, &v) == FMM_OK && v == 1 + 8 + 64);
    CHECK(fmm_plan_info(plan, 999, &v) == FMM_ERR_INVALID_ARG);

    /* the size query, then the copy, of the unit surface */
    CHECK(fmm_plan_get_array(plan, FMM_ARRAY_SURFACE, NULL, 0, &need) == FMM_OK);
    CHECK(need == (int64_t)sizeof surf);
    CHECK(fmm_plan_get_array(plan, FMM_ARRAY_SURFACE, surf, 8, NULL) == FMM_ERR_INVALID_ARG);
    CHECK(fmm_plan_get_array(plan, FMM_ARRAY_SURFACE, surf, need, NULL) == FMM_OK);
    for (i = 0; i < 56; ++i) {
        double m = 0;
        int d;
        for (d = 0; d < 3; ++d) {
            double a = surf[3 * i + d] < 0 ? -surf[3 * i + d] : surf[3 * i + d];
            if (a > m) m = a;
        }
        CHECK(m == 1.0); /* every surface point lies on the cube's boundary */
    }

    /* a host-only plan refuses to evaluate, with a message */
    CHECK(fmm_evaluate(plan, q, 1, phi, NULL) == FMM_ERR_INVALID_ARG);
    CHECK(strlen(fmm_last_error()) > 0);
    CHECK(fmm_plan_set_option(plan, FMM_OPT_M2L_MODE, 7.0) == FMM_ERR_INVALID_ARG);
    CHECK(fmm_set_operator_cache(NULL) == FMM_OK);

    /* invalid creation arguments come back as statuses */
    plan = (fmm_destroy(plan), NULL);
    CHECK(fmm_plan_create_ex(x, NULL, 0, 4, 32, &o, &plan) == FMM_ERR_INVALID_ARG);
    CHECK(plan == NULL);
    CHECK(fmm_plan_create_ex(x, NULL, N, 1, 32, &o, &plan) == FMM_ERR_INVALID_ARG);
    fmm_destroy(NULL);
    puts("ok");
    return 0;
}
