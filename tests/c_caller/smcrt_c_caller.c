/*
 * A plain C caller of the library's C-ABI (include/smcrt.h): the pencil-beam
 * sphere (radius 1 cm, mu_a 1, mu_s 10 /cm, g 0.9, n 1.38 in air; 50^3 grid
 * over the 2 cm cube) run through smcrt_run in FP64 and in mixed precision,
 * and once through the serving calls (smcrt_submit / smcrt_wait).  Prints
 * each run's integer tallies and a checksum of its fluence map, one line per
 * run, for the test that compares them with the same runs made through the
 * Python binding.  Usage: smcrt_c_caller <packets> <stepping 0|1>.
 */
#include <stdio.h>
#include <stdlib.h>

#include "smcrt.h"

static void print_run(const char *name, const smcrt_totals *t, const int64_t *flu, size_t cells)
{
    /* order-independent checksum of the map: sum and sum of index * value */
    long long s0 = 0, s1 = 0;
    for (size_t i = 0; i < cells; ++i) {
        s0 += (long long)flu[i];
        s1 += (long long)((unsigned long long)flu[i] * (unsigned long long)(i + 1));
    }
    printf("%s %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld\n", name, (long long)t->R, (long long)t->T,
           (long long)t->A, (long long)t->killed, (long long)t->gain, (long long)t->packets,
           (long long)t->scatters, (long long)t->steps, s0, s1);
}

int main(int argc, char **argv)
{
    const uint64_t n = argc > 1 ? strtoull(argv[1], NULL, 10) : 100000;
    const int stepping = argc > 2 ? atoi(argv[2]) : SMCRT_STEP_SEGMENT;
    smcrt_prim sphere = {SMCRT_SPHERE, 0, {0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0}};
    smcrt_csg_node program = {SMCRT_OP_PRIM, 0, 0.0};
    smcrt_region tissue = {0, 1, 1.0, 10.0, 0.9, 1.38};
    smcrt_scene scene = {&sphere, 1, &program, 1, &tissue, 1, 1.0,
                         {-1.25, -1.25, -1.25}, {1.25, 1.25, 1.25},
                         1e-6, 100000, stepping, 0, NULL, 0, 0};
    smcrt_source beam = {SMCRT_SRC_PENCIL, 0, {0.0, 0.0, 1.2}, {0.0, 0.0, -1.0}, 0.0};
    smcrt_grid grid = {{-1.0, -1.0, -1.0}, {1.0, 1.0, 1.0}, {50, 50, 50}, 0};
    const size_t cells = (size_t)50 * 50 * 50;
    int64_t *flu = calloc(cells, sizeof(int64_t));
    smcrt_totals t;
    smcrt_ctx *ctx = NULL;
    int rc = flu ? smcrt_create(&ctx, 0, 0) : SMCRT_ERR_NO_MEMORY;
    if (rc == SMCRT_OK) rc = smcrt_run(ctx, &scene, &beam, &grid, n, 1, SMCRT_FP64, flu, &t);
    if (rc == SMCRT_OK) print_run("run_fp64", &t, flu, cells);
    if (rc == SMCRT_OK) rc = smcrt_run(ctx, &scene, &beam, &grid, n, 1, SMCRT_MIXED, flu, &t);
    if (rc == SMCRT_OK) print_run("run_mixed", &t, flu, cells);
    if (rc == SMCRT_OK) {
        uint64_t job = 0;
        double latency = 0.0;
        rc = smcrt_submit(ctx, &scene, &beam, &grid, n, 1, SMCRT_MIXED, &job);
        if (rc == SMCRT_OK) rc = smcrt_wait(ctx, job, -1.0, flu, &t, &latency);
        if (rc == SMCRT_OK) print_run("served_mixed", &t, flu, cells);
    }
    if (rc != SMCRT_OK) fprintf(stderr, "smcrt: %s (%d)\n", smcrt_strerror(rc), rc);
    if (ctx) smcrt_destroy(ctx);
    free(flu);
    return rc != SMCRT_OK;
}
