/* A plain C caller of libsdm (no CUDA headers, no Python): one cell of super-droplets read from a
 * binary file, stepped through the C ABI of include/sdm.h, the result written back.
 *
 *   capi_example IN OUT STEPS [KERNEL]
 *
 * IN holds, little-endian: n (u64), xi[n] (u64), v[n] (f64), dv (f64), golovin_b (f64), dt (f64),
 * seed (u64).  OUT receives n (u64), xi[n], v[n] after STEPS coalescence steps (FP64 decisions,
 * PRP shuffle contract), then the summed step statistics n_pairs, n_collisions, n_removed (u64).
 * KERNEL is the sdm_kernel_id of the cell (default 0, Golovin).  Exit status 0 on success; any
 * error is printed with sdm_status_str and returns 1. */
#include <stdio.h>
#include <stdlib.h>

#include "sdm.h"

static int check(sdm_status s, const char* where)
{
    if (s != SDM_OK) {
        fprintf(stderr, "%s: %s\n", where, sdm_status_str(s));
        return 1;
    }
    return 0;
}

int main(int argc, char** argv)
{
    if (argc < 4) {
        fprintf(stderr, "usage: %s IN OUT STEPS [KERNEL]\n", argv[0]);
        return 1;
    }
    const uint32_t steps = (uint32_t)strtoul(argv[3], NULL, 10);
    const uint8_t kernel = argc > 4 ? (uint8_t)strtoul(argv[4], NULL, 10) : 0u;
    FILE* f = fopen(argv[1], "rb");
    if (!f) { perror(argv[1]); return 1; }
    uint64_t n = 0;
    if (fread(&n, sizeof n, 1, f) != 1 || n == 0) { fprintf(stderr, "bad input\n"); fclose(f); return 1; }
    uint64_t* xi = malloc(sizeof(uint64_t) * n);
    double* v = malloc(sizeof(double) * n);
    uint32_t* cell = calloc(n, sizeof(uint32_t));        /* every SD in cell 0 */
    double dv = 0, b = 0, dt = 0;
    uint64_t seed = 0;
    int bad = !xi || !v || !cell;
    bad = bad || fread(xi, sizeof(uint64_t), n, f) != n || fread(v, sizeof(double), n, f) != n;
    bad = bad || fread(&dv, sizeof dv, 1, f) != 1 || fread(&b, sizeof b, 1, f) != 1;
    bad = bad || fread(&dt, sizeof dt, 1, f) != 1 || fread(&seed, sizeof seed, 1, f) != 1;
    fclose(f);
    if (bad) { fprintf(stderr, "bad input\n"); return 1; }

    sdm_state* st = NULL;
    if (check(sdm_alloc(&st, n, 1, 1, NULL, NULL, 0), "sdm_alloc")) return 1;
    int err = check(sdm_init_state(st, xi, v, cell, n, &dv, &kernel, 0), "sdm_init_state");
    sdm_step_params p = {0};
    p.dt = dt;
    p.golovin_b = b;
    p.seed = seed;
    p.step = 0;
    p.precision = SDM_PREC_FP64;
    p.shuffle = SDM_SHUFFLE_PRP;
    sdm_step_stats stats = {0};
    if (!err) err = check(sdm_coalescence_step(st, &p, steps, &stats), "sdm_coalescence_step");
    if (!err) err = check(sdm_get_state(st, xi, v, NULL, NULL, 0), "sdm_get_state");
    if (!err) err = check(sdm_sync(st), "sdm_sync");
    sdm_free(st);
    if (!err) {
        FILE* o = fopen(argv[2], "wb");
        if (!o) { perror(argv[2]); return 1; }
        const uint64_t tail[3] = {stats.n_pairs, stats.n_collisions, stats.n_removed};
        err = fwrite(&n, sizeof n, 1, o) != 1 || fwrite(xi, sizeof(uint64_t), n, o) != n ||
              fwrite(v, sizeof(double), n, o) != n || fwrite(tail, sizeof(uint64_t), 3, o) != 3;
        fclose(o);
    }
    free(xi);
    free(v);
    free(cell);
    return err ? 1 : 0;
}
