/* CPU implementation of the bitgen definition in bitgen.h. */
#include "bitgen.h"
#include <pthread.h>
#include <stdlib.h>

static uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t key_of(uint64_t seed, int matrix_id) {
    return (seed << 32) ^ ((uint64_t)matrix_id << 62);
}

uint64_t bitgen_draw(uint64_t seed, int matrix_id, uint64_t counter) {
    return mix(key_of(seed, matrix_id) + (counter + 1) * BITGEN_GAMMA);
}

typedef struct {
    uint64_t *out;
    int64_t cols, row_lo, row_hi, out_row0;
    uint64_t key, theta;
    int mode;
} fill_job;

static void *fill_worker(void *p) {
    fill_job *j = (fill_job *)p;
    int64_t wpr = j->cols / 64;
    for (int64_t i = j->row_lo; i < j->row_hi; i++) {
        uint64_t *row = j->out + (i - j->out_row0) * wpr;
        for (int64_t w = 0; w < wpr; w++) {
            uint64_t word = 0;
            if (j->mode == BITGEN_DENSE) {
                uint64_t q = (uint64_t)(i * wpr + w);
                word = mix(j->key + (q + 1) * BITGEN_GAMMA);
            } else {
                for (int b = 0; b < 64; b++) {
                    uint64_t e = (uint64_t)(i * j->cols + w * 64 + b);
                    if (mix(j->key + (e + 1) * BITGEN_GAMMA) < j->theta) word |= 1ULL << b;
                }
            }
            row[w] = word;
        }
    }
    return NULL;
}

void bitgen_fill_rows(uint64_t *out, int64_t cols, int64_t row0, int64_t nrows,
                      uint64_t seed, int matrix_id, int mode, uint64_t theta,
                      int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrows) nthreads = (int)(nrows > 0 ? nrows : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    fill_job *jobs = (fill_job *)malloc(sizeof(fill_job) * nthreads);
    uint64_t key = key_of(seed, matrix_id);
    for (int t = 0; t < nthreads; t++) {
        jobs[t].out = out;
        jobs[t].cols = cols;
        jobs[t].row_lo = row0 + nrows * t / nthreads;
        jobs[t].row_hi = row0 + nrows * (t + 1) / nthreads;
        jobs[t].out_row0 = row0;
        jobs[t].key = key;
        jobs[t].theta = theta;
        jobs[t].mode = mode;
        pthread_create(&th[t], NULL, fill_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}
