/*
 * bitgen — seeded, counter-based Bernoulli bit matrices.
 *
 * This module only makes inputs. It holds none of the arithmetic of the
 * matrix products; both the CPU oracle and the GPU path consume what it
 * produces, and the CPU and GPU implementations below are written
 * independently from the same published definition of SplitMix64
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014; the 64-bit finaliser constants are Stafford's "Mix13").
 *
 * Definition (both implementations follow it word for word):
 *
 *   gamma      = 0x9e3779b97f4a7c15
 *   mix(z)     : z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9
 *                z = (z ^ (z >> 27)) * 0x94d049bb133111eb
 *                return z ^ (z >> 31)
 *   key(seed, id) = (seed << 32) ^ (id << 62)        id: 0 = A, 1 = B, ...
 *   draw(key, c)  = mix(key + (c + 1) * gamma)       (the c-th SplitMix64 output)
 *
 * Matrix layout: rows x cols bits, row-major, cols a multiple of 64, bit j of
 * row i is bit (j % 64) of 64-bit word i*(cols/64) + j/64 (LSB first).
 *
 *   mode BITGEN_DENSE     (p = 1/2): word q = draw(key, q), all 64 bits used.
 *   mode BITGEN_THRESHOLD (p = theta / 2^64): bit e = i*cols + j is 1 iff
 *                          draw(key, e) < theta (unsigned compare).
 */
#ifndef BITGEN_H
#define BITGEN_H
#include <stdint.h>

#define BITGEN_DENSE 0
#define BITGEN_THRESHOLD 1
#define BITGEN_GAMMA 0x9e3779b97f4a7c15ULL

#ifdef __cplusplus
extern "C" {
#endif

/* CPU: fill rows [row0, row0 + nrows) of a rows x cols matrix into out
 * (nrows * cols/64 words). Uses nthreads POSIX threads (<= 0: one). */
void bitgen_fill_rows(uint64_t *out, int64_t cols, int64_t row0, int64_t nrows,
                      uint64_t seed, int matrix_id, int mode, uint64_t theta,
                      int nthreads);

/* CPU: one draw, for tests of the definition itself. */
uint64_t bitgen_draw(uint64_t seed, int matrix_id, uint64_t counter);

/* GPU (libbitgen_cuda.so): same contract on device memory, asynchronous on
 * `stream` (a cudaStream_t, 0 = legacy default). Returns a cudaError_t. */
int bitgen_fill_rows_device(uint64_t *out, int64_t cols, int64_t row0, int64_t nrows,
                            uint64_t seed, int matrix_id, int mode, uint64_t theta,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif
