// GPU implementation of the bitgen definition in bitgen.h (written separately
// from bitgen.c; tests check the two bit for bit).
#include <cuda_runtime.h>
#include <stdint.h>
#include "bitgen.h"

namespace {

__device__ __forceinline__ uint64_t sm64_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// One thread per 64-bit output word; grid-stride over the requested rows.
__global__ void fill_kernel(uint64_t* __restrict__ out, int64_t cols, int64_t row0,
                            int64_t nrows, uint64_t key, int mode, uint64_t theta) {
    const int64_t wpr = cols / 64;
    const int64_t total = nrows * wpr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / wpr, w = t - r * wpr;
        const int64_t i = row0 + r;
        uint64_t word = 0;
        if (mode == BITGEN_DENSE) {
            const uint64_t q = (uint64_t)(i * wpr + w);
            word = sm64_finalise(key + (q + 1) * BITGEN_GAMMA);
        } else {
            const uint64_t e0 = (uint64_t)(i * cols + w * 64);
#pragma unroll 8
            for (int b = 0; b < 64; b++) {
                const uint64_t v = sm64_finalise(key + (e0 + b + 1) * BITGEN_GAMMA);
                word |= (uint64_t)(v < theta) << b;
            }
        }
        out[t] = word;
    }
}

}  // namespace

extern "C" int bitgen_fill_rows_device(uint64_t* out, int64_t cols, int64_t row0,
                                       int64_t nrows, uint64_t seed, int matrix_id, int mode,
                                       uint64_t theta, void* stream) {
    if (cols <= 0 || cols % 64 != 0 || nrows < 0 || row0 < 0) return (int)cudaErrorInvalidValue;
    if (nrows == 0) return 0;
    const uint64_t key = (seed << 32) ^ ((uint64_t)matrix_id << 62);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t total = nrows * (cols / 64);
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
    if (blocks > cap) blocks = cap;
    fill_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(out, cols, row0, nrows, key,
                                                                   mode, theta);
    return (int)cudaGetLastError();
}
