// Bit-matrix transpose (Sec. 3.5: the paper transposes the right operand so
// that both operands of the inner product run along k; it does this on the
// host with recursive 64x64 word transposes). Here: on the GPU, one warp per
// 64x64 bit block, the recursive block swap done with warp shuffles.
//
// HBM-bound: reads rows*cols/8 bytes and writes the same. A CTA moves a tile
// of 256 rows x 256 columns (16 blocks) through shared memory so that both
// the loads and the stores touch 32 contiguous bytes per row.
#include "internal.h"

namespace bmm {
namespace {

constexpr int TILE_R = 256;       // input rows per CTA
constexpr int TILE_W = 4;         // input words (64 columns each) per CTA
constexpr int PADW = TILE_W + 1;  // padded shared row (conflict-free 8-byte accesses)

__device__ __forceinline__ uint64_t swap_step(uint64_t v, int lane, int j, uint64_t mask) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, v, j);
    if ((lane & j) == 0) {
        const uint64_t t = ((v >> j) ^ other) & mask;
        return v ^ (t << j);
    }
    const uint64_t t = ((other >> j) ^ v) & mask;
    return v ^ t;
}

__global__ void __launch_bounds__(256) transpose_kernel(const uint64_t* __restrict__ X,
                                                        int64_t pitch, uint64_t* __restrict__ Xt,
                                                        int64_t tpitch, int64_t rows,
                                                        int64_t cols) {
    __shared__ uint64_t tin[TILE_R][PADW];
    __shared__ uint64_t tout[TILE_W * 64][PADW];
    const int t = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * TILE_R;
    const int64_t w0 = (int64_t)blockIdx.x * TILE_W;  // first input word (column / 64)
    const int64_t xw = cols / 64, tw = rows / 64;

    {
        const int64_t r = r0 + t;
#pragma unroll
        for (int q = 0; q < TILE_W; q++)
            tin[t][q] = (r < rows && w0 + q < xw) ? X[r * pitch + w0 + q] : 0ull;
    }
    __syncthreads();

    const int warp = t >> 5, lane = t & 31;
    for (int b = warp; b < (TILE_R / 64) * TILE_W; b += 8) {
        const int rb = b / TILE_W, cb = b % TILE_W;
        uint64_t lo = tin[rb * 64 + lane][cb];
        uint64_t hi = tin[rb * 64 + lane + 32][cb];
        {  // swap the off-diagonal 32x32 blocks (rows lane and lane+32 live in one thread)
            const uint64_t tt = ((lo >> 32) ^ hi) & 0x00000000FFFFFFFFull;
            hi ^= tt;
            lo ^= tt << 32;
        }
        lo = swap_step(lo, lane, 16, 0x0000FFFF0000FFFFull);
        hi = swap_step(hi, lane, 16, 0x0000FFFF0000FFFFull);
        lo = swap_step(lo, lane, 8, 0x00FF00FF00FF00FFull);
        hi = swap_step(hi, lane, 8, 0x00FF00FF00FF00FFull);
        lo = swap_step(lo, lane, 4, 0x0F0F0F0F0F0F0F0Full);
        hi = swap_step(hi, lane, 4, 0x0F0F0F0F0F0F0F0Full);
        lo = swap_step(lo, lane, 2, 0x3333333333333333ull);
        hi = swap_step(hi, lane, 2, 0x3333333333333333ull);
        lo = swap_step(lo, lane, 1, 0x5555555555555555ull);
        hi = swap_step(hi, lane, 1, 0x5555555555555555ull);
        tout[cb * 64 + lane][rb] = lo;
        tout[cb * 64 + lane + 32][rb] = hi;
    }
    __syncthreads();

    {
        const int64_t orow = w0 * 64 + t;  // output row = input column
        const int64_t ow0 = r0 / 64;
#pragma unroll
        for (int q = 0; q < TILE_R / 64; q++)
            if (orow < cols && ow0 + q < tw) Xt[orow * tpitch + ow0 + q] = tout[t][q];
    }
}

}  // namespace

cudaError_t launch_transpose_pitched(const uint64_t* X, int64_t pitch, uint64_t* Xt,
                                     int64_t tpitch, int64_t rows, int64_t cols,
                                     cudaStream_t s) {
    const int64_t gx = (cols / 64 + TILE_W - 1) / TILE_W;
    const int64_t gy = (rows + TILE_R - 1) / TILE_R;
    if (gx <= 0 || gy <= 0) return cudaSuccess;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    TraceScope ts(BMM_PHASE_TRANSPOSE, s);
    transpose_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(X, pitch, Xt, tpitch, rows,
                                                                      cols);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const uint64_t* X, uint64_t* Xt, int64_t rows, int64_t cols,
                             cudaStream_t s) {
    return launch_transpose_pitched(X, cols / 64, Xt, rows / 64, rows, cols, s);
}

}  // namespace bmm
