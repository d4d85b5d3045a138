// Bit-matrix transpose (Sec. 3.5: the paper transposes the right operand so
// that both operands of the inner product run along k; it does this on the
// host with recursive 64x64 word transposes). Here: on the GPU, one warp per
// 64x64 bit block, the recursive block swap done with warp shuffles.
//
// HBM-bound: reads rows*cols/8 bytes and writes the same. A CTA moves a tile
// of 512 rows x 512 columns (8 x 8 blocks of 64 x 64) through shared memory,
// so both the loads and the stores touch 64 contiguous bytes per row, and the
// tile is transposed in place: a warp takes a block and its mirror image
// across the diagonal, transposes both in registers and writes each into the
// other's place.
#include "internal.h"

namespace bmm {
namespace {

constexpr int TILE_B = 8;           // 64 x 64 blocks per tile side
constexpr int TILE_R = 64 * TILE_B; // input rows per CTA
constexpr int TILE_W = TILE_B;      // input words (64 columns each) per CTA
constexpr int PADW = TILE_W + 1;    // padded shared row (spreads a block column over the banks)

__device__ __forceinline__ uint64_t swap_step(uint64_t v, int lane, int j, uint64_t mask) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, v, j);
    if ((lane & j) == 0) {
        const uint64_t t = ((v >> j) ^ other) & mask;
        return v ^ (t << j);
    }
    const uint64_t t = ((other >> j) ^ v) & mask;
    return v ^ t;
}

// Transposes the 64 x 64 bit block whose rows lane and lane + 32 this thread
// holds (lo, hi): afterwards lo / hi are rows lane and lane + 32 of the
// transposed block.
__device__ __forceinline__ void transpose_block(uint64_t& lo, uint64_t& hi, int lane) {
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
}

// One CTA tile: input rows [512 by, 512 by + 512), words [8 bx, 8 bx + 8).
// Entries outside the matrix read as zero and are not written.
__device__ __forceinline__ void transpose_tile(const uint64_t* __restrict__ X, int64_t pitch,
                                               uint64_t* __restrict__ Xt, int64_t tpitch,
                                               int64_t rows, int64_t cols, int64_t bx,
                                               int64_t by) {
    __shared__ uint64_t tile[TILE_R][PADW];
    const int t = threadIdx.x;
    const int64_t r0 = by * TILE_R;
    const int64_t w0 = bx * TILE_W;  // first input word (column / 64)
    const int64_t xw = cols / 64, tw = rows / 64;

    // load: eight consecutive lanes read one row's 64 bytes
#pragma unroll
    for (int i = t; i < TILE_R * TILE_W; i += 256) {
        const int r = i / TILE_W, q = i % TILE_W;
        const int64_t gr = r0 + r;
        tile[r][q] = (gr < rows && w0 + q < xw) ? X[gr * pitch + w0 + q] : 0ull;
    }
    __syncthreads();

    // blocks (rb, cb) and (cb, rb) trade places, transposed
    const int warp = t >> 5, lane = t & 31;
    for (int u = warp; u < TILE_B * (TILE_B + 1) / 2; u += 8) {
        int rb = 0, rem = u;  // u-th pair with rb <= cb, row by row
        while (rem >= TILE_B - rb) {
            rem -= TILE_B - rb;
            rb++;
        }
        const int cb = rb + rem;
        uint64_t lo = tile[rb * 64 + lane][cb], hi = tile[rb * 64 + lane + 32][cb];
        uint64_t lo2 = 0, hi2 = 0;
        if (cb != rb) {
            lo2 = tile[cb * 64 + lane][rb];
            hi2 = tile[cb * 64 + lane + 32][rb];
        }
        __syncwarp();
        transpose_block(lo, hi, lane);
        tile[cb * 64 + lane][rb] = lo;
        tile[cb * 64 + lane + 32][rb] = hi;
        if (cb != rb) {
            transpose_block(lo2, hi2, lane);
            tile[rb * 64 + lane][cb] = lo2;
            tile[rb * 64 + lane + 32][cb] = hi2;
        }
    }
    __syncthreads();

    // store: output row c (input column w0*64 + c) gets words [r0/64, r0/64 + 8)
    const int64_t ow0 = r0 / 64;
#pragma unroll
    for (int i = t; i < TILE_R * TILE_W; i += 256) {
        const int c = i / TILE_W, q = i % TILE_W;
        const int64_t orow = w0 * 64 + c;
        if (orow < cols && ow0 + q < tw) Xt[orow * tpitch + ow0 + q] = tile[c][q];
    }
}

__global__ void __launch_bounds__(256) transpose_kernel(const uint64_t* __restrict__ X,
                                                        int64_t pitch, uint64_t* __restrict__ Xt,
                                                        int64_t tpitch, int64_t rows,
                                                        int64_t cols) {
    transpose_tile(X, pitch, Xt, tpitch, rows, cols, blockIdx.x, blockIdx.y);
}

// Many transposes in one launch: CTA b takes tile b - first[i] of problem i,
// where first[] is the exclusive prefix of the problems' tile counts.
__global__ void __launch_bounds__(256) transpose_batched_kernel(const TransposeJob* __restrict__ jobs,
                                                                const int64_t* __restrict__ first,
                                                                int count) {
    const int64_t b = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last i with first[i] <= b
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const TransposeJob j = jobs[lo];
    const int64_t local = b - first[lo];
    const int64_t gx = (j.cols / 64 + TILE_W - 1) / TILE_W;
    transpose_tile(j.X, j.pitch, j.Xt, j.tpitch, j.rows, j.cols, local % gx, local / gx);
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

int64_t transpose_tiles(int64_t rows, int64_t cols) {
    return ((cols / 64 + TILE_W - 1) / TILE_W) * ((rows + TILE_R - 1) / TILE_R);
}

cudaError_t launch_transpose_batched(const TransposeJob* jobs, const int64_t* first, int count,
                                     int64_t total_tiles, cudaStream_t s) {
    if (count <= 0 || total_tiles <= 0) return cudaSuccess;
    if (total_tiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
    TraceScope ts(BMM_PHASE_TRANSPOSE, s);
    transpose_batched_kernel<<<(unsigned)total_tiles, 256, 0, s>>>(jobs, first, count);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const uint64_t* X, uint64_t* Xt, int64_t rows, int64_t cols,
                             cudaStream_t s) {
    return launch_transpose_pitched(X, cols / 64, Xt, rows / 64, rows, cols, s);
}

}  // namespace bmm
