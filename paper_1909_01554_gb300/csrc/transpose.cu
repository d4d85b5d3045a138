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
#include <mutex>

#include "internal.h"

namespace bmm {
namespace {

constexpr int MAX_DEV = 64;  // per-device one-time kernel attributes

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

// ---- the same tile through the tensor memory accelerator -------------------
// Strided 64-byte row segments moved by load/store instructions reach about
// half of HBM bandwidth on this part; TMA copies of the same boxes reach ~0.9
// (measured with plain tile copies). So where both row pitches are even
// (16-byte strides) the tile comes in as two TMA boxes of 256 rows x 64 bytes,
// 64-byte swizzled, is transposed in place in shared memory, and leaves as
// two TMA boxes. Out-of-range parts of a tile load as zero and are clipped
// from the stores by the TMA unit.
constexpr int TMA_TILE_BYTES = TILE_R * TILE_W * 8;  // 32 KB: 512 rows x 64 bytes
constexpr int TMA_SMEM = TMA_TILE_BYTES + 1024;      // + alignment of the swizzle atoms

// Byte offset of word w of row r in a tile the TMA unit wrote with the
// 64-byte swizzle: 16-byte chunk c of row r sits at chunk c ^ ((r >> 1) & 3).
__device__ __forceinline__ uint32_t swz(int r, int w) {
    return (uint32_t)(r * 64 + ((((w >> 1) ^ (r >> 1)) & 3) << 4) + ((w & 1) << 3));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Every tile's transpose in shared memory, as transpose_tile does it, on the
// swizzled layout.
__device__ __forceinline__ void transpose_swizzled(uint8_t* t) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto at = [&](int r, int w) { return reinterpret_cast<uint64_t*>(t + swz(r, w)); };
    for (int u = warp; u < TILE_B * (TILE_B + 1) / 2; u += 8) {
        int rb = 0, rem = u;
        while (rem >= TILE_B - rb) {
            rem -= TILE_B - rb;
            rb++;
        }
        const int cb = rb + rem;
        uint64_t lo = *at(rb * 64 + lane, cb), hi = *at(rb * 64 + lane + 32, cb);
        uint64_t lo2 = 0, hi2 = 0;
        if (cb != rb) {
            lo2 = *at(cb * 64 + lane, rb);
            hi2 = *at(cb * 64 + lane + 32, rb);
        }
        __syncwarp();
        transpose_block(lo, hi, lane);
        *at(cb * 64 + lane, rb) = lo;
        *at(cb * 64 + lane + 32, rb) = hi;
        if (cb != rb) {
            transpose_block(lo2, hi2, lane);
            *at(rb * 64 + lane, cb) = lo2;
            *at(rb * 64 + lane + 32, cb) = hi2;
        }
    }
}

constexpr uint64_t TMA_WAIT_NS = 2000000000ull;  // 2 s

// One tile: input words [8 bx, 8 bx + 8), rows [512 by, 512 by + 512) of the
// map mx; output (map mt) rows [512 bx, ...), words [8 by, ...). A wait that
// gives up records DEVERR_TIMEOUT and the CTA skips its stores.
__device__ __forceinline__ void transpose_tile_tma(const CUtensorMap* mx, const CUtensorMap* mt,
                                                   int64_t bx, int64_t by, int64_t cols,
                                                   uint8_t* t, uint64_t* bar, uint32_t* err) {
    const uint32_t b = smem_addr(bar), ts = smem_addr(t);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                     "r"((uint32_t)TMA_TILE_BYTES)
                     : "memory");
        for (int h = 0; h < 2; h++)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(ts + h * (TMA_TILE_BYTES / 2)),
                "l"(reinterpret_cast<uint64_t>(mx)), "r"((int)(bx * TILE_W)),
                "r"((int)(by * TILE_R + h * (TILE_R / 2))), "r"(b)
                : "memory");
    }
    uint32_t ok = 0;
    uint64_t t0 = 0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t i = 1; !ok; i++) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(b)
            : "memory");
        if (!ok && (i & 255u) == 0) {
            uint64_t now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            if (now - t0 > TMA_WAIT_NS) break;
        }
    }
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicOr(err, DEVERR_TIMEOUT);
        return;
    }
    transpose_swizzled(t);
    // the generic-proxy writes above, before the TMA unit reads the tile
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        // (a box that starts past the last output row has nothing to store)
        for (int h = 0; h < 2 && bx * TILE_R + h * (TILE_R / 2) < cols; h++)
            asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                             reinterpret_cast<uint64_t>(mt)),
                         "r"((int)(by * TILE_W)), "r"((int)(bx * TILE_R + h * (TILE_R / 2))),
                         "r"(ts + h * (TMA_TILE_BYTES / 2))
                         : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        // the stores must have read the tile before the CTA's shared memory goes
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
}

__global__ void __launch_bounds__(256) transpose_tma_kernel(const __grid_constant__ CUtensorMap mx,
                                                            const __grid_constant__ CUtensorMap mt,
                                                            int64_t cols, uint32_t* err) {
    extern __shared__ __align__(1024) uint8_t tma_raw[];
    __shared__ __align__(8) uint64_t bar;
    uint8_t* t = (uint8_t*)(((uintptr_t)tma_raw + 1023) & ~(uintptr_t)1023);
    transpose_tile_tma(&mx, &mt, blockIdx.x, blockIdx.y, cols, t, &bar, err);
}

// TMA-form jobs of a batch in one launch (as transpose_batched_kernel).
__global__ void __launch_bounds__(256) transpose_tma_batched_kernel(
    const TmaTransposeJob* __restrict__ jobs, const int64_t* __restrict__ first, int count,
    uint32_t* err) {
    extern __shared__ __align__(1024) uint8_t tma_raw[];
    __shared__ __align__(8) uint64_t bar;
    uint8_t* t = (uint8_t*)(((uintptr_t)tma_raw + 1023) & ~(uintptr_t)1023);
    const int64_t b = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last i with first[i] <= b
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const TmaTransposeJob* j = jobs + lo;
    const int64_t local = b - first[lo], gx = j->gx;
    transpose_tile_tma(&j->mx, &j->mt, local % gx, local / gx, j->cols, t, &bar, err);
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

// The TMA form needs 16-byte aligned bases and row strides, and whole boxes
// inside each dimension of the maps.
bool tma_transposable(const uint64_t* X, int64_t pitch, const uint64_t* Xt, int64_t tpitch,
                      int64_t rows, int64_t cols) {
    return ((uintptr_t)X & 15) == 0 && ((uintptr_t)Xt & 15) == 0 && pitch % 2 == 0 &&
           tpitch % 2 == 0 && rows >= TILE_R && cols >= TILE_R && rows / 64 <= 0x7fffffff &&
           cols <= 0x7fffffff && rows <= 0x7fffffff;
}

cudaError_t tma_attr() {
    static bool done[MAX_DEV] = {false};
    static cudaError_t err[MAX_DEV];
    static std::mutex mu;
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAX_DEV) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[d]) {
        err[d] = cudaFuncSetAttribute(transpose_tma_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM);
        if (err[d] == cudaSuccess)
            err[d] = cudaFuncSetAttribute(transpose_tma_batched_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM);
        done[d] = true;
    }
    return err[d];
}

bool make_transpose_tma_job(TmaTransposeJob* out, const TransposeJob& j) {
    if (device_cc() != 103 || !tma_transposable(j.X, j.pitch, j.Xt, j.tpitch, j.rows, j.cols) ||
        tma_attr() != cudaSuccess)
        return false;
    out->gx = (j.cols / 64 + TILE_W - 1) / TILE_W;
    out->cols = j.cols;
    return make_map_2d(&out->mx, j.X, j.cols / 64, j.rows, j.pitch * 8, TILE_W, TILE_R / 2, true) &&
           make_map_2d(&out->mt, j.Xt, j.rows / 64, j.cols, j.tpitch * 8, TILE_W, TILE_R / 2,
                       true);
}

cudaError_t launch_transpose_tma_batched(const TmaTransposeJob* jobs, const int64_t* first,
                                         int count, int64_t total_tiles, cudaStream_t s) {
    if (count <= 0 || total_tiles <= 0) return cudaSuccess;
    if (total_tiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
    cudaError_t e = tma_attr();
    if (e != cudaSuccess) return e;
    uint32_t* err = device_error_word();
    if (!err) return cudaErrorMemoryAllocation;
    TraceScope ts(BMM_PHASE_TRANSPOSE, s);
    transpose_tma_batched_kernel<<<(unsigned)total_tiles, 256, TMA_SMEM, s>>>(jobs, first, count,
                                                                           err);
    return cudaGetLastError();
}

cudaError_t launch_transpose_loadstore(const uint64_t* X, uint64_t* Xt, int64_t rows,
                                       int64_t cols, cudaStream_t s) {
    const int64_t gx = (cols / 64 + TILE_W - 1) / TILE_W;
    const int64_t gy = (rows + TILE_R - 1) / TILE_R;
    if (gx <= 0 || gy <= 0) return cudaSuccess;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    TraceScope ts(BMM_PHASE_TRANSPOSE, s);
    transpose_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(X, cols / 64, Xt, rows / 64,
                                                                      rows, cols);
    return cudaGetLastError();
}

cudaError_t launch_transpose_pitched(const uint64_t* X, int64_t pitch, uint64_t* Xt,
                                     int64_t tpitch, int64_t rows, int64_t cols,
                                     cudaStream_t s) {
    const int64_t gx = (cols / 64 + TILE_W - 1) / TILE_W;
    const int64_t gy = (rows + TILE_R - 1) / TILE_R;
    if (gx <= 0 || gy <= 0) return cudaSuccess;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    CUtensorMap mx, mt;
    uint32_t* err = nullptr;
    if (device_cc() == 103 && tma_transposable(X, pitch, Xt, tpitch, rows, cols) &&
        tma_attr() == cudaSuccess && (err = device_error_word()) != nullptr &&
        make_map_2d(&mx, X, cols / 64, rows, pitch * 8, TILE_W, TILE_R / 2, true) &&
        make_map_2d(&mt, Xt, rows / 64, cols, tpitch * 8, TILE_W, TILE_R / 2, true)) {
        TraceScope ts(BMM_PHASE_TRANSPOSE, s);
        transpose_tma_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, TMA_SMEM, s>>>(mx, mt, cols,
                                                                                   err);
        return cudaGetLastError();
    }
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
