// XOR passes of the Strassen-like recursions over packed words: basis changes
// (Secs. 3.6 and 3.13), the expanding parallel layer (Sec. 3.9, Alg. 1), the
// compressing parallel layer (Sec. 3.11, Alg. 2) with up to two levels merged
// in registers (Sec. 3.15), and the depth-first combine / fold passes of the
// serial layer (Sec. 3.8, Eqs. rec-in and rec-out).
//
// All are HBM-bound streaming kernels: one thread per 64-bit word position of
// the leaf-sized block, coalesced along the row, every input word read once
// and every output word written once.
#include "internal.h"
#include "plan.h"
#include "slp.h"

namespace bmm {
namespace {

// Stored block (r, c) of an operand for block index q = 2*i + j of the paper's
// operand. The right operand is held transposed (Bt = B^T), so block (j, k)
// of B is the transpose of stored block (k, j).
template <int OPERAND>
__device__ __forceinline__ void stored_block(int q, int& r, int& c) {
    if (OPERAND == 0) {
        r = q >> 1;
        c = q & 1;
    } else {
        r = q & 1;
        c = q >> 1;
    }
}

// The blocks an expanding pass reads: the block X itself (mask 0), or the
// quadrants `mask` selects of the parent block X of twice the size, XORed
// together (the input combination of a depth-first level, Eq. rec-in, fused
// into the pass). Returns how many, with their offsets in words from X;
// brows x bw is the expanded block's size in words.
template <int OPERAND>
__device__ __forceinline__ int source_blocks(uint32_t mask, int64_t pitch, int64_t brows,
                                             int64_t bw, int64_t (&off)[4]) {
    if (mask == 0) {
        off[0] = 0;
        return 1;
    }
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!((mask >> q) & 1u)) continue;
        int r, c;
        stored_block<OPERAND>(q, r, c);
        off[cnt++] = r * brows * pitch + c * bw;
    }
    return cnt;
}

// The blocks a compressing pass writes: C itself (dest 0), or the quadrants
// `dest` selects of the parent C (the output fold of a depth-first level,
// Eq. rec-out, fused into the pass): block q becomes v where bit q of
// `first` is set, else is XORed with v.
__device__ __forceinline__ int dest_blocks(uint32_t dest, uint32_t first, int64_t ldc,
                                           int64_t brows, int64_t bw, int64_t (&off)[4],
                                           bool (&overwrite)[4]) {
    if (dest == 0) {
        off[0] = 0;
        overwrite[0] = true;
        return 1;
    }
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!((dest >> q) & 1u)) continue;
        off[cnt] = (q >> 1) * brows * ldc + (q & 1) * bw;
        overwrite[cnt++] = (first >> q) & 1u;
    }
    return cnt;
}

template <int V, int OPERAND, typename Wd>
__device__ __forceinline__ void combine_level(const Wd* in, Wd* out) {
    if (OPERAND == 0)
        slp::alpha<V>(in, out);
    else
        slp::beta<V>(in, out);
}

// Expanding pass over D merged levels: basis change (phi / psi) then the
// operand combinations (alpha / beta) at every level, from 4^D input words
// to 7^D leaf words per position. Leaf index H = h_1 7^(D-1) + ... + h_D
// (level 1 most significant). rows x wcols is the expanded block; with a
// non-zero mask it is formed on the fly from its parent X (src_word).
template <int V, int D, int OPERAND>
__global__ void __launch_bounds__(256, 2) expand_kernel(const uint64_t* __restrict__ X, int64_t pitch,
                                                     int64_t rows, int64_t wcols, uint32_t mask,
                                                     uint64_t* __restrict__ leaves) {
    const int64_t lr = rows >> D, lw = wcols >> D;
    const int64_t leaf_words = lr * lw;
    const int64_t total = leaf_words;
    int64_t soff[4];
    const int nsrc = source_blocks<OPERAND>(mask, pitch, rows, wcols, soff);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / lw, w = t - i * lw;
        if (D == 1) {
            uint64_t x[4] = {0, 0, 0, 0}, y[7];
            for (int u = 0; u < nsrc; u++) {
                const uint64_t* src = X + soff[u];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    int r, c;
                    stored_block<OPERAND>(q, r, c);
                    x[q] ^= src[(r * lr + i) * pitch + c * lw + w];
                }
            }
            slp::phi<V>(x);
            combine_level<V, OPERAND>(x, y);
#pragma unroll
            for (int h = 0; h < 7; h++) leaves[h * leaf_words + t] = y[h];
        } else {
            uint64_t x[4][4];  // [level-1 block][level-2 block]
#pragma unroll
            for (int q1 = 0; q1 < 4; q1++)
#pragma unroll
                for (int q2 = 0; q2 < 4; q2++) x[q1][q2] = 0;
            for (int u = 0; u < nsrc; u++) {  // 16 independent loads per source block
                const uint64_t* src = X + soff[u];
#pragma unroll
                for (int q1 = 0; q1 < 4; q1++)
#pragma unroll
                    for (int q2 = 0; q2 < 4; q2++) {
                        int r1, c1, r2, c2;
                        stored_block<OPERAND>(q1, r1, c1);
                        stored_block<OPERAND>(q2, r2, c2);
                        x[q1][q2] ^= src[(r1 * 2 * lr + r2 * lr + i) * pitch + c1 * 2 * lw +
                                         c2 * lw + w];
                    }
            }
            // basis change at level 2 (within each level-1 block) and at level 1
#pragma unroll
            for (int q1 = 0; q1 < 4; q1++) slp::phi<V>(x[q1]);
#pragma unroll
            for (int q2 = 0; q2 < 4; q2++) {
                uint64_t v[4] = {x[0][q2], x[1][q2], x[2][q2], x[3][q2]};
                slp::phi<V>(v);
#pragma unroll
                for (int q1 = 0; q1 < 4; q1++) x[q1][q2] = v[q1];
            }
            // level-2 combinations, then level-1 combinations (Yates)
            uint64_t y[4][7];
#pragma unroll
            for (int q1 = 0; q1 < 4; q1++) combine_level<V, OPERAND>(x[q1], y[q1]);
#pragma unroll
            for (int h2 = 0; h2 < 7; h2++) {
                uint64_t v[4] = {y[0][h2], y[1][h2], y[2][h2], y[3][h2]}, z[7];
                combine_level<V, OPERAND>(v, z);
#pragma unroll
                for (int h1 = 0; h1 < 7; h1++) leaves[(h1 * 7 + h2) * leaf_words + t] = z[h1];
            }
        }
    }
}

// Compressing pass over D merged levels: gamma then the inverse basis change
// chi at every level, from 7^D leaf products to 4^D output words, written
// into C or folded into its parent (dst_word).
template <int V, int D>
__global__ void __launch_bounds__(256, 2) compress_kernel(const uint64_t* __restrict__ leaves,
                                                       int64_t lr, int64_t lw,
                                                       uint64_t* __restrict__ C, int64_t ldc,
                                                       uint32_t dest, uint32_t first) {
    const int64_t leaf_words = lr * lw;
    int64_t doff[4];
    bool over[4];
    const int ndst = dest_blocks(dest, first, ldc, lr << D, lw << D, doff, over);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < leaf_words;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / lw, w = t - i * lw;
        if (D == 1) {
            uint64_t q[7], c[4];
#pragma unroll
            for (int h = 0; h < 7; h++) q[h] = leaves[h * leaf_words + t];
            slp::gamma<V>(q, c);
            slp::chi<V>(c);
            for (int u = 0; u < ndst; u++) {  // all old words loaded before any store
                uint64_t* dst = C + doff[u];
                uint64_t old[4] = {0, 0, 0, 0};
                if (!over[u]) {
#pragma unroll
                    for (int b = 0; b < 4; b++) old[b] = dst[((b >> 1) * lr + i) * ldc + (b & 1) * lw + w];
                }
#pragma unroll
                for (int b = 0; b < 4; b++)
                    dst[((b >> 1) * lr + i) * ldc + (b & 1) * lw + w] = old[b] ^ c[b];
            }
        } else {
            uint64_t u[7][4];  // [h1][level-2 block]
#pragma unroll
            for (int h1 = 0; h1 < 7; h1++) {
                uint64_t q[7];
#pragma unroll
                for (int h2 = 0; h2 < 7; h2++) q[h2] = leaves[(h1 * 7 + h2) * leaf_words + t];
                slp::gamma<V>(q, u[h1]);
            }
            uint64_t c[4][4];  // [level-1 block][level-2 block]
#pragma unroll
            for (int b2 = 0; b2 < 4; b2++) {
                uint64_t q[7] = {u[0][b2], u[1][b2], u[2][b2], u[3][b2], u[4][b2], u[5][b2], u[6][b2]};
                uint64_t v[4];
                slp::gamma<V>(q, v);
                slp::chi<V>(v);  // level-1 inverse basis change
#pragma unroll
                for (int b1 = 0; b1 < 4; b1++) c[b1][b2] = v[b1];
            }
#pragma unroll
            for (int b1 = 0; b1 < 4; b1++) slp::chi<V>(c[b1]);  // level-2 inverse basis change
            for (int u = 0; u < ndst; u++) {  // all old words loaded before any store
                uint64_t* dst = C + doff[u];
                uint64_t old[4][4];
#pragma unroll
                for (int b1 = 0; b1 < 4; b1++)
#pragma unroll
                    for (int b2 = 0; b2 < 4; b2++) {
                        const int64_t row = (b1 >> 1) * 2 * lr + (b2 >> 1) * lr + i;
                        const int64_t col = (b1 & 1) * 2 * lw + (b2 & 1) * lw + w;
                        old[b1][b2] = over[u] ? 0ull : dst[row * ldc + col];
                    }
#pragma unroll
                for (int b1 = 0; b1 < 4; b1++)
#pragma unroll
                    for (int b2 = 0; b2 < 4; b2++) {
                        const int64_t row = (b1 >> 1) * 2 * lr + (b2 >> 1) * lr + i;
                        const int64_t col = (b1 & 1) * 2 * lw + (b2 & 1) * lw + w;
                        dst[row * ldc + col] = old[b1][b2] ^ c[b1][b2];
                    }
            }
        }
    }
}

// Depth-first input combination (Eq. rec-in with the basis change folded in):
// dst = XOR of the blocks of X selected by `mask` (bit q = block q of the
// paper's operand; OPERAND 1 reads the transposed right operand).
template <int OPERAND>
__global__ void __launch_bounds__(256) combine_kernel(const uint64_t* __restrict__ X, int64_t pitch,
                                                      int64_t hr, int64_t hw, uint32_t mask,
                                                      uint64_t* __restrict__ dst) {
    const int64_t total = hr * hw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / hw, w = t - i * hw;
        uint64_t acc = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (!((mask >> q) & 1u)) continue;
            int r, c;
            stored_block<OPERAND>(q, r, c);
            acc ^= X[(r * hr + i) * pitch + c * hw + w];
        }
        dst[t] = acc;
    }
}

// Depth-first output fold (Eq. rec-out): for each block q of C in `dest`,
// C_q = R (bit q of `first`) or C_q ^= R.
__global__ void __launch_bounds__(256) fold_kernel(const uint64_t* __restrict__ R, int64_t hr,
                                                   int64_t hw, uint64_t* __restrict__ C, int64_t ldc,
                                                   uint32_t dest, uint32_t first) {
    const int64_t total = hr * hw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / hw, w = t - i * hw;
        const uint64_t v = R[t];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (!((dest >> q) & 1u)) continue;
            uint64_t* p = C + ((q >> 1) * hr + i) * ldc + (q & 1) * hw + w;
            *p = ((first >> q) & 1u) ? v : (*p ^ v);
        }
    }
}

// One in-place basis-change level over all parent blocks at depth `level-1`.
template <int V, int INV>
__global__ void __launch_bounds__(256) basis_level_kernel(uint64_t* __restrict__ X, int64_t pitch,
                                                          int64_t rows, int64_t wcols, int level) {
    const int64_t hr = rows >> level, hw = wcols >> level;
    const int64_t half_r = rows >> 1, half_w = wcols >> 1;
    const int64_t total = half_r * half_w;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rho = t / half_w, omega = t - rho * half_w;
        const int64_t pr = rho / hr, i = rho - pr * hr;
        const int64_t pc = omega / hw, w = omega - pc * hw;
        uint64_t* base = X + (pr * 2 * hr + i) * pitch + pc * 2 * hw + w;
        uint64_t x[4];
#pragma unroll
        for (int q = 0; q < 4; q++) x[q] = base[(q >> 1) * hr * pitch + (q & 1) * hw];
        if (INV)
            slp::chi<V>(x);
        else
            slp::phi<V>(x);
#pragma unroll
        for (int q = 1; q < 4; q++) base[(q >> 1) * hr * pitch + (q & 1) * hw] = x[q];
    }
}

unsigned grid_for(int64_t items) {
    const int64_t cap = (int64_t)sm_count() * 8;
    int64_t b = (items + 255) / 256;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <int V>
cudaError_t launch_expand_v(int operand, int d, const uint64_t* X, int64_t pitch, int64_t rows,
                            int64_t wcols, uint32_t mask, uint64_t* leaves, cudaStream_t s) {
    const unsigned g = grid_for((rows >> d) * (wcols >> d));
    TraceScope ts(BMM_PHASE_XOR, s);
    if (d == 1) {
        if (operand == 0)
            expand_kernel<V, 1, 0><<<g, 256, 0, s>>>(X, pitch, rows, wcols, mask, leaves);
        else
            expand_kernel<V, 1, 1><<<g, 256, 0, s>>>(X, pitch, rows, wcols, mask, leaves);
    } else {
        if (operand == 0)
            expand_kernel<V, 2, 0><<<g, 256, 0, s>>>(X, pitch, rows, wcols, mask, leaves);
        else
            expand_kernel<V, 2, 1><<<g, 256, 0, s>>>(X, pitch, rows, wcols, mask, leaves);
    }
    return cudaGetLastError();
}

template <int V>
cudaError_t launch_compress_v(int d, const uint64_t* leaves, int64_t lr, int64_t lw, uint64_t* C,
                              int64_t ldc, uint32_t dest, uint32_t first, cudaStream_t s) {
    const unsigned g = grid_for(lr * lw);
    TraceScope ts(BMM_PHASE_XOR, s);
    if (d == 1)
        compress_kernel<V, 1><<<g, 256, 0, s>>>(leaves, lr, lw, C, ldc, dest, first);
    else
        compress_kernel<V, 2><<<g, 256, 0, s>>>(leaves, lr, lw, C, ldc, dest, first);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_expand(int variant, int operand, int d, const uint64_t* X, int64_t pitch,
                          int64_t rows, int64_t wcols, uint32_t mask, uint64_t* leaves,
                          cudaStream_t s) {
    switch (variant) {
        case 0: return launch_expand_v<0>(operand, d, X, pitch, rows, wcols, mask, leaves, s);
        case 1: return launch_expand_v<1>(operand, d, X, pitch, rows, wcols, mask, leaves, s);
        default: return launch_expand_v<2>(operand, d, X, pitch, rows, wcols, mask, leaves, s);
    }
}

cudaError_t launch_compress(int variant, int d, const uint64_t* leaves, int64_t lr, int64_t lw,
                            uint64_t* C, int64_t ldc, uint32_t dest, uint32_t first,
                            cudaStream_t s) {
    switch (variant) {
        case 0: return launch_compress_v<0>(d, leaves, lr, lw, C, ldc, dest, first, s);
        case 1: return launch_compress_v<1>(d, leaves, lr, lw, C, ldc, dest, first, s);
        default: return launch_compress_v<2>(d, leaves, lr, lw, C, ldc, dest, first, s);
    }
}

cudaError_t launch_combine(int operand, const uint64_t* X, int64_t pitch, int64_t hr, int64_t hw,
                           uint32_t mask, uint64_t* dst, cudaStream_t s) {
    const unsigned g = grid_for(hr * hw);
    TraceScope ts(BMM_PHASE_XOR, s);
    if (operand == 0)
        combine_kernel<0><<<g, 256, 0, s>>>(X, pitch, hr, hw, mask, dst);
    else
        combine_kernel<1><<<g, 256, 0, s>>>(X, pitch, hr, hw, mask, dst);
    return cudaGetLastError();
}

cudaError_t launch_fold(const uint64_t* R, int64_t hr, int64_t hw, uint64_t* C, int64_t ldc,
                        uint32_t dest, uint32_t first, cudaStream_t s) {
    TraceScope ts(BMM_PHASE_XOR, s);
    fold_kernel<<<grid_for(hr * hw), 256, 0, s>>>(R, hr, hw, C, ldc, dest, first);
    return cudaGetLastError();
}

bmm_status run_basis_change(int variant, int inverse, uint64_t* X, int64_t pitch, int64_t rows,
                            int64_t cols, int depth, cudaStream_t s) {
    const int64_t wcols = cols / 64;
    if (variant == 0) return BMM_OK;  // standard basis: identity
    for (int level = 1; level <= depth; level++) {
        const unsigned g = grid_for((rows / 2) * (wcols / 2));
        TraceScope ts(BMM_PHASE_XOR, s);
        if (variant == 1) {
            if (inverse)
                basis_level_kernel<1, 1><<<g, 256, 0, s>>>(X, pitch, rows, wcols, level);
            else
                basis_level_kernel<1, 0><<<g, 256, 0, s>>>(X, pitch, rows, wcols, level);
        } else {
            if (inverse)
                basis_level_kernel<2, 1><<<g, 256, 0, s>>>(X, pitch, rows, wcols, level);
            else
                basis_level_kernel<2, 0><<<g, 256, 0, s>>>(X, pitch, rows, wcols, level);
        }
        BMM_CUDA_TRY(cudaGetLastError());
    }
    return BMM_OK;
}

}  // namespace bmm
