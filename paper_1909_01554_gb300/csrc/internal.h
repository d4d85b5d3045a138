// Internal declarations shared by the translation units of libbmm.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bmm.h"

namespace bmm {

constexpr int OP_GF2 = 0;
constexpr int OP_BOOL = 1;

// Device-side failure word (one per device, allocated on first use). Kernels
// whose bounded waits give up OR a code into it and return.
constexpr uint32_t DEVERR_TIMEOUT = 1u;

uint32_t* device_error_word();  // nullptr if allocation failed

// Records a CUDA error for bmm_last_cuda_error() and maps it to a status.
bmm_status cuda_fail(cudaError_t e);
#define BMM_CUDA_TRY(expr)                              \
    do {                                                \
        cudaError_t bmm_e_ = (expr);                    \
        if (bmm_e_ != cudaSuccess) return cuda_fail(bmm_e_); \
    } while (0)

// The argument checks every product entry point shares: null pointers,
// sizes (positive multiples of 64), 16-byte alignment, C overlapping A or B.
bmm_status check_product_args(const uint64_t* A, const uint64_t* B, const uint64_t* C,
                              int64_t m, int64_t k, int64_t n);

// Tracing hooks: wrap every kernel launch in a TraceScope.
void trace_launch_begin(int phase, cudaStream_t s, void** token);
void trace_launch_end(void* token, cudaStream_t s);
struct TraceScope {
    void* tok = nullptr;
    cudaStream_t s;
    TraceScope(int phase, cudaStream_t st) : s(st) { trace_launch_begin(phase, s, &tok); }
    ~TraceScope() { trace_launch_end(tok, s); }
};

// Number of SMs of the current device (cached per device).
int sm_count();
// Compute capability major*10 + minor of the current device.
int device_cc();

// ---- base-case paths --------------------------------------------------------
bool tc_path_available();  // tensor-core kernels: sm_103a and the TMA map encoder
bool tc_pair_available();  // e4m3 operands on SM pairs (clusters of two)
bool tc_fp4_available();   // e2m1 operands on SM pairs
// The base-case path BMM_PATH_AUTO resolves to on the current device.
int auto_path();
inline bool is_tc_path(int path) {
    return path == BMM_PATH_TC_FP8 || path == BMM_PATH_TC_FP8_PAIR ||
           path == BMM_PATH_TC_FP4_PAIR;
}

// A 2-D TMA map over uint64 words (words x rows, row stride in bytes, a
// multiple of 16), box of box_words x box_rows, optionally 64-byte swizzled.
// False if the driver's encoder is unavailable or refuses the arguments.
bool make_map_2d(CUtensorMap* map, const void* base, int64_t words, int64_t rows,
                 int64_t stride_bytes, int box_words, int box_rows, bool swizzle64);

// ---- launchers (each returns a launch error, or cudaSuccess) -------------
cudaError_t launch_transpose(const uint64_t* X, uint64_t* Xt, int64_t rows, int64_t cols,
                             cudaStream_t s);
// Always the load/store form, which needs no device memory of the library's
// own (the TMA form records bounded-wait timeouts in the device error word).
cudaError_t launch_transpose_loadstore(const uint64_t* X, uint64_t* Xt, int64_t rows,
                                       int64_t cols, cudaStream_t s);
// X is rows x cols with row pitch `pitch` words; Xt is cols x rows, row pitch tpitch words.
cudaError_t launch_transpose_pitched(const uint64_t* X, int64_t pitch, uint64_t* Xt,
                                     int64_t tpitch, int64_t rows, int64_t cols,
                                     cudaStream_t s);

// One transpose of a batch: Xt (cols x rows, pitch tpitch) = X^T (rows x cols, pitch pitch).
struct TransposeJob {
    const uint64_t* X;
    uint64_t* Xt;
    int64_t pitch, tpitch, rows, cols;
};
// CTA tiles one transpose takes (the batched launch needs their prefix sums).
int64_t transpose_tiles(int64_t rows, int64_t cols);
// A transpose of a batch in its TMA form (device memory, aligned as its maps).
struct TmaTransposeJob {
    CUtensorMap mx, mt;  // X (words x rows) and Xt (words x cols), 64-byte swizzled boxes
    int64_t gx, cols;    // tiles along X's words; Xt's rows
};
// Fills the TMA form of a job; false where it does not apply (odd pitches,
// unaligned bases, less than a 512 x 512 tile a side, no TMA on the device):
// such a job goes to launch_transpose_batched.
bool make_transpose_tma_job(TmaTransposeJob* out, const TransposeJob& j);
// All TMA-form jobs in one launch; first[i] = tiles of jobs 0..i-1 (device).
cudaError_t launch_transpose_tma_batched(const TmaTransposeJob* jobs, const int64_t* first,
                                         int count, int64_t total_tiles, cudaStream_t s);
// All jobs in one launch; first[i] = tiles of jobs 0..i-1 (device arrays).
cudaError_t launch_transpose_batched(const TransposeJob* jobs, const int64_t* first, int count,
                                     int64_t total_tiles, cudaStream_t s);

// CUDA-core base case: C (m x n, row pitch ldc words) = A (m x k, pitch lda)
// times Bt^T (Bt n x k, pitch ldb), GF(2) or Boolean.
// Leaf h of a batch of `count` starts at A + h*strideA, Bt + h*strideB,
// C + h*strideC (words).
cudaError_t launch_popc_nt(int op, const uint64_t* A, int64_t lda, int64_t strideA,
                           const uint64_t* Bt, int64_t ldb, int64_t strideB, uint64_t* C,
                           int64_t ldc, int64_t strideC, int64_t count, int64_t m, int64_t k,
                           int64_t n, cudaStream_t s);

// Batched CUDA-core base case: one problem C (m x n, pitch ldc) = A (m x k,
// pitch lda) times Bt^T (Bt n x k, pitch ldb), and one 128 x 128 tile of it.
struct PopcJob {
    const uint64_t* A;
    const uint64_t* Bt;
    uint64_t* C;
    int64_t lda, ldb, ldc, m, k, n;
    int32_t op, pad;
};
struct PopcTile {
    int32_t job, tm, tn, pad;
};
constexpr int POPC_TILE = 128;
// Every tile of the (device) list in one persistent launch; the list is
// walked in order, CTA b taking tiles b, b + grid, ...
cudaError_t launch_popc_batched(const PopcJob* jobs, const PopcTile* tiles, int64_t count,
                                cudaStream_t s);
// CTAs of that launch (resident blocks per SM x SMs).
int popc_batched_grid();

// Combined standard-basis operators of one Strassen level as 0/1 masks:
// xi[h] bit q = block q of A enters product h, eta[h] likewise for B,
// zeta[q] bit h = product h enters block q of C (blocks q = 2*row + col).
struct LevelMasks {
    uint32_t xi[7], eta[7], zeta[4];
};

// The binary product of each block of a batch through one Strassen level run
// inside the CUDA-core kernel: C (m x n) = A (m x k) Bt^T (Bt n x k), the
// seven quadrant products formed, multiplied and recombined in one launch
// (strides and pitches as launch_popc_nt). m even; k and n multiples of 128.
cudaError_t launch_popc_level(const uint64_t* A, int64_t lda, int64_t strideA, const uint64_t* Bt,
                              int64_t ldb, int64_t strideB, uint64_t* C, int64_t ldc,
                              int64_t strideC, int64_t count, int64_t m, int64_t k, int64_t n,
                              const LevelMasks& masks, cudaStream_t s);
// The same on the tensor cores (e2m1 operands, SM pairs): every quadrant's k a
// whole number of 512-bit packed stages (k a multiple of 1024), even pitches
// and strides; BMM_ERR_UNSUPPORTED otherwise or without the tensor path.
bmm_status run_tc_level(const uint64_t* A, int64_t lda, int64_t strideA, const uint64_t* Bt,
                        int64_t ldb, int64_t strideB, uint64_t* C, int64_t ldc, int64_t strideC,
                        int64_t count, int64_t m, int64_t k, int64_t n, const LevelMasks& masks,
                        cudaStream_t s);

}  // namespace bmm
