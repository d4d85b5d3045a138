// Descriptors shared by the batched form of the tensor-core base case and
// the host code that plans it.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "internal.h"

namespace bmm {

// One product of the batch, as the persistent kernel sees it (global memory;
// CUtensorMap's own alignment keeps the TMA maps inside usable in place).
struct TcProblem {
    CUtensorMap mapA;  // A (m x k), 3-D map (k words, m rows, 1)
    CUtensorMap mapB;  // Bt (n x k)
    uint64_t* C;
    int64_t ldc;       // words
    int32_t m, n, nks, op;  // nks: k stages (128 bits e4m3, 256 bits e2m1)
};

// One output tile (TC_TILE_M rows, or 2 * TC_TILE_M for an SM pair, x
// TC_TILE_N columns) of one problem; tm counts tiles of that height.
// It repeats the problem fields the epilogue needs, so a role reads one item
// per tile rather than an item and then its problem.
struct TcWorkItem {
    int32_t prob, tm, tn;
    int32_t nks;   // the problem's k stages; may be odd: the last packed stage
                   // then runs only its first operand stage's MMAs
    int32_t n128;  // 1: the tile's MMAs are N = 128 (its columns past 128 lie beyond n)
    int32_t op, m, n;
    uint64_t* C;
    int64_t ldc;
};

constexpr int TC_TILE_M = 128;
constexpr int TC_TILE_N = 256;
// CTA pairs of the e4m3 (fp4 false) or e2m1 kernel that can be resident at
// once (0: SM pairs unavailable).
int tc_pair_slots(bool fp4);

// Fills the host copy of a problem descriptor (TMA maps need k % 128 == 0
// and even pitches) for the single-SM or the SM-pair kernel, e4m3 or e2m1
// operands (e2m1 only on SM pairs). Returns false if a map cannot be encoded.
bool tc_make_problem(TcProblem* out, const uint64_t* A, int64_t lda, const uint64_t* Bt,
                     int64_t ldb, uint64_t* C, int64_t ldc, int64_t m, int64_t k, int64_t n,
                     int op, bool pair, bool fp4);

// The batched kernel's one-time launch setup on the current device (done
// when a plan is made, so that a plan's first run can be captured).
cudaError_t tc_prepare_batched(bool pair, bool fp4);

// One persistent launch over the per-unit work lists; a unit is one CTA, or
// one CTA pair when `pair`. unit_ptr has 2 * (units + 1) entries: the first
// units + 1 delimit each unit's items, entry units + 1 + u is unit u's
// number of packed stages (two k stages each, the last one possibly half).
cudaError_t tc_launch_batched(const TcProblem* d_probs, const TcWorkItem* d_items,
                              const int32_t* d_unit_ptr, int units, bool pair, bool fp4,
                              cudaStream_t s);

}  // namespace bmm
