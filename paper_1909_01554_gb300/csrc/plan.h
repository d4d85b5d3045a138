// Planning and execution of one product: which base-case path, how many
// Strassen levels run depth-first (serial layer, Sec. 3.8) and how many run
// breadth-first in fused XOR passes (parallel layers, Secs. 3.9 and 3.11),
// and how the scratch memory is laid out.
#pragma once

#include "internal.h"

namespace bmm {

struct Plan {
    int op = OP_GF2;
    int path = BMM_PATH_POPC;  // resolved base-case path
    int variant = BMM_VARIANT_SELF_INVERSE;
    int depth = 0;             // total Strassen levels (0 = cubic)
    int serial = 0;            // of which depth-first (top) levels
    int kernel_level = 0;      // 1: the innermost level runs inside the base-case kernel
    int64_t m = 0, k = 0, n = 0;
    // k the kernels run with: the tensor-core paths need every leaf's k to be
    // a multiple of 128 bits, so k is rounded up with zero columns of A and
    // zero rows of B (the product is unchanged); kp == k otherwise.
    int64_t kp = 0;
    uint64_t workspace_bytes = 0;
};

bmm_status make_plan(int op, int64_t m, int64_t k, int64_t n, const bmm_opts* opts, Plan* out);

// Scratch bytes of a plan with these sizes, Strassen depth and depth-first
// levels, k padded to kp (a padded copy of A when kp != k).
uint64_t workspace_padded(int64_t m, int64_t k, int64_t kp, int64_t n, int depth, int serial);

// Bytes the plan's streaming passes move through HBM: the transpose of B and
// every XOR pass (depth-first combine / fold, breadth-first expand /
// compress), not counting the base case.
uint64_t plan_pass_bytes(const Plan& p);

// The autotuner's recorded choice for (op, m, k, n) on the current device:
// base-case path and Strassen depth. False if the shape was not tuned.
bool tuned_choice(int op, int64_t m, int64_t k, int64_t n, int* path, int* depth);

bmm_status execute_plan(const Plan& p, const uint64_t* A, const uint64_t* B, uint64_t* C,
                        void* workspace, cudaStream_t s);

// C (pitch ldc) = A (pitch lda) * Bt^T (pitch ldb): the base case on one path.
bmm_status run_base_product(int op, int path, const uint64_t* A, int64_t lda, const uint64_t* Bt,
                            int64_t ldb, uint64_t* C, int64_t ldc, int64_t m, int64_t k,
                            int64_t n, cudaStream_t s);

// Batched base case over `count` leaves of equal shape:
// A_h = A + h*strideA, Bt_h = Bt + h*strideB, C_h = C + h*strideC (words),
// each with its own row pitch (lda, ldb, ldc words).
bmm_status run_base_product_batched(int op, int path, const uint64_t* A, int64_t lda,
                                    int64_t strideA, const uint64_t* Bt, int64_t ldb,
                                    int64_t strideB, uint64_t* C, int64_t ldc, int64_t strideC,
                                    int64_t count, int64_t m, int64_t k, int64_t n,
                                    cudaStream_t s);

bmm_status run_basis_change(int variant, int inverse, uint64_t* X, int64_t pitch, int64_t rows,
                            int64_t cols, int depth, cudaStream_t s);

bmm_status run_batched(int op, int32_t count, const uint64_t* const* A,
                       const uint64_t* const* B, uint64_t* const* C, const int64_t* m,
                       const int64_t* k, const int64_t* n, cudaStream_t s);

}  // namespace bmm
