/*
 * bmm.h — C ABI of the GB300 (sm_103a) bit-matrix multiplication library.
 *
 * Products of bit matrices after Karppa & Kaski, "Engineering Boolean Matrix
 * Multiplication for Multiple-Accelerator Shared-Memory Architectures"
 * (arXiv:1909.01554):
 *   Boolean product  C_ij = OR_k  (A_ik AND B_kj)   over (0,1,OR,AND)  (Sec. 1; Sec. 3.18)
 *   binary product   C_ij = XOR_k (A_ik AND B_kj)   over GF(2)         (Sec. 2.4; Eq. c-equals-ab)
 * The binary product may run through the alternative-basis Strassen
 * recurrences of Sec. 2.2 (self-inverse, Thm. 1) or Sec. 2.3 (chaining,
 * Thm. 2), or Strassen–Winograd in the standard basis (Sec. 2.1), down to a
 * cubic base-case block product (Sec. 3.10).
 *
 * Matrix layout (all entry points): row-major, bit-packed into uint64 words,
 * least significant index in the bits of a word (Sec. 3.4 linearisation):
 * bit j of row i of an R x K matrix is bit (j % 64) of word i*(K/64) + j/64.
 * So A (m x k) has m*k/64 words, B (k x n) has k*n/64 words, C (m x n) has
 * m*n/64 words.
 *
 * Ownership: every matrix pointer is DEVICE memory owned by the caller, on
 * the current CUDA device. A and B are read only (the library never writes
 * them); C is overwritten (not accumulated). Buffers must not overlap.
 * Alignment: every pointer must be 16-byte aligned (TMA copies need 16 B).
 *
 * Execution: asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 * stream). C is valid once the stream has completed. Scratch memory is
 * allocated stream-ordered (cudaMallocAsync) unless the caller passes one in
 * bmm_opts.workspace. No entry point falls back to the CPU: failures are
 * returned as a status.
 *
 * Errors: sizes must be positive multiples of 64 (BMM_ERR_INVALID); null or
 * overlapping pointers give BMM_ERR_INVALID; misaligned pointers give
 * BMM_ERR_ALIGN. Device-side waits are bounded: a kernel whose wait times out
 * records it and returns early; bmm_stream_status() then reports
 * BMM_ERR_TIMEOUT and C is undefined.
 */
#ifndef BMM_H
#define BMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *bmm_stream_t; /* a cudaStream_t */

typedef enum {
    BMM_OK = 0,
    BMM_ERR_INVALID = 1,     /* bad size, null/overlapping pointer, bad option */
    BMM_ERR_ALIGN = 2,       /* pointer not 16-byte aligned */
    BMM_ERR_NOMEM = 3,       /* scratch allocation failed or caller workspace too small */
    BMM_ERR_CUDA = 4,        /* a CUDA runtime/driver call failed: bmm_last_cuda_error() */
    BMM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up; results undefined */
    BMM_ERR_UNSUPPORTED = 6  /* valid request this build/device does not support */
} bmm_status;

/* Base-case block product (Sec. 3.10 inner layer). */
typedef enum {
    BMM_PATH_AUTO = 0,    /* the fastest path for the shape on this device */
    BMM_PATH_TC_FP8 = 1,  /* tcgen05 tensor cores, bits -> e4m3, FP32 accumulate */
    BMM_PATH_TC_I8 = 2,   /* 8-bit integer tensor MMA: sm_103a has none, so requests
                             for it return BMM_ERR_UNSUPPORTED */
    BMM_PATH_POPC = 3,    /* CUDA cores: LOP3 AND-XOR / AND-OR over 32-bit words */
    BMM_PATH_TC_FP8_PAIR = 4, /* as TC_FP8, two SMs per 256 x 256 tile (cta_group::2) */
    BMM_PATH_TC_FP4_PAIR = 5  /* as TC_FP8_PAIR with bits -> e2m1 nibbles and the
                                 block-scaled 4-bit MMA (kind::mxf4, unit-free scale
                                 2^-6), FP32 accumulate: twice the k per MMA */
} bmm_path;

/* 2x2 recursion for the binary product. */
typedef enum {
    BMM_VARIANT_WINOGRAD = 0,     /* Strassen–Winograd, standard basis (Eqs. sw-*) */
    BMM_VARIANT_SELF_INVERSE = 1, /* alternative basis, self-inverse (Eqs. mb-*, Thm. 1) */
    BMM_VARIANT_CHAINING = 2      /* alternative basis, chaining (Eqs. ab-*, Thm. 2) */
} bmm_variant;

typedef struct {
    int32_t path;            /* bmm_path */
    int32_t strassen_depth;  /* -1 auto, 0 cubic, d > 0: d levels (binary product only) */
    int32_t variant;         /* bmm_variant, used when strassen_depth != 0 */
    int32_t serial_depth;    /* -1 auto; top levels run depth-first (Sec. 3.8) */
    void *workspace;         /* optional device scratch; NULL: stream-ordered allocation */
    uint64_t workspace_bytes;
    int32_t kernel_level;    /* 1: the innermost Strassen level runs inside the base-case
                                kernel (a level shifted into the inner layer, Sec. 3.15),
                                which forms each of the 7 products' operands from
                                the quadrants as it stages them and folds the products
                                into the C quadrants on chip (no leaf operands or
                                leaf products in HBM). Binary product on the CUDA-core
                                path (BMM_PATH_POPC) or the e2m1 tensor path
                                (BMM_PATH_TC_FP4_PAIR; k is then padded so that every
                                quadrant's k is a multiple of 512 bits), or AUTO where
                                it resolves to one of them; other paths give
                                BMM_ERR_UNSUPPORTED; a plan without Strassen levels
                                ignores it. 0 (default): every level in XOR passes */
} bmm_opts;

/* Fills opts with the defaults (auto path, auto depth, self-inverse variant). */
void bmm_opts_default(bmm_opts *opts);

/* C = A B over GF(2). A: m x k, B: k x n, C: m x n (Sec. 2.4, Eq. c-equals-ab). */
bmm_status bmm_gf2(const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m, int64_t k,
                   int64_t n, bmm_stream_t stream);

/* C = A B over the Boolean algebra (Sec. 1, Sec. 3.18). Always cubic: the
 * Boolean semiring has no additive inverse, so no Strassen recursion applies. */
bmm_status bmm_bool(const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m, int64_t k,
                    int64_t n, bmm_stream_t stream);

/* As above with explicit options (opts may be NULL for the defaults). */
bmm_status bmm_gf2_ex(const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m, int64_t k,
                      int64_t n, const bmm_opts *opts, bmm_stream_t stream);
bmm_status bmm_bool_ex(const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m, int64_t k,
                       int64_t n, const bmm_opts *opts, bmm_stream_t stream);

/* Scratch bytes the call with these arguments needs (op: 0 binary, 1 Boolean). */
bmm_status bmm_workspace_size(int32_t op, int64_t m, int64_t k, int64_t n, const bmm_opts *opts,
                              uint64_t *bytes);

/* What the planner resolves the options to for these sizes: the base-case
 * path, the Strassen depth and how many of its top levels run depth-first,
 * the variant, the number of base-case leaves (7^depth) and the scratch size.
 * kp is the k the base case runs with (the tensor paths pad k with zero
 * columns of A and zero rows of B so that every leaf's k is a multiple of
 * 128 bits); pass_bytes the bytes that the plan's streaming passes (the
 * transpose of B, the padded copy of A, every XOR pass of Secs. 3.8-3.11)
 * read and write in HBM, the base case not counted: with the leaves' MACs it
 * gives the Strassen path's bound (MACs at the tensor peak + pass_bytes at
 * the HBM bandwidth). */
typedef struct {
    int32_t path;
    int32_t strassen_depth;
    int32_t serial_depth;
    int32_t variant;
    int64_t leaves;
    uint64_t workspace_bytes;
    int32_t kernel_level;    /* 1: the innermost of the levels runs inside the base case */
    int64_t kp;
    uint64_t pass_bytes;
} bmm_plan_info;
bmm_status bmm_plan(int32_t op, int64_t m, int64_t k, int64_t n, const bmm_opts *opts,
                    bmm_plan_info *info);

/* Autotuner (Sec. 3.17: once memory capacity has fixed what it must, the few
 * remaining parameter choices are made by measurement). Times the candidate
 * base-case paths (tensor cores on SM pairs or single SMs where available,
 * CUDA cores) and, for the binary product (op 0), every Strassen depth 0..4
 * the sizes allow with leaves of at least 256 bits a side, and records the
 * fastest (path, depth) for (op, m, k, n) on the current device; products
 * whose options leave both path and depth to the library (bmm_gf2, bmm_bool,
 * or bmm_opts_default) then use it. The depth-first level count stays with
 * the planner's memory rule. Work is issued on `stream` with scratch of its
 * own (stream-ordered; operands are synthetic), and the call synchronises it.
 * A candidate is timed as a whole product when the product is small (its
 * operands and scratch use at most a quarter of free memory and the cubic
 * product would take under ~0.1 s); otherwise its leaf products are timed on
 * a leaf-shaped proxy of at most 16384 bits a side, scaled to the leaf count
 * and size, and its streaming passes are charged plan bytes at the measured
 * device copy bandwidth. flags: BMM_TUNE_MODEL forces the second way.
 * Errors: BMM_ERR_INVALID for bad op or sizes (as for the products),
 * BMM_ERR_NOMEM if scratch cannot be had. */
#define BMM_TUNE_MODEL 1u
typedef struct {
    bmm_opts best;     /* path and strassen_depth chosen; other fields default */
    double est_ms;     /* its measured (or modelled) time per product */
    int32_t measured;  /* 1: whole products timed; 0: leaf proxies + pass model */
    int32_t candidates;
} bmm_tune_result;
bmm_status bmm_autotune(int32_t op, int64_t m, int64_t k, int64_t n, uint32_t flags,
                        bmm_stream_t stream, bmm_tune_result *result);

/* Forgets every recorded choice (all devices). */
void bmm_autotune_clear(void);

/* Batched independent products C_i = A_i B_i, i < count, of individual sizes
 * (each a multiple of 64), all in one persistent launch of the base case.
 * op[i]: 0 binary, 1 Boolean (cubic; the batch may mix them). The pointer
 * and size arrays are HOST memory; the matrices are device memory as above.
 * These one-shot forms build a plan, run it on `stream` and wait for the
 * stream before freeing the plan, so they return with the products done. */
bmm_status bmm_batched(int32_t count, const int32_t *op, const uint64_t *const *A,
                       const uint64_t *const *B, uint64_t *const *C, const int64_t *m,
                       const int64_t *k, const int64_t *n, bmm_stream_t stream);
bmm_status bmm_gf2_batched(int32_t count, const uint64_t *const *A, const uint64_t *const *B,
                           uint64_t *const *C, const int64_t *m, const int64_t *k,
                           const int64_t *n, bmm_stream_t stream);
bmm_status bmm_bool_batched(int32_t count, const uint64_t *const *A, const uint64_t *const *B,
                            uint64_t *const *C, const int64_t *m, const int64_t *k,
                            const int64_t *n, bmm_stream_t stream);

/* Reusable batch plan. create decides, per problem, its base case (the
 * tensor cores or the CUDA cores) and its tile form (a last column tile of
 * N = 128 where at most 128 of its 256 columns lie inside n; k in operand
 * stages of 256 bits for e2m1, 128 for e4m3, so half a packed stage at the
 * end is not multiplied) from a cost model measured on the device: per
 * stage of k and per tile of each kernel, from synthetic batches timed the
 * first time a plan on that device and tensor path needs it (Sec. 3.17:
 * what memory does not fix is chosen by measurement; that first create
 * takes some tens of milliseconds longer). A binary problem gets the
 * Strassen depth a single product of its shape would get (Sec. 3.8: the
 * rule keeps leaves of at least 8192 bits, so depth 0 for any side below
 * 16384, or a tuned record for the shape); one with depth > 0 leaves the
 * batched launches and runs, after them, as its own Strassen product
 * (transpose, XOR passes, leaves) in scratch that the plan holds, sized for
 * the largest such problem; an AUTO entry of a plan on the device's
 * automatic tensor path leaves its path to that single-product planner too.
 * The rest run cubic in the batched launches. It then builds, on the current device, TMA maps
 * per problem, the tensor tile work list and its assignment to SM pairs
 * (longest first onto the least loaded pair, by model cost), the CUDA-core
 * tile list, and scratch for the transposed B's; it allocates device memory
 * and copies to it synchronously. run launches on `stream` the batched
 * transposes of every B (a TMA launch for those whose row pitches are even,
 * a load/store launch for the rest), row padding for tensor problems with
 * k/64 odd, one persistent tensor-core launch and, when some problem chose
 * the CUDA cores, one persistent CUDA-core launch, then the Strassen
 * problems one after another; it allocates nothing and
 * does not synchronise, and it reads the matrices named at create time, so new data
 * in the same buffers needs no new plan. Every run of a plan uses the plan's
 * own scratch (the transposed B's, padded A's, the Strassen problems'
 * scratch), so two runs of one plan must not overlap on the GPU (order them
 * on one stream, or make a plan per stream). destroy frees the plan; call it
 * only after the runs have completed. */
typedef struct bmm_batched_plan_s *bmm_batched_plan;
bmm_status bmm_batched_plan_create(int32_t count, const int32_t *op, const uint64_t *const *A,
                                   const uint64_t *const *B, uint64_t *const *C, const int64_t *m,
                                   const int64_t *k, const int64_t *n, bmm_batched_plan *plan);
/* As create, every problem on base-case `path` (bmm_path; AUTO as create,
 * the model choosing per problem; an explicit tensor path the device lacks:
 * BMM_ERR_UNSUPPORTED; tail tile forms still follow the model). */
bmm_status bmm_batched_plan_create_ex(int32_t count, const int32_t *op, const uint64_t *const *A,
                                      const uint64_t *const *B, uint64_t *const *C,
                                      const int64_t *m, const int64_t *k, const int64_t *n,
                                      int32_t path, bmm_batched_plan *plan);
bmm_status bmm_batched_plan_run(bmm_batched_plan plan, bmm_stream_t stream);
bmm_status bmm_batched_plan_destroy(bmm_batched_plan plan);
/* As create with the base case named per problem: paths[i] is
 * BMM_PATH_AUTO (the model chooses), BMM_PATH_POPC, or a tensor path; every
 * tensor entry must name the same tensor path (else BMM_ERR_INVALID), and
 * AUTO entries choose between it (or, if none is named, the device's
 * automatic tensor path) and the CUDA cores. paths is host memory. */
bmm_status bmm_batched_plan_create_paths(int32_t count, const int32_t *op,
                                         const uint64_t *const *A, const uint64_t *const *B,
                                         uint64_t *const *C, const int64_t *m, const int64_t *k,
                                         const int64_t *n, const int32_t *paths,
                                         bmm_batched_plan *plan);
/* The plan's tensor path (bmm_path, never AUTO) if any problem runs on the
 * tensor cores, else BMM_PATH_POPC. */
bmm_status bmm_batched_plan_path(bmm_batched_plan plan, int32_t *path);

/* What a plan decided for problem i (0 <= i < count). */
typedef struct {
    int32_t path;           /* base case: a tensor path or BMM_PATH_POPC */
    int32_t tile_m, tile_n; /* rows and columns of C per tile */
    int32_t tail_n;         /* columns the MMAs of its last column tile cover (tile_n or 128) */
    int32_t k_step;         /* bits of k per step the tiles run in (k is padded to whole steps) */
    int64_t k_steps;        /* steps of k per tile */
    int32_t strassen_depth; /* 0: cubic in the batched launches; > 0: its own
                               Strassen product (tile fields: its leaves';
                               est_us 0: the model covers the batched launches) */
    double est_us;          /* the model's time for all its tiles on one unit (CTA pair or CTA) */
} bmm_batched_choice;
bmm_status bmm_batched_plan_choice(bmm_batched_plan plan, int32_t i, bmm_batched_choice *out);

/* Totals of a plan. macs_needed is sum of m k n; macs_issued the MACs the
 * base case computes: tiles padded to whole tiles and k steps, and for a
 * Strassen problem 7^d leaves of (m k n) / 8^d. est_ms covers the batched
 * launches only. */
typedef struct {
    int32_t problems, tensor_problems, popc_problems;
    int32_t tensor_path;          /* the tensor path the plan uses for tensor problems */
    int64_t tensor_tiles, tensor_tiles_n128, popc_tiles;
    double macs_needed, macs_issued;
    double est_ms;                /* the model's base-case time of one run */
    int32_t model_measured;       /* 1: the model was measured on this device */
    int32_t strassen_problems;    /* problems run as their own Strassen products
                                     (counted in tensor_ or popc_problems too) */
} bmm_batched_stats;
bmm_status bmm_batched_plan_stats(bmm_batched_plan plan, bmm_batched_stats *out);

/* The batched cost model for a tensor path (AUTO: the device's automatic
 * one; BMM_PATH_POPC: the CUDA-core part only) on the current device,
 * measured now if it was not yet (synchronises the device). Times are
 * nanoseconds on one unit of the launch. */
typedef struct {
    int32_t path;
    int32_t measured;
    int32_t tensor_units;          /* CTA pairs (or CTAs) of the tensor launch */
    double tensor_stage_ns;        /* per operand stage of an N = 256 tile */
    double tensor_stage_n128_ns;   /* per operand stage of an N = 128 tile */
    double tensor_tile_ns;         /* per tile */
    int32_t popc_units;            /* CTAs of the CUDA-core launch */
    double popc_stage_ns;          /* per 256-bit stage of k of a 128 x 128 tile */
    double popc_tile_ns;           /* per tile */
} bmm_batched_model_info;
bmm_status bmm_batched_model(int32_t path, bmm_batched_model_info *out);

/* ---- operands in host memory: the host layer (Secs. 3.12-3.14, Alg. 3) ---
 *
 * C = A B with A, B and C in host memory (same packed row-major layout as on
 * the device), for products whose operands need not fit the device. Binary
 * product: the host expands `host_depth` Strassen levels into 7^host_depth
 * sub-instances (each block combination of A and B that the combined masks
 * of those levels select, Eq. igen), the device solves each with its own
 * plan, and the host adds every solution into the C blocks it belongs to
 * (Eq. iagg); host threads generate and aggregate while the device computes
 * and the host link copies, all double-buffered. Boolean product (no
 * additive inverse), or host_depth 0: C is computed in blocks that fit the
 * device, streaming row panels of A and column panels of B from the
 * caller's arrays and C blocks back into C.
 *
 * Pinned host memory (cudaHostAlloc / cudaHostRegister) lets the copies run
 * asynchronously; pageable memory works with staged copies. The calls block
 * until C is complete in host memory; `stream` carries the device work.
 * Errors: as bmm_gf2 (sizes, alignment, overlap of C with A or B);
 * BMM_ERR_NOMEM if no blocking fits `device_bytes` or host staging cannot
 * be pinned; host_depth > 0 for the Boolean product is BMM_ERR_INVALID; a
 * host_depth whose 64 * 2^host_depth does not divide m, k and n is
 * BMM_ERR_UNSUPPORTED. */
typedef struct {
    bmm_opts device;        /* options of each product on the device (path, Strassen
                               depth, variant; also the host levels' variant);
                               the workspace fields are ignored */
    uint64_t device_bytes;  /* device memory the call may use; 0: 80 % of free memory */
    int32_t host_depth;     /* binary product: Strassen levels on the host; -1: none
                               if the whole product fits, else the fewest that make a
                               sub-instance fit, else blocks of C; 0: never */
    int32_t threads;        /* host threads for generation and aggregation; 0: all */
} bmm_host_opts;

void bmm_host_opts_default(bmm_host_opts *opts);

/* What a host-memory product with these arguments does (no device needed
 * when opts->device_bytes is non-zero). */
typedef struct {
    int32_t host_depth;             /* Strassen levels run on the host */
    int64_t sub_m, sub_k, sub_n;    /* shape of one device product */
    int64_t count;                  /* device products */
    uint64_t device_bytes;          /* device memory the call needs (estimate) */
    uint64_t staging_bytes;         /* pinned host staging it allocates */
    uint64_t upload_bytes, download_bytes;  /* host <-> device traffic */
} bmm_host_plan_info;

bmm_status bmm_host_plan(int32_t op, int64_t m, int64_t k, int64_t n, const bmm_host_opts *opts,
                         bmm_host_plan_info *info);
bmm_status bmm_gf2_host(const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m, int64_t k,
                        int64_t n, const bmm_host_opts *opts, bmm_stream_t stream);
/* The host-memory products keep their pinned staging and device buffers
 * between calls on a device (allocating them is a large share of one call);
 * calls on one device are serialised. This frees them on every device. */
void bmm_host_release(void);
bmm_status bmm_bool_host(const uint64_t *A, const uint64_t *B, uint64_t *C, int64_t m, int64_t k,
                         int64_t n, const bmm_host_opts *opts, bmm_stream_t stream);

/* ---- the steps of the path, exported for tests and experiments ---------- */

/* Bit transpose: Xt (cols x rows) = X^T (X is rows x cols). The paper
 * transposes the right operand so both operands run along k (Sec. 3.5).
 * Tiles of 512 x 512 bits move through shared memory by TMA where both row
 * pitches are even and the matrix has a whole tile a side, else by loads and
 * stores. */
bmm_status bmm_transpose(const uint64_t *X, uint64_t *Xt, int64_t rows, int64_t cols,
                         bmm_stream_t stream);

/* Base-case product in the "NT" form: C (m x n) = A (m x k) times the
 * transpose of Bt (n x k), over GF(2) (op 0) or Boolean (op 1), on one path
 * (Sec. 3.10; Sec. 3.18). `path` must be explicit (not BMM_PATH_AUTO); the
 * tensor-core paths need k % 128 == 0 and an sm_103 device, else
 * BMM_ERR_UNSUPPORTED. */
bmm_status bmm_base_product(int32_t op, int32_t path, const uint64_t *A, const uint64_t *Bt,
                            uint64_t *C, int64_t m, int64_t k, int64_t n, bmm_stream_t stream);

/* In-place basis change of X (rows x cols) over `depth` levels of 2x2 blocks:
 * inverse = 0 applies phi (= psi), inverse = 1 applies chi
 * (Eqs. mb-fwdbasisrecurrence / mb-revbasisrecurrence for the self-inverse
 * variant, ab-fwdbasisrecurrence / ab-revbasisrecurrence for chaining; the
 * identity for Strassen–Winograd). rows, cols divisible by 64 * 2^depth. */
bmm_status bmm_basis_change(int32_t variant, int32_t inverse, uint64_t *X, int64_t rows,
                            int64_t cols, int32_t depth, bmm_stream_t stream);

/* ---- fixed-scratch product ------------------------------------------------ */

/* Bytes of the device array bmm_product_noalloc uses as scratch. */
#define BMM_NOALLOC_SCRATCH_BYTES (8u << 20)

/* C = A B, cubic, over GF(2) (op 0) or the Boolean algebra (op 1), with the
 * same layouts, alignment and argument checks as bmm_gf2 / bmm_bool, but
 * without allocating any memory. The paper has no counterpart: this entry
 * point is for callers that cannot allocate device memory while they run,
 * such as applications whose framework reserves nearly all of HBM in its
 * own pool (a library allocation could fail or fragment it), latency-bound
 * loops in which an allocation might synchronise the device, and
 * deployments that fix all device memory when the library is loaded.
 *
 * Its only scratch, the transpose of B (k x n bits), lives in one static
 * device array of BMM_NOALLOC_SCRATCH_BYTES bytes that every GPU loading
 * this library keeps until the process exits. Sizes with k*n/8 larger than
 * that return BMM_ERR_NOMEM. Every call looks the array's device address up
 * (cudaGetSymbolAddress, with the calling device current); the first call
 * on a device also loads this library's device code there, so make that
 * first call before any stream capture begins. All calls share the one
 * array and it keeps the last call's contents; each call writes every word
 * it later reads, so nothing needs clearing, but calls whose work overlaps
 * on the GPU (for example on two streams at once) race on it and must be
 * serialised by the caller. With tracing on (bmm_trace_enable), launches
 * also create CUDA events. */
bmm_status bmm_product_noalloc(int32_t op, const uint64_t *A, const uint64_t *B, uint64_t *C,
                               int64_t m, int64_t k, int64_t n, bmm_stream_t stream);

/* ---- tracing -------------------------------------------------------------- */

/* Phases that tracing times separately. */
typedef enum {
    BMM_PHASE_BASE = 0,      /* base-case block products (tensor or CUDA-core) */
    BMM_PHASE_XOR = 1,       /* expand / compress / combine / fold / basis-change passes */
    BMM_PHASE_TRANSPOSE = 2, /* bit transposes */
    BMM_PHASE_COUNT = 3
} bmm_phase;

/* Starts (enable = 1) or stops (0) recording a CUDA event pair around every
 * kernel launch, on the stream the kernel is launched on. Starting clears
 * what was recorded before. Process-wide; not for concurrent callers. */
void bmm_trace_enable(int32_t enable);

/* Synchronises the recorded events and returns, for one phase, how many
 * kernels were launched and their summed device time in milliseconds. */
bmm_status bmm_trace_read(int32_t phase, int64_t *launches, double *milliseconds);

/* Kernels launched by this library in this process so far (always counted). */
int64_t bmm_launch_count(void);

/* ---- status ------------------------------------------------------------- */

/* Synchronises `stream` and reports device-side failures recorded since the
 * last call (BMM_ERR_TIMEOUT after a bounded wait gave up), else BMM_OK. */
bmm_status bmm_stream_status(bmm_stream_t stream);

/* Launches one thread that waits, with the same bounded wait the kernels
 * use, on a barrier nothing ever arrives on, for limit_ns nanoseconds (at
 * most 10 s). The wait gives up, records the timeout and the kernel returns;
 * the next bmm_stream_status() reports BMM_ERR_TIMEOUT and clears it. A test
 * of the failure path that faults and hangs nothing. */
bmm_status bmm_selftest_wait_timeout(int64_t limit_ns, bmm_stream_t stream);

/* Name of a status code (static string). */
const char *bmm_status_string(bmm_status status);

/* The cudaError_t behind the last BMM_ERR_CUDA on this thread. */
int32_t bmm_last_cuda_error(void);

/* 1 if the current device can run the tensor-core paths (sm_103), else 0. */
int32_t bmm_device_supported(void);

#ifdef __cplusplus
}
#endif

#endif /* BMM_H */
