// Tensor-core base-case block product for sm_103a (Sec. 3.10 inner layer,
// re-designed for tcgen05): C = A * Bt^T over GF(2) or the Boolean algebra,
// A (m x k) and Bt (n x k) packed along k.
//
// The bit product is an integer dot product of 0/1 vectors: count_ij =
// sum_k A_ik Bt_jk. GF(2) takes count mod 2, Boolean takes count > 0. The
// tensor cores compute the counts exactly: bits are expanded to e4m3 bytes
// (value 2^-6, products 2^-12, FP32 accumulation exact while counts stay
// below 2^23). sm_103a has no 8-bit integer MMA (ptxas rejects
// tcgen05.mma kind::i8 for this target), so FP8 is the exact tensor format.
//
// Persistent kernel, one CTA per SM, warp-specialised (18 warps):
//   warp 16     TMA producer: packed tiles of 128 rows of A and 256 rows of
//               Bt (128 in a pair, below), 256 bits of k each (32-byte rows),
//               into a PSTAGES-deep shared ring (cp.async.bulk.tensor,
//               mbarrier complete_tx). Each packed stage feeds two operand
//               stages of 128 bits.
//   Bt expansion (8 warps; 4 in a pair): each packed 32-bit word becomes
//               32 bytes of the K-major, 128-byte-swizzled canonical UMMA
//               layout; a warp expands 4 whole rows of a packed stage at a
//               time.
//   A expansion (4 warps, one per TMEM lane quarter): one row per thread,
//               every packed stage: 256 bits -> 256 e4m3 bytes (both operand
//               stages) written straight into TMEM with one tcgen05.st.
//   epilogue (4 warps; 8 in a pair, two per lane quarter splitting the
//               columns): tcgen05.ld 32 lanes x 32 columns at a time, parity
//               or non-zero test, bits packed in registers with a shallow
//               tree (one row per thread) and stored as 64-bit words.
//   warp 17     MMA issuer: per packed stage, 2 x 4 tcgen05.mma (M=128,
//               N=256, K=32; A from TMEM, B from shared memory) into the TMEM
//               accumulator and one commit that frees the operand slot.
// SM pairs (PAIR): two CTAs of a cluster on two SMs share one 256 x 256 tile
// through tcgen05.mma.cta_group::2 (M=256). Each CTA expands its own 128 rows
// of A into its TMEM and its own 128 of the tile's 256 Bt rows into its
// shared memory; the even CTA issues the MMAs, which read both CTAs'
// operands and accumulate each CTA's 128 rows in its own TMEM. The gating
// barriers (operand stage full, accumulator empty) live in the even CTA and
// both CTAs' producers and epilogues arrive there; the commits that free an
// operand stage or publish the accumulator are multicast to both CTAs.
// The two operand stages a packed stage fills form one slot with one "full"
// barrier (every producer arrives) and one "empty" barrier (one commit).
// Every producer handles every packed stage in order, so the MMA issuer's
// wait on a slot covers the slots before it too: with four or more slots it
// checks one barrier per two packed stages (a check costs ~190 cycles of
// latency, even when the phase is already complete). TMEM stores share the tensor pipe's issue path
// with the MMAs, so A goes in with one wide store per packed stage. Keeping
// A in TMEM means shared memory carries only Bt (written once, read once by
// the tensor core). Long k is flushed from TMEM in chunks of `kchunk` stages
// (the epilogue folds parities / ORs across chunks).
//
// Within every 32-element group of k the expansion permutes k (byte t of
// output word j holds bit 8t + j of the packed word); A and Bt use the same
// permutation, so the contraction is unchanged.
//
// e2m1 form (FP4): every bit becomes a 4-bit e2m1 value under a uniform
// block scale, twice the k per MMA (kind::mxf4); an operand stage then holds
// 256 bits of k and a packed stage 512.
//
// Batched form (BATCHED): each unit walks its own list of work items, one
// tile of one problem each (per-problem TMA maps); a tile may run N = 128
// MMAs (a tail with at most 128 columns inside n) and may end in half a
// packed stage. Uniform form: the tiles of `count` equal leaves.
//
// Every mbarrier wait is bounded (wall clock, ~2 s). A wait that gives up
// records BMM device error DEVERR_TIMEOUT and makes its role stop; the CTA
// then drains its own in-flight copies and MMAs (again bounded), frees TMEM
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "plan.h"
#include "tc_batched.h"

namespace bmm {
namespace {

constexpr int BM = TC_TILE_M;    // rows of C per tile (UMMA M, TMEM lanes)
constexpr int BN = TC_TILE_N;    // columns of C per tile (UMMA N)
constexpr int SUB = 2;           // operand stages per packed stage
constexpr int KS_MIN = 128;      // k granularity of the operands (both formats)
// 18 warps: an SM sub-partition (16 K registers) holds at most five of
// them, which leaves 96 registers per thread (the A expansion keeps 64
// output words live for one wide TMEM store). Warps 0..15 are split between
// Bt expansion, A expansion (one warp per TMEM lane quarter) and the
// epilogue as the layout below gives; then the TMA and MMA warps.
constexpr int AEXP_WARPS = 4;
constexpr int TMA_WARP = 16;
constexpr int MMA_WARP = 17;
constexpr int THREADS = 18 * 32;
// Tile raster: groups of GROUP_M row-tiles, column by column within a
// group. Each Bt tile is read from DRAM once per group while the group's
// rows of A (32 x 256 rows x k bits: 32 MiB at k = 32768 for pairs) stay in
// L2 (measured: 64 row-tiles no longer fit and A is re-read).
constexpr int GROUP_M = 32;

// An operand stage is 128 bytes of expanded operand per row in both
// formats: 128 k as e4m3 bytes, or 256 k as e2m1 nibbles (two per byte).
// One tcgen05.mma consumes 32 bytes of k per row (K = 32 e4m3, K = 64 e2m1),
// so the descriptors and TMEM columns advance the same way in both.
constexpr int ACC_COL = 0;               // accumulator: TMEM columns [0, BN)
constexpr int A_COL = BN;                // A ring: columns [BN, BN + ESTAGES * A_STAGE_COLS)
constexpr int A_STAGE_COLS = 32;         // 128 bytes of a row = 32 columns of 32 bits
constexpr int A_MMA_COLS = 8;            // 32 bytes of a row per MMA
constexpr int MMAS_PER_STAGE = 4;
constexpr int SF_COL = 448;              // e2m1: block scales, columns [448, 512)
constexpr int SF_COLS = 64;
constexpr int TMEM_COLS = 512;

// Per-CTA shapes and shared-memory layout. A CTA always owns 128 rows of C
// (its 128 TMEM lanes) and the matching 128 rows of A. A CTA on its own
// (cta_group::1) also expands all 256 Bt rows of its 128 x 256 tile. In a
// pair (a cluster of two CTAs on two SMs, cta_group::2, one 256 x 256 tile)
// each CTA expands only its half of the Bt rows, and the pair's MMAs read
// both halves: per SM, half the shared-memory traffic and a third less
// expansion work for the same number of MACs.
// LEVEL: the in-kernel Strassen level (below). Its packed stages hold up to
// six quadrant tiles (the A quadrants one product combines, then its Bt
// quadrants; at most six for every variant's products), so the ring is two
// packed stages deep.
template <bool PAIR, bool FP4, bool LEVEL = false>
struct Lay {
    static constexpr int KS = FP4 ? 256 : 128;  // k (bits) per operand stage
    static constexpr int KP = SUB * KS;         // k (bits) per packed (TMA) stage
    static constexpr int MMA_K = FP4 ? 64 : 32; // k per tcgen05.mma
    // ring depths: packed stages (shared) and operand stages (Bt in shared,
    // A in TMEM); a pair's smaller operand stages leave room for deeper rings.
    // The e2m1 form gives up two operand stages of TMEM to the block scales.
    static constexpr int PSTAGES = LEVEL ? 2 : PAIR ? 6 : 4;
    static constexpr int ESTAGES = PAIR ? (FP4 ? 6 : 8) : 4;
    // operand slots: the two operand stages one packed stage fills
    static constexpr int OSLOTS = ESTAGES / SUB;
    // packed stages the MMA issuer covers with one wait (needs more slots
    // than that, or the producers cannot run ahead)
    static constexpr int WAITG = OSLOTS >= 4 ? 2 : 1;
    // barriers: full_p[P], empty_p[P], full_o[O], empty_o[O], acc_full, acc_empty, drain
    static constexpr int NBARS = 2 * PSTAGES + 2 * OSLOTS + 3;
    // warps: Bt expansion [0, BEXP_WARPS), A expansion [AEXP_WARP0, +4),
    // epilogue [EPI_WARP0, TMA_WARP). A CTA alone has twice the Bt rows, a
    // pair's MMA issuer gains most from a short accumulator drain.
    static constexpr int BEXP_WARPS = PAIR ? 4 : 8;
    static constexpr int AEXP_WARP0 = BEXP_WARPS;
    static constexpr int EPI_WARP0 = AEXP_WARP0 + AEXP_WARPS;
    static constexpr int EPI_WARPS = TMA_WARP - EPI_WARP0;
    static_assert(AEXP_WARP0 % 4 == 0 && EPI_WARP0 % 4 == 0 && EPI_WARPS % 4 == 0,
                  "warp % 4 is the TMEM lane quarter");
    static constexpr int TILE_M = PAIR ? 2 * BM : BM;  // rows of C per tile
    static constexpr int BROWS = PAIR ? BN / 2 : BN;   // Bt rows held by one CTA
    static constexpr int PA_BYTES = BM * KP / 8;       // packed A per packed stage
    static constexpr int PB_BYTES = BROWS * KP / 8;    // packed Bt per packed stage
    static constexpr int EB_BYTES = BROWS * 128;       // expanded Bt per operand stage
    static constexpr int QTILES = 6;                   // LEVEL: quadrant tiles per stage
    static constexpr int OFF_EB = 0;
    static constexpr int OFF_PA = OFF_EB + ESTAGES * EB_BYTES;
    static constexpr int OFF_PB = OFF_PA + PSTAGES * PA_BYTES;  // (not LEVEL)
    static constexpr int PSTAGE_BYTES = QTILES * PA_BYTES;      // LEVEL: one packed stage
    // LEVEL: every epilogue thread's words of the four C quadrants (4 x 4
    // words, lane-interleaved), in shared memory beside the registers the
    // accumulator loads need
    static constexpr int QOUT_BYTES = LEVEL ? EPI_WARPS * 32 * 16 * 4 : 0;
    static constexpr int OFF_QOUT = LEVEL ? OFF_PA + PSTAGES * PSTAGE_BYTES : 0;
    // batched: two work items per epilogue warp, fetched a tile ahead
    static constexpr int OFF_ITEMS = LEVEL ? OFF_QOUT + QOUT_BYTES : OFF_PB + PSTAGES * PB_BYTES;
    static constexpr int ITEM_BYTES = 48;
    static constexpr int OFF_BAR = OFF_ITEMS + EPI_WARPS * 2 * ITEM_BYTES;
    static constexpr int OFF_TMEM_SLOT = OFF_BAR + NBARS * 8;
    static constexpr int SMEM_BYTES = OFF_TMEM_SLOT + 16 + 1024;  // + alignment slack
    static_assert(EB_BYTES % 1024 == 0, "swizzle atoms stay 1024-byte aligned");
    static_assert(A_COL + ESTAGES * A_STAGE_COLS <= (FP4 ? SF_COL : TMEM_COLS), "TMEM budget");
    static_assert(SF_COL + SF_COLS <= TMEM_COLS, "TMEM budget");
    static_assert(KS / MMA_K == MMAS_PER_STAGE && MMA_K * (FP4 ? 4 : 8) == 32 * A_MMA_COLS,
                  "an MMA reads 32 bytes of k per row");
    static_assert(ESTAGES % SUB == 0, "a packed stage's operand stages are adjacent in TMEM");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
    static_assert(!LEVEL || (PAIR && PA_BYTES == PB_BYTES), "LEVEL: equal quadrant tiles");
};

constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity. Returns false
// (after recording the timeout) if it did not complete within WAIT_NS.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, uint32_t* err,
                                            uint64_t limit_ns = WAIT_NS) {
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; i++) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255u) == 0 && globaltimer() - t0 > limit_ns) {
            atomicOr(err, DEVERR_TIMEOUT);
            return false;
        }
    }
}

// Arrive on the barrier at the same shared-memory offset in CTA `cta` of
// the cluster. What the waiter goes on to use is this CTA's own shared
// memory and TMEM, read by the pair's tensor cores; the writer orders it
// with fence.proxy.async.shared::cta or tcgen05.fence before arriving, so a
// CTA-scope arrive is enough (a cluster-scope release costs a memory barrier).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar, uint32_t cta) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(bar), "r"(cta));
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of both CTAs of the cluster (no thread may have exited).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Self-test of the bounded wait: one thread waits on a barrier that nothing
// arrives on, gives up after limit_ns, records the timeout and returns.
__global__ void wait_selftest_kernel(uint32_t* err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    fence_barrier_init();
    mbar_wait_slow(b, 0, err, limit_ns);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* err) {
    if (mbar_try(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, err);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzled canonical layout: each row's 128 bytes of k sit at row * 128,
// 8-row groups form 1024-byte atoms (SBO = 1024 between them), and within an
// atom the 16-byte chunk c of row r is stored at chunk c ^ (r % 8). The
// start address may point k bytes into the first row (k < 128): the swizzle
// is applied to absolute address bits, so atoms must be 1024-byte aligned.
// Adding 2 to the descriptor advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // LBO: unused for swizzled K-major, 1 by convention
    d |= (uint64_t)(1024u >> 4) << 32;   // SBO: 8-row atom stride
    d |= (uint64_t)1 << 46;              // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;              // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor for kind::f8f6f4: D format (1 = F32), A and B
// format 0 (E4M3), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int M, int N = BN>
__host__ __device__ constexpr uint32_t instr_desc(uint32_t dfmt) {
    return (dfmt << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor for kind::mxf4 (block-scaled e2m1, FP32
// accumulate): A and B format 1 (E2M1) at bits 7 and 10, both K-major,
// N >> 3 at bit 17, scale format 1 (UE8M0) at bit 23, M >> 4 at bit 24;
// scale-factor data ids 0 and K = 64 (bit 31 clear).
template <int M, int N = BN>
__host__ __device__ constexpr uint32_t instr_desc_mxf4() {
    return (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (1u << 23) |
           ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) += A (TMEM) x B (shared, descriptor). PAIR: cta_group::2, issued
// by the even CTA of the pair; A, B and D are the two CTAs' halves at the
// same TMEM / shared-memory addresses.
template <bool PAIR>
__device__ __forceinline__ void mma_f8_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t db,
                                          uint32_t idesc, uint32_t accumulate) {
    if (PAIR)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
            "r"(tmem_a), "l"(db), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
            "r"(tmem_a), "l"(db), "r"(idesc), "r"(accumulate)
            : "memory");
}

// As mma_f8_ta for e2m1 operands with block scales: every 32 k of a row of
// A (B) is scaled by the UE8M0 byte the tensor core reads from TMEM at
// tmem_sfa (tmem_sfb); here every scale byte holds the same value.
template <bool PAIR>
__device__ __forceinline__ void mma_f4_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t db,
                                          uint32_t idesc, uint32_t tmem_sfa, uint32_t tmem_sfb,
                                          uint32_t accumulate) {
    if (PAIR)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X"
            " [%0], [%1], %2, %3, [%4], [%5], p;\n\t}" ::"r"(tmem_d),
            "r"(tmem_a), "l"(db), "r"(idesc), "r"(tmem_sfa), "r"(tmem_sfb), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X"
            " [%0], [%1], %2, %3, [%4], [%5], p;\n\t}" ::"r"(tmem_d),
            "r"(tmem_a), "l"(db), "r"(idesc), "r"(tmem_sfa), "r"(tmem_sfb), "r"(accumulate)
            : "memory");
}

// Arrive on `bar` once every MMA this thread issued so far has completed.
// PAIR: on the barrier at the same offset in each CTA of `mask`.
template <bool PAIR>
__device__ __forceinline__ void mma_commit(uint32_t bar, uint16_t mask = 3) {
    if (PAIR)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
            " [%0], %1;" ::"r"(bar),
            "h"(mask)
            : "memory");
    else
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
            : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t slot) {
    if (PAIR) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc(uint32_t tmem) {
    if (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
}

// 32 lanes x 64 columns (one row per thread), then wait for the load.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
        "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
        "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, "
        "[%64];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]),
          "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]),
          "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]),
          "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]),
          "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]),
          "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 lanes x 64 columns: one row per thread, 64 consecutive 32-bit columns
// (both operand stages of a packed stage in one instruction; TMEM stores
// share the tensor pipe's issue path with the MMAs, so fewer, wider ones).
__device__ __forceinline__ void tmem_st64(uint32_t taddr, const uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, "
        "%33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, "
        "%49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63, %64};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31]), "r"(v[32]), "r"(v[33]), "r"(v[34]), "r"(v[35]),
        "r"(v[36]), "r"(v[37]), "r"(v[38]), "r"(v[39]), "r"(v[40]), "r"(v[41]), "r"(v[42]),
        "r"(v[43]), "r"(v[44]), "r"(v[45]), "r"(v[46]), "r"(v[47]), "r"(v[48]), "r"(v[49]),
        "r"(v[50]), "r"(v[51]), "r"(v[52]), "r"(v[53]), "r"(v[54]), "r"(v[55]), "r"(v[56]),
        "r"(v[57]), "r"(v[58]), "r"(v[59]), "r"(v[60]), "r"(v[61]), "r"(v[62]), "r"(v[63])
        : "memory");
}

// ---------------------------------------------------------------- expansion
// Packed word x holds 32 consecutive k of one row. Output word j (j = 0..7)
// gets bit (8t + j) of x in byte t, moved to bit 3 of that byte (e4m3 0x08 =
// 2^-6). The moves are multiplications by powers of two (left) or high
// halves of them (right) with factors the compiler cannot see, so they run
// on the FMA pipe and leave the integer pipe the masks alone.
struct Spread {
    uint32_t f[8];  // f[j]: 2^(3-j) for j <= 3 (low product), 2^(35-j) for j > 3 (high)
    uint32_t g[4];  // spread4: 2, 1 (low products), 2^31, 2^30 (high)
};

__device__ __forceinline__ void spread8(uint32_t x, const Spread& sp, uint32_t* y) {
    constexpr uint32_t mask = 0x08080808u;
    y[0] = (x * sp.f[0]) & mask;
    y[1] = (x * sp.f[1]) & mask;
    y[2] = (x * sp.f[2]) & mask;
    y[3] = x & mask;
    y[4] = __umulhi(x, sp.f[4]) & mask;
    y[5] = __umulhi(x, sp.f[5]) & mask;
    y[6] = __umulhi(x, sp.f[6]) & mask;
    y[7] = __umulhi(x, sp.f[7]) & mask;
}

// e2m1 form: output word j (j = 0..3) gets bit (4t + j) of x in nibble t,
// moved to bit 1 of the nibble (e2m1 0x2 = 1.0, scaled by 2^-6 at the MMA,
// so products are 2^-12 as in the e4m3 form).
__device__ __forceinline__ void spread4(uint32_t x, const Spread& sp, uint32_t* y) {
    constexpr uint32_t mask = 0x22222222u;
    y[0] = (x * sp.g[0]) & mask;
    y[1] = x & mask;
    y[2] = __umulhi(x, sp.g[2]) & mask;
    y[3] = __umulhi(x, sp.g[3]) & mask;
}

// UE8M0 block scale 2^-6 (biased exponent 121) in every byte.
constexpr uint32_t SCALE_WORD = 0x79797979u;

// 32 result bits of one accumulator row slice -> one word, bit j from v[j].
// GF(2): v[j] = count * 2^-12 exactly; adding 2^11 puts count's LSB in bit 0.
// Boolean: any non-zero count. Each bit goes in with one funnel shift (the
// word shifts right by one and takes the bit at the top), in four
// independent chains of eight that are merged at the end.
template <int OP>
__device__ __forceinline__ uint32_t pack_bits(const uint32_t* v) {
    uint32_t c[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 8; j++)
#pragma unroll
        for (int g = 0; g < 4; g++) {
            const uint32_t x = v[8 * g + j];
            const uint32_t bit = OP == OP_GF2 ? __float_as_uint(__uint_as_float(x) + 2048.0f)
                                              : min(x, 1u);  // fp32 counts are >= 0
            c[g] = __funnelshift_r(c[g], bit, 1);  // bit 0 of `bit` enters at bit 31
        }
    // chain g holds bits 8g..8g+7 in its top byte
    return (c[0] >> 24) | (c[1] >> 16) | (c[2] >> 8) | c[3];
}

struct TileCoord {
    int leaf, tm, tn;
};

__device__ __forceinline__ TileCoord tile_of(int t, int tiles_m, int tiles_n) {
    const int per_leaf = tiles_m * tiles_n;
    TileCoord c;
    c.leaf = t / per_leaf;
    int r = t - c.leaf * per_leaf;
    const int group = GROUP_M * tiles_n;
    const int g = r / group;
    const int first_m = g * GROUP_M;
    const int gm = min(GROUP_M, tiles_m - first_m);
    const int in = r - g * group;
    c.tm = first_m + in % gm;
    c.tn = in / gm;
    return c;
}

struct Params {
    // uniform form: one shape, `count` leaves side by side
    uint64_t* C;
    int64_t ldc, strideC;
    int m, n, nks, op;
    int tiles_m, tiles_n, total_tiles;
    // batched form: per-problem descriptors and per-CTA work lists
    const TcProblem* probs;
    const TcWorkItem* items;
    const int32_t* cta_ptr;
    int kchunk;  // stages per flush (both forms)
    uint32_t* err;
    Spread sp;
    // LEVEL: each leaf is a block of 2m x 2k times 2k x 2n bits whose seven
    // quadrant products run here (m, n, nks: one quadrant product); qkw:
    // words of k per quadrant; nibble h of xi4 / eta4: the A / B quadrants
    // product h combines; bits 7q..7q+6 of zeta7: the products C quadrant q
    // sums.
    uint32_t xi4, eta4, zeta7;
    int qkw;
};

// Everything a role needs about one output tile.
struct Tile {
    const CUtensorMap* ma;
    const CUtensorMap* mb;
    uint64_t* C;  // leaf's C
    int64_t ldc;
    int m, n, nks, op, tm, tn, leaf;
    int n128;     // batched: N = 128 MMAs (columns 128.. of the tile lie past n)
};

// Scheduling unit: a CTA, or a CTA pair (consecutive blockIdx.x, one cluster).
template <bool PAIR>
__device__ __forceinline__ int unit_id() {
    return PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
}
template <bool PAIR>
__device__ __forceinline__ int unit_count() {
    return PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
}

template <bool BATCHED, bool PAIR>
__device__ __forceinline__ int tile_count(const Params& p) {
    const int u = unit_id<PAIR>();
    if (BATCHED) return p.cta_ptr[u + 1] - p.cta_ptr[u];
    int c = 0;
    for (int t = u; t < p.total_tiles; t += unit_count<PAIR>()) c++;
    return c;
}

// A batched tile from its work item.
__device__ __forceinline__ Tile tile_of_item(const Params& p, const TcWorkItem& w) {
    Tile t;
    const TcProblem* d = p.probs + w.prob;
    t.ma = &d->mapA;
    t.mb = &d->mapB;
    t.C = w.C;
    t.ldc = w.ldc;
    t.m = w.m;
    t.n = w.n;
    t.nks = w.nks;
    t.op = w.op;
    t.tm = w.tm;
    t.tn = w.tn;
    t.leaf = 0;
    t.n128 = w.n128;
    return t;
}

// 16 bytes global -> shared, asynchronous (cp.async; wait with cp_async_wait_all).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// items: batched, this unit's slice of the work list (read once per kernel,
// so that fetching a tile's item is one load, not two dependent ones).
template <bool BATCHED, bool PAIR>
__device__ __forceinline__ Tile tile_get(const Params& p, const TcWorkItem* items, int idx,
                                         const CUtensorMap* tmA, const CUtensorMap* tmB) {
    Tile t;
    if (BATCHED) {
        const TcWorkItem w = items[idx];
        const TcProblem* d = p.probs + w.prob;
        t.ma = &d->mapA;
        t.mb = &d->mapB;
        t.C = w.C;
        t.ldc = w.ldc;
        t.m = w.m;
        t.n = w.n;
        t.nks = w.nks;
        t.op = w.op;
        t.tm = w.tm;
        t.tn = w.tn;
        t.leaf = 0;
        t.n128 = w.n128;
    } else {
        const TileCoord c =
            tile_of(unit_id<PAIR>() + idx * unit_count<PAIR>(), p.tiles_m, p.tiles_n);
        t.ma = tmA;
        t.mb = tmB;
        t.C = p.C + (int64_t)c.leaf * p.strideC;
        t.ldc = p.ldc;
        t.m = p.m;
        t.n = p.n;
        t.nks = p.nks;
        t.op = p.op;
        t.tm = c.tm;
        t.tn = c.tn;
        t.leaf = c.leaf;
        t.n128 = 0;
    }
    return t;
}

// What the MMA issuer needs of a tile: its k stages, and (batched) N = 128.
struct TileK {
    int nks, n128;
};
template <bool BATCHED>
__device__ __forceinline__ TileK tile_k(const Params& p, const TcWorkItem* items, int idx) {
    if (BATCHED) {
        const TcWorkItem* w = items + idx;
        return {w->nks, w->n128};
    }
    return {p.nks, 0};
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// The in-kernel Strassen level (LEVEL; a level shifted from the expanding
// and compressing passes into the inner layer, Sec. 3.15), binary product
// only: every leaf of the launch is a block of 2m x 2k times 2k x 2n bits,
// and a CTA pair takes one 256 x 256 tile position of the quadrant-sized
// product and runs the block's seven quadrant products there, one after the
// other. For product h the TMA producer loads, per packed stage, the tiles
// of the A quadrants that xi_h = alpha_h phi selects and of the Bt quadrants
// that eta_h = beta_h psi selects (the combined operators of Eqs. mb-* /
// ab-* / sw-*), the expansion warps XOR them as they expand, so the seven
// operands never exist in HBM, and the epilogue XORs the product's parity
// bits into the C quadrants that zeta = chi gamma sends it to, in
// registers; the four quadrant words of the position leave once, after the
// seventh product.
template <bool BATCHED, bool PAIR, bool FP4, bool LEVEL = false>
__global__ void __launch_bounds__(THREADS, 1)
    tc_nt_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const Params p) {
    static_assert(!LEVEL || (!BATCHED && PAIR), "the in-kernel level runs on SM pairs");
    using LY = Lay<PAIR, FP4, LEVEL>;
    constexpr int PSTAGES = LY::PSTAGES, OSLOTS = LY::OSLOTS, KP = LY::KP;
    constexpr int BEXP_WARPS = LY::BEXP_WARPS, EPI_WARP0 = LY::EPI_WARP0,
                  EPI_WARPS = LY::EPI_WARPS;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + LY::OFF_BAR;
    auto full_p = [&](int s) { return bar0 + 8u * s; };
    auto empty_p = [&](int s) { return bar0 + 8u * (PSTAGES + s); };
    auto full_o = [&](int q) { return bar0 + 8u * (2 * PSTAGES + q); };
    auto empty_o = [&](int q) { return bar0 + 8u * (2 * PSTAGES + OSLOTS + q); };
    const uint32_t acc_full = bar0 + 8u * (2 * PSTAGES + 2 * OSLOTS);
    const uint32_t acc_empty = acc_full + 8u;
    const uint32_t drain_bar = acc_full + 16u;
    uint32_t* tmem_slot = (uint32_t*)(smem + LY::OFF_TMEM_SLOT);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // In a pair, CTA 0 issues the MMAs and holds the barriers that gate them
    // (full_o, acc_empty); both CTAs' producers and epilogues arrive there.
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    constexpr uint32_t CTAS = PAIR ? 2u : 1u;
    auto arrive_leader = [&](uint32_t bar) {
        if (PAIR)
            mbar_arrive_cluster(bar, 0);
        else
            mbar_arrive(bar);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; s++) {
            mbar_init(full_p(s), 1);
            mbar_init(empty_p(s), BEXP_WARPS + AEXP_WARPS);  // every expansion warp reads every stage
        }
        for (int q = 0; q < OSLOTS; q++) {
            mbar_init(full_o(q), CTAS * (BEXP_WARPS + AEXP_WARPS));
            mbar_init(empty_o(q), 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, CTAS * EPI_WARPS);
        mbar_init(drain_bar, 1);
        fence_barrier_init();
    }
    if (warp == MMA_WARP) tmem_alloc<PAIR>(smem_u32(tmem_slot));
    if (!BATCHED && warp == TMA_WARP && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA))
                     : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB))
                     : "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();  // the peer's barriers exist before anything arrives on them
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int kchunk = p.kchunk;
    const int my_tiles = tile_count<BATCHED, PAIR>(p);
    const TcWorkItem* my_items = BATCHED ? p.items + p.cta_ptr[unit_id<PAIR>()] : nullptr;
    int total_pit = 0;  // packed stages this CTA runs (batched: from the plan)
    if (BATCHED)
        total_pit = p.cta_ptr[unit_count<PAIR>() + 1 + unit_id<PAIR>()];
    else
        total_pit = my_tiles * (LEVEL ? 7 : 1) * (p.nks / SUB);
    // LEVEL: a packed stage's quadrant tiles, A's first (sub-buffer j)
    auto qtile = [&](int s, int j) {
        return (uint32_t)(LY::OFF_PA + s * LY::PSTAGE_BYTES + j * LY::PA_BYTES);
    };

    if (warp == TMA_WARP) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int pit = 0;  // packed stages issued
            bool ok = true;
            // Batched: a tile's work item is read two tiles ahead and its
            // TMA maps prefetched one tile ahead, so neither the item load
            // nor a map fetch stalls the copies of the tile before it.
            Tile nxt = my_tiles > 0 ? tile_get<BATCHED, PAIR>(p, my_items, 0, &tmA, &tmB) : Tile{};
            Tile nxt2 = my_tiles > 1 ? tile_get<BATCHED, PAIR>(p, my_items, 1, &tmA, &tmB) : nxt;
            if (BATCHED && my_tiles > 0) {
                prefetch_tensormap(nxt.ma);
                prefetch_tensormap(nxt.mb);
            }
            for (int i = 0; ok && i < my_tiles; i++) {
                const Tile tc = nxt;
                nxt = nxt2;
                if (BATCHED && i + 1 < my_tiles) {
                    prefetch_tensormap(nxt.ma);
                    prefetch_tensormap(nxt.mb);
                }
                if (i + 2 < my_tiles)
                    nxt2 = tile_get<BATCHED, PAIR>(p, my_items, i + 2, &tmA, &tmB);
                const int arow = tc.tm * LY::TILE_M + (int)rank * BM;
                // an N = 128 tile takes 64 of its columns from each CTA of a pair
                const int brow =
                    tc.tn * BN + (int)rank * (BATCHED && tc.n128 ? LY::BROWS / 2 : LY::BROWS);
                if (LEVEL) {
                    // A quadrant (r, c) at rows r m, words c qkw; B block (r, c)
                    // is stored transposed, as Bt rows c n, words r qkw
                    for (int h = 0; ok && h < 7; h++) {
                        const uint32_t xa = (p.xi4 >> (4 * h)) & 0xFu;
                        const uint32_t xb = (p.eta4 >> (4 * h)) & 0xFu;
                        const uint32_t bytes = (uint32_t)(__popc(xa) + __popc(xb)) * LY::PA_BYTES;
                        for (int kp = 0; kp < tc.nks / SUB; kp++, pit++) {
                            const int s = pit % PSTAGES;
                            if (!mbar_wait(empty_p(s), ((pit / PSTAGES) & 1) ^ 1, p.err)) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_tx(full_p(s), bytes);
                            int j = 0;
                            for (int q = 0; q < 4; q++)
                                if ((xa >> q) & 1u)
                                    tma_load_3d(sbase + qtile(s, j++), tc.ma,
                                                (q & 1) * p.qkw + kp * (KP / 64),
                                                (q >> 1) * tc.m + arow, tc.leaf, full_p(s));
                            for (int q = 0; q < 4; q++)
                                if ((xb >> q) & 1u)
                                    tma_load_3d(sbase + qtile(s, j++), tc.mb,
                                                (q >> 1) * p.qkw + kp * (KP / 64),
                                                (q & 1) * tc.n + brow, tc.leaf, full_p(s));
                        }
                    }
                    continue;
                }
                for (int kp = 0; kp < (tc.nks + SUB - 1) / SUB; kp++, pit++) {
                    const int s = pit % PSTAGES;
                    if (!mbar_wait(empty_p(s), ((pit / PSTAGES) & 1) ^ 1, p.err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(full_p(s), LY::PA_BYTES + LY::PB_BYTES);
                    tma_load_3d(sbase + LY::OFF_PA + s * LY::PA_BYTES, tc.ma, kp * (KP / 64), arow,
                                tc.leaf, full_p(s));
                    tma_load_3d(sbase + LY::OFF_PB + s * LY::PB_BYTES, tc.mb, kp * (KP / 64), brow,
                                tc.leaf, full_p(s));
                }
            }
            // drain: the copies of the last issued stages must land before exit
            for (int j = 1; j <= PSTAGES && j <= pit; j++) {
                const int i = pit - j;
                if (!mbar_wait(full_p(i % PSTAGES), (i / PSTAGES) & 1, p.err)) break;
            }
        }
    } else if (FP4 && warp < BEXP_WARPS) {
        // ---------------------------------------------------- Bt expansion, e2m1
        // Per packed stage: items of 2 rows x 16 packed words (both operand
        // stages). Lane = (half h, row rr of the item, word wl of the half):
        // word w = 8h + wl goes to 16-byte chunk wl of operand stage 2q + h.
        // A quarter-warp holds the 8 chunks of one row: 8 distinct bank groups.
        const int h = lane >> 4, rr = (lane >> 3) & 1, wl = lane & 7;
        const Spread sp = p.sp;
        int lv_k = 0, lv_h = 0;  // LEVEL: packed stage within the product, the product
        for (int pit = 0; pit < total_pit; pit++) {
            const int s = pit % PSTAGES;
            const int q = pit % OSLOTS;
            if (!mbar_wait(full_p(s), (pit / PSTAGES) & 1, p.err) ||
                !mbar_wait(empty_o(q), ((pit / OSLOTS) & 1) ^ 1, p.err))
                break;
            constexpr int ITEMS = (LY::BROWS / 2) / BEXP_WARPS;
            uint8_t* eb = smem + LY::OFF_EB + (2 * q + h) * LY::EB_BYTES;
            uint32_t x[ITEMS];
            if (LEVEL) {
                // S_h: the XOR of the Bt quadrant tiles, stored after A's
                const int j0 = __popc((p.xi4 >> (4 * lv_h)) & 0xFu);
                const int nb = __popc((p.eta4 >> (4 * lv_h)) & 0xFu);
#pragma unroll
                for (int i = 0; i < ITEMS; i++) x[i] = 0u;
                for (int j = 0; j < nb; j++) {
                    const uint32_t* pb = reinterpret_cast<const uint32_t*>(smem + qtile(s, j0 + j));
#pragma unroll
                    for (int i = 0; i < ITEMS; i++)
                        x[i] ^= pb[((warp + BEXP_WARPS * i) * 2 + rr) * 16 + 8 * h + wl];
                }
                if (++lv_k == p.nks / SUB) {
                    lv_k = 0;
                    if (++lv_h == 7) lv_h = 0;
                }
            } else {
                const uint32_t* pb =
                    reinterpret_cast<const uint32_t*>(smem + LY::OFF_PB + s * LY::PB_BYTES);
#pragma unroll
                for (int i = 0; i < ITEMS; i++)
                    x[i] = pb[((warp + BEXP_WARPS * i) * 2 + rr) * 16 + 8 * h + wl];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_p(s));
#pragma unroll
            for (int i = 0; i < ITEMS; i++) {
                const int row = (warp + BEXP_WARPS * i) * 2 + rr;
                uint32_t y[4];
                spread4(x[i], sp, y);
                *reinterpret_cast<uint4*>(eb + row * 128 + ((wl ^ (row & 7)) * 16)) =
                    make_uint4(y[0], y[1], y[2], y[3]);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) arrive_leader(full_o(q));
        }
    } else if (warp < BEXP_WARPS) {
        // ---------------------------------------------------- Bt expansion (shared)
        // Per packed stage: items of 4 rows x 8 packed words (both operand
        // stages). Lane = (half h, row rr of the item, word wl of the half):
        // word w = 4h + wl of the row goes to operand stage 2q + h of slot q.
        // A quarter-warp then holds two adjacent rows (opposite parity) x 4
        // words of one half, whose swizzled 16-byte chunks are 8 distinct bank
        // groups.
        const int h = lane >> 4, rr = (lane >> 2) & 3, wl = lane & 3;
        const Spread sp = p.sp;
        static_assert(SUB == 2, "a packed stage feeds two operand stages");
        for (int pit = 0; pit < total_pit; pit++) {
            const int s = pit % PSTAGES;
            const int q = pit % OSLOTS;
            if (!mbar_wait(full_p(s), (pit / PSTAGES) & 1, p.err) ||
                !mbar_wait(empty_o(q), ((pit / OSLOTS) & 1) ^ 1, p.err))
                break;
            constexpr int ITEMS = (LY::BROWS / 4) / BEXP_WARPS;
            const uint32_t* pb =
                reinterpret_cast<const uint32_t*>(smem + LY::OFF_PB + s * LY::PB_BYTES);
            uint8_t* eb = smem + LY::OFF_EB + (2 * q + h) * LY::EB_BYTES;
            uint32_t x[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; i++)
                x[i] = pb[((warp + BEXP_WARPS * i) * 4 + rr) * 8 + 4 * h + wl];
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_p(s));
#pragma unroll
            for (int i = 0; i < ITEMS; i++) {
                const int row = (warp + BEXP_WARPS * i) * 4 + rr;
                uint8_t* rowp = eb + row * 128;
                uint32_t y[8];
                spread8(x[i], sp, y);
                *reinterpret_cast<uint4*>(rowp + (((2 * wl) ^ (row & 7)) * 16)) =
                    make_uint4(y[0], y[1], y[2], y[3]);
                *reinterpret_cast<uint4*>(rowp + (((2 * wl + 1) ^ (row & 7)) * 16)) =
                    make_uint4(y[4], y[5], y[6], y[7]);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) arrive_leader(full_o(q));
        }
    } else if (warp < EPI_WARP0) {
        // ---------------------------------------------------- A expansion (TMEM)
        // One warp per TMEM lane quarter, one row per thread, every packed
        // stage: 256 bits -> 256 e4m3 bytes = both operand stages of the
        // slot, adjacent TMEM columns, one store.
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        const Spread sp = p.sp;
        const uint32_t tlane = (uint32_t)(32 * quarter) << 16;
        if (FP4) {
            // block scales for this lane quarter, before the first full_o arrive
            uint32_t f[64];
#pragma unroll
            for (int i = 0; i < 64; i++) f[i] = SCALE_WORD;
            tmem_st64(tmem + tlane + (uint32_t)SF_COL, f);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        int lv_k = 0, lv_h = 0;  // LEVEL: packed stage within the product, the product
        for (int pit = 0; pit < total_pit; pit++) {
            const int s = pit % PSTAGES;
            const int q = pit % OSLOTS;
            if (!mbar_wait(full_p(s), (pit / PSTAGES) & 1, p.err)) break;
            constexpr int NV = KP / 128;  // 16-byte vectors per packed row
            uint4 xv[NV];
            if (LEVEL) {
                // T_h: the XOR of the A quadrant tiles
                const int na = __popc((p.xi4 >> (4 * lv_h)) & 0xFu);
#pragma unroll
                for (int v = 0; v < NV; v++) xv[v] = make_uint4(0u, 0u, 0u, 0u);
                for (int j = 0; j < na; j++) {
                    const uint4* src =
                        reinterpret_cast<const uint4*>(smem + qtile(s, j) + row * (KP / 8));
#pragma unroll
                    for (int v = 0; v < NV; v++) {
                        const uint4 t = src[v];
                        xv[v].x ^= t.x;
                        xv[v].y ^= t.y;
                        xv[v].z ^= t.z;
                        xv[v].w ^= t.w;
                    }
                }
                if (++lv_k == p.nks / SUB) {
                    lv_k = 0;
                    if (++lv_h == 7) lv_h = 0;
                }
            } else {
                const uint4* src = reinterpret_cast<const uint4*>(smem + LY::OFF_PA +
                                                                  s * LY::PA_BYTES + row * (KP / 8));
#pragma unroll
                for (int v = 0; v < NV; v++) xv[v] = src[v];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_p(s));
            if (!mbar_wait(empty_o(q), ((pit / OSLOTS) & 1) ^ 1, p.err)) break;
            tc_fence_after();  // the slot's MMAs (seen complete) before our TMEM stores
            uint32_t y[64];
#pragma unroll
            for (int v = 0; v < NV; v++) {
                if (FP4) {
                    spread4(xv[v].x, sp, y + 16 * v);
                    spread4(xv[v].y, sp, y + 16 * v + 4);
                    spread4(xv[v].z, sp, y + 16 * v + 8);
                    spread4(xv[v].w, sp, y + 16 * v + 12);
                } else {
                    spread8(xv[v].x, sp, y + 32 * v);
                    spread8(xv[v].y, sp, y + 32 * v + 8);
                    spread8(xv[v].z, sp, y + 32 * v + 16);
                    spread8(xv[v].w, sp, y + 32 * v + 24);
                }
            }
            tmem_st64(tmem + tlane + (uint32_t)(A_COL + 2 * q * A_STAGE_COLS), y);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive_leader(full_o(q));
        }
    } else if (warp == MMA_WARP) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc =
                FP4 ? instr_desc_mxf4<LY::TILE_M>() : instr_desc<LY::TILE_M>(1u);
            constexpr uint32_t idesc128 = FP4 ? instr_desc_mxf4<LY::TILE_M, BN / 2>()
                                              : instr_desc<LY::TILE_M, BN / 2>(1u);
            // operand stage e's descriptor: the start-address field (bytes >> 4)
            // moves by EB_BYTES >> 4 per stage; every stage lies below 256 KB,
            // so no carry
            const uint64_t db_base = smem_desc_sw128(sbase + LY::OFF_EB);
            // The issuing thread's own instructions sit on the tensor pipe's
            // critical path (one extra branch per stage measured 5 %), so the
            // slot and its phase are running counters, not divisions.
            static_assert(LY::WAITG == 1 || LY::WAITG == 2, "wait groups of one or two slots");
            int seg = 0, pit = 0;
            int q = 0;         // pit % OSLOTS
            uint32_t ph = 0;   // (pit / OSLOTS) & 1
            bool ok = true;
            // a tile's k stages are loaded one tile ahead (batched: from the
            // work list in global memory, off the issue path)
            // (batched: items read two tiles ahead of their use)
            TileK tk_next = my_tiles > 0 ? tile_k<BATCHED>(p, my_items, 0) : TileK{0, 0};
            TileK tk_next2 = my_tiles > 1 ? tile_k<BATCHED>(p, my_items, 1) : tk_next;
            // LEVEL: every tile position runs seven products, each an
            // accumulator tile of its own
            const int mma_tiles = LEVEL ? 7 * my_tiles : my_tiles;
            for (int i = 0; ok && i < mma_tiles; i++) {
                const int nks = tk_next.nks;
                const uint32_t id = BATCHED && tk_next.n128 ? idesc128 : idesc;
                tk_next = tk_next2;
                if (i + 2 < mma_tiles) tk_next2 = tile_k<BATCHED>(p, my_items, i + 2);
                int kin = 0;
                for (int ks = 0; ks < nks; ks += SUB, pit++) {
                    // Every producer fills the slots in order, so one wait on
                    // the last of WAITG consecutive slots covers them all. At a
                    // tile's first stage the operands are checked before the
                    // (longer) wait for the epilogue to free the accumulator.
                    const bool group = (pit & (LY::WAITG - 1)) == 0;
                    if (group) {
                        int qw = q;
                        uint32_t phw = ph;
                        if (LY::WAITG == 2 && pit + 1 < total_pit && ++qw == OSLOTS) {
                            qw = 0;
                            phw ^= 1u;
                        }
                        if (!mbar_wait(full_o(qw), phw, p.err)) {
                            ok = false;
                            break;
                        }
                    }
                    if (kin == 0) {
                        if (!mbar_wait(acc_empty, (seg & 1) ^ 1, p.err)) {
                            ok = false;
                            break;
                        }
                    }
                    if (group || kin == 0) tc_fence_after();
#pragma unroll
                    for (int sub = 0; sub < SUB; sub++) {
                        // batched: an odd k-stage count ends in half a packed
                        // stage, whose second operand stage is all padding
                        if (BATCHED && sub > 0 && ks + sub >= nks) break;
                        const int e = 2 * q + sub;
                        const uint32_t ta = tmem + (uint32_t)(A_COL + e * A_STAGE_COLS);
                        const uint64_t db = db_base + (uint64_t)(e * (LY::EB_BYTES >> 4));
#pragma unroll
                        for (int j = 0; j < MMAS_PER_STAGE; j++) {
                            const uint32_t acc = (kin > 0 || sub > 0 || j > 0) ? 1u : 0u;
                            if (FP4)
                                mma_f4_ta<PAIR>(tmem + ACC_COL, ta + j * A_MMA_COLS, db + 2 * j,
                                                BATCHED ? id : idesc, tmem + SF_COL,
                                                tmem + SF_COL + SF_COLS / 2, acc);
                            else
                                mma_f8_ta<PAIR>(tmem + ACC_COL, ta + j * A_MMA_COLS, db + 2 * j,
                                                BATCHED ? id : idesc, acc);
                        }
                    }
                    mma_commit<PAIR>(empty_o(q));
                    if (++q == OSLOTS) {
                        q = 0;
                        ph ^= 1u;
                    }
                    kin += SUB;
                    if (kin >= kchunk || ks + SUB >= nks) {
                        mma_commit<PAIR>(acc_full);
                        seg++;
                        kin = 0;
                    }
                }
            }
            if (!ok) {  // wait (bounded) for every MMA this thread issued
                mma_commit<PAIR>(drain_bar, 1);
                mbar_wait(drain_bar, 0, p.err);
            }
        }
    } else if (warp < TMA_WARP) {
        // ---------------------------------------------------- epilogue
        // EPI_WARPS / 4 warps per TMEM lane quarter, splitting the columns.
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
        const int chalf = (warp - EPI_WARP0) >> 2;
        const uint32_t tlane = (uint32_t)(32 * quarter) << 16;
        constexpr int CW = BN / (EPI_WARPS / 4) / 32;  // 32-column chunks per warp
        int seg = 0;
        bool ok = true;
        // batched: each tile's work item is copied into this warp's shared
        // slot while the tile before it runs, off the accumulator hand-off path
        const uint32_t islot =
            sbase + (uint32_t)(LY::OFF_ITEMS + (warp - EPI_WARP0) * 2 * LY::ITEM_BYTES);
        static_assert(sizeof(TcWorkItem) == LY::ITEM_BYTES, "three 16-byte copies per item");
        auto fetch_item = [&](int idx) {
            if (lane < 3)
                cp_async16(islot + (uint32_t)((idx & 1) * LY::ITEM_BYTES + 16 * lane),
                           reinterpret_cast<const uint8_t*>(my_items + idx) + 16 * lane);
        };
        if (BATCHED && my_tiles > 0) fetch_item(0);
        for (int i = 0; ok && i < my_tiles; i++) {
            Tile tc;
            if (BATCHED) {
                cp_async_wait_all();
                __syncwarp();
                TcWorkItem w;
                std::memcpy(&w, smem + (islot - sbase) + (i & 1) * LY::ITEM_BYTES, sizeof(w));
                __syncwarp();
                if (i + 1 < my_tiles) fetch_item(i + 1);
                tc = tile_of_item(p, w);
            } else {
                tc = tile_get<BATCHED, PAIR>(p, my_items, i, &tmA, &tmB);
            }
            const int nseg = (tc.nks + kchunk - 1) / kchunk;
            const bool gf2 = tc.op == OP_GF2;
            // an N = 128 tile writes no accumulator column past 128: the warps
            // that drain those columns only hand the accumulator back
            const bool idle = BATCHED && PAIR && tc.n128 && chalf == 1;
            // LEVEL: this thread's words of the four C quadrants, summed over
            // the position's seven products: word (q, c) at qo[(CW q + c) 32]
            static_assert(!LEVEL || CW == 4, "four words per quadrant");
            uint32_t* qo = reinterpret_cast<uint32_t*>(smem + LY::OFF_QOUT) +
                           (warp - EPI_WARP0) * 32 * 16 + lane;
            if (LEVEL)
#pragma unroll
                for (int j = 0; j < 16; j++) qo[32 * j] = 0u;
            uint32_t out[1][CW];
#pragma unroll
            for (int c = 0; c < CW; c++) out[0][c] = 0u;
            for (int h = 0; ok && h < (LEVEL ? 7 : 1); h++) {
            // LEVEL: the C quadrants product h goes to (bit q)
            uint32_t zq = 0;
            if (LEVEL)
                for (int q = 0; q < 4; q++) zq |= ((p.zeta7 >> (7 * q + h)) & 1u) << q;
            uint32_t words[LEVEL ? 1 : CW];
#pragma unroll
            for (int c = 0; c < (LEVEL ? 1 : CW); c++) words[c] = 0u;
            for (int g = 0; g < nseg; g++, seg++) {
                if (!mbar_wait(acc_full, seg & 1, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (idle) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) arrive_leader(acc_empty);
                    continue;
                }
                if (LEVEL) {
                    // parities are XOR-linear: each chunk folds straight into
                    // the quadrants product h goes to
#pragma unroll
                    for (int c = 0; c < CW; c += 2) {
                        uint32_t v[64];
                        tmem_ld64(tmem + tlane + (uint32_t)(ACC_COL + 32 * (CW * chalf + c)), v);
                        if (c + 2 == CW) {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) arrive_leader(acc_empty);
                        }
                        const uint32_t b0 = pack_bits<OP_GF2>(v), b1 = pack_bits<OP_GF2>(v + 32);
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            if ((zq >> q) & 1u) {
                                qo[32 * (CW * q + c)] ^= b0;
                                qo[32 * (CW * q + c + 1)] ^= b1;
                            }
                    }
                    continue;
                }
                // 64 columns per load: half the load-wait round trips of 32
#pragma unroll
                for (int c = 0; c < CW; c += 2) {
                    uint32_t v[64];
                    tmem_ld64(tmem + tlane + (uint32_t)(ACC_COL + 32 * (CW * chalf + c)), v);
                    if (c + 2 == CW) {
                        // every column this warp drains is in registers: hand the
                        // accumulator back before packing the last chunk
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) arrive_leader(acc_empty);
                    }
                    if (gf2) {
                        words[c] ^= pack_bits<OP_GF2>(v);
                        words[c + 1] ^= pack_bits<OP_GF2>(v + 32);
                    } else {
                        words[c] |= pack_bits<OP_BOOL>(v);
                        words[c + 1] |= pack_bits<OP_BOOL>(v + 32);
                    }
                }
            }
            if (!LEVEL) {
#pragma unroll
                for (int c = 0; c < CW; c++) out[0][c] = words[c];
            }
            }
            if (!ok) break;
            const int64_t row =
                (int64_t)tc.tm * LY::TILE_M + (int64_t)rank * BM + 32 * quarter + lane;
            if (LEVEL) {
                // quadrant (r, c) of the block's C: rows r m, words c n/64
                const int64_t w0 = (int64_t)tc.tn * (BN / 64) + chalf * (CW / 2);
                const int64_t nw = tc.n / 64;
                if (row < tc.m) {
#pragma unroll
                    for (int q = 0; q < (LEVEL ? 4 : 1); q++) {
                        uint64_t* crow = tc.C + ((q >> 1) * (int64_t)tc.m + row) * tc.ldc +
                                         (q & 1) * nw;
#pragma unroll
                        for (int c = 0; c < CW / 2; c++)
                            if (w0 + c < nw)
                                crow[w0 + c] = (uint64_t)qo[32 * (CW * q + 2 * c)] |
                                               ((uint64_t)qo[32 * (CW * q + 2 * c + 1)] << 32);
                    }
                }
            } else if (row < tc.m) {
                uint64_t* crow = tc.C + row * tc.ldc;
                const int64_t w0 = (int64_t)tc.tn * (BN / 64) + chalf * (CW / 2);
                const int64_t nw = tc.n / 64;
#pragma unroll
                for (int c = 0; c < CW / 2; c++)
                    if (w0 + c < nw)
                        crow[w0 + c] = (uint64_t)out[0][2 * c] | ((uint64_t)out[0][2 * c + 1] << 32);
            }
        }
        // a loop left early (a wait gave up) may still have an item copy in
        // flight into this warp's slot
        if (BATCHED) cp_async_wait_all();
    }

    tc_fence_before();
    __syncthreads();
    // A pair leaves together: the peer's remote arrivals and the MMAs that
    // read its shared memory and TMEM are over before either CTA frees TMEM.
    if (PAIR) cluster_sync();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc<PAIR>(tmem);
    }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return fn;
}

// 3-D map over uint64 words: (k/64 words, rows, leaves), box (box_words,
// box_rows, 1). Boxes that run past k or the rows are zero-filled, which
// adds nothing to the counts.
bool make_map(CUtensorMap* map, const uint64_t* base, int64_t kwords, int64_t rows,
              int64_t pitch, int64_t count, int64_t stride, int box_rows, int box_words) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kwords, (cuuint64_t)rows, (cuuint64_t)count};
    const int64_t leaf_stride = count > 1 ? stride : rows * pitch;
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * 8), (cuuint64_t)(leaf_stride * 8)};
    cuuint32_t box[3] = {(cuuint32_t)box_words, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)base, dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

// 2-D map over uint64 words (inner words, outer rows, row stride in bytes),
// box (box_words, box_rows), 64-byte swizzle when asked (box rows of 64 B).
bool make_map_2d(CUtensorMap* map, const void* base, int64_t words, int64_t rows,
                 int64_t stride_bytes, int box_words, int box_rows, bool swizzle64) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)words, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)stride_bytes};
    cuuint32_t box[2] = {(cuuint32_t)box_words, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r =
        fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE,
           swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

constexpr int MAX_DEVICES = 64;

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// Per-device one-time setup (function attributes and occupancy are per device).
std::mutex g_setup_mu;

template <bool BATCHED, bool PAIR, bool FP4, bool LEVEL = false>
cudaError_t set_smem_attr() {
    static bool done[MAX_DEVICES] = {false};
    static cudaError_t err[MAX_DEVICES];
    const int d = current_device();
    if (d < 0 || d >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!done[d]) {
        err[d] = cudaFuncSetAttribute(tc_nt_kernel<BATCHED, PAIR, FP4, LEVEL>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Lay<PAIR, FP4, LEVEL>::SMEM_BYTES);
        done[d] = true;
    }
    return err[d];
}

cudaLaunchConfig_t pair_config(unsigned units, size_t smem, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * units);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// CTA pairs of the e4m3 (FP4 false) or e2m1 kernel that can be resident at
// once on the current device (clusters of two on one TPC); 0 if cluster
// launches are unavailable.
template <bool FP4>
int pair_slots() {
    static int slots[MAX_DEVICES];
    static bool done[MAX_DEVICES] = {false};
    const int d = current_device();
    if (d < 0 || d >= MAX_DEVICES) return 0;
    if (set_smem_attr<false, true, FP4>() != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!done[d]) {
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg =
            pair_config((unsigned)sm_count(), Lay<true, FP4>::SMEM_BYTES, at);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc_nt_kernel<false, true, FP4>, &cfg) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            n = 0;
        }
        slots[d] = n;
        done[d] = true;
    }
    return slots[d];
}

// units: CTAs (single) or CTA pairs (PAIR) to launch.
template <bool BATCHED, bool PAIR, bool FP4, bool LEVEL = false>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const Params& prm, int units,
                      cudaStream_t s) {
    static_assert(PAIR || !FP4, "the e2m1 form runs on SM pairs");
    const cudaError_t e = set_smem_attr<BATCHED, PAIR, FP4, LEVEL>();
    if (e != cudaSuccess) return e;
    if (!PAIR) {
        tc_nt_kernel<BATCHED, false, false>
            <<<units, THREADS, Lay<false, false>::SMEM_BYTES, s>>>(ma, mb, prm);
        return cudaGetLastError();
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = pair_config((unsigned)units, Lay<PAIR, FP4, LEVEL>::SMEM_BYTES, at);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, tc_nt_kernel<BATCHED, PAIR, FP4, LEVEL>, ma, mb, prm);
}

// CTA pairs of the in-kernel-level kernel (e2m1) that can be resident at once.
int level_slots() {
    static int slots[MAX_DEVICES];
    static bool done[MAX_DEVICES] = {false};
    const int d = current_device();
    if (d < 0 || d >= MAX_DEVICES) return 0;
    if (set_smem_attr<false, true, true, true>() != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!done[d]) {
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg =
            pair_config((unsigned)sm_count(), Lay<true, true, true>::SMEM_BYTES, at);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc_nt_kernel<false, true, true, true>, &cfg) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            n = 0;
        }
        slots[d] = n;
        done[d] = true;
    }
    return slots[d];
}

Spread spread_factors() {
    Spread sp;
    for (int j = 0; j < 8; j++) sp.f[j] = j <= 3 ? (1u << (3 - j)) : (1u << (35 - j));
    sp.g[0] = 2u;
    sp.g[1] = 1u;
    sp.g[2] = 1u << 31;
    sp.g[3] = 1u << 30;
    return sp;
}

// k bits per operand stage of a tensor path.
int64_t stage_bits(int path) { return path == BMM_PATH_TC_FP4_PAIR ? 256 : 128; }

}  // namespace

bool tc_path_available() { return device_cc() == 103 && encode_fn() != nullptr; }

// SM pairs need cluster launches with both CTAs of a pair resident at once.
bool tc_pair_available() { return tc_path_available() && pair_slots<false>() > 0; }
bool tc_fp4_available() { return tc_path_available() && pair_slots<true>() > 0; }

// Longest run of k stages accumulated before the counts are flushed from
// TMEM: both formats read parity through an FP32 value count * 2^-12, exact
// while count < 2^23: at most 65534 stages of 128 k, or 32766 of 256.
int tc_kchunk_stages(int path, int nks) {
    // a multiple of the operand stages per packed stage (flushes happen between packed stages)
    const int cap = path == BMM_PATH_TC_FP4_PAIR ? 32766 : 65534;
    return nks < cap ? nks : cap;
}

bmm_status run_tc_strided(int op, int path, const uint64_t* A, int64_t lda, int64_t strideA,
                          const uint64_t* Bt, int64_t ldb, int64_t strideB, uint64_t* C,
                          int64_t ldc, int64_t strideC, int64_t count, int64_t m, int64_t k,
                          int64_t n, cudaStream_t s) {
    const bool fp4 = path == BMM_PATH_TC_FP4_PAIR;
    const bool pair = fp4 || path == BMM_PATH_TC_FP8_PAIR;
    if (!tc_path_available() || (path != BMM_PATH_TC_FP8 && !pair)) return BMM_ERR_UNSUPPORTED;
    if (k % KS_MIN || (lda & 1) || (ldb & 1) ||
        (count > 1 && ((strideA & 1) || (strideB & 1))))
        return BMM_ERR_UNSUPPORTED;
    if (m <= 0 || n <= 0 || k <= 0 || count <= 0) return BMM_OK;
    // tile and stage indices are 32-bit in the kernel
    if (m > 0x7fffffffLL || n > 0x7fffffffLL || k / KS_MIN > 0x3fffffffLL)
        return BMM_ERR_UNSUPPORTED;
    const int slots = fp4 ? pair_slots<true>() : pair ? pair_slots<false>() : sm_count();
    if (slots <= 0) return BMM_ERR_UNSUPPORTED;
    uint32_t* err = device_error_word();
    if (!err) return BMM_ERR_NOMEM;
    const int64_t kp = SUB * stage_bits(path);  // k bits per packed stage
    const int tile_m = pair ? Lay<true, false>::TILE_M : Lay<false, false>::TILE_M;
    const int brows = pair ? Lay<true, false>::BROWS : Lay<false, false>::BROWS;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, k / 64, m, lda, count, strideA, BM, (int)(kp / 64)) ||
        !make_map(&mb, Bt, k / 64, n, ldb, count, strideB, brows, (int)(kp / 64)))
        return BMM_ERR_CUDA;
    Params prm{};
    prm.C = C;
    prm.ldc = ldc;
    prm.strideC = strideC;
    prm.m = (int)m;
    prm.n = (int)n;
    prm.nks = (int)((k + kp - 1) / kp) * SUB;  // whole packed stages; the tail is zero-filled
    prm.op = op;
    prm.kchunk = tc_kchunk_stages(path, prm.nks);
    prm.tiles_m = (int)((m + tile_m - 1) / tile_m);
    prm.tiles_n = (int)((n + BN - 1) / BN);
    const int64_t total = (int64_t)prm.tiles_m * prm.tiles_n * count;
    if (total > 0x7fffffff) return BMM_ERR_UNSUPPORTED;
    prm.total_tiles = (int)total;
    prm.err = err;
    prm.sp = spread_factors();
    TraceScope ts(BMM_PHASE_BASE, s);
    const int units = prm.total_tiles < slots ? prm.total_tiles : slots;
    const cudaError_t e = fp4    ? launch_tc<false, true, true>(ma, mb, prm, units, s)
                          : pair ? launch_tc<false, true, false>(ma, mb, prm, units, s)
                                 : launch_tc<false, false, false>(ma, mb, prm, units, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return BMM_OK;
}

// The binary product of each block of a batch through one Strassen level run
// inside the e2m1 SM-pair kernel: block h is C (m x n, pitch ldc) = A (m x k,
// pitch lda) times Bt (n x k, pitch ldb)^T at A + h strideA, Bt + h strideB,
// C + h strideC (words). m and n even, k a multiple of 2 x 512 bits (every
// quadrant's k whole packed stages, so no copy reads into the neighbouring
// quadrant), even pitches and strides.
bmm_status run_tc_level(const uint64_t* A, int64_t lda, int64_t strideA, const uint64_t* Bt,
                        int64_t ldb, int64_t strideB, uint64_t* C, int64_t ldc, int64_t strideC,
                        int64_t count, int64_t m, int64_t k, int64_t n, const LevelMasks& masks,
                        cudaStream_t s) {
    using LY = Lay<true, true, true>;
    if (!tc_path_available()) return BMM_ERR_UNSUPPORTED;
    if (m % 2 || n % 2 || k % (2 * LY::KP) || (lda & 1) || (ldb & 1) ||
        (count > 1 && ((strideA & 1) || (strideB & 1))))
        return BMM_ERR_UNSUPPORTED;
    if (m <= 0 || n <= 0 || k <= 0 || count <= 0) return BMM_OK;
    if (m > 0x7fffffffLL || n > 0x7fffffffLL || k / KS_MIN > 0x3fffffffLL)
        return BMM_ERR_UNSUPPORTED;
    const int slots = level_slots();
    if (slots <= 0) return BMM_ERR_UNSUPPORTED;
    uint32_t* err = device_error_word();
    if (!err) return BMM_ERR_NOMEM;
    const int64_t hm = m / 2, hk = k / 2, hn = n / 2;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, k / 64, m, lda, count, strideA, BM, LY::KP / 64) ||
        !make_map(&mb, Bt, k / 64, n, ldb, count, strideB, LY::BROWS, LY::KP / 64))
        return BMM_ERR_CUDA;
    Params prm{};
    prm.C = C;
    prm.ldc = ldc;
    prm.strideC = strideC;
    prm.m = (int)hm;
    prm.n = (int)hn;
    prm.nks = (int)(hk / LY::KP) * SUB;
    prm.op = OP_GF2;
    prm.kchunk = tc_kchunk_stages(BMM_PATH_TC_FP4_PAIR, prm.nks);
    prm.tiles_m = (int)((hm + LY::TILE_M - 1) / LY::TILE_M);
    prm.tiles_n = (int)((hn + BN - 1) / BN);
    const int64_t total = (int64_t)prm.tiles_m * prm.tiles_n * count;
    if (total > 0x7fffffff / 7) return BMM_ERR_UNSUPPORTED;
    prm.total_tiles = (int)total;
    prm.err = err;
    prm.sp = spread_factors();
    for (int h = 0; h < 7; h++) {
        // a packed stage holds at most QTILES quadrant tiles (every variant's
        // products combine at most six)
        if (__builtin_popcount(masks.xi[h] & 0xFu) + __builtin_popcount(masks.eta[h] & 0xFu) >
            LY::QTILES)
            return BMM_ERR_UNSUPPORTED;
        prm.xi4 |= (masks.xi[h] & 0xFu) << (4 * h);
        prm.eta4 |= (masks.eta[h] & 0xFu) << (4 * h);
    }
    for (int q = 0; q < 4; q++) prm.zeta7 |= (masks.zeta[q] & 0x7Fu) << (7 * q);
    prm.qkw = (int)(hk / 64);
    TraceScope ts(BMM_PHASE_BASE, s);
    const int units = prm.total_tiles < slots ? prm.total_tiles : slots;
    const cudaError_t e = launch_tc<false, true, true, true>(ma, mb, prm, units, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return BMM_OK;
}

}  // namespace bmm

namespace bmm {

int tc_pair_slots(bool fp4) {
    if (!tc_path_available()) return 0;
    return fp4 ? pair_slots<true>() : pair_slots<false>();
}

bool tc_make_problem(TcProblem* out, const uint64_t* A, int64_t lda, const uint64_t* Bt,
                     int64_t ldb, uint64_t* C, int64_t ldc, int64_t m, int64_t k, int64_t n,
                     int op, bool pair, bool fp4) {
    if (k % KS_MIN || (lda & 1) || (ldb & 1) || (fp4 && !pair)) return false;
    const int64_t kp = SUB * stage_bits(fp4 ? BMM_PATH_TC_FP4_PAIR : BMM_PATH_TC_FP8);
    if (!make_map(&out->mapA, A, k / 64, m, lda, 1, 0, BM, (int)(kp / 64)) ||
        !make_map(&out->mapB, Bt, k / 64, n, ldb, 1, 0,
                  pair ? Lay<true, false>::BROWS : Lay<false, false>::BROWS, (int)(kp / 64)))
        return false;
    out->C = C;
    out->ldc = ldc;
    out->m = (int32_t)m;
    out->n = (int32_t)n;
    out->nks = (int32_t)(((k + kp - 1) / kp) * SUB);
    out->op = op;
    return true;
}

int tc_problem_kchunk(bool fp4) {
    return tc_kchunk_stages(fp4 ? BMM_PATH_TC_FP4_PAIR : BMM_PATH_TC_FP8, 0x7fffffff);
}

cudaError_t tc_prepare_batched(bool pair, bool fp4) {
    if (fp4 && !pair) return cudaErrorInvalidValue;
    return fp4    ? set_smem_attr<true, true, true>()
           : pair ? set_smem_attr<true, true, false>()
                  : set_smem_attr<true, false, false>();
}

cudaError_t tc_launch_batched(const TcProblem* d_probs, const TcWorkItem* d_items,
                              const int32_t* d_unit_ptr, int units, bool pair, bool fp4,
                              cudaStream_t s) {
    if (fp4 && !pair) return cudaErrorInvalidValue;
    uint32_t* err = device_error_word();
    if (!err) return cudaErrorMemoryAllocation;
    Params prm{};
    prm.probs = d_probs;
    prm.items = d_items;
    prm.cta_ptr = d_unit_ptr;
    prm.kchunk = tc_problem_kchunk(fp4);
    prm.err = err;
    prm.sp = spread_factors();
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    TraceScope ts(BMM_PHASE_BASE, s);
    return fp4    ? launch_tc<true, true, true>(dummy, dummy, prm, units, s)
           : pair ? launch_tc<true, true, false>(dummy, dummy, prm, units, s)
                  : launch_tc<true, false, false>(dummy, dummy, prm, units, s);
}

}  // namespace bmm

extern "C" bmm_status bmm_selftest_wait_timeout(int64_t limit_ns, bmm_stream_t stream) {
    using namespace bmm;
    if (limit_ns <= 0 || limit_ns > 10000000000LL) return BMM_ERR_INVALID;
    uint32_t* err = device_error_word();
    if (!err) return BMM_ERR_NOMEM;
    wait_selftest_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(err, (uint64_t)limit_ns);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BMM_OK : cuda_fail(e);
}
