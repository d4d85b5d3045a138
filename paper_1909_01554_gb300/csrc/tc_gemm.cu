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
// Persistent kernel, one CTA per SM, warp-specialised (22 warps):
//   warp 20     TMA producer: packed tiles of 128 rows of A and 256 rows of
//               Bt, 256 bits of k each (32-byte rows), into a PSTAGES-deep
//               shared ring (cp.async.bulk.tensor, mbarrier complete_tx).
//               Each packed stage feeds two operand stages of 128 bits.
//   warps 8-15  A expansion: one row per thread, 256 bits -> 256 e4m3
//               bytes (two operand stages) written straight into TMEM with
//               tcgen05.st; two warps per TMEM lane quarter take alternate
//               packed stages.
//   warps 0-7   Bt expansion: each packed 32-bit word becomes 32 bytes of
//               the K-major, 128-byte-swizzled canonical UMMA layout; a warp
//               expands 4 whole rows of a packed stage at a time.
//   warp 21     MMA issuer: per packed stage, one wait, then for each of its
//               two operand stages 4 x tcgen05.mma (M=128, N=256, K=32; A
//               from TMEM, B from shared memory) into the TMEM accumulator
//               and one commit that frees that operand stage.
//   warps 16-19 epilogue: tcgen05.ld 32 lanes x 32 columns at a time, parity
//               or non-zero test, bits packed in registers with a shallow
//               tree (one row per thread) and stored as 64-bit words.
// The A and Bt halves of an operand stage share one "full" barrier (all
// producers arrive) and one "empty" barrier (one commit). Every producer
// arrives on the first operand stage of a packed stage before the second,
// and commits complete in order, so waiting for the second stage's barrier
// covers both: each role checks one barrier per packed stage (a check costs
// ~190 cycles of latency, even when the phase is already complete). Keeping A in TMEM
// means shared memory carries only Bt (written once, read once by the tensor
// core). Long k is flushed from TMEM in chunks of `kchunk` stages (the
// epilogue folds parities / ORs across chunks).
//
// Within every 32-element group of k the expansion permutes k (byte t of
// output word j holds bit 8t + j of the packed word); A and Bt use the same
// permutation, so the contraction is unchanged.
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
constexpr int KS = 128;          // k (bits) per operand stage
constexpr int KP = TC_PACKED_BITS;  // k (bits) per packed (TMA) stage
constexpr int SUB = KP / KS;     // operand stages per packed stage
constexpr int MMA_K = 32;        // k per tcgen05.mma for 8-bit operands
constexpr int PSTAGES = 4;       // packed ring depth (shared)
constexpr int ESTAGES = 4;       // operand ring depth (Bt in shared, A in TMEM)
// 22 warps: an SM sub-partition (16 K registers) holds at most six of them,
// which caps registers at 80 per thread.
constexpr int BEXP_WARPS = 8;    // warps 0..7
constexpr int AEXP_WARP0 = 8;    // warps 8..15: two per TMEM lane quarter, alternate stages
constexpr int EPI_WARP0 = 16;    // warps 16..19 (warp % 4 = TMEM lane quarter)
constexpr int TMA_WARP = 20;
constexpr int MMA_WARP = 21;
constexpr int THREADS = 22 * 32;
constexpr int GROUP_M = 16;      // tile raster: 16 row-tiles per group

constexpr int PA_BYTES = BM * KP / 8;    // 4 KB packed A per packed stage
constexpr int PB_BYTES = BN * KP / 8;    // 8 KB packed Bt per packed stage
constexpr int EB_BYTES = BN * KS;        // 32 KB expanded Bt per operand stage
constexpr int ACC_COL = 0;               // accumulator: TMEM columns [0, BN)
constexpr int A_COL = BN;                // A ring: columns [BN, BN + ESTAGES * KS / 4)
constexpr int A_STAGE_COLS = KS / 4;     // 4 e4m3 per 32-bit column
constexpr int TMEM_COLS = 512;
static_assert(A_COL + ESTAGES * A_STAGE_COLS <= TMEM_COLS, "TMEM budget");

constexpr int OFF_EB = 0;
constexpr int OFF_PA = OFF_EB + ESTAGES * EB_BYTES;
constexpr int OFF_PB = OFF_PA + PSTAGES * PA_BYTES;
constexpr int OFF_BAR = OFF_PB + PSTAGES * PB_BYTES;
// barriers: full_p[P], empty_p[P], full_e[E], empty_e[E], acc_full, acc_empty, drain
constexpr int NBARS = 2 * PSTAGES + 2 * ESTAGES + 3;
constexpr int OFF_TMEM_SLOT = OFF_BAR + NBARS * 8;
constexpr int SMEM_BYTES = OFF_TMEM_SLOT + 16 + 1024;  // + alignment slack

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
__host__ __device__ constexpr uint32_t instr_desc(uint32_t dfmt) {
    return (dfmt << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// D (TMEM) += A (TMEM) x B (shared, descriptor).
__device__ __forceinline__ void mma_f8_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t db,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31])
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

// 32 result bits of one accumulator row slice -> one word, bit j from v[j].
// GF(2): v[j] = count * 2^-12 exactly; adding 2^11 puts count's LSB in bit 0.
// Boolean: any non-zero count. Packed with a 5-level tree of multiply-adds.
template <int OP>
__device__ __forceinline__ uint32_t pack_bits(const uint32_t (&v)[32]) {
    uint32_t b[32];
#pragma unroll
    for (int j = 0; j < 32; j++) {
        if (OP == OP_GF2)
            b[j] = __float_as_uint(__uint_as_float(v[j]) + 2048.0f) & 1u;
        else
            b[j] = min(v[j], 1u);  // fp32 counts are >= 0: non-zero bits <=> count > 0
    }
#pragma unroll
    for (int w = 1; w < 32; w *= 2)
#pragma unroll
        for (int j = 0; j < 32; j += 2 * w) b[j] = b[j + w] * (1u << w) + b[j];
    return b[0];
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
};

// Everything a role needs about one output tile.
struct Tile {
    const CUtensorMap* ma;
    const CUtensorMap* mb;
    uint64_t* C;  // leaf's C
    int64_t ldc;
    int m, n, nks, op, tm, tn, leaf;
};

template <bool BATCHED>
__device__ __forceinline__ int tile_count(const Params& p) {
    if (BATCHED) return p.cta_ptr[blockIdx.x + 1] - p.cta_ptr[blockIdx.x];
    int c = 0;
    for (int t = blockIdx.x; t < p.total_tiles; t += gridDim.x) c++;
    return c;
}

template <bool BATCHED>
__device__ __forceinline__ Tile tile_get(const Params& p, int idx, const CUtensorMap* tmA,
                                         const CUtensorMap* tmB) {
    Tile t;
    if (BATCHED) {
        const TcWorkItem w = p.items[p.cta_ptr[blockIdx.x] + idx];
        const TcProblem* d = p.probs + w.prob;
        t.ma = &d->mapA;
        t.mb = &d->mapB;
        t.C = d->C;
        t.ldc = d->ldc;
        t.m = d->m;
        t.n = d->n;
        t.nks = d->nks;
        t.op = d->op;
        t.tm = w.tm;
        t.tn = w.tn;
        t.leaf = 0;
    } else {
        const TileCoord c = tile_of(blockIdx.x + idx * gridDim.x, p.tiles_m, p.tiles_n);
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
    }
    return t;
}

template <bool BATCHED>
__device__ __forceinline__ int tile_nks(const Params& p, int idx) {
    if (BATCHED) return p.probs[p.items[p.cta_ptr[blockIdx.x] + idx].prob].nks;
    return p.nks;
}

template <bool BATCHED>
__global__ void __launch_bounds__(THREADS, 1)
    tc_nt_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const Params p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + OFF_BAR;
    auto full_p = [&](int s) { return bar0 + 8u * s; };
    auto empty_p = [&](int s) { return bar0 + 8u * (PSTAGES + s); };
    auto full_e = [&](int s) { return bar0 + 8u * (2 * PSTAGES + s); };
    auto empty_e = [&](int s) { return bar0 + 8u * (2 * PSTAGES + ESTAGES + s); };
    const uint32_t acc_full = bar0 + 8u * (2 * PSTAGES + 2 * ESTAGES);
    const uint32_t acc_empty = acc_full + 8u;
    const uint32_t drain_bar = acc_full + 16u;
    uint32_t* tmem_slot = (uint32_t*)(smem + OFF_TMEM_SLOT);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; s++) {
            mbar_init(full_p(s), 1);
            mbar_init(empty_p(s), BEXP_WARPS + 4);  // 8 Bt warps + the 4 A warps of that stage
        }
        for (int s = 0; s < ESTAGES; s++) {
            mbar_init(full_e(s), BEXP_WARPS + 4);  // 8 Bt warps + the 4 A warps of that stage
            mbar_init(empty_e(s), 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 4);
        mbar_init(drain_bar, 1);
        fence_barrier_init();
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (!BATCHED && warp == TMA_WARP && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA))
                     : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB))
                     : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int kchunk = p.kchunk;
    const int my_tiles = tile_count<BATCHED>(p);
    int total_it = 0;  // operand stages this CTA runs
    for (int i = 0; i < my_tiles; i++) total_it += tile_nks<BATCHED>(p, i);

    if (warp == TMA_WARP) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int pit = 0;  // packed stages issued
            bool ok = true;
            for (int i = 0; ok && i < my_tiles; i++) {
                const Tile tc = tile_get<BATCHED>(p, i, &tmA, &tmB);
                for (int kp = 0; kp < tc.nks / SUB; kp++, pit++) {
                    const int s = pit % PSTAGES;
                    if (!mbar_wait(empty_p(s), ((pit / PSTAGES) & 1) ^ 1, p.err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(full_p(s), PA_BYTES + PB_BYTES);
                    tma_load_3d(sbase + OFF_PA + s * PA_BYTES, tc.ma, kp * (KP / 64), tc.tm * BM,
                                tc.leaf, full_p(s));
                    tma_load_3d(sbase + OFF_PB + s * PB_BYTES, tc.mb, kp * (KP / 64), tc.tn * BN,
                                tc.leaf, full_p(s));
                }
            }
            // drain: the copies of the last issued stages must land before exit
            for (int j = 1; j <= PSTAGES && j <= pit; j++) {
                const int i = pit - j;
                if (!mbar_wait(full_p(i % PSTAGES), (i / PSTAGES) & 1, p.err)) break;
            }
        }
    } else if (warp < BEXP_WARPS) {
        // ---------------------------------------------------- Bt expansion (shared)
        // Per packed stage: 64 items of 4 rows x 8 packed words (both operand
        // stages). Lane = (half h, row rr of the item, word wl of the half):
        // word w = 4h + wl of the row goes to operand stage 2*pit + h. A
        // quarter-warp then holds two adjacent rows (opposite parity) x 4 words
        // of one half, whose swizzled 16-byte chunks are 8 distinct bank groups.
        const int h = lane >> 4, rr = (lane >> 2) & 3, wl = lane & 3;
        const Spread sp = p.sp;
        const int total_pit = total_it / SUB;
        static_assert(SUB == 2, "a packed stage feeds two operand stages");
        for (int pit = 0; pit < total_pit; pit++) {
            const int s = pit % PSTAGES;
            const int it0 = pit * SUB;
            const int se0 = it0 % ESTAGES, se1 = (it0 + 1) % ESTAGES;
            if (!mbar_wait(full_p(s), (pit / PSTAGES) & 1, p.err) ||
                !mbar_wait(empty_e(se1), (((it0 + 1) / ESTAGES) & 1) ^ 1, p.err))
                break;
            constexpr int ITEMS = (BN / 4) / BEXP_WARPS;
            const uint32_t* pb = reinterpret_cast<const uint32_t*>(smem + OFF_PB + s * PB_BYTES);
            uint8_t* eb = smem + OFF_EB + (h ? se1 : se0) * EB_BYTES;
            uint32_t x[ITEMS];
#pragma unroll
            for (int q = 0; q < ITEMS; q++)
                x[q] = pb[((warp + BEXP_WARPS * q) * 4 + rr) * 8 + 4 * h + wl];
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_p(s));
#pragma unroll
            for (int q = 0; q < ITEMS; q++) {
                const int row = (warp + BEXP_WARPS * q) * 4 + rr;
                uint8_t* rowp = eb + row * 128;
                uint32_t y[8];
                spread8(x[q], sp, y);
                *reinterpret_cast<uint4*>(rowp + (((2 * wl) ^ (row & 7)) * 16)) =
                    make_uint4(y[0], y[1], y[2], y[3]);
                *reinterpret_cast<uint4*>(rowp + (((2 * wl + 1) ^ (row & 7)) * 16)) =
                    make_uint4(y[4], y[5], y[6], y[7]);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(full_e(se0));
                mbar_arrive(full_e(se1));
            }
        }
    } else if (warp < EPI_WARP0) {
        // ---------------------------------------------------- A expansion (TMEM)
        const int quarter = warp & 3;
        const int parity = (warp - AEXP_WARP0) >> 2;  // this warp takes packed stages pit % 2 == parity
        const int row = 32 * quarter + lane;
        const Spread sp = p.sp;
        const uint32_t tlane = (uint32_t)(32 * quarter) << 16;
        const int total_pit = total_it / SUB;
        for (int pit = parity; pit < total_pit; pit += 2) {
            const int s = pit % PSTAGES;
            const int it0 = pit * SUB;
            const int se0 = it0 % ESTAGES, se1 = (it0 + 1) % ESTAGES;
            if (!mbar_wait(full_p(s), (pit / PSTAGES) & 1, p.err))
                break;
            const uint4* src = reinterpret_cast<const uint4*>(smem + OFF_PA + s * PA_BYTES +
                                                              row * (KP / 8));
            const uint4 xa = src[0], xb = src[1];
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_p(s));
            uint32_t y[32];
            if (!mbar_wait(empty_e(se1), (((it0 + 1) / ESTAGES) & 1) ^ 1, p.err)) break;
            spread8(xa.x, sp, y);
            spread8(xa.y, sp, y + 8);
            spread8(xa.z, sp, y + 16);
            spread8(xa.w, sp, y + 24);
            tmem_st32(tmem + tlane + (uint32_t)(A_COL + se0 * A_STAGE_COLS), y);
            spread8(xb.x, sp, y);
            spread8(xb.y, sp, y + 8);
            spread8(xb.z, sp, y + 16);
            spread8(xb.w, sp, y + 24);
            tmem_st32(tmem + tlane + (uint32_t)(A_COL + se1 * A_STAGE_COLS), y);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(full_e(se0));
                mbar_arrive(full_e(se1));
            }
        }
    } else if (warp == MMA_WARP) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(1u);
            uint64_t db0[ESTAGES];
#pragma unroll
            for (int s = 0; s < ESTAGES; s++) db0[s] = smem_desc_sw128(sbase + OFF_EB + s * EB_BYTES);
            int seg = 0, pit = 0;
            bool ok = true;
            for (int i = 0; ok && i < my_tiles; i++) {
                const int nks = tile_nks<BATCHED>(p, i);
                int kin = 0;
                for (int ks = 0; ks < nks; ks += SUB, pit++) {
                    if (kin == 0) {
                        if (!mbar_wait(acc_empty, (seg & 1) ^ 1, p.err)) {
                            ok = false;
                            break;
                        }
                    }
                    const int it0 = pit * SUB;
                    if (!mbar_wait(full_e((it0 + 1) % ESTAGES), ((it0 + 1) / ESTAGES) & 1, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int sub = 0; sub < SUB; sub++) {
                        const int se = (it0 + sub) % ESTAGES;
                        const uint32_t ta = tmem + (uint32_t)(A_COL + se * A_STAGE_COLS);
                        uint64_t db = db0[0];
#pragma unroll
                        for (int s = 1; s < ESTAGES; s++)
                            if (se == s) db = db0[s];
#pragma unroll
                        for (int j = 0; j < KS / MMA_K; j++)
                            mma_f8_ta(tmem + ACC_COL, ta + j * (MMA_K / 4), db + 2 * j, idesc,
                                      (kin > 0 || sub > 0 || j > 0) ? 1u : 0u);
                        mma_commit(empty_e(se));
                    }
                    kin += SUB;
                    if (kin >= kchunk || ks + SUB >= nks) {
                        mma_commit(acc_full);
                        seg++;
                        kin = 0;
                    }
                }
            }
            if (!ok) {  // wait (bounded) for every MMA this thread issued
                mma_commit(drain_bar);
                mbar_wait(drain_bar, 0, p.err);
            }
        }
    } else if (warp < TMA_WARP) {
        // ---------------------------------------------------- epilogue
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
        const uint32_t tlane = (uint32_t)(32 * quarter) << 16;
        int seg = 0;
        bool ok = true;
        for (int i = 0; ok && i < my_tiles; i++) {
            const Tile tc = tile_get<BATCHED>(p, i, &tmA, &tmB);
            const int nseg = (tc.nks + kchunk - 1) / kchunk;
            const bool gf2 = tc.op == OP_GF2;
            uint32_t words[BN / 32];
#pragma unroll
            for (int c = 0; c < BN / 32; c++) words[c] = 0u;
            for (int g = 0; g < nseg; g++, seg++) {
                if (!mbar_wait(acc_full, seg & 1, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll 2
                for (int c = 0; c < BN / 32; c++) {
                    uint32_t v[32];
                    tmem_ld32(tmem + tlane + (uint32_t)(ACC_COL + 32 * c), v);
                    if (gf2)
                        words[c] ^= pack_bits<OP_GF2>(v);
                    else
                        words[c] |= pack_bits<OP_BOOL>(v);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
            }
            if (!ok) break;
            const int64_t row = (int64_t)tc.tm * BM + 32 * quarter + lane;
            if (row < tc.m) {
                uint64_t* crow = tc.C + row * tc.ldc;
                const int64_t w0 = (int64_t)tc.tn * (BN / 64);
                const int64_t nw = tc.n / 64;
#pragma unroll
                for (int c = 0; c < BN / 64; c++)
                    if (w0 + c < nw)
                        crow[w0 + c] = (uint64_t)words[2 * c] | ((uint64_t)words[2 * c + 1] << 32);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
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

// 3-D map over uint64 words: (k/64 words, rows, leaves), box (KP/64, box_rows, 1).
// Boxes that run past k or the rows are zero-filled, which adds nothing to
// the counts.
bool make_map(CUtensorMap* map, const uint64_t* base, int64_t kwords, int64_t rows,
              int64_t pitch, int64_t count, int64_t stride, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kwords, (cuuint64_t)rows, (cuuint64_t)count};
    const int64_t leaf_stride = count > 1 ? stride : rows * pitch;
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * 8), (cuuint64_t)(leaf_stride * 8)};
    cuuint32_t box[3] = {(cuuint32_t)(KP / 64), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)base, dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <bool BATCHED>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const Params& prm, int grid,
                      cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_nt_kernel<BATCHED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tc_nt_kernel<BATCHED><<<grid, THREADS, SMEM_BYTES, s>>>(ma, mb, prm);
    return cudaGetLastError();
}

Spread spread_factors() {
    Spread sp;
    for (int j = 0; j < 8; j++) sp.f[j] = j <= 3 ? (1u << (3 - j)) : (1u << (35 - j));
    return sp;
}

}  // namespace

bool tc_path_available() { return device_cc() == 103 && encode_fn() != nullptr; }

// Longest run of k stages accumulated before the counts are flushed from
// TMEM: the e4m3 path reads parity through an FP32 value count * 2^-12,
// exact while count < 2^23 (at most 65534 stages of 128); S32 needs none.
int tc_kchunk_stages(int path, int nks) {
    // a multiple of the operand stages per packed stage (flushes happen between packed stages)
    const int cap = 65534;
    if (path == BMM_PATH_TC_FP8) return nks < cap ? nks : cap;
    return nks;
}

bmm_status run_tc_strided(int op, int path, const uint64_t* A, int64_t lda, int64_t strideA,
                          const uint64_t* Bt, int64_t ldb, int64_t strideB, uint64_t* C,
                          int64_t ldc, int64_t strideC, int64_t count, int64_t m, int64_t k,
                          int64_t n, cudaStream_t s) {
    if (!tc_path_available() || path != BMM_PATH_TC_FP8) return BMM_ERR_UNSUPPORTED;
    if (k % KS || (lda & 1) || (ldb & 1) || (count > 1 && ((strideA & 1) || (strideB & 1))))
        return BMM_ERR_UNSUPPORTED;
    if (m <= 0 || n <= 0 || k <= 0 || count <= 0) return BMM_OK;
    uint32_t* err = device_error_word();
    if (!err) return BMM_ERR_NOMEM;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, k / 64, m, lda, count, strideA, BM) ||
        !make_map(&mb, Bt, k / 64, n, ldb, count, strideB, BN))
        return BMM_ERR_CUDA;
    Params prm{};
    prm.C = C;
    prm.ldc = ldc;
    prm.strideC = strideC;
    prm.m = (int)m;
    prm.n = (int)n;
    prm.nks = (int)((k + KP - 1) / KP) * SUB;  // whole packed stages; the tail is zero-filled
    prm.op = op;
    prm.kchunk = tc_kchunk_stages(path, prm.nks);
    prm.tiles_m = (int)((m + BM - 1) / BM);
    prm.tiles_n = (int)((n + BN - 1) / BN);
    const int64_t total = (int64_t)prm.tiles_m * prm.tiles_n * count;
    if (total > 0x7fffffff) return BMM_ERR_UNSUPPORTED;
    prm.total_tiles = (int)total;
    prm.err = err;
    prm.sp = spread_factors();
    TraceScope ts(BMM_PHASE_BASE, s);
    const int grid = prm.total_tiles < sm_count() ? prm.total_tiles : sm_count();
    const cudaError_t e = launch_tc<false>(ma, mb, prm, grid, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return BMM_OK;
}

}  // namespace bmm

namespace bmm {

bool tc_make_problem(TcProblem* out, const uint64_t* A, int64_t lda, const uint64_t* Bt,
                     int64_t ldb, uint64_t* C, int64_t ldc, int64_t m, int64_t k, int64_t n,
                     int op) {
    if (k % KS || (lda & 1) || (ldb & 1)) return false;
    if (!make_map(&out->mapA, A, k / 64, m, lda, 1, 0, BM) ||
        !make_map(&out->mapB, Bt, k / 64, n, ldb, 1, 0, BN))
        return false;
    out->C = C;
    out->ldc = ldc;
    out->m = (int32_t)m;
    out->n = (int32_t)n;
    out->nks = (int32_t)(((k + KP - 1) / KP) * SUB);
    out->op = op;
    return true;
}

cudaError_t tc_launch_batched(const TcProblem* d_probs, const TcWorkItem* d_items,
                              const int32_t* d_cta_ptr, int grid, cudaStream_t s) {
    uint32_t* err = device_error_word();
    if (!err) return cudaErrorMemoryAllocation;
    Params prm{};
    prm.probs = d_probs;
    prm.items = d_items;
    prm.cta_ptr = d_cta_ptr;
    prm.kchunk = 65534;
    prm.err = err;
    prm.sp = spread_factors();
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    TraceScope ts(BMM_PHASE_BASE, s);
    return launch_tc<true>(dummy, dummy, prm, grid, s);
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
