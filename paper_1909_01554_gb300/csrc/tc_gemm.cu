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
// Persistent kernel, one CTA per SM, warp-specialised:
//   warp 12     TMA producer: packed 128 x 128-bit tiles of A and 256 x
//               128-bit tiles of Bt into a PSTAGES-deep shared ring
//               (cp.async.bulk.tensor, mbarrier complete_tx).
//   warps 0-7   expansion: each packed 32-bit word becomes 32 bytes of the
//               K-major, no-swizzle canonical UMMA layout (8-row x 16-byte
//               core matrices), into an ESTAGES-deep ring.
//   warp 13     MMA issuer: 4 x tcgen05.mma (M=128, N=256, K=32) per stage
//               into one of two TMEM accumulators (2 x 256 columns); commits
//               release operand stages and publish finished accumulators.
//   warps 8-11  epilogue: tcgen05.ld 32 lanes x 32 columns at a time, parity
//               or non-zero test, bits repacked in registers (one row per
//               thread) and stored as 64-bit words.
// The two accumulators let the epilogue of one tile overlap the main loop of
// the next; the same mechanism flushes long k in chunks (kchunk stages).
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

#include <mutex>

#include "plan.h"

namespace bmm {
namespace {

constexpr int BM = 128;          // rows of C per tile (UMMA M, TMEM lanes)
constexpr int BN = 256;          // columns of C per tile (UMMA N)
constexpr int KS = 128;          // k (bits) per stage
constexpr int MMA_K = 32;        // k per tcgen05.mma for 8-bit operands
constexpr int PSTAGES = 6;       // packed ring depth
constexpr int ESTAGES = 3;       // expanded ring depth
constexpr int EXP_WARPS = 8;
// warps 8..11: epilogue (warp % 4 = TMEM lane quarter)
constexpr int TMA_WARP = 12;
constexpr int MMA_WARP = 13;
constexpr int THREADS = 14 * 32;
constexpr int GROUP_M = 16;      // tile raster: 16 row-tiles per group

constexpr int PA_BYTES = BM * KS / 8;    // 2 KB packed A per stage
constexpr int PB_BYTES = BN * KS / 8;    // 4 KB packed Bt per stage
constexpr int EA_BYTES = BM * KS;        // 16 KB expanded A per stage
constexpr int EB_BYTES = BN * KS;        // 32 KB expanded Bt per stage
constexpr int TMEM_COLS = 2 * BN;        // two fp32/s32 accumulators

constexpr int OFF_EA = 0;
constexpr int OFF_EB = OFF_EA + ESTAGES * EA_BYTES;
constexpr int OFF_PA = OFF_EB + ESTAGES * EB_BYTES;
constexpr int OFF_PB = OFF_PA + PSTAGES * PA_BYTES;
constexpr int OFF_BAR = OFF_PB + PSTAGES * PB_BYTES;
// barriers: full_p[P], empty_p[P], full_e[E], empty_e[E], acc_full[2], acc_empty[2], drain
constexpr int NBARS = 2 * PSTAGES + 2 * ESTAGES + 5;
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
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, uint32_t* err) {
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; i++) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255u) == 0 && globaltimer() - t0 > WAIT_NS) {
            atomicOr(err, DEVERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* err) {
    if (mbar_try(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, err);
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// LBO = byte distance between core matrices adjacent along K, SBO = between
// core matrices adjacent along M/N (8-row groups).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    // base offset 0, relative LBO mode, swizzle none (bits 61-63 = 0)
    return d;
}

// Instruction descriptor for kind::f8f6f4: D format (1 = F32), A and B
// format 0 (E4M3), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t dfmt) {
    return (dfmt << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
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

// ---------------------------------------------------------------- expansion
// Packed word x holds 32 consecutive k of one row. Output word j (j = 0..7)
// gets bit (8t + j) of x in byte t, moved to bit T of that byte:
// T = 3 gives e4m3 0x08 = 2^-6, T = 0 gives u8 1.
template <int T, int J>
__device__ __forceinline__ uint32_t spread(uint32_t x) {
    constexpr uint32_t mask = 0x01010101u << T;
    if constexpr (T >= J)
        return (x << (T - J)) & mask;
    else
        return (x >> (J - T)) & mask;
}

template <int T>
__device__ __forceinline__ void expand_word(uint32_t x, uint32_t dst) {
    const uint32_t y0 = spread<T, 0>(x), y1 = spread<T, 1>(x), y2 = spread<T, 2>(x),
                   y3 = spread<T, 3>(x), y4 = spread<T, 4>(x), y5 = spread<T, 5>(x),
                   y6 = spread<T, 6>(x), y7 = spread<T, 7>(x);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(y0), "r"(y1), "r"(y2),
                 "r"(y3)
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + 128), "r"(y4), "r"(y5),
                 "r"(y6), "r"(y7)
                 : "memory");
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
    uint64_t* C;
    int64_t ldc, strideC;
    int m, n, nks, kchunk;  // kchunk: stages per accumulator flush
    int tiles_m, tiles_n, total_tiles;
    uint32_t* err;
};

template <int OP>
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
    auto acc_full = [&](int b) { return bar0 + 8u * (2 * PSTAGES + 2 * ESTAGES + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (2 * PSTAGES + 2 * ESTAGES + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * PSTAGES + 2 * ESTAGES + 4);
    uint32_t* tmem_slot = (uint32_t*)(smem + OFF_TMEM_SLOT);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; s++) {
            mbar_init(full_p(s), 1);
            mbar_init(empty_p(s), EXP_WARPS);
        }
        for (int s = 0; s < ESTAGES; s++) {
            mbar_init(full_e(s), EXP_WARPS);
            mbar_init(empty_e(s), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), 4);
        }
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
    if (warp == TMA_WARP && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA))
                     : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB))
                     : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int nks = p.nks;
    const int kchunk = p.kchunk;

    if (warp == TMA_WARP) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < p.total_tiles; t += gridDim.x) {
                const TileCoord tc = tile_of(t, p.tiles_m, p.tiles_n);
                for (int ks = 0; ks < nks; ks++, it++) {
                    const int s = it % PSTAGES;
                    if (!mbar_wait(empty_p(s), ((it / PSTAGES) & 1) ^ 1, p.err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(full_p(s), PA_BYTES + PB_BYTES);
                    tma_load_3d(sbase + OFF_PA + s * PA_BYTES, &tmA, ks * (KS / 64), tc.tm * BM,
                                tc.leaf, full_p(s));
                    tma_load_3d(sbase + OFF_PB + s * PB_BYTES, &tmB, ks * (KS / 64), tc.tn * BN,
                                tc.leaf, full_p(s));
                }
            }
            // drain: the copies of the last issued stages must land before exit
            for (int j = 1; j <= PSTAGES && j <= it; j++) {
                const int i = it - j;
                if (!mbar_wait(full_p(i % PSTAGES), (i / PSTAGES) & 1, p.err)) break;
            }
        }
    } else if (warp < EXP_WARPS) {
        // ---------------------------------------------------- expansion
        constexpr int TBIT = 3;  // e4m3 0x08
        const int ri = lane & 7, wq = lane >> 3;
        int it = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < p.total_tiles; t += gridDim.x) {
            for (int ks = 0; ks < nks; ks++, it++) {
                const int sp = it % PSTAGES, se = it % ESTAGES;
                if (!mbar_wait(full_p(sp), (it / PSTAGES) & 1, p.err) ||
                    !mbar_wait(empty_e(se), ((it / ESTAGES) & 1) ^ 1, p.err)) {
                    ok = false;
                    break;
                }
                const uint32_t pa = sbase + OFF_PA + sp * PA_BYTES;
                const uint32_t pb = sbase + OFF_PB + sp * PB_BYTES;
                const uint32_t ea = sbase + OFF_EA + se * EA_BYTES;
                const uint32_t eb = sbase + OFF_EB + se * EB_BYTES;
                // 48 row groups of 8 rows (16 of A, 32 of Bt); lane = (row in group, word)
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    const int g = warp + EXP_WARPS * q;
                    uint32_t src, dst;
                    if (g < BM / 8) {
                        src = pa + (g * 8 + ri) * (KS / 8) + wq * 4;
                        dst = ea + g * 1024 + (2 * wq) * 128 + ri * 16;
                    } else {
                        const int gb = g - BM / 8;
                        src = pb + (gb * 8 + ri) * (KS / 8) + wq * 4;
                        dst = eb + gb * 1024 + (2 * wq) * 128 + ri * 16;
                    }
                    uint32_t x;
                    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(x) : "r"(src) : "memory");
                    expand_word<TBIT>(x, dst);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty_p(sp));
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(full_e(se));
            }
        }
    } else if (warp == MMA_WARP) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(1u);
            int it = 0, seg = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < p.total_tiles; t += gridDim.x) {
                int b = 0;
                for (int ks = 0; ks < nks; ks++, it++) {
                    const int kin = ks % kchunk;
                    if (kin == 0) {
                        b = seg & 1;
                        if (!mbar_wait(acc_empty(b), ((seg >> 1) & 1) ^ 1, p.err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    const int se = it % ESTAGES;
                    if (!mbar_wait(full_e(se), (it / ESTAGES) & 1, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ea = sbase + OFF_EA + se * EA_BYTES;
                    const uint32_t eb = sbase + OFF_EB + se * EB_BYTES;
#pragma unroll
                    for (int j = 0; j < KS / MMA_K; j++) {
                        const uint64_t da = smem_desc(ea + j * 256, 128, 1024);
                        const uint64_t db = smem_desc(eb + j * 256, 128, 1024);
                        mma_f8(tmem + (uint32_t)(b * BN), da, db, idesc,
                               (kin > 0 || j > 0) ? 1u : 0u);
                    }
                    mma_commit(empty_e(se));
                    if (kin == kchunk - 1 || ks == nks - 1) {
                        mma_commit(acc_full(b));
                        seg++;
                    }
                }
            }
            if (!ok) {  // wait (bounded) for every MMA this thread issued
                mma_commit(drain_bar);
                mbar_wait(drain_bar, 0, p.err);
            }
        }
    } else {
        // ---------------------------------------------------- epilogue
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
        const int nseg = (nks + kchunk - 1) / kchunk;
        int seg = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < p.total_tiles; t += gridDim.x) {
            const TileCoord tc = tile_of(t, p.tiles_m, p.tiles_n);
            uint32_t words[BN / 32];
#pragma unroll
            for (int c = 0; c < BN / 32; c++) words[c] = 0u;
            for (int g = 0; g < nseg; g++, seg++) {
                const int b = seg & 1;
                if (!mbar_wait(acc_full(b), (seg >> 1) & 1, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < BN / 32; c++) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * BN + 32 * c),
                              v);
                    uint32_t wbits = 0;
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        // value = count * 2^-12, exact; + 2^11 puts count's LSB in bit 0
                        const uint32_t bit =
                            (OP == OP_GF2)
                                ? (__float_as_uint(__uint_as_float(v[j]) + 2048.0f) & 1u)
                                : (v[j] != 0u ? 1u : 0u);
                        wbits |= bit << j;
                    }
                    if (OP == OP_GF2)
                        words[c] ^= wbits;
                    else
                        words[c] |= wbits;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty(b));
            }
            if (!ok) break;
            const int64_t row = (int64_t)tc.tm * BM + 32 * quarter + lane;
            if (row < p.m) {
                uint64_t* crow = p.C + (int64_t)tc.leaf * p.strideC + row * p.ldc;
                const int64_t w0 = (int64_t)tc.tn * (BN / 64);
                const int64_t nw = p.n / 64;
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

// 3-D map over uint64 words: (k/64 words, rows, leaves), box (KS/64, box_rows, 1).
bool make_map(CUtensorMap* map, const uint64_t* base, int64_t kwords, int64_t rows,
              int64_t pitch, int64_t count, int64_t stride, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kwords, (cuuint64_t)rows, (cuuint64_t)count};
    const int64_t leaf_stride = count > 1 ? stride : rows * pitch;
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * 8), (cuuint64_t)(leaf_stride * 8)};
    cuuint32_t box[3] = {(cuuint32_t)(KS / 64), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void*)base, dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int OP>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const Params& prm,
                      cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_nt_kernel<OP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = prm.total_tiles < sm_count() ? prm.total_tiles : sm_count();
    tc_nt_kernel<OP><<<grid, THREADS, SMEM_BYTES, s>>>(ma, mb, prm);
    return cudaGetLastError();
}

}  // namespace

bool tc_path_available() { return device_cc() == 103 && encode_fn() != nullptr; }

// Longest run of k stages accumulated before the counts are flushed from
// TMEM: the e4m3 path reads parity through an FP32 value count * 2^-12,
// exact while count < 2^23 (at most 65535 stages of 128); S32 needs none.
int tc_kchunk_stages(int path, int nks) {
    if (path == BMM_PATH_TC_FP8) return nks < 65535 ? nks : 65535;
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
    Params prm;
    prm.C = C;
    prm.ldc = ldc;
    prm.strideC = strideC;
    prm.m = (int)m;
    prm.n = (int)n;
    prm.nks = (int)(k / KS);
    prm.kchunk = tc_kchunk_stages(path, prm.nks);
    prm.tiles_m = (int)((m + BM - 1) / BM);
    prm.tiles_n = (int)((n + BN - 1) / BN);
    const int64_t total = (int64_t)prm.tiles_m * prm.tiles_n * count;
    if (total > 0x7fffffff) return BMM_ERR_UNSUPPORTED;
    prm.total_tiles = (int)total;
    prm.err = err;
    TraceScope ts(BMM_PHASE_BASE, s);
    const cudaError_t e =
        (op == OP_GF2) ? launch_tc<OP_GF2>(ma, mb, prm, s) : launch_tc<OP_BOOL>(ma, mb, prm, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return BMM_OK;
}

}  // namespace bmm
