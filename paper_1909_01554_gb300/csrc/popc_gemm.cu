// CUDA-core base-case block product (Sec. 3.10 inner layer; Sec. 3.18 for the
// Boolean variant), in the "NT" form C = A * Bt^T with both operands packed
// along k.
//
// Per 32-bit word of k, one LOP3 computes acc = acc XOR (a AND b) for the
// binary product, or acc = acc OR (a AND b) for the Boolean product: 32 ANDs
// and 32 XORs/ORs, 64 bit operations per lane instruction. After the k loop
// the binary result is the parity of acc (POPC), the Boolean result is
// acc != 0 (the paper's popcount-parity check and nonzero test, Sec. 4).
//
// Tiling: a CTA of 256 threads owns a 128 x 128 tile of C; thread (tx, ty)
// accumulates rows ty + 16 i and columns tx + 16 j (i, j < 8), 64 independent
// 32-bit accumulators. k advances 256 bits per stage through a 3-stage
// cp.async ring in shared memory; each thread reads its operands with 128-bit
// shared loads (4 words of k), so the inner loop is 64 LOP3 per 4 shared
// loads of 16 bytes. Rows are padded to 48 bytes, which keeps every
// quarter-warp's 128-bit loads on distinct banks. The epilogue gathers the
// result bits of a warp with ballots and writes whole 64-bit words.
#include <algorithm>
#include <mutex>

#include "internal.h"

namespace bmm {
namespace {

constexpr int BM = 128, BN = 128;
constexpr int KW64 = 4;    // 64-bit words of k per stage (256 bits)
constexpr int LD = 12;     // padded shared row in 32-bit words (48 bytes)
constexpr int STAGES = 3;
constexpr int MAX_DEVICES = 64;  // per-device one-time kernel attributes
constexpr int SMEM_BYTES = STAGES * (BM + BN) * LD * 4;
// The in-kernel level: double-buffered operand tiles, and a ring of raw
// quadrant words (2 words x 2 operands x 4 quadrants per thread and stage).
constexpr int LEVEL_STAGES = 2;
constexpr int RAW_SLOTS = 3;
constexpr int LEVEL_SMEM_BYTES = LEVEL_STAGES * (BM + BN) * LD * 4 + RAW_SLOTS * 2 * 2 * 4 * 256 * 8;

// 64-bit words of a stage row (KW64) that one thread copies: VW = 2 (16-byte
// copies, two threads per row) where every copied pair is 16-byte aligned,
// else VW = 1 (8-byte copies, four threads per row, two rows per thread).
template <int VW>
struct LevelMap {
    static constexpr int TPR = KW64 / VW;   // threads per stage row
    static constexpr int U = TPR / 2;       // rows per thread (256 threads, 128 rows)
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One k stage of the CTA's tile: 2 x 4 words of k per thread, 64 LOP3 per
// four 16-byte shared loads per operand row.
template <int OP>
__device__ __forceinline__ void tile_stage(const uint32_t* a_s, const uint32_t* b_s, int tx, int ty,
                                           uint32_t (&acc)[8][8]) {
#pragma unroll
    for (int kk = 0; kk < 2 * KW64; kk += 4) {
        uint4 a[8], b[8];
#pragma unroll
        for (int i = 0; i < 8; i++)
            a[i] = *reinterpret_cast<const uint4*>(&a_s[(ty + 16 * i) * LD + kk]);
#pragma unroll
        for (int j = 0; j < 8; j++)
            b[j] = *reinterpret_cast<const uint4*>(&b_s[(tx + 16 * j) * LD + kk]);
#pragma unroll
        for (int i = 0; i < 8; i++)
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (OP == OP_GF2) {
                    acc[i][j] ^= a[i].x & b[j].x;
                    acc[i][j] ^= a[i].y & b[j].y;
                    acc[i][j] ^= a[i].z & b[j].z;
                    acc[i][j] ^= a[i].w & b[j].w;
                } else {
                    acc[i][j] |= a[i].x & b[j].x;
                    acc[i][j] |= a[i].y & b[j].y;
                    acc[i][j] |= a[i].z & b[j].z;
                    acc[i][j] |= a[i].w & b[j].w;
                }
            }
    }
}

// Epilogue gather. Lanes 0-15 of a warp hold row ty0 = 2*warp, lanes 16-31
// row ty0+1; lane tx holds column tx + 16 j. One ballot per (i, j) yields 16
// bits of two rows; lane L keeps the 64-bit word (i = L/4, row half (L/2)%2,
// word L%2) of the tile, at tile row 2*warp + half + 16*i, tile word L%2.
template <int OP>
__device__ __forceinline__ uint64_t tile_word(const uint32_t (&acc)[8][8], int lane) {
    uint64_t myword = 0;
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const bool bit = (OP == OP_GF2) ? ((__popc(acc[i][j]) & 1) != 0) : (acc[i][j] != 0u);
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            const int w = j >> 2, sh = 16 * (j & 3);
            if (lane == i * 4 + 0 + w) myword |= (uint64_t)(bal & 0xffffu) << sh;
            if (lane == i * 4 + 2 + w) myword |= (uint64_t)(bal >> 16) << sh;
        }
    return myword;
}

// One 128 x 128 tile of C (rows row0.., columns col0..) = A * Bt^T over the
// whole of k: the cp.async ring, the LOP3 loop and the ballot epilogue.
template <int OP>
__device__ __forceinline__ void popc_tile(const uint64_t* __restrict__ A, int64_t lda,
                                          const uint64_t* __restrict__ Bt, int64_t ldb,
                                          uint64_t* __restrict__ C, int64_t ldc, int64_t m,
                                          int64_t k, int64_t n, int64_t row0, int64_t col0,
                                          uint32_t* smem) {
    uint32_t* sA = smem;                      // [STAGES][BM][LD]
    uint32_t* sB = smem + STAGES * BM * LD;   // [STAGES][BN][LD]

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t kwords = k / 64;
    const int nk = (int)((kwords + KW64 - 1) / KW64);

    auto load_stage = [&](int s, int kt) {
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int c = tid + q * 256;  // 512 chunks of 8 bytes per operand
            const int r = c >> 2, w = c & 3;
            const int64_t kw = (int64_t)kt * KW64 + w;
            const bool okk = kw < kwords;
            {
                const bool ok = okk && (row0 + r < m);
                const uint64_t* src = ok ? A + (row0 + r) * lda + kw : A;
                cp_async8(&sA[(s * BM + r) * LD + 2 * w], src, ok ? 8 : 0);
            }
            {
                const bool ok = okk && (col0 + r < n);
                const uint64_t* src = ok ? Bt + (col0 + r) * ldb + kw : Bt;
                cp_async8(&sB[(s * BN + r) * LD + 2 * w], src, ok ? 8 : 0);
            }
        }
    };

    uint32_t acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0u;

#pragma unroll
    for (int s = 0; s < STAGES - 1; s++) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }

    for (int kt = 0; kt < nk; kt++) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nt = kt + STAGES - 1;
            if (nt < nk) load_stage(nt % STAGES, nt);
            cp_async_commit();
        }
        tile_stage<OP>(sA + (kt % STAGES) * BM * LD, sB + (kt % STAGES) * BN * LD, tx, ty, acc);
    }
    cp_async_wait<0>();

    const int warp = tid >> 5, lane = tid & 31;
    const uint64_t myword = tile_word<OP>(acc, lane);
    {
        const int i = lane >> 2, half = (lane >> 1) & 1, w = lane & 1;
        const int64_t row = row0 + 2 * warp + half + 16 * i;
        const int64_t cw = col0 / 64 + w;
        if (row < m && cw < n / 64) C[row * ldc + cw] = myword;
    }
}

template <int OP>
__global__ void __launch_bounds__(256, 1)
    popc_nt_kernel(const uint64_t* __restrict__ A, int64_t lda, int64_t strideA,
                   const uint64_t* __restrict__ Bt, int64_t ldb, int64_t strideB,
                   uint64_t* __restrict__ C, int64_t ldc, int64_t strideC, int64_t m, int64_t k,
                   int64_t n) {
    extern __shared__ __align__(16) uint32_t smem[];
    popc_tile<OP>(A + (int64_t)blockIdx.z * strideA, lda, Bt + (int64_t)blockIdx.z * strideB, ldb,
                  C + (int64_t)blockIdx.z * strideC, ldc, m, k, n, (int64_t)blockIdx.y * BM,
                  (int64_t)blockIdx.x * BN, smem);
}

// Products of uneven sizes in one persistent launch: CTA b takes tiles b,
// b + gridDim.x, ... of the list (ordered longest first by the planner), each
// a 128 x 128 tile of one problem's C over that problem's whole k.
__global__ void __launch_bounds__(256, 1)
    popc_batched_kernel(const PopcJob* __restrict__ jobs, const PopcTile* __restrict__ tiles,
                        int64_t count) {
    extern __shared__ __align__(16) uint32_t smem[];
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const PopcTile w = tiles[t];
        const PopcJob j = jobs[w.job];
        __syncthreads();  // the previous tile's last stage has been read by every thread
        if (j.op == OP_GF2)
            popc_tile<OP_GF2>(j.A, j.lda, j.Bt, j.ldb, j.C, j.ldc, j.m, j.k, j.n,
                              (int64_t)w.tm * BM, (int64_t)w.tn * BN, smem);
        else
            popc_tile<OP_BOOL>(j.A, j.lda, j.Bt, j.ldb, j.C, j.ldc, j.m, j.k, j.n,
                               (int64_t)w.tm * BM, (int64_t)w.tn * BN, smem);
    }
}

// One Strassen level inside the kernel (a level shifted from the expanding
// and compressing layers into the inner layer, Sec. 3.15): the binary
// product C (2hm x 2hn) = A (2hm x 2hk) * Bt (2hn x 2hk)^T of one block,
// through its seven quadrant-sized products. The CTA owns one 128 x 128
// tile position of the quadrant-sized product and runs the seven products
// there one after the other. Product h reads, per word of k, the quadrants
// of A that xi_h selects and the quadrants of B that eta_h selects and XORs
// them as they are staged (the combined input operators xi = alpha phi and
// eta = beta psi of one level), so its operands never exist in HBM. Its
// result bits are XORed into each C quadrant that zeta = chi gamma sends it
// to, in registers; the four quadrant words leave once, after the seventh
// product.
//
// Staging: each thread copies its own words of every selected quadrant with
// cp.async into a ring of RAW_SLOTS stages laid out per thread (consecutive
// threads, consecutive words: conflict-free), two stages ahead of the
// compute; once its own copies of a stage have landed (wait_group, no
// barrier needed), it XORs them and stores the combined words into the
// double-buffered operand tile that the LOP3 loop reads. The source
// addresses are formed once per product and advance by one stage per step.
template <int VW>
__global__ void __launch_bounds__(256, 1)
    popc_level_kernel(const uint64_t* __restrict__ A, int64_t lda, int64_t strideA,
                      const uint64_t* __restrict__ Bt, int64_t ldb, int64_t strideB,
                      uint64_t* __restrict__ C, int64_t ldc, int64_t strideC, int64_t hm,
                      int64_t hk, int64_t hn, uint32_t xi4, uint32_t eta4, uint32_t zeta7) {
    using LM = LevelMap<VW>;
    constexpr int U = LM::U, TPR = LM::TPR;
    A += (int64_t)blockIdx.z * strideA;
    Bt += (int64_t)blockIdx.z * strideB;
    C += (int64_t)blockIdx.z * strideC;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* sA = smem;                           // [LEVEL_STAGES][BM][LD]
    uint32_t* sB = smem + LEVEL_STAGES * BM * LD;  // [LEVEL_STAGES][BN][LD]
    // [RAW_SLOTS][U][2 operands][4 quadrants][256 threads][VW words]
    uint64_t* raw = reinterpret_cast<uint64_t*>(smem + LEVEL_STAGES * (BM + BN) * LD);
    static_assert(U * VW == 2, "the ring holds two words per thread, operand and quadrant");

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;
    const int64_t hkw = hk / 64;  // words of k per quadrant
    const int nk = (int)((hkw + KW64 - 1) / KW64);
    auto raw_at = [&](int slot, int u, int op, int q) {
        return raw + (((((slot * U + u) * 2 + op) * 4 + q) * 256 + tid) * VW);
    };

    // This thread's rows r and first words w of every stage, and its first
    // source word in each quadrant: A block (i, j) at rows i*hm, words j*hkw;
    // B block (i, j) is stored transposed in Bt, at rows j*hn, words i*hkw
    // (block q = 2i + j). Rows past the block read nothing.
    int rr[U], ww[U];
    bool rowa[U], rowb[U];
    const uint64_t* pa[U][4];
    const uint64_t* pb[U][4];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int c = tid + u * 256;
        rr[u] = c / TPR;
        ww[u] = (c % TPR) * VW;
        rowa[u] = row0 + rr[u] < hm;
        rowb[u] = col0 + rr[u] < hn;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            pa[u][q] = rowa[u] ? A + (row0 + rr[u] + (q >> 1) * hm) * lda + (q & 1) * hkw + ww[u]
                               : A;
            pb[u][q] = rowb[u] ? Bt + (col0 + rr[u] + (q & 1) * hn) * ldb + (q >> 1) * hkw + ww[u]
                               : Bt;
        }
    }

    uint64_t out[4] = {0, 0, 0, 0};  // this thread's word of each C quadrant
    for (int h = 0; h < 7; h++) {
        const uint32_t xa = (xi4 >> (4 * h)) & 0xFu, xb = (eta4 >> (4 * h)) & 0xFu;
        // this thread's words of every selected quadrant of stage kt, copied
        // into ring slot kt % RAW_SLOTS
        auto issue = [&](int kt) {
            const int slot = kt % RAW_SLOTS;
            const int64_t adv = (int64_t)kt * KW64;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const bool kv = adv + ww[u] < hkw;
                const bool oka = kv && rowa[u], okb = kv && rowb[u];
                const int bytes_a = oka ? 8 * VW : 0, bytes_b = okb ? 8 * VW : 0;
                // a copy that reads nothing still gets an address inside the
                // operand (its base)
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if ((xa >> q) & 1u) {
                        const uint64_t* src = oka ? pa[u][q] + adv : A;
                        if (VW == 2)
                            cp_async16(raw_at(slot, u, 0, q), src, bytes_a);
                        else
                            cp_async8(raw_at(slot, u, 0, q), src, bytes_a);
                    }
                    if ((xb >> q) & 1u) {
                        const uint64_t* src = okb ? pb[u][q] + adv : Bt;
                        if (VW == 2)
                            cp_async16(raw_at(slot, u, 1, q), src, bytes_b);
                        else
                            cp_async8(raw_at(slot, u, 1, q), src, bytes_b);
                    }
                }
            }
        };
        // stage kt's words (landed) XORed into operand buffer `buf`
        auto combine = [&](int kt, int buf) {
            const int slot = kt % RAW_SLOTS;
#pragma unroll
            for (int u = 0; u < U; u++) {
                uint64_t a[VW], b[VW];
#pragma unroll
                for (int v = 0; v < VW; v++) a[v] = b[v] = 0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if ((xa >> q) & 1u) {
                        const uint64_t* x = raw_at(slot, u, 0, q);
                        if (VW == 2) {
                            const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(x);
                            a[0] ^= t.x;
                            a[VW - 1] ^= t.y;
                        } else {
                            a[0] ^= x[0];
                        }
                    }
                    if ((xb >> q) & 1u) {
                        const uint64_t* x = raw_at(slot, u, 1, q);
                        if (VW == 2) {
                            const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(x);
                            b[0] ^= t.x;
                            b[VW - 1] ^= t.y;
                        } else {
                            b[0] ^= x[0];
                        }
                    }
                }
                uint32_t* da = &sA[(buf * BM + rr[u]) * LD + 2 * ww[u]];
                uint32_t* db = &sB[(buf * BN + rr[u]) * LD + 2 * ww[u]];
                if (VW == 2) {
                    *reinterpret_cast<ulonglong2*>(da) = make_ulonglong2(a[0], a[VW - 1]);
                    *reinterpret_cast<ulonglong2*>(db) = make_ulonglong2(b[0], b[VW - 1]);
                } else {
                    *reinterpret_cast<uint64_t*>(da) = a[0];
                    *reinterpret_cast<uint64_t*>(db) = b[0];
                }
            }
        };

        uint32_t acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; i++)
#pragma unroll
            for (int j = 0; j < 8; j++) acc[i][j] = 0u;
        // Every copy group of the previous product has been waited for, and
        // its last stage ended at a barrier: the ring and buffer 0 are free.
        issue(0);
        cp_async_commit();
        if (nk > 1) issue(1);
        cp_async_commit();
        cp_async_wait<1>();  // stage 0
        combine(0, 0);
        __syncthreads();
        for (int kt = 0; kt < nk; kt++) {
            // slot (kt+2) % RAW_SLOTS held stage kt-1, combined in the
            // previous iteration by this same thread
            if (kt + 2 < nk) issue(kt + 2);
            cp_async_commit();
            tile_stage<OP_GF2>(sA + (kt & 1) * BM * LD, sB + (kt & 1) * BN * LD, tx, ty, acc);
            if (kt + 1 < nk) {
                cp_async_wait<1>();  // stage kt+1 (only stage kt+2 may be in flight)
                // buffer (kt+1)&1 was last read in stage kt-1, which every
                // thread finished before the barrier that ended it
                combine(kt + 1, (kt + 1) & 1);
            }
            __syncthreads();
        }
        const uint64_t word = tile_word<OP_GF2>(acc, lane);
#pragma unroll
        for (int q = 0; q < 4; q++)
            if ((zeta7 >> (7 * q + h)) & 1u) out[q] ^= word;
    }
    {
        const int i = lane >> 2, half = (lane >> 1) & 1, w = lane & 1;
        const int64_t row = row0 + 2 * warp + half + 16 * i;
        const int64_t cw = col0 / 64 + w;
        const int64_t hnw = hn / 64;
        if (row < hm && cw < hnw) {
#pragma unroll
            for (int q = 0; q < 4; q++)
                C[((q >> 1) * hm + row) * ldc + (q & 1) * hnw + cw] = out[q];
        }
    }
}

template <int VW>
cudaError_t level_attr() {
    static bool done[MAX_DEVICES] = {false};
    static cudaError_t err[MAX_DEVICES];
    static std::mutex mu;
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAX_DEVICES)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[d]) {
        err[d] = cudaFuncSetAttribute(popc_level_kernel<VW>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      LEVEL_SMEM_BYTES);
        done[d] = true;
    }
    return err[d];
}

}  // namespace

cudaError_t launch_popc_nt(int op, const uint64_t* A, int64_t lda, int64_t strideA,
                           const uint64_t* Bt, int64_t ldb, int64_t strideB, uint64_t* C,
                           int64_t ldc, int64_t strideC, int64_t count, int64_t m, int64_t k,
                           int64_t n, cudaStream_t s) {
    const int64_t gx = (n + BN - 1) / BN, gy = (m + BM - 1) / BM;
    if (gx <= 0 || gy <= 0 || count <= 0) return cudaSuccess;
    if (gy > 65535 || count > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)count);
    static_assert(SMEM_BYTES <= 48 * 1024, "fits the default dynamic shared memory limit");
    TraceScope ts(BMM_PHASE_BASE, s);
    if (op == OP_GF2)
        popc_nt_kernel<OP_GF2><<<grid, 256, SMEM_BYTES, s>>>(A, lda, strideA, Bt, ldb, strideB, C,
                                                             ldc, strideC, m, k, n);
    else
        popc_nt_kernel<OP_BOOL><<<grid, 256, SMEM_BYTES, s>>>(A, lda, strideA, Bt, ldb, strideB,
                                                              C, ldc, strideC, m, k, n);
    return cudaGetLastError();
}

int popc_batched_grid() {
    static int grid[MAX_DEVICES] = {0};
    static std::mutex mu;
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAX_DEVICES) return sm_count();
    std::lock_guard<std::mutex> lk(mu);
    if (!grid[d]) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, popc_batched_kernel, 256,
                                                          SMEM_BYTES) != cudaSuccess ||
            per < 1) {
            (void)cudaGetLastError();
            per = 1;
        }
        grid[d] = per * sm_count();
    }
    return grid[d];
}

cudaError_t launch_popc_batched(const PopcJob* jobs, const PopcTile* tiles, int64_t count,
                                cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int64_t g = std::min<int64_t>(count, popc_batched_grid());
    TraceScope ts(BMM_PHASE_BASE, s);
    popc_batched_kernel<<<(unsigned)g, 256, SMEM_BYTES, s>>>(jobs, tiles, count);
    return cudaGetLastError();
}

cudaError_t launch_popc_level(const uint64_t* A, int64_t lda, int64_t strideA, const uint64_t* Bt,
                              int64_t ldb, int64_t strideB, uint64_t* C, int64_t ldc,
                              int64_t strideC, int64_t count, int64_t m, int64_t k, int64_t n,
                              const LevelMasks& masks, cudaStream_t s) {
    if (m % 2 || k % 128 || n % 128) return cudaErrorInvalidValue;
    const int64_t hm = m / 2, hk = k / 2, hn = n / 2;
    const int64_t gx = (hn + BN - 1) / BN, gy = (hm + BM - 1) / BM;
    if (gx <= 0 || gy <= 0 || count <= 0) return cudaSuccess;
    if (gy > 65535 || count > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)count);
    static_assert(LEVEL_SMEM_BYTES <= 227 * 1024, "fits one CTA's shared memory");
    // 16-byte copies where every copied word pair starts 16-byte aligned:
    // even pitches, even quadrant widths, 16-byte aligned bases and strides
    const bool wide = hk / 64 % 2 == 0 && lda % 2 == 0 && ldb % 2 == 0 && strideA % 2 == 0 &&
                      strideB % 2 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)Bt % 16 == 0;
    cudaError_t e = wide ? level_attr<2>() : level_attr<1>();
    if (e != cudaSuccess) return e;
    // the masks packed into three words: nibble h of xi4 / eta4 = xi[h] /
    // eta[h]; bits 7q..7q+6 of zeta7 = zeta[q]
    uint32_t xi4 = 0, eta4 = 0, zeta7 = 0;
    for (int h = 0; h < 7; h++) {
        xi4 |= (masks.xi[h] & 0xFu) << (4 * h);
        eta4 |= (masks.eta[h] & 0xFu) << (4 * h);
    }
    for (int q = 0; q < 4; q++) zeta7 |= (masks.zeta[q] & 0x7Fu) << (7 * q);
    TraceScope ts(BMM_PHASE_BASE, s);
    if (wide)
        popc_level_kernel<2><<<grid, 256, LEVEL_SMEM_BYTES, s>>>(
            A, lda, strideA, Bt, ldb, strideB, C, ldc, strideC, hm, hk, hn, xi4, eta4, zeta7);
    else
        popc_level_kernel<1><<<grid, 256, LEVEL_SMEM_BYTES, s>>>(
            A, lda, strideA, Bt, ldb, strideB, C, ldc, strideC, hm, hk, hn, xi4, eta4, zeta7);
    return cudaGetLastError();
}

}  // namespace bmm
