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
#include "internal.h"

namespace bmm {
namespace {

constexpr int BM = 128, BN = 128;
constexpr int KW64 = 4;    // 64-bit words of k per stage (256 bits)
constexpr int LD = 12;     // padded shared row in 32-bit words (48 bytes)
constexpr int STAGES = 3;
constexpr int SMEM_BYTES = STAGES * (BM + BN) * LD * 4;

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc),
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

template <int OP>
__global__ void __launch_bounds__(256, 1)
    popc_nt_kernel(const uint64_t* __restrict__ A, int64_t lda, int64_t strideA,
                   const uint64_t* __restrict__ Bt, int64_t ldb, int64_t strideB,
                   uint64_t* __restrict__ C, int64_t ldc, int64_t strideC, int64_t m, int64_t k,
                   int64_t n) {
    A += (int64_t)blockIdx.z * strideA;
    Bt += (int64_t)blockIdx.z * strideB;
    C += (int64_t)blockIdx.z * strideC;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* sA = smem;                      // [STAGES][BM][LD]
    uint32_t* sB = smem + STAGES * BM * LD;   // [STAGES][BN][LD]

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;
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
        const uint32_t* a_s = sA + (kt % STAGES) * BM * LD;
        const uint32_t* b_s = sB + (kt % STAGES) * BN * LD;
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
    cp_async_wait<0>();

    // Epilogue. Lanes 0-15 of a warp hold row ty0 = 2*warp, lanes 16-31 row ty0+1;
    // lane tx holds column tx + 16 j. One ballot per (i, j) yields 16 bits of two
    // rows; lane L keeps the 64-bit word (i = L/4, row half (L/2)%2, word L%2).
    const int warp = tid >> 5, lane = tid & 31;
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
    {
        const int i = lane >> 2, half = (lane >> 1) & 1, w = lane & 1;
        const int64_t row = row0 + 2 * warp + half + 16 * i;
        const int64_t cw = col0 / 64 + w;
        if (row < m && cw < n / 64) C[row * ldc + cw] = myword;
    }
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

}  // namespace bmm
