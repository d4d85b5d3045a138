// Planner and executor for one product (the accelerator-side layers of
// Sec. 3.4 on a single GPU with all operands resident in HBM):
//   transpose B -> Bt (Sec. 3.5), then `serial` depth-first levels
//   (Sec. 3.8: combine, recurse, fold, reusing scratch across the 7
//   branches), then `depth - serial` breadth-first levels merged into one
//   expanding pass per operand (Sec. 3.9, 3.15), the batched base case over
//   the 7^d leaves (Sec. 3.10), and one compressing pass (Sec. 3.11).
#include <cstring>

#include "plan.h"
#include "slp.h"

namespace bmm {

cudaError_t launch_expand(int variant, int operand, int d, const uint64_t* X, int64_t pitch,
                          int64_t rows, int64_t wcols, uint32_t mask, uint64_t* leaves,
                          cudaStream_t s);
cudaError_t launch_compress(int variant, int d, const uint64_t* leaves, int64_t lr, int64_t lw,
                            uint64_t* C, int64_t ldc, uint32_t dest, uint32_t first,
                            cudaStream_t s);
cudaError_t launch_combine(int operand, const uint64_t* X, int64_t pitch, int64_t hr, int64_t hw,
                           uint32_t mask, uint64_t* dst, cudaStream_t s);
cudaError_t launch_fold(const uint64_t* R, int64_t hr, int64_t hw, uint64_t* C, int64_t ldc,
                        uint32_t dest, uint32_t first, cudaStream_t s);
bmm_status run_tc_strided(int op, int path, const uint64_t* A, int64_t lda, int64_t strideA,
                          const uint64_t* Bt, int64_t ldb, int64_t strideB, uint64_t* C,
                          int64_t ldc, int64_t strideC, int64_t count, int64_t m, int64_t k,
                          int64_t n, cudaStream_t s);

namespace {

constexpr uint64_t ALIGN = 256;
uint64_t round_up(uint64_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

constexpr int MAX_MERGED = 2;  // breadth-first levels merged in registers

int ipow7(int d) {
    int r = 1;
    while (d-- > 0) r *= 7;
    return r;
}

bool divisible(int64_t m, int64_t k, int64_t n, int d) {
    const int64_t unit = (int64_t)64 << d;
    return (m % ((int64_t)1 << d) == 0) && (m >> d) % 64 == 0 && k % unit == 0 && n % unit == 0;
}

// The last depth-first level hands its branches straight to the
// breadth-first passes: its input combination is done by the expanding pass
// (reading the parent's quadrants) and its output fold by the compressing
// pass, so that level needs no branch buffers.
bool fused_last_serial(int depth, int serial) { return serial > 0 && depth > serial; }

// Bytes of scratch for a plan: Bt, the depth-first branch buffers of every
// serial level, and the breadth-first leaves at the bottom.
uint64_t workspace_for(int64_t m, int64_t k, int64_t n, int depth, int serial) {
    uint64_t b = round_up((uint64_t)k * n / 8);  // Bt
    const int bufs = fused_last_serial(depth, serial) ? serial - 1 : serial;
    for (int l = 1; l <= bufs; l++) {
        b += round_up((uint64_t)(m >> l) * (k >> l) / 8);
        b += round_up((uint64_t)(n >> l) * (k >> l) / 8);
        b += round_up((uint64_t)(m >> l) * (n >> l) / 8);
    }
    const int dp = depth - serial;
    if (dp > 0) {
        const uint64_t r = (uint64_t)ipow7(dp);
        b += round_up(r * (uint64_t)(m >> depth) * (k >> depth) / 8);
        b += round_up(r * (uint64_t)(n >> depth) * (k >> depth) / 8);
        b += round_up(r * (uint64_t)(m >> depth) * (n >> depth) / 8);
    }
    return b;
}

struct Exec {
    const Plan& p;
    const int od;  // levels outside the base case (the last one may run inside it)
    char* ws;
    cudaStream_t s;
    uint32_t xi[7], eta[7], zeta[4];
    uint64_t* Bt = nullptr;
    uint64_t* Apad = nullptr;  // A with k padded to kp (only when kp != k)
    uint64_t* T[8] = {nullptr};
    uint64_t* S[8] = {nullptr};
    uint64_t* R[8] = {nullptr};
    uint64_t *TL = nullptr, *SL = nullptr, *QL = nullptr;

    Exec(const Plan& plan, void* w, cudaStream_t st)
        : p(plan), od(plan.depth - plan.kernel_level), ws((char*)w), s(st) {
        switch (p.variant) {
            case 0: slp::level_masks<0>(xi, eta, zeta); break;
            case 1: slp::level_masks<1>(xi, eta, zeta); break;
            default: slp::level_masks<2>(xi, eta, zeta); break;
        }
        uint64_t off = 0;
        auto take = [&](uint64_t bytes) {
            uint64_t* q = (uint64_t*)(ws + off);
            off += round_up(bytes);
            return q;
        };
        Bt = take((uint64_t)p.kp * p.n / 8);
        if (p.kp != p.k) Apad = take((uint64_t)p.m * p.kp / 8);
        const int bufs = fused_last_serial(od, p.serial) ? p.serial - 1 : p.serial;
        for (int l = 1; l <= bufs; l++) {
            T[l] = take((uint64_t)(p.m >> l) * (p.kp >> l) / 8);
            S[l] = take((uint64_t)(p.n >> l) * (p.kp >> l) / 8);
            R[l] = take((uint64_t)(p.m >> l) * (p.n >> l) / 8);
        }
        const int dp = od - p.serial;
        if (dp > 0) {
            const uint64_t r = (uint64_t)ipow7(dp);
            TL = take(r * (uint64_t)(p.m >> od) * (p.kp >> od) / 8);
            SL = take(r * (uint64_t)(p.n >> od) * (p.kp >> od) / 8);
            QL = take(r * (uint64_t)(p.m >> od) * (p.n >> od) / 8);
        }
    }

    // The product of `count` blocks below the outer levels (strides in words):
    // the base case, or the innermost Strassen level with the base case
    // inside one kernel.
    bmm_status blocks(const uint64_t* A, int64_t lda, int64_t sa, const uint64_t* B, int64_t ldb,
                      int64_t sb, uint64_t* C, int64_t ldc, int64_t sc, int64_t count, int64_t m,
                      int64_t k, int64_t n) {
        if (p.kernel_level) {
            LevelMasks lm;
            std::memcpy(lm.xi, xi, sizeof xi);
            std::memcpy(lm.eta, eta, sizeof eta);
            std::memcpy(lm.zeta, zeta, sizeof zeta);
            if (p.path == BMM_PATH_TC_FP4_PAIR)
                return run_tc_level(A, lda, sa, B, ldb, sb, C, ldc, sc, count, m, k, n, lm, s);
            BMM_CUDA_TRY(launch_popc_level(A, lda, sa, B, ldb, sb, C, ldc, sc, count, m, k, n, lm,
                                           s));
            return BMM_OK;
        }
        return run_base_product_batched(p.op, p.path, A, lda, sa, B, ldb, sb, C, ldc, sc, count,
                                        m, k, n, s);
    }

    bmm_status level(int l, const uint64_t* A, int64_t lda, const uint64_t* B, int64_t ldb,
                     uint64_t* C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
        if (l < p.serial) {
            const int64_t hm = m / 2, hk = k / 2, hn = n / 2;
            uint32_t first = 0xF;
            if (l + 1 == p.serial && fused_last_serial(od, p.serial)) {
                for (int h = 0; h < 7; h++) {
                    uint32_t dest = 0;
                    for (int q = 0; q < 4; q++) dest |= ((zeta[q] >> h) & 1u) << q;
                    if (!dest) continue;
                    bmm_status st = leaves(A, lda, xi[h], B, ldb, eta[h], C, ldc, dest,
                                           first & dest, hm, hk, hn);
                    if (st != BMM_OK) return st;
                    first &= ~dest;
                }
                return BMM_OK;
            }
            for (int h = 0; h < 7; h++) {
                BMM_CUDA_TRY(launch_combine(0, A, lda, hm, hk / 64, xi[h], T[l + 1], s));
                BMM_CUDA_TRY(launch_combine(1, B, ldb, hn, hk / 64, eta[h], S[l + 1], s));
                bmm_status st = level(l + 1, T[l + 1], hk / 64, S[l + 1], hk / 64, R[l + 1],
                                      hn / 64, hm, hk, hn);
                if (st != BMM_OK) return st;
                uint32_t dest = 0;
                for (int q = 0; q < 4; q++) dest |= ((zeta[q] >> h) & 1u) << q;
                if (dest) {
                    BMM_CUDA_TRY(launch_fold(R[l + 1], hm, hn / 64, C, ldc, dest, first & dest, s));
                    first &= ~dest;
                }
            }
            return BMM_OK;
        }
        if (od == l) return blocks(A, lda, 0, B, ldb, 0, C, ldc, 0, 1, m, k, n);
        return leaves(A, lda, 0, B, ldb, 0, C, ldc, 0, 0, m, k, n);
    }

    // The breadth-first levels below an m x k x n block: expand both operands
    // into the leaves, the batched base case, compress into C. With non-zero
    // masks the block's operands are combinations of the quadrants of A / B
    // (their parents) and the result is folded into the quadrants `dest` of
    // C (its parent), as a depth-first level would.
    bmm_status leaves(const uint64_t* A, int64_t lda, uint32_t amask, const uint64_t* B,
                      int64_t ldb, uint32_t bmask, uint64_t* C, int64_t ldc, uint32_t dest,
                      uint32_t first, int64_t m, int64_t k, int64_t n) {
        const int dp = od - p.serial;
        const int64_t lm = m >> dp, lk = k >> dp, ln = n >> dp;
        BMM_CUDA_TRY(launch_expand(p.variant, 0, dp, A, lda, m, k / 64, amask, TL, s));
        BMM_CUDA_TRY(launch_expand(p.variant, 1, dp, B, ldb, n, k / 64, bmask, SL, s));
        const int64_t count = ipow7(dp);
        bmm_status st = blocks(TL, lk / 64, lm * lk / 64, SL, lk / 64, ln * lk / 64, QL, ln / 64,
                               lm * ln / 64, count, lm, lk, ln);
        if (st != BMM_OK) return st;
        BMM_CUDA_TRY(launch_compress(p.variant, dp, QL, lm, ln / 64, C, ldc, dest, first, s));
        return BMM_OK;
    }
};

}  // namespace

// Scratch of a plan with k padded to kp (the padded copy of A when kp != k).
uint64_t workspace_padded(int64_t m, int64_t k, int64_t kp, int64_t n, int depth, int serial) {
    return workspace_for(m, kp, n, depth, serial) + (kp != k ? round_up((uint64_t)m * kp / 8) : 0);
}

bmm_status make_plan(int op, int64_t m, int64_t k, int64_t n, const bmm_opts* opts, Plan* out) {
    bmm_opts o;
    bmm_opts_default(&o);
    if (opts) o = *opts;
    Plan p;
    p.op = op;
    p.m = m;
    p.k = k;
    p.n = n;
    if (o.variant < 0 || o.variant > 2) return BMM_ERR_INVALID;
    if (o.kernel_level < 0 || o.kernel_level > 1) return BMM_ERR_INVALID;
    p.variant = o.variant;
    if (o.path < BMM_PATH_AUTO || o.path > BMM_PATH_TC_FP4_PAIR) return BMM_ERR_INVALID;
    if (is_tc_path(o.path) && !tc_path_available()) return BMM_ERR_UNSUPPORTED;
    if (o.path == BMM_PATH_TC_FP4_PAIR && !tc_fp4_available()) return BMM_ERR_UNSUPPORTED;
    // recursion depth
    if (op == OP_BOOL) {
        if (o.strassen_depth > 0) return BMM_ERR_INVALID;  // no additive inverse
        p.depth = 0;
    } else if (o.strassen_depth >= 0) {
        p.depth = o.strassen_depth;
        if (p.depth > 6) return BMM_ERR_UNSUPPORTED;
        if (p.depth > 0 && !divisible(m, k, n, p.depth)) return BMM_ERR_UNSUPPORTED;
    } else {
        // Auto: recurse while every leaf dimension stays >= 8192 (below that the
        // base case loses efficiency faster than 7/8 of the work is saved).
        int d = 0;
        while (d < 4 && divisible(m, k, n, d + 1) && (m >> (d + 1)) >= 8192 &&
               (k >> (d + 1)) >= 8192 && (n >> (d + 1)) >= 8192)
            d++;
        p.depth = d;
    }
    // A tuned choice (bmm_autotune) replaces the rules below when both the
    // path and the depth are left to the library.
    int tpath = 0, tdepth = 0;
    const bool tuned = o.path == BMM_PATH_AUTO && o.strassen_depth < 0 && o.kernel_level == 0 &&
                       tuned_choice(op, m, k, n, &tpath, &tdepth) &&
                       (tdepth == 0 || (op == OP_GF2 && divisible(m, k, n, tdepth)));
    if (tuned) {
        p.depth = tdepth;
        o.path = tpath;
    }
    // base-case path (auto_path below); the tensor paths pad k so that every
    // leaf's k is a multiple of 128 bits
    p.path = o.path == BMM_PATH_AUTO ? auto_path() : o.path;
    // The innermost level inside the base-case kernel: the CUDA-core kernel
    // and the e2m1 SM-pair kernel have that form; a plan without Strassen
    // levels has no level to move.
    p.kernel_level = (o.kernel_level && p.depth > 0) ? 1 : 0;
    if (p.kernel_level && p.path != BMM_PATH_POPC && p.path != BMM_PATH_TC_FP4_PAIR)
        return BMM_ERR_UNSUPPORTED;
    p.kp = k;
    if (is_tc_path(p.path)) {
        // leaf k a multiple of 128 bits; with the level in the tensor kernel,
        // of its 512-bit packed stage (a quadrant's copies stay inside it)
        const int64_t unit = (int64_t)(p.kernel_level ? 512 : 128) << p.depth;
        p.kp = (k + unit - 1) / unit * unit;
    }
    const int od = p.depth - p.kernel_level;  // levels run by the XOR passes
    // depth-first levels: at least od - MAX_MERGED; more while the
    // breadth-first scratch does not fit in free device memory.
    int serial_min = od > MAX_MERGED ? od - MAX_MERGED : 0;
    if (o.serial_depth >= 0) {
        if (o.serial_depth > od) return BMM_ERR_INVALID;
        p.serial = o.serial_depth < serial_min ? serial_min : o.serial_depth;
    } else {
        p.serial = serial_min;
        size_t fr = 0, tot = 0;
        if (!(o.workspace) && cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
            while (p.serial < od &&
                   workspace_padded(m, k, p.kp, n, od, p.serial) > (uint64_t)(fr * 0.9))
                p.serial++;
        }
    }
    p.workspace_bytes = workspace_padded(m, k, p.kp, n, od, p.serial);
    *out = p;
    return BMM_OK;
}

uint64_t plan_pass_bytes(const Plan& p) {
    uint32_t xi[7], eta[7], zeta[4];
    switch (p.variant) {
        case 0: slp::level_masks<0>(xi, eta, zeta); break;
        case 1: slp::level_masks<1>(xi, eta, zeta); break;
        default: slp::level_masks<2>(xi, eta, zeta); break;
    }
    auto bits = [](uint32_t x) { return (uint64_t)__builtin_popcount(x); };
    const int d = p.depth - p.kernel_level, dp = d - p.serial;
    const bool fused = fused_last_serial(d, p.serial);
    const uint64_t r = (uint64_t)ipow7(dp > 0 ? dp : 0);
    const uint64_t la = (uint64_t)(p.m >> d) * (p.kp >> d) / 8;
    const uint64_t lb = (uint64_t)(p.n >> d) * (p.kp >> d) / 8;
    const uint64_t lc = (uint64_t)(p.m >> d) * (p.n >> d) / 8;
    // transpose: B read, Bt written with its padding columns
    uint64_t total = (uint64_t)p.k * p.n / 8 + (uint64_t)p.kp * p.n / 8;
    if (p.kp != p.k) total += (uint64_t)p.m * p.k / 8 + (uint64_t)p.m * p.kp / 8;  // padded A
    uint64_t reps = 1;                              // executions of the current level
    for (int l = 0; l < p.serial; l++, reps *= 7) {
        const uint64_t a = (uint64_t)(p.m >> (l + 1)) * (p.kp >> (l + 1)) / 8;
        const uint64_t b = (uint64_t)(p.n >> (l + 1)) * (p.kp >> (l + 1)) / 8;
        const uint64_t c = (uint64_t)(p.m >> (l + 1)) * (p.n >> (l + 1)) / 8;
        const bool last_fused = fused && l + 1 == p.serial;
        uint64_t per = 0;
        uint32_t first = 0xF;
        for (int h = 0; h < 7; h++) {
            uint32_t dest = 0;
            for (int q = 0; q < 4; q++) dest |= ((zeta[q] >> h) & 1u) << q;
            if (last_fused) {  // expand reads the parent's quadrants, compress folds
                if (!dest) continue;
                per += bits(xi[h]) * a + r * la + bits(eta[h]) * b + r * lb;
                per += r * lc + bits(dest) * c + bits(dest & ~first) * c;
            } else {  // combine into branch buffers, fold the branch result
                per += (bits(xi[h]) + 1) * a + (bits(eta[h]) + 1) * b;
                if (dest) per += c + bits(dest) * c + bits(dest & ~first) * c;
            }
            first &= ~dest;
        }
        total += reps * per;
    }
    if (dp > 0 && !fused) {
        const int s = p.serial;
        const uint64_t in_a = (uint64_t)(p.m >> s) * (p.kp >> s) / 8;
        const uint64_t in_b = (uint64_t)(p.n >> s) * (p.kp >> s) / 8;
        const uint64_t out_c = (uint64_t)(p.m >> s) * (p.n >> s) / 8;
        total += reps * (in_a + r * la + in_b + r * lb + r * lc + out_c);
    }
    return total;
}

bmm_status execute_plan(const Plan& p, const uint64_t* A, const uint64_t* B, uint64_t* C,
                        void* workspace, cudaStream_t s) {
    Exec ex(p, workspace, s);
    const uint64_t* Aop = A;
    if (p.kp != p.k) {
        // zero pad columns k..kp of A (a pitched copy) and of B^T
        const size_t wb = (size_t)(p.k / 8), pb = (size_t)(p.kp / 8);
        BMM_CUDA_TRY(cudaMemset2DAsync((char*)ex.Apad + wb, pb, 0, pb - wb, (size_t)p.m, s));
        BMM_CUDA_TRY(cudaMemcpy2DAsync(ex.Apad, pb, A, wb, wb, (size_t)p.m,
                                       cudaMemcpyDeviceToDevice, s));
        BMM_CUDA_TRY(cudaMemset2DAsync((char*)ex.Bt + wb, pb, 0, pb - wb, (size_t)p.n, s));
        Aop = ex.Apad;
    }
    BMM_CUDA_TRY(launch_transpose_pitched(B, p.n / 64, ex.Bt, p.kp / 64, p.k, p.n, s));
    return ex.level(0, Aop, p.kp / 64, ex.Bt, p.kp / 64, C, p.n / 64, p.m, p.kp, p.n);
}

// Base case for BMM_PATH_AUTO: the tensor cores wherever the device has
// them; on SM pairs where clusters can be launched (faster at every measured
// size from 4096^3 up), with e2m1 operands (twice the e4m3 rate from 8192^3
// up); else the CUDA-core kernel.
int auto_path() {
    if (!tc_path_available()) return BMM_PATH_POPC;
    if (tc_fp4_available()) return BMM_PATH_TC_FP4_PAIR;
    return tc_pair_available() ? BMM_PATH_TC_FP8_PAIR : BMM_PATH_TC_FP8;
}

bmm_status run_base_product(int op, int path, const uint64_t* A, int64_t lda, const uint64_t* Bt,
                            int64_t ldb, uint64_t* C, int64_t ldc, int64_t m, int64_t k,
                            int64_t n, cudaStream_t s) {
    return run_base_product_batched(op, path, A, lda, 0, Bt, ldb, 0, C, ldc, 0, 1, m, k, n, s);
}

bmm_status run_base_product_batched(int op, int path, const uint64_t* A, int64_t lda,
                                    int64_t strideA, const uint64_t* Bt, int64_t ldb,
                                    int64_t strideB, uint64_t* C, int64_t ldc, int64_t strideC,
                                    int64_t count, int64_t m, int64_t k, int64_t n,
                                    cudaStream_t s) {
    if (count <= 0) return BMM_OK;
    if (path == BMM_PATH_POPC) {
        BMM_CUDA_TRY(launch_popc_nt(op, A, lda, strideA, Bt, ldb, strideB, C, ldc, strideC, count,
                                    m, k, n, s));
        return BMM_OK;
    }
    return run_tc_strided(op, path, A, lda, strideA, Bt, ldb, strideB, C, ldc, strideC, count, m,
                          k, n, s);
}

}  // namespace bmm
