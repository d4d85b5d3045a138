// C ABI entry points (include/bmm.h): argument checks, path planning,
// stream-ordered scratch, and the sequence of kernels for each product.
#include <cstring>
#include <mutex>

#include "internal.h"
#include "plan.h"

namespace bmm {

namespace {
thread_local int32_t t_last_cuda_error = 0;
std::mutex g_mu;
uint32_t* g_err_word[64] = {nullptr};
int g_sms[64] = {0};
int g_cc[64] = {0};

int cur_dev() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}
}  // namespace

bmm_status cuda_fail(cudaError_t e) {
    t_last_cuda_error = (int32_t)e;
    if (e == cudaErrorMemoryAllocation) return BMM_ERR_NOMEM;
    return BMM_ERR_CUDA;
}

uint32_t* device_error_word() {
    const int d = cur_dev();
    if (d < 0 || d >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_err_word[d]) {
        void* p = nullptr;
        if (cudaMalloc(&p, 256) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, 256) != cudaSuccess) return nullptr;
        g_err_word[d] = (uint32_t*)p;
    }
    return g_err_word[d];
}

int sm_count() {
    const int d = cur_dev();
    if (d >= 0 && d < 64 && g_sms[d]) return g_sms[d];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    if (d >= 0 && d < 64) g_sms[d] = v;
    return v > 0 ? v : 1;
}

int device_cc() {
    const int d = cur_dev();
    if (d >= 0 && d < 64 && g_cc[d]) return g_cc[d];
    int ma = 0, mi = 0;
    cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, d);
    cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, d);
    const int v = ma * 10 + mi;
    if (d >= 0 && d < 64) g_cc[d] = v;
    return v;
}

// ---------------------------------------------------------------- checks
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static bool overlaps(const void* a, uint64_t abytes, const void* b, uint64_t bbytes) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

bmm_status check_product_args(const uint64_t* A, const uint64_t* B, const uint64_t* C,
                              int64_t m, int64_t k, int64_t n) {
    if (!A || !B || !C) return BMM_ERR_INVALID;
    if (m <= 0 || k <= 0 || n <= 0 || m % 64 || k % 64 || n % 64) return BMM_ERR_INVALID;
    if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return BMM_ERR_ALIGN;
    const uint64_t ab = (uint64_t)m * (uint64_t)k / 8, bb = (uint64_t)k * (uint64_t)n / 8,
                   cb = (uint64_t)m * (uint64_t)n / 8;
    if (overlaps(C, cb, A, ab) || overlaps(C, cb, B, bb)) return BMM_ERR_INVALID;
    return BMM_OK;
}

// Scratch: caller workspace when given, else stream-ordered allocation.
struct Scratch {
    void* base = nullptr;
    uint64_t bytes = 0;
    bool owned = false;
    cudaStream_t s = nullptr;
    bmm_status acquire(uint64_t need, const bmm_opts* o, cudaStream_t st) {
        s = st;
        bytes = need;
        if (need == 0) return BMM_OK;
        if (o && o->workspace) {
            if (o->workspace_bytes < need) return BMM_ERR_NOMEM;
            if (!aligned16(o->workspace)) return BMM_ERR_ALIGN;
            base = o->workspace;
            return BMM_OK;
        }
        const cudaError_t e = cudaMallocAsync(&base, need, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            base = nullptr;
            return cuda_fail(e);
        }
        owned = true;
        return BMM_OK;
    }
    ~Scratch() {
        if (owned && base) cudaFreeAsync(base, s);
    }
};

}  // namespace bmm

using namespace bmm;

extern "C" {

void bmm_opts_default(bmm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->path = BMM_PATH_AUTO;
    o->strassen_depth = -1;
    o->variant = BMM_VARIANT_SELF_INVERSE;
    o->serial_depth = -1;
}

const char* bmm_status_string(bmm_status s) {
    switch (s) {
        case BMM_OK: return "BMM_OK";
        case BMM_ERR_INVALID: return "BMM_ERR_INVALID";
        case BMM_ERR_ALIGN: return "BMM_ERR_ALIGN";
        case BMM_ERR_NOMEM: return "BMM_ERR_NOMEM";
        case BMM_ERR_CUDA: return "BMM_ERR_CUDA";
        case BMM_ERR_TIMEOUT: return "BMM_ERR_TIMEOUT";
        case BMM_ERR_UNSUPPORTED: return "BMM_ERR_UNSUPPORTED";
    }
    return "BMM_ERR_UNKNOWN";
}

int32_t bmm_last_cuda_error(void) { return t_last_cuda_error; }

int32_t bmm_device_supported(void) { return device_cc() == 103 ? 1 : 0; }

bmm_status bmm_stream_status(bmm_stream_t stream) {
    BMM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t* w = device_error_word();
    if (!w) return BMM_ERR_NOMEM;
    uint32_t v = 0;
    BMM_CUDA_TRY(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
    if (v) {
        BMM_CUDA_TRY(cudaMemset(w, 0, sizeof(uint32_t)));
        return BMM_ERR_TIMEOUT;
    }
    return BMM_OK;
}

bmm_status bmm_transpose(const uint64_t* X, uint64_t* Xt, int64_t rows, int64_t cols,
                         bmm_stream_t stream) {
    if (!X || !Xt || rows <= 0 || cols <= 0 || rows % 64 || cols % 64) return BMM_ERR_INVALID;
    if (overlaps(X, (uint64_t)rows * cols / 8, Xt, (uint64_t)rows * cols / 8))
        return BMM_ERR_INVALID;
    BMM_CUDA_TRY(launch_transpose(X, Xt, rows, cols, (cudaStream_t)stream));
    return BMM_OK;
}

bmm_status bmm_base_product(int32_t op, int32_t path, const uint64_t* A, const uint64_t* Bt,
                            uint64_t* C, int64_t m, int64_t k, int64_t n, bmm_stream_t stream) {
    if (op != OP_GF2 && op != OP_BOOL) return BMM_ERR_INVALID;
    bmm_status st = check_product_args(A, Bt, C, m, k, n);
    if (st != BMM_OK) return st;
    return run_base_product(op, path, A, k / 64, Bt, k / 64, C, n / 64, m, k, n,
                            (cudaStream_t)stream);
}

bmm_status bmm_workspace_size(int32_t op, int64_t m, int64_t k, int64_t n, const bmm_opts* opts,
                              uint64_t* bytes) {
    if (!bytes || (op != OP_GF2 && op != OP_BOOL)) return BMM_ERR_INVALID;
    if (m <= 0 || k <= 0 || n <= 0 || m % 64 || k % 64 || n % 64) return BMM_ERR_INVALID;
    Plan p;
    bmm_status st = make_plan(op, m, k, n, opts, &p);
    if (st != BMM_OK) return st;
    *bytes = p.workspace_bytes;
    return BMM_OK;
}

bmm_status bmm_plan(int32_t op, int64_t m, int64_t k, int64_t n, const bmm_opts* opts,
                    bmm_plan_info* info) {
    if (!info || (op != OP_GF2 && op != OP_BOOL)) return BMM_ERR_INVALID;
    if (m <= 0 || k <= 0 || n <= 0 || m % 64 || k % 64 || n % 64) return BMM_ERR_INVALID;
    Plan p;
    bmm_status st = make_plan(op, m, k, n, opts, &p);
    if (st != BMM_OK) return st;
    info->path = p.path;
    info->strassen_depth = p.depth;
    info->serial_depth = p.serial;
    info->variant = p.variant;
    int64_t leaves = 1;
    for (int i = 0; i < p.depth; i++) leaves *= 7;
    info->leaves = leaves;
    info->workspace_bytes = p.workspace_bytes;
    info->kernel_level = p.kernel_level;
    info->kp = p.kp;
    info->pass_bytes = plan_pass_bytes(p);
    return BMM_OK;
}

static bmm_status product(int op, const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m,
                          int64_t k, int64_t n, const bmm_opts* opts, bmm_stream_t stream) {
    bmm_status st = check_product_args(A, B, C, m, k, n);
    if (st != BMM_OK) return st;
    Plan p;
    st = make_plan(op, m, k, n, opts, &p);
    if (st != BMM_OK) return st;
    Scratch ws;
    st = ws.acquire(p.workspace_bytes, opts, (cudaStream_t)stream);
    if (st != BMM_OK) return st;
    return execute_plan(p, A, B, C, ws.base, (cudaStream_t)stream);
}

bmm_status bmm_gf2(const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m, int64_t k,
                   int64_t n, bmm_stream_t stream) {
    return product(OP_GF2, A, B, C, m, k, n, nullptr, stream);
}
bmm_status bmm_bool(const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m, int64_t k,
                    int64_t n, bmm_stream_t stream) {
    return product(OP_BOOL, A, B, C, m, k, n, nullptr, stream);
}
bmm_status bmm_gf2_ex(const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m, int64_t k,
                      int64_t n, const bmm_opts* opts, bmm_stream_t stream) {
    return product(OP_GF2, A, B, C, m, k, n, opts, stream);
}
bmm_status bmm_bool_ex(const uint64_t* A, const uint64_t* B, uint64_t* C, int64_t m, int64_t k,
                       int64_t n, const bmm_opts* opts, bmm_stream_t stream) {
    return product(OP_BOOL, A, B, C, m, k, n, opts, stream);
}

bmm_status bmm_basis_change(int32_t variant, int32_t inverse, uint64_t* X, int64_t rows,
                            int64_t cols, int32_t depth, bmm_stream_t stream) {
    if (!X || depth < 0 || variant < 0 || variant > 2) return BMM_ERR_INVALID;
    const int64_t unit = (int64_t)64 << depth;
    if (rows <= 0 || cols <= 0 || rows % unit || cols % unit) return BMM_ERR_INVALID;
    if (!aligned16(X)) return BMM_ERR_ALIGN;
    return run_basis_change(variant, inverse, X, cols / 64, rows, cols, depth,
                            (cudaStream_t)stream);
}

bmm_status bmm_gf2_batched(int32_t count, const uint64_t* const* A, const uint64_t* const* B,
                           uint64_t* const* C, const int64_t* m, const int64_t* k,
                           const int64_t* n, bmm_stream_t stream) {
    return run_batched(OP_GF2, count, A, B, C, m, k, n, (cudaStream_t)stream);
}
bmm_status bmm_bool_batched(int32_t count, const uint64_t* const* A, const uint64_t* const* B,
                            uint64_t* const* C, const int64_t* m, const int64_t* k,
                            const int64_t* n, bmm_stream_t stream) {
    return run_batched(OP_BOOL, count, A, B, C, m, k, n, (cudaStream_t)stream);
}

}  // extern "C"
