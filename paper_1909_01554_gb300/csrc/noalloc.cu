// bmm_product_noalloc: the cubic product with its only scratch buffer (the
// transposed right operand) held in a fixed, file-scope device array instead
// of memory allocated per call.
//
// Some callers cannot allocate device memory while they run: applications
// whose framework reserves almost all of HBM in its own pool up front (a
// library-side cudaMalloc or cudaMallocAsync could then fail or fragment
// that pool), latency-critical loops where an allocation may synchronise
// the device, and deployments that must fix every byte of device memory
// when the library loads. This entry point serves them: it launches the same
// transpose and CUDA-core base-case kernels as bmm_gf2/bmm_bool, and never
// calls an allocator.
#include <mutex>

#include "internal.h"

namespace bmm {
namespace {

constexpr uint64_t NOALLOC_WORDS = (uint64_t)BMM_NOALLOC_SCRATCH_BYTES / 8;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS];

std::mutex g_noalloc_mu;
uint64_t* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array on the current device. In host code
// the array's name only stands in for the symbol, so the address is looked
// up once per device (with that device current) and cached.
bmm_status noalloc_scratch(uint64_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return BMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        g_noalloc_ptr[dev] = (uint64_t*)p;
    }
    *out = g_noalloc_ptr[dev];
    return BMM_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

bool overlaps(const void* a, uint64_t abytes, const void* b, uint64_t bbytes) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

}  // namespace
}  // namespace bmm

using namespace bmm;

extern "C" bmm_status bmm_product_noalloc(int32_t op, const uint64_t* A, const uint64_t* B,
                                          uint64_t* C, int64_t m, int64_t k, int64_t n,
                                          bmm_stream_t stream) {
    if (op != OP_GF2 && op != OP_BOOL) return BMM_ERR_INVALID;
    if (!A || !B || !C) return BMM_ERR_INVALID;
    if (m <= 0 || k <= 0 || n <= 0 || m % 64 || k % 64 || n % 64) return BMM_ERR_INVALID;
    if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return BMM_ERR_ALIGN;
    const uint64_t cb = (uint64_t)m * (uint64_t)n / 8;
    if (overlaps(C, cb, A, (uint64_t)m * (uint64_t)k / 8) ||
        overlaps(C, cb, B, (uint64_t)k * (uint64_t)n / 8))
        return BMM_ERR_INVALID;
    // B^T (n x k bits) must fit the fixed array.
    if ((uint64_t)k * (uint64_t)n / 8 > (uint64_t)BMM_NOALLOC_SCRATCH_BYTES) return BMM_ERR_NOMEM;
    uint64_t* Bt = nullptr;
    bmm_status st = noalloc_scratch(&Bt);
    if (st != BMM_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    // The transpose writes every word of B^T that the product reads, so the
    // array needs no clearing between calls.
    cudaError_t e = launch_transpose(B, Bt, k, n, s);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_popc_nt(op, A, k / 64, 0, Bt, k / 64, 0, C, n / 64, 0, 1, m, k, n, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return BMM_OK;
}
