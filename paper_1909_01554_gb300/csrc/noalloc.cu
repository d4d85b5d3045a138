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
#include "internal.h"

namespace bmm {
namespace {

constexpr uint64_t NOALLOC_WORDS = (uint64_t)BMM_NOALLOC_SCRATCH_BYTES / 8;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS];

// Device address of the scratch array on the current device. In host code
// the array's name only stands in for the symbol, so the address is looked up
// with the calling device current, on every call: it is a table lookup that
// allocates nothing, and a cached address would go stale if the device's
// context were reset and the module loaded again at another address. The
// first lookup on a device loads the module's device code.
bmm_status noalloc_scratch(uint64_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    *out = (uint64_t*)p;
    return BMM_OK;
}

}  // namespace
}  // namespace bmm

using namespace bmm;

extern "C" bmm_status bmm_product_noalloc(int32_t op, const uint64_t* A, const uint64_t* B,
                                          uint64_t* C, int64_t m, int64_t k, int64_t n,
                                          bmm_stream_t stream) {
    if (op != OP_GF2 && op != OP_BOOL) return BMM_ERR_INVALID;
    // the checks of bmm_gf2 / bmm_bool: null, size, alignment and overlap
    bmm_status st = check_product_args(A, B, C, m, k, n);
    if (st != BMM_OK) return st;
    // B^T (n x k bits) must fit the fixed array.
    if ((uint64_t)k * (uint64_t)n / 8 > (uint64_t)BMM_NOALLOC_SCRATCH_BYTES) return BMM_ERR_NOMEM;
    uint64_t* Bt = nullptr;
    st = noalloc_scratch(&Bt);
    if (st != BMM_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    // The transpose writes every word of B^T that the product reads, so the
    // array needs no clearing between calls.
    cudaError_t e = launch_transpose_loadstore(B, Bt, k, n, s);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_popc_nt(op, A, k / 64, 0, Bt, k / 64, 0, C, n / 64, 0, 1, m, k, n, s);
    if (e != cudaSuccess) return cuda_fail(e);
    return BMM_OK;
}
