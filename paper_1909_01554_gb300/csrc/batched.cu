// Batched products of uneven sizes (placeholder until the persistent kernel lands).
#include "plan.h"

namespace bmm {

bmm_status run_batched(int, int32_t, const uint64_t* const*, const uint64_t* const*,
                       uint64_t* const*, const int64_t*, const int64_t*, const int64_t*,
                       cudaStream_t) {
    return BMM_ERR_UNSUPPORTED;
}

}  // namespace bmm
