// Tensor-core (tcgen05) time transform.
#include "tacaw_api_internal.h"

namespace tacaw {

int spectrum_tc(tacaw_ctx* ctx, const float2*, const double2*, int64_t, int64_t, int64_t, int32_t precision,
                const int32_t*, int64_t, float*, Scratch&) {
  return set_err(ctx, TACAW_EINVAL, "precision %d is not available in this build", precision);
}

}  // namespace tacaw
