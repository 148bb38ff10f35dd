// Serving loop (tacaw_submit / tacaw_poll).
#include "tacaw_api_internal.h"

namespace tacaw {

void serving_shutdown(tacaw_ctx*) {}

}  // namespace tacaw
