// Learned preconditioner for the Davidson solver (placeholder until the
// network kernels land: requesting it is refused, never served by another path).
#include "bse_internal.h"
#include "mlp.h"

namespace bse {
void mlp_precondition(const MlpNet*, int, int, const double*, const double*, const double2*,
                      int64_t, double2*, int64_t, cudaStream_t) {
  throw Error(BSE_ERR_UNSUPPORTED, "the MLP preconditioner is not available in this build");
}
}  // namespace bse
