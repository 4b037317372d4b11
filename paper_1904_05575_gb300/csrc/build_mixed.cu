// Split-precision tensor-core build (tcgen05).  Placeholder until the
// tensor-core kernels land: the request is refused, never served by another path.
#include "bse_internal.h"

namespace bse {
bool mixed_supported(int) { return false; }
void build_mixed(const Problem&, int, cudaStream_t) {
  throw Error(BSE_ERR_UNSUPPORTED, "split-precision build is not available in this build");
}
}  // namespace bse
