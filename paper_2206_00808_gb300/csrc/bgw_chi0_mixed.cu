// Mixed-precision contraction: not built yet.
#include "bgw_mixed.h"

namespace bgw {
size_t mixed_workspace_bytes(long, int, int) { return 0; }
cudaError_t herk_mixed(const void *, int, int, const double *, int, void *, void *, cudaStream_t,
                       int *) {
    return cudaErrorNotSupported;
}
}  // namespace bgw
