// Tensor-core split-BF16 evaluation path (placeholder until the tcgen05 kernel lands).
#include "tc_internal.h"

namespace scff {
size_t tc_workspace_bytes(const PairSetDev &, int, int, int, int) { return 0; }
cudaError_t launch_tc_form_factor(const TcArgs &, int64_t *, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace scff
