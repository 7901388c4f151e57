// tcgen05 split-precision contraction (placeholder until the kernel lands).
#include "internal.h"

namespace cutqc {
bool tc_supported(const Contraction&) { return false; }
size_t tc_workspace_bytes(const Contraction&) { return 0; }
void launch_tc_bf16x3(const Contraction&, void*, size_t, cudaStream_t) {
  fail(CUTQC_ERR_UNSUPPORTED, "tensor-core path not built");
}
}  // namespace cutqc
