// k_mlp_tc.cu -- K-c on tcgen05 tensor cores (placeholder until the kernel lands).
#include "amnerf_internal.h"

namespace amnerf {
size_t tc_leaf_stride_bytes(int, int, int, int) { return 0; }
void pack_tc_leaf(const float*, uint8_t*, int, int, int, int) {}
cudaError_t launch_mlp_tc(cudaStream_t, const MlpArgs&, int, int) { return cudaErrorNotSupported; }
}  // namespace amnerf
