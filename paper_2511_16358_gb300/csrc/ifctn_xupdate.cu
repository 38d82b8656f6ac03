// ifctn_xupdate.cu -- instantiations of the standalone X update of the per-stage
// path (eq. (updateX) fused with the reconstruction and the stop-test sums),
// in a translation unit of their own so they build in parallel with the
// persistent kernel.
#include "ifctn_persistent_impl.cuh"

namespace ifctn {
template cudaError_t launch_xupdate_slab<float>(const SweepParams<float>&, double*, int, cudaStream_t);
template cudaError_t launch_xupdate_slab<double>(const SweepParams<double>&, double*, int, cudaStream_t);
}  // namespace ifctn
