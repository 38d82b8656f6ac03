// Warp-pipelined contraction kernels, FP32 tensors.
#include "ifctn_contract_warp.cuh"

namespace ifctn {
template cudaError_t launch_contract_warp<float>(const ContractArgs<float>&, int, cudaStream_t);
}  // namespace ifctn
