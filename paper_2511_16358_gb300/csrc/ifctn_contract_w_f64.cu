// Warp-pipelined contraction kernels, FP64 tensors.
#include "ifctn_contract_warp.cuh"

namespace ifctn {
template cudaError_t launch_contract_warp<double>(const ContractArgs<double>&, int, cudaStream_t);
}  // namespace ifctn
