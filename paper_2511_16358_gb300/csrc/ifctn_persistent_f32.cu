// ifctn_persistent_f32.cu -- float instantiations of the streaming contraction kernels and
// of the persistent sweep kernel (one translation unit per dtype so the two
// compile in parallel).
#include "ifctn_contract_kernels.cuh"
#include "ifctn_persistent_impl.cuh"

namespace ifctn {
template cudaError_t launch_contract<float>(const ContractArgs<float>&, cudaStream_t);
template cudaError_t launch_contract_finish<float>(const Shape&, int, const ContractPlan&, const UnitDesc*,
                                                 const float*, const float*, double*, const int*, cudaStream_t);
template int persistent_smem_bytes<float>(const SweepParams<float>&);
template cudaError_t launch_persistent<float>(const SweepParams<float>&, int, int, cudaStream_t);
template int persistent_max_grid<float>(int);
template cudaError_t launch_persistent_multi<float>(const SweepParams<float>*, int, int, int, cudaStream_t);
template int persistent_multi_max_grid<float>(int);
template cudaError_t launch_solve_cols<float>(const SweepParams<float>&, int, cudaStream_t);
}  // namespace ifctn
