// ifctn_persistent_f64.cu -- double instantiations of the streaming contraction kernels and
// of the persistent sweep kernel (one translation unit per dtype so the two
// compile in parallel).
#include "ifctn_contract_kernels.cuh"
#include "ifctn_persistent_impl.cuh"

namespace ifctn {
template cudaError_t launch_contract<double>(const ContractArgs<double>&, cudaStream_t);
template cudaError_t launch_contract_finish<double>(const Shape&, int, const ContractPlan&, const UnitDesc*,
                                                 const double*, const double*, double*, const int*, cudaStream_t);
template int persistent_smem_bytes<double>(const SweepParams<double>&);
template cudaError_t launch_persistent<double>(const SweepParams<double>&, int, int, cudaStream_t);
template int persistent_max_grid<double>(int);
template cudaError_t launch_persistent_multi<double>(const SweepParams<double>*, int, int, int, cudaStream_t);
template int persistent_multi_max_grid<double>(int);
template cudaError_t launch_solve_cols<double>(const SweepParams<double>&, int, cudaStream_t);
}  // namespace ifctn
