// ifctn_selftest.cu -- exercises the failure path of the bounded device waits.
//
// Every wait of the library's kernels (the software grid barrier of the
// persistent sweep, the mbarrier phases of the TMA rings) gives up after a
// clock budget, records FLAG_TIMEOUT in the context's flag word and lets the
// kernel return, so that the host reports IFCTN_ETIMEOUT and the CUDA context
// stays usable.  This kernel runs both waits with a short budget on
// conditions that nothing will ever satisfy -- a grid barrier that one CTA
// never joins, and an mbarrier phase whose announced bytes no copy delivers --
// so that the expiry path can be tested without a hung or faulting kernel.
#include "ifctn_persistent_impl.cuh"

namespace ifctn {
namespace {

__global__ void k_wait_selftest(int* flags, unsigned* count, long long budget) {
    __shared__ __align__(8) uint64_t bar;
    if (blockIdx.x != 0) return;  // CTA 1 never arrives at the barrier
    unsigned nb = 0;
    grid_barrier(count, nb, flags, gridDim.x, budget);  // waits for 2 arrivals, 1 comes
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, 16);  // 16 bytes announced, no copy issued
        mbar_wait_bounded(&bar, 0, flags, budget);
    }
    __syncthreads();
}

}  // namespace

cudaError_t launch_wait_selftest(int* flags, unsigned* count, long long budget, cudaStream_t st) {
    k_wait_selftest<<<2, 32, 0, st>>>(flags, count, budget);
    return cudaGetLastError();
}

}  // namespace ifctn
