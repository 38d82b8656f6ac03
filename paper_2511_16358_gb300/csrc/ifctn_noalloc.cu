// ifctn_noalloc.cu -- reconstruction that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is entirely
// owned by another allocator (a framework's caching allocator that has
// reserved the device), code on a latency-critical path that must not pay for
// an allocation (cudaMalloc may synchronise the device), or code with a fixed,
// audited memory footprint.  For them, ifctn_reconstruct_noalloc computes
// iFCTN(G) from device-resident factors into a caller-provided device buffer
// and keeps its only scratch -- the pair matrices W_{p,q} = G_{p,q}^T G_{q,p}
// -- in the file-scope array below, which every GPU that loads this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ifctn.h"
#include "ifctn_api_internal.h"
#include "ifctn_launch.h"

namespace {

// 8 MiB of scratch: the pair matrices of one call, in the tensor dtype.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
ifctn_status scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        ifctn::set_error("no usable current CUDA device");
        return IFCTN_ECUDA;
    }
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            ifctn::set_error(std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                             cudaGetErrorString(e));
            return IFCTN_ECUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return IFCTN_OK;
}

// True when p is device (or managed) memory that the current device owns.
// Memory of another GPU is refused: the scratch array and the launches are
// on the current device, and reaching another GPU's memory from there either
// faults or crosses the interconnect.
bool is_current_device_pointer(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

template <typename T>
ifctn_status run(const ifctn::Shape& sh, const double* factors, void* out, cudaStream_t st, void* scratch) {
    T* W = static_cast<T*>(scratch);
    cudaError_t e = ifctn::launch_pairs<T>(sh, factors, W, st);
    if (e == cudaSuccess) e = ifctn::launch_reconstruct<T>(sh, W, static_cast<T*>(out), nullptr, 1216, st);
    if (e != cudaSuccess) {
        ifctn::set_error(std::string("reconstruction launch failed: ") + cudaGetErrorString(e));
        return IFCTN_ECUDA;
    }
    return IFCTN_OK;
}

}  // namespace

extern "C" ifctn_status ifctn_reconstruct_noalloc(int32_t order, const int64_t* dims, const int32_t* ranks,
                                                   int32_t precision, const double* factors, void* out,
                                                   void* cuda_stream) {
    if (!dims || !ranks || !factors || !out) {
        ifctn::set_error("null argument");
        return IFCTN_EINVAL;
    }
    ifctn_problem p;
    memset(&p, 0, sizeof(p));
    p.order = order;
    for (int k = 0; k < 4 && k < order; ++k) p.dims[k] = dims[k];
    for (int i = 0; i < 16; ++i) p.ranks[i] = ranks[i];
    p.rho = 1.0;
    p.precision = precision;
    ifctn::Shape sh;
    ifctn_status rs = ifctn::build_shape(&p, sh);
    if (rs != IFCTN_OK) return rs;
    const size_t esz = precision == IFCTN_FP64 ? 8 : 4;
    const size_t need = static_cast<size_t>(sh.wsize) * esz;
    if (need > NOALLOC_SCRATCH_BYTES) {
        ifctn::set_error("pair matrices need " + std::to_string(need) + " bytes of scratch, more than the " +
                         std::to_string(NOALLOC_SCRATCH_BYTES) + "-byte static array of the allocation-free path");
        return IFCTN_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        ifctn::set_error("no usable current CUDA device");
        return IFCTN_ECUDA;
    }
    if (!is_current_device_pointer(factors, dev) || !is_current_device_pointer(out, dev)) {
        ifctn::set_error("the allocation-free path needs factors and out in memory of the current device (" +
                         std::to_string(dev) + ")");
        return IFCTN_EINVAL;
    }
    void* scratch = nullptr;
    rs = scratch_for_current_device(&scratch);
    if (rs != IFCTN_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    return precision == IFCTN_FP64 ? run<double>(sh, factors, out, st, scratch)
                                   : run<float>(sh, factors, out, st, scratch);
}
