// ifctn_api_internal.h -- host-side declarations shared by the API and the server.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/ifctn.h"
#include "ifctn_internal.cuh"

namespace ifctn {

void set_error(const std::string& m);
ifctn_status build_shape(const ifctn_problem* p, Shape& s);
int mode_q(const Shape& s, int k);
// tune_timing: a context created while IFCTN_TUNE_CACHE names a file may time
// launch-shape candidates for shapes the cache lacks (false: cache lookups only)
ifctn_status create_ctx(const ifctn_problem* prob, const void* obs, const uint8_t* mask, const double* init,
                        void* stream, ifctn_ctx** out, bool tune_timing);
size_t ctx_device_bytes(const ifctn_ctx* c);
// serving: element size of a context whose sweeps run as one persistent
// launch (4 or 8), else 0; and one cooperative launch running nsweeps[i]
// sweeps of every ctxs[i] (same kind) on a slice of the grid each, on stream
// bst (returns once the launch is enqueued)
int ctx_batch_kind(const ifctn_ctx* c);
ifctn_status ctx_run_batch(ifctn_ctx* const* ctxs, const int* nsweeps, int njobs, cudaStream_t bst);
// asynchronous use by the server: enqueue n sweeps (tolerance tol) on the
// context's stream without waiting.
ifctn_status ctx_enqueue(ifctn_ctx* c, int n, double tol, bool reset);
cudaStream_t ctx_stream(ifctn_ctx* c);
// caps the persistent grid (the server gives each resident job a share)
void ctx_set_grid_cap(ifctn_ctx* c, int g);

}  // namespace ifctn
