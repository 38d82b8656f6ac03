// ifctn_launch.h -- host-side launchers of the iFCTN kernels (one TU per group).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "ifctn_internal.cuh"

namespace ifctn {

// The dynamic shared-memory limit of a kernel is one setting per function and
// device for the whole process, while several contexts (each with its own
// plan) may launch the same kernel: only ever raise it.
inline cudaError_t raise_dyn_smem(const void* func, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cur;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    int& c = cur[std::make_pair(func, dev)];
    if (bytes <= c) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) c = bytes;
    return e;
}

template <typename T>
struct ContractArgs {
    const T* X;
    const T* Gt;  // cherry factors in the tensor dtype
    const T* W;   // pair matrices in the tensor dtype
    Shape sh;
    int k;
    ContractPlan pl;
    const UnitDesc* units;
    T* part;
    int* flags;
    const int* done;
};

// M_k partials (Prop. 1: M_k = X_(k) Z_k, Z_k generated on the fly).
template <typename T>
cudaError_t launch_contract(const ContractArgs<T>& a, cudaStream_t st);

// Warp-pipelined variant for tensors streamed from HBM (plan.warp = 1).
template <typename T>
cudaError_t launch_contract_warp(const ContractArgs<T>& a, int grid, cudaStream_t st);
// M_k = reduction of the partials (FP64 output, I_k x Q_k).
template <typename T>
cudaError_t launch_contract_finish(const Shape& sh, int k, const ContractPlan& pl,
                                   const UnitDesc* units, const T* part, const T* Gt, double* Mk,
                                   const int* done, cudaStream_t st);

// K_k = Z_k^T Z_k via the mode-by-mode chain (t1, t2 scratch; output in T).
template <typename T>
cudaError_t launch_gram(const Shape& sh, int k, const T* Gt, const T* W, T* t1, T* t2, T* Kk,
                        const int* done, cudaStream_t st);

// Order-3 tensors with edge ranks above RMAX (Shape::wide): the mode
// systems as chains of batched products (contraction: modes c1 then c2; Gram:
// d1 then d2) and the column solves with H in shared memory.
struct WideChain {
    int c1, c2, d1, d2;
};
WideChain wide_chain(const Shape& s, int k);
long long wide_v_elems(const Shape& s, int k);  // first contraction link's output (V)
long long wide_t_elems(const Shape& s, int k);  // first Gram link's output
template <typename T>
cudaError_t launch_wide_contract(const Shape& s, int k, const T* X, const T* Gt, const T* W, T* V, const int* done,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_wide_finish(const Shape& s, int k, const T* Gt, const T* V, double* Mk, const int* done,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_wide_gram(const Shape& s, int k, const T* Gt, const T* W, T* Tg, T* Kk, const int* done,
                             cudaStream_t st);
// The first two steps of the order-4 Gram chain (T2 of k_gram_io: t1 scratch of
// I_o I_c R_{k,l}(R_{k,l}+1)/2 entries) as two batched products over i_o, the
// alternative to one CTA per i_o (selected by IFCTN_GRAM_GEMM=1).
template <typename T>
cudaError_t launch_gram4_gemm(const Shape& s, int k, const T* Gt, const T* W, T* t1, T* t2, const int* done,
                              cudaStream_t st);

// Column solves of mode k with one CTA per column (order 3 or 4; ranks up to
// WIDE_RMAX, Q_k up to WIDE_QMAX): H in shared memory, FP64 Cholesky, W refresh.
template <typename T>
cudaError_t launch_cta_solve(const Shape& s, int k, double rho, const double* Mk, const T* Kk, double* Gd, T* Gt,
                             T* W, int* flags, const int* done, cudaStream_t st);

// eq. (updateX) fused with the reconstruction and the sweep's reductions.
template <typename T>
cudaError_t launch_xupdate(const Shape& sh, double rho, T* X, const uint32_t* maskbits, const T* W,
                           double* xpart, int nblocks, const int* done, cudaStream_t st);

// Reconstruction only (out may be null: then only sum of squares into xpart).
template <typename T>
cudaError_t launch_reconstruct(const Shape& sh, const T* W, T* out, double* xpart, int nblocks,
                               cudaStream_t st);

// RSE / RMSE partial sums against a ground truth.
template <typename T>
cudaError_t launch_metrics(const Shape& sh, const T* X, const T* Xt, const uint32_t* maskbits,
                           double* mpart, int nblocks, const int* done, cudaStream_t st);

// All pair matrices from the FP64 master factors.
template <typename T>
cudaError_t launch_pairs(const Shape& sh, const double* Gd, T* W, cudaStream_t st);

// X^0 = P_Omega(O) and the mask bitset.
template <typename T>
cudaError_t launch_init_x(long long P, const T* O, const uint8_t* mask, T* X, cudaStream_t st);
cudaError_t launch_pack_mask(long long P, const uint8_t* mask, uint32_t* bits, cudaStream_t st);

// FP64 master -> working-dtype copy of the factors.
template <typename T>
cudaError_t launch_cast_factors(int n, const double* Gd, T* Gt, cudaStream_t st);

// Fixed-order reduction of the sweep partials into the log record.
struct SweepStat {
    double rel_change, objective, rse, rmse, dx2, x2;
    int sweep, converged, flags, pad;
};
cudaError_t launch_finalize(const double* xpart, int nblocks, const double* mpart, int mblocks,
                            long long nmiss_total, const double* tol, SweepStat* log, int log_cap,
                            int* sweep_counter, int* done, const int* flags, cudaStream_t st);

cudaError_t launch_finalize8(const double* xpart, int nblocks, int met, long long nmiss, const double* tol,
                             SweepStat* log, int log_cap, int* sweep_counter, int* done, const int* flags,
                             cudaStream_t st);

// Sum of squares of xpart[0] slots (used for the default initial scaling).
cudaError_t launch_sum_partials(const double* xpart, int nblocks, int stride, int slot,
                                double* out, cudaStream_t st);

// scale factors in place by a device scalar: G *= s^(1/(N(N-1)))
cudaError_t launch_scale_factors(int n, double* Gd, const double* ratio, double expo,
                                 cudaStream_t st);

template <typename T>
cudaError_t launch_sumsq(long long P, const T* X, double* part, int nblocks, cudaStream_t st);
cudaError_t launch_count_bits(long long nwords, const uint32_t* bits, double* part, int nblocks,
                              cudaStream_t st);
cudaError_t launch_to_double(long long n, const float* a, double* b, cudaStream_t st);
// Failure-path diagnostic: a grid barrier one CTA never joins and an mbarrier
// phase no copy completes, each bounded by `budget` clock cycles (sets
// FLAG_TIMEOUT in *flags; *count must be zero).
cudaError_t launch_wait_selftest(int* flags, unsigned* count, long long budget, cudaStream_t st);

}  // namespace ifctn
