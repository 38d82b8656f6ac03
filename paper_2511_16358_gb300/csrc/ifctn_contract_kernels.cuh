// ifctn_contract_kernels.cuh -- the streaming mode-k contraction M_k = X_(k) Z_k.
// (standalone kernels; instantiated per dtype in ifctn_persistent_f{32,64}.cu)
//
// Prop. 1 writes the mode-k sub-network as
//     Z_k(i_{-k}, r) = S_k(i_{-k}) * prod_{m != k} G_{m,k}(r_m, i_m),
//     S_k = broadcast product of W_{p,q} = G_{p,q}^T G_{q,p} over pairs p,q != k,
// and eq. (updateG) needs, for every column j of every G_{k,i}, the vector
// A_j^T x_j.  All of these are contractions of one matrix,
//     M_k(j, r) = sum_{i_{-k}} X(i_k = j, i_{-k}) Z_k(i_{-k}, r),
// against the Kronecker vector E_j of the other columns G_{k,m}(:, j), so the
// whole mode needs a single pass over X.  Z_k is never formed: its entries are
// built on the fly from the small W and G matrices (the "coefficient builder").
//
// The pass is one-read HBM streaming.  The tensor is cut into slabs (all
// entries sharing the indices of modes 0..N-3); each CTA takes a list of slabs
// and moves contiguous slab tiles into a shared-memory ring with 1-D TMA bulk
// copies (cp.async.bulk + mbarrier), several stages ahead of the compute.
// Inside a tile the contraction is hierarchical, so each tensor entry costs
// about R_{k,B} + 2 FMAs:
//   ROW kernel (k is not the last mode): a thread owns one row a of mode N-2,
//     contracts the contiguous mode N-1 in registers (u = R values), folds the
//     row into a register tile z over one more mode, and the remaining modes
//     are contracted at the flush or in the finisher.
//   COL kernel (k is the last mode): a thread owns one column b, contracts
//     mode N-2 in registers and folds slabs into z the same way.
// Partials are written per work unit and reduced by the finisher in a fixed
// order, so results are deterministic (no atomics).
#pragma once
#include "ifctn_contract_dev.cuh"
#include "ifctn_plan.h"

namespace ifctn {
namespace {
using namespace cdev;

template <typename T, int RB>
__global__ void __launch_bounds__(256) k_contract_row(const __grid_constant__ ContractArgs<T> A) {
    pdl_begin();
    if (*A.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    if (threadIdx.x == 0) {
        for (int i = 0; i < A.pl.nstages; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int pipe = 0;
    row_unit_body<T, RB>(A, blockIdx.x, smem + 128, bars, pipe, nullptr);
}

template <typename T, int RA>
__global__ void __launch_bounds__(256) k_contract_col(const __grid_constant__ ContractArgs<T> A) {
    pdl_begin();
    if (*A.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    if (threadIdx.x == 0) {
        for (int i = 0; i < A.pl.nstages; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int pipe = 0;
    col_unit_body<T, RA>(A, blockIdx.x, smem + 128, bars, pipe);
}

// ---------------------------------------------------------------------------
// finisher: M_k(row, q) from the partials (fixed order)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_contract_finish(const __grid_constant__ Shape s, const int k,
                                                         const __grid_constant__ ContractPlan pl,
                                                         const UnitDesc* __restrict__ units,
                                                         const T* __restrict__ part,
                                                         const T* __restrict__ Gt,
                                                         double* __restrict__ Mk,
                                                         const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    const int Ik = s.I[k], Q = pl.Q, Qp = pl.Qp;
    const long long total = static_cast<long long>(Ik) * Q;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int row = static_cast<int>(idx / Q), q = static_cast<int>(idx - static_cast<long long>(row) * Q);
        T acc = T(0);
        if (pl.kcase == CASE_F) {
            for (int sl = 0; sl < pl.nslot; ++sl)
                acc += part[(static_cast<size_t>(row) * pl.nslot + sl) * Q + q];
        } else {
            const int rd = pl.dmode >= 0 ? q / Qp : 0;
            const int qp = q - rd * Qp;
            const bool colcase = pl.kcase == CASE_COL;
            for (int un = 0; un < pl.nunits; ++un) {
                const int lo = colcase ? units[un].b0 : units[un].a0;
                const int hi = colcase ? units[un].b1 : units[un].a1;
                if (row < lo || row >= hi) continue;
                T v = part[(static_cast<size_t>(un) * pl.nrow + row) * Qp + qp];
                if (pl.dmode >= 0) v *= gfac(Gt, s, pl.dmode, k, rd, units[un].key);
                acc += v;
            }
        }
        Mk[idx] = static_cast<double>(acc);
    }
}

template <typename T, int R>
cudaError_t launch_row_r(const ContractArgs<T>& a, cudaStream_t st) {
    auto kern = k_contract_row<T, R>;
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), a.pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.pl.nunits, a.pl.nthreads, a.pl.smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int R>
cudaError_t launch_col_r(const ContractArgs<T>& a, cudaStream_t st) {
    auto kern = k_contract_col<T, R>;
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), a.pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.pl.nunits, a.pl.nthreads, a.pl.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_contract(const ContractArgs<T>& a, cudaStream_t st) {
    if (a.pl.warp) return launch_contract_warp<T>(a, a.pl.grid, st);
    const bool col = a.pl.kcase == CASE_COL;
    switch (a.pl.R1) {
#define IFCTN_CASE(R) \
    case R:           \
        return col ? launch_col_r<T, R>(a, st) : launch_row_r<T, R>(a, st);
        IFCTN_CASE(1)
        IFCTN_CASE(2)
        IFCTN_CASE(3)
        IFCTN_CASE(4)
        IFCTN_CASE(5)
        IFCTN_CASE(6)
        IFCTN_CASE(7)
        IFCTN_CASE(8)
#undef IFCTN_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

// Row-parallel finisher for the unit-keyed partials (CASE_A, CASE_COL): one CTA
// per output row; thread (g, qp) sums the units g, g + ng, ... that cover the
// row, times G_{d,k}(rd, key) for every rd of the deferred mode d, and the
// groups are added in a fixed order (deterministic).
template <typename T>
__global__ void __launch_bounds__(1024) k_contract_finish_rows(const __grid_constant__ Shape s, const int k, const __grid_constant__ ContractPlan pl,
                                                               const UnitDesc* __restrict__ units,
                                                               const T* __restrict__ part, const T* __restrict__ Gt,
                                                               double* __restrict__ Mk, const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    extern __shared__ __align__(16) unsigned char fsm[];
    T* red = reinterpret_cast<T*>(fsm);  // [blockDim.x][RMAX]
    const int row = blockIdx.x;
    const int Qp = pl.Qp;
    const int ng = blockDim.x / Qp;
    const int g = threadIdx.x / Qp, qp = threadIdx.x - g * Qp;
    const bool colcase = pl.kcase == CASE_COL;
    const int Rd = pl.dmode >= 0 ? s.R[k][pl.dmode] : 1;
    T acc[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) acc[r] = T(0);
    if (g < ng) {
        // the units that cover this row: a stride when the plan knows it
        const int u0 = pl.fin_mod > 0 ? row / pl.fin_div : 0;
        const int us = pl.fin_mod > 0 ? pl.fin_mod : 1;
#pragma unroll 4
        for (int un = u0 + g * us; un < pl.nunits; un += ng * us) {
            const UnitDesc u = units[un];
            const int lo = colcase ? u.b0 : u.a0, hi = colcase ? u.b1 : u.a1;
            if (row < lo || row >= hi) continue;
            const T v = part[(static_cast<size_t>(un) * pl.nrow + row) * Qp + qp];
            if (pl.dmode >= 0) {
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < Rd) acc[r] = fma(gfac(Gt, s, pl.dmode, k, r, u.key), v, acc[r]);
            } else {
                acc[0] += v;
            }
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
            if (r < Rd) red[(g * RMAX + r) * Qp + qp] = acc[r];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < Rd * Qp; q += blockDim.x) {
        const int rd = q / Qp, qq = q - rd * Qp;
        T a = T(0);
        for (int gg = 0; gg < ng; ++gg) a += red[(gg * RMAX + rd) * Qp + qq];
        Mk[static_cast<size_t>(row) * pl.Q + q] = static_cast<double>(a);
    }
}

template <typename T>
cudaError_t launch_contract_finish(const Shape& sh, int k, const ContractPlan& pl,
                                   const UnitDesc* units, const T* part, const T* Gt, double* Mk,
                                   const int* done, cudaStream_t st) {
    if (pl.kcase != CASE_F && pl.Qp <= 256) {
        // one CTA per output row; with few rows and many units a row gets up to
        // 1024 threads, so that each sums fewer units (the kernel is latency-bound)
        const int per_row = pl.nunits / (pl.fin_mod > 0 ? pl.fin_mod : 1);
        int threads = 256;
        while (threads < 1024 && sh.I[k] * (threads / 256) < 2 * num_sms() && per_row / (threads / pl.Qp) > 4)
            threads *= 2;
        const int smem = threads * RMAX * static_cast<int>(sizeof(T));
        cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(k_contract_finish_rows<T>), smem);
        if (e != cudaSuccess) return e;
        k_contract_finish_rows<T><<<sh.I[k], threads, smem, st>>>(sh, k, pl, units, part, Gt, Mk, done);
        return cudaGetLastError();
    }
    const long long total = static_cast<long long>(sh.I[k]) * pl.Q;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 1216) blocks = 1216;
    if (blocks < 1) blocks = 1;
    k_contract_finish<T><<<blocks, 256, 0, st>>>(sh, k, pl, units, part, Gt, Mk, done);
    return cudaGetLastError();
}

}  // namespace ifctn
