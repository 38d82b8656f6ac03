// ifctn_persistent.h -- parameters of the persistent sweep kernel.
#pragma once
#include "ifctn_launch.h"

namespace ifctn {

template <typename T>
struct SweepParams {
    Shape sh;
    ContractPlan pl[MAXN];
    const UnitDesc* units[MAXN];
    int gunits[MAXN];        // Gram work units of phase 1, per mode
    T* X;
    const uint32_t* mb;
    const T* Xt;             // ground truth for RSE/RMSE, or null
    double* Gd;
    T* Gt;
    T* W;
    T* part;
    T* gbuf;                 // Gram intermediate T2
    T* Kk;
    double* Mk[MAXN];
    double* xpart;           // 2 x grid x 8 per-CTA sums (double buffered by sweep)
    SweepStat* log;
    int log_cap;
    int* counter;
    int* done;
    int* flags;
    const double* tol;
    unsigned* bar_count;
    unsigned* bar_gen;
    double rho;
    long long nmiss;
    int nsweeps;
    int nstages;
    int solve_k_in_smem;
    int gram_chunk;
    unsigned long long* tstamp;  // optional phase timestamps of the first sweep
    double inv1p;                // 1 / (1 + rho), precomputed
    double tolv;                 // stop tolerance of this launch (0 = none)
    int xu_rows;                 // X update: rows of a slab per work unit
    int xu_wab_smem;             // X update: W_{A,B} kept in shared memory
};

template <typename T>
int persistent_smem_bytes(const SweepParams<T>& p);
template <typename T>
int persistent_max_grid(int smem);
template <typename T>
cudaError_t launch_persistent(const SweepParams<T>& p, int grid, int smem, cudaStream_t st);
// the column solves of mode k with the W_{k,.} refresh (per-stage path)
template <typename T>
cudaError_t launch_solve_cols(const SweepParams<T>& p, int k, cudaStream_t st);
// the X update of the per-stage path: per-CTA sums (6 of 8 slots) into xpart
template <typename T>
cudaError_t launch_xupdate_slab(const SweepParams<T>& p, double* xpart, int nblocks, cudaStream_t st);

}  // namespace ifctn
