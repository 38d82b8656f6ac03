// ifctn_persistent.h -- parameters of the persistent sweep kernel.
#pragma once
#include "ifctn_launch.h"

namespace ifctn {

// Row stride of K_k when the solve holds it in shared memory: odd, so that the
// lanes of a warp, which read K at rows a multiple of the stride apart, fall on
// different banks (an even Q such as 36 or 192 put them on one bank: 8- to
// 24-way conflicts).
__host__ __device__ inline int k_stride(int Q) { return Q | 1; }

constexpr int PERSISTENT_THREADS = 256;  // threads per CTA of the persistent kernel

template <typename T>
struct SweepParams {
    Shape sh;
    ContractPlan pl[MAXN];
    const UnitDesc* units[MAXN];
    int gunits[MAXN];        // Gram work units of phase 1, per mode
    int gram_iob[MAXN];      // io values per Gram unit (order 3), per mode
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
    double rho;
    long long nmiss;
    int nsweeps;
    int nstages;
    int solve_k_in_smem;
    int gram_chunk;
    unsigned long long* tstamp;  // optional phase timestamps of one sweep (stamp_sweep)
    const int* stab[MAXN];       // per-mode index tables of the column solves (solve_stage_tables)
    int stamp_mode;              // mode whose first column's solve sub-steps are timestamped
    int stamp_sweep;             // sweep of the launch whose phases are timestamped
    double inv1p;                // 1 / (1 + rho), precomputed
    double tolv;                 // stop tolerance of this launch (0 = none)
    int xu_rows;                 // X update: rows of a slab per work unit
    int xu_wab_smem;             // X update: W_{A,B} kept in shared memory
    int xu_variant;              // X update (per-stage path): batch / residency variant
    int solve_nw;                // warps of a CTA that take columns in the solve (0: all); the rest help stage and refresh
    int cta0, ncta;              // the job's slice of the launch's grid (first CTA, CTA count)
};

// Index tables of the column solves of mode k (the same for every column):
// for each stage slot ti of the non-k modes (ranks Rm, last slot fastest)
//   cbt[ti][o]  K index of (o, c = 0), o over the other slots' combinations
//   dgt[ti][o]  digits of o, 3 bits per slot
//   lnt[ti][l]  lane l's first (o, o2) of the H sums, o | o2 << 16 (l < 32),
//               and at l = 32 the step of 32 combinations, dq | dr << 16
// laid out [cbt 3Q][dgt 3Q][lnt 3 x SOLVE_TAB_LANE] (Q = product of Rm).
constexpr int SOLVE_TAB_LANE = 33;
__host__ __device__ inline int solve_tab_ints(int Q) { return 6 * Q + 3 * SOLVE_TAB_LANE; }
inline void solve_stage_tables(const Shape& s, int k, int* out) {
    int Rm[3] = {1, 1, 1}, st[3] = {1, 1, 1}, nm = 0, Q = 1;
    for (int q = 0; q < s.N; ++q)
        if (q != k) {
            Rm[nm] = s.R[k][q];
            Q *= Rm[nm++];
        }
    for (int t = nm - 2; t >= 0; --t) st[t] = st[t + 1] * Rm[t + 1];
    int* cbt = out;
    int* dgt = out + 3 * Q;
    int* lnt = out + 6 * Q;
    for (int i = 0; i < solve_tab_ints(Q); ++i) out[i] = 0;
    for (int ti = 0; ti < nm; ++ti) {
        const int Ri = Rm[ti], sp = st[ti], Qo = Q / Ri;
        for (int o = 0; o < Qo; ++o) {
            const int hi = o / sp;
            cbt[ti * Q + o] = hi * Ri * sp + (o - hi * sp);
            int rem = o, pk = 0;
            for (int t = nm - 1; t >= 0; --t) {
                if (t == ti) continue;
                pk |= (rem % Rm[t]) << (3 * t);
                rem /= Rm[t];
            }
            dgt[ti * Q + o] = pk;
        }
        for (int l = 0; l < 32; ++l) lnt[ti * SOLVE_TAB_LANE + l] = (l / Qo) | ((l % Qo) << 16);
        lnt[ti * SOLVE_TAB_LANE + 32] = (32 / Qo) | ((32 % Qo) << 16);
    }
}

template <typename T>
int persistent_smem_bytes(const SweepParams<T>& p);
template <typename T>
int persistent_max_grid(int smem);
template <typename T>
cudaError_t launch_persistent(const SweepParams<T>& p, int grid, int smem, cudaStream_t st);
// several jobs in one cooperative launch (jobs: device array, slices in
// ascending cta0 covering [0, grid)); the occupancy-limited grid of that kernel
template <typename T>
cudaError_t launch_persistent_multi(const SweepParams<T>* jobs, int njobs, int grid, int smem, cudaStream_t st);
template <typename T>
int persistent_multi_max_grid(int smem);
// the column solves of mode k with the W_{k,.} refresh (per-stage path)
template <typename T>
cudaError_t launch_solve_cols(const SweepParams<T>& p, int k, cudaStream_t st);
// the X update of the per-stage path: per-CTA sums (6 of 8 slots) into xpart
template <typename T>
cudaError_t launch_xupdate_slab(const SweepParams<T>& p, double* xpart, int nblocks, cudaStream_t st);

}  // namespace ifctn
