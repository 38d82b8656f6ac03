// ifctn_persistent_impl.cuh -- the whole PAM run (Algorithm 1) in one cooperative
// launch.
//
// One sweep is a chain of dependent phases (per mode k: contraction + Gram
// partials, their reduction, the column solves; then the X update).  Issued
// as separate kernels every phase pays a launch and a cold start, which
// dominates for tensors that live in L2.  Here one persistent grid (as many
// CTAs as fit co-resident, guaranteed by a cooperative launch) runs every
// phase of every sweep and separates them with a software grid barrier:
//
//   mode k:  P1  streaming contraction units (TMA-fed, ifctn_contract_dev.cuh)
//                + Gram chain units, grid-strided over CTAs        | barrier
//            P2  K_k and M_k reductions of the partials, one lane
//                group per output                                   | barrier
//            P3  column solves of eq. (updateG) + W_{k,.} refresh   | barrier
//   then     P4  fused reconstruct + masked X update (eq. (updateX))| barrier
//            P5  every CTA reduces the per-CTA sums in the same fixed
//                order, so all CTAs take the same stop decision.
//
// All reductions are fixed-order, so the factors and the tensor do not depend
// on the grid size.  Every wait is bounded; on expiry a flag is raised and
// the kernel returns.
#pragma once
#include <algorithm>
#include <type_traits>

#include "ifctn_contract_dev.cuh"
#include "ifctn_persistent.h"

namespace ifctn {
namespace {

using cdev::contract_col_unit;
using cdev::contract_row_unit;

constexpr int PT = PERSISTENT_THREADS;
constexpr int PW = PT / 32;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}



// Software grid barrier over the nctas CTAs of one job (the grid is
// co-resident: cooperative launch; several jobs can share a launch, each with
// its own counter).  The arrival counter only grows during a launch (the host
// zeroes it before each launch): barrier number b of the launch is passed
// once it reaches b * nctas.  Thread 0 of a CTA arrives with a release reduction and
// spins with acquire loads until the target, bounded by a clock budget (on
// expiry: timeout flag, and the kernel returns).  Every CTA passes the same
// sequence of barriers, so `nb` (this CTA's count of barriers passed) agrees.
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned& nb, int* flags, unsigned nctas,
                                             long long budget = WAIT_BUDGET_CYCLES) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    ++nb;
    if (threadIdx.x == 0) {
        const unsigned target = nb * nctas;
        red_release_add_u32(count, 1u);
        const long long t0 = clock64();
        while (ld_acquire_u32(count) < target) {
            if (clock64() - t0 > budget) {
                atomicOr(flags, FLAG_TIMEOUT);
                break;
            }
        }
    }
    __syncthreads();
    return (*reinterpret_cast<volatile int*>(flags) & FLAG_TIMEOUT) == 0;
}

__device__ __forceinline__ int nonk(const Shape& s, int k, int* m) {
    int t = 0;
    for (int q = 0; q < s.N; ++q)
        if (q != k) m[t++] = q;
    return t;
}

// sum over a group of L lanes (L a power of two, groups aligned in the warp)
template <typename T>
__device__ __forceinline__ T group_sum(T v, int L) {
    for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int pow2_at_least(int x) {
    int L = 1;
    while (L < x && L < 32) L <<= 1;
    return L;
}

// Hint the L2 with the tensor span of a CTA's next contraction unit while it
// works on the current one (bulk prefetch, no shared memory involved).
template <typename T>
__device__ __forceinline__ void prefetch_unit(const SweepParams<T>& p, int k, int uidx) {
    const UnitDesc u = p.units[k][uidx];
    const Shape& s = p.sh;
    const long long e0 = (static_cast<long long>(u.f0) * s.IA + u.a0) * s.IB;
    long long n = static_cast<long long>(u.a1 - u.a0) * s.IB;
    if (u.fstride == 1) n += static_cast<long long>(u.ns - 1) * s.IA * s.IB;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p.X + e0) & ~uintptr_t(15);
    uintptr_t hi = (reinterpret_cast<uintptr_t>(p.X + e0 + n) + 15) & ~uintptr_t(15);
    if (hi - lo > (1u << 20)) hi = lo + (1u << 20);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(static_cast<unsigned>(hi - lo))
                 : "memory");
}

// The out-of-line unit bodies read their arguments through a reference; the
// per-mode arguments live in shared memory (built once per launch), so those
// reads are shared loads rather than loads from a per-thread stack copy.
template <typename T>
__device__ void build_contract_args(const SweepParams<T>& p, ContractArgs<T>* a) {
    for (int k = 0; k < p.sh.N; ++k) {
        a[k].X = p.X;
        a[k].Gt = p.Gt;
        a[k].W = p.W;
        a[k].sh = p.sh;
        a[k].k = k;
        a[k].pl = p.pl[k];
        a[k].units = p.units[k];
        a[k].part = p.part;
        a[k].flags = p.flags;
        a[k].done = p.done;
    }
}

template <typename T>
__device__ bool contract_dispatch(const ContractArgs<T>& a, int uidx, unsigned char* smem, uint64_t* bars,
                                  int& pipe, int* wtag) {
    const bool col = a.pl.kcase == CASE_COL;
    switch (a.pl.R1) {
#define IFCTN_PCASE(R) \
    case R:            \
        return col ? contract_col_unit<T, R>(a, uidx, smem, bars, pipe) : contract_row_unit<T, R>(a, uidx, smem, bars, pipe, wtag);
        IFCTN_PCASE(1)
        IFCTN_PCASE(2)
        IFCTN_PCASE(3)
        IFCTN_PCASE(4)
        IFCTN_PCASE(5)
        IFCTN_PCASE(6)
        IFCTN_PCASE(7)
        IFCTN_PCASE(8)
#undef IFCTN_PCASE
        default:
            return false;
    }
}

// ---------------------------------------------------------------------------
// Gram units (phase 1).  Non-k modes ascending: [o, l] (N=3), [o, c, l] (N=4).
//   N=3: T2[io][x][y] = sum_il W_ol(io,il)^2 g_l(x,il) g_l(y,il)
//   N=4: T1[ic][x][y] = W_oc(io,ic)^2 sum_il (W_ol(io,il) W_cl(ic,il))^2 g_l g_l
//        T2[io][(xc,xl)][(yc,yl)] = sum_ic g_c(xc,ic) g_c(yc,ic) T1[ic][xl][yl]
// with g_m = G_{m,k}.  K_k = sum_io g_o g_o^T (x) T2[io] is formed in phase 2.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void gram_unit(const SweepParams<T>& p, int k, int gu, unsigned char* smem) {
    const Shape& s = p.sh;
    int m[3];
    nonk(s, k, m);
    T* sm = reinterpret_cast<T*>(smem);
    const int tid = threadIdx.x;
    if (s.N == 3) {
        const int o = m[0], l = m[1];
        const int Io = s.I[o], Il = s.I[l], Rl = s.R[k][l];
        const int iob = p.gram_iob[k];
        const int io0 = gu * iob, io1 = min(Io, io0 + iob);
        // rows at an odd stride: the threads of a warp read different rows at
        // the same il without bank conflicts
        const int ld = Il | 1;
        T* gl = sm;  // Rl x ld
        for (int r = 0; r < Rl; ++r) stage_async(gl + r * ld, p.Gt + s.goff[l][k] + r * Il, Il);
        T* wr = gl + Rl * ld;  // (io1-io0) x ld
        for (int r = 0; r < io1 - io0; ++r)
            stage_async(wr + r * ld, p.W + s.woff[o][l] + static_cast<long long>(io0 + r) * Il, Il);
        stage_wait();
        const int nout = (io1 - io0) * Rl * Rl;
        for (int idx = tid; idx < nout; idx += PT) {
            const int y = idx % Rl, x = (idx / Rl) % Rl, ir = idx / (Rl * Rl);
            const T* gx = gl + x * ld;
            const T* gy = gl + y * ld;
            const T* w2 = wr + ir * ld;
            T a0 = T(0), a1 = T(0);
            int il = 0;
            for (; il + 1 < Il; il += 2) {
                a0 = fma(w2[il] * w2[il], gx[il] * gy[il], a0);
                a1 = fma(w2[il + 1] * w2[il + 1], gx[il + 1] * gy[il + 1], a1);
            }
            if (il < Il) a0 = fma(w2[il] * w2[il], gx[il] * gy[il], a0);
            p.gbuf[(static_cast<long long>(io0 + ir) * Rl + x) * Rl + y] = a0 + a1;
        }
        __syncthreads();
        return;
    }
    // N = 4: one io per unit
    const int o = m[0], c = m[1], l = m[2];
    const int io = gu;
    const int Ic = s.I[c], Il = s.I[l], Rc = s.R[k][c], Rl = s.R[k][l];
    const int Q2 = Rc * Rl;
    T* gl = sm;                    // Rl x Il
    T* gc = gl + Rl * Il;          // Rc x Ic
    T* wol = gc + Rc * Ic;         // Il
    T* t2a = wol + Il;             // Q2 x Q2 accumulators
    T* t1 = t2a + Q2 * Q2;         // chunk x Rl x Rl
    stage_async(gl, p.Gt + s.goff[l][k], Rl * Il);
    stage_async(gc, p.Gt + s.goff[c][k], Rc * Ic);
    stage_async(wol, p.W + s.woff[o][l] + static_cast<long long>(io) * Il, Il);
    for (int idx = tid; idx < Q2 * Q2; idx += PT) t2a[idx] = T(0);
    const int chunk = max(1, min(Ic, p.gram_chunk));
    stage_wait();
    for (int ic0 = 0; ic0 < Ic; ic0 += chunk) {
        const int nc = min(chunk, Ic - ic0);
        for (int idx = tid; idx < nc * Rl * Rl; idx += PT) {
            const int y = idx % Rl, x = (idx / Rl) % Rl, icr = idx / (Rl * Rl);
            const int ic = ic0 + icr;
            const T* wcl = p.W + s.woff[c][l] + static_cast<long long>(ic) * Il;
            const T* gx = gl + x * Il;
            const T* gy = gl + y * Il;
            T acc = T(0);
            for (int il = 0; il < Il; ++il) {
                const T w = wol[il] * wcl[il];
                acc = fma(w * w, gx[il] * gy[il], acc);
            }
            const T woc = p.W[s.woff[o][c] + static_cast<long long>(io) * Ic + ic];
            t1[idx] = acc * woc * woc;
        }
        __syncthreads();
        for (int idx = tid; idx < Q2 * Q2; idx += PT) {
            const int Y = idx % Q2, X = idx / Q2;
            const int xc = X / Rl, xl = X - xc * Rl, yc = Y / Rl, yl = Y - yc * Rl;
            T acc = t2a[idx];
            for (int icr = 0; icr < nc; ++icr) {
                const int ic = ic0 + icr;
                acc = fma(gc[xc * Ic + ic] * gc[yc * Ic + ic], t1[(icr * Rl + xl) * Rl + yl], acc);
            }
            t2a[idx] = acc;
        }
        __syncthreads();
    }
    T* dst = p.gbuf + static_cast<long long>(io) * Q2 * Q2;
    for (int idx = tid; idx < Q2 * Q2; idx += PT) dst[idx] = t2a[idx];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Phase 2: K_k and M_k from the partials.  A group of L lanes reduces one
// output; the groups of the whole grid share the outputs.
// ---------------------------------------------------------------------------
// The CTA's index within its job and the job's CTA count: a launch can run
// several jobs on consecutive slices of its grid (cta0 = the slice's first CTA).
template <typename T>
__device__ __forceinline__ int vbid(const SweepParams<T>& p) {
    return static_cast<int>(blockIdx.x) - p.cta0;
}

template <typename T>
__device__ void reduce_phase(const SweepParams<T>& p, int k, unsigned char* smem, bool stamp = false) {
    const int VB = vbid(p), VG = p.ncta;  // this job's CTA index and grid size
    const Shape& s = p.sh;
    // sub-step timestamps (slots 52..55) of CTA 0, thread 0, when `stamp` is set
    auto rstamp = [&](int n) {
        if (stamp && p.tstamp && VB == 0 && threadIdx.x == 0) p.tstamp[52 + n] = gtimer();
    };
    rstamp(0);
    const ContractPlan& pl = p.pl[k];
    int m[3];
    const int nm = nonk(s, k, m);
    const int o = m[0], Io = s.I[o], Ro = s.R[k][o];
    int Q2 = 1;
    for (int t = 1; t < nm; ++t) Q2 *= s.R[k][m[t]];
    const int Q = Ro * Q2;
    const int lane = threadIdx.x & 31;
    const long long gwarp = static_cast<long long>(VB) * PW + (threadIdx.x >> 5);
    const long long nwarps = static_cast<long long>(VG) * PW;
    // --- K (upper triangle, mirrored) ---
    {
        const int L = pow2_at_least((Io + 3) / 4);
        const int per = 32 / L;
        const long long gid = gwarp * per + lane / L;
        const long long ngroups = nwarps * per;
        const int sub = lane % L;
        const long long nout = static_cast<long long>(Q) * (Q + 1) / 2;
        const long long iters = (nout + ngroups - 1) / ngroups;
        for (long long it = 0; it < iters; ++it) {
            const long long out = gid + it * ngroups;
            T acc = T(0);
            int row = 0, col = 0;
            if (out < nout) {
                // out -> (row <= col) in row-major upper-triangle order
                long long r = 0, rem = out;
                while (rem >= Q - r) {
                    rem -= Q - r;
                    ++r;
                }
                row = static_cast<int>(r);
                col = static_cast<int>(r + rem);
                const int xo = row / Q2, X = row - xo * Q2, yo = col / Q2, Y = col - yo * Q2;
                const T* gx = p.Gt + s.goff[o][k] + xo * Io;
                const T* gy = p.Gt + s.goff[o][k] + yo * Io;
                // unrolled so that a lane's loads are in flight together
                if (nm == 1) {
#pragma unroll 8
                    for (int io = sub; io < Io; io += L) acc = fma(gx[io], gy[io], acc);
                } else {
                    const T* tp = p.gbuf + static_cast<long long>(X) * Q2 + Y;
                    const long long st = static_cast<long long>(Q2) * Q2;
#pragma unroll 8
                    for (int io = sub; io < Io; io += L) acc = fma(gx[io] * gy[io], tp[io * st], acc);
                }
            }
            acc = group_sum(acc, L);
            if (out < nout && sub == 0) {
                p.Kk[static_cast<long long>(row) * Q + col] = acc;
                p.Kk[static_cast<long long>(col) * Q + row] = acc;
            }
        }
    }
    rstamp(1);
    // --- M, units covering every row: column tiles of TW columns (narrower
    // when 32-wide tiles would leave CTAs idle); within a warp the lanes of a
    // column split the units and meet by shuffles, warps meet in shared memory ---
    if (pl.kcase != CASE_F && pl.key_div > 0) {
        const int Qp = pl.Qp;
        const int ncol = pl.nrow * Qp;
        int TW = 32;
        while (TW > 8 && (ncol + TW - 1) / TW < VG) TW >>= 1;
        const int SUBS = 32 / TW;
        const int ntile = (ncol + TW - 1) / TW;
        const int Rd = pl.dmode >= 0 ? s.R[k][pl.dmode] : 1;
        const int nu = pl.nunits;
        T* coef = reinterpret_cast<T*>(smem);      // Rd x nu
        T* red = coef + ((Rd * nu + 3) & ~3);      // PW x RMAX x 32
        if (VB < ntile) {
            if (pl.dmode >= 0 && pl.key_div == 1 && nu == s.I[pl.dmode]) {
                // coef(rd, u) = G_{d,k}(rd, u): the whole table, one copy
                stage_async(coef, p.Gt + s.goff[pl.dmode][k], Rd * nu);
                stage_wait();
            } else {
#pragma unroll 4
                for (int idx = threadIdx.x; idx < Rd * nu; idx += PT) {
                    const int rdd = idx / nu, u = idx - rdd * nu;
                    coef[idx] = pl.dmode >= 0 ? gfac(p.Gt, s, pl.dmode, k, rdd, u / pl.key_div) : T(1);
                }
                __syncthreads();
            }
            rstamp(2);
            const int warp = threadIdx.x >> 5;
            const int cl = lane % TW, sub = lane / TW;
            for (int tile = VB; tile < ntile; tile += VG) {
                const int c = tile * TW + cl;
                const bool valid = c < ncol;
                T acc[RMAX];
#pragma unroll
                for (int r = 0; r < RMAX; ++r) acc[r] = T(0);
                const T* pc = p.part + c;
                // batches of UB units: every load of a batch in flight before its FMAs
                constexpr int UB = 8;
                const int ustep = PW * SUBS;
                for (int u0 = warp * SUBS + sub; u0 < nu; u0 += ustep * UB) {
                    T vv[UB];
#pragma unroll
                    for (int t = 0; t < UB; ++t) {
                        const int u = u0 + t * ustep;
                        vv[t] = (valid && u < nu) ? pc[static_cast<size_t>(u) * ncol] : T(0);
                    }
#pragma unroll
                    for (int t = 0; t < UB; ++t) {
                        const int u = u0 + t * ustep;
                        if (u < nu)
#pragma unroll
                            for (int r = 0; r < RMAX; ++r)
                                if (r < Rd) acc[r] = fma(coef[r * nu + u], vv[t], acc[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < Rd)
                        for (int o = TW; o < 32; o <<= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
                if (sub == 0)
#pragma unroll
                    for (int r = 0; r < RMAX; ++r)
                        if (r < Rd) red[(warp * RMAX + r) * 32 + cl] = acc[r];
                __syncthreads();
                for (int idx = threadIdx.x; idx < Rd * TW; idx += PT) {
                    const int r = idx / TW, ln = idx - r * TW;
                    const int cc = tile * TW + ln;
                    if (cc < ncol) {
                        T v = T(0);
                        for (int w2 = 0; w2 < PW; ++w2) v += red[(w2 * RMAX + r) * 32 + ln];
                        const int row = cc / Qp, qp = cc - row * Qp;
                        p.Mk[k][static_cast<long long>(row) * Q + r * Qp + qp] = static_cast<double>(v);
                    }
                }
                __syncthreads();
            }
        }
        rstamp(3);
        return;
    }
    // --- M ---
    {
        const int Ik = s.I[k], Qp = pl.Qp;
        const bool isF = pl.kcase == CASE_F;
        const int nterm = isF ? pl.nslot : pl.nunits;
        const int L = pow2_at_least((nterm + 1) / 2);
        const int per = 32 / L;
        const long long gid = gwarp * per + lane / L;
        const long long ngroups = nwarps * per;
        const int sub = lane % L;
        const long long nout = static_cast<long long>(Ik) * Q;
        const long long iters = (nout + ngroups - 1) / ngroups;
        const bool colcase = pl.kcase == CASE_COL;
        for (long long it = 0; it < iters; ++it) {
            const long long out = gid + it * ngroups;
            T acc = T(0);
            if (out < nout) {
                const int row = static_cast<int>(out / Q), q = static_cast<int>(out - static_cast<long long>(row) * Q);
                if (isF) {
                    for (int sl = sub; sl < pl.nslot; sl += L)
                        acc += p.part[(static_cast<size_t>(row) * pl.nslot + sl) * Q + q];
                } else if (pl.key_div > 0) {
                    // every unit covers every row; the deferred key is u / key_div
                    const int rd = pl.dmode >= 0 ? q / Qp : 0;
                    const int qp = q - rd * Qp;
                    const T* pp0 = p.part + static_cast<size_t>(row) * Qp + qp;
                    const size_t ust = static_cast<size_t>(pl.nrow) * Qp;
                    if (pl.dmode >= 0) {
                        const T* gd = p.Gt + s.goff[pl.dmode][k] + rd * s.I[pl.dmode];
#pragma unroll 4
                        for (int u = sub; u < pl.nunits; u += L) acc = fma(pp0[u * ust], gd[u / pl.key_div], acc);
                    } else {
#pragma unroll 4
                        for (int u = sub; u < pl.nunits; u += L) acc += pp0[u * ust];
                    }
                } else {
                    const int rd = pl.dmode >= 0 ? q / Qp : 0;
                    const int qp = q - rd * Qp;
                    const UnitDesc* un = p.units[k];
                    for (int u = sub; u < pl.nunits; u += L) {
                        const int lo = colcase ? un[u].b0 : un[u].a0;
                        const int hi = colcase ? un[u].b1 : un[u].a1;
                        if (row < lo || row >= hi) continue;
                        T v = p.part[(static_cast<size_t>(u) * pl.nrow + row) * Qp + qp];
                        if (pl.dmode >= 0) v *= gfac(p.Gt, s, pl.dmode, k, rd, un[u].key);
                        acc += v;
                    }
                }
            }
            acc = group_sum(acc, L);
            if (out < nout && sub == 0) p.Mk[k][out] = static_cast<double>(acc);
        }
    }
}

// ---------------------------------------------------------------------------
// Phase 3: eq. (updateG) for every column j of mode k, one warp per column
// (columns dealt round-robin over the CTAs first, so every SM gets work).
// H = E_j^T K_k E_j and b = E_j^T M_k(j,:) + rho g_old with E_j the Kronecker
// product of the current columns G_{k,m}(:,j), m != i (identity in slot i);
// stages i ascending (Gauss-Seidel within the column).
//
// (H + rho I) g = b is solved by an LDL^T factorisation (the matrix is SPD
// with eigenvalues >= rho, so no pivoting) that every lane of the warp runs
// in registers.  FP64 path: the factorisation and the solves in FP64.  Mixed
// path: the factorisation in FP32 followed by a step of iterative refinement
// whose residual b - (H + rho I) g is formed in two-float arithmetic (about
// 48 significant bits from FP32 instructions only), which recovers the
// accuracy of an FP64 solve for the conditioning these systems have without
// GB300's FP64 pipe (one FP64 instruction per 64 cycles of a warp scheduler).
// (One refinement step: H itself carries the FP32 rounding of the
// contractions, so further steps would not change the result's accuracy.)
// ---------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ F recip_nr(F d) {
    // reciprocal: hardware FP32 estimate (rcp.approx, about 1 ulp), refined by
    // Newton-Raphson x <- x (2 - d x): once in FP32, twice more in FP64.  The
    // mixed path's factorisation only has to be good enough for one step of
    // FP64 iterative refinement.
    float xf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xf) : "f"(static_cast<float>(d)));
    const float df = static_cast<float>(d);
    xf = xf * (2.0f - df * xf);
    F x = static_cast<F>(xf);
    if (sizeof(F) == 8) {
        x = x * (F(2) - d * x);
        x = x * (F(2) - d * x);
    }
    return x;
}


// Sub-step timestamps of one column (slots 40..55 of the timestamp buffer):
// taken by lane 0 of warp 0 of CTA 0 on its first column when `stamp` is set.
#define IFCTN_SSTAMP(n)                                                        \
    do {                                                                       \
        if (stamp_col && lane == 0) p.tstamp[40 + (n)] = gtimer();             \
    } while (0)

// Shared-memory layout of the solve phase (byte offsets from the phase's base):
//   per-warp scratch (WSD doubles: the current columns in FP64 and in T (with
//   the low parts of their two-float form on the mixed path), H and b of a
//   stage, the solution), the tables G_{i,k} (T), the per-stage index tables
//   of the CTA, per-warp omega and M_k row in T (Qa entries each), K_k (T, when
//   kept in shared memory), per-warp M_k row (FP64, the cp.async target).
constexpr int WSD = 2 * RMAX * RMAX + 11 * RMAX;  // doubles per warp
// offsets inside a warp's scratch, in doubles (vs, gd) and in T (the rest)
constexpr int SC_VS = 0, SC_GD = 3 * RMAX, SC_T = 4 * RMAX;
constexpr int SC_AF = 0, SC_HV = RMAX * RMAX, SC_XF = 2 * RMAX * RMAX, SC_BV = SC_XF + RMAX, SC_VT = SC_BV + RMAX,
              SC_VLO_T = SC_VT + 3 * RMAX;  // T offset where the FP32 low parts start
constexpr int TAB_LANE = SOLVE_TAB_LANE;

struct SolveLayout {
    long long gik, tab, warp, wstride, K, Ms, total;
};

__host__ __device__ inline SolveLayout solve_layout(int Q, int tot, int sz, bool ksm) {
    SolveLayout L;
    const long long Qa = (Q + 3) & ~3;
    L.gik = static_cast<long long>(PW) * WSD * 8;
    L.tab = (L.gik + static_cast<long long>(tot) * sz + 15) & ~15LL;
    L.warp = (L.tab + static_cast<long long>(solve_tab_ints(Q)) * 4 + 15) & ~15LL;
    L.wstride = Qa * 2 * sz;
    L.K = (L.warp + PW * L.wstride + 15) & ~15LL;
    L.Ms = (L.K + (ksm ? static_cast<long long>(Q) * k_stride(Q) * sz : 0) + 15) & ~15LL;
    L.total = L.Ms + static_cast<long long>(PW) * Q * 8;
    return L;
}

template <typename T>
__device__ __forceinline__ T* warp_scratch_t(unsigned char* smem, int w) {
    return reinterpret_cast<T*>(reinterpret_cast<double*>(smem) + w * WSD + SC_T);
}


// Butterfly reduce-scatter across the warp: v[V] per lane (V = 32 or 64) ->
// the warp sums of value index lane (V = 32) or 2 lane, 2 lane + 1 (V = 64)
// in v[0] (, v[1]).  Each level sends half of the values still held to the
// partner lane, so the whole reduction is V - V/32 shuffles in five levels.
template <typename T, int V>
__device__ __forceinline__ void warp_reduce_scatter(T (&v)[V], int lane) {
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int o = 16 >> lv;
        const int n = V >> (lv + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < V / 2; ++i) {
            if (i < n) {
                const T send = up ? v[i] : v[i + n];
                const T keep = up ? v[i + n] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
}

// LDL^T of the SPD matrix A (lower triangle used) in registers, in place:
// unit-lower L below the diagonal, D on it, 1/D in id.  False if a pivot is
// not positive.
template <typename F, int RI>
__device__ __forceinline__ bool ldlt_regs(F (&A)[RI][RI], F (&id)[RI]) {
    bool ok = true;
#pragma unroll
    for (int c = 0; c < RI; ++c) {
        F d = A[c][c];
#pragma unroll
        for (int t = 0; t < c; ++t) d -= A[c][t] * A[c][t] * A[t][t];
        ok = ok && (d > F(0));
        A[c][c] = d;
        const F inv = recip_nr<F>(d);
        id[c] = inv;
#pragma unroll
        for (int r = c + 1; r < RI; ++r) {
            F v = A[r][c];
#pragma unroll
            for (int t = 0; t < c; ++t) v -= A[r][t] * A[c][t] * A[t][t];
            A[r][c] = v * inv;
        }
    }
    return ok;
}

// L D L^T x = b in registers (x holds b on entry)
template <typename F, int RI>
__device__ __forceinline__ void ldlt_solve_regs(const F (&A)[RI][RI], const F (&id)[RI], F (&x)[RI]) {
#pragma unroll
    for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int t = 0; t < r; ++t) x[r] -= A[r][t] * x[t];
#pragma unroll
    for (int r = 0; r < RI; ++r) x[r] *= id[r];
#pragma unroll
    for (int r = RI - 1; r >= 0; --r)
#pragma unroll
        for (int t = r + 1; t < RI; ++t) x[r] -= A[t][r] * x[t];
}

// Error-free transformations in FP32: a + b = s + e and a * b = p + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// One stage (slot ti, Ri = RI values) of the column solve, by one warp:
//   H(c, c2) = sum_{o, o2} omega(o) omega(o2) K[(o2, c2), (o, c)] + rho [c = c2]
//   b(c)     = sum_o omega(o) M_k(j, (o, c)) + rho g_old(c)
//   (H) g = b
// where (o, c) is the K index with digit c in slot ti, cb[o] the index of
// (o, 0) and sp the index step of the slot.  Lanes take (o, o2) combinations
// (lane's first one (o_0, o2_0), then steps of 32) and keep every pair
// c <= c2 (K is symmetric, so H is) and every b(c) in registers; one
// reduce-scatter leaves value q with lane q, which writes it out.  Every lane
// then factorises H and solves in registers.
//   FP64 path: all of it in FP64; the new column goes to gd.
//   Mixed path: FP32 factorisation and solve, then one step of refinement
//   whose residual b - H g is formed by lane r for row r in two-float
//   arithmetic (error-free products and sums of the FP32 sums, rho and the
//   old value as hi + lo pairs: about 48 significant bits, no FP64
//   instruction); the new column as a two-float pair replaces (ghi, glo).
// Returns false (uniformly) when H is not numerically SPD or the result is
// not finite; the old column is then left in place.
template <typename T, int RI>
__device__ __forceinline__ bool stage_solve(const T* __restrict__ K, const T* __restrict__ om,
                                            const int* __restrict__ cb, const T* __restrict__ mrow, int Q, int LK,
                                            int Qo, int sp, int lane, int olane, int dq, int dr, T rhoT, float rhi,
                                            float rlo, T* ghi, float* glo, T* Af, T* Hv, T* xf, T* bv, double* gd,
                                            unsigned long long* ts) {
    constexpr bool MIXED = sizeof(T) == 4;
    constexpr int NP = RI * (RI + 1) / 2;
    constexpr int V = NP + RI <= 32 ? 32 : 64;
    // optional sub-step timestamps (one profiled column): ts[0..3]
    auto stamp = [&](int n) {
        if (ts && lane == 0) ts[n] = gtimer();
    };
    T v[V];
#pragma unroll
    for (int q = 0; q < V; ++q) v[q] = T(0);
    (void)Q;
    const int spQ = sp * LK;  // K(row, col) at row * LK + col
    const int n = Qo * Qo;
    int o = olane & 0xffff;
    int o2 = olane >> 16;
    for (int f = lane; f < n; f += 32) {
        const T w = om[o] * om[o2];
        const T* kr = K + cb[o2] * LK + cb[o];
        int q = 0;
#pragma unroll
        for (int c2 = 0; c2 < RI; ++c2)
#pragma unroll
            for (int c = 0; c <= c2; ++c, ++q) v[q] = fma(kr[c2 * spQ + c * sp], w, v[q]);
        o += dq;
        o2 += dr;
        if (o2 >= Qo) {
            o2 -= Qo;
            ++o;
        }
    }
    for (int o1 = lane; o1 < Qo; o1 += 32) {
        const T w = om[o1];
        const T* mr = mrow + cb[o1];
#pragma unroll
        for (int c = 0; c < RI; ++c) v[NP + c] = fma(w, mr[c * sp], v[NP + c]);
    }
    stamp(0);
    warp_reduce_scatter<T, V>(v, lane);
#pragma unroll
    for (int h = 0; h < V / 32; ++h) {
        const int idx = V == 32 ? lane : 2 * lane + h;
        const T val = v[h];
        if (idx < NP) {
            int c2 = 0;
            while ((c2 + 1) * (c2 + 2) / 2 <= idx) ++c2;
            const int c = idx - c2 * (c2 + 1) / 2;
            const T hv = c == c2 ? val + rhoT : val;
            Af[c2 * RI + c] = hv;
            Af[c * RI + c2] = hv;
            if (MIXED) {
                Hv[c2 * RI + c] = val;
                Hv[c * RI + c2] = val;
            }
        } else if (idx < NP + RI) {
            const int c = idx - NP;
            bv[c] = val;
            xf[c] = fma(rhoT, ghi[c], val);
        }
    }
    __syncwarp();
    stamp(1);
    T A[RI][RI], id[RI], x[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
#pragma unroll
        for (int c = 0; c <= r; ++c) A[r][c] = Af[r * RI + c];
        x[r] = xf[r];
    }
    bool ok = ldlt_regs<T, RI>(A, id);
    ldlt_solve_regs<T, RI>(A, id, x);
    stamp(2);
    T xl = T(0);
#pragma unroll
    for (int r = 0; r < RI; ++r)
        if (lane == r) xl = x[r];
    if constexpr (MIXED) {
        // residual of row r: b_r - sum_t H(r, t) x_t, with b_r = bv_r + rho g_old(r)
        // and H(r, r) = Hv(r, r) + rho, in two-float arithmetic
        float rr = 0.f;
        if (lane < RI) {
            float sum = bv[lane], err = 0.f, p, pe, se;
            const float gh = ghi[lane], gl = glo[lane];
            two_prod(rhi, gh, p, pe);
            two_sum(sum, p, sum, se);
            err += pe + se + fmaf(rhi, gl, rlo * gh);
#pragma unroll
            for (int t = 0; t < RI; ++t) {
                two_prod(-Hv[lane * RI + t], x[t], p, pe);
                two_sum(sum, p, sum, se);
                err += pe + se;
            }
            two_prod(-rhi, xl, p, pe);
            two_sum(sum, p, sum, se);
            err += pe + se - rlo * xl;
            rr = sum + err;
        }
        float cr[RI];
#pragma unroll
        for (int t = 0; t < RI; ++t) cr[t] = __shfl_sync(0xffffffffu, rr, t);
        ldlt_solve_regs<float, RI>(A, id, cr);
        float cl = 0.f;
#pragma unroll
        for (int r = 0; r < RI; ++r)
            if (lane == r) cl = cr[r];
        float nh, nl;
        two_sum(xl, cl, nh, nl);
        if (lane < RI && !isfinite(nh)) ok = false;
        const bool all = __all_sync(0xffffffffu, ok) != 0;
        if (all && lane < RI) {
            ghi[lane] = nh;
            glo[lane] = nl;
        }
        stamp(3);
        return all;
    } else {
        if (lane < RI) {
            gd[lane] = xl;
            if (!isfinite(xl)) ok = false;
        }
        stamp(3);
        return __all_sync(0xffffffffu, ok) != 0;
    }
}

template <typename T>
__device__ void solve_phase(const SweepParams<T>& p, int k, unsigned char* smem, bool stamp = false) {
    const int VB = vbid(p), VG = p.ncta;  // this job's CTA index and grid size
    const Shape& s = p.sh;
    const int Ik = s.I[k];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    bool stamp_col = stamp && p.tstamp && VB == 0 && warp == 0;
    IFCTN_SSTAMP(0);
    if (VB >= Ik) return;  // no columns for this CTA
    constexpr bool MIXED = sizeof(T) == 4;
    int m[3];
    const int nm = nonk(s, k, m);
    int Rm[3] = {1, 1, 1}, st[3] = {1, 1, 1};
    int Q = 1;
    for (int t = 0; t < nm; ++t) {
        Rm[t] = s.R[k][m[t]];
        Q *= Rm[t];
    }
    for (int t = nm - 2; t >= 0; --t) st[t] = st[t + 1] * Rm[t + 1];
    int gko[3];
    int tot = 0;
    for (int t = 0; t < nm; ++t) {
        gko[t] = tot;
        tot += Rm[t] * s.I[m[t]];
    }
    const bool ksm = p.solve_k_in_smem != 0;
    const SolveLayout L = solve_layout(Q, tot, static_cast<int>(sizeof(T)), ksm);
    double* my = reinterpret_cast<double*>(smem) + warp * WSD;
    double* vs = my + SC_VS;  // 3 x RMAX current columns (FP64, fetched)
    double* gd = my + SC_GD;  // RMAX: new column (FP64 path)
    T* sc = warp_scratch_t<T>(smem, warp);
    T* Af = sc + SC_AF;  // RMAX*RMAX: H + rho I
    T* Hv = sc + SC_HV;  // RMAX*RMAX: H's sums (mixed path)
    T* xf = sc + SC_XF;  // RMAX: b
    T* bv = sc + SC_BV;  // RMAX: b's sums (mixed path)
    T* vt = sc + SC_VT;  // 3 x RMAX: current columns in T (high parts on the mixed path)
    float* vlo = reinterpret_cast<float*>(sc + SC_VLO_T);  // 3 x RMAX: low parts (mixed path)
    T* gik = reinterpret_cast<T*>(smem + L.gik);
    int* cbt = reinterpret_cast<int*>(smem + L.tab);  // [nm][Q] K index of (o, 0)
    int* dgt = cbt + 3 * Q;                            // [nm][Q] digits of o, 3 bits per slot
    int* lnt = dgt + 3 * Q;                            // [nm][TAB_LANE]: lane's first (o, o2); steps
    const int Qa = (Q + 3) & ~3;
    T* om = reinterpret_cast<T*>(smem + L.warp + warp * L.wstride);
    T* mf = om + Qa;
    T* Ks = reinterpret_cast<T*>(smem + L.K);
    double* Ms = reinterpret_cast<double*>(smem + L.Ms) + static_cast<size_t>(warp) * Q;
    const T* mrow = MIXED ? mf : reinterpret_cast<const T*>(Ms);
    // the current columns G_{k,m}(:, j) and the row M_k(j, :) of a column,
    // copied asynchronously (the first column's together with the tables)
    auto fetch_column = [&](int j) {
        for (int t = 0; t < nm; ++t)
            for (int r = lane; r < Rm[t]; r += 32)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(vs + t * RMAX + r)),
                             "l"(p.Gd + s.goff[k][m[t]] + r * Ik + j)
                             : "memory");
        const double* Mj = p.Mk[k] + static_cast<long long>(j) * Q;
        for (int q = lane; q < Q; q += 32)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(Ms + q)), "l"(Mj + q) : "memory");
    };
    // what the first column needs (its data, K, the index tables) in one
    // cp.async group; the tables G_{i,k}, read only by the W refresh, in a
    // second group that is waited for before the refresh
    const int NWc = p.solve_nw > 0 ? p.solve_nw : PW;  // warps that take columns (the others help stage and refresh)
    const int j0 = warp < NWc ? warp * VG + VB : Ik;
    if (j0 < Ik) fetch_column(j0);
    if (ksm) {  // rows at the odd stride k_stride(Q)
        const int LKs = k_stride(Q);
        if (LKs == Q) {
            stage_async(Ks, p.Kk, Q * Q);
        } else {
            for (int idx = threadIdx.x; idx < Q * Q; idx += blockDim.x) {
                const int r = idx / Q, c = idx - r * Q;
                if (sizeof(T) == 4)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(Ks + r * LKs + c)),
                                 "l"(p.Kk + idx)
                                 : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(Ks + r * LKs + c)),
                                 "l"(p.Kk + idx)
                                 : "memory");
            }
        }
    }
    stage_async(cbt, p.stab[k], solve_tab_ints(Q));
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int t = 0; t < nm; ++t) stage_async(gik + gko[t], p.Gt + s.goff[m[t]][k], Rm[t] * s.I[m[t]]);
    asm volatile("cp.async.commit_group;" ::: "memory");
    const T* K = ksm ? Ks : p.Kk;
    const int LK = ksm ? k_stride(Q) : Q;
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    IFCTN_SSTAMP(1);
    const double rho = p.rho;
    const T rhoT = static_cast<T>(rho);
    const float rhi = static_cast<float>(rho);
    const float rlo = static_cast<float>(rho - static_cast<double>(rhi));
    // W refresh by the whole CTA when every warp has at most one column
    const bool cta_refresh = static_cast<long long>(VG) * NWc >= Ik;
    if (!cta_refresh) {  // every warp refreshes its columns: the tables first
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
    }
    for (int j = j0; j < Ik; j += VG * NWc) {
        if (j != j0) {
            fetch_column(j);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
        }
        // the column vectors (two-float pairs on the mixed path) and the M_k
        // row in T, converted once per column
        for (int idx = lane; idx < nm * RMAX; idx += 32) {
            const int t = idx / RMAX, r = idx - t * RMAX;
            if (r < Rm[t]) {
                const double g = vs[idx];
                const T h = static_cast<T>(g);
                vt[idx] = h;
                if (MIXED) vlo[idx] = static_cast<float>(g - static_cast<double>(h));
            }
        }
        if (MIXED)
            for (int q = lane; q < Q; q += 32) mf[q] = static_cast<T>(Ms[q]);
        __syncwarp();
        IFCTN_SSTAMP(2);
        unsigned changed = 0;  // slots whose column was updated
        for (int ti = 0; ti < nm; ++ti) {
            const int i = m[ti], Ri = Rm[ti], sp = st[ti];
            const int Qo = Q / Ri;
            // omega(o) = prod over slots t != ti of v_t(digit_t(o))
            for (int o = lane; o < Qo; o += 32) {
                const int pk = dgt[ti * Q + o];
                T w = T(1);
                for (int t = 0; t < nm; ++t)
                    if (t != ti) w *= vt[t * RMAX + ((pk >> (3 * t)) & 7)];
                om[o] = w;
            }
            __syncwarp();
            if (ti == 0) IFCTN_SSTAMP(3);
            const int* cb = cbt + ti * Q;
            const int olane = lnt[ti * TAB_LANE + lane];
            const int steps = lnt[ti * TAB_LANE + 32];
            const int dq = steps & 0xffff, dr = steps >> 16;
            T* gh = vt + ti * RMAX;
            float* gl = vlo + ti * RMAX;
            unsigned long long* sts = (stamp_col && ti == 0) ? p.tstamp + 44 : nullptr;
            bool okc;
            switch (Ri) {
#define IFCTN_SOLVE_CASE(R)                                                                                     \
    case R:                                                                                                     \
        okc = stage_solve<T, R>(K, om, cb, mrow, Q, LK, Qo, sp, lane, olane, dq, dr, rhoT, rhi, rlo, gh, gl, Af, Hv, \
                                xf, bv, gd, sts);                                                               \
        break;
                IFCTN_SOLVE_CASE(1)
                IFCTN_SOLVE_CASE(2)
                IFCTN_SOLVE_CASE(3)
                IFCTN_SOLVE_CASE(4)
                IFCTN_SOLVE_CASE(5)
                IFCTN_SOLVE_CASE(6)
                IFCTN_SOLVE_CASE(7)
                default:
                    okc = stage_solve<T, 8>(K, om, cb, mrow, Q, LK, Qo, sp, lane, olane, dq, dr, rhoT, rhi, rlo, gh, gl,
                                            Af, Hv, xf, bv, gd, sts);
                    break;
#undef IFCTN_SOLVE_CASE
            }
            if (!okc && lane == 0) atomicOr(p.flags, FLAG_NOTSPD);  // the old column stays
            if (ti == 0) IFCTN_SSTAMP(8);
            if (okc) {
                changed |= 1u << ti;
                for (int r = lane; r < Ri; r += 32) {
                    if (MIXED) {
                        p.Gt[s.goff[k][i] + r * Ik + j] = gh[r];
                    } else {
                        const double g = gd[r];
                        vs[ti * RMAX + r] = g;
                        vt[ti * RMAX + r] = static_cast<T>(g);
                        p.Gd[s.goff[k][i] + r * Ik + j] = g;
                        p.Gt[s.goff[k][i] + r * Ik + j] = static_cast<T>(g);
                    }
                }
            }
            __syncwarp();
            if (ti == 0) IFCTN_SSTAMP(9);
        }
        if (MIXED) {
            // FP64 master copy of the updated slots: hi + lo
            for (int idx = lane; idx < nm * RMAX; idx += 32) {
                const int t = idx / RMAX, r = idx - t * RMAX;
                if (r < Rm[t] && ((changed >> t) & 1u)) {
                    const double g = static_cast<double>(vt[idx]) + static_cast<double>(vlo[idx]);
                    vs[idx] = g;
                    p.Gd[s.goff[k][m[t]] + r * Ik + j] = g;
                }
            }
        }
        IFCTN_SSTAMP(10);
        if (cta_refresh) continue;  // done below by the whole CTA
        // refresh W_{k,i}(j, :) for every i != k (in the tensor dtype)
        for (int t = 0; t < nm; ++t) {
            const int i = m[t], Ri = Rm[t], Ii = s.I[i];
            const T* gk = gik + gko[t];
            T v[RMAX];
#pragma unroll
            for (int r = 0; r < RMAX; ++r) v[r] = r < Ri ? vt[t * RMAX + r] : T(0);
            for (int b = lane; b < Ii; b += 32) {
                T w = T(0);
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < Ri) w = fma(v[r], gk[r * Ii + b], w);
                if (k < i)
                    p.W[s.woff[k][i] + static_cast<long long>(j) * Ii + b] = w;
                else
                    p.W[s.woff[i][k] + static_cast<long long>(b) * Ik + j] = w;
            }
        }
        __syncwarp();
        IFCTN_SSTAMP(11);
        stamp_col = false;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (cta_refresh) {
        // columns of this CTA: j = w * VG + VB, their new
        // G_{k,i}(:, j) in warp w's scratch (same arithmetic as per warp)
        const int ncol = min(NWc, (Ik - VB + VG - 1) / VG);
        for (int t = 0; t < nm; ++t) {
            const int i = m[t], Ri = Rm[t], Ii = s.I[i];
            const T* gk = gik + gko[t];
            for (int idx = tid; idx < ncol * Ii; idx += blockDim.x) {
                const int w = idx / Ii, b = idx - w * Ii;
                const int j = w * VG + VB;
                const T* vtw = warp_scratch_t<T>(smem, w) + SC_VT + t * RMAX;
                T acc = T(0);
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    if (r < Ri) acc = fma(vtw[r], gk[r * Ii + b], acc);
                if (k < i)
                    p.W[s.woff[k][i] + static_cast<long long>(j) * Ii + b] = acc;
                else
                    p.W[s.woff[i][k] + static_cast<long long>(b) * Ik + j] = acc;
            }
        }
        if (stamp && p.tstamp && VB == 0 && threadIdx.x == 0) p.tstamp[40 + 11] = gtimer();
    }
}
#undef IFCTN_SSTAMP

// ---------------------------------------------------------------------------
// Phase 4: eq. (updateX) fused with the reconstruction and the sums of the
// stop test, the objective and (optionally) RSE / RMSE.
// ---------------------------------------------------------------------------
struct Walk4 {
    int i0, i1, a, b;
};

__device__ __forceinline__ void walk4_from(const Shape& s, long long e, Walk4& w) {
    w.b = static_cast<int>(e % s.IB);
    long long r = e / s.IB;
    w.a = static_cast<int>(r % s.IA);
    long long f = r / s.IA;
    if (s.N == 4) {
        w.i1 = static_cast<int>(f % s.I[1]);
        w.i0 = static_cast<int>(f / s.I[1]);
    } else {
        w.i0 = static_cast<int>(f);
        w.i1 = 0;
    }
}

__device__ __forceinline__ void walk4_inc(const Shape& s, Walk4& w) {
    if (++w.b == s.IB) {
        w.b = 0;
        if (++w.a == s.IA) {
            w.a = 0;
            if (s.N == 4) {
                if (++w.i1 == s.I[1]) {
                    w.i1 = 0;
                    ++w.i0;
                }
            } else {
                ++w.i0;
            }
        }
    }
}

// a fixed element stride decomposed into single-carry digit increments
struct Step4 {
    int d0, d1, da, db;
};

__device__ __forceinline__ Step4 step4_of(const Shape& s, long long d) {
    Step4 t;
    t.db = static_cast<int>(d % s.IB);
    long long r = d / s.IB;
    t.da = static_cast<int>(r % s.IA);
    long long f = r / s.IA;
    if (s.N == 4) {
        t.d1 = static_cast<int>(f % s.I[1]);
        t.d0 = static_cast<int>(f / s.I[1]);
    } else {
        t.d0 = static_cast<int>(f);
        t.d1 = 0;
    }
    return t;
}

__device__ __forceinline__ void walk4_add(const Shape& s, Walk4& w, const Step4& t) {
    w.b += t.db;
    int ca = 0;
    if (w.b >= s.IB) {
        w.b -= s.IB;
        ca = 1;
    }
    w.a += t.da + ca;
    int cf = 0;
    if (w.a >= s.IA) {
        w.a -= s.IA;
        cf = 1;
    }
    if (s.N == 4) {
        w.i1 += t.d1 + cf;
        int c0 = 0;
        if (w.i1 >= s.I[1]) {
            w.i1 -= s.I[1];
            c0 = 1;
        }
        w.i0 += t.d0 + c0;
    } else {
        w.i0 += t.d0 + cf;
    }
}

template <typename T>
__device__ __forceinline__ T recon4(const Shape& s, const T* __restrict__ W, const Walk4& w) {
    const int N = s.N, Am = N - 2, Bm = N - 1;
    T v = W[s.woff[Am][Bm] + static_cast<long long>(w.a) * s.IB + w.b];
    if (N >= 3)
        v *= W[s.woff[0][Am] + static_cast<long long>(w.i0) * s.IA + w.a] *
             W[s.woff[0][Bm] + static_cast<long long>(w.i0) * s.IB + w.b];
    if (N == 4)
        v *= W[s.woff[1][Am] + static_cast<long long>(w.i1) * s.IA + w.a] *
             W[s.woff[1][Bm] + static_cast<long long>(w.i1) * s.IB + w.b] *
             W[s.woff[0][1] + static_cast<long long>(w.i0) * s.I[1] + w.i1];
    return v;
}

template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static constexpr int n = 4; };
template <> struct V16<double> { using type = double2; static constexpr int n = 2; };
__device__ __forceinline__ float v16get(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ double v16get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ void v16set(float4& v, int i, float x) {
    if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ void v16set(double2& v, int i, double x) {
    if (i == 0) v.x = x; else v.y = x;
}

template <typename T>
__device__ __forceinline__ void xelem(const SweepParams<T>& p, const T rho, const T inv1p, const long long e,
                                      const T xo, T& xn, const T rec, const bool obs, T (&fa)[6], const bool met) {
    xn = obs ? xo : (rec + rho * xo) * inv1p;
    const T d = xn - xo, r = xn - rec;
    fa[0] = fma(d, d, fa[0]);
    fa[1] = fma(xo, xo, fa[1]);
    fa[2] = fma(r, r, fa[2]);
    if (met) {
        const T xt = p.Xt[e];
        const T de = xt - xn;
        fa[3] = fma(de, de, fa[3]);
        fa[4] = fma(xt, xt, fa[4]);
        if (!obs) fa[5] = fma(de, de, fa[5]);
    }
}

template <typename T>
__device__ __forceinline__ void xacc(const SweepParams<T>& p, const T rho, const T inv1p, const long long e,
                                     const T rec, const bool obs, T (&fa)[6], const bool met) {
    const T xo = p.X[e];
    const T xn = obs ? xo : (rec + rho * xo) * inv1p;
    p.X[e] = xn;
    const T d = xn - xo, r = xn - rec;
    fa[0] = fma(d, d, fa[0]);
    fa[1] = fma(xo, xo, fa[1]);
    fa[2] = fma(r, r, fa[2]);
    if (met) {
        const T xt = p.Xt[e];
        const T de = xt - xn;
        fa[3] = fma(de, de, fa[3]);
        fa[4] = fma(xt, xt, fa[4]);
        if (!obs) fa[5] = fma(de, de, fa[5]);
    }
}

// eq. (updateX) over the slab geometry: a work unit is a contiguous range of
// rows (row = (slab f, a)), possibly spanning several slabs.  Per unit, the
// factors alpha(row) = prod_{p in F} W_{p,A}(i_p, a) and, per slab,
// beta(f, b) = C_f prod_{p in F} W_{p,B}(i_p, b) with C_f = W_{0,1}(i0, i1)
// (N = 4) are built in shared memory, and W_{A,B} is kept in shared memory
// when it fits, so that iFCTN(G)(i) = alpha(row) beta(f, b) W_{A,B}(a, b)
// costs three shared loads per entry.
// XB4: 16-byte vectors of X a thread holds in flight per batch (the loads of
// a batch are all issued before its stores).
// VEC_ONLY: compiled for the 16-byte path alone (the caller guarantees it
// applies), which leaves the registers of the element-wise path unused.
template <typename T, int XB4 = 4, bool VEC_ONLY = false>
__device__ void xupdate_phase(const SweepParams<T>& p, double* out6, unsigned char* smem) {
    const int VB = vbid(p), VG = p.ncta;  // this job's CTA index and grid size
    const Shape& s = p.sh;
    const int N = s.N, IA = s.IA, IB = s.IB, Am = N - 2, Bm = N - 1;
    const T rho = static_cast<T>(p.rho), inv1p = static_cast<T>(p.inv1p);
    const bool met = p.Xt != nullptr;
    const bool wsm = p.xu_wab_smem != 0;
    const int RU = p.xu_rows;
    const int SU = (RU + IA - 1) / IA + 1;  // slabs a unit can touch
    constexpr int VN = 16 / static_cast<int>(sizeof(T));
    T* wab = reinterpret_cast<T*>(smem);
    T* alpha = wab + (wsm ? IA * IB : 0);
    T* beta = alpha + (RU + VN - 1) / VN * VN;  // 16-byte aligned rows
    // 16-byte path: rows of whole 16-byte chunks (every chunk inside one row and
    // one 32-bit mask word) with W_{A,B} in shared memory
    const bool vec = wsm && IB % VN == 0;
    const T* WAB = p.W + s.woff[Am][Bm];
    if (wsm) stage_async(wab, WAB, IA * IB);
    asm volatile("cp.async.wait_all;" ::: "memory");
    const T* wab_r = wsm ? wab : WAB;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    T fa[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T run2[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    const long long rows_total = static_cast<long long>(s.nF) * IA;
    const long long nunit = (rows_total + RU - 1) / RU;
    for (long long un = VB; un < nunit; un += VG) {
        const long long r0 = un * RU;
        const int nr = static_cast<int>(min(static_cast<long long>(RU), rows_total - r0));
        const long long f0 = rows_total < (1LL << 32)
                                 ? static_cast<long long>(static_cast<unsigned>(r0) / static_cast<unsigned>(IA))
                                 : r0 / IA;
        const int a00 = static_cast<int>(r0 - f0 * IA);
        const int nsl = static_cast<int>((r0 + nr - 1) / IA - f0) + 1;
        __syncthreads();  // previous unit done with alpha / beta
        // slab and row of unit row rl from the unit's first ones (32-bit
        // divisions of small numbers; the slab count is below 2^31)
        for (int rl = threadIdx.x; rl < nr; rl += PT) {
            const unsigned ar = static_cast<unsigned>(a00 + rl);
            const unsigned df = ar / static_cast<unsigned>(IA);
            const int a = static_cast<int>(ar - df * static_cast<unsigned>(IA));
            const unsigned f = static_cast<unsigned>(f0) + df;
            int i0 = 0, i1 = 0;
            if (N == 4) {
                i0 = static_cast<int>(f / static_cast<unsigned>(s.I[1]));
                i1 = static_cast<int>(f - static_cast<unsigned>(i0) * static_cast<unsigned>(s.I[1]));
            } else {
                i0 = static_cast<int>(f);
            }
            T v = T(1);
            if (N >= 3) v *= p.W[s.woff[0][Am] + static_cast<long long>(i0) * IA + a];
            if (N == 4) v *= p.W[s.woff[1][Am] + static_cast<long long>(i1) * IA + a];
            alpha[rl] = v;
        }
        for (int idx = threadIdx.x; idx < nsl * IB; idx += PT) {
            const int sl = idx / IB, b = idx - sl * IB;
            const unsigned f = static_cast<unsigned>(f0 + sl);
            int i0 = 0, i1 = 0;
            if (N == 4) {
                i0 = static_cast<int>(f / static_cast<unsigned>(s.I[1]));
                i1 = static_cast<int>(f - static_cast<unsigned>(i0) * static_cast<unsigned>(s.I[1]));
            } else {
                i0 = static_cast<int>(f);
            }
            T v = N == 4 ? p.W[s.woff[0][1] + static_cast<long long>(i0) * s.I[1] + i1] : T(1);
            if (N >= 3) v *= p.W[s.woff[0][Bm] + static_cast<long long>(i0) * IB + b];
            if (N == 4) v *= p.W[s.woff[1][Bm] + static_cast<long long>(i1) * IB + b];
            beta[idx] = v;
        }
        __syncthreads();
        (void)SU;
        const long long e0 = r0 * IB;
        const int n = nr * IB;
        if (VEC_ONLY || vec) {
            const int nch = IB / VN;
            const int n4 = nr * nch;
            int rl4 = threadIdx.x / nch, c4 = threadIdx.x - rl4 * nch;
            int a4 = a00 + rl4, sl4 = 0;
            while (a4 >= IA) {
                a4 -= IA;
                ++sl4;
            }
            const int drl4 = PT / nch, dc4 = PT - drl4 * nch;
            for (int ob = 0; ob < n4; ob += XB4 * PT) {
                T xo[XB4][VN], rec[XB4][VN];
                uint32_t wd[XB4];
#pragma unroll
                for (int t = 0; t < XB4; ++t) {
                    const int o = ob + t * PT + threadIdx.x;
                    if (o < n4) {
                        const long long e = e0 + static_cast<long long>(o) * VN;
                        if constexpr (sizeof(T) == 4) {
                            const float4 v = *reinterpret_cast<const float4*>(p.X + e);
                            xo[t][0] = v.x;
                            xo[t][1] = v.y;
                            xo[t][2] = v.z;
                            xo[t][3] = v.w;
                        } else {
                            const double2 v = *reinterpret_cast<const double2*>(p.X + e);
                            xo[t][0] = v.x;
                            xo[t][1] = v.y;
                        }
                        wd[t] = p.mb[e >> 5];
                        const T al = alpha[rl4];
                        const T* wr = wab + a4 * IB + c4 * VN;
                        const T* br = beta + sl4 * IB + c4 * VN;
#pragma unroll
                        for (int j = 0; j < VN; ++j) rec[t][j] = wr[j] * al * br[j];
                    }
                    c4 += dc4;
                    int step = drl4;
                    if (c4 >= nch) {
                        c4 -= nch;
                        ++step;
                    }
                    rl4 += step;
                    a4 += step;
                    while (a4 >= IA) {
                        a4 -= IA;
                        ++sl4;
                    }
                }
#pragma unroll
                for (int t = 0; t < XB4; ++t) {
                    const int o = ob + t * PT + threadIdx.x;
                    if (o < n4) {
                        const long long e = e0 + static_cast<long long>(o) * VN;
                        // the vector's VN mask bits (a whole chunk lies in one 32-bit word)
                        const uint32_t ob4 = wd[t] >> (static_cast<unsigned>(e) & 31u);
                        T xn[VN];
#pragma unroll
                        for (int j = 0; j < VN; ++j) {
                            const bool obs = (ob4 >> j) & 1u;
                            xn[j] = obs ? xo[t][j] : (rec[t][j] + rho * xo[t][j]) * inv1p;
                            const T d = xn[j] - xo[t][j], r = xn[j] - rec[t][j];
                            fa[0] = fma(d, d, fa[0]);
                            fa[1] = fma(xo[t][j], xo[t][j], fa[1]);
                            fa[2] = fma(r, r, fa[2]);
                        }
                        if (met) {
#pragma unroll
                            for (int j = 0; j < VN; ++j) {
                                const bool obs = (ob4 >> j) & 1u;
                                const T xt = p.Xt[e + j];
                                const T de = xt - xn[j];
                                fa[3] = fma(de, de, fa[3]);
                                fa[4] = fma(xt, xt, fa[4]);
                                if (!obs) fa[5] = fma(de, de, fa[5]);
                            }
                        }
                        if constexpr (sizeof(T) == 4)
                            *reinterpret_cast<float4*>(p.X + e) = make_float4(xn[0], xn[1], xn[2], xn[3]);
                        else
                            *reinterpret_cast<double2*>(p.X + e) = make_double2(xn[0], xn[1]);
                    }
                }
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    run2[t] += fa[t];
                    fa[t] = T(0);
                }
            }
            continue;
        }
        // walker over (row-in-unit, b) and the slab-local row index a
        int rl = threadIdx.x / IB, b = threadIdx.x - (threadIdx.x / IB) * IB;
        int a = a00 + rl, sl = 0;
        while (a >= IA) {
            a -= IA;
            ++sl;
        }
        const int drl = PT / IB, db = PT - drl * IB;
        // batches of XB entries per thread (stride PT): every load of a batch
        // is issued before any store, so they overlap in flight
        constexpr int XB = 8;
        for (int ob = 0; ob < n; ob += XB * PT) {
            T xo[XB], rec[XB];
            uint32_t wd[XB];
#pragma unroll
            for (int t = 0; t < XB; ++t) {
                const int o = ob + t * PT + threadIdx.x;
                if (o < n) {
                    const long long e = e0 + o;
                    xo[t] = p.X[e];
                    wd[t] = p.mb[e >> 5];
                    rec[t] = wab_r[static_cast<long long>(a) * IB + b] * alpha[rl] * beta[sl * IB + b];
                }
                b += db;
                int step = drl;
                if (b >= IB) {
                    b -= IB;
                    ++step;
                }
                rl += step;
                a += step;
                while (a >= IA) {
                    a -= IA;
                    ++sl;
                }
            }
#pragma unroll
            for (int t = 0; t < XB; ++t) {
                const int o = ob + t * PT + threadIdx.x;
                if (o < n) {
                    const long long e = e0 + o;
                    const bool obs = (wd[t] >> (e & 31)) & 1u;
                    const T xn = obs ? xo[t] : (rec[t] + rho * xo[t]) * inv1p;
                    p.X[e] = xn;
                    const T d = xn - xo[t], r = xn - rec[t];
                    fa[0] = fma(d, d, fa[0]);
                    fa[1] = fma(xo[t], xo[t], fa[1]);
                    fa[2] = fma(r, r, fa[2]);
                    if (met) {
                        const T xt = p.Xt[e];
                        const T de = xt - xn;
                        fa[3] = fma(de, de, fa[3]);
                        fa[4] = fma(xt, xt, fa[4]);
                        if (!obs) fa[5] = fma(de, de, fa[5]);
                    }
                }
            }
            // two-level accumulation: batch sums fold into running sums in the
            // tensor dtype; FP64 only once per thread (GB300's FP64 pipe is narrow)
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                run2[t] += fa[t];
                fa[t] = T(0);
            }
        }
    }
    (void)acc;
    // per-CTA sums: warp reduction in the tensor dtype, FP64 across warps
    __shared__ double sh[PW][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 6; ++t) run2[t] = warp_sum(run2[t]);
    if (lane == 0)
        for (int t = 0; t < 6; ++t) sh[warp][t] = static_cast<double>(run2[t]);
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int w2 = 0; w2 < PW; ++w2) v += sh[w2][threadIdx.x];
        out6[threadIdx.x] = v;
    }
    __syncthreads();
}

// Standalone form of the X update for the per-stage (graph) path.  XB4
// vectors in flight per thread and MINB resident CTAs per SM set the bytes in
// flight per SM (XB4 x 16 B x 256 threads x MINB).
template <typename T, int XB4, int MINB, bool VEC_ONLY>
__global__ void __launch_bounds__(PT, MINB) k_xupdate_slab(const __grid_constant__ SweepParams<T> p,
                                                           double* __restrict__ xpart) {
    pdl_begin();
    if (*reinterpret_cast<volatile const int*>(p.done)) return;
    extern __shared__ __align__(128) unsigned char xsm[];
    xupdate_phase<T, XB4, VEC_ONLY>(p, xpart + 8 * blockIdx.x, xsm);
}


// The column solves of mode k for the per-stage path: the solve phase above
// on a grid of ceil(I_k / PW) CTAs, so every warp takes one column and the
// CTA refreshes the W_{k,.} entries of its columns before it exits.
template <typename T>
__global__ void __launch_bounds__(PT) k_solve_cols(const __grid_constant__ SweepParams<T> p, const int k) {
    pdl_begin();
    if (*reinterpret_cast<volatile const int*>(p.done)) return;
    extern __shared__ __align__(128) unsigned char ssm[];
    solve_phase<T>(p, k, ssm);
}


// CTA 0 stamps the end of every phase of one sweep of the launch (profiling aid)
#define IFCTN_STAMP(p, sw, slot)                                                        \
    do {                                                                              \
        if ((p).tstamp && (sw) == (p).stamp_sweep && vbid(p) == 0 && threadIdx.x == 0 &&            \
            (slot) < 64)                                                              \
            (p).tstamp[(slot)] = gtimer();                                            \
    } while (0)

// All sweeps of one job on the CTAs [p.cta0, p.cta0 + p.ncta) of the launch.
template <typename T>
__device__ __forceinline__ void sweep_body(const SweepParams<T>& p, unsigned char* smem) {
    const int VB = vbid(p), VG = p.ncta;  // this job's CTA index and grid size
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* work = smem + 128;
    __shared__ ContractArgs<T> cargs[MAXN];
    if (threadIdx.x == 0) {
        for (int i = 0; i < p.nstages; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        build_contract_args<T>(p, cargs);
    }
    __syncthreads();
    if (*reinterpret_cast<volatile const int*>(p.done)) return;
    int pipe = 0;
    unsigned nbar = 0;  // grid barriers passed in this launch
    const Shape& s = p.sh;
    __shared__ int redc;
    __shared__ int wtag;
    for (int sw = 0; sw < p.nsweeps; ++sw) {
        IFCTN_STAMP(p, sw, 0);
        for (int k = 0; k < s.N; ++k) {
            const int nU = p.pl[k].nunits, nG = p.gunits[k];
            if (threadIdx.x == 0) wtag = 0;  // W_{A,B} changes between modes
            __syncthreads();
            // Gram units first (they start the longest dependency-free work),
            // then the contraction units; a Gram unit clobbers the shared
            // W_{A,B} cache, so the tag is cleared around it
            for (int w = VB; w < nU + nG; w += VG) {
                if (w < nG) {
                    if (threadIdx.x == 0) wtag = 0;
                    gram_unit<T>(p, k, w, work);
                    if (threadIdx.x == 0 && w + VG >= nG &&
                        w + VG < nU + nG)
                        prefetch_unit<T>(p, k, w + VG - nG);
                } else {
                    const int cu = w - nG;
                    if (threadIdx.x == 0 && cu + VG < nU)
                        prefetch_unit<T>(p, k, cu + VG);
                    if (!contract_dispatch<T>(cargs[k], cu, work, bars, pipe, &wtag)) return;
                }
            }
            IFCTN_STAMP(p, sw, 1 + 6 * k);
            if (p.tstamp && sw == p.stamp_sweep && threadIdx.x == 0 && k < 4 && VB < 512)
                p.tstamp[64 + k * 512 + VB] = gtimer();
            if (!grid_barrier(p.bar_count, nbar, p.flags, VG)) return;
            IFCTN_STAMP(p, sw, 2 + 6 * k);
            reduce_phase<T>(p, k, work, sw == p.stamp_sweep && k == p.stamp_mode);
            IFCTN_STAMP(p, sw, 3 + 6 * k);
            if (!grid_barrier(p.bar_count, nbar, p.flags, VG)) return;
            IFCTN_STAMP(p, sw, 4 + 6 * k);
            solve_phase<T>(p, k, work, sw == p.stamp_sweep && k == p.stamp_mode);
            IFCTN_STAMP(p, sw, 5 + 6 * k);
            if (!grid_barrier(p.bar_count, nbar, p.flags, VG)) return;
            IFCTN_STAMP(p, sw, 6 + 6 * k);
        }
        double* xp = p.xpart + 8LL * VG * (sw & 1);
        xupdate_phase<T>(p, xp + 8 * VB, work);
        IFCTN_STAMP(p, sw, 25);
        if (!grid_barrier(p.bar_count, nbar, p.flags, VG)) return;
        IFCTN_STAMP(p, sw, 26);
        // Stop decision (only when a tolerance is set): every CTA sums the
        // per-CTA FP64 values in the same order as the log record below and
        // applies the same formula, so all CTAs take the decision the log
        // reports, without another barrier.  The FP64 log record is written
        // by the last CTA, which carries the least work in the next phases.
        bool conv = false;
        if (p.tolv > 0) {
            if (threadIdx.x < 32) {
                double a0 = 0.0, a1 = 0.0;
                for (int b = threadIdx.x; b < VG; b += 32) {
                    a0 += reinterpret_cast<volatile double*>(xp)[8 * b + 0];
                    a1 += reinterpret_cast<volatile double*>(xp)[8 * b + 1];
                }
                a0 = warp_sum(a0);
                a1 = warp_sum(a1);
                if (threadIdx.x == 0) {
                    const double rel = a1 > 0 ? sqrt(a0) / sqrt(a1) : (a0 > 0 ? INFINITY : 0.0);
                    redc = rel < p.tolv ? 1 : 0;
                }
            }
            __syncthreads();
            conv = redc != 0;
        }
        if (VB == VG - 1 && threadIdx.x < 32) {
            double a[6] = {0, 0, 0, 0, 0, 0};
            for (int b = threadIdx.x; b < VG; b += 32)
                for (int t = 0; t < 6; ++t) a[t] += reinterpret_cast<volatile double*>(xp)[8 * b + t];
            for (int t = 0; t < 6; ++t) a[t] = warp_sum(a[t]);
            if (threadIdx.x == 0) {
                const double dx2 = a[0], x2 = a[1];
                SweepStat r;
                r.rel_change = x2 > 0 ? sqrt(dx2) / sqrt(x2) : (dx2 > 0 ? INFINITY : 0.0);
                r.objective = 0.5 * a[2];
                if (p.Xt) {
                    r.rse = a[4] > 0 ? sqrt(a[3]) / sqrt(a[4]) : NAN;
                    r.rmse = p.nmiss > 0 ? sqrt(a[5] / static_cast<double>(p.nmiss)) : 0.0;
                } else {
                    r.rse = NAN;
                    r.rmse = NAN;
                }
                r.dx2 = dx2;
                r.x2 = x2;
                const int sidx = *p.counter;
                r.sweep = sidx + 1;
                r.converged = conv ? 1 : 0;
                r.flags = *p.flags;
                r.pad = 0;
                if (!isfinite(r.rel_change) || !isfinite(r.objective)) r.flags |= FLAG_NONFINITE;
                p.log[sidx % p.log_cap] = r;
                *p.counter = sidx + 1;
                if (conv) *p.done = 1;
            }
        }
        if (conv) return;
        // xpart is double-buffered by sweep parity: the buffer read here is
        // rewritten two sweeps later, after many more grid barriers.
    }
}

template <typename T>
__global__ void __launch_bounds__(PT, 2) k_sweep_persistent(const __grid_constant__ SweepParams<T> p) {
    extern __shared__ __align__(128) unsigned char smem[];
    sweep_body<T>(p, smem);
}

// Several jobs in one cooperative launch: job j runs on the CTAs
// [jobs[j].cta0, jobs[j].cta0 + jobs[j].ncta) (slices in ascending order,
// covering the grid), exactly as it would run alone on a grid of that size;
// its parameters are copied to shared memory once.
template <typename T>
__global__ void __launch_bounds__(PT, 2) k_sweep_multi(const SweepParams<T>* __restrict__ jobs, const int njobs) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) SweepParams<T> sp;
    int j = 0;
    while (j + 1 < njobs && jobs[j + 1].cta0 <= static_cast<int>(blockIdx.x)) ++j;
    {
        const int* src = reinterpret_cast<const int*>(jobs + j);
        int* dst = reinterpret_cast<int*>(&sp);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(SweepParams<T>) / sizeof(int)); i += blockDim.x)
            dst[i] = src[i];
    }
    __syncthreads();
    sweep_body<T>(sp, smem);
}

}  // namespace

template <typename T>
int persistent_smem_bytes(const SweepParams<T>& p) {
    const Shape& s = p.sh;
    long long need = 0;
    for (int k = 0; k < s.N; ++k) {
        need = std::max<long long>(need, p.pl[k].smem - 128);
        int m[3], nm = 0;
        for (int q = 0; q < s.N; ++q)
            if (q != k) m[nm++] = q;
        int Q = 1, tot = 0;
        for (int t = 0; t < nm; ++t) {
            Q *= s.R[k][m[t]];
            tot += s.R[k][m[t]] * s.I[m[t]];
        }
        need = std::max(need, solve_layout(Q, tot, static_cast<int>(sizeof(T)), p.solve_k_in_smem != 0).total);
        // reduce_phase (column tiles): coefficients + cross-warp sums
        need = std::max<long long>(need, (static_cast<long long>(RMAX) * p.pl[k].nunits + 4 +
                                          static_cast<long long>(PW) * RMAX * 32) * sizeof(T));
        if (nm == 2) {
            const int l = m[1];
            need = std::max<long long>(need, static_cast<long long>(s.R[k][l] + p.gram_iob[k]) * (s.I[l] | 1) * sizeof(T));
        } else if (nm == 3) {
            const int c = m[1], l = m[2];
            const long long Q2 = static_cast<long long>(s.R[k][c]) * s.R[k][l];
            const int chunk = std::max(1, std::min(s.I[c], p.gram_chunk));
            need = std::max<long long>(need, (static_cast<long long>(s.R[k][l]) * s.I[l] + s.R[k][c] * s.I[c] + s.I[l] +
                                              Q2 * Q2 + static_cast<long long>(chunk) * s.R[k][l] * s.R[k][l]) *
                                                 sizeof(T));
        }
    }
    // xupdate: W_{A,B} (when kept in shared memory) + alpha + beta (+ alignment of beta)
    need = std::max<long long>(need, (16 + static_cast<long long>(p.xu_wab_smem ? s.IA * s.IB : 0) + p.xu_rows +
                                      static_cast<long long>((p.xu_rows + s.IA - 1) / s.IA + 1) * s.IB) *
                                         sizeof(T));
    return static_cast<int>(need + 128 + 256);
}

template <typename T>
cudaError_t launch_persistent(const SweepParams<T>& p0, int grid, int smem, cudaStream_t st) {
    SweepParams<T> p = p0;
    p.cta0 = 0;
    p.ncta = grid;
    void* args[] = {&p};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_sweep_persistent<T>), dim3(grid), dim3(PT), args,
                                       smem, st);
}

template <typename T>
cudaError_t launch_persistent_multi(const SweepParams<T>* jobs, int njobs, int grid, int smem, cudaStream_t st) {
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(k_sweep_multi<T>), smem);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<SweepParams<T>**>(&jobs), &njobs};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_sweep_multi<T>), dim3(grid), dim3(PT), args, smem,
                                       st);
}

template <typename T>
int persistent_multi_max_grid(int smem) {
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(k_sweep_multi<T>), smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_multi<T>, PT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per * sms;
}

template <typename T, int XB4, int MINB, bool VEC_ONLY>
cudaError_t launch_xupdate_slab_v(const SweepParams<T>& p0, double* xpart, int nblocks, cudaStream_t st) {
    SweepParams<T> p = p0;
    p.cta0 = 0;
    p.ncta = nblocks;
    const int smem = static_cast<int>((static_cast<long long>(p.xu_wab_smem ? p.sh.IA * p.sh.IB : 0) + p.xu_rows +
                                       static_cast<long long>((p.xu_rows + p.sh.IA - 1) / p.sh.IA + 1) * p.sh.IB) *
                                      sizeof(T)) + 64;
    auto kern = k_xupdate_slab<T, XB4, MINB, VEC_ONLY>;
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, PT, smem, st>>>(p, xpart);
    return cudaGetLastError();
}

// p.xu_variant picks the batch and residency of the 16-byte path (1: 8
// vectors, 2 CTAs/SM; 2: 4 vectors, 3 CTAs/SM; 3: 4 vectors, 4 CTAs/SM);
// 0, and every shape the 16-byte path does not apply to, runs the generic
// kernel (4 vectors, 2 CTAs/SM).
template <typename T>
cudaError_t launch_xupdate_slab(const SweepParams<T>& p, double* xpart, int nblocks, cudaStream_t st) {
    constexpr int VN = 16 / static_cast<int>(sizeof(T));
    const bool vec = p.xu_wab_smem != 0 && p.sh.IB % VN == 0;
    switch (vec ? p.xu_variant : 0) {
        case 1: return launch_xupdate_slab_v<T, 8, 2, true>(p, xpart, nblocks, st);
        case 2: return launch_xupdate_slab_v<T, 4, 3, true>(p, xpart, nblocks, st);
        case 3: return launch_xupdate_slab_v<T, 4, 4, true>(p, xpart, nblocks, st);
        default: return launch_xupdate_slab_v<T, 4, 2, false>(p, xpart, nblocks, st);
    }
}

template <typename T>
cudaError_t launch_solve_cols(const SweepParams<T>& p0, int k, cudaStream_t st) {
    const Shape& s = p0.sh;
    int Q = 1, tot = 0;
    for (int q = 0; q < s.N; ++q)
        if (q != k) {
            Q *= s.R[k][q];
            tot += s.R[k][q] * s.I[q];
        }
    SweepParams<T> p = p0;
    const int sz = static_cast<int>(sizeof(T));
    p.solve_k_in_smem = solve_layout(Q, tot, sz, true).total + 64 <= 220 * 1024 ? 1 : 0;
    const int smem = static_cast<int>(solve_layout(Q, tot, sz, p.solve_k_in_smem != 0).total + 64);
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(k_solve_cols<T>), smem);
    if (e != cudaSuccess) return e;
    // Warps of a CTA that take columns: as few as spread the columns over
    // every SM, so that columns do not queue on one SM's shared-memory pipe
    // while others idle (the assembly of H reads K_k from shared memory); all
    // PT threads still stage K_k and the tables and refresh W.  With nw warps
    // and ncta = ceil(I_k / nw) CTAs, column j = w ncta + CTA is taken by warp
    // w < nw, and every CTA refreshes its own columns.
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nw = std::max(1, std::min(PW, (s.I[k] + sms - 1) / std::max(1, sms)));
    p.solve_nw = nw;
    p.cta0 = 0;
    p.ncta = (s.I[k] + nw - 1) / nw;
    k_solve_cols<T><<<p.ncta, PT, smem, st>>>(p, k);
    return cudaGetLastError();
}

template <typename T>
int persistent_max_grid(int smem) {
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(k_sweep_persistent<T>), smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_persistent<T>, PT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per * sms;
}

}  // namespace ifctn
