// ifctn_contract_dev.cuh -- per-unit device code of the streaming mode-k
// contraction M_k = X_(k) Z_k (see ifctn_contract.cu for the design).  Used by
// the standalone contraction kernels and by the persistent sweep kernel.
#pragma once
#include "ifctn_launch.h"

namespace ifctn {
namespace cdev {

__device__ __forceinline__ void decode_f(const Shape& s, long long f, int& i0, int& i1) {
    if (s.N == 4) {
        i0 = static_cast<int>(f / s.I[1]);
        i1 = static_cast<int>(f - static_cast<long long>(i0) * s.I[1]);
    } else {
        i0 = static_cast<int>(f);
        i1 = 0;
    }
}

// Level-2 fold shared by CASE_A and COL: z(r2, r) += coef(r2) * u(r), where
// r2 runs over mode l2 (mode 1 for N = 4, mode 0 for N = 3) and coef carries
// G_{l2,k} and, for N = 4, the pair matrix W_{0,1}.
template <typename T, int R>
__device__ __forceinline__ void fold_outer(const Shape& s, const T* Gt, const T* W, int k, int l2,
                                           int Rl2, int i0, int i1, const T (&u)[R],
                                           T (&z)[RMAX][R]) {
    if (l2 < 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) z[0][r] += u[r];
    } else if (s.N == 4) {
        const T w01 = W[s.woff[0][1] + static_cast<long long>(i0) * s.I[1] + i1];
#pragma unroll
        for (int r2 = 0; r2 < RMAX; ++r2)
            if (r2 < Rl2) {
                const T c = gfac(Gt, s, 1, k, r2, i1) * w01;
#pragma unroll
                for (int r = 0; r < R; ++r) z[r2][r] = fma(c, u[r], z[r2][r]);
            }
    } else if (s.N == 3) {
#pragma unroll
        for (int r2 = 0; r2 < RMAX; ++r2)
            if (r2 < Rl2) {
                const T c = gfac(Gt, s, 0, k, r2, i0);
#pragma unroll
                for (int r = 0; r < R; ++r) z[r2][r] = fma(c, u[r], z[r2][r]);
            }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) z[0][r] += u[r];
    }
}

// Byte range [lo, hi) covering elements [e0, e0+n) rounded out to 16 bytes.
template <typename T>
__device__ __forceinline__ void tile_range(const T* X, long long e0, long long n, uintptr_t& lo,
                                           uintptr_t& hi) {
    lo = reinterpret_cast<uintptr_t>(X + e0) & ~uintptr_t(15);
    hi = (reinterpret_cast<uintptr_t>(X + e0 + n) + 15) & ~uintptr_t(15);
}

// Bounded drain of stages issued but never consumed (error path only).
static __device__ void drain(uint64_t* bars, int S, int from, int to, int* flags) {
    for (int it = from; it < to; ++it) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&bars[it % S], static_cast<unsigned>((it / S) & 1)))
            if (clock64() - t0 > 200000000LL) break;
    }
    (void)flags;
}

// ---------------------------------------------------------------------------
// ROW kernel: k in F (CASE_F) or k = N-2 (CASE_A)
// ---------------------------------------------------------------------------
template <typename T, int RB>
__device__ __noinline__ bool contract_row_unit(const ContractArgs<T>& A, const int uidx, unsigned char* smem,
                                  uint64_t* bars, int& pipe, int* wtag) {
    const Shape& s = A.sh;
    const ContractPlan& pl = A.pl;
    const int N = s.N, k = A.k, IA = s.IA, IB = s.IB;
    const int Bm = N - 1, Am = N - 2;
    const int TA = pl.TA, G = pl.G, S = pl.nstages;
    constexpr int RBP = RB | 1;
    const bool isF = pl.kcase == CASE_F;
    const UnitDesc u = A.units[uidx];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int g = tid / TA, al = tid - g * TA;
    const bool in_grid = g < G;

    const bool split = pl.split != 0;
    const int GS = split ? 1 : G;  // slabs per stage
    T* stage = reinterpret_cast<T*>(smem);
    T* psi = stage + static_cast<size_t>(S) * GS * pl.sub_elems;
    T* wab = psi + static_cast<size_t>(GS) * IB * RBP;
    T* red = wab + (isF ? static_cast<size_t>(TA) * IB : 0);

    const int na_tot = u.a1 - u.a0;
    const int npass = (na_tot + TA - 1) / TA;
    const int nbatch = (u.ns + GS - 1) / GS;
    const int nst = npass * nbatch;
    // split mode: group g covers columns [bg0, bg1) of every row
    const int bg0 = split ? static_cast<int>(static_cast<long long>(IB) * g / G) : 0;
    const int bg1 = split ? static_cast<int>(static_cast<long long>(IB) * (g + 1) / G) : IB;

    T* outs = red + static_cast<size_t>(nwarp) * pl.Q;
    if (isF)
        for (int q = tid; q < pl.Q; q += nthr) outs[q] = T(0);
    __syncthreads();

    auto issue = [&](int it) {
        const int p = it / nbatch, bt = it - p * nbatch;
        const int a0 = u.a0 + p * TA;
        const int na = min(TA, u.a1 - a0);
        const int buf = (pipe + it) % S;
        const int gmax = min(GS, u.ns - bt * GS);
        unsigned total = 0;
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * GS + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            total += static_cast<unsigned>(hi - lo);
        }
        mbar_arrive_expect_tx(&bars[buf], total);
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * GS + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            bulk_g2s(stage + (static_cast<size_t>(buf) * GS + gg) * pl.sub_elems,
                     reinterpret_cast<const void*>(lo), static_cast<unsigned>(hi - lo), &bars[buf]);
        }
    };
    if (tid == 0)
        for (int it = 0; it < min(S, nst); ++it) issue(it);

    T z[RMAX][RB];
#pragma unroll
    for (int r2 = 0; r2 < RMAX; ++r2)
#pragma unroll
        for (int r = 0; r < RB; ++r) z[r2][r] = T(0);

    for (int it = 0; it < nst; ++it) {
        const int p = it / nbatch, bt = it - p * nbatch;
        const int a0 = u.a0 + p * TA;
        const int na = min(TA, u.a1 - a0);
        const int buf = (pipe + it) % S;
        const unsigned par = static_cast<unsigned>(((pipe + it) / S) & 1);
        // pair matrix W_{A,B} rows of this pass; a caller may keep them across
        // units through *wtag (the first row + 1 of the rows held, 0 = none)
        const bool wload = isF && bt == 0 && !(wtag && *wtag == a0 + 1 && na == TA);
        if (wload) stage_async(wab, A.W + s.woff[Am][Bm] + static_cast<long long>(a0) * IB, na * IB);
        const int gsl = split ? 0 : g;  // this thread's slab within the stage
        const int sidx = bt * GS + gsl;
        const bool has = in_grid && sidx < u.ns;
        long long f = 0;
        int i0 = 0, i1 = 0;
        if (has) {
            f = u.f0 + static_cast<long long>(sidx) * u.fstride;
            decode_f(s, f, i0, i1);
        }
        // psi(b, r) = prod_{p in F, p != k} W_{p,B}(i_p, b) * G_{B,k}(r, b)
        if (split ? (bt < u.ns) : has) {
            if (split && !has) {  // padding threads help fill the shared table
                f = u.f0 + static_cast<long long>(bt) * u.fstride;
                decode_f(s, f, i0, i1);
            }
            T* pg = psi + static_cast<size_t>(gsl) * IB * RBP;
            const int t0 = split ? tid : al, tst = split ? nthr : TA;
#pragma unroll 4
            for (int idx = t0; idx < IB * RB; idx += tst) {
                const int b = idx / RB, r = idx - b * RB;
                T om = T(1);
                if (N >= 3 && k != 0) om *= A.W[s.woff[0][Bm] + static_cast<long long>(i0) * IB + b];
                if (N == 4 && k != 1) om *= A.W[s.woff[1][Bm] + static_cast<long long>(i1) * IB + b];
                pg[b * RBP + r] = om * gfac(A.Gt, s, Bm, k, r, b);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        if (wload && wtag && tid == 0) *wtag = (na == TA) ? a0 + 1 : 0;
        const bool ok = mbar_wait_bounded(&bars[buf], par, A.flags);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bars, S, pipe + it + 1, pipe + min(nst, it + S), A.flags);
            return false;
        }
        if (has && al < na) {
            const long long e0 = (f * IA + a0) * IB;
            const int shift = static_cast<int>((reinterpret_cast<uintptr_t>(A.X + e0) & 15) / sizeof(T));
            const T* xr = stage + (static_cast<size_t>(buf) * GS + gsl) * pl.sub_elems + shift +
                          static_cast<size_t>(al) * IB;
            const T* pg = psi + static_cast<size_t>(gsl) * IB * RBP;
            T uu[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) uu[r] = T(0);
            const int blen = bg1 - bg0;
            const int bst = (pl.skew && blen > 0) ? bg0 + (al % blen) : bg0;
            if (isF) {
                const T* wr = wab + static_cast<size_t>(al) * IB;
                for (int b = bst; b < bg1; ++b) {
                    const T x = xr[b] * wr[b];
                    const T* pr = pg + b * RBP;
#pragma unroll
                    for (int r = 0; r < RB; ++r) uu[r] = fma(x, pr[r], uu[r]);
                }
                for (int b = bg0; b < bst; ++b) {
                    const T x = xr[b] * wr[b];
                    const T* pr = pg + b * RBP;
#pragma unroll
                    for (int r = 0; r < RB; ++r) uu[r] = fma(x, pr[r], uu[r]);
                }
                if (N == 4) {
                    // coef(r2) = G_{o,k}(r2, i_o) W_{o,A}(i_o, a), o = the other F mode
                    const int o = 1 - k;
                    const int io = o == 0 ? i0 : i1;
                    const T alpha = A.W[s.woff[o][Am] + static_cast<long long>(io) * IA + a0 + al];
#pragma unroll
                    for (int r2 = 0; r2 < RMAX; ++r2)
                        if (r2 < pl.Rl2) {
                            const T c = gfac(A.Gt, s, o, k, r2, io) * alpha;
#pragma unroll
                            for (int r = 0; r < RB; ++r) z[r2][r] = fma(c, uu[r], z[r2][r]);
                        }
                } else {
#pragma unroll
                    for (int r = 0; r < RB; ++r) z[0][r] += uu[r];
                }
            } else {
                for (int b = bst; b < bg1; ++b) {
                    const T x = xr[b];
                    const T* pr = pg + b * RBP;
#pragma unroll
                    for (int r = 0; r < RB; ++r) uu[r] = fma(x, pr[r], uu[r]);
                }
                for (int b = bg0; b < bst; ++b) {
                    const T x = xr[b];
                    const T* pr = pg + b * RBP;
#pragma unroll
                    for (int r = 0; r < RB; ++r) uu[r] = fma(x, pr[r], uu[r]);
                }
                fold_outer<T, RB>(s, A.Gt, A.W, k, pl.l2, pl.Rl2, i0, i1, uu, z);
            }
        }
        __syncthreads();
        if (tid == 0 && it + S < nst) {
            fence_proxy_async();
            issue(it + S);
        }
        if (bt == nbatch - 1) {  // end of a pass over rows [a0, a0+na)
            const bool act = in_grid && al < na;
            if (isF) {
                // out(r2, rA, rB) += sum_a G_{A,k}(rA, a) z_a(r2, rB)
                T gA[RMAX];
#pragma unroll
                for (int rA = 0; rA < RMAX; ++rA)
                    gA[rA] = (act && rA < pl.RA) ? gfac(A.Gt, s, Am, k, rA, a0 + al) : T(0);
                T* wsum = red;
#pragma unroll
                for (int r2 = 0; r2 < RMAX; ++r2)
                    if (r2 < pl.Rl2)
#pragma unroll
                        for (int rA = 0; rA < RMAX; ++rA)
                            if (rA < pl.RA)
#pragma unroll
                                for (int r = 0; r < RB; ++r) {
                                    const T v = warp_sum(gA[rA] * z[r2][r]);
                                    if (lane == 0) wsum[warp * pl.Q + (r2 * pl.RA + rA) * RB + r] = v;
                                }
                __syncthreads();
                for (int q = tid; q < pl.Q; q += nthr) {
                    T acc = T(0);
                    for (int w = 0; w < nwarp; ++w) acc += wsum[w * pl.Q + q];
                    outs[q] += acc;
                }
                __syncthreads();
            } else {
                const int Qp = pl.Qp;
#pragma unroll
                for (int r2 = 0; r2 < RMAX; ++r2)
                    if (r2 < pl.Rl2)
#pragma unroll
                        for (int r = 0; r < RB; ++r) red[tid * Qp + r2 * RB + r] = act ? z[r2][r] : T(0);
                __syncthreads();
                for (int idx = tid; idx < na * Qp; idx += nthr) {
                    const int row = idx / Qp, q = idx - row * Qp;
                    T acc = T(0);
                    for (int gg = 0; gg < G; ++gg) acc += red[(gg * TA + row) * Qp + q];
                    A.part[(static_cast<size_t>(uidx) * IA + a0 + row) * Qp + q] = acc;
                }
                __syncthreads();
            }
#pragma unroll
            for (int r2 = 0; r2 < RMAX; ++r2)
#pragma unroll
                for (int r = 0; r < RB; ++r) z[r2][r] = T(0);
        }
    }
    if (isF)
        for (int q = tid; q < pl.Q; q += nthr)
            A.part[(static_cast<size_t>(u.key) * pl.nslot + u.slot) * pl.Q + q] = outs[q];
    __syncthreads();
    pipe += nst;
    return true;
}

// ---------------------------------------------------------------------------
// COL kernel: k = N-1 (the contiguous mode is the output index)
// ---------------------------------------------------------------------------
template <typename T, int RA>
__device__ __noinline__ bool contract_col_unit(const ContractArgs<T>& A, const int uidx, unsigned char* smem,
                                  uint64_t* bars, int& pipe) {
    const Shape& s = A.sh;
    const ContractPlan& pl = A.pl;
    const int N = s.N, k = A.k, IA = s.IA, IB = s.IB;
    const int Am = N - 2;
    const int TB = pl.TA, G = pl.G, S = pl.nstages, TAc = pl.TAc;
    constexpr int RAP = RA | 1;
    const UnitDesc u = A.units[uidx];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int g = tid / TB, bl = tid - g * TB;
    const bool in_grid = g < G;
    const int b = u.b0 + bl;
    const bool colok = in_grid && b < u.b1;

    const bool split = pl.split != 0;
    const int GS = split ? 1 : G;  // slabs per stage
    T* stage = reinterpret_cast<T*>(smem);
    T* phi = stage + static_cast<size_t>(S) * GS * pl.sub_elems;
    T* red = phi + static_cast<size_t>(GS) * TAc * RAP;

    const int na_tot = u.a1 - u.a0;
    const int nch = (na_tot + TAc - 1) / TAc;
    const int nbatch = (u.ns + GS - 1) / GS;
    const int nst = nbatch * nch;

    __syncthreads();

    auto issue = [&](int it) {
        const int bt = it / nch, c = it - bt * nch;
        const int a0 = u.a0 + c * TAc;
        const int na = min(TAc, u.a1 - a0);
        const int buf = (pipe + it) % S;
        const int gmax = min(GS, u.ns - bt * GS);
        unsigned total = 0;
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * GS + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            total += static_cast<unsigned>(hi - lo);
        }
        mbar_arrive_expect_tx(&bars[buf], total);
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * GS + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            bulk_g2s(stage + (static_cast<size_t>(buf) * GS + gg) * pl.sub_elems,
                     reinterpret_cast<const void*>(lo), static_cast<unsigned>(hi - lo), &bars[buf]);
        }
    };
    if (tid == 0)
        for (int it = 0; it < min(S, nst); ++it) issue(it);

    T z[RMAX][RA], uu[RA];
#pragma unroll
    for (int r2 = 0; r2 < RMAX; ++r2)
#pragma unroll
        for (int r = 0; r < RA; ++r) z[r2][r] = T(0);
#pragma unroll
    for (int r = 0; r < RA; ++r) uu[r] = T(0);

    for (int it = 0; it < nst; ++it) {
        const int bt = it / nch, c = it - bt * nch;
        const int a0 = u.a0 + c * TAc;
        const int na = min(TAc, u.a1 - a0);
        const int buf = (pipe + it) % S;
        const unsigned par = static_cast<unsigned>(((pipe + it) / S) & 1);
        const int gsl = split ? 0 : g;
        const int sidx = bt * GS + gsl;
        const bool has = in_grid && sidx < u.ns;
        long long f = 0;
        int i0 = 0, i1 = 0;
        if (has) {
            f = u.f0 + static_cast<long long>(sidx) * u.fstride;
            decode_f(s, f, i0, i1);
        }
        // phi(a, r) = prod_{p in F} W_{p,A}(i_p, a) * G_{A,k}(r, a)
        if (split ? (bt < u.ns) : has) {
            if (split && !has) {
                f = u.f0 + static_cast<long long>(bt) * u.fstride;
                decode_f(s, f, i0, i1);
            }
            T* pg = phi + static_cast<size_t>(gsl) * TAc * RAP;
            const int t0 = split ? tid : bl, tst = split ? nthr : TB;
#pragma unroll 4
            for (int idx = t0; idx < na * RA; idx += tst) {
                const int ar = idx / RA, r = idx - ar * RA;
                const int a = a0 + ar;
                T om = T(1);
                if (N >= 3) om *= A.W[s.woff[0][Am] + static_cast<long long>(i0) * IA + a];
                if (N == 4) om *= A.W[s.woff[1][Am] + static_cast<long long>(i1) * IA + a];
                pg[ar * RAP + r] = om * gfac(A.Gt, s, Am, k, r, a);
            }
        }
        __syncthreads();
        const bool ok = mbar_wait_bounded(&bars[buf], par, A.flags);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bars, S, pipe + it + 1, pipe + min(nst, it + S), A.flags);
            return false;
        }
        if (has && colok) {
            const long long e0 = (f * IA + a0) * IB;
            const int shift = static_cast<int>((reinterpret_cast<uintptr_t>(A.X + e0) & 15) / sizeof(T));
            const T* xr = stage + (static_cast<size_t>(buf) * GS + gsl) * pl.sub_elems + shift + b;
            const T* pg = phi + static_cast<size_t>(gsl) * TAc * RAP;
            const int ar0 = split ? g : 0, ars = split ? G : 1;
            for (int ar = ar0; ar < na; ar += ars) {
                const T x = xr[static_cast<size_t>(ar) * IB];
                const T* pr = pg + ar * RAP;
#pragma unroll
                for (int r = 0; r < RA; ++r) uu[r] = fma(x, pr[r], uu[r]);
            }
        }
        if (c == nch - 1) {
            if (has && colok) fold_outer<T, RA>(s, A.Gt, A.W, k, pl.l2, pl.Rl2, i0, i1, uu, z);
#pragma unroll
            for (int r = 0; r < RA; ++r) uu[r] = T(0);
        }
        __syncthreads();
        if (tid == 0 && it + S < nst) {
            fence_proxy_async();
            issue(it + S);
        }
    }
    const int Qp = pl.Qp;
#pragma unroll
    for (int r2 = 0; r2 < RMAX; ++r2)
        if (r2 < pl.Rl2)
#pragma unroll
            for (int r = 0; r < RA; ++r) red[tid * Qp + r2 * RA + r] = colok ? z[r2][r] : T(0);
    __syncthreads();
    const int nb = u.b1 - u.b0;
    for (int idx = tid; idx < nb * Qp; idx += nthr) {
        const int row = idx / Qp, q = idx - row * Qp;
        T acc = T(0);
        for (int gg = 0; gg < G; ++gg) acc += red[(gg * TB + row) * Qp + q];
        A.part[(static_cast<size_t>(uidx) * IB + u.b0 + row) * Qp + q] = acc;
    }
    __syncthreads();
    pipe += nst;
    return true;
}

}  // namespace cdev
}  // namespace ifctn
