// ifctn_contract_dev.cuh -- per-unit device code of the streaming mode-k
// contraction M_k = X_(k) Z_k (design notes in ifctn_contract_kernels.cuh).
// Used by the standalone contraction kernels and by the persistent sweep
// kernel.
//
// Every pipeline stage is one mbarrier phase fed by 1-D TMA bulk copies: the
// X tile of each slab of the stage plus the few short W vectors that slab
// needs (the rows of W_{p,B} or W_{p,A} that build the coefficient table, the
// row of W_{o,A} of the level-2 weight, or the scalar W_{0,1}(i0,i1)).  The
// static G_{m,k} tables are staged once per unit.  So no global load sits on
// the per-stage path: a stage waits only for its own bulk copies.
#pragma once
#include "ifctn_launch.h"

namespace ifctn {
namespace cdev {

// slab index f (< 2^31) -> F-mode indices, in 32-bit arithmetic
__device__ __forceinline__ void decode_f(const Shape& s, long long f, int& i0, int& i1) {
    const int fi = static_cast<int>(f);
    if (s.N == 4) {
        const unsigned q = static_cast<unsigned>(fi) / static_cast<unsigned>(s.I[1]);
        i0 = static_cast<int>(q);
        i1 = fi - i0 * s.I[1];
    } else {
        i0 = fi;
        i1 = 0;
    }
}

// Byte range [lo, hi) covering elements [p, p+n) rounded out to 16 bytes.
template <typename T>
__device__ __forceinline__ void range16(const T* p, long long n, uintptr_t& lo, uintptr_t& hi) {
    lo = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15);
    hi = (reinterpret_cast<uintptr_t>(p + n) + 15) & ~uintptr_t(15);
}

template <typename T>
__device__ __forceinline__ int shift16(const T* p) {
    return static_cast<int>((reinterpret_cast<uintptr_t>(p) & 15) / sizeof(T));
}

// Short W vectors a slab's stage carries (element offsets into W, lengths).
struct Aux {
    int n;
    long long off[3];
    int len[3];
};

// ROW kind (k != N-1): the psi rows W_{p,B}(i_p, :) for F modes p != k, then
// (CASE_F, N = 4) the row W_{o,A}(i_o, a0:a0+na), or (CASE_A, N = 4) W_{0,1}(i0,i1).
__device__ __forceinline__ Aux row_aux(const Shape& s, int k, bool isF, long long f, int a0, int na) {
    int i0, i1;
    decode_f(s, f, i0, i1);
    const int N = s.N, Am = N - 2, Bm = N - 1;
    Aux a;
    a.n = 0;
    if (N >= 3 && k != 0) {
        a.off[a.n] = s.woff[0][Bm] + static_cast<long long>(i0) * s.IB;
        a.len[a.n++] = s.IB;
    }
    if (N == 4 && k != 1) {
        a.off[a.n] = s.woff[1][Bm] + static_cast<long long>(i1) * s.IB;
        a.len[a.n++] = s.IB;
    }
    if (isF && N == 4) {
        const int o = 1 - k, io = o == 0 ? i0 : i1;
        a.off[a.n] = s.woff[o][Am] + static_cast<long long>(io) * s.IA + a0;
        a.len[a.n++] = na;
    }
    if (!isF && N == 4) {
        a.off[a.n] = s.woff[0][1] + static_cast<long long>(i0) * s.I[1] + i1;
        a.len[a.n++] = 1;
    }
    return a;
}

// COL kind (k = N-1): the phi rows W_{p,A}(i_p, a0:a0+na) for every F mode p,
// then (N = 4) W_{0,1}(i0,i1).
__device__ __forceinline__ Aux col_aux(const Shape& s, long long f, int a0, int na) {
    int i0, i1;
    decode_f(s, f, i0, i1);
    const int N = s.N, Am = N - 2;
    Aux a;
    a.n = 0;
    if (N >= 3) {
        a.off[a.n] = s.woff[0][Am] + static_cast<long long>(i0) * s.IA + a0;
        a.len[a.n++] = na;
    }
    if (N == 4) {
        a.off[a.n] = s.woff[1][Am] + static_cast<long long>(i1) * s.IA + a0;
        a.len[a.n++] = na;
        a.off[a.n] = s.woff[0][1] + static_cast<long long>(i0) * s.I[1] + i1;
        a.len[a.n++] = 1;
    }
    return a;
}

// Issues one slab's bulk copies (X tile + aux vectors) into the stage buffer at
// element offset `base` and returns their byte count.  A stage's copies are
// issued before its single arrive.expect_tx: the barrier's transaction count may
// run negative in between, and the phase cannot complete before that arrive
// (arrival count 1), so the count is armed once with the stage total.
template <typename T>
__device__ __forceinline__ unsigned slab_copies(const T* X, const T* W, long long e0, long long n, const Aux& ax,
                                                T* buf, unsigned base, int xcap, int SL, uint64_t* bar) {
    uintptr_t lo, hi;
    range16(X + e0, n, lo, hi);
    unsigned total = static_cast<unsigned>(hi - lo);
    bulk_g2s(buf + base, reinterpret_cast<const void*>(lo), static_cast<unsigned>(hi - lo), bar);
    for (int j = 0; j < ax.n; ++j) {
        range16(W + ax.off[j], ax.len[j], lo, hi);
        total += static_cast<unsigned>(hi - lo);
        bulk_g2s(buf + base + xcap + j * SL, reinterpret_cast<const void*>(lo), static_cast<unsigned>(hi - lo), bar);
    }
    return total;
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
// ROW kind: k in F (CASE_F) or k = N-2 (CASE_A).  A thread owns row a of the
// slab tile, contracts the contiguous mode B in registers (u, RB values) and
// folds the row into z over the level-2 mode.
// ---------------------------------------------------------------------------
template <typename T, int RB>
__device__ __forceinline__ bool row_unit_body(const ContractArgs<T>& A, const int uidx, unsigned char* smem,
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
    const int SL = pl.aux_slot, xcap = pl.sub_elems - 3 * SL;
    const int npsi = (N >= 3 && k != 0 ? 1 : 0) + (N == 4 && k != 1 ? 1 : 0);

    T* stage = reinterpret_cast<T*>(smem);
    T* psi = stage + static_cast<size_t>(S) * GS * pl.sub_elems;
    T* wab = psi + static_cast<size_t>(GS) * IB * RBP;
    T* red = wab + (isF ? static_cast<size_t>(TA) * IB : 0);
    T* outs = red + static_cast<size_t>(nwarp) * pl.Q;
    T* gtab = red + (isF ? static_cast<size_t>(nwarp + 1) * pl.Q : static_cast<size_t>(nthr) * pl.Qp);
    const int l2 = pl.l2;
    const int nB = pl.R1 * IB;
    const int nL = l2 >= 0 ? pl.Rl2 * s.I[l2] : 0;
    const int nA = isF ? pl.RA * IA : 0;
    const bool gsm = pl.gtab_smem != 0;
    const T* gB = gsm ? gtab : A.Gt + s.goff[Bm][k];
    const T* gL = l2 >= 0 ? (gsm ? gtab + nB : A.Gt + s.goff[l2][k]) : nullptr;
    const T* gA = isF ? (gsm ? gtab + nB + nL : A.Gt + s.goff[Am][k]) : nullptr;

    const int na_tot = u.a1 - u.a0;
    const int npass = (na_tot + TA - 1) / TA;
    const int nbatch = (u.ns + GS - 1) / GS;
    const int nst = npass * nbatch;
    // split mode: group g covers columns [bg0, bg1) of every row
    const int bg0 = split ? static_cast<int>(static_cast<long long>(IB) * g / G) : 0;
    const int bg1 = split ? static_cast<int>(static_cast<long long>(IB) * (g + 1) / G) : IB;

    auto issue = [&](int it) {
        const int p = it / nbatch, bt = it - p * nbatch;
        const int a0 = u.a0 + p * TA;
        const int na = min(TA, u.a1 - a0);
        const int buf = (pipe + it) % S;
        const int gmax = min(GS, u.ns - bt * GS);
        T* sbuf = stage + static_cast<size_t>(buf) * GS * pl.sub_elems;
        unsigned total = 0;
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * GS + gg) * u.fstride;
            const Aux ax = row_aux(s, k, isF, f, a0, na);
            total += slab_copies(A.X, A.W, (f * IA + a0) * IB, static_cast<long long>(na) * IB, ax, sbuf,
                                 static_cast<unsigned>(gg * pl.sub_elems), xcap, SL, &bars[buf]);
        }
        mbar_arrive_expect_tx(&bars[buf], total);
    };
    if (tid == 0)
        for (int it = 0; it < min(S, nst); ++it) issue(it);
    if (isF)
        for (int q = tid; q < pl.Q; q += nthr) outs[q] = T(0);
    if (gsm) {
        stage_async(gtab, A.Gt + s.goff[Bm][k], nB);
        if (nL) stage_async(gtab + nB, A.Gt + s.goff[l2][k], nL);
        if (nA) stage_async(gtab + nB + nL, A.Gt + s.goff[Am][k], nA);
    }
    stage_wait();

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
        const bool ok = mbar_wait_bounded(&bars[buf], par, A.flags);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bars, S, pipe + it + 1, pipe + min(nst, it + S), A.flags);
            return false;
        }
        // psi(b, r) = prod_{p in F, p != k} W_{p,B}(i_p, b) * G_{B,k}(r, b), from
        // the rows the stage brought along
        {
            const bool build = split ? (bt < u.ns) : has;
            if (build) {
                const long long fb = u.f0 + static_cast<long long>(bt * GS + gsl) * u.fstride;
                const Aux ax = row_aux(s, k, isF, fb, a0, na);
                const T* sub = stage + (static_cast<size_t>(buf) * GS + gsl) * pl.sub_elems;
                const T* w0 = npsi > 0 ? sub + xcap + shift16(A.W + ax.off[0]) : nullptr;
                const T* w1 = npsi > 1 ? sub + xcap + SL + shift16(A.W + ax.off[1]) : nullptr;
                T* pg = psi + static_cast<size_t>(gsl) * IB * RBP;
                const int t0 = split ? tid : al, tst = split ? nthr : TA;
                for (int idx = t0; idx < IB * RB; idx += tst) {
                    const int b = idx / RB, r = idx - b * RB;
                    T om = T(1);
                    if (npsi > 0) om *= w0[b];
                    if (npsi > 1) om *= w1[b];
                    pg[b * RBP + r] = om * gB[r * IB + b];
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        if (wload && wtag && tid == 0) *wtag = (na == TA) ? a0 + 1 : 0;
        if (has && al < na) {
            const long long f = u.f0 + static_cast<long long>(sidx) * u.fstride;
            int i0, i1;
            decode_f(s, f, i0, i1);
            const T* sub = stage + (static_cast<size_t>(buf) * GS + gsl) * pl.sub_elems;
            const T* xr = sub + shift16(A.X + (f * IA + a0) * IB) + static_cast<size_t>(al) * IB;
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
            }
            // level-2 fold: z(r2, r) += coef(r2) u(r)
            if (l2 < 0) {
#pragma unroll
                for (int r = 0; r < RB; ++r) z[0][r] += uu[r];
            } else {
                const Aux ax = row_aux(s, k, isF, f, a0, na);
                T scale = T(1);
                int il2;
                if (isF) {  // N = 4: coef = G_{o,k}(r2, i_o) W_{o,A}(i_o, a)
                    il2 = l2 == 0 ? i0 : i1;
                    scale = (sub + xcap + npsi * SL + shift16(A.W + ax.off[npsi]))[al];
                } else if (N == 4) {  // coef = G_{1,k}(r2, i1) W_{0,1}(i0, i1)
                    il2 = i1;
                    scale = (sub + xcap + npsi * SL + shift16(A.W + ax.off[npsi]))[0];
                } else {  // N = 3: coef = G_{0,k}(r2, i0)
                    il2 = i0;
                }
                const T* gl = gL + il2;
                const int Il2 = s.I[l2];
#pragma unroll
                for (int r2 = 0; r2 < RMAX; ++r2)
                    if (r2 < pl.Rl2) {
                        const T c = gl[r2 * Il2] * scale;
#pragma unroll
                        for (int r = 0; r < RB; ++r) z[r2][r] = fma(c, uu[r], z[r2][r]);
                    }
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
                T gAv[RMAX];
#pragma unroll
                for (int rA = 0; rA < RMAX; ++rA) gAv[rA] = (act && rA < pl.RA) ? gA[rA * IA + a0 + al] : T(0);
                T* wsum = red;
#pragma unroll
                for (int r2 = 0; r2 < RMAX; ++r2)
                    if (r2 < pl.Rl2)
#pragma unroll
                        for (int rA = 0; rA < RMAX; ++rA)
                            if (rA < pl.RA)
#pragma unroll
                                for (int r = 0; r < RB; ++r) {
                                    const T v = warp_sum(gAv[rA] * z[r2][r]);
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
// COL kind: k = N-1 (the contiguous mode is the output index).  A thread owns
// column b, contracts mode A in registers and folds each slab into z.
// ---------------------------------------------------------------------------
template <typename T, int RA>
__device__ __forceinline__ bool col_unit_body(const ContractArgs<T>& A, const int uidx, unsigned char* smem,
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
    const int SL = pl.aux_slot, xcap = pl.sub_elems - 3 * SL;
    const int nphi = (N >= 3 ? 1 : 0) + (N == 4 ? 1 : 0);

    T* stage = reinterpret_cast<T*>(smem);
    T* phi = stage + static_cast<size_t>(S) * GS * pl.sub_elems;
    T* red = phi + static_cast<size_t>(GS) * TAc * RAP;
    T* gtab = red + static_cast<size_t>(nthr) * pl.Qp;
    const int l2 = pl.l2;
    const int nAg = pl.R1 * IA;
    const int nL = l2 >= 0 ? pl.Rl2 * s.I[l2] : 0;
    const bool gsm = pl.gtab_smem != 0;
    const T* gAt = gsm ? gtab : A.Gt + s.goff[Am][k];
    const T* gL = l2 >= 0 ? (gsm ? gtab + nAg : A.Gt + s.goff[l2][k]) : nullptr;

    const int na_tot = u.a1 - u.a0;
    const int nch = (na_tot + TAc - 1) / TAc;
    const int nbatch = (u.ns + GS - 1) / GS;
    const int nst = nbatch * nch;

    auto issue = [&](int it) {
        const int bt = it / nch, c = it - bt * nch;
        const int a0 = u.a0 + c * TAc;
        const int na = min(TAc, u.a1 - a0);
        const int buf = (pipe + it) % S;
        const int gmax = min(GS, u.ns - bt * GS);
        T* sbuf = stage + static_cast<size_t>(buf) * GS * pl.sub_elems;
        unsigned total = 0;
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * GS + gg) * u.fstride;
            const Aux ax = col_aux(s, f, a0, na);
            total += slab_copies(A.X, A.W, (f * IA + a0) * IB, static_cast<long long>(na) * IB, ax, sbuf,
                                 static_cast<unsigned>(gg * pl.sub_elems), xcap, SL, &bars[buf]);
        }
        mbar_arrive_expect_tx(&bars[buf], total);
    };
    if (tid == 0)
        for (int it = 0; it < min(S, nst); ++it) issue(it);
    if (gsm) {
        stage_async(gtab, A.Gt + s.goff[Am][k], nAg);
        if (nL) stage_async(gtab + nAg, A.Gt + s.goff[l2][k], nL);
    }
    stage_wait();

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
        const bool ok = mbar_wait_bounded(&bars[buf], par, A.flags);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bars, S, pipe + it + 1, pipe + min(nst, it + S), A.flags);
            return false;
        }
        // phi(a, r) = prod_{p in F} W_{p,A}(i_p, a) * G_{A,k}(r, a), from the
        // rows the stage brought along
        {
            const bool build = split ? (bt < u.ns) : has;
            if (build) {
                const long long fb = u.f0 + static_cast<long long>(bt * GS + gsl) * u.fstride;
                const Aux ax = col_aux(s, fb, a0, na);
                const T* sub = stage + (static_cast<size_t>(buf) * GS + gsl) * pl.sub_elems;
                const T* w0 = nphi > 0 ? sub + xcap + shift16(A.W + ax.off[0]) : nullptr;
                const T* w1 = nphi > 1 ? sub + xcap + SL + shift16(A.W + ax.off[1]) : nullptr;
                T* pg = phi + static_cast<size_t>(gsl) * TAc * RAP;
                const int t0 = split ? tid : bl, tst = split ? nthr : TB;
                for (int idx = t0; idx < na * RA; idx += tst) {
                    const int ar = idx / RA, r = idx - ar * RA;
                    T om = T(1);
                    if (nphi > 0) om *= w0[ar];
                    if (nphi > 1) om *= w1[ar];
                    pg[ar * RAP + r] = om * gAt[r * IA + a0 + ar];
                }
            }
        }
        __syncthreads();
        if (has && colok) {
            const long long f = u.f0 + static_cast<long long>(sidx) * u.fstride;
            const T* sub = stage + (static_cast<size_t>(buf) * GS + gsl) * pl.sub_elems;
            const T* xr = sub + shift16(A.X + (f * IA + a0) * IB) + b;
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
            if (has && colok) {
                if (l2 < 0) {
#pragma unroll
                    for (int r = 0; r < RA; ++r) z[0][r] += uu[r];
                } else {
                    const long long f = u.f0 + static_cast<long long>(sidx) * u.fstride;
                    int i0, i1;
                    decode_f(s, f, i0, i1);
                    T scale = T(1);
                    int il2 = i0;
                    if (N == 4) {  // coef = G_{1,k}(r2, i1) W_{0,1}(i0, i1)
                        const Aux ax = col_aux(s, f, a0, na);
                        const T* sub = stage + (static_cast<size_t>(buf) * GS + gsl) * pl.sub_elems;
                        scale = (sub + xcap + nphi * SL + shift16(A.W + ax.off[nphi]))[0];
                        il2 = i1;
                    }
                    const T* gl = gL + il2;
                    const int Il2 = s.I[l2];
#pragma unroll
                    for (int r2 = 0; r2 < RMAX; ++r2)
                        if (r2 < pl.Rl2) {
                            const T cf = gl[r2 * Il2] * scale;
#pragma unroll
                            for (int r = 0; r < RA; ++r) z[r2][r] = fma(cf, uu[r], z[r2][r]);
                        }
                }
            }
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

// Out-of-line entry points used by the persistent kernel (one copy of each
// body per rank instead of one per call site).  The standalone kernels inline
// the bodies instead, which leaves them the whole register file.
template <typename T, int RB>
__device__ __noinline__ bool contract_row_unit(const ContractArgs<T>& A, const int uidx, unsigned char* smem,
                                               uint64_t* bars, int& pipe, int* wtag) {
    return row_unit_body<T, RB>(A, uidx, smem, bars, pipe, wtag);
}

template <typename T, int RA>
__device__ __noinline__ bool contract_col_unit(const ContractArgs<T>& A, const int uidx, unsigned char* smem,
                                               uint64_t* bars, int& pipe) {
    return col_unit_body<T, RA>(A, uidx, smem, bars, pipe);
}

}  // namespace cdev
}  // namespace ifctn
