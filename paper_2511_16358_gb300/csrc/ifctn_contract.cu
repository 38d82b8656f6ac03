// ifctn_contract.cu -- the streaming mode-k contraction M_k = X_(k) Z_k.
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
#include "ifctn_launch.h"

namespace ifctn {
namespace {

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
__device__ __forceinline__ void fold_outer(const Shape& s, const T* Gt, const T* W, int k,
                                           int Rl2, int i0, int i1, const T (&u)[R],
                                           T (&z)[RMAX][R]) {
    if (s.N == 4) {
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
__device__ void drain(uint64_t* bars, int S, int from, int to, int* flags) {
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
__global__ void __launch_bounds__(256) k_contract_row(const ContractArgs<T> A) {
    if (*A.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const Shape& s = A.sh;
    const ContractPlan& pl = A.pl;
    const int N = s.N, k = A.k, IA = s.IA, IB = s.IB;
    const int Bm = N - 1, Am = N - 2;
    const int TA = pl.TA, G = pl.G, S = pl.nstages;
    constexpr int RBP = RB | 1;
    const bool isF = pl.kcase == CASE_F;
    const UnitDesc u = A.units[blockIdx.x];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int g = tid / TA, al = tid - g * TA;
    const bool in_grid = g < G;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    T* stage = reinterpret_cast<T*>(smem + 128);
    T* psi = stage + static_cast<size_t>(S) * G * pl.sub_elems;
    T* wab = psi + static_cast<size_t>(G) * IB * RBP;
    T* red = wab + (isF ? static_cast<size_t>(TA) * IB : 0);

    const int na_tot = u.a1 - u.a0;
    const int npass = (na_tot + TA - 1) / TA;
    const int nbatch = (u.ns + G - 1) / G;
    const int nst = npass * nbatch;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    T* outs = red + static_cast<size_t>(nwarp) * pl.Q;
    if (isF)
        for (int q = tid; q < pl.Q; q += nthr) outs[q] = T(0);
    __syncthreads();

    auto issue = [&](int it) {
        const int p = it / nbatch, bt = it - p * nbatch;
        const int a0 = u.a0 + p * TA;
        const int na = min(TA, u.a1 - a0);
        const int buf = it % S;
        const int gmax = min(G, u.ns - bt * G);
        unsigned total = 0;
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * G + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            total += static_cast<unsigned>(hi - lo);
        }
        mbar_arrive_expect_tx(&bars[buf], total);
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * G + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            bulk_g2s(stage + (static_cast<size_t>(buf) * G + gg) * pl.sub_elems,
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
        const int buf = it % S;
        const unsigned par = static_cast<unsigned>((it / S) & 1);
        if (isF && bt == 0) {  // pair matrix W_{A,B} rows of this pass
            const T* src = A.W + s.woff[Am][Bm] + static_cast<long long>(a0) * IB;
            for (int idx = tid; idx < na * IB; idx += nthr) wab[idx] = src[idx];
        }
        const int sidx = bt * G + g;
        const bool has = in_grid && sidx < u.ns;
        long long f = 0;
        int i0 = 0, i1 = 0;
        if (has) {
            f = u.f0 + static_cast<long long>(sidx) * u.fstride;
            decode_f(s, f, i0, i1);
            // psi(b, r) = prod_{p in F, p != k} W_{p,B}(i_p, b) * G_{B,k}(r, b)
            T* pg = psi + static_cast<size_t>(g) * IB * RBP;
            for (int idx = al; idx < IB * RB; idx += TA) {
                const int b = idx / RB, r = idx - b * RB;
                T om = T(1);
                if (N >= 3 && k != 0) om *= A.W[s.woff[0][Bm] + static_cast<long long>(i0) * IB + b];
                if (N == 4 && k != 1) om *= A.W[s.woff[1][Bm] + static_cast<long long>(i1) * IB + b];
                pg[b * RBP + r] = om * gfac(A.Gt, s, Bm, k, r, b);
            }
        }
        __syncthreads();
        const bool ok = mbar_wait_bounded(&bars[buf], par, A.flags);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bars, S, it + 1, min(nst, it + S), A.flags);
            return;
        }
        if (has && al < na) {
            const long long e0 = (f * IA + a0) * IB;
            const int shift = static_cast<int>((reinterpret_cast<uintptr_t>(A.X + e0) & 15) / sizeof(T));
            const T* xr = stage + (static_cast<size_t>(buf) * G + g) * pl.sub_elems + shift +
                          static_cast<size_t>(al) * IB;
            const T* pg = psi + static_cast<size_t>(g) * IB * RBP;
            T uu[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) uu[r] = T(0);
            const int bst = pl.skew ? (al % IB) : 0;
            if (isF) {
                const T* wr = wab + static_cast<size_t>(al) * IB;
                for (int b = bst; b < IB; ++b) {
                    const T x = xr[b] * wr[b];
                    const T* pr = pg + b * RBP;
#pragma unroll
                    for (int r = 0; r < RB; ++r) uu[r] = fma(x, pr[r], uu[r]);
                }
                for (int b = 0; b < bst; ++b) {
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
                for (int b = bst; b < IB; ++b) {
                    const T x = xr[b];
                    const T* pr = pg + b * RBP;
#pragma unroll
                    for (int r = 0; r < RB; ++r) uu[r] = fma(x, pr[r], uu[r]);
                }
                for (int b = 0; b < bst; ++b) {
                    const T x = xr[b];
                    const T* pr = pg + b * RBP;
#pragma unroll
                    for (int r = 0; r < RB; ++r) uu[r] = fma(x, pr[r], uu[r]);
                }
                fold_outer<T, RB>(s, A.Gt, A.W, k, pl.Rl2, i0, i1, uu, z);
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
                    A.part[(static_cast<size_t>(blockIdx.x) * IA + a0 + row) * Qp + q] = acc;
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
}

// ---------------------------------------------------------------------------
// COL kernel: k = N-1 (the contiguous mode is the output index)
// ---------------------------------------------------------------------------
template <typename T, int RA>
__global__ void __launch_bounds__(256) k_contract_col(const ContractArgs<T> A) {
    if (*A.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const Shape& s = A.sh;
    const ContractPlan& pl = A.pl;
    const int N = s.N, k = A.k, IA = s.IA, IB = s.IB;
    const int Am = N - 2;
    const int TB = pl.TA, G = pl.G, S = pl.nstages, TAc = pl.TAc;
    constexpr int RAP = RA | 1;
    const UnitDesc u = A.units[blockIdx.x];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int g = tid / TB, bl = tid - g * TB;
    const bool in_grid = g < G;
    const int b = u.b0 + bl;
    const bool colok = in_grid && b < u.b1;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    T* stage = reinterpret_cast<T*>(smem + 128);
    T* phi = stage + static_cast<size_t>(S) * G * pl.sub_elems;
    T* red = phi + static_cast<size_t>(G) * TAc * RAP;

    const int na_tot = u.a1 - u.a0;
    const int nch = (na_tot + TAc - 1) / TAc;
    const int nbatch = (u.ns + G - 1) / G;
    const int nst = nbatch * nch;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int it) {
        const int bt = it / nch, c = it - bt * nch;
        const int a0 = u.a0 + c * TAc;
        const int na = min(TAc, u.a1 - a0);
        const int buf = it % S;
        const int gmax = min(G, u.ns - bt * G);
        unsigned total = 0;
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * G + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            total += static_cast<unsigned>(hi - lo);
        }
        mbar_arrive_expect_tx(&bars[buf], total);
        for (int gg = 0; gg < gmax; ++gg) {
            const long long f = u.f0 + static_cast<long long>(bt * G + gg) * u.fstride;
            uintptr_t lo, hi;
            tile_range(A.X, (f * IA + a0) * IB, static_cast<long long>(na) * IB, lo, hi);
            bulk_g2s(stage + (static_cast<size_t>(buf) * G + gg) * pl.sub_elems,
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
        const int buf = it % S;
        const unsigned par = static_cast<unsigned>((it / S) & 1);
        const int sidx = bt * G + g;
        const bool has = in_grid && sidx < u.ns;
        long long f = 0;
        int i0 = 0, i1 = 0;
        if (has) {
            f = u.f0 + static_cast<long long>(sidx) * u.fstride;
            decode_f(s, f, i0, i1);
            // phi(a, r) = prod_{p in F} W_{p,A}(i_p, a) * G_{A,k}(r, a)
            T* pg = phi + static_cast<size_t>(g) * TAc * RAP;
            for (int idx = bl; idx < na * RA; idx += TB) {
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
            if (tid == 0) drain(bars, S, it + 1, min(nst, it + S), A.flags);
            return;
        }
        if (has && colok) {
            const long long e0 = (f * IA + a0) * IB;
            const int shift = static_cast<int>((reinterpret_cast<uintptr_t>(A.X + e0) & 15) / sizeof(T));
            const T* xr = stage + (static_cast<size_t>(buf) * G + g) * pl.sub_elems + shift + b;
            const T* pg = phi + static_cast<size_t>(g) * TAc * RAP;
            for (int ar = 0; ar < na; ++ar) {
                const T x = xr[static_cast<size_t>(ar) * IB];
                const T* pr = pg + ar * RAP;
#pragma unroll
                for (int r = 0; r < RA; ++r) uu[r] = fma(x, pr[r], uu[r]);
            }
        }
        if (c == nch - 1) {
            if (has && colok) fold_outer<T, RA>(s, A.Gt, A.W, k, pl.Rl2, i0, i1, uu, z);
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
        A.part[(static_cast<size_t>(blockIdx.x) * IB + u.b0 + row) * Qp + q] = acc;
    }
}

// ---------------------------------------------------------------------------
// finisher: M_k(row, q) from the partials (fixed order)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_contract_finish(const Shape s, const int k,
                                                         const ContractPlan pl,
                                                         const UnitDesc* __restrict__ units,
                                                         const T* __restrict__ part,
                                                         const T* __restrict__ Gt,
                                                         double* __restrict__ Mk,
                                                         const int* __restrict__ done) {
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
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.pl.nunits, a.pl.nthreads, a.pl.smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int R>
cudaError_t launch_col_r(const ContractArgs<T>& a, cudaStream_t st) {
    auto kern = k_contract_col<T, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.pl.nunits, a.pl.nthreads, a.pl.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_contract(const ContractArgs<T>& a, cudaStream_t st) {
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

template <typename T>
cudaError_t launch_contract_finish(const Shape& sh, int k, const ContractPlan& pl,
                                   const UnitDesc* units, const T* part, const T* Gt, double* Mk,
                                   const int* done, cudaStream_t st) {
    const long long total = static_cast<long long>(sh.I[k]) * pl.Q;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 1216) blocks = 1216;
    if (blocks < 1) blocks = 1;
    k_contract_finish<T><<<blocks, 256, 0, st>>>(sh, k, pl, units, part, Gt, Mk, done);
    return cudaGetLastError();
}

template cudaError_t launch_contract<float>(const ContractArgs<float>&, cudaStream_t);
template cudaError_t launch_contract<double>(const ContractArgs<double>&, cudaStream_t);
template cudaError_t launch_contract_finish<float>(const Shape&, int, const ContractPlan&,
                                                   const UnitDesc*, const float*, const float*,
                                                   double*, const int*, cudaStream_t);
template cudaError_t launch_contract_finish<double>(const Shape&, int, const ContractPlan&,
                                                    const UnitDesc*, const double*, const double*,
                                                    double*, const int*, cudaStream_t);

}  // namespace ifctn
