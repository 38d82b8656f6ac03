// ifctn_wide.cu -- mode systems of order-3 tensors whose edge ranks exceed
// the register-resident kernels' limit (R_{k,l} up to WIDE_RMAX, Q_k up to
// WIDE_QMAX), as in the multispectral rank grid of Sec. 5.2 (R_{1,2} up to
// 36), and column solves with one CTA per column: for those tensors (and,
// when selected for testing, on the sweep graph of order-3 and order-4
// tensors; the warp-per-column solve is faster there on GB300).
//
// For mode k with other modes a < b, the regrouped systems of eq. (updateG)
// (Prop. 1: M_k = X_(k) Z_k, K_k = Z_k^T Z_k; Q_k index q = r_a R_{k,b} + r_b)
// are formed as two chains of contractions.  Each link is a batched matrix
// product whose operands are generated while they are loaded, from X, the pair
// matrices W and the factors G_{m,k}:
//
//   contraction (c1, c2 the other modes; c1 contracted first)
//     V(j, i_c2, r1)        = sum_{i_c1} X(i) W_{c1,c2}(i_c1, i_c2) G_{c1,k}(r1, i_c1)
//     M_k(j, (r_c1, r_c2))  = sum_{i_c2} G_{c2,k}(r_c2, i_c2) V(j, i_c2, r_c1)
//   Gram (d1 summed first)
//     T(i_d2, r1, r1')      = sum_{i_d1} W_{d1,d2}(i_d1, i_d2)^2 G_{d1,k}(r1, i_d1) G_{d1,k}(r1', i_d1)
//     K_k((r1,r2),(r1',r2')) = sum_{i_d2} G_{d2,k}(r2, i_d2) G_{d2,k}(r2', i_d2) T(i_d2, r1, r1')
//
// X is read once per mode, by the first link, whose contracted mode is the
// contiguous one (mode 2) unless k is: the loads stay coalesced.  The column
// solves assemble H = E_j^T K_k E_j + rho I and b = E_j^T M_k(j,:)^T + rho g in
// the tensor dtype with all threads of a CTA, factorise H by Cholesky in FP64
// in shared memory, and refresh W_{k,i}(j, :) with the new columns
// (Algorithm 1's order: i != k ascending, each stage using the column the
// previous one produced).
#include <cuda_runtime.h>

#include <algorithm>

#include "ifctn_launch.h"
#include "ifctn_persistent.h"

namespace ifctn {
namespace {

constexpr int WT = 256;  // threads of every kernel in this file
constexpr int BK = 16;   // reduction depth of one shared-memory tile

// C[b](m, n) = sum_i A[b](m, i) B[b](i, n) for every batch b; Op generates
// the operands (a, bm), stores the result (store) and names the sizes.  Each
// CTA computes BM x BN outputs, TM x TN per thread, in the tensor dtype.
template <typename T, int BM, int BN, int TM, int TN, class Op>
__global__ void __launch_bounds__(WT) k_wide_gemm(const __grid_constant__ Op op, const int* __restrict__ done) {
    static_assert((BM / TM) * (BN / TN) == WT, "thread layout");
    pdl_begin();
    if (*done) return;
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int mt_n = (op.M + BM - 1) / BM, nt_n = (op.N + BN - 1) / BN;
    for (int b = blockIdx.z; b < op.batch; b += gridDim.z)
        for (int mt = blockIdx.y; mt < mt_n; mt += gridDim.y)
            for (int nt = blockIdx.x; nt < nt_n; nt += gridDim.x) {
                const int m0 = mt * BM, n0 = nt * BN;
                T acc[TM][TN];
#pragma unroll
                for (int u = 0; u < TM; ++u)
#pragma unroll
                    for (int v = 0; v < TN; ++v) acc[u][v] = T(0);
                for (int k0 = 0; k0 < op.K; k0 += BK) {
                    for (int e = tid; e < BK * BM; e += WT) {
                        int kk, mm;
                        if (op.a_m_fast) {
                            mm = e % BM;
                            kk = e / BM;
                        } else {
                            kk = e % BK;
                            mm = e / BK;
                        }
                        const int m = m0 + mm, i = k0 + kk;
                        As[kk][mm] = (m < op.M && i < op.K) ? op.a(b, m, i) : T(0);
                    }
                    for (int e = tid; e < BK * BN; e += WT) {
                        int kk, nn;
                        if (op.b_n_fast) {
                            nn = e % BN;
                            kk = e / BN;
                        } else {
                            kk = e % BK;
                            nn = e / BK;
                        }
                        const int n = n0 + nn, i = k0 + kk;
                        Bs[kk][nn] = (n < op.N && i < op.K) ? op.bm(b, i, n) : T(0);
                    }
                    __syncthreads();
#pragma unroll
                    for (int kk = 0; kk < BK; ++kk) {
                        T av[TM], bv[TN];
#pragma unroll
                        for (int u = 0; u < TM; ++u) av[u] = As[kk][ty * TM + u];
#pragma unroll
                        for (int v = 0; v < TN; ++v) bv[v] = Bs[kk][tx * TN + v];
#pragma unroll
                        for (int u = 0; u < TM; ++u)
#pragma unroll
                            for (int v = 0; v < TN; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int u = 0; u < TM; ++u)
#pragma unroll
                    for (int v = 0; v < TN; ++v) {
                        const int m = m0 + ty * TM + u, n = n0 + tx * TN + v;
                        if (m < op.M && n < op.N) op.store(b, m, n, acc[u][v]);
                    }
            }
}

// First link of the contraction: batch b = i_c2, m = j, n = r1, i = i_c1.
template <typename T>
struct OpContract1 {
    const T* X;
    const T* W;  // W_{c1,c2} or W_{c2,c1}, at its offset
    const T* G;  // G_{c1,k}
    T* V;
    long long sk, sc1, sc2;  // strides of modes k, c1, c2 in X
    int wsi, wsb;            // W_{c1,c2}(i, b) at W[i * wsi + b * wsb]
    int Ic1, Ic2, R1;
    int M, N, K, batch;
    bool a_m_fast, b_n_fast;
    __device__ T a(int b, int m, int i) const { return X[m * sk + i * sc1 + b * sc2]; }
    __device__ T bm(int b, int i, int n) const {
        return W[static_cast<long long>(i) * wsi + static_cast<long long>(b) * wsb] * G[static_cast<long long>(n) * Ic1 + i];
    }
    __device__ void store(int b, int m, int n, T v) const {
        V[(static_cast<long long>(m) * Ic2 + b) * R1 + n] = v;
    }
};

// Second link: batch b = j, m = r_c2, n = r_c1, i = i_c2; M_k in FP64.
template <typename T>
struct OpContract2 {
    const T* G;  // G_{c2,k}
    const T* V;
    double* Mk;
    int Ic2, R1, Q, qsm, qsn;  // q = m * qsm + n * qsn
    int M, N, K, batch;
    bool a_m_fast, b_n_fast;
    __device__ T a(int, int m, int i) const { return G[static_cast<long long>(m) * Ic2 + i]; }
    __device__ T bm(int b, int i, int n) const { return V[(static_cast<long long>(b) * Ic2 + i) * R1 + n]; }
    __device__ void store(int b, int m, int n, T v) const {
        Mk[static_cast<long long>(b) * Q + m * qsm + n * qsn] = static_cast<double>(v);
    }
};

// First link of the Gram: m = i_d2, n = (r1, r1'), i = i_d1.
template <typename T>
struct OpGram1 {
    const T* W;  // W_{d1,d2}(i, m) at W[i * wsi + m * wsb]
    const T* G;  // G_{d1,k}
    T* Tg;
    int wsi, wsb, Id1, R1;
    int M, N, K, batch;
    bool a_m_fast, b_n_fast;
    __device__ T a(int, int m, int i) const {
        const T w = W[static_cast<long long>(i) * wsi + static_cast<long long>(m) * wsb];
        return w * w;
    }
    __device__ T bm(int, int i, int n) const {
        const int r = n / R1, rp = n - r * R1;
        return G[static_cast<long long>(r) * Id1 + i] * G[static_cast<long long>(rp) * Id1 + i];
    }
    __device__ void store(int, int m, int n, T v) const { Tg[static_cast<long long>(m) * N + n] = v; }
};

// Second link: m = (r2, r2'), n = (r1, r1'), i = i_d2; K_k(q, q') with
// q = r1 * s1 + r2 * s2.
template <typename T>
struct OpGram2 {
    const T* G;  // G_{d2,k}
    const T* Tg;
    T* Kk;
    int Id2, R1, R2, Q, s1, s2;
    int M, N, K, batch;
    bool a_m_fast, b_n_fast;
    __device__ T a(int, int m, int i) const {
        const int r = m / R2, rp = m - r * R2;
        return G[static_cast<long long>(r) * Id2 + i] * G[static_cast<long long>(rp) * Id2 + i];
    }
    __device__ T bm(int, int i, int n) const { return Tg[static_cast<long long>(i) * N + n]; }
    __device__ void store(int, int m, int n, T v) const {
        const int r2 = m / R2, r2p = m - r2 * R2;
        const int r1 = n / R1, r1p = n - r1 * R1;
        Kk[static_cast<long long>(r1 * s1 + r2 * s2) * Q + r1p * s1 + r2p * s2] = v;
    }
};

// Order-4 Gram, other modes o < c < l of k (o the batch): pairs p = (x, y),
// x <= y, of the l-slot rank run over NP = R_l (R_l + 1) / 2 in row order.
__device__ __forceinline__ void pair_of(int p, int R, int& x, int& y) {
    x = 0;
    while (p >= R - x) {
        p -= R - x;
        ++x;
    }
    y = x + p;
}

// First link: t1[o][ic][p] = W_{o,c}(o, ic)^2 sum_{il} W_{c,l}(ic, il)^2 W_{o,l}(o, il)^2 G_{l,k}(x_p, il) G_{l,k}(y_p, il);
// batch b = i_o, m = i_c, n = p, i = i_l.
template <typename T>
struct OpGram4a {
    const T* Wcl;  // W_{c,l}(ic, il) at Wcl[ic * cs_c + il * cs_l]
    const T* Wol;  // W_{o,l}(io, il) at Wol[io * os_o + il * os_l]
    const T* Woc;  // W_{o,c}(io, ic) at Woc[io * ws_o + ic * ws_c]
    const T* Gl;   // G_{l,k}
    T* t1;
    int cs_c, cs_l, os_o, os_l, ws_o, ws_c, Il, RL;
    int M, N, K, batch;
    bool a_m_fast, b_n_fast;
    __device__ T a(int, int m, int i) const {
        const T w = Wcl[static_cast<long long>(m) * cs_c + static_cast<long long>(i) * cs_l];
        return w * w;
    }
    __device__ T bm(int b, int i, int n) const {
        int x, y;
        pair_of(n, RL, x, y);
        const T w = Wol[static_cast<long long>(b) * os_o + static_cast<long long>(i) * os_l];
        return w * w * Gl[static_cast<long long>(x) * Il + i] * Gl[static_cast<long long>(y) * Il + i];
    }
    __device__ void store(int b, int m, int n, T v) const {
        const T w = Woc[static_cast<long long>(b) * ws_o + static_cast<long long>(m) * ws_c];
        t1[(static_cast<long long>(b) * M + m) * N + n] = v * w * w;
    }
};

// Second link: T2[o][(xc, xl), (yc, yl)] = sum_{ic} G_{c,k}(xc, ic) G_{c,k}(yc, ic) t1[o][ic][p(xl, yl)],
// both (xl, yl) and (yl, xl); batch b = i_o, m = (xc, yc), n = p, i = i_c.
template <typename T>
struct OpGram4b {
    const T* Gc;  // G_{c,k}
    const T* t1;
    T* T2;
    int Ic, Rc, RL, NP;
    int M, N, K, batch;
    bool a_m_fast, b_n_fast;
    __device__ T a(int, int m, int i) const {
        const int xc = m / Rc, yc = m - xc * Rc;
        return Gc[static_cast<long long>(xc) * Ic + i] * Gc[static_cast<long long>(yc) * Ic + i];
    }
    __device__ T bm(int b, int i, int n) const { return t1[(static_cast<long long>(b) * Ic + i) * NP + n]; }
    __device__ void store(int b, int m, int n, T v) const {
        const int xc = m / Rc, yc = m - xc * Rc;
        int xl, yl;
        pair_of(n, RL, xl, yl);
        const int Q2 = Rc * RL;
        T* out = T2 + static_cast<long long>(b) * Q2 * Q2;
        out[(xc * RL + xl) * Q2 + yc * RL + yl] = v;
        if (xl != yl) out[(xc * RL + yl) * Q2 + yc * RL + xl] = v;
    }
};

template <typename T, class Op>
cudaError_t launch_gemm(const Op& op, const int* done, cudaStream_t st) {
    if (op.M <= 0 || op.N <= 0 || op.batch <= 0) return cudaSuccess;
    if (op.N <= 16) {
        constexpr int BM = 128, BN = 16;
        dim3 grid(1, std::min((op.M + BM - 1) / BM, 65535), std::min(op.batch, 65535));
        k_wide_gemm<T, BM, BN, 8, 1, Op><<<grid, WT, 0, st>>>(op, done);
    } else {
        constexpr int BM = 64, BN = 64;
        dim3 grid(std::min((op.N + BN - 1) / BN, 65535), std::min((op.M + BM - 1) / BM, 65535),
                  std::min(op.batch, 65535));
        k_wide_gemm<T, BM, BN, 4, 4, Op><<<grid, WT, 0, st>>>(op, done);
    }
    return cudaGetLastError();
}

// W_{p,q}(i_p, i_q) as W[i_p * sp + i_q * sq] from the pointer returned.
template <typename T>
const T* pair_view(const Shape& s, const T* W, int p, int q, int& sp, int& sq) {
    if (p < q) {
        sp = s.I[q];
        sq = 1;
        return W + s.woff[p][q];
    }
    sp = 1;
    sq = s.I[p];
    return W + s.woff[q][p];
}

void other_modes(int k, int& a, int& b) {
    a = k == 0 ? 1 : 0;
    b = k == 2 ? 1 : 2;
}

// ---------------------------------------------------------------------------
// column solves, one CTA per column
// ---------------------------------------------------------------------------
constexpr int HPART = 4096;  // partial sums of H held in shared memory

// The other modes of k (ascending), their ranks, the Q_k index stride of each
// slot (slot 0 most significant) and Q_k.
struct Slots {
    int nm, Q, Rx;
    int m[3], R[3], st[3];
};

__host__ __device__ inline Slots slots_of(const Shape& s, int k) {
    Slots q;
    q.nm = 0;
    for (int t = 0; t < s.N; ++t)
        if (t != k) q.m[q.nm++] = t;
    q.Q = 1;
    q.Rx = 1;
    for (int t = 0; t < q.nm; ++t) {
        q.R[t] = s.R[k][q.m[t]];
        q.Q *= q.R[t];
        q.Rx = q.R[t] > q.Rx ? q.R[t] : q.Rx;
    }
    for (int t = 0; t < 3; ++t) q.st[t] = 1;
    for (int t = q.nm - 2; t >= 0; --t) q.st[t] = q.st[t + 1] * q.R[t + 1];
    return q;
}

// Shared-memory layout of the solve (bytes): H, b, the current columns of the
// slots, M_k(j, :), the partial sums of H, the weights and K offsets of the
// other slots' digit combinations, optionally K_k at an odd row stride.
struct CtaSolveLayout {
    long long H, bv, gc, Mr, part, om, cbo, K, bad, total;
};

__host__ __device__ inline CtaSolveLayout cta_solve_layout(const Slots& q, int sz, bool kstage) {
    CtaSolveLayout L;
    L.H = 0;
    L.bv = L.H + 8LL * q.Rx * q.Rx;
    L.gc = L.bv + 8LL * q.Rx;
    L.Mr = L.gc + 8LL * 3 * WIDE_RMAX;
    L.part = L.Mr + 8LL * q.Q;
    L.om = L.part + static_cast<long long>(sz) * HPART;
    L.cbo = (L.om + static_cast<long long>(sz) * q.Q + 15) & ~15LL;
    L.K = (L.cbo + 4LL * q.Q + 15) & ~15LL;
    L.bad = L.K + (kstage ? static_cast<long long>(sz) * q.Q * k_stride(q.Q) : 0);
    L.total = L.bad + 16;
    return L;
}

// Row c and column c' <= c of entry e of a lower triangle stored by rows.
__device__ __forceinline__ void tri_index(int e, int& c, int& cp) {
    // FP32 estimate (e < 2^12 here), corrected exactly below: no FP64 on a
    // pipe that GB300 keeps narrow
    c = static_cast<int>((sqrtf(8.0f * static_cast<float>(e) + 1.0f) - 1.0f) * 0.5f);
    while (c * (c + 1) / 2 > e) --c;
    while ((c + 1) * (c + 2) / 2 <= e) ++c;
    cp = e - c * (c + 1) / 2;
}

// One CTA per column j of mode k (grid-stride over j), stages i != k in order
// (each using the columns the previous ones produced).  For stage ti the other
// slots' digit combinations o get the weight w(o) = prod_t G_{k,m_t}(d_t, j)
// and the K_k offset cb(o); then
//   H(c, c') = sum_{o,o'} w(o) w(o') K_k(cb(o) + c sp, cb(o') + c' sp) + rho [c = c']
//   b(c)     = sum_o w(o) M_k(j, cb(o) + c sp) + rho g_old(c)
// (sp the stride of slot ti), summed in the tensor dtype by (entry, group of
// o) work items with fixed owners and added in a fixed order, factorised by
// Cholesky in FP64 in shared memory, solved by one warp.
template <typename T>
__global__ void __launch_bounds__(WT) k_cta_solve(const __grid_constant__ Shape s, const int k, const double rho,
                                                  const double* __restrict__ Mk, const T* __restrict__ Kk,
                                                  double* __restrict__ Gd, T* __restrict__ Gt, T* __restrict__ W,
                                                  int* __restrict__ flags, const int* __restrict__ done,
                                                  const int kstage) {
    pdl_begin();
    if (*done) return;
    extern __shared__ __align__(16) unsigned char wsm[];
    const Slots q = slots_of(s, k);
    const int Q = q.Q, Ik = s.I[k], nm = q.nm;
    const CtaSolveLayout L = cta_solve_layout(q, static_cast<int>(sizeof(T)), kstage != 0);
    double* H = reinterpret_cast<double*>(wsm + L.H);
    double* bv = reinterpret_cast<double*>(wsm + L.bv);
    double* gc = reinterpret_cast<double*>(wsm + L.gc);  // [3][WIDE_RMAX]
    double* Mr = reinterpret_cast<double*>(wsm + L.Mr);
    T* part = reinterpret_cast<T*>(wsm + L.part);
    T* om = reinterpret_cast<T*>(wsm + L.om);
    int* cbo = reinterpret_cast<int*>(wsm + L.cbo);
    int* bad = reinterpret_cast<int*>(wsm + L.bad);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T* K = Kk;
    int LK = Q;
    if (kstage) {  // K_k once per CTA, rows at the odd stride k_stride(Q)
        T* Ks = reinterpret_cast<T*>(wsm + L.K);
        LK = k_stride(Q);
        for (int idx = tid; idx < Q * Q; idx += WT) {
            const int r = idx / Q, c = idx - r * Q;
            Ks[r * LK + c] = Kk[idx];
        }
        K = Ks;
    }
    for (int j = blockIdx.x; j < Ik; j += gridDim.x) {
        for (int t = 0; t < nm; ++t)
            for (int r = tid; r < q.R[t]; r += WT) gc[t * WIDE_RMAX + r] = Gd[s.goff[k][q.m[t]] + r * Ik + j];
        for (int c = tid; c < Q; c += WT) Mr[c] = Mk[static_cast<long long>(j) * Q + c];
        __syncthreads();
        for (int ti = 0; ti < nm; ++ti) {
            const int Ri = q.R[ti], sp = q.st[ti], Qo = Q / Ri;
            for (int o = tid; o < Qo; o += WT) {  // digits of o over the slots t != ti, last slot fastest
                int rem = o, cb = 0;
                double w = 1.0;
                for (int t = nm - 1; t >= 0; --t) {
                    if (t == ti) continue;
                    const int d = rem % q.R[t];
                    rem /= q.R[t];
                    w *= gc[t * WIDE_RMAX + d];
                    cb += d * q.st[t];
                }
                om[o] = static_cast<T>(w);
                cbo[o] = cb;
            }
            __syncthreads();
            const int ne = Ri * (Ri + 1) / 2;
            const int ng = max(1, min(Qo, HPART / ne));
            const int og = (Qo + ng - 1) / ng;
            for (int it = tid; it < ne * ng; it += WT) {
                const int e = it / ng, g = it - e * ng;
                int c, cp;
                tri_index(e, c, cp);
                T acc = T(0);
                const int o1 = min(Qo, (g + 1) * og);
                for (int o = g * og; o < o1; ++o) {
                    const T* kr = K + static_cast<long long>(cbo[o] + c * sp) * LK + cp * sp;
                    T inner = T(0);
                    for (int o2 = 0; o2 < Qo; ++o2) inner = fma(om[o2], kr[cbo[o2]], inner);
                    acc = fma(om[o], inner, acc);
                }
                part[g * ne + e] = acc;
            }
            for (int c = tid; c < Ri; c += WT) {
                T acc = T(0);
                for (int o = 0; o < Qo; ++o) acc = fma(om[o], static_cast<T>(Mr[cbo[o] + c * sp]), acc);
                bv[c] = static_cast<double>(acc) + rho * gc[ti * WIDE_RMAX + c];
            }
            if (tid == 0) *bad = 0;
            __syncthreads();
            for (int e = tid; e < ne; e += WT) {
                double h = 0.0;
                for (int g = 0; g < ng; ++g) h += static_cast<double>(part[g * ne + e]);
                int c, cp;
                tri_index(e, c, cp);
                H[c * Ri + cp] = h + (c == cp ? rho : 0.0);
            }
            __syncthreads();
            // Cholesky H = L L^T, lower triangle in place
            for (int c = 0; c < Ri; ++c) {
                if (tid == 0) {
                    double d = H[c * Ri + c];
                    if (!(d > 0.0) || !isfinite(d)) {
                        *bad = 1;
                        d = 1.0;
                    }
                    H[c * Ri + c] = sqrt(d);
                }
                __syncthreads();
                const double d = H[c * Ri + c];
                for (int r = c + 1 + tid; r < Ri; r += WT) H[r * Ri + c] /= d;
                __syncthreads();
                const int nt = Ri - c - 1;
                for (int e = tid; e < nt * (nt + 1) / 2; e += WT) {
                    int rr, tt;
                    tri_index(e, rr, tt);
                    const int r = c + 1 + rr, t = c + 1 + tt;
                    H[r * Ri + t] -= H[r * Ri + c] * H[t * Ri + c];
                }
                __syncthreads();
            }
            // L y = b, then L^T g = y, by warp 0
            if (warp == 0) {
                for (int r = 0; r < Ri; ++r) {
                    double v = 0.0;
                    for (int t = lane; t < r; t += 32) v += H[r * Ri + t] * bv[t];
                    v = warp_sum(v);
                    if (lane == 0) bv[r] = (bv[r] - v) / H[r * Ri + r];
                    __syncwarp();
                }
                for (int r = Ri - 1; r >= 0; --r) {
                    double v = 0.0;
                    for (int t = r + 1 + lane; t < Ri; t += 32) v += H[t * Ri + r] * bv[t];
                    v = warp_sum(v);
                    if (lane == 0) bv[r] = (bv[r] - v) / H[r * Ri + r];
                    __syncwarp();
                }
                bool fin = true;
                for (int r = lane; r < Ri; r += 32) fin = fin && isfinite(bv[r]);
                if (!__all_sync(0xffffffffu, fin) && lane == 0) *bad = 1;
            }
            __syncthreads();
            if (*bad) {
                if (tid == 0) atomicOr(flags, FLAG_NOTSPD);  // the old column stays
            } else {
                const int i = q.m[ti];
                for (int c = tid; c < Ri; c += WT) {
                    const double g = bv[c];
                    gc[ti * WIDE_RMAX + c] = g;
                    Gd[s.goff[k][i] + c * Ik + j] = g;
                    Gt[s.goff[k][i] + c * Ik + j] = static_cast<T>(g);
                }
            }
            __syncthreads();
        }
        // W_{k,i}(j, :) from the new columns, in the tensor dtype
        for (int t = 0; t < nm; ++t) {
            const int i = q.m[t], Ri = q.R[t], Ii = s.I[i];
            const T* gik = Gt + s.goff[i][k];
            for (int b2 = tid; b2 < Ii; b2 += WT) {
                T w = T(0);
                for (int r = 0; r < Ri; ++r)
                    w = fma(static_cast<T>(gc[t * WIDE_RMAX + r]), gik[static_cast<long long>(r) * Ii + b2], w);
                if (k < i)
                    W[s.woff[k][i] + static_cast<long long>(j) * Ii + b2] = w;
                else
                    W[s.woff[i][k] + static_cast<long long>(b2) * Ik + j] = w;
            }
        }
        __syncthreads();
    }
}

}  // namespace

WideChain wide_chain(const Shape& s, int k) {
    WideChain c;
    int a, b;
    other_modes(k, a, b);
    // contraction: the contiguous mode first unless it is k (coalesced loads
    // of X either way); for k = 2 the order with fewer multiply-adds
    if (k != 2) {
        c.c1 = 2;
        c.c2 = k == 0 ? 1 : 0;
    } else {
        const int Q = s.R[k][a] * s.R[k][b];
        const double ca = static_cast<double>(s.P) * s.R[k][a] + static_cast<double>(s.I[k]) * s.I[b] * Q;
        const double cb = static_cast<double>(s.P) * s.R[k][b] + static_cast<double>(s.I[k]) * s.I[a] * Q;
        c.c1 = ca <= cb ? a : b;
        c.c2 = ca <= cb ? b : a;
    }
    // Gram: the mode with the cheaper chain summed first
    const double Ia = s.I[a], Ib = s.I[b], Ra = s.R[k][a], Rb = s.R[k][b];
    const double Q2 = Ra * Ra * Rb * Rb;
    const double ga = Ia * Ib * Ra * Ra + Ib * Q2;
    const double gb = Ia * Ib * Rb * Rb + Ia * Q2;
    c.d1 = ga <= gb ? a : b;
    c.d2 = ga <= gb ? b : a;
    return c;
}

long long wide_v_elems(const Shape& s, int k) {
    const WideChain c = wide_chain(s, k);
    return static_cast<long long>(s.I[k]) * s.I[c.c2] * s.R[k][c.c1];
}

long long wide_t_elems(const Shape& s, int k) {
    const WideChain c = wide_chain(s, k);
    return static_cast<long long>(s.I[c.d2]) * s.R[k][c.d1] * s.R[k][c.d1];
}

template <typename T>
cudaError_t launch_wide_contract(const Shape& s, int k, const T* X, const T* Gt, const T* W, T* V, const int* done,
                                 cudaStream_t st) {
    const WideChain c = wide_chain(s, k);
    const long long str[3] = {static_cast<long long>(s.I[1]) * s.I[2], s.I[2], 1};
    OpContract1<T> op;
    op.X = X;
    op.W = pair_view(s, W, c.c1, c.c2, op.wsi, op.wsb);
    op.G = Gt + s.goff[c.c1][k];
    op.V = V;
    op.sk = str[k];
    op.sc1 = str[c.c1];
    op.sc2 = str[c.c2];
    op.Ic1 = s.I[c.c1];
    op.Ic2 = s.I[c.c2];
    op.R1 = s.R[k][c.c1];
    op.M = s.I[k];
    op.N = op.R1;
    op.K = op.Ic1;
    op.batch = op.Ic2;
    op.a_m_fast = op.sk == 1;
    op.b_n_fast = false;
    return launch_gemm<T>(op, done, st);
}

template <typename T>
cudaError_t launch_wide_finish(const Shape& s, int k, const T* Gt, const T* V, double* Mk, const int* done,
                               cudaStream_t st) {
    const WideChain c = wide_chain(s, k);
    OpContract2<T> op;
    op.G = Gt + s.goff[c.c2][k];
    op.V = V;
    op.Mk = Mk;
    op.Ic2 = s.I[c.c2];
    op.R1 = s.R[k][c.c1];
    const int R2 = s.R[k][c.c2];
    op.Q = op.R1 * R2;
    // q = r_a R_{k,b} + r_b (a < b the other modes)
    if (c.c2 < c.c1) {
        op.qsm = op.R1;
        op.qsn = 1;
    } else {
        op.qsm = 1;
        op.qsn = R2;
    }
    op.M = R2;
    op.N = op.R1;
    op.K = op.Ic2;
    op.batch = s.I[k];
    op.a_m_fast = false;
    op.b_n_fast = true;
    return launch_gemm<T>(op, done, st);
}

template <typename T>
cudaError_t launch_wide_gram(const Shape& s, int k, const T* Gt, const T* W, T* Tg, T* Kk, const int* done,
                             cudaStream_t st) {
    const WideChain c = wide_chain(s, k);
    const int R1 = s.R[k][c.d1], R2 = s.R[k][c.d2];
    OpGram1<T> g1;
    int sp, sq;
    g1.W = pair_view(s, W, c.d1, c.d2, sp, sq);
    g1.wsi = sp;
    g1.wsb = sq;
    g1.G = Gt + s.goff[c.d1][k];
    g1.Tg = Tg;
    g1.Id1 = s.I[c.d1];
    g1.R1 = R1;
    g1.M = s.I[c.d2];
    g1.N = R1 * R1;
    g1.K = g1.Id1;
    g1.batch = 1;
    g1.a_m_fast = sq == 1;
    g1.b_n_fast = false;
    cudaError_t e = launch_gemm<T>(g1, done, st);
    if (e != cudaSuccess) return e;
    OpGram2<T> g2;
    g2.G = Gt + s.goff[c.d2][k];
    g2.Tg = Tg;
    g2.Kk = Kk;
    g2.Id2 = s.I[c.d2];
    g2.R1 = R1;
    g2.R2 = R2;
    g2.Q = R1 * R2;
    // q = r_a R_{k,b} + r_b (a < b the other modes)
    if (c.d1 < c.d2) {
        g2.s1 = R2;
        g2.s2 = 1;
    } else {
        g2.s1 = 1;
        g2.s2 = R1;
    }
    g2.M = R2 * R2;
    g2.N = R1 * R1;
    g2.K = g2.Id2;
    g2.batch = 1;
    g2.a_m_fast = false;
    g2.b_n_fast = true;
    return launch_gemm<T>(g2, done, st);
}

template <typename T>
cudaError_t launch_gram4_gemm(const Shape& s, int k, const T* Gt, const T* W, T* t1, T* t2, const int* done,
                              cudaStream_t st) {
    int m[3], nm = 0;
    for (int q = 0; q < s.N; ++q)
        if (q != k) m[nm++] = q;
    if (nm != 3) return cudaErrorInvalidValue;
    const int o = m[0], c = m[1], l = m[2];
    const int RL = s.R[k][l], Rc = s.R[k][c], NP = RL * (RL + 1) / 2;
    OpGram4a<T> a;
    a.Wcl = pair_view(s, W, c, l, a.cs_c, a.cs_l);
    a.Wol = pair_view(s, W, o, l, a.os_o, a.os_l);
    a.Woc = pair_view(s, W, o, c, a.ws_o, a.ws_c);
    a.Gl = Gt + s.goff[l][k];
    a.t1 = t1;
    a.Il = s.I[l];
    a.RL = RL;
    a.M = s.I[c];
    a.N = NP;
    a.K = s.I[l];
    a.batch = s.I[o];
    a.a_m_fast = a.cs_c == 1;
    a.b_n_fast = false;
    cudaError_t e = launch_gemm<T>(a, done, st);
    if (e != cudaSuccess) return e;
    OpGram4b<T> b;
    b.Gc = Gt + s.goff[c][k];
    b.t1 = t1;
    b.T2 = t2;
    b.Ic = s.I[c];
    b.Rc = Rc;
    b.RL = RL;
    b.NP = NP;
    b.M = Rc * Rc;
    b.N = NP;
    b.K = s.I[c];
    b.batch = s.I[o];
    b.a_m_fast = false;
    b.b_n_fast = true;
    return launch_gemm<T>(b, done, st);
}

template <typename T>
cudaError_t launch_cta_solve(const Shape& s, int k, double rho, const double* Mk, const T* Kk, double* Gd, T* Gt,
                             T* W, int* flags, const int* done, cudaStream_t st) {
    const Slots q = slots_of(s, k);
    if (s.N < 3 || q.Rx > WIDE_RMAX || q.Q > WIDE_QMAX) return cudaErrorInvalidValue;
    const int sz = static_cast<int>(sizeof(T));
    // K_k staged in shared memory when the whole layout stays within about
    // half of an SM's shared memory (two CTAs a SM)
    int kstage = cta_solve_layout(q, sz, true).total <= 110 * 1024 ? 1 : 0;
    const int smem = static_cast<int>(cta_solve_layout(q, sz, kstage != 0).total);
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(k_cta_solve<T>), smem);
    if (e != cudaSuccess) return e;
    k_cta_solve<T><<<std::min(s.I[k], 65535), WT, smem, st>>>(s, k, rho, Mk, Kk, Gd, Gt, W, flags, done, kstage);
    return cudaGetLastError();
}

#define IFCTN_WIDE_INST(T)                                                                                         \
    template cudaError_t launch_wide_contract<T>(const Shape&, int, const T*, const T*, const T*, T*, const int*, \
                                                 cudaStream_t);                                                   \
    template cudaError_t launch_wide_finish<T>(const Shape&, int, const T*, const T*, double*, const int*,        \
                                               cudaStream_t);                                                     \
    template cudaError_t launch_wide_gram<T>(const Shape&, int, const T*, const T*, T*, T*, const int*,           \
                                             cudaStream_t);                                                       \
    template cudaError_t launch_cta_solve<T>(const Shape&, int, double, const double*, const T*, double*, T*, T*, \
                                             int*, const int*, cudaStream_t);                                     \
    template cudaError_t launch_gram4_gemm<T>(const Shape&, int, const T*, const T*, T*, T*, const int*,         \
                                              cudaStream_t);
IFCTN_WIDE_INST(float)
IFCTN_WIDE_INST(double)
#undef IFCTN_WIDE_INST

}  // namespace ifctn
