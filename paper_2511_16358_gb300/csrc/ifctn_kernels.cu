// ifctn_kernels.cu -- Gram chain, proximal solves, fused X update and helpers.
#include <cstdlib>
#include <cstring>

#include "ifctn_launch.h"

namespace ifctn {
namespace {

__device__ __forceinline__ int nonk_modes(const Shape& s, int k, int* m) {
    int t = 0;
    for (int q = 0; q < s.N; ++q)
        if (q != k) m[t++] = q;
    return t;
}

template <typename T>
__device__ __forceinline__ T to_t(double v) { return static_cast<T>(v); }

// ---------------------------------------------------------------------------
// Gram K_k = Z_k^T Z_k (Prop. 1): sum over i_{-k} of S_k^2 times the Kronecker
// product of G_{m,k}(:,i_m) G_{m,k}(:,i_m)^T, contracted one mode at a time.
// Non-k modes in ascending order: [o] (N=2), [o, l] (N=3), [o, c, l] (N=4).
//   t1 (N=3):  T2[io][x][y]      = sum_il W_ol(io,il)^2 g_l(x,il) g_l(y,il)
//   t1 (N=4):  T1[io][ic][x][y]  = W_oc(io,ic)^2 sum_il (W_ol W_cl)^2 g_l g_l
//   t2 (N=4):  T2[io][X][Y]      = sum_ic g_c(xc,ic) g_c(yc,ic) T1[io][ic][xl][yl]
//   fin:       K[(xo,X),(yo,Y)]  = sum_io g_o(xo,io) g_o(yo,io) T2[io][X][Y]
// with g_m = G_{m,k}.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gram_t1(const __grid_constant__ Shape s, const int k, const T* __restrict__ Gt,
                                                 const T* __restrict__ W, T* __restrict__ out,
                                                 const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    int m[3];
    nonk_modes(s, k, m);
    const int o = m[0];
    const int l = s.N == 3 ? m[1] : m[2];
    const int c = s.N == 4 ? m[1] : -1;
    const int Io = s.I[o], Il = s.I[l], Ic = c >= 0 ? s.I[c] : 1;
    const int Rl = s.R[k][l];
    const long long total = static_cast<long long>(Io) * Ic * Rl * Rl;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int y = static_cast<int>(idx % Rl);
        const int x = static_cast<int>((idx / Rl) % Rl);
        const long long oc = idx / (static_cast<long long>(Rl) * Rl);
        const int ic = static_cast<int>(oc % Ic);
        const int io = static_cast<int>(oc / Ic);
        const T* gx = Gt + s.goff[l][k] + x * Il;
        const T* gy = Gt + s.goff[l][k] + y * Il;
        const T* wol = W + s.woff[o][l] + static_cast<long long>(io) * Il;
        T acc = T(0);
        if (c < 0) {
            for (int il = 0; il < Il; ++il) {
                const T w = wol[il];
                acc = fma(w * w, gx[il] * gy[il], acc);
            }
        } else {
            const T* wcl = W + s.woff[c][l] + static_cast<long long>(ic) * Il;
            for (int il = 0; il < Il; ++il) {
                const T w = wol[il] * wcl[il];
                acc = fma(w * w, gx[il] * gy[il], acc);
            }
            const T woc = W[s.woff[o][c] + static_cast<long long>(io) * Ic + ic];
            acc *= woc * woc;
        }
        out[idx] = acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gram_t2(const __grid_constant__ Shape s, const int k, const T* __restrict__ Gt,
                                                 const T* __restrict__ t1, T* __restrict__ t2,
                                                 const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    int m[3];
    nonk_modes(s, k, m);
    const int o = m[0], c = m[1], l = m[2];
    const int Io = s.I[o], Ic = s.I[c];
    const int Rc = s.R[k][c], Rl = s.R[k][l];
    const int Q2 = Rc * Rl;
    const long long total = static_cast<long long>(Io) * Q2 * Q2;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int Y = static_cast<int>(idx % Q2);
        const int X = static_cast<int>((idx / Q2) % Q2);
        const int io = static_cast<int>(idx / (static_cast<long long>(Q2) * Q2));
        const int xc = X / Rl, xl = X - xc * Rl, yc = Y / Rl, yl = Y - yc * Rl;
        const T* gx = Gt + s.goff[c][k] + xc * Ic;
        const T* gy = Gt + s.goff[c][k] + yc * Ic;
        const T* tp = t1 + static_cast<long long>(io) * Ic * Rl * Rl + xl * Rl + yl;
        T acc = T(0);
        for (int ic = 0; ic < Ic; ++ic) acc = fma(gx[ic] * gy[ic], tp[static_cast<long long>(ic) * Rl * Rl], acc);
        t2[idx] = acc;
    }
}

// Pair index p of the upper triangle (x <= y, row-major) of an R x R block.
__device__ __forceinline__ void pair_xy(int p, int R, int& x, int& y) {
    int r = p, xx = 0;
    while (r >= R - xx) {
        r -= R - xx;
        ++xx;
    }
    x = xx;
    y = xx + r;
}

// NP consecutive elements from 16-byte aligned shared memory (NP a multiple
// of 16 / sizeof(T)).
template <typename T, int NP>
__device__ __forceinline__ void ld_vec(const T* __restrict__ p, T (&o)[NP]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < NP; i += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + i);
            o[i] = v.x;
            o[i + 1] = v.y;
            o[i + 2] = v.z;
            o[i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NP; i += 2) {
            const double2 v = *reinterpret_cast<const double2*>(p + i);
            o[i] = v.x;
            o[i + 1] = v.y;
        }
    }
}

// Fused first two steps of the chain for N = 4 (non-k modes o < c < l), one
// CTA per io, with T1 kept in shared memory:
//   h(il, p)  = W_ol(io, il)^2 g_l(x, il) g_l(y, il),                 p = (x <= y)
//   T1(ic, p) = W_oc(io, ic)^2 sum_il W_cl(ic, il)^2 h(il, p)
//   T2[io][(xc, xl)][(yc, yl)] = sum_ic g_c(xc, ic) g_c(yc, ic) T1(ic, p(xl, yl))
// A warp takes 32 consecutive ic (lane = ic) and streams W_cl through a
// 32 x 33 shared tile (rows read coalesced, columns read without bank
// conflicts); every lane keeps all pairs p of its ic in registers.
constexpr int GRAM_WARPS = 8;

template <typename T, int RL>
__host__ __device__ constexpr int gram_npp() {
    constexpr int NP = RL * (RL + 1) / 2, VN = 16 / static_cast<int>(sizeof(T));
    return (NP + VN - 1) / VN * VN;
}

template <typename T>
long long gram_io_smem(int RL, int Il, int Ic, int Rc) {
    const int NP = RL * (RL + 1) / 2, VN = 16 / static_cast<int>(sizeof(T));
    const int NPP = (NP + VN - 1) / VN * VN;
    return (static_cast<long long>(Il) * NPP + static_cast<long long>(Ic) * NP + static_cast<long long>(Rc) * Ic +
            GRAM_WARPS * 32 * 33) * sizeof(T) + 16;
}

template <typename T, int RL>
__global__ void __launch_bounds__(GRAM_WARPS * 32) k_gram_io(const __grid_constant__ Shape s, const int k,
                                                             const T* __restrict__ Gt, const T* __restrict__ W,
                                                             T* __restrict__ t2, const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    extern __shared__ __align__(16) unsigned char gsm[];
    constexpr int NP = RL * (RL + 1) / 2;
    constexpr int NPP = gram_npp<T, RL>();
    int m[3];
    nonk_modes(s, k, m);
    const int o = m[0], c = m[1], l = m[2];
    const int Ic = s.I[c], Il = s.I[l];
    const int Rc = s.R[k][c];
    const int io = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T* hs = reinterpret_cast<T*>(gsm);  // [Il][NPP]
    T* t1s = hs + Il * NPP;              // [Ic][NP]
    T* gcs = t1s + Ic * NP;              // [Rc][Ic]
    T* tile = gcs + Rc * Ic + warp * 32 * 33;
    const T* gl = Gt + s.goff[l][k];
    const T* wol = W + s.woff[o][l] + static_cast<long long>(io) * Il;
    const T* woc = W + s.woff[o][c] + static_cast<long long>(io) * Ic;
    const T* wcl = W + s.woff[c][l];
    for (int idx = tid; idx < Il * NPP; idx += blockDim.x) {
        const int il = idx / NPP, p = idx - il * NPP;
        T v = T(0);
        if (p < NP) {
            int x, y;
            pair_xy(p, RL, x, y);
            const T w = wol[il];
            v = w * w * gl[x * Il + il] * gl[y * Il + il];
        }
        hs[idx] = v;
    }
    for (int idx = tid; idx < Rc * Ic; idx += blockDim.x) gcs[idx] = Gt[s.goff[c][k] + idx];
    __syncthreads();
    for (int ic0 = warp * 32; ic0 < Ic; ic0 += GRAM_WARPS * 32) {
        const int ic = ic0 + lane;
        const int nr = min(32, Ic - ic0);
        T acc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q] = T(0);
        for (int il0 = 0; il0 < Il; il0 += 32) {
            const int nil = min(32, Il - il0);
            __syncwarp();
            if (lane < nil)
                for (int r = 0; r < nr; ++r) tile[r * 33 + lane] = wcl[static_cast<long long>(ic0 + r) * Il + il0 + lane];
            __syncwarp();
            if (lane < nr) {
                for (int j = 0; j < nil; ++j) {
                    T bw = tile[lane * 33 + j];
                    bw *= bw;
                    T hv[NPP];
                    ld_vec<T, NPP>(hs + (il0 + j) * NPP, hv);
#pragma unroll
                    for (int q = 0; q < NP; ++q) acc[q] = fma(bw, hv[q], acc[q]);
                }
            }
        }
        if (lane < nr) {
            const T wo = woc[ic];
            const T w2 = wo * wo;
#pragma unroll
            for (int q = 0; q < NP; ++q) t1s[ic * NP + q] = acc[q] * w2;
        }
    }
    __syncthreads();
    const int Q2 = Rc * RL;
    T* out = t2 + static_cast<long long>(io) * Q2 * Q2;
    for (int idx = tid; idx < Rc * Rc * NP; idx += blockDim.x) {
        const int xy = idx / NP, p = idx - xy * NP;
        const int xc = xy / Rc, yc = xy - xc * Rc;
        int xl, yl;
        pair_xy(p, RL, xl, yl);
        const T* ga = gcs + xc * Ic;
        const T* gb = gcs + yc * Ic;
        const T* tp = t1s + p;
        T a0 = T(0), a1 = T(0);
        int ic = 0;
        for (; ic + 1 < Ic; ic += 2) {
            a0 = fma(ga[ic] * gb[ic], tp[ic * NP], a0);
            a1 = fma(ga[ic + 1] * gb[ic + 1], tp[(ic + 1) * NP], a1);
        }
        if (ic < Ic) a0 = fma(ga[ic] * gb[ic], tp[ic * NP], a0);
        const T v = a0 + a1;
        out[(xc * RL + xl) * Q2 + yc * RL + yl] = v;
        if (xl != yl) out[(xc * RL + yl) * Q2 + yc * RL + xl] = v;
    }
}

// Last step: K[(xo, X), (yo, Y)] = sum_io g_o(xo, io) g_o(yo, io) T2[io][X][Y]
// (N = 3, 4; for N = 2 directly sum_io g_o(xo, io) g_o(yo, io)).  A CTA takes
// 32 consecutive entries of K (lane = entry); its warps split the io range and
// their sums are added in a fixed order.
template <typename T>
__global__ void __launch_bounds__(GRAM_WARPS * 32) k_gram_fin(const __grid_constant__ Shape s, const int k,
                                                              const T* __restrict__ Gt, const T* __restrict__ t2,
                                                              T* __restrict__ K, const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    __shared__ T red[GRAM_WARPS][32];
    int m[3];
    const int nm = nonk_modes(s, k, m);
    const int o = m[0];
    const int Io = s.I[o];
    int Q2 = 1;
    for (int t = 1; t < nm; ++t) Q2 *= s.R[k][m[t]];
    const int Q = s.R[k][o] * Q2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long idx = blockIdx.x * 32LL + lane;
    const bool act = idx < static_cast<long long>(Q) * Q;
    const int per = (Io + GRAM_WARPS - 1) / GRAM_WARPS;
    const int io0 = warp * per, io1 = min(Io, io0 + per);
    T acc = T(0);
    if (act) {
        const int col = static_cast<int>(idx % Q), row = static_cast<int>(idx / Q);
        const int xo = row / Q2, X = row - xo * Q2, yo = col / Q2, Y = col - yo * Q2;
        const T* gx = Gt + s.goff[o][k] + xo * Io;
        const T* gy = Gt + s.goff[o][k] + yo * Io;
        if (nm == 1) {
            for (int io = io0; io < io1; ++io) acc = fma(gx[io], gy[io], acc);
        } else {
            const T* tp = t2 + static_cast<long long>(X) * Q2 + Y;
            const long long st = static_cast<long long>(Q2) * Q2;
            for (int io = io0; io < io1; ++io) acc = fma(gx[io] * gy[io], tp[io * st], acc);
        }
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && act) {
        T v = red[0][lane];
#pragma unroll
        for (int w = 1; w < GRAM_WARPS; ++w) v += red[w][lane];
        K[idx] = v;
    }
}

// ---------------------------------------------------------------------------
// Element index walker over the slab geometry (i0, i1 = F modes; a, b = the
// last two modes) with carries, so no division runs per element.
// ---------------------------------------------------------------------------
struct Walk {
    int i0, i1, a, b;
};

__device__ __forceinline__ void walk_from(const Shape& s, long long e, Walk& w) {
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

__device__ __forceinline__ void walk_inc(const Shape& s, Walk& w) {
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

// advance by a fixed stride decomposed as (d0, d1, da, db) with single carries
struct Stride {
    int d0, d1, da, db;
};

__device__ __forceinline__ Stride stride_of(const Shape& s, long long d) {
    Stride t;
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

__device__ __forceinline__ void walk_add(const Shape& s, Walk& w, const Stride& t) {
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

// iFCTN(G)(i) = prod_{p<q} W_{p,q}(i_p, i_q) at the walker position
template <typename T>
__device__ __forceinline__ T recon_at(const Shape& s, const T* __restrict__ W, const Walk& w) {
    const int N = s.N, Am = N - 2, Bm = N - 1;
    T v = W[s.woff[Am][Bm] + static_cast<long long>(w.a) * s.IB + w.b];
    if (N >= 3) {
        v *= W[s.woff[0][Am] + static_cast<long long>(w.i0) * s.IA + w.a] *
             W[s.woff[0][Bm] + static_cast<long long>(w.i0) * s.IB + w.b];
    }
    if (N == 4) {
        v *= W[s.woff[1][Am] + static_cast<long long>(w.i1) * s.IA + w.a] *
             W[s.woff[1][Bm] + static_cast<long long>(w.i1) * s.IB + w.b] *
             W[s.woff[0][1] + static_cast<long long>(w.i0) * s.I[1] + w.i1];
    }
    return v;
}

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int n = 2;
};

__device__ __forceinline__ float vget(const float4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ double vget(const double2& v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ void vset(float4& v, int i, float x) {
    if (i == 0) v.x = x;
    else if (i == 1) v.y = x;
    else if (i == 2) v.z = x;
    else v.w = x;
}
__device__ __forceinline__ void vset(double2& v, int i, double x) {
    if (i == 0) v.x = x;
    else v.y = x;
}

template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* out) {
    __shared__ double sh[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = warp_sum(v[t]);
    if (lane == 0)
#pragma unroll
        for (int t = 0; t < NV; ++t) sh[warp][t] = v[t];
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += sh[w][threadIdx.x];
        out[threadIdx.x] = acc;
    }
}

// ---------------------------------------------------------------------------
// eq. (updateX): X <- P_{Omega^c}((iFCTN(G) + rho X)/(1+rho)) + P_Omega(X),
// fused with the reconstruction and the sweep reductions
//   xpart[blk] = { ||X1-X0||^2, ||X0||^2, ||X1 - iFCTN(G)||^2 }.
// One read and one write of X plus the mask bitset; grid-stride over 16-byte
// vectors.  FP32 accumulation in short runs, carried in FP64.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_xupdate(const __grid_constant__ Shape s, const T rho, const T inv1p,
                                                 T* __restrict__ X, const uint32_t* __restrict__ mb,
                                                 const T* __restrict__ W, double* __restrict__ xpart,
                                                 const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    using V = typename Vec<T>::type;
    constexpr int NV = Vec<T>::n;
    const long long P = s.P;
    const long long nvec = P / NV;
    const long long gtid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    double acc[3] = {0.0, 0.0, 0.0};
    T fa[3] = {T(0), T(0), T(0)};
    int run = 0;
    Walk w;
    walk_from(s, gtid * NV, w);
    const Stride stp = stride_of(s, gstr * NV - NV);
    V* Xv = reinterpret_cast<V*>(X);
    for (long long v = gtid; v < nvec; v += gstr) {
        V xv = Xv[v];
        const long long e0 = v * NV;
        const uint32_t word = mb[e0 >> 5];
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const T xo = vget(xv, t);
            const T rec = recon_at(s, W, w);
            const bool obs = (word >> ((e0 + t) & 31)) & 1u;
            const T xn = obs ? xo : (rec + rho * xo) * inv1p;
            vset(xv, t, xn);
            const T d = xn - xo, r = xn - rec;
            fa[0] = fma(d, d, fa[0]);
            fa[1] = fma(xo, xo, fa[1]);
            fa[2] = fma(r, r, fa[2]);
            walk_inc(s, w);
        }
        Xv[v] = xv;
        walk_add(s, w, stp);
        if (++run == 16) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                acc[t] += static_cast<double>(fa[t]);
                fa[t] = T(0);
            }
            run = 0;
        }
    }
    if (gtid == 0) {  // ragged tail
        Walk wt;
        walk_from(s, nvec * NV, wt);
        for (long long e = nvec * NV; e < P; ++e) {
            const T xo = X[e];
            const T rec = recon_at(s, W, wt);
            const bool obs = (mb[e >> 5] >> (e & 31)) & 1u;
            const T xn = obs ? xo : (rec + rho * xo) * inv1p;
            X[e] = xn;
            const T d = xn - xo, r = xn - rec;
            fa[0] = fma(d, d, fa[0]);
            fa[1] = fma(xo, xo, fa[1]);
            fa[2] = fma(r, r, fa[2]);
            walk_inc(s, wt);
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) acc[t] += static_cast<double>(fa[t]);
    block_sum_store<3>(acc, xpart + 3 * blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(256) k_reconstruct(const __grid_constant__ Shape s, const T* __restrict__ W,
                                                     T* __restrict__ out, double* __restrict__ xpart) {
    pdl_begin();
    const long long P = s.P;
    const long long gtid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    double acc[3] = {0.0, 0.0, 0.0};
    T fa = T(0);
    int run = 0;
    if (gtid < P) {
        Walk w;
        walk_from(s, gtid, w);
        const Stride stp = stride_of(s, gstr);
        for (long long e = gtid; e < P; e += gstr) {
            const T rec = recon_at(s, W, w);
            if (out) out[e] = rec;
            fa = fma(rec, rec, fa);
            if (++run == 64) {
                acc[0] += static_cast<double>(fa);
                fa = T(0);
                run = 0;
            }
            walk_add(s, w, stp);
        }
    }
    acc[0] += static_cast<double>(fa);
    if (xpart) block_sum_store<3>(acc, xpart + 3 * blockIdx.x);
}

// RSE / RMSE sums: { ||Xt-X||^2, ||Xt||^2, sum over missing (Xt-X)^2 }
template <typename T>
__global__ void __launch_bounds__(256) k_metrics(const long long P, const T* __restrict__ X,
                                                 const T* __restrict__ Xt, const uint32_t* __restrict__ mb,
                                                 double* __restrict__ mpart, const int* __restrict__ done) {
    pdl_begin();
    if (*done) return;
    const long long gtid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    double acc[3] = {0.0, 0.0, 0.0};
    T fa[3] = {T(0), T(0), T(0)};
    int run = 0;
    for (long long e = gtid; e < P; e += gstr) {
        const T d = Xt[e] - X[e];
        const bool obs = (mb[e >> 5] >> (e & 31)) & 1u;
        fa[0] = fma(d, d, fa[0]);
        fa[1] = fma(Xt[e], Xt[e], fa[1]);
        if (!obs) fa[2] = fma(d, d, fa[2]);
        if (++run == 64) {
            for (int t = 0; t < 3; ++t) {
                acc[t] += static_cast<double>(fa[t]);
                fa[t] = T(0);
            }
            run = 0;
        }
    }
    for (int t = 0; t < 3; ++t) acc[t] += static_cast<double>(fa[t]);
    block_sum_store<3>(acc, mpart + 3 * blockIdx.x);
}

template <typename T>
__global__ void k_pairs(const __grid_constant__ Shape s, const double* __restrict__ Gd, T* __restrict__ W) {
    pdl_begin();
    const long long gtid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long idx = gtid; idx < s.wsize; idx += gstr) {
        int p = 0, q = 1;
        for (int pp = 0; pp < s.N; ++pp)
            for (int qq = pp + 1; qq < s.N; ++qq)
                if (idx >= s.woff[pp][qq]) {
                    p = pp;
                    q = qq;
                }
        // the last pair whose offset is <= idx (offsets increase in (p,q) order)
        const long long rel = idx - s.woff[p][q];
        const int a = static_cast<int>(rel / s.I[q]), b = static_cast<int>(rel % s.I[q]);
        const int R = s.R[p][q];
        double acc = 0.0;
        for (int r = 0; r < R; ++r)
            acc = fma(Gd[s.goff[p][q] + r * s.I[p] + a], Gd[s.goff[q][p] + r * s.I[q] + b], acc);
        W[idx] = to_t<T>(acc);
    }
}

template <typename T>
__global__ void k_init_x(const long long P, const T* __restrict__ O, const uint8_t* __restrict__ mask,
                         T* __restrict__ X) {
    pdl_begin();
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < P; e += gstr)
        X[e] = mask[e] ? O[e] : T(0);
}

__global__ void k_pack_mask(const long long P, const uint8_t* __restrict__ mask, uint32_t* __restrict__ bits) {
    pdl_begin();
    const long long nw = (P + 31) / 32;
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long wd = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; wd < nw; wd += gstr) {
        uint32_t v = 0;
        for (int t = 0; t < 32; ++t) {
            const long long e = wd * 32 + t;
            if (e < P && mask[e]) v |= (1u << t);
        }
        bits[wd] = v;
    }
}

template <typename T>
__global__ void k_cast(const int n, const double* __restrict__ a, T* __restrict__ b) {
    pdl_begin();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = to_t<T>(a[i]);
}

__global__ void k_finalize(const double* __restrict__ xpart, const int nblocks, const double* __restrict__ mpart,
                           const int mblocks, const long long nmiss, const double* __restrict__ tolp,
                           SweepStat* __restrict__ log, const int cap, int* __restrict__ counter,
                           int* __restrict__ done, const int* __restrict__ flags) {
    pdl_begin();
    if (*done) return;
    __shared__ double sh[256][6];
    const int t = threadIdx.x;
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int b = t; b < nblocks; b += blockDim.x)
        for (int c = 0; c < 3; ++c) a[c] += xpart[3 * b + c];
    if (mpart)
        for (int b = t; b < mblocks; b += blockDim.x)
            for (int c = 0; c < 3; ++c) a[3 + c] += mpart[3 * b + c];
    for (int c = 0; c < 6; ++c) sh[t][c] = a[c];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (t < h)
            for (int c = 0; c < 6; ++c) sh[t][c] += sh[t + h][c];
        __syncthreads();
    }
    if (t == 0) {
        const double tol = *tolp;
        const double dx2 = sh[0][0], x2 = sh[0][1], ob = sh[0][2];
        SweepStat r;
        r.rel_change = x2 > 0 ? sqrt(dx2) / sqrt(x2) : (dx2 > 0 ? INFINITY : 0.0);
        r.objective = 0.5 * ob;
        if (mpart) {
            r.rse = sh[0][4] > 0 ? sqrt(sh[0][3]) / sqrt(sh[0][4]) : NAN;
            r.rmse = nmiss > 0 ? sqrt(sh[0][5] / static_cast<double>(nmiss)) : 0.0;
        } else {
            r.rse = NAN;
            r.rmse = NAN;
        }
        r.dx2 = dx2;
        r.x2 = x2;
        const int sidx = *counter;
        r.sweep = sidx + 1;
        r.converged = (tol > 0 && r.rel_change < tol) ? 1 : 0;
        r.flags = *flags;
        r.pad = 0;
        if (!isfinite(r.rel_change) || !isfinite(r.objective)) r.flags |= FLAG_NONFINITE;
        log[sidx % cap] = r;
        *counter = sidx + 1;
        if (r.converged) *done = 1;
    }
}

// Fixed-order reduction of the per-CTA sums of the slab X update (8-double
// stride: ||X1-X0||^2, ||X0||^2, ||X1-rec||^2, then the three RSE/RMSE sums).
__global__ void k_finalize8(const double* __restrict__ xpart, const int nblocks, const int met, const long long nmiss,
                            const double* __restrict__ tolp, SweepStat* __restrict__ log, const int cap,
                            int* __restrict__ counter, int* __restrict__ done, const int* __restrict__ flags) {
    pdl_begin();
    if (*done) return;
    __shared__ double sh[256][6];
    const int t = threadIdx.x;
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int b = t; b < nblocks; b += blockDim.x)
        for (int c = 0; c < 6; ++c) a[c] += xpart[8 * b + c];
    for (int c = 0; c < 6; ++c) sh[t][c] = a[c];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (t < h)
            for (int c = 0; c < 6; ++c) sh[t][c] += sh[t + h][c];
        __syncthreads();
    }
    if (t == 0) {
        const double tol = *tolp;
        const double dx2 = sh[0][0], x2 = sh[0][1];
        SweepStat r;
        r.rel_change = x2 > 0 ? sqrt(dx2) / sqrt(x2) : (dx2 > 0 ? INFINITY : 0.0);
        r.objective = 0.5 * sh[0][2];
        if (met) {
            r.rse = sh[0][4] > 0 ? sqrt(sh[0][3]) / sqrt(sh[0][4]) : NAN;
            r.rmse = nmiss > 0 ? sqrt(sh[0][5] / static_cast<double>(nmiss)) : 0.0;
        } else {
            r.rse = NAN;
            r.rmse = NAN;
        }
        r.dx2 = dx2;
        r.x2 = x2;
        const int sidx = *counter;
        r.sweep = sidx + 1;
        r.converged = (tol > 0 && r.rel_change < tol) ? 1 : 0;
        r.flags = *flags;
        r.pad = 0;
        if (!isfinite(r.rel_change) || !isfinite(r.objective)) r.flags |= FLAG_NONFINITE;
        log[sidx % cap] = r;
        *counter = sidx + 1;
        if (r.converged) *done = 1;
    }
}

__global__ void k_sum_partials(const double* __restrict__ xpart, const int nblocks, const int stride,
                               const int slot, double* __restrict__ out) {
    pdl_begin();
    __shared__ double sh[256];
    double a = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a += xpart[stride * b + slot];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_scale(const int n, double* __restrict__ Gd, const double* __restrict__ ratio, const double expo) {
    pdl_begin();
    const double sc = pow(*ratio, expo);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) Gd[i] *= sc;
}

inline int grid_for(long long n, int block, int cap) {
    long long g = (n + block - 1) / block;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

}  // namespace

template <typename T, int RL>
cudaError_t launch_gram_io(const Shape& sh, int k, const T* Gt, const T* W, T* t2, const int* done, int smem,
                           cudaStream_t st) {
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(k_gram_io<T, RL>), smem);
    if (e != cudaSuccess) return e;
    int m[3], nm = 0;
    for (int q = 0; q < sh.N; ++q)
        if (q != k) m[nm++] = q;
    k_gram_io<T, RL><<<sh.I[m[0]], GRAM_WARPS * 32, smem, st>>>(sh, k, Gt, W, t2, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram(const Shape& sh, int k, const T* Gt, const T* W, T* t1, T* t2, T* Kk,
                        const int* done, cudaStream_t st) {
    int m[3], nm = 0;
    for (int q = 0; q < sh.N; ++q)
        if (q != k) m[nm++] = q;
    // IFCTN_GRAM_GEMM=1: the first two steps as two batched products over i_o
    // instead of one CTA per i_o (measured 2.3x slower on the 288x400x60x24
    // shape's modes 2 and 3; kept selectable, and tested, as the alternative)
    const char* ge = getenv("IFCTN_GRAM_GEMM");
    const bool gemm = nm == 3 && ge && strcmp(ge, "1") == 0;
    if (gemm) {
        cudaError_t e = launch_gram4_gemm<T>(sh, k, Gt, W, t1, t2, done, st);
        if (e != cudaSuccess) return e;
    } else if (nm == 3) {
        const int RL = sh.R[k][m[2]];
        const long long smem = gram_io_smem<T>(RL, sh.I[m[2]], sh.I[m[1]], sh.R[k][m[1]]);
        if (smem <= 200 * 1024) {
            cudaError_t e;
            const int sm = static_cast<int>(smem);
            switch (RL) {
                case 1: e = launch_gram_io<T, 1>(sh, k, Gt, W, t2, done, sm, st); break;
                case 2: e = launch_gram_io<T, 2>(sh, k, Gt, W, t2, done, sm, st); break;
                case 3: e = launch_gram_io<T, 3>(sh, k, Gt, W, t2, done, sm, st); break;
                case 4: e = launch_gram_io<T, 4>(sh, k, Gt, W, t2, done, sm, st); break;
                case 5: e = launch_gram_io<T, 5>(sh, k, Gt, W, t2, done, sm, st); break;
                case 6: e = launch_gram_io<T, 6>(sh, k, Gt, W, t2, done, sm, st); break;
                case 7: e = launch_gram_io<T, 7>(sh, k, Gt, W, t2, done, sm, st); break;
                default: e = launch_gram_io<T, 8>(sh, k, Gt, W, t2, done, sm, st); break;
            }
            if (e != cudaSuccess) return e;
        } else {  // T1 too large for shared memory: through global memory
            const long long n1 = static_cast<long long>(sh.I[m[0]]) * sh.I[m[1]] * RL * RL;
            k_gram_t1<T><<<grid_for(n1, 256, 2432), 256, 0, st>>>(sh, k, Gt, W, t1, done);
            const int Q2 = sh.R[k][m[1]] * RL;
            const long long n2 = static_cast<long long>(sh.I[m[0]]) * Q2 * Q2;
            k_gram_t2<T><<<grid_for(n2, 256, 2432), 256, 0, st>>>(sh, k, Gt, t1, t2, done);
        }
    } else if (nm == 2) {
        const long long n1 = static_cast<long long>(sh.I[m[0]]) * sh.R[k][m[1]] * sh.R[k][m[1]];
        k_gram_t1<T><<<grid_for(n1, 256, 2432), 256, 0, st>>>(sh, k, Gt, W, t2, done);
    }
    int Q = 1;
    for (int t = 0; t < nm; ++t) Q *= sh.R[k][m[t]];
    const long long nK = static_cast<long long>(Q) * Q;
    k_gram_fin<T><<<static_cast<int>((nK + 31) / 32), GRAM_WARPS * 32, 0, st>>>(sh, k, Gt, t2, Kk, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xupdate(const Shape& sh, double rho, T* X, const uint32_t* maskbits, const T* W,
                           double* xpart, int nblocks, const int* done, cudaStream_t st) {
    k_xupdate<T><<<nblocks, 256, 0, st>>>(sh, static_cast<T>(rho), static_cast<T>(1.0 / (1.0 + rho)), X,
                                          maskbits, W, xpart, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reconstruct(const Shape& sh, const T* W, T* out, double* xpart, int nblocks,
                               cudaStream_t st) {
    k_reconstruct<T><<<nblocks, 256, 0, st>>>(sh, W, out, xpart);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_metrics(const Shape& sh, const T* X, const T* Xt, const uint32_t* maskbits,
                           double* mpart, int nblocks, const int* done, cudaStream_t st) {
    k_metrics<T><<<nblocks, 256, 0, st>>>(sh.P, X, Xt, maskbits, mpart, done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pairs(const Shape& sh, const double* Gd, T* W, cudaStream_t st) {
    k_pairs<T><<<grid_for(sh.wsize, 256, 4096), 256, 0, st>>>(sh, Gd, W);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_x(long long P, const T* O, const uint8_t* mask, T* X, cudaStream_t st) {
    k_init_x<T><<<grid_for(P, 256, 8192), 256, 0, st>>>(P, O, mask, X);
    return cudaGetLastError();
}

cudaError_t launch_pack_mask(long long P, const uint8_t* mask, uint32_t* bits, cudaStream_t st) {
    k_pack_mask<<<grid_for((P + 31) / 32, 256, 8192), 256, 0, st>>>(P, mask, bits);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cast_factors(int n, const double* Gd, T* Gt, cudaStream_t st) {
    k_cast<T><<<grid_for(n, 256, 1024), 256, 0, st>>>(n, Gd, Gt);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* xpart, int nblocks, const double* mpart, int mblocks,
                            long long nmiss_total, const double* tol, SweepStat* log, int log_cap,
                            int* sweep_counter, int* done, const int* flags, cudaStream_t st) {
    k_finalize<<<1, 256, 0, st>>>(xpart, nblocks, mpart, mblocks, nmiss_total, tol, log, log_cap,
                                  sweep_counter, done, flags);
    return cudaGetLastError();
}

cudaError_t launch_finalize8(const double* xpart, int nblocks, int met, long long nmiss, const double* tol,
                             SweepStat* log, int log_cap, int* sweep_counter, int* done, const int* flags,
                             cudaStream_t st) {
    k_finalize8<<<1, 256, 0, st>>>(xpart, nblocks, met, nmiss, tol, log, log_cap, sweep_counter, done, flags);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* xpart, int nblocks, int stride, int slot, double* out,
                                cudaStream_t st) {
    k_sum_partials<<<1, 256, 0, st>>>(xpart, nblocks, stride, slot, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_factors(int n, double* Gd, const double* ratio, double expo, cudaStream_t st) {
    k_scale<<<grid_for(n, 256, 1024), 256, 0, st>>>(n, Gd, ratio, expo);
    return cudaGetLastError();
}

#define IFCTN_INST(T)                                                                                    \
    template cudaError_t launch_gram<T>(const Shape&, int, const T*, const T*, T*, T*, T*, const int*,   \
                                        cudaStream_t);                                                   \
    template cudaError_t launch_xupdate<T>(const Shape&, double, T*, const uint32_t*, const T*, double*,  \
                                           int, const int*, cudaStream_t);                               \
    template cudaError_t launch_reconstruct<T>(const Shape&, const T*, T*, double*, int, cudaStream_t);  \
    template cudaError_t launch_metrics<T>(const Shape&, const T*, const T*, const uint32_t*, double*,    \
                                           int, const int*, cudaStream_t);                               \
    template cudaError_t launch_pairs<T>(const Shape&, const double*, T*, cudaStream_t);                 \
    template cudaError_t launch_init_x<T>(long long, const T*, const uint8_t*, T*, cudaStream_t);        \
    template cudaError_t launch_cast_factors<T>(int, const double*, T*, cudaStream_t);
IFCTN_INST(float)
IFCTN_INST(double)
#undef IFCTN_INST

}  // namespace ifctn

namespace ifctn {
namespace {
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(const long long P, const T* __restrict__ X, double* __restrict__ part) {
    pdl_begin();
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    double acc[3] = {0.0, 0.0, 0.0};
    T fa = T(0);
    int run = 0;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < P; e += gstr) {
        fa = fma(X[e], X[e], fa);
        if (++run == 64) {
            acc[0] += static_cast<double>(fa);
            fa = T(0);
            run = 0;
        }
    }
    acc[0] += static_cast<double>(fa);
    block_sum_store<3>(acc, part + 3 * blockIdx.x);
}

__global__ void __launch_bounds__(256) k_count_bits(const long long nwords, const uint32_t* __restrict__ bits,
                                                    double* __restrict__ part) {
    pdl_begin();
    const long long gstr = static_cast<long long>(gridDim.x) * blockDim.x;
    double acc[3] = {0.0, 0.0, 0.0};
    long long c = 0;
    for (long long w = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; w < nwords; w += gstr)
        c += __popc(bits[w]);
    acc[0] = static_cast<double>(c);
    block_sum_store<3>(acc, part + 3 * blockIdx.x);
}

__global__ void k_to_double_f(const long long n, const float* __restrict__ a, double* __restrict__ b) {
    pdl_begin();
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        b[i] = static_cast<double>(a[i]);
}
}  // namespace

template <typename T>
cudaError_t launch_sumsq(long long P, const T* X, double* part, int nblocks, cudaStream_t st) {
    k_sumsq<T><<<nblocks, 256, 0, st>>>(P, X, part);
    return cudaGetLastError();
}
template cudaError_t launch_sumsq<float>(long long, const float*, double*, int, cudaStream_t);
template cudaError_t launch_sumsq<double>(long long, const double*, double*, int, cudaStream_t);

cudaError_t launch_count_bits(long long nwords, const uint32_t* bits, double* part, int nblocks,
                              cudaStream_t st) {
    k_count_bits<<<nblocks, 256, 0, st>>>(nwords, bits, part);
    return cudaGetLastError();
}

cudaError_t launch_to_double(long long n, const float* a, double* b, cudaStream_t st) {
    k_to_double_f<<<grid_for(n, 256, 4096), 256, 0, st>>>(n, a, b);
    return cudaGetLastError();
}
}  // namespace ifctn
