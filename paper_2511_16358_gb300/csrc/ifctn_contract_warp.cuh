// ifctn_contract_warp.cuh -- warp-pipelined streaming contraction
// M_k = X_(k) Z_k (Prop. 1) for tensors that stream from HBM.
//
// The arithmetic is the one of the CTA kernels (ifctn_contract_dev.cuh):
// Z_k is never formed; per slab (entries sharing modes 0..N-3) the
// contiguous mode is contracted first against a small coefficient table and
// the result is folded over one more mode in registers.  What changes is the
// organisation, which here is chosen for bandwidth:
//   - one CTA of NWARP = 16 warps per SM (at most 128 registers a thread),
//     looping over work units;
//   - every warp runs its own ring of S shared-memory stages, each one
//     mbarrier phase fed by a single 1-D TMA bulk copy of the task's rows, so
//     the per-tile path waits only on the warp's own copy and a __syncwarp --
//     the CTA meets once per unit, to reduce;
//   - the few W entries a task needs besides its tile are loaded by the
//     lanes that use them, one task ahead, into registers (small TMA copies
//     cost more issue time than they save);
//   - ROW kind (k != N-1): a lane owns one row of the unit for the whole
//     unit and reads it with 16-byte shared loads (skewed where rows would
//     share banks); the coefficient-table row of a column is a broadcast;
//   - COL kind (k = N-1): a lane owns one column; the coefficient table row
//     of a tensor row is a broadcast load.
// Partials go to the same per-unit slots as the CTA kernels and are reduced by
// the same finisher, in a fixed order (deterministic, no atomics).
#pragma once
#include <type_traits>

#include "ifctn_contract_dev.cuh"

namespace ifctn {
namespace wdev {
using namespace cdev;

constexpr int NWARP = 16;
constexpr int MISC_OFF = 512;  // bytes: mbarriers (NWARP x at most 4 stages) live in [0, 512)

// NP consecutive elements from 16-byte aligned shared memory.
template <typename T, int NP>
__device__ __forceinline__ void ld_row(const T* __restrict__ p, T (&o)[NP]) {
    if constexpr (sizeof(T) == 4) {
        static_assert(NP % 4 == 0, "float rows are read in float4");
#pragma unroll
        for (int i = 0; i < NP; i += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + i);
            o[i] = v.x;
            o[i + 1] = v.y;
            o[i + 2] = v.z;
            o[i + 3] = v.w;
        }
    } else {
        static_assert(NP % 2 == 0, "double rows are read in double2");
#pragma unroll
        for (int i = 0; i < NP; i += 2) {
            const double2 v = *reinterpret_cast<const double2*>(p + i);
            o[i] = v.x;
            o[i + 1] = v.y;
        }
    }
}

// Bounded wait, uniform across the warp.  After the first expiry (abort flag
// set) later waits give in-flight copies only a short grace period.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, unsigned par, volatile int* abortf, int* flags) {
    bool ok = mbar_try_wait(bar, par);
    if (!ok) {
        const long long lim = *abortf ? 2000000LL : 4000000000LL;
        const long long t0 = clock64();
        while (!(ok = mbar_try_wait(bar, par))) {
            if (clock64() - t0 > lim) {
                atomicOr(flags, FLAG_TIMEOUT);
                *abortf = 1;
                break;
            }
        }
    }
    return __all_sync(0xffffffffu, ok) != 0;
}

// Waits until at most S-1 of this thread's cp.async groups are pending (the
// group of the oldest stage of an S-stage ring is then complete).
__device__ __forceinline__ void cp_async_wait_ring(int S) {
    if (S <= 2) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else if (S == 3) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else asm volatile("cp.async.wait_group 3;" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(sizeof(T))
                 : "memory");
}

// One task: slab f, rows [a0, a0 + na).
struct Task {
    long long f;
    int a0, na;
};

// Unit fields the issue path needs, cached while the cursor stays in a unit.
struct UnitCur {
    int ui, ns, nrb, nt;
    long long f0, fstride;
    int a0, a1;
};

__device__ __forceinline__ void load_unit(const UnitDesc* units, int ui, int rbk, UnitCur& c) {
    const UnitDesc u = units[ui];
    c.ui = ui;
    c.ns = u.ns;
    c.nrb = (u.a1 - u.a0 + rbk - 1) / rbk;
    c.nt = u.ns * c.nrb;
    c.f0 = u.f0;
    c.fstride = u.fstride;
    c.a0 = u.a0;
    c.a1 = u.a1;
}

// Slab f -> (i0, i1) with the plan's multiplier instead of a division (N = 4).
__device__ __forceinline__ void decode_f_fast(const Shape& s, const ContractPlan& pl, long long f, int& i0, int& i1) {
    const int fi = static_cast<int>(f);
    if (s.N == 4) {
        i0 = static_cast<int>((static_cast<unsigned long long>(static_cast<unsigned>(fi)) * pl.fdiv_m) >> pl.fdiv_s);
        i1 = fi - i0 * s.I[1];
    } else {
        i0 = fi;
        i1 = 0;
    }
}

__device__ __forceinline__ Task task_at(const UnitCur& c, int t, int rbk) {
    const int sidx = c.nrb == 1 ? t : t / c.nrb;
    const int rb = t - sidx * c.nrb;
    Task k;
    k.f = c.f0 + static_cast<long long>(sidx) * c.fstride;
    k.a0 = c.a0 + rb * rbk;
    k.na = min(rbk, c.a1 - k.a0);
    return k;
}

// ---------------------------------------------------------------------------
// ROW kind.  Fold modes:
//   CASE_F, N = 4: z_a(r2, rB) over the other F mode l2 with coefficient
//                  G_{l2,k}(r2, i_l2) W_{l2,A}(i_l2, a); G_{A,k} applied per
//                  unit (rows fixed per lane);
//   CASE_F, N = 3 (foldA): z(rA, rB) += G_{A,k}(rA, a) u_a(rB) directly;
//   CASE_A:        z_a(r2, rB) over l2 (N = 4: G_{1,k}(r2,i1) W_{0,1}(i0,i1);
//                  N = 3: G_{0,k}(r2, i0)); the row a is the output row.
// The few W entries a task needs besides its tile (the rows W_{p,B}(i_p, :)
// of the coefficient table, the fold weight) are loaded by the lanes that use
// them, one task ahead, into registers.
// ---------------------------------------------------------------------------

// RPL rows per lane (1, or 2 for tasks of up to 64 rows: twice the independent
// work per coefficient-table load and per task overhead); RCT the rank of the
// register fold when fixed at compile time (0: any, up to RMAX; the z
// registers are then sized for RMAX).
template <typename T, int RB, int RPL, int RCT, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_contract_roww(const __grid_constant__ ContractArgs<T> A) {
    pdl_begin();
    static_assert(RPL == 1 || RPL == 2, "one or two rows per lane");
    if (*A.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int VN = 16 / static_cast<int>(sizeof(T));
    constexpr int RBP = (RB + VN - 1) / VN * VN;
    constexpr int ZR = RCT > 0 ? RCT : RMAX;
    // two accumulator sets (shorter FMA chains) while registers allow; with two
    // rows per lane the rows are the independent chains
    constexpr bool SPLIT = RPL == 1 && RB <= 5;
    const Shape& s = A.sh;
    const ContractPlan& pl = A.pl;
    const int N = s.N, k = A.k, IA = s.IA, IB = s.IB, Am = N - 2, Bm = N - 1;
    const bool isF = pl.kcase == CASE_F;
    const bool foldA = isF && N == 3;
    const bool vec = pl.vec != 0;
    const int PS = vec ? RB : RBP;  // row stride of the coefficient table
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int S = pl.nstages, TC = pl.sub_elems;
    const int RBK = pl.TAc, LDX = pl.ldx, XR = pl.xr, ZW = pl.zw;
    const int l2 = pl.l2;
    const int RC = RCT > 0 ? RCT : (foldA ? pl.RA : pl.Rl2);
    // F modes p != k whose rows W_{p,B}(i_p, :) enter the coefficient table
    const int p0 = (N == 4) ? (k == 0 ? 1 : 0) : (N == 3 && k != 0 ? 0 : -1);
    const bool two_psi = N == 4 && k == 2;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    int* misc = reinterpret_cast<int*>(smem + MISC_OFF);  // [0] abort, [1 + w] z slot of warp w
    volatile int* abortf = misc;
    T* tiles = reinterpret_cast<T*>(smem + pl.off_tile);
    T* psi = reinterpret_cast<T*>(smem + pl.off_tab) + static_cast<size_t>(warp) * IB * PS;
    T* gtab = reinterpret_cast<T*>(smem + pl.off_gtab);
    T* wab = reinterpret_cast<T*>(smem + pl.off_wab);
    T* zs = reinterpret_cast<T*>(smem + pl.off_zs);
    const int nB = pl.R1 * IB;
    const int nL = l2 >= 0 ? pl.Rl2 * s.I[l2] : 0;
    const int nA = isF ? pl.RA * IA : 0;
    const T* gB = gtab;
    const T* gL = gtab + nB;
    const T* gA = gtab + nB + nL;

    if (tid == 0) {
        for (int i = 0; i < NW * S; ++i) mbar_init(&bars[i], 1);
        misc[0] = 0;
        fence_mbar_init();
    }
    stage_async(gtab, A.Gt + s.goff[Bm][k], nB);
    if (nL) stage_async(gtab + nB, A.Gt + s.goff[l2][k], nL);
    if (nA) stage_async(gtab + nB + nL, A.Gt + s.goff[Am][k], nA);
    stage_wait();

    // per-warp ring of the W entries each task needs besides its tile, filled
    // by cp.async at issue time and waited for with the stage.  Slot layout:
    // [0, IBP) the row W_{p0,B}(i_p0, :), [IBP, 2 IBP) the row W_{1,B}(i1, :)
    // (N = 4, k = 2), then the fold weights of the task's rows (32 RPL; b =
    // lane + 32 m and row = lane + 32 q are lane-owned).
    const int IBP = (IB + 31) & ~31;
    const int AUXW = pl.auxw;
    const int AUX_W1 = IBP, AUX_FW = two_psi ? 2 * IBP : IBP;
    T* auxr = reinterpret_cast<T*>(smem + pl.off_aux) + static_cast<size_t>(warp) * S * AUXW;

    // bases of the W rows a task needs (fixed for the launch), and the element
    // offsets of X and W_{A,B} within their 16-byte chunk, so that a task's
    // tile offset needs only 32-bit arithmetic (the offset mod VN is that of
    // the low 32 bits)
    const T* Wpsi0 = A.W + s.woff[p0 >= 0 ? p0 : 0][Bm];
    const T* Wpsi1 = A.W + s.woff[1][Bm];
    const T* Wfold = (isF && N == 4) ? A.W + s.woff[1 - k][Am] : A.W + s.woff[0][1];
    const unsigned xmis = static_cast<unsigned>(shift16(A.X));
    const unsigned wmis = static_cast<unsigned>(shift16(A.W + s.woff[Am][Bm]));
    auto tile_shift = [&](unsigned mis, long long f, int a0) {
        return static_cast<int>((mis + (static_cast<unsigned>(f) * static_cast<unsigned>(IA) + static_cast<unsigned>(a0)) *
                                           static_cast<unsigned>(IB)) &
                                static_cast<unsigned>(VN - 1));
    };

    // issue path: the task's rows of X (and, N = 3 k = 0, of W_{A,B}) by TMA
    // (lane 0), its W entries by every lane, one cp.async group per issue
    UnitCur ic = {};
    int ct = warp;
    auto settle = [&]() {
        while (ic.ui < pl.nunits && ct >= ic.nt) {
            ct = warp;
            const int nu = ic.ui + gridDim.x;
            if (nu < pl.nunits) load_unit(A.units, nu, RBK, ic);
            else ic.ui = nu;
        }
    };
    auto issue_next = [&](int st) {
        if (ic.ui >= pl.nunits) {
            cp_async_commit();  // empty group: keeps one group per stage
            return;
        }
        const Task tk = task_at(ic, ct, RBK);
        {
            int i0, i1;
            decode_f_fast(s, pl, tk.f, i0, i1);
            T* ax = auxr + st * AUXW;
            if (p0 >= 0) {
                const T* r = Wpsi0 + static_cast<long long>(p0 == 0 ? i0 : i1) * IB;
                for (int b = lane; b < IB; b += 32) cp_async_elem(ax + b, r + b);
            }
            if (two_psi) {
                const T* r = Wpsi1 + static_cast<long long>(i1) * IB;
                for (int b = lane; b < IB; b += 32) cp_async_elem(ax + AUX_W1 + b, r + b);
            }
            if (isF && N == 4) {
                const int io = k == 1 ? i0 : i1;  // the other F mode o = 1 - k
                const T* r = Wfold + static_cast<long long>(io) * IA + tk.a0 + lane;
#pragma unroll
                for (int q = 0; q < RPL; ++q)
                    if (lane + 32 * q < tk.na) cp_async_elem(ax + AUX_FW + 32 * q + lane, r + 32 * q);
            } else if (!isF && N == 4) {
                cp_async_elem(ax + AUX_FW + lane, Wfold + static_cast<long long>(i0) * s.I[1] + i1);
            }
            cp_async_commit();
        }
        if (lane == 0) {
            T* buf = tiles + (static_cast<size_t>(warp) * S + st) * TC;
            uint64_t* bar = &bars[warp * S + st];
            uintptr_t xlo, xhi, wlo = 0, whi = 0;
            range16(A.X + (tk.f * IA + tk.a0) * IB, static_cast<long long>(tk.na) * IB, xlo, xhi);
            if (foldA)
                range16(A.W + s.woff[Am][Bm] + static_cast<long long>(tk.a0) * IB, static_cast<long long>(tk.na) * IB,
                        wlo, whi);
            mbar_arrive_expect_tx(bar, static_cast<unsigned>((xhi - xlo) + (whi - wlo)));
            fence_proxy_async();
            bulk_g2s(buf, reinterpret_cast<const void*>(xlo), static_cast<unsigned>(xhi - xlo), bar);
            if (foldA) bulk_g2s(buf + XR, reinterpret_cast<const void*>(wlo), static_cast<unsigned>(whi - wlo), bar);
        }
        ct += NW;
        settle();
    };
    ic.ui = blockIdx.x;
    if (ic.ui < pl.nunits) load_unit(A.units, ic.ui, RBK, ic);
    settle();
    for (int i = 0; i < S; ++i) issue_next(i);

    int st = 0;        // ring stage of the next task this warp consumes
    unsigned par = 0;  // and the mbarrier phase parity it waits for
    for (int ui = blockIdx.x; ui < pl.nunits; ui += gridDim.x) {
        UnitCur uc;
        load_unit(A.units, ui, RBK, uc);
        const int nt = uc.nt;
        const int nru = uc.a1 - uc.a0;
        const UnitDesc u = A.units[ui];
        if (isF && !foldA) {  // W_{A,B} rows of the unit, padded to an odd number of 16-byte chunks
            for (int idx = tid; idx < nru * IB; idx += blockDim.x) {
                const int r = idx / IB, b = idx - r * IB;
                asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(wab + r * LDX + b)),
                             "l"(A.W + s.woff[Am][Bm] + static_cast<long long>(uc.a0 + r) * IB + b), "n"(sizeof(T))
                             : "memory");
            }
        }
        stage_wait();

        T z[RPL][ZR][RB];
#pragma unroll
        for (int q = 0; q < RPL; ++q)
#pragma unroll
            for (int r2 = 0; r2 < ZR; ++r2)
#pragma unroll
                for (int r = 0; r < RB; ++r) z[q][r2][r] = T(0);

        int zslot = -1;
        for (int t = warp; t < nt; t += NW) {
            T* buf = tiles + (static_cast<size_t>(warp) * S + st) * TC;
            const T* ax = auxr + st * AUXW;
            cp_async_wait_ring(S);  // this lane's W entries of the task
            const bool ok = warp_wait(&bars[warp * S + st], par, abortf, A.flags) && !*abortf;
            const Task tk = task_at(uc, t, RBK);
            if (ok) {
                int i0, i1;
                decode_f_fast(s, pl, tk.f, i0, i1);
                // coefficient table psi(b, r) = prod_{p in F, p != k} W_{p,B}(i_p, b) G_{B,k}(r, b)
                for (int b = lane; b < IB; b += 32) {
                    const T om = (p0 >= 0 ? ax[b] : T(1)) * (two_psi ? ax[AUX_W1 + b] : T(1));
#pragma unroll
                    for (int r = 0; r < RBP; ++r)
                        if (r < RB) psi[b * PS + r] = om * gB[r * IB + b];
                        else if (!vec) psi[b * PS + r] = T(0);
                }
                __syncwarp();
                bool va[RPL];
                const T* xr[RPL];
                const T* wr[RPL];
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    va[q] = lane + 32 * q < tk.na;
                    const int row = va[q] ? lane + 32 * q : 0;
                    xr[q] = buf + tile_shift(xmis, tk.f, tk.a0) + row * IB;
                    wr[q] = nullptr;
                    if (foldA) wr[q] = buf + XR + tile_shift(wmis, 0, tk.a0) + row * IB;
                    else if (isF)
                        wr[q] = wab + static_cast<size_t>(tk.a0 - uc.a0 + row) * LDX;
                }
                T u0[RPL][RB], u1[RPL][RB];
#pragma unroll
                for (int q = 0; q < RPL; ++q)
#pragma unroll
                    for (int r = 0; r < RB; ++r) u0[q][r] = u1[q][r] = T(0);
                if (vec) {
                    // one 16-byte chunk b..b+VN-1 of the lane's rows; with_w: the
                    // rows are multiplied by W_{A,B} first
                    auto chunk = [&](int b, auto with_w) {
                        T p[VN * RB];
                        ld_row<T, VN * RB>(psi + b * RB, p);
#pragma unroll
                        for (int q = 0; q < RPL; ++q) {
                            T xa[VN];
                            ld_row<T, VN>(xr[q] + b, xa);
                            if constexpr (decltype(with_w)::value) {
                                T wa[VN];
                                ld_row<T, VN>(wr[q] + b, wa);
#pragma unroll
                                for (int j = 0; j < VN; ++j) xa[j] *= wa[j];
                            }
#pragma unroll
                            for (int j = 0; j < VN; ++j)
#pragma unroll
                                for (int r = 0; r < RB; ++r) {
                                    if (SPLIT && (j & 1)) u1[q][r] = fma(xa[j], p[j * RB + r], u1[q][r]);
                                    else u0[q][r] = fma(xa[j], p[j * RB + r], u0[q][r]);
                                }
                        }
                    };
                    const bool hw = wr[0] != nullptr;  // the same for every row of the task
                    if (!pl.skew) {
                        if (hw) {
#pragma unroll 2
                            for (int b = 0; b < IB; b += VN) chunk(b, std::true_type{});
                        } else {
#pragma unroll 2
                            for (int b = 0; b < IB; b += VN) chunk(b, std::false_type{});
                        }
                    } else {
                        // each lane starts at its own chunk, so that rows that share
                        // banks are read apart
                        const int nch = IB / VN;
                        int c = lane % nch;
#pragma unroll 2
                        for (int ic2 = 0; ic2 < nch; ++ic2, c = (c + 1 == nch) ? 0 : c + 1) {
                            if (hw) chunk(c * VN, std::true_type{});
                            else chunk(c * VN, std::false_type{});
                        }
                    }
                } else {
#pragma unroll 4
                    for (int b = 0; b < IB; ++b) {
                        T p[RBP];
                        ld_row<T, RBP>(psi + b * RBP, p);
#pragma unroll
                        for (int q = 0; q < RPL; ++q) {
                            T xa = xr[q][b];
                            if (wr[q]) xa *= wr[q][b];
#pragma unroll
                            for (int r = 0; r < RB; ++r) {
                                if (SPLIT && (b & 1)) u1[q][r] = fma(xa, p[r], u1[q][r]);
                                else u0[q][r] = fma(xa, p[r], u0[q][r]);
                            }
                        }
                    }
                }
                if constexpr (SPLIT) {
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
#pragma unroll
                        for (int r = 0; r < RB; ++r) u0[q][r] += u1[q][r];
                }
                // fold the rows into z
                if (foldA) {
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        const T* ga = gA + tk.a0 + (va[q] ? lane + 32 * q : 0);
#pragma unroll
                        for (int r2 = 0; r2 < ZR; ++r2)
                            if (r2 < RC) {
                                const T c0 = va[q] ? ga[r2 * IA] : T(0);
#pragma unroll
                                for (int r = 0; r < RB; ++r) z[0][r2][r] = fma(c0, u0[q][r], z[0][r2][r]);
                            }
                    }
                } else if (l2 < 0) {
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
#pragma unroll
                        for (int r = 0; r < RB; ++r) z[q][0][r] += va[q] ? u0[q][r] : T(0);
                } else {
                    // coefficient G_{l2,k}(r2, i_l2) times the fold weight
                    const int il2 = isF ? (l2 == 0 ? i0 : i1) : (N == 4 ? i1 : i0);
                    const T* gl = gL + il2;
                    const int Il2 = s.I[l2];
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        const T sc = va[q] ? ((N == 4) ? ax[AUX_FW + (isF ? 32 * q : 0) + lane] : T(1)) : T(0);
#pragma unroll
                        for (int r2 = 0; r2 < ZR; ++r2)
                            if (r2 < RC) {
                                const T c0 = gl[r2 * Il2] * sc;
#pragma unroll
                                for (int r = 0; r < RB; ++r) z[q][r2][r] = fma(c0, u0[q][r], z[q][r2][r]);
                            }
                    }
                }
            }
            __syncwarp();
            if (t + NW < nt) {
                issue_next(st);  // the stage is free again
            } else {
                zslot = st;  // keeps z for the unit reduction; refilled after it
            }
            if (++st == S) {
                st = 0;
                par ^= 1u;
            }
        }
        // ---- unit end: reduce over warps (fixed order) ----
        const int nwk = min(NW, nt);
        if (zslot >= 0) {
            T* zb = tiles + (static_cast<size_t>(warp) * S + zslot) * TC;
            if (foldA) {
#pragma unroll
                for (int r2 = 0; r2 < ZR; ++r2)
                    if (r2 < RC)
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            const T v = warp_sum(z[0][r2][r]);
                            if (lane == 0) zb[r2 * RB + r] = v;
                        }
            } else {
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    const int row = lane + 32 * q;
                    if (row < nru) {
#pragma unroll
                        for (int r2 = 0; r2 < ZR; ++r2)
                            if (r2 < RC)
#pragma unroll
                                for (int r = 0; r < RB; ++r) zb[row * ZW + r2 * RB + r] = z[q][r2][r];
                    }
                }
            }
            if (lane == 0) misc[1 + warp] = zslot;
        }
        __syncthreads();
        auto zbuf = [&](int w) { return tiles + (static_cast<size_t>(w) * S + misc[1 + w]) * TC; };
        const bool aborted = *abortf != 0;  // uniform: no warp writes it between the two barriers
        if (!aborted) {
            if (foldA) {
                for (int q = tid; q < pl.Q; q += blockDim.x) {
                    T acc = T(0);
                    for (int w = 0; w < nwk; ++w) acc += zbuf(w)[q];
                    A.part[(static_cast<size_t>(u.key) * pl.nslot + u.slot) * pl.Q + q] = acc;
                }
            } else if (isF) {
                for (int idx = tid; idx < nru * ZW; idx += blockDim.x) {
                    T acc = T(0);
                    for (int w = 0; w < nwk; ++w) acc += zbuf(w)[idx];
                    zs[idx] = acc;
                }
                __syncthreads();
                const int RA = pl.RA;
                for (int q = tid; q < pl.Q; q += blockDim.x) {
                    const int r2 = q / (RA * RB), rem = q - r2 * RA * RB;
                    const int rA = rem / RB, rB = rem - rA * RB;
                    T acc = T(0);
                    for (int row = 0; row < nru; ++row)
                        acc = fma(gA[rA * IA + uc.a0 + row], zs[row * ZW + r2 * RB + rB], acc);
                    A.part[(static_cast<size_t>(u.key) * pl.nslot + u.slot) * pl.Q + q] = acc;
                }
            } else {
                for (int idx = tid; idx < nru * ZW; idx += blockDim.x) {
                    const int row = idx / ZW, q = idx - row * ZW;
                    T acc = T(0);
                    for (int w = 0; w < nwk; ++w) acc += zbuf(w)[idx];
                    A.part[(static_cast<size_t>(ui) * IA + uc.a0 + row) * pl.Qp + q] = acc;
                }
            }
        }
        __syncthreads();
        if (zslot >= 0) issue_next(zslot);
    }
}

// ---------------------------------------------------------------------------
// COL kind (k = N-1): lane = column b of the unit's 32-column chunk; level 1
// over rows a against phi(a, r) = prod_{p in F} W_{p,A}(i_p, a) G_{A,k}(r, a)
// (built per task, lane = row); fold per task over l2 (N = 4:
// G_{1,k}(r2, i1) W_{0,1}(i0, i1), i0 deferred to the finisher; N = 3:
// G_{0,k}(r2, i0)).
// ---------------------------------------------------------------------------

template <typename T, int RA, int RPL, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_contract_colw(const __grid_constant__ ContractArgs<T> A) {
    pdl_begin();
    if (*A.done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int VN = 16 / static_cast<int>(sizeof(T));
    constexpr bool SPLIT = RA <= 5;
    const Shape& s = A.sh;
    const ContractPlan& pl = A.pl;
    const int N = s.N, k = A.k, IA = s.IA, IB = s.IB, Am = N - 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const int S = pl.nstages, TC = pl.sub_elems;
    const int RBK = pl.TAc, ZW = pl.zw;
    const int l2 = pl.l2;
    const int RC = pl.Rl2;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    int* misc = reinterpret_cast<int*>(smem + MISC_OFF);
    volatile int* abortf = misc;
    T* tiles = reinterpret_cast<T*>(smem + pl.off_tile);
    // phi rows of a task (up to 32 RPL, lane-owned: a = lane + 32 q), RA values
    // each, plus VN zero rows of padding
    constexpr int PR = 32 * RPL;
    T* phi = reinterpret_cast<T*>(smem + pl.off_tab) + static_cast<size_t>(warp) * (PR + VN) * RA;
    T* gtab = reinterpret_cast<T*>(smem + pl.off_gtab);
    const int nAg = pl.R1 * IA;
    const int nL = l2 >= 0 ? RC * s.I[l2] : 0;
    const T* gAt = gtab;
    const T* gL = gtab + nAg;
    // per-warp ring of the W entries of a task (phi row weights W_{0,A}(i0, a)
    // at [0, PR) and W_{1,A}(i1, a) at [PR, 2 PR), a = lane + 32 q; W_{0,1}(i0,
    // i1) at [2 PR, 2 PR + 32)), filled by cp.async at issue time
    const int AUXW = pl.auxw;
    T* auxr = reinterpret_cast<T*>(smem + pl.off_aux) + static_cast<size_t>(warp) * S * AUXW;

    if (tid == 0) {
        for (int i = 0; i < NW * S; ++i) mbar_init(&bars[i], 1);
        misc[0] = 0;
        fence_mbar_init();
    }
    stage_async(gtab, A.Gt + s.goff[Am][k], nAg);
    if (nL) stage_async(gtab + nAg, A.Gt + s.goff[l2][k], nL);
    stage_wait();

    UnitCur ic = {};
    int ct = warp;
    auto settle = [&]() {
        while (ic.ui < pl.nunits && ct >= ic.nt) {
            ct = warp;
            const int nu = ic.ui + gridDim.x;
            if (nu < pl.nunits) load_unit(A.units, nu, RBK, ic);
            else ic.ui = nu;
        }
    };
    auto issue_next = [&](int st) {
        if (ic.ui >= pl.nunits) {
            cp_async_commit();
            return;
        }
        const Task tk = task_at(ic, ct, RBK);
        {
            int i0, i1;
            decode_f_fast(s, pl, tk.f, i0, i1);
            T* ax = auxr + st * AUXW;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int a = lane + 32 * q;
                if (a < tk.na) {
                    if (N >= 3) cp_async_elem(ax + a, A.W + s.woff[0][Am] + static_cast<long long>(i0) * IA + tk.a0 + a);
                    if (N == 4)
                        cp_async_elem(ax + PR + a, A.W + s.woff[1][Am] + static_cast<long long>(i1) * IA + tk.a0 + a);
                }
            }
            if (N == 4) cp_async_elem(ax + 2 * PR + lane, A.W + s.woff[0][1] + static_cast<long long>(i0) * s.I[1] + i1);
            cp_async_commit();
        }
        if (lane == 0) {
            T* buf = tiles + (static_cast<size_t>(warp) * S + st) * TC;
            uint64_t* bar = &bars[warp * S + st];
            uintptr_t lo, hi;
            range16(A.X + (tk.f * IA + tk.a0) * IB, static_cast<long long>(tk.na) * IB, lo, hi);
            mbar_arrive_expect_tx(bar, static_cast<unsigned>(hi - lo));
            fence_proxy_async();
            bulk_g2s(buf, reinterpret_cast<const void*>(lo), static_cast<unsigned>(hi - lo), bar);
        }
        ct += NW;
        settle();
    };
    ic.ui = blockIdx.x;
    if (ic.ui < pl.nunits) load_unit(A.units, ic.ui, RBK, ic);
    settle();
    for (int i = 0; i < S; ++i) issue_next(i);

    int st = 0;        // ring stage of the next task this warp consumes
    unsigned par = 0;  // and the mbarrier phase parity it waits for
    for (int ui = blockIdx.x; ui < pl.nunits; ui += gridDim.x) {
        UnitCur uc;
        load_unit(A.units, ui, RBK, uc);
        const UnitDesc u = A.units[ui];
        const int nt = uc.nt;
        const int nb = u.b1 - u.b0;
        const bool colok = lane < nb;
        T z[RMAX][RA];
#pragma unroll
        for (int r2 = 0; r2 < RMAX; ++r2)
#pragma unroll
            for (int r = 0; r < RA; ++r) z[r2][r] = T(0);
        int zslot = -1;
        for (int t = warp; t < nt; t += NW) {
            T* buf = tiles + (static_cast<size_t>(warp) * S + st) * TC;
            const T* ax = auxr + st * AUXW;
            cp_async_wait_ring(S);
            const bool ok = warp_wait(&bars[warp * S + st], par, abortf, A.flags) && !*abortf;
            const Task tk = task_at(uc, t, RBK);
            if (ok) {
                int i0, i1;
                decode_f_fast(s, pl, tk.f, i0, i1);
                // phi rows (lane-owned rows a = lane + 32 q); rows past na are zero
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    const int a = lane + 32 * q;
                    const T om = (a < tk.na) ? (N >= 3 ? ax[a] : T(1)) * (N == 4 ? ax[PR + a] : T(1)) : T(0);
#pragma unroll
                    for (int r = 0; r < RA; ++r)
                        phi[a * RA + r] = a < tk.na ? om * gAt[r * IA + tk.a0 + a] : T(0);
                }
                if (lane < VN) {  // padding rows PR.. of the last chunk
#pragma unroll
                    for (int r = 0; r < RA; ++r) phi[(PR + lane) * RA + r] = T(0);
                }
                __syncwarp();
                const T* xt = buf + shift16(A.X + (tk.f * IA + tk.a0) * IB) + u.b0 + (colok ? lane : 0);
                T u0[RA], u1[RA];
#pragma unroll
                for (int r = 0; r < RA; ++r) u0[r] = u1[r] = T(0);
                // whole chunks of VN rows, then the ragged last one, whose rows
                // past na read row na - 1 (their phi rows are zero)
                const int nfull = tk.na / VN * VN;
                const T* xa = xt;
                for (int a = 0; a < nfull; a += VN, xa += static_cast<size_t>(VN) * IB) {
                    T p[VN * RA];
                    ld_row<T, VN * RA>(phi + a * RA, p);
#pragma unroll
                    for (int j = 0; j < VN; ++j) {
                        const T x = xa[static_cast<size_t>(j) * IB];
#pragma unroll
                        for (int r = 0; r < RA; ++r) {
                            if (SPLIT && (j & 1)) u1[r] = fma(x, p[j * RA + r], u1[r]);
                            else u0[r] = fma(x, p[j * RA + r], u0[r]);
                        }
                    }
                }
                if (nfull < tk.na) {
                    const int a = nfull;
                    T p[VN * RA];
                    ld_row<T, VN * RA>(phi + a * RA, p);
#pragma unroll
                    for (int j = 0; j < VN; ++j) {
                        const int ar = min(a + j, tk.na - 1);
                        const T x = xt[static_cast<size_t>(ar) * IB];
#pragma unroll
                        for (int r = 0; r < RA; ++r) {
                            if (SPLIT && (j & 1)) u1[r] = fma(x, p[j * RA + r], u1[r]);
                            else u0[r] = fma(x, p[j * RA + r], u0[r]);
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < RA; ++r) u0[r] += u1[r];
                if (l2 < 0) {
#pragma unroll
                    for (int r = 0; r < RA; ++r) z[0][r] += colok ? u0[r] : T(0);
                } else {
                    const T scale = colok ? (N == 4 ? ax[2 * PR + lane] : T(1)) : T(0);
                    const int il2 = N == 4 ? i1 : i0;
                    const T* gl = gL + il2;
                    const int Il2 = s.I[l2];
#pragma unroll
                    for (int r2 = 0; r2 < RMAX; ++r2)
                        if (r2 < RC) {
                            const T cf = gl[r2 * Il2] * scale;
#pragma unroll
                            for (int r = 0; r < RA; ++r) z[r2][r] = fma(cf, u0[r], z[r2][r]);
                        }
                }
            }
            __syncwarp();
            if (t + NW < nt)
                issue_next(st);
            else
                zslot = st;
            if (++st == S) {
                st = 0;
                par ^= 1u;
            }
        }
        const int nwk = min(NW, nt);
        if (zslot >= 0) {
            T* zb = tiles + (static_cast<size_t>(warp) * S + zslot) * TC;
            if (colok)
#pragma unroll
                for (int r2 = 0; r2 < RMAX; ++r2)
                    if (r2 < RC)
#pragma unroll
                        for (int r = 0; r < RA; ++r) zb[lane * ZW + r2 * RA + r] = z[r2][r];
            if (lane == 0) misc[1 + warp] = zslot;
        }
        __syncthreads();
        const bool aborted = *abortf != 0;
        if (!aborted) {
            for (int idx = tid; idx < nb * ZW; idx += blockDim.x) {
                const int col = idx / ZW, q = idx - col * ZW;
                T acc = T(0);
                for (int w = 0; w < nwk; ++w) acc += (tiles + (static_cast<size_t>(w) * S + misc[1 + w]) * TC)[idx];
                A.part[(static_cast<size_t>(ui) * IB + u.b0 + col) * pl.Qp + q] = acc;
            }
        }
        __syncthreads();
        if (zslot >= 0) issue_next(zslot);
    }
}

template <typename T, int R, int RPL = 1, int RCT = 0, int NW = NWARP>
cudaError_t launch_roww_r(const ContractArgs<T>& a, int grid, cudaStream_t st) {
    auto kern = k_contract_roww<T, R, RPL, RCT, NW>;
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), a.pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NW * 32, a.pl.smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int R, int RPL = 1, int NW = NWARP>
cudaError_t launch_colw_r(const ContractArgs<T>& a, int grid, cudaStream_t st) {
    auto kern = k_contract_colw<T, R, RPL, NW>;
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), a.pl.smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NW * 32, a.pl.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wdev

template <typename T>
cudaError_t launch_contract_warp(const ContractArgs<T>& a, int grid, cudaStream_t st) {
    const bool col = a.pl.kcase == CASE_COL;
    // the plan's warps per CTA must be those of the instantiation it selects
    const int nw_want = a.pl.rpl == 2 ? (col ? 12 : wdev::NWARP) : (a.pl.nwarp == 8 ? 8 : wdev::NWARP);
    if (a.pl.nwarp != nw_want) return cudaErrorInvalidValue;
    if (!col && a.pl.rpl == 2) {  // two rows per lane: instantiated for equal ranks R_{k,B} = R_{k,l2}
        switch (a.pl.R1) {
            case 2: return wdev::launch_roww_r<T, 2, 2, 2>(a, grid, st);
            case 3: return wdev::launch_roww_r<T, 3, 2, 3>(a, grid, st);
            case 4: return wdev::launch_roww_r<T, 4, 2, 4>(a, grid, st);
            case 5: return wdev::launch_roww_r<T, 5, 2, 5>(a, grid, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (col && a.pl.rpl == 2) {  // tasks of up to 64 rows: 12 warps (their rings fit shared memory)
        switch (a.pl.R1) {
#define IFCTN_CASE(R) \
    case R:           \
        return wdev::launch_colw_r<T, R, 2, 12>(a, grid, st);
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
    if (a.pl.nwarp == 8) {  // long rows: 8 warps, each with twice the shared memory of the 16-warp plan
        switch (a.pl.R1) {
#define IFCTN_CASE(R) \
    case R:           \
        return col ? wdev::launch_colw_r<T, R, 1, 8>(a, grid, st) : wdev::launch_roww_r<T, R, 1, 0, 8>(a, grid, st);
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
    switch (a.pl.R1) {
#define IFCTN_CASE(R) \
    case R:           \
        return col ? wdev::launch_colw_r<T, R>(a, grid, st) : wdev::launch_roww_r<T, R>(a, grid, st);
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

}  // namespace ifctn
