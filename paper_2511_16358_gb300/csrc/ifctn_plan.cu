// ifctn_plan.cu -- host-side checks and launch planning: the validated shape
// of a problem (sizes, ranks, packed offsets) and the work units and
// shared-memory carve-up of every mode's streaming contraction (M_k = X_(k) Z_k,
// Prop. 1), for the CTA kernels of the persistent path and the warp-pipelined
// kernels of the sweep graph.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ifctn_api_internal.h"
#include "ifctn_plan.h"

namespace ifctn {

namespace {

constexpr int STAGE_BYTES = 32 * 1024;
constexpr int NSTAGES = 3;

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Split [0, len) into n nearly equal chunks; returns chunk c's [lo, hi).
inline void chunk(int len, int n, int c, int& lo, int& hi) {
    lo = static_cast<int>(static_cast<long long>(len) * c / n);
    hi = static_cast<int>(static_cast<long long>(len) * (c + 1) / n);
}

}  // namespace

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

ifctn_status build_shape(const ifctn_problem* p, Shape& s) {
    if (!p) {
        set_error("null problem");
        return IFCTN_EINVAL;
    }
    memset(&s, 0, sizeof(s));
    s.N = p->order;
    if (s.N < 2 || s.N > 4) {
        set_error("order must be 2..4");
        return IFCTN_EINVAL;
    }
    // Every size the kernels index with 32-bit integers (I_k, the slab count,
    // the packed factor and pair-matrix arrays) must stay below 2^31, and the
    // entry count below 2^40 (far beyond device memory), so that no product
    // below overflows.
    constexpr long long MAX_ENTRIES = 1LL << 40;
    s.P = 1;
    for (int k = 0; k < s.N; ++k) {
        if (p->dims[k] < 1 || p->dims[k] > (1 << 30)) {
            set_error("dims must be in 1..2^30");
            return IFCTN_EINVAL;
        }
        s.I[k] = static_cast<int>(p->dims[k]);
        s.P *= p->dims[k];
        if (s.P > MAX_ENTRIES) {
            set_error("tensor has more than 2^40 entries");
            return IFCTN_EINVAL;
        }
    }
    // Edge ranks up to RMAX for every order; order-3 tensors also take ranks
    // up to WIDE_RMAX with every Q_k <= WIDE_QMAX (the kernels of ifctn_wide.cu).
    const int rmax = s.N == 3 ? WIDE_RMAX : RMAX;
    for (int k = 0; k < s.N; ++k)
        for (int l = 0; l < s.N; ++l) {
            if (k == l) continue;
            const int r = p->ranks[k * 4 + l];
            if (r < 1 || r > rmax || r != p->ranks[l * 4 + k]) {
                set_error(s.N == 3 ? "ranks must be symmetric and in 1..64" : "ranks must be symmetric and in 1..8");
                return IFCTN_EINVAL;
            }
            s.R[k][l] = r;
            if (r > RMAX) s.wide = 1;
        }
    if (s.wide)
        for (int k = 0; k < s.N; ++k) {
            long long q = 1;
            for (int l = 0; l < s.N; ++l)
                if (l != k) q *= s.R[k][l];
            if (q > WIDE_QMAX) {
                set_error("with ranks above 8, every Q_k (product of a mode's edge ranks) must be <= 4096");
                return IFCTN_EINVAL;
            }
        }
    if (!(p->rho > 0.0) || !std::isfinite(p->rho)) {
        set_error("rho must be > 0");
        return IFCTN_EINVAL;
    }
    if (p->max_sweeps < 0 || p->tol < 0) {
        set_error("max_sweeps and tol must be >= 0");
        return IFCTN_EINVAL;
    }
    if (p->precision != IFCTN_FP64 && p->precision != IFCTN_MIXED) {
        set_error("unknown precision");
        return IFCTN_EINVAL;
    }
    long long off = 0;
    for (int k = 0; k < s.N; ++k)
        for (int l = 0; l < s.N; ++l) {
            if (k == l) continue;
            s.goff[k][l] = static_cast<int>(off);
            off += static_cast<long long>(s.R[k][l]) * s.I[k];
            if (off > INT_MAX) {
                set_error("packed factor array has 2^31 or more entries");
                return IFCTN_EINVAL;
            }
        }
    s.gsize = static_cast<int>(off);
    off = 0;
    for (int p2 = 0; p2 < s.N; ++p2)
        for (int q = p2 + 1; q < s.N; ++q) {
            s.woff[p2][q] = static_cast<int>(off);
            off += static_cast<long long>(s.I[p2]) * s.I[q];
            if (off > INT_MAX) {
                set_error("pair matrices have 2^31 or more entries");
                return IFCTN_EINVAL;
            }
        }
    s.wsize = static_cast<int>(off);
    s.IA = s.I[s.N - 2];
    s.IB = s.I[s.N - 1];
    long long nf = 1;
    for (int m = 0; m < s.N - 2; ++m) nf *= s.I[m];
    if (nf > INT_MAX) {
        set_error("more than 2^31 - 1 slabs (product of all but the last two sizes)");
        return IFCTN_EINVAL;
    }
    s.nF = static_cast<int>(nf);
    return IFCTN_OK;
}

int mode_q(const Shape& s, int k) {
    int q = 1;
    for (int m = 0; m < s.N; ++m)
        if (m != k) q *= s.R[k][m];
    return q;
}

// Launch geometry of the mode-k contraction and its work units.

// Largest number of pipeline stages any unit of the plan consumes.
static int max_unit_stages(const ContractPlan& pl, const std::vector<UnitDesc>& units) {
    int mx = 1;
    const int GS = pl.split ? 1 : pl.G;
    for (const UnitDesc& u : units) {
        const int nb = (u.ns + GS - 1) / GS;
        int n = 1;
        if (pl.kcase == CASE_COL)
            n = nb * ((u.a1 - u.a0 + pl.TAc - 1) / pl.TAc);
        else
            n = nb * ((u.a1 - u.a0 + pl.TA - 1) / pl.TA);
        mx = std::max(mx, n);
    }
    return mx;
}

ContractPlan plan_contract(const Shape& s, int k, int sz, std::vector<UnitDesc>& units) {
    ContractPlan pl;
    memset(&pl, 0, sizeof(pl));
    const int N = s.N, Am = N - 2, Bm = N - 1, IA = s.IA, IB = s.IB;
    const int target = 4 * num_sms();
    pl.Q = mode_q(s, k);
    pl.nstages = NSTAGES;
    units.clear();
    auto add = [&](int f0, int fstride, int ns, int key, int a0, int a1, int b0, int b1, int slot) {
        UnitDesc u;
        memset(&u, 0, sizeof(u));
        u.f0 = f0;
        u.fstride = fstride;
        u.ns = ns;
        u.key = key;
        u.a0 = a0;
        u.a1 = a1;
        u.b0 = b0;
        u.b1 = b1;
        u.slot = slot;
        units.push_back(u);
    };
    if (k == Bm) {  // COL
        pl.kcase = CASE_COL;
        pl.R1 = s.R[k][Am];
        const bool slab3 = N == 3 && s.P * sz <= L2_RESIDENT_BYTES;
        if (N == 4) {
            pl.l2 = 1;
            pl.dmode = 0;
        } else if (N == 3 && !slab3) {
            pl.l2 = 0;
            pl.dmode = -1;
        } else if (N == 3) {
            pl.l2 = -1;
            pl.dmode = 0;
        } else {
            pl.l2 = -1;
            pl.dmode = -1;
        }
        pl.Rl2 = pl.l2 >= 0 ? s.R[k][pl.l2] : 1;
        pl.Qp = pl.Rl2 * pl.R1;
        const int TB = std::min(IB, 256);
        const int nbch = cdiv(IB, TB);
        const int gmax = std::max(1, 256 / TB);
        int maxns = 1;
        if (N == 4) {
            const int I0 = s.I[0], I1 = s.I[1];
            const int nsmin = gmax;
            int nC = std::max(1, std::min(cdiv(target, static_cast<long long>(I0) * nbch), std::max(1, I1 / nsmin)));
            for (int i0 = 0; i0 < I0; ++i0)
                for (int c = 0; c < nC; ++c)
                    for (int bc = 0; bc < nbch; ++bc) {
                        int lo, hi, b0, b1;
                        chunk(I1, nC, c, lo, hi);
                        chunk(IB, nbch, bc, b0, b1);
                        add(i0 * I1 + lo, 1, hi - lo, i0, 0, IA, b0, b1, 0);
                        maxns = std::max(maxns, hi - lo);
                    }
        } else if (N == 3 && slab3) {
            for (int i0 = 0; i0 < s.I[0]; ++i0)
                for (int bc = 0; bc < nbch; ++bc) {
                    int b0, b1;
                    chunk(IB, nbch, bc, b0, b1);
                    add(i0, 1, 1, i0, 0, IA, b0, b1, 0);
                }
        } else if (N == 3) {
            const int I0 = s.I[0];
            const int nsmin = std::max(gmax, cdiv(4LL * pl.Qp, IA));
            int nC = std::max(1, std::min(cdiv(target, nbch), std::max(1, I0 / nsmin)));
            for (int c = 0; c < nC; ++c)
                for (int bc = 0; bc < nbch; ++bc) {
                    int lo, hi, b0, b1;
                    chunk(I0, nC, c, lo, hi);
                    chunk(IB, nbch, bc, b0, b1);
                    add(lo, 1, hi - lo, -1, 0, IA, b0, b1, 0);
                    maxns = std::max(maxns, hi - lo);
                }
        } else {
            const int nAC = std::max(1, std::min(cdiv(target, nbch), cdiv(IA, 64)));
            for (int ac = 0; ac < nAC; ++ac)
                for (int bc = 0; bc < nbch; ++bc) {
                    int a0, a1, b0, b1;
                    chunk(IA, nAC, ac, a0, a1);
                    chunk(IB, nbch, bc, b0, b1);
                    add(0, 1, 1, -1, a0, a1, b0, b1, 0);
                }
        }
        // a unit with a single slab and no register fold: the groups split its rows
        pl.split = (maxns == 1 && pl.l2 < 0) ? 1 : 0;
        int G = pl.split ? std::max(1, std::min(gmax, IA / 4)) : std::max(1, std::min(gmax, maxns));
        {  // the unit's G_{A,k} and G_{l2,k} tables, staged in shared memory when small
            const long long ge = static_cast<long long>(pl.R1) * IA + (pl.l2 >= 0 ? pl.Rl2 * s.I[pl.l2] : 0);
            pl.gtab_smem = ge * sz <= 48 * 1024 ? 1 : 0;
            pl.gtab_elems = pl.gtab_smem ? static_cast<int>(ge) : 0;
        }
        for (;;) {
            const int GS = pl.split ? 1 : G;
            int TAc = std::max(1, std::min(IA, STAGE_BYTES / (GS * IB * sz)));
            const int nthr = 256;
            const int SL = round_up(TAc + 32 / sz, 16 / sz);
            const int sub = round_up(TAc * IB + 32 / sz, 16 / sz) + 3 * SL;
            const long long smem = 128 + static_cast<long long>(NSTAGES) * GS * sub * sz +
                                   static_cast<long long>(GS) * TAc * (pl.R1 | 1) * sz +
                                   static_cast<long long>(nthr) * pl.Qp * sz +
                                   static_cast<long long>(pl.gtab_elems) * sz;
            pl.aux_slot = SL;
            if (smem <= SMEM_LIMIT || G == 1) {
                pl.TA = TB;
                pl.TAc = TAc;
                pl.G = G;
                pl.nthreads = nthr;
                pl.sub_elems = sub;
                pl.smem = static_cast<int>(smem);
                break;
            }
            --G;
        }
        {
            const int need = std::min(NSTAGES, max_unit_stages(pl, units));
            if (need < NSTAGES) {
                const int GS = pl.split ? 1 : pl.G;
                pl.smem -= (NSTAGES - need) * GS * pl.sub_elems * sz;
                pl.nstages = need;
            }
        }
        pl.nrow = IB;
        pl.nunits = static_cast<int>(units.size());
        pl.part_elems = static_cast<long long>(pl.nunits) * IB * pl.Qp;
        pl.key_div = 0;
        if (nbch == 1 && N >= 3) {
            if (N == 3 && slab3) pl.key_div = 1;
            else if (N == 4) pl.key_div = static_cast<int>(units.size()) / s.I[0];
            else pl.key_div = 1 << 30;  // no deferral: any positive value
        }
        return pl;
    }
    // ROW kinds
    pl.R1 = s.R[k][Bm];
    const bool isF = k < Am;
    pl.kcase = isF ? CASE_F : CASE_A;
    if (isF) {
        pl.RA = s.R[k][Am];
        pl.dmode = -1;
        if (N == 4) {
            pl.l2 = 1 - k;
            pl.Rl2 = s.R[k][pl.l2];
        } else {
            pl.l2 = -1;
            pl.Rl2 = 1;
        }
        pl.Qp = pl.Q;
    } else {
        if (N == 4) {
            pl.l2 = 1;
            pl.dmode = 0;
        } else if (N == 3 && s.P * sz <= L2_RESIDENT_BYTES) {
            pl.l2 = -1;
            pl.dmode = 0;
        } else if (N == 3) {
            pl.l2 = 0;
            pl.dmode = -1;
        } else {
            pl.l2 = -1;
            pl.dmode = -1;
        }
        pl.Rl2 = pl.l2 >= 0 ? s.R[k][pl.l2] : 1;
        pl.Qp = pl.Rl2 * pl.R1;
    }
    const int rows_cap = std::max(1, STAGE_BYTES / (IB * sz));
    const int TA = std::min(std::min(IA, rows_cap), 256);
    const int gmax = std::max(1, std::min(256 / TA, STAGE_BYTES / (TA * IB * sz)));
    int maxns = 1;
    if (isF && N == 4) {
        const int o = 1 - k, Io = s.I[o], Ik = s.I[k], I1 = s.I[1];
        int nOC = std::max(1, std::min(cdiv(target, Ik), std::max(1, Io / gmax)));
        for (int j = 0; j < Ik; ++j)
            for (int oc = 0; oc < nOC; ++oc) {
                int lo, hi;
                chunk(Io, nOC, oc, lo, hi);
                if (k == 0)
                    add(j * I1 + lo, 1, hi - lo, j, 0, IA, 0, IB, oc);
                else
                    add(lo * I1 + j, I1, hi - lo, j, 0, IA, 0, IB, oc);
                maxns = std::max(maxns, hi - lo);
            }
        pl.nslot = nOC;
        pl.part_elems = static_cast<long long>(Ik) * nOC * pl.Q;
    } else if (isF) {  // N = 3, k = 0: one slab per output row
        for (int j = 0; j < s.I[0]; ++j) add(j, 1, 1, j, 0, IA, 0, IB, 0);
        pl.nslot = 1;
        pl.part_elems = static_cast<long long>(s.I[0]) * pl.Q;
    } else if (N == 4) {
        const int I0 = s.I[0], I1 = s.I[1];
        const int nsmin = std::max(gmax, cdiv(4LL * pl.Qp, IB));
        int nC = std::max(1, std::min(cdiv(target, I0), std::max(1, I1 / nsmin)));
        for (int i0 = 0; i0 < I0; ++i0)
            for (int c = 0; c < nC; ++c) {
                int lo, hi;
                chunk(I1, nC, c, lo, hi);
                add(i0 * I1 + lo, 1, hi - lo, i0, 0, IA, 0, IB, 0);
                maxns = std::max(maxns, hi - lo);
            }
    } else if (N == 3 && pl.dmode == 0) {
        for (int i0 = 0; i0 < s.I[0]; ++i0) add(i0, 1, 1, i0, 0, IA, 0, IB, 0);
    } else if (N == 3) {
        const int I0 = s.I[0];
        const int nsmin = std::max(gmax, cdiv(4LL * pl.Qp, IB));
        int nC = std::max(1, std::min(target, std::max(1, I0 / nsmin)));
        for (int c = 0; c < nC; ++c) {
            int lo, hi;
            chunk(I0, nC, c, lo, hi);
            add(lo, 1, hi - lo, -1, 0, IA, 0, IB, 0);
            maxns = std::max(maxns, hi - lo);
        }
    } else {  // N = 2: one slab, split into row chunks of TA
        const int nAC = cdiv(IA, TA);
        for (int ac = 0; ac < nAC; ++ac) {
            int a0 = ac * TA, a1 = std::min(IA, a0 + TA);
            add(0, 1, 1, -1, a0, a1, 0, IB, 0);
        }
    }
    if (!isF) pl.part_elems = static_cast<long long>(units.size()) * IA * pl.Qp;
    // a unit with a single slab and no register fold: the groups split its columns
    pl.split = (maxns == 1 && pl.Rl2 == 1 && (pl.l2 < 0 || isF)) ? 1 : 0;
    int G = pl.split ? std::max(1, std::min(std::max(1, 256 / TA), IB / 4)) : std::max(1, std::min(gmax, maxns));
    {  // the unit's G_{B,k}, G_{l2,k} and (CASE_F) G_{A,k} tables
        const long long ge = static_cast<long long>(pl.R1) * IB + (pl.l2 >= 0 ? pl.Rl2 * s.I[pl.l2] : 0) +
                             (isF ? static_cast<long long>(pl.RA) * IA : 0);
        pl.gtab_smem = ge * sz <= 48 * 1024 ? 1 : 0;
        pl.gtab_elems = pl.gtab_smem ? static_cast<int>(ge) : 0;
    }
    for (;;) {
        const int GS = pl.split ? 1 : G;
        const int nthr = 256;
        const int nwarp = nthr / 32;
        const int SL = round_up(std::max(IB, TA) + 32 / sz, 16 / sz);
        const int sub = round_up(TA * IB + 32 / sz, 16 / sz) + 3 * SL;
        pl.aux_slot = SL;
        long long smem = 128 + static_cast<long long>(NSTAGES) * GS * sub * sz +
                         static_cast<long long>(GS) * IB * (pl.R1 | 1) * sz +
                         static_cast<long long>(pl.gtab_elems) * sz;
        if (isF)
            smem += static_cast<long long>(TA) * IB * sz + static_cast<long long>(nwarp + 1) * pl.Q * sz;
        else
            smem += static_cast<long long>(nthr) * pl.Qp * sz;
        if (smem <= SMEM_LIMIT || G == 1) {
            pl.TA = TA;
            pl.G = G;
            pl.nthreads = nthr;
            pl.sub_elems = sub;
            pl.smem = static_cast<int>(smem);
            break;
        }
        --G;
    }
    pl.skew = (IB % 2 == 0) ? 1 : 0;
    {
        const int need = std::min(NSTAGES, max_unit_stages(pl, units));
        if (need < NSTAGES) {
            const int GS = pl.split ? 1 : pl.G;
            pl.smem -= (NSTAGES - need) * GS * pl.sub_elems * sz;
            pl.nstages = need;
        }
    }
    pl.nrow = IA;
    pl.nunits = static_cast<int>(units.size());
    pl.key_div = 0;
    if (!isF && N >= 3) {
        if (N == 3 && pl.dmode == 0) pl.key_div = 1;
        else if (N == 4) pl.key_div = static_cast<int>(units.size()) / s.I[0];
        else pl.key_div = 1 << 30;
    }
    return pl;
}


// Plan of the warp-pipelined kernels (one CTA of 8 warps per SM, a TMA ring
// per warp).  Returns warp = 0 when the shape does not fit their shared-memory
// layout; the CTA kernels then run the mode.
// Chunk count for splitting S slabs (t tasks each) into the units of a
// warp-pipelined contraction, `outer` units per chunk.  A unit ends in a CTA
// barrier, so its tasks should split evenly over the NW warps, and the
// units evenly over the SMs.  Cost model, in task times: the most units a
// CTA runs times (tasks a warp runs per unit + per-unit overhead E).  The
// candidates are c0 (the balance-driven default) and every divisor c of S
// whose units give each warp the same number of tasks; the default is left
// only for a predicted gain above 3 %.
int warp_unit_chunks(int S, int t, long long outer, int c0, int NW, int sms) {
    constexpr double E = 0.4;
    auto cost = [&](int c) {
        const long long nu = outer * c;
        const long long per_cta = (nu + sms - 1) / sms;
        const long long tasks = static_cast<long long>((S + c - 1) / c) * t;
        return static_cast<double>(per_cta) * (static_cast<double>((tasks + NW - 1) / NW) + E);
    };
    int best = c0;
    double bc = cost(c0);
    for (int c = 1; c <= S; ++c) {
        if (S % c != 0 || (static_cast<long long>(S / c) * t) % NW != 0) continue;
        if (outer * c > 64LL * sms) break;
        const double v = cost(c);
        if (v < bc && v < 0.97 * cost(c0)) {  // leave the default only for a clear gain
            bc = v;
            best = c;
        }
    }
    return best;
}

// IFCTN_CW_RPL=1 keeps the warp contraction at one row per lane (timing and
// tuning); otherwise two rows per lane are used where the plan allows them.
bool rows_per_lane_allowed() {
    const char* e = getenv("IFCTN_CW_RPL");
    return !(e && strcmp(e, "1") == 0);
}

WarpKnobs default_warp_knobs() {
    WarpKnobs kn;
    kn.rpl = rows_per_lane_allowed() ? 1 : 0;
    return kn;
}

namespace {

// The plan with NW0 warps a CTA (12 for the COL kernel with tasks of up to 64
// rows) and at most XBYTES of X in a one-row-per-lane task; pl.warp = 0 when
// the rings do not fit.
ContractPlan plan_contract_warp_at(const Shape& s, int k, int sz, std::vector<UnitDesc>& units,
                                   const WarpKnobs& kn, int NW0, int XBYTES) {
    // two rows per lane only with the 16-warp CTA (12 for COL): the kernels
    // are instantiated for those
    const bool rpl_allowed = kn.rpl != 0 && NW0 == 16;
    int NW = NW0;
    ContractPlan pl;
    memset(&pl, 0, sizeof(pl));
    const int N = s.N, Am = N - 2, Bm = N - 1, IA = s.IA, IB = s.IB;
    const int VN = 16 / sz;
    const int sms = num_sms();
    // work units: enough for balance; where the partials are kept per unit
    // (CASE_A, COL) fewer, since the finisher sums over them
    const int target = (k < N - 2) ? 8 * sms : 4 * sms;
    // rows per task: at most cap, split evenly
    auto balanced = [](int rows, int cap) {
        cap = std::max(1, std::min(rows, cap));
        return cdiv(rows, cdiv(rows, cap));
    };
    pl.Q = mode_q(s, k);
    units.clear();
    auto add = [&](int f0, int fstride, int ns, int key, int a0, int a1, int b0, int b1, int slot) {
        UnitDesc u;
        memset(&u, 0, sizeof(u));
        u.f0 = f0;
        u.fstride = fstride;
        u.ns = ns;
        u.key = key;
        u.a0 = a0;
        u.a1 = a1;
        u.b0 = b0;
        u.b1 = b1;
        u.slot = slot;
        units.push_back(u);
    };
    long long tab_elems = 0, gtab_elems = 0, wab_elems = 0, zs_elems = 0, zmin = 0;
    int xregion = 0;
    if (k == Bm) {  // COL
        pl.kcase = CASE_COL;
        pl.R1 = s.R[k][Am];
        if (N == 4) {
            pl.l2 = 1;
            pl.dmode = 0;
        } else if (N == 3) {
            pl.l2 = 0;
            pl.dmode = -1;
        } else {
            pl.l2 = -1;
            pl.dmode = -1;
        }
        pl.Rl2 = pl.l2 >= 0 ? s.R[k][pl.l2] : 1;
        pl.Qp = pl.Rl2 * pl.R1;
        pl.zw = pl.Qp;
        const int nbc = cdiv(IB, 32);
        pl.vec = 0;
        pl.ldx = IB;
        // a lane builds one row of the coefficient table: at most 32 rows a task,
        // or 64 (two rows a lane, 12 warps so that their rings fit) when the
        // rows are short enough (IFCTN_CW_RPL=1 keeps 32)
        int RBK = balanced(IA, std::min(32, std::max(1, XBYTES / (sz * IB))));
        pl.rpl = 1;
        if (rpl_allowed) {
            const int RBK2 = balanced(IA, std::min(64, std::max(1, 2 * XBYTES / (sz * IB))));
            if (RBK2 > 32) {
                RBK = RBK2;
                pl.rpl = 2;
                NW = 12;
            }
        }
        pl.TAc = RBK;
        const int nrb = cdiv(IA, RBK);
        if (N == 4) {
            const int I0 = s.I[0], I1 = s.I[1];
            int nC = std::max(1, std::min(std::min(cdiv(target, static_cast<long long>(I0) * nbc),
                                                   std::max(1, I1 * nrb / NW)), I1));
            if (kn.chunking == 0) nC = warp_unit_chunks(I1, nrb, static_cast<long long>(I0) * nbc, nC, NW, sms);
            if (kn.chunking == 2) nC = 1;
            for (int i0 = 0; i0 < I0; ++i0)
                for (int c = 0; c < nC; ++c)
                    for (int bc = 0; bc < nbc; ++bc) {
                        int lo, hi;
                        chunk(I1, nC, c, lo, hi);
                        if (hi <= lo) continue;
                        add(i0 * I1 + lo, 1, hi - lo, i0, 0, IA, bc * 32, std::min(IB, bc * 32 + 32), 0);
                    }
        } else if (N == 3) {
            const int I0 = s.I[0];
            const int nC = std::max(1, std::min(std::min(cdiv(target, nbc), std::max(1, I0 * nrb / NW)), I0));
            for (int c = 0; c < nC; ++c)
                for (int bc = 0; bc < nbc; ++bc) {
                    int lo, hi;
                    chunk(I0, nC, c, lo, hi);
                    if (hi <= lo) continue;
                    add(lo, 1, hi - lo, -1, 0, IA, bc * 32, std::min(IB, bc * 32 + 32), 0);
                }
        } else {
            const int nrc = std::max(1, std::min(cdiv(target, nbc), cdiv(nrb, NW)));
            for (int rc = 0; rc < nrc; ++rc)
                for (int bc = 0; bc < nbc; ++bc) {
                    int lo, hi;
                    chunk(nrb, nrc, rc, lo, hi);
                    if (hi <= lo) continue;
                    add(0, 1, 1, -1, lo * RBK, std::min(IA, hi * RBK), bc * 32, std::min(IB, bc * 32 + 32), 0);
                }
        }
        pl.nrow = IB;
        pl.nunits = static_cast<int>(units.size());
        pl.part_elems = static_cast<long long>(pl.nunits) * IB * pl.Qp;
        pl.fin_div = 32;  // units covering column b: b / 32, b / 32 + nbc, ...
        pl.fin_mod = nbc;
        xregion = round_up(RBK * IB + 32 / sz, VN);
        tab_elems = static_cast<long long>(NW) * (32 * pl.rpl + VN) * pl.R1;
        gtab_elems = static_cast<long long>(pl.R1) * IA + (pl.l2 >= 0 ? static_cast<long long>(pl.Rl2) * s.I[pl.l2] : 0);
        zmin = 32LL * pl.zw;
        pl.aux_slot = 0;
    } else {  // ROW
        const bool isF = k < Am;
        pl.kcase = isF ? CASE_F : CASE_A;
        pl.R1 = s.R[k][Bm];
        const bool foldA = isF && N == 3;
        if (isF) {
            pl.RA = s.R[k][Am];
            pl.dmode = -1;
            if (N == 4) {
                pl.l2 = 1 - k;
                pl.Rl2 = s.R[k][pl.l2];
                pl.zw = pl.Rl2 * pl.R1;
            } else {
                pl.l2 = -1;
                pl.Rl2 = 1;
                pl.zw = pl.RA * pl.R1;
            }
            pl.Qp = pl.Q;
        } else {
            if (N == 4) {
                pl.l2 = 1;
                pl.dmode = 0;
            } else if (N == 3) {
                pl.l2 = 0;
                pl.dmode = -1;
            } else {
                pl.l2 = -1;
                pl.dmode = -1;
            }
            pl.Rl2 = pl.l2 >= 0 ? s.R[k][pl.l2] : 1;
            pl.Qp = pl.Rl2 * pl.R1;
            pl.zw = pl.Qp;
        }
        // 16-byte rows are read with 16-byte loads (N = 3, k = 0 reads rows of
        // W_{A,B} the same way, whose start must then be aligned too).  Eight
        // consecutive rows of nch 16-byte chunks fall on 8/gcd(nch, 8) bank
        // groups; from a 4-way conflict on, lanes read their chunks skewed.
        pl.vec = (IB % VN == 0 && (!foldA || s.woff[Am][Bm] % VN == 0)) ? 1 : 0;
        if (pl.vec) {
            const int nch = IB / VN;
            int g = nch, m = 8;
            while (m) {
                const int t = g % m;
                g = m;
                m = t;
            }
            pl.skew = g >= 4 ? 1 : 0;
        }
        // W_{A,B} rows of a unit (staged per unit): padded to an odd number of chunks
        int ldx = round_up(IB, VN);
        if ((ldx / VN) % 2 == 0) ldx += VN;
        pl.ldx = ldx;
        // a lane owns one row: tasks of up to 32 rows; rows too long for 16 of
        // them in a task leave the mode to the CTA kernels.  Order 4 with equal
        // ranks R_{k,B} = R_{k,l2} (2..5) and more than 32 rows: two rows per
        // lane, tasks of up to 64 rows (IFCTN_CW_RPL=1 or 2 forces the choice
        // where both are possible).
        int RBK = balanced(IA, std::min(32, XBYTES / (sz * IB)));
        if (RBK < std::min(IA, 16)) {
            units.clear();
            pl.warp = 0;
            return pl;
        }
        pl.rpl = 1;
        if (rpl_allowed && N == 4 && pl.Rl2 == pl.R1 && pl.R1 >= 2 && pl.R1 <= 5) {
            const int RBK2 = balanced(IA, std::min(64, 2 * XBYTES / (sz * IB)));
            if (RBK2 > 32) {
                RBK = RBK2;
                pl.rpl = 2;
            }
        }
        pl.TAc = RBK;
        const int nrc = cdiv(IA, RBK);
        if (isF && N == 4) {
            const int o = 1 - k, Io = s.I[o], Ik = s.I[k], I1 = s.I[1];
            int nOC = std::max(1, std::min(cdiv(target, static_cast<long long>(Ik) * nrc), std::max(1, Io / NW)));
            if (kn.chunking == 0) nOC = warp_unit_chunks(Io, 1, static_cast<long long>(Ik) * nrc, nOC, NW, sms);
            if (kn.chunking == 2) nOC = 1;
            for (int j = 0; j < Ik; ++j)
                for (int oc = 0; oc < nOC; ++oc)
                    for (int rc = 0; rc < nrc; ++rc) {
                        int lo, hi;
                        chunk(Io, nOC, oc, lo, hi);
                        const int a0 = rc * RBK, a1 = std::min(IA, a0 + RBK);
                        if (k == 0)
                            add(j * I1 + lo, 1, hi - lo, j, a0, a1, 0, IB, oc * nrc + rc);
                        else
                            add(lo * I1 + j, I1, hi - lo, j, a0, a1, 0, IB, oc * nrc + rc);
                    }
            pl.nslot = nOC * nrc;
            pl.part_elems = static_cast<long long>(Ik) * pl.nslot * pl.Q;
            wab_elems = static_cast<long long>(RBK) * ldx;
            zs_elems = static_cast<long long>(RBK) * pl.zw;
        } else if (foldA) {  // N = 3, k = 0: one slab per output row, split by rows
            const int I0 = s.I[0];
            const int nu = std::max(1, std::min(cdiv(target, I0), cdiv(nrc, NW)));
            for (int j = 0; j < I0; ++j)
                for (int c = 0; c < nu; ++c) {
                    int lo, hi;
                    chunk(nrc, nu, c, lo, hi);
                    add(j, 1, 1, j, lo * RBK, std::min(IA, hi * RBK), 0, IB, c);
                }
            pl.nslot = nu;
            pl.part_elems = static_cast<long long>(I0) * nu * pl.Q;
            pl.xr = round_up(RBK * IB + 32 / sz, VN);
        } else if (N == 4) {
            const int I0 = s.I[0], I1 = s.I[1];
            int nC = std::max(1, std::min(cdiv(target, static_cast<long long>(I0) * nrc), std::max(1, I1 / NW)));
            if (kn.chunking == 0) nC = warp_unit_chunks(I1, 1, static_cast<long long>(I0) * nrc, nC, NW, sms);
            if (kn.chunking == 2) nC = 1;
            for (int i0 = 0; i0 < I0; ++i0)
                for (int c = 0; c < nC; ++c)
                    for (int rc = 0; rc < nrc; ++rc) {
                        int lo, hi;
                        chunk(I1, nC, c, lo, hi);
                        if (hi <= lo) continue;
                        add(i0 * I1 + lo, 1, hi - lo, i0, rc * RBK, std::min(IA, rc * RBK + RBK), 0, IB, 0);
                    }
        } else if (N == 3) {
            const int I0 = s.I[0];
            const int nC = std::max(1, std::min(cdiv(target, nrc), std::max(1, I0 / NW)));
            for (int c = 0; c < nC; ++c)
                for (int rc = 0; rc < nrc; ++rc) {
                    int lo, hi;
                    chunk(I0, nC, c, lo, hi);
                    if (hi <= lo) continue;
                    add(lo, 1, hi - lo, -1, rc * RBK, std::min(IA, rc * RBK + RBK), 0, IB, 0);
                }
        } else {
            for (int rc = 0; rc < nrc; ++rc) add(0, 1, 1, -1, rc * RBK, std::min(IA, rc * RBK + RBK), 0, IB, 0);
        }
        pl.nrow = IA;
        pl.nunits = static_cast<int>(units.size());
        if (!isF) {
            pl.part_elems = static_cast<long long>(pl.nunits) * IA * pl.Qp;
            pl.fin_div = RBK;  // units covering row a: a / RBK, a / RBK + nrc, ...
            pl.fin_mod = nrc;
        }
        xregion = round_up(RBK * IB + 32 / sz, VN);
        if (foldA) xregion *= 2;
        const int RBP = round_up(pl.R1, VN);
        tab_elems = static_cast<long long>(NW) * IB * (pl.vec ? pl.R1 : RBP);
        gtab_elems = static_cast<long long>(pl.R1) * IB +
                     (pl.l2 >= 0 ? static_cast<long long>(pl.Rl2) * s.I[pl.l2] : 0) +
                     (isF ? static_cast<long long>(pl.RA) * IA : 0);
        zmin = foldA ? pl.zw : static_cast<long long>(RBK) * pl.zw;
        pl.aux_slot = 0;
    }
    long long tc = xregion;
    tc = std::max(tc, zmin);
    tc = (tc + VN - 1) / VN * VN;
    pl.sub_elems = static_cast<int>(tc);
    auto r128 = [](long long b) { return (b + 127) / 128 * 128; };
    const long long limit = 225 * 1024;
    // per-warp ring of a task's W entries (cp.async), elements a stage: COL the
    // row weights of two F modes (32 or 64 rows each), W_{0,1}(i0, i1); ROW one row W_{p,B}(i_p, :)
    // (two for N = 4, k = 2) padded to whole warps, then the fold weights of up
    // to 32 rows per lane row
    const long long auxw = (k == Bm) ? 64LL * std::max(1, pl.rpl) + 32
                                     : (N == 4 && k == 2 ? 2LL : 1LL) * round_up(IB, 32) + 32LL * std::max(1, pl.rpl);
    pl.auxw = static_cast<int>(auxw);
    // with two rows per lane the unit-end sums (zs) share the per-warp
    // coefficient tables' space: those are rewritten only by the next unit's
    // tasks, after the unit end's last CTA barrier
    const bool zs_in_tab = pl.rpl == 2 && zs_elems <= tab_elems;
    for (int S = 4; S >= 2; --S) {
        if (kn.stages > 0 && S != kn.stages) continue;
        const long long off_tile = 640;
        const long long off_tab = off_tile + r128(static_cast<long long>(NW) * S * tc * sz);
        const long long off_gtab = off_tab + r128(tab_elems * sz);
        const long long off_wab = off_gtab + r128(gtab_elems * sz);
        const long long off_zs = zs_in_tab ? off_tab : off_wab + r128(wab_elems * sz);
        const long long off_aux = zs_in_tab ? off_wab + r128(wab_elems * sz) : off_zs + r128(zs_elems * sz);
        const long long total = off_aux + static_cast<long long>(NW) * S * auxw * sz;
        if (total <= limit) {
            pl.nstages = S;
            pl.off_tile = static_cast<int>(off_tile);
            pl.off_tab = static_cast<int>(off_tab);
            pl.off_gtab = static_cast<int>(off_gtab);
            pl.off_wab = static_cast<int>(off_wab);
            pl.off_zs = static_cast<int>(off_zs);
            pl.off_aux = static_cast<int>(off_aux);
            pl.smem = static_cast<int>(total);
            pl.warp = 1;
            break;
        }
    }
    pl.nwarp = NW;
    if (!pl.warp && pl.rpl == 2) {
        WarpKnobs k1 = kn;
        k1.rpl = 0;
        return plan_contract_warp_at(s, k, sz, units, k1, NW0, XBYTES);
    }
    pl.grid = std::max(1, std::min(pl.nunits, sms));
    if (N == 4) {  // i0 = f / I_1 without a division: exact for f < 2^31 (Granlund-Montgomery, rounded-up multiplier)
        const unsigned long long d = static_cast<unsigned long long>(s.I[1]);
        int l = 0;
        while ((1ULL << l) < d) ++l;
        pl.fdiv_s = 32 + l;
        pl.fdiv_m = ((1ULL << pl.fdiv_s) + d - 1) / d;
    }
    if (!pl.warp) units.clear();
    return pl;
}

}  // namespace

// The first plan whose rings fit and whose tasks have at least three quarters
// of min(IA, 32) rows (or the fitting plan with the most rows a task): 16 warps a CTA,
// then 8 with twice the shared memory each; the X budget of a task as the knob
// gives it, doubled, quadrupled (long rows fill fewer lanes).
ContractPlan plan_contract_warp(const Shape& s, int k, int sz, std::vector<UnitDesc>& units,
                                const WarpKnobs& kn) {
    const int rows = s.IA;  // rows of mode A: what a task splits, for both kinds
    ContractPlan best;
    memset(&best, 0, sizeof(best));
    std::vector<UnitDesc> bu;
    for (int nw : {16, 8})
        for (int xf = 1; xf <= 4; xf *= 2) {
            std::vector<UnitDesc> u;
            const ContractPlan p = plan_contract_warp_at(s, k, sz, u, kn, nw, kn.xbytes * xf);
            if (!p.warp) continue;
            const int want = std::min(rows, 32) * 3 / 4;
            if (p.TAc >= want) {
                units = u;
                return p;
            }
            if (!best.warp || p.TAc > best.TAc) {
                best = p;
                bu = u;
            }
        }
    units = bu;
    return best;
}

}  // namespace ifctn
