// ifctn_internal.cuh -- shared definitions of the iFCTN sm_103a kernels.
//
// Notation follows the paper (Gan & Cui, iFCTN): X is I_0 x ... x I_{N-1}
// (0-based here), cherry factor G_{k,l} is R_{k,l} x I_k, and
// W_{p,q} = G_{p,q}^T G_{q,p} (I_p x I_q) is the pair matrix whose broadcast
// product over pairs without k is S_k of Prop. 1.  The model is
// X(i) = prod_{p<q} W_{p,q}(i_p, i_q) (eq. (iFCTN) with every rank sum
// carried out pair by pair).
//
// Geometry used by every streaming kernel.  The C-order tensor is viewed as
// nF "slabs" of IA x IB entries: B = mode N-1 (contiguous), A = mode N-2,
// and the slab index f runs over modes 0..N-3 (F modes).  For N = 2 there is
// one slab (A = mode 0, B = mode 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ifctn {

constexpr int MAXN = 4;
constexpr int RMAX = 8;
// Order-3 tensors may have edge ranks above RMAX (the multispectral rank grid
// of Sec. 5.2 reaches R_{1,2} = 36): their mode systems and column solves run
// on the kernels of ifctn_wide.cu, up to these limits.
constexpr int WIDE_RMAX = 64;
constexpr int WIDE_QMAX = 4096;

enum : int { FLAG_TIMEOUT = 1, FLAG_NOTSPD = 2, FLAG_NONFINITE = 4 };

struct Shape {
    int N;
    int I[MAXN];
    int R[MAXN][MAXN];
    long long P;
    int goff[MAXN][MAXN];  // element offset of G_{k,l} in the packed factor array
    int woff[MAXN][MAXN];  // element offset of W_{p,q} (p<q) in the packed pair array
    int gsize, wsize;
    int nF, IA, IB;        // slab count and slab sizes
    int wide;              // 1: some R_{k,l} > RMAX (order 3): the kernels of ifctn_wide.cu
};

// One work unit of a streaming contraction: a list of slabs
// {f0 + s*fstride : s < ns}, rows [a0,a1) and columns [b0,b1) of each slab,
// and a key (output row for k in F, deferred-mode index otherwise).
struct UnitDesc {
    int f0, fstride, ns, key;
    int a0, a1, b0, b1;
    int slot, pad0, pad1, pad2;
};

enum ContractCase : int { CASE_F = 0, CASE_A = 1, CASE_COL = 2 };

struct ContractPlan {
    int kcase;
    int l2;          // level-2 mode (accumulated in registers), -1 none
    int dmode;       // mode deferred to the finisher, -1 none
    int R1;          // rank of the level-1 (in-register) contraction
    int Rl2;         // rank of the level-2 mode (1 if none)
    int RA;          // CASE_F: rank R_{k,A} applied at the flush
    int Qp;          // width of one partial row
    int Q;           // Q_k
    int TA;          // ROW: rows per pass; COL: columns per CTA (TB)
    int TAc;         // COL: rows per chunk
    int G;           // groups per CTA (each group one slab per stage)
    int nthreads;
    int nunits;
    int nslot;       // CASE_F: partial slots per output row
    int nrow;        // CASE_A: IA, COL: IB (rows of a partial)
    int sub_elems;   // capacity of one group's stage sub-buffer (elements)
    int nstages;
    int smem;        // dynamic shared memory bytes
    int skew;        // ROW: rotate the b loop (IB even)
    int split;       // 1: one slab per stage, the G groups split its reduction
                     //    range (ROW: columns b, COL: rows a); 0: groups take
                     //    different slabs
    int aux_slot;    // elements per auxiliary-vector slot in a stage sub-buffer
    int gtab_smem;   // 1: the unit's G_{m,k} tables are staged in shared memory
    int gtab_elems;  // their size (elements)
    int key_div;     // > 0: every unit covers all rows and its deferred key is
                     //      unit / key_div (no descriptor loads in the reduction)
    // warp-pipelined kernels (HBM-streaming tensors)
    int warp;        // 1: k_contract_roww / k_contract_colw run this mode
    int vec;         // ROW: rows copied one by one into a padded layout and read
                     //      with 16-byte loads; COL: only the unit's columns copied
    int ldx;         // row stride of the X tile in shared memory (elements)
    int xr;          // ROW, N = 3, k = 0: offset of the W_{A,B} rows in a stage
    int zw;          // width of one register-fold row (elements)
    int grid;        // CTAs (one per SM)
    int off_tile, off_tab, off_gtab, off_wab, off_zs, off_aux;  // shared-memory carve-up (bytes)
    int fin_div, fin_mod;  // > 0: the units covering output row r are r / fin_div + n * fin_mod
    int auxw;        // warp kernels: elements of a warp's per-stage ring slot of W entries
    int rpl;         // warp kernels: rows per lane (1, or 2 for tasks of up to 64 rows)
    int nwarp;       // warp kernels: warps per CTA
    int fdiv_s;      // warp kernels, N = 4: slab f = i0 I_1 + i1 has i0 = (f * fdiv_m) >> fdiv_s
    unsigned long long fdiv_m;
    long long part_elems;
};

// Launch-shape choices of the warp-pipelined contraction that the planner
// leaves open (the autotuner times them): rows per lane allowed (1) or not,
// ring stages per warp (0 = as many as fit, else 2..4), X bytes of a
// one-row-per-lane task, and the unit chunking (0 = the cost model that gives
// every warp of a unit the same number of tasks, 1 = balance across SMs only,
// 2 = the fewest units: one per output row or deferred index, which leaves
// the finisher the fewest partials to reduce).
struct WarpKnobs {
    int rpl = 1;
    int stages = 0;
    int xbytes = 4096;
    int chunking = 0;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Programmatic dependent launch: the sweep graph's kernel-to-kernel edges let a
// kernel be launched while its predecessor still runs.  Every kernel that can
// sit in that graph first waits until its predecessors have completed and
// their writes are visible (a no-op for an ordinary launch), then lets its own
// dependents launch, so their launch latency and block scheduling overlap
// this kernel's run instead of following it.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Clock budget of every bounded device wait (about 2 s at 2 GHz).
constexpr long long WAIT_BUDGET_CYCLES = 4000000000LL;

// Waits for phase `parity` of the barrier with a clock budget (WAIT_BUDGET_CYCLES
// unless a shorter one is given).  On expiry it records FLAG_TIMEOUT and
// returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* flags,
                                                  long long budget = WAIT_BUDGET_CYCLES) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) {
            atomicOr(flags, FLAG_TIMEOUT);
            return false;
        }
    }
    return true;
}

// 1-D TMA bulk copy global -> shared, completion signalled on `bar`.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Asynchronous element-wise copy global -> shared by all threads of the CTA
// (cp.async: every copy is in flight before any wait).  Completes at
// stage_wait(), which also synchronises the CTA.
template <typename T>
__device__ __forceinline__ void stage_async(T* dst, const T* src, int n) {
    int i0 = 0;
    if (((smem_u32(dst) | static_cast<unsigned>(reinterpret_cast<uintptr_t>(src))) & 15u) == 0) {
        // both 16-byte aligned: 16-byte copies, then the elements of the tail
        constexpr int E = 16 / static_cast<int>(sizeof(T));
        const int nv = n / E;
        for (int v = threadIdx.x; v < nv; v += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + v * E)), "l"(src + v * E)
                         : "memory");
        i0 = nv * E;
    }
    for (int i = i0 + threadIdx.x; i < n; i += blockDim.x) {
        if (sizeof(T) == 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst + i)), "l"(src + i) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst + i)), "l"(src + i) : "memory");
    }
}

__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// W_{p,q}(a, b) for any p != q (stored for p<q)
template <typename T>
__device__ __forceinline__ T wpair(const T* W, const Shape& s, int p, int q, int ip, int iq) {
    return p < q ? W[s.woff[p][q] + (long long)ip * s.I[q] + iq]
                 : W[s.woff[q][p] + (long long)iq * s.I[p] + ip];
}

// G_{m,k}(r, i)
template <typename T>
__device__ __forceinline__ T gfac(const T* G, const Shape& s, int m, int k, int r, int i) {
    return G[s.goff[m][k] + r * s.I[m] + i];
}

#endif  // __CUDACC__

}  // namespace ifctn
