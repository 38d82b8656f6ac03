// ifctn_api.cu -- host runtime and C ABI of the iFCTN library.
//
// A context owns every device buffer of one completion problem, plans the
// launch geometry of each mode once, and captures one PAM sweep (Algorithm 1,
// one pass of its loop) into a CUDA graph that is replayed per sweep.  The
// Gram chain of mode k runs on a side branch of the graph, concurrently with
// the HBM-streaming contraction of the same mode.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ifctn.h"
#include "ifctn_api_internal.h"
#include "ifctn_launch.h"
#include "ifctn_persistent.h"
#include "ifctn_plan.h"

namespace ifctn {

thread_local std::string g_last_error;

void set_error(const std::string& m) { g_last_error = m; }

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                         \
            return IFCTN_ECUDA;                                                                    \
        }                                                                                          \
    } while (0)

namespace {

constexpr int LOG_CAP = 4096;

}  // namespace

}  // namespace ifctn

using namespace ifctn;

namespace {

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count) {
        n = count;
        return cudaMalloc(reinterpret_cast<void**>(&p), std::max<size_t>(count, 1) * sizeof(T) + 64);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
    }
};

}  // namespace

struct ifctn_ctx {
    virtual ~ifctn_ctx() {}
    virtual ifctn_status sweep(int n, ifctn_stats* out) = 0;
    virtual ifctn_status complete(void* out_X, ifctn_stats* out) = 0;
    virtual ifctn_status reconstruct(void* out) = 0;
    virtual ifctn_status get_factors(double* out) = 0;
    virtual ifctn_status set_factors(const double* in) = 0;
    virtual ifctn_status get_x(void* out) = 0;
    virtual ifctn_status set_x(const void* in) = 0;
    virtual ifctn_status set_truth(const void* xt, int log) = 0;
    virtual ifctn_status get_log(ifctn_stats* out, int max, int* n) = 0;
    virtual ifctn_status mode_system(int k, double* Mk, double* Kk) = 0;
    virtual int kernels_per_sweep() const = 0;
    virtual size_t device_bytes() const = 0;
    virtual ifctn_status enqueue(int n, double tol, bool reset) = 0;
    virtual ifctn_status launch_stage(int stage, int k) = 0;
    virtual ifctn_status wait_selftest(long long budget) = 0;
    virtual ifctn_status tune(const char* path, int* ntimed) = 0;
    virtual ifctn_status sweep_exchange(int n, ifctn_allreduce_fn fn, void* user, ifctn_stats* out) = 0;
    virtual long long launch_total() const = 0;
    virtual ifctn_status phase_times(double* out, int max, int* n) = 0;
    virtual void set_grid_cap(int g) = 0;
    virtual cudaStream_t stream() const = 0;
    // batched persistent launches (serving): the element size of the context's
    // dtype when its sweeps run as one persistent launch, else 0
    virtual int batch_kind() const = 0;
};

namespace ifctn {

// Tensors that do not stay in L2 stream through the per-stage kernels (graph
// path, warp-pipelined contraction); the rest run as one persistent launch.
// IFCTN_PATH=graph or =persistent overrides the choice (testing, tuning).
bool choose_graph_only(const Shape& sh, int sz) {
    const char* e = getenv("IFCTN_PATH");
    if (e && strcmp(e, "graph") == 0) return true;
    if (e && strcmp(e, "persistent") == 0) return false;
    return sh.P * static_cast<long long>(sz) > L2_RESIDENT_BYTES;
}

// NVTX range over a scope (header-only NVTX3: free unless a profiler injects a
// tool).  The host-side enqueue of each stage is named, so that a timeline shows
// the stages of the per-stage path, the exchange of the sharded sweep, tuning
// and graph or persistent sweep launches.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
const char* const kModeSystems[MAXN] = {"ifctn mode 1 contraction+Gram", "ifctn mode 2 contraction+Gram",
                                        "ifctn mode 3 contraction+Gram", "ifctn mode 4 contraction+Gram"};
const char* const kModeSolves[MAXN] = {"ifctn mode 1 solves", "ifctn mode 2 solves", "ifctn mode 3 solves",
                                       "ifctn mode 4 solves"};

#ifndef IFCTN_SOURCE_DIGEST
#define IFCTN_SOURCE_DIGEST "unversioned"
#endif

// The autotuner's selection rule: the fastest candidate, except that the
// planner's default (candidate 0) is kept unless the fastest beats it by 2 %
// or more (timings of nearly equal shapes differ by noise, and the default
// is what every other context of the shape runs when no cache is used).
int tune_choose(int n, const double* secs) {
    if (n <= 0) return -1;
    int best = 0;
    for (int i = 1; i < n; ++i)
        if (secs[i] < secs[best]) best = i;
    return secs[best] <= 0.98 * secs[0] ? best : 0;
}

template <typename T>
struct Engine : ifctn_ctx {
    Shape sh;
    ifctn_problem prob;
    cudaStream_t st = nullptr, side = nullptr;
    bool own_stream = false;
    cudaEvent_t ev_fork[MAXN] = {}, ev_join[MAXN] = {};
    DevBuf<T> X, Xt, Gt, W, Kk, t1, t2, part, tmpT;
    DevBuf<double> Gd, Mk[MAXN], xpart, mpart, scal, tmpD, tol;
    DevBuf<uint32_t> maskbits;
    DevBuf<UnitDesc> units;
    DevBuf<SweepStat> log;
    DevBuf<int> ints;  // [0] counter, [1] done, [2] flags
    DevBuf<int> stab;  // index tables of the column solves, per mode (solve_stage_tables)
    int stab_off[MAXN] = {};
    ContractPlan plan[MAXN];
    int unit_off[MAXN] = {};
    int xblocks = 0;
    long long nmiss = 0, nobs = 0;
    bool truth = false, logm = false;
    cudaGraphExec_t gexec = nullptr;
    int launches = 0;
    size_t bytes = 0;
    // persistent path
    bool persistent = false;
    bool graph_only = false;  // HBM-sized tensor (or forced): per-stage kernels, warp-pipelined contraction
    int pgrid = 0, psmem = 0, grid_cap = 0;
    SweepParams<T> pp;
    DevBuf<unsigned> bar;
    DevBuf<unsigned long long> tstamp;  // [0,64): phase ends; [64 + k*512 + cta]: per-CTA phase-1 ends
    long long launch_count = 0;
    int ex_sweeps = 0;  // sweeps run by sweep_exchange
    // creation-time tuning (IFCTN_TUNE_CACHE) may time candidates; contexts
    // of served jobs only read the cache, so a job never pays for timing
    bool tune_timing = true;
    int force_path = 0;  // 1: sweep graph of per-stage kernels, 2: persistent launch, 0: by size
    DevBuf<T> snapX;
    DevBuf<double> snapG;

    // Saves the initial state (X, G) so that sweeps timed to choose the
    // execution path can be undone by restore_snapshot().
    ifctn_status snapshot() {
        if (snapX.alloc(sh.P) != cudaSuccess || snapG.alloc(sh.gsize) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation failed");
            return IFCTN_ENOMEM;
        }
        CK(cudaMemcpyAsync(snapX.p, X.p, sh.P * sizeof(T), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(snapG.p, Gd.p, sh.gsize * sizeof(double), cudaMemcpyDeviceToDevice, st));
        return IFCTN_OK;
    }
    // Back to the saved state, with the sweep counter, log and flags as at creation.
    ifctn_status restore_snapshot() {
        CK(cudaMemcpyAsync(X.p, snapX.p, sh.P * sizeof(T), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(Gd.p, snapG.p, sh.gsize * sizeof(double), cudaMemcpyDeviceToDevice, st));
        ifctn_status rs = refresh_factors();
        if (rs != IFCTN_OK) return rs;
        CK(cudaMemsetAsync(ints.p, 0, 4 * sizeof(int), st));
        CK(cudaStreamSynchronize(st));
        snapX.release();
        snapG.release();
        return IFCTN_OK;
    }
    // Device seconds of m sweeps after m warm-up sweeps (CUDA events on the
    // context's stream), from and back to the saved state.
    ifctn_status time_sweeps(int m, double* sec) {
        ifctn_status rs = snapshot();
        if (rs != IFCTN_OK) return rs;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        rs = enqueue(m, 0.0, true);
        if (rs == IFCTN_OK && cudaEventRecord(e0, st) != cudaSuccess) rs = IFCTN_ECUDA;
        if (rs == IFCTN_OK) rs = enqueue(m, 0.0, true);
        if (rs == IFCTN_OK && cudaEventRecord(e1, st) != cudaSuccess) rs = IFCTN_ECUDA;
        float ms = 0.f;
        if (rs == IFCTN_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rs = IFCTN_ECUDA;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rs == IFCTN_OK) rs = check_flags();
        if (rs != IFCTN_OK) return rs;
        *sec = 1e-3 * ms;
        return restore_snapshot();
    }
    double cur_tol = 0.0;

    int* counter() { return ints.p; }
    int* done() { return ints.p + 1; }
    int* flags() { return ints.p + 2; }

    ~Engine() override {
        if (st) cudaStreamSynchronize(st);
        if (gexec) cudaGraphExecDestroy(gexec);
        for (int k = 0; k < MAXN; ++k) {
            if (ev_fork[k]) cudaEventDestroy(ev_fork[k]);
            if (ev_join[k]) cudaEventDestroy(ev_join[k]);
            Mk[k].release();
        }
        bar.release();
        tstamp.release();
        X.release(); Xt.release(); Gt.release(); W.release(); Kk.release(); t1.release(); t2.release();
        part.release(); tmpT.release(); Gd.release(); xpart.release(); mpart.release(); scal.release();
        tmpD.release(); tol.release(); maskbits.release(); units.release(); log.release(); ints.release();
        stab.release();
        if (side) cudaStreamDestroy(side);
        if (own_stream && st) cudaStreamDestroy(st);
    }

    size_t device_bytes() const override { return bytes; }

    template <typename U>
    cudaError_t alloc(DevBuf<U>& b, size_t n) {
        bytes += n * sizeof(U) + 64;
        return b.alloc(n);
    }

    ifctn_status init(const ifctn_problem* p, const void* obs, const uint8_t* mask, const double* init_f,
                      void* stream) {
        prob = *p;
        ifctn_status rs = build_shape(p, sh);
        if (rs != IFCTN_OK) return rs;
        if (!obs || !mask) {
            set_error("obs and mask are required");
            return IFCTN_EINVAL;
        }
        if (stream) {
            st = static_cast<cudaStream_t>(stream);
        } else {
            CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            own_stream = true;
        }
        CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        for (int k = 0; k < MAXN; ++k) {
            CK(cudaEventCreateWithFlags(&ev_fork[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ev_join[k], cudaEventDisableTiming));
        }
        const int sz = sizeof(T);
        std::vector<UnitDesc> all;
        long long maxpart = 1, maxt1 = 1, maxt2 = 1, maxK = 1;
        graph_only = force_path == 1 ? true : force_path == 2 ? false : choose_graph_only(sh, sz);
        if (sh.wide) {
            // ranks above RMAX: the per-stage kernels of ifctn_wide.cu (t1 holds
            // the contraction's first link, t2 the Gram's)
            if (force_path == 2) {
                set_error("the persistent path needs every edge rank <= 8");
                return IFCTN_EINVAL;
            }
            graph_only = true;
            for (int k = 0; k < sh.N; ++k) {
                memset(&plan[k], 0, sizeof(plan[k]));
                plan[k].Q = mode_q(sh, k);
                plan[k].nstages = 1;
                unit_off[k] = 0;
                const long long Q = plan[k].Q;
                maxK = std::max(maxK, Q * Q);
                maxt1 = std::max(maxt1, wide_v_elems(sh, k));
                maxt2 = std::max(maxt2, wide_t_elems(sh, k));
            }
        }
        for (int k = 0; k < sh.N && !sh.wide; ++k) {
            std::vector<UnitDesc> u;
            plan[k].warp = 0;
            if (graph_only) plan[k] = plan_contract_warp(sh, k, sz, u, default_warp_knobs());
            if (!plan[k].warp) plan[k] = plan_contract(sh, k, sz, u);
            if (plan[k].smem > SMEM_LIMIT && !plan[k].warp) {
                set_error("tensor shape needs more shared memory than available");
                return IFCTN_EINVAL;
            }
            unit_off[k] = static_cast<int>(all.size());
            all.insert(all.end(), u.begin(), u.end());
            maxpart = std::max(maxpart, plan[k].part_elems);
            const int Q = mode_q(sh, k);
            maxK = std::max<long long>(maxK, static_cast<long long>(Q) * Q);
            int m[3], nm = 0;
            for (int q = 0; q < sh.N; ++q)
                if (q != k) m[nm++] = q;
            if (nm == 3) {
                maxt1 = std::max<long long>(maxt1, static_cast<long long>(sh.I[m[0]]) * sh.I[m[1]] *
                                                       sh.R[k][m[2]] * sh.R[k][m[2]]);
                const long long Q2 = static_cast<long long>(sh.R[k][m[1]]) * sh.R[k][m[2]];
                maxt2 = std::max<long long>(maxt2, sh.I[m[0]] * Q2 * Q2);
            } else if (nm == 2) {
                maxt2 = std::max<long long>(maxt2, static_cast<long long>(sh.I[m[0]]) * sh.R[k][m[1]] *
                                                       sh.R[k][m[1]]);
            }
        }
        xblocks = 4 * num_sms();
        const int xpart_n = std::max(3 * xblocks, 16 * 4 * num_sms());
        const long long P = sh.P;
        bool ok = alloc(X, P) == cudaSuccess && alloc(Gt, sh.gsize) == cudaSuccess &&
                  alloc(W, sh.wsize) == cudaSuccess && alloc(Kk, maxK) == cudaSuccess &&
                  alloc(t1, maxt1) == cudaSuccess && alloc(t2, maxt2) == cudaSuccess &&
                  alloc(part, maxpart) == cudaSuccess && alloc(Gd, sh.gsize) == cudaSuccess &&
                  alloc(xpart, xpart_n) == cudaSuccess && alloc(mpart, 3 * xblocks) == cudaSuccess &&
                  alloc(bar, 4) == cudaSuccess && alloc(tstamp, 64 + 4 * 512) == cudaSuccess &&
                  alloc(scal, 8) == cudaSuccess && alloc(tol, 1) == cudaSuccess &&
                  alloc(maskbits, (P + 31) / 32) == cudaSuccess && alloc(units, all.size()) == cudaSuccess &&
                  alloc(log, LOG_CAP) == cudaSuccess && alloc(ints, 4) == cudaSuccess;
        for (int k = 0; k < sh.N && ok; ++k)
            ok = alloc(Mk[k], static_cast<size_t>(sh.I[k]) * mode_q(sh, k)) == cudaSuccess;
        std::vector<int> tabs;
        for (int k = 0; k < sh.N && !sh.wide; ++k) {
            stab_off[k] = static_cast<int>(tabs.size());
            const int n = solve_tab_ints(mode_q(sh, k));
            tabs.resize(tabs.size() + (n + 3) / 4 * 4, 0);  // 16-byte aligned blocks
            solve_stage_tables(sh, k, tabs.data() + stab_off[k]);
        }
        if (tabs.empty()) tabs.resize(4, 0);  // the wide kernels use no index tables
        if (ok) ok = alloc(stab, tabs.size()) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            set_error("device allocation failed");
            return IFCTN_ENOMEM;
        }
        if (!all.empty())
            CK(cudaMemcpyAsync(units.p, all.data(), all.size() * sizeof(UnitDesc), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(stab.p, tabs.data(), tabs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(ints.p, 0, 4 * sizeof(int), st));
        CK(cudaMemsetAsync(bar.p, 0, 4 * sizeof(unsigned), st));
        CK(cudaMemsetAsync(tol.p, 0, sizeof(double), st));
        // inputs: mask bytes and O go through a scratch buffer
        {
            uint8_t* dmask = nullptr;
            T* dO = nullptr;
            CK(cudaMallocAsync(reinterpret_cast<void**>(&dmask), P, st));
            CK(cudaMemcpyAsync(dmask, mask, P, cudaMemcpyDefault, st));
            CK(launch_pack_mask(P, dmask, maskbits.p, st));
            CK(cudaMallocAsync(reinterpret_cast<void**>(&dO), P * sizeof(T), st));
            CK(cudaMemcpyAsync(dO, obs, P * sizeof(T), cudaMemcpyDefault, st));
            CK(launch_init_x<T>(P, dO, dmask, X.p, st));
            CK(cudaFreeAsync(dO, st));
            CK(cudaFreeAsync(dmask, st));
        }
        // |Omega| and its complement
        CK(launch_count_bits((P + 31) / 32, maskbits.p, xpart.p, xblocks, st));
        CK(launch_sum_partials(xpart.p, xblocks, 3, 0, scal.p, st));
        double hs[1];
        CK(cudaMemcpyAsync(hs, scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        nobs = static_cast<long long>(hs[0] + 0.5);
        nmiss = P - nobs;
        if (init_f) {
            CK(cudaMemcpyAsync(Gd.p, init_f, sh.gsize * sizeof(double), cudaMemcpyDefault, st));
        } else {
            rs = default_factors();
            if (rs != IFCTN_OK) return rs;
        }
        rs = refresh_factors();
        if (rs != IFCTN_OK) return rs;
        CK(cudaStreamSynchronize(st));
        setup_persistent();
        // launch shapes from the tuning cache named by IFCTN_TUNE_CACHE (timed
        // and added to it where the cache has no entry for this shape)
        if (const char* path = getenv("IFCTN_TUNE_CACHE")) {
            if (*path && graph_only && !sh.wide) {
                rs = tune(path, nullptr, !tune_timing);
                if (rs != IFCTN_OK) return rs;
                return IFCTN_OK;  // tune() rebuilt the graph
            }
        }
        return build_graph();
    }

    // ---- autotuning of the streaming contraction's launch shape ----------
    // Key of mode k of this problem in the tuning cache: the library's source
    // digest, the dtype, the shape and ranks, the mode and the SM count.
    std::string tune_key(int k) const {
        std::string key = std::string("ifctn-tune-v1 ") + IFCTN_SOURCE_DIGEST + (sizeof(T) == 4 ? " f32 " : " f64 ");
        key += "N" + std::to_string(sh.N);
        for (int m = 0; m < sh.N; ++m) key += "," + std::to_string(sh.I[m]);
        key += " R";
        for (int p2 = 0; p2 < sh.N; ++p2)
            for (int q = p2 + 1; q < sh.N; ++q) key += std::to_string(sh.R[p2][q]) + ".";
        key += " k" + std::to_string(k) + " sms" + std::to_string(num_sms());
        return key;
    }

    // Device seconds of the mode-k contraction and its finisher with plan pl
    // and units u (the median of 5 runs after one warm-up, CUDA events on the
    // context's stream); unit descriptors and partials in scratch buffers.
    ifctn_status time_contract(int k, const ContractPlan& pl, const std::vector<UnitDesc>& u, double* sec) {
        DevBuf<UnitDesc> du;
        DevBuf<T> dp;
        if (du.alloc(u.size()) != cudaSuccess || dp.alloc(std::max<long long>(pl.part_elems, 1)) != cudaSuccess) {
            du.release();
            dp.release();
            cudaGetLastError();
            set_error("device allocation failed while tuning");
            return IFCTN_ENOMEM;
        }
        ContractArgs<T> a = cargs(k);
        a.pl = pl;
        a.units = du.p;
        a.part = dp.p;
        cudaEvent_t e[6];
        for (auto& ev : e) cudaEventCreate(&ev);
        // the contraction and the finisher that reduces its per-unit partials
        // into M_k: both change with the plan
        auto pair = [&]() {
            cudaError_t r = launch_contract<T>(a, st);
            if (r == cudaSuccess)
                r = launch_contract_finish<T>(sh, k, pl, du.p, dp.p, Gt.p, Mk[k].p, done(), st);
            return r;
        };
        cudaError_t err = cudaMemcpyAsync(du.p, u.data(), u.size() * sizeof(UnitDesc), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = pair();
        for (int i = 0; i < 5 && err == cudaSuccess; ++i) {
            err = cudaEventRecord(e[i], st);
            if (err == cudaSuccess) err = pair();
        }
        if (err == cudaSuccess) err = cudaEventRecord(e[5], st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        std::vector<double> t;
        for (int i = 0; i < 5 && err == cudaSuccess; ++i) {
            float ms = 0.f;
            err = cudaEventElapsedTime(&ms, e[i], e[i + 1]);
            t.push_back(1e-3 * ms);
        }
        for (auto& ev : e) cudaEventDestroy(ev);
        du.release();
        dp.release();
        if (err != cudaSuccess) {
            set_error(std::string("tuning launch failed: ") + cudaGetErrorString(err));
            return IFCTN_ECUDA;
        }
        std::sort(t.begin(), t.end());
        *sec = t[t.size() / 2];
        return IFCTN_OK;
    }

    // For every mode whose contraction runs the warp-pipelined kernels: takes
    // the launch shape from the cache at `path` (nullable) when it holds this
    // key, else times the planner's candidates (rows per lane, ring stages,
    // task size, unit chunking), keeps the fastest by the rule of
    // tune_choose(), and appends it to the cache.  Then re-lays the unit
    // descriptors and rebuilds the sweep graph.
    ifctn_status tune(const char* path, int* ntimed) override { return tune(path, ntimed, false); }

    ifctn_status tune(const char* path, int* ntimed, bool lookup_only) {
        NvtxRange nr("ifctn tune");
        int timed = 0;
        if (sh.wide) {  // the kernels of ifctn_wide.cu have no launch-shape choices
            if (ntimed) *ntimed = 0;
            return IFCTN_OK;
        }
        std::vector<std::string> lines;
        if (path && *path) {
            if (FILE* f = fopen(path, "r")) {
                char buf[1024];
                while (fgets(buf, sizeof(buf), f)) lines.emplace_back(buf);
                fclose(f);
            }
        }
        const int sz = sizeof(T);
        CK(cudaMemsetAsync(done(), 0, sizeof(int), st));
        std::vector<UnitDesc> all;
        long long maxpart = 1;
        ContractPlan np[MAXN];
        int noff[MAXN] = {};
        for (int k = 0; k < sh.N; ++k) {
            std::vector<UnitDesc> u;
            np[k] = plan[k];
            if (plan[k].warp) {
                const std::string key = tune_key(k);
                WarpKnobs chosen = default_warp_knobs();
                bool cached = false;
                for (const std::string& ln : lines) {
                    if (ln.compare(0, key.size(), key) == 0 && ln.size() > key.size() && ln[key.size()] == ' ') {
                        int v[4];
                        if (sscanf(ln.c_str() + key.size(), " rpl=%d stages=%d xbytes=%d chunking=%d", &v[0], &v[1],
                                   &v[2], &v[3]) == 4) {
                            chosen.rpl = v[0];
                            chosen.stages = v[1];
                            chosen.xbytes = v[2];
                            chosen.chunking = v[3];
                            cached = true;
                        }
                    }
                }
                if (!cached && !lookup_only) {
                    std::vector<WarpKnobs> cands(1, default_warp_knobs());
                    for (int rpl : {1, 0})
                        for (int stg : {0, 2, 3})
                            for (int xb : {4096, 2048, 8192})
                                for (int ch : {0, 1, 2}) {
                                    WarpKnobs w;
                                    w.rpl = rpl;
                                    w.stages = stg;
                                    w.xbytes = xb;
                                    w.chunking = ch;
                                    cands.push_back(w);
                                }
                    std::vector<ContractPlan> cp;
                    std::vector<std::vector<UnitDesc>> cu;
                    std::vector<double> secs;
                    std::vector<int> which;
                    for (size_t c = 0; c < cands.size(); ++c) {
                        std::vector<UnitDesc> uc;
                        ContractPlan pc = plan_contract_warp(sh, k, sz, uc, cands[c]);
                        if (!pc.warp) continue;
                        bool dup = false;  // the same plan and units as a candidate timed already
                        for (size_t j = 0; j < cp.size() && !dup; ++j)
                            dup = memcmp(&cp[j], &pc, sizeof(pc)) == 0 && cu[j].size() == uc.size() &&
                                  memcmp(cu[j].data(), uc.data(), uc.size() * sizeof(UnitDesc)) == 0;
                        if (dup) continue;
                        double t = 0;
                        ifctn_status rs = time_contract(k, pc, uc, &t);
                        if (rs != IFCTN_OK) return rs;
                        ++timed;
                        cp.push_back(pc);
                        cu.push_back(uc);
                        secs.push_back(t);
                        which.push_back(static_cast<int>(c));
                    }
                    const int pick = which.empty() ? 0 : which[tune_choose(static_cast<int>(secs.size()), secs.data())];
                    chosen = cands[pick];
                    if (path && *path && !which.empty()) {
                        if (FILE* f = fopen(path, "a")) {
                            const int pi = tune_choose(static_cast<int>(secs.size()), secs.data());
                            fprintf(f, "%s rpl=%d stages=%d xbytes=%d chunking=%d seconds=%.9g default_seconds=%.9g\n",
                                    key.c_str(), chosen.rpl, chosen.stages, chosen.xbytes, chosen.chunking, secs[pi],
                                    secs[0]);
                            fclose(f);
                        }
                    }
                }
                np[k] = plan_contract_warp(sh, k, sz, u, chosen);
                if (!np[k].warp) np[k] = plan_contract(sh, k, sz, u);
            } else {
                np[k] = plan_contract(sh, k, sz, u);
            }
            noff[k] = static_cast<int>(all.size());
            all.insert(all.end(), u.begin(), u.end());
            maxpart = std::max(maxpart, np[k].part_elems);
        }
        CK(cudaStreamSynchronize(st));
        if (all.size() > units.n) {
            units.release();
            if (units.alloc(all.size()) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation failed");
                return IFCTN_ENOMEM;
            }
        }
        if (static_cast<size_t>(maxpart) > part.n) {
            part.release();
            if (part.alloc(maxpart) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation failed");
                return IFCTN_ENOMEM;
            }
        }
        if (!all.empty())
            CK(cudaMemcpyAsync(units.p, all.data(), all.size() * sizeof(UnitDesc), cudaMemcpyHostToDevice, st));
        for (int k = 0; k < sh.N; ++k) {
            plan[k] = np[k];
            unit_off[k] = noff[k];
            pp.pl[k] = plan[k];
            pp.units[k] = units.p + unit_off[k];
        }
        pp.part = part.p;
        CK(cudaStreamSynchronize(st));
        if (ntimed) *ntimed = timed;
        return build_graph();
    }

    // The whole run in one cooperative launch when the grid fits co-resident.
    void setup_persistent() {
        memset(&pp, 0, sizeof(pp));
        pp.sh = sh;
        int m[3];
        bool k_fits = true;
        for (int k = 0; k < sh.N; ++k) {
            pp.pl[k] = plan[k];
            pp.units[k] = units.p + unit_off[k];
            pp.stab[k] = stab.p + stab_off[k];
            int nm = 0;
            for (int q = 0; q < sh.N; ++q)
                if (q != k) m[nm++] = q;
            // order 3: a Gram unit takes iob values of i_o, one output per thread
            // (iob R^2 <= threads); enough of them per unit that the Gram units fit on
            // the CTAs the contraction units leave free (one work item per CTA)
            pp.gram_iob[k] = 2;
            if (nm == 2) {
                const int Io = sh.I[m[0]], Rl = sh.R[k][m[1]];
                const int free_ctas = 2 * num_sms() - plan[k].nunits;
                const int cap = std::max(2, PERSISTENT_THREADS / (Rl * Rl));
                if (free_ctas > 0) pp.gram_iob[k] = std::max(2, std::min(cap, cdiv(Io, free_ctas)));
                pp.gunits[k] = cdiv(Io, pp.gram_iob[k]);
            } else {
                pp.gunits[k] = nm == 3 ? sh.I[m[0]] : 0;
            }
            const long long Q = mode_q(sh, k);
            if (Q * k_stride(static_cast<int>(Q)) * static_cast<long long>(sizeof(T)) > 96 * 1024) k_fits = false;
        }
        pp.solve_k_in_smem = k_fits ? 1 : 0;
        int gc = 1 << 30;
        for (int k = 0; k < sh.N; ++k) {
            int nm = 0;
            for (int q = 0; q < sh.N; ++q)
                if (q != k) m[nm++] = q;
            if (nm == 3) {
                const int Rl = sh.R[k][m[2]];
                gc = std::min(gc, std::max(1, static_cast<int>(32 * 1024 / (Rl * Rl * sizeof(T)))));
            }
        }
        pp.gram_chunk = gc == (1 << 30) ? 1 : gc;
        pp.X = X.p;
        pp.mb = maskbits.p;
        pp.Xt = nullptr;
        pp.Gd = Gd.p;
        pp.Gt = Gt.p;
        pp.W = W.p;
        pp.part = part.p;
        pp.gbuf = t2.p;
        pp.Kk = Kk.p;
        for (int k = 0; k < sh.N; ++k) pp.Mk[k] = Mk[k].p;
        pp.xpart = xpart.p;
        pp.log = log.p;
        pp.log_cap = LOG_CAP;
        pp.counter = counter();
        pp.done = done();
        pp.flags = flags();
        pp.tol = tol.p;
        pp.bar_count = bar.p;
        pp.rho = prob.rho;
        pp.inv1p = 1.0 / (1.0 + prob.rho);
        pp.nmiss = nmiss;
        // One pipeline counter runs through every mode of the persistent
        // kernel, and an mbarrier's phase parity follows from it only if the
        // ring has the same number of stages in every mode: give each mode the
        // largest stage count (and the shared memory that goes with it).
        pp.nstages = 1;
        for (int k = 0; k < sh.N; ++k) pp.nstages = std::max(pp.nstages, plan[k].nstages);
        for (int k = 0; k < sh.N; ++k) {
            ContractPlan& q = pp.pl[k];
            if (q.nstages < pp.nstages) {
                const int GS = q.split ? 1 : q.G;
                q.smem += (pp.nstages - q.nstages) * GS * q.sub_elems * static_cast<int>(sizeof(T));
                q.nstages = pp.nstages;
            }
        }
        pp.tstamp = tstamp.p;
        // profiling aid: the mode whose first column is timestamped (default the last)
        pp.stamp_mode = sh.N - 1;
        if (const char* e = getenv("IFCTN_STAMP_MODE")) {
            const int v = atoi(e);
            if (v >= 0 && v < sh.N) pp.stamp_mode = v;
        }
        pp.stamp_sweep = 0;
        if (const char* e = getenv("IFCTN_STAMP_SWEEP")) pp.stamp_sweep = std::max(0, atoi(e));
        {
            // X-update work units: contiguous row ranges of 2K..16K entries,
            // about one per CTA of the persistent grid (each unit pays the
            // latency of building its row and slab factors)
            const long long target_units = 2LL * num_sms();
            const long long rows_total = static_cast<long long>(sh.nF) * sh.IA;
            long long rows = std::max<long long>(1, rows_total / target_units);
            // IFCTN_XU_ENTRIES overrides the 16K-entry cap (timing and tuning)
            long long cap = 16384;
            if (const char* e = getenv("IFCTN_XU_ENTRIES")) cap = std::max(1024LL, atoll(e));
            rows = std::max<long long>(rows, std::max(1, 2048 / sh.IB));
            rows = std::min<long long>(rows, std::max<long long>(1, cap / sh.IB));
            rows = std::min<long long>(rows, rows_total);
            pp.xu_rows = static_cast<int>(std::max<long long>(rows, 1));
            pp.xu_wab_smem = static_cast<long long>(sh.IA) * sh.IB * sizeof(T) <= 64 * 1024 ? 1 : 0;
            // 16-byte path, FP32: 4 vectors a thread in flight, 4 CTAs per SM
            // (measured on the 288x400x60x24 shape: 307 us against 341 us for the
            // generic kernel's 2 CTAs per SM); IFCTN_XU_VARIANT overrides (timing)
            pp.xu_variant = sizeof(T) == 4 ? 3 : 1;  // FP64: 8 vectors, 2 CTAs/SM (no register spill)
            if (const char* e = getenv("IFCTN_XU_VARIANT")) pp.xu_variant = std::max(0, std::min(3, atoi(e)));
        }
        psmem = persistent_smem_bytes<T>(pp);
        persistent = false;
        // One launch per run pays off when the tensor stays in L2 and the
        // phases are latency-bound; HBM-sized tensors stream better through
        // the per-stage kernels at full occupancy (graph path).
        if (graph_only) return;
        if (psmem > 227 * 1024) return;
        int g = persistent_max_grid<T>(psmem);
        if (grid_cap > 0) g = std::min(g, grid_cap);
        if (const char* e = getenv("IFCTN_GRID_CAP"))  // timing of the grid size
            if (atoi(e) > 0) g = std::min(g, atoi(e));
        if (g < 1 || 16LL * g > static_cast<long long>(xpart.n)) return;
        pgrid = g;
        persistent = true;
    }

    ifctn_status launch_run(int n) {
        NvtxRange nr("ifctn sweeps");
        if (n <= 0) return IFCTN_OK;
        if (persistent) {
            // at most 65536 sweeps a launch: the grid barrier's arrival counter
            // (zeroed before each launch) then stays far below 2^32
            for (int s0 = 0; s0 < n; s0 += 65536) {
                pp.nsweeps = std::min(65536, n - s0);
                pp.tolv = cur_tol;
                pp.Xt = (logm && truth) ? Xt.p : nullptr;
                CK(cudaMemsetAsync(bar.p, 0, 4 * sizeof(unsigned), st));
                CK(launch_persistent<T>(pp, pgrid, psmem, st));
                ++launch_count;
            }
        } else {
            for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(gexec, st));
            launch_count += static_cast<long long>(n) * launches;
        }
        return IFCTN_OK;
    }

    // seeded splitmix64 U(0,1) entries, scaled so ||iFCTN(G0)|| = ||P_Omega(O)|| / sqrt(|Omega|/P)
    ifctn_status default_factors() {
        std::vector<double> g(sh.gsize);
        uint64_t seed = prob.seed;
        for (int i = 0; i < sh.gsize; ++i) {
            uint64_t z = seed + static_cast<uint64_t>(i + 1) * 0x9E3779B97F4A7C15ULL;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
            z ^= z >> 31;
            g[i] = static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0);
        }
        CK(cudaMemcpyAsync(Gd.p, g.data(), sh.gsize * sizeof(double), cudaMemcpyHostToDevice, st));
        ifctn_status rs = refresh_factors();
        if (rs != IFCTN_OK) return rs;
        CK(launch_reconstruct<T>(sh, W.p, nullptr, xpart.p, xblocks, st));
        CK(launch_sum_partials(xpart.p, xblocks, 3, 0, scal.p, st));
        CK(launch_sumsq<T>(sh.P, X.p, xpart.p, xblocks, st));
        CK(launch_sum_partials(xpart.p, xblocks, 3, 0, scal.p + 1, st));
        double h[2];
        CK(cudaMemcpyAsync(h, scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const double rec2 = h[0], obs2 = h[1];
        if (rec2 > 0 && obs2 > 0 && nobs > 0) {
            const double target = std::sqrt(obs2 * static_cast<double>(sh.P) / static_cast<double>(nobs));
            const double ratio = target / std::sqrt(rec2);
            const double sc = std::pow(ratio, 1.0 / (sh.N * (sh.N - 1)));
            for (auto& v : g) v *= sc;
            CK(cudaMemcpyAsync(Gd.p, g.data(), sh.gsize * sizeof(double), cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));
        }
        return IFCTN_OK;
    }

    ifctn_status refresh_factors() {
        CK(launch_cast_factors<T>(sh.gsize, Gd.p, Gt.p, st));
        CK(launch_pairs<T>(sh, Gd.p, W.p, st));
        return IFCTN_OK;
    }

    // The stages of mode k on stream s: the register-resident kernels, or the
    // kernels of ifctn_wide.cu when some edge rank exceeds RMAX (t1 then holds
    // the contraction's first link, t2 the Gram's).
    cudaError_t stage_contract(int k, cudaStream_t s) {
        if (sh.wide) return launch_wide_contract<T>(sh, k, X.p, Gt.p, W.p, t1.p, done(), s);
        return launch_contract<T>(cargs(k), s);
    }
    cudaError_t stage_finish(int k, cudaStream_t s) {
        if (sh.wide) return launch_wide_finish<T>(sh, k, Gt.p, t1.p, Mk[k].p, done(), s);
        return launch_contract_finish<T>(sh, k, plan[k], units.p + unit_off[k], part.p, Gt.p, Mk[k].p, done(), s);
    }
    cudaError_t stage_gram(int k, cudaStream_t s) {
        if (sh.wide) return launch_wide_gram<T>(sh, k, Gt.p, W.p, t2.p, Kk.p, done(), s);
        return launch_gram<T>(sh, k, Gt.p, W.p, t1.p, t2.p, Kk.p, done(), s);
    }
    cudaError_t stage_solve(int k, cudaStream_t s) {
        if (cta_solve(k))
            return launch_cta_solve<T>(sh, k, prob.rho, Mk[k].p, Kk.p, Gd.p, Gt.p, W.p, flags(), done(), s);
        return launch_solve_cols<T>(pp, k, s);
    }
    // One CTA per column for ranks above RMAX; otherwise a warp per column,
    // whose mixed-precision solve runs no FP64 instruction (the CTA solve's
    // FP64 Cholesky and sums measured 3-5x slower on GB300 for the 288x400x60x24
    // shape's modes).  IFCTN_CTA_SOLVE=1 selects the CTA solve on the sweep
    // graph of order 3 and 4 (testing).
    bool cta_solve(int k) const {
        (void)k;
        if (sh.wide) return true;
        if (!graph_only || sh.N < 3) return false;
        const char* e = getenv("IFCTN_CTA_SOLVE");
        return e && strcmp(e, "1") == 0;
    }
    int mode_system_launches() const { return sh.wide ? 4 : 3; }

    ContractArgs<T> cargs(int k) {
        ContractArgs<T> a;
        a.X = X.p;
        a.Gt = Gt.p;
        a.W = W.p;
        a.sh = sh;
        a.k = k;
        a.pl = plan[k];
        a.units = units.p + unit_off[k];
        a.part = part.p;
        a.flags = flags();
        a.done = done();
        return a;
    }

    // mode-k systems: Gram on the side stream, contraction on the main one
    cudaError_t enqueue_mode_systems(int k) {
        NvtxRange r(kModeSystems[k]);
        cudaError_t e;
        if ((e = cudaEventRecord(ev_fork[k], st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ev_fork[k], 0)) != cudaSuccess) return e;
        if ((e = stage_gram(k, side)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev_join[k], side)) != cudaSuccess) return e;
        if ((e = stage_contract(k, st)) != cudaSuccess) return e;
        if ((e = stage_finish(k, st)) != cudaSuccess) return e;
        return cudaStreamWaitEvent(st, ev_join[k], 0);
    }

    cudaError_t enqueue_sweep() {
        cudaError_t e;
        for (int k = 0; k < sh.N; ++k) {
            if ((e = enqueue_mode_systems(k)) != cudaSuccess) return e;
            NvtxRange r(kModeSolves[k]);
            if ((e = stage_solve(k, st)) != cudaSuccess) return e;
        }
        NvtxRange r("ifctn X update");
        pp.Xt = (logm && truth) ? Xt.p : nullptr;
        const int xb = slab_xblocks();
        if ((e = launch_xupdate_slab<T>(pp, xpart.p, xb, st)) != cudaSuccess) return e;
        return launch_finalize8(xpart.p, xb, (logm && truth) ? 1 : 0, nmiss, tol.p, log.p, LOG_CAP, counter(),
                                done(), flags(), st);
    }

    int slab_xblocks() const { return static_cast<int>(std::min<long long>(xpart.n / 8, 8LL * num_sms())); }

    // kernel launches of one sweep: the kernel nodes of its captured graph
    static int count_kernel_nodes(cudaGraph_t g) {
        size_t n = 0;
        if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
        std::vector<cudaGraphNode_t> nodes(n);
        if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
        int kn = 0;
        for (size_t i = 0; i < n; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
        }
        return kn;
    }
    int kernels_per_sweep() const override { return launches; }

    // Turns every kernel-to-kernel edge of the captured sweep graph into a
    // programmatic one (the downstream kernel may launch once every block of
    // the upstream one has started; it waits in griddepcontrol.wait for the
    // upstream kernel's completion and writes before it reads anything), so
    // consecutive kernels' launch latencies overlap.  IFCTN_PDL=0 keeps the
    // ordinary edges (timing).  Returns false if the graph could not be
    // restored to a consistent state.
    static bool programmatic_edges(cudaGraph_t g) {
        if (const char* v = getenv("IFCTN_PDL"))
            if (strcmp(v, "0") == 0) return true;
        size_t ne = 0;
        if (cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &ne) != cudaSuccess || ne == 0) {
            cudaGetLastError();
            return true;
        }
        std::vector<cudaGraphNode_t> from(ne), to(ne);
        std::vector<cudaGraphEdgeData> ed(ne);
        if (cudaGraphGetEdges(g, from.data(), to.data(), ed.data(), &ne) != cudaSuccess) {
            cudaGetLastError();
            return true;
        }
        for (size_t i = 0; i < ne; ++i) {
            cudaGraphNodeType tf, tt;
            if (cudaGraphNodeGetType(from[i], &tf) != cudaSuccess || cudaGraphNodeGetType(to[i], &tt) != cudaSuccess)
                return false;
            if (tf != cudaGraphNodeTypeKernel || tt != cudaGraphNodeTypeKernel) continue;
            if (ed[i].type != cudaGraphDependencyTypeDefault || ed[i].from_port != 0) continue;
            cudaGraphEdgeData pe;
            memset(&pe, 0, sizeof(pe));
            pe.from_port = cudaGraphKernelNodePortProgrammatic;
            pe.type = cudaGraphDependencyTypeProgrammatic;
            if (cudaGraphRemoveDependencies(g, &from[i], &to[i], &ed[i], 1) != cudaSuccess) {
                cudaGetLastError();
                continue;  // the ordinary edge is still there
            }
            if (cudaGraphAddDependencies(g, &from[i], &to[i], &pe, 1) != cudaSuccess) {
                cudaGetLastError();
                if (cudaGraphAddDependencies(g, &from[i], &to[i], &ed[i], 1) != cudaSuccess) return false;
            }
        }
        return true;
    }

    ifctn_status build_graph() {
        if (gexec) {
            cudaGraphExecDestroy(gexec);
            gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_sweep();
        cudaError_t e2 = cudaStreamEndCapture(st, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            set_error(std::string("sweep capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
            return IFCTN_ECUDA;
        }
        launches = count_kernel_nodes(g);
        if (!programmatic_edges(g)) {
            cudaGraphDestroy(g);
            cudaGetLastError();
            set_error("could not make the sweep graph's kernel edges programmatic");
            return IFCTN_ECUDA;
        }
        e = cudaGraphInstantiate(&gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
            return IFCTN_ECUDA;
        }
        return IFCTN_OK;
    }

    // Reports a failure recorded by a kernel once: the flag word is cleared
    // when it is read, so the context can be used again (its state is that of
    // the interrupted call; set_factors / set_x restore a checkpoint).
    ifctn_status check_flags() {
        int f[3];
        CK(cudaMemcpyAsync(f, ints.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (f[2] & (FLAG_TIMEOUT | FLAG_NOTSPD)) {
            CK(cudaMemsetAsync(flags(), 0, sizeof(int), st));
            CK(cudaStreamSynchronize(st));
        }
        if (f[2] & FLAG_TIMEOUT) {
            set_error("a bounded device wait expired");
            return IFCTN_ETIMEOUT;
        }
        if (f[2] & FLAG_NOTSPD) {
            set_error("a proximal normal-equation matrix was not positive definite");
            return IFCTN_ENOTSPD;
        }
        return IFCTN_OK;
    }

    ifctn_status last_stats(ifctn_stats* out) {
        int cnt = 0;
        CK(cudaMemcpyAsync(&cnt, counter(), sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (!out) return IFCTN_OK;
        memset(out, 0, sizeof(*out));
        out->rel_change = out->objective = out->rse = out->rmse = NAN;
        if (cnt == 0) return IFCTN_OK;
        SweepStat r;
        CK(cudaMemcpy(&r, log.p + ((cnt - 1) % LOG_CAP), sizeof(r), cudaMemcpyDeviceToHost));
        out->sweeps_done = r.sweep;
        out->converged = r.converged;
        out->rel_change = r.rel_change;
        out->objective = r.objective;
        out->rse = r.rse;
        out->rmse = r.rmse;
        return IFCTN_OK;
    }

    ifctn_status run(int n, double tolv, ifctn_stats* out) {
        if (n < 0) {
            set_error("n must be >= 0");
            return IFCTN_EINVAL;
        }
        CK(cudaMemcpyAsync(tol.p, &tolv, sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(done(), 0, sizeof(int), st));
        cur_tol = tolv;
        const int chunkn = (tolv > 0 && !persistent) ? 16 : (1 << 30);
        int doneh = 0;
        for (int s = 0; s < n;) {
            const int m = std::min(chunkn, n - s);
            ifctn_status rs0 = launch_run(m);
            if (rs0 != IFCTN_OK) return rs0;
            s += m;
            if (tolv > 0 && s < n) {
                CK(cudaMemcpyAsync(&doneh, done(), sizeof(int), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (doneh) break;
            }
        }
        ifctn_status rs = check_flags();
        if (rs != IFCTN_OK) return rs;
        return last_stats(out);
    }

    ifctn_status sweep(int n, ifctn_stats* out) override { return run(n, 0.0, out); }

    ifctn_status enqueue(int n, double tolv, bool reset) override {
        if (reset) {
            CK(cudaMemcpyAsync(tol.p, &tolv, sizeof(double), cudaMemcpyHostToDevice, st));
            CK(cudaMemsetAsync(done(), 0, sizeof(int), st));
            cur_tol = tolv;
        }
        return launch_run(n);
    }
    cudaStream_t stream() const override { return st; }
    long long launch_total() const override { return launch_count; }
    ifctn_status phase_times(double* out, int max, int* n) override {
        std::vector<unsigned long long> h(64 + 4 * 512);
        CK(cudaMemcpyAsync(h.data(), tstamp.p, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        auto rel = [&](unsigned long long t) {
            return (t >= h[0] && h[0]) ? 1e-9 * static_cast<double>(t - h[0]) : NAN;
        };
        int cnt = 0;
        for (int i = 0; i < 26 && cnt < max; ++i) out[cnt++] = rel(h[i + 1]);
        // then, per mode, the latest per-CTA end of phase 1 and the mean
        for (int k = 0; k < sh.N && cnt + 1 < max; ++k) {
            double mx = 0, sm = 0;
            int c = 0;
            for (int b = 0; b < std::min(pgrid, 512); ++b) {
                const double v = rel(h[64 + k * 512 + b]);
                if (v == v) {
                    mx = std::max(mx, v);
                    sm += v;
                    ++c;
                }
            }
            out[cnt++] = mx;
            out[cnt++] = c ? sm / c : NAN;
        }
        // sub-steps of the profiled mode's first column solve, then of its
        // reduction phase (CTA 0)
        for (int i = 40; i < 56 && cnt < max; ++i) out[cnt++] = rel(h[i]);
        if (n) *n = persistent ? cnt : 0;
        return IFCTN_OK;
    }
    int batch_kind() const override { return persistent ? static_cast<int>(sizeof(T)) : 0; }

    // Prepares n sweeps of this context for a launch shared with other jobs:
    // the per-launch state (grid-barrier counter) is reset on stream bst, and
    // *out receives the launch parameters for the CTA slice [cta0, cta0 + ncta).
    ifctn_status batch_prepare(int n, cudaStream_t bst, int cta0, int ncta, SweepParams<T>* out) {
        pp.nsweeps = n;
        pp.tolv = cur_tol;
        pp.Xt = (logm && truth) ? Xt.p : nullptr;
        CK(cudaMemsetAsync(bar.p, 0, 4 * sizeof(unsigned), bst));
        *out = pp;
        out->cta0 = cta0;
        out->ncta = ncta;
        ++launch_count;
        return IFCTN_OK;
    }

    void set_grid_cap(int g) override {
        grid_cap = g;
        setup_persistent();
        build_graph();
    }

    ifctn_status launch_stage(int stage, int k) override {
        if (k < 0 || k >= sh.N) {
            set_error("mode out of range");
            return IFCTN_EINVAL;
        }
        switch (stage) {
            case 0: CK(stage_contract(k, st)); break;
            case 1: CK(stage_gram(k, st)); break;
            case 2: CK(stage_solve(k, st)); break;
            case 3: CK(launch_xupdate_slab<T>(pp, xpart.p, slab_xblocks(), st)); break;
            case 4: CK(stage_finish(k, st)); break;
            default: set_error("unknown stage"); return IFCTN_EINVAL;
        }
        return IFCTN_OK;
    }

    // n sweeps of a slab of a tensor split along its first mode (see
    // ifctn_sweep_exchange): the per-stage kernels, with the partial M_k and
    // K_k of every mode k >= 1 and the stop-test sums combined by `fn`.
    ifctn_status sweep_exchange(int n, ifctn_allreduce_fn fn, void* user, ifctn_stats* out) override {
        if (n < 0 || !fn) {
            set_error(n < 0 ? "n must be >= 0" : "null allreduce function");
            return IFCTN_EINVAL;
        }
        CK(cudaMemsetAsync(done(), 0, sizeof(int), st));
        long long need = 8;
        for (int k = 1; k < sh.N; ++k) {
            const long long Q = mode_q(sh, k);
            need = std::max(need, static_cast<long long>(sh.I[k]) * Q + Q * Q);
        }
        if (tmpD.n < static_cast<size_t>(need)) {
            tmpD.release();
            if (tmpD.alloc(need) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation failed");
                return IFCTN_ENOMEM;
            }
        }
        std::vector<double> hb(need);
        std::vector<T> kt;
        double sums[3] = {0, 0, 0};
        NvtxRange nr("ifctn sharded sweeps");
        for (int s_ = 0; s_ < n; ++s_) {
            for (int k = 0; k < sh.N; ++k) {
                NvtxRange mr(kModeSystems[k]);
                CK(stage_contract(k, st));
                CK(stage_finish(k, st));
                CK(stage_gram(k, st));
                launch_count += mode_system_launches();
                if (k > 0) {  // M_k and K_k are sums over the slab's entries: combine them
                    const long long Q = mode_q(sh, k), nm = static_cast<long long>(sh.I[k]) * Q;
                    CK(cudaMemcpyAsync(hb.data(), Mk[k].p, nm * sizeof(double), cudaMemcpyDeviceToHost, st));
                    if (sizeof(T) == sizeof(double)) {
                        CK(cudaMemcpyAsync(hb.data() + nm, Kk.p, Q * Q * sizeof(double), cudaMemcpyDeviceToHost, st));
                    } else {
                        CK(launch_to_double(Q * Q, reinterpret_cast<const float*>(Kk.p), tmpD.p, st));
                        CK(cudaMemcpyAsync(hb.data() + nm, tmpD.p, Q * Q * sizeof(double), cudaMemcpyDeviceToHost, st));
                        ++launch_count;
                    }
                    CK(cudaStreamSynchronize(st));
                    NvtxRange xr("ifctn exchange");
                    if (fn(user, hb.data(), nm + Q * Q) != 0) {
                        set_error("the allreduce function failed");
                        return IFCTN_EINVAL;
                    }
                    CK(cudaMemcpyAsync(Mk[k].p, hb.data(), nm * sizeof(double), cudaMemcpyHostToDevice, st));
                    kt.assign(Q * Q, T(0));
                    for (long long i = 0; i < Q * Q; ++i) kt[i] = static_cast<T>(hb[nm + i]);
                    CK(cudaMemcpyAsync(Kk.p, kt.data(), Q * Q * sizeof(T), cudaMemcpyHostToDevice, st));
                    CK(cudaStreamSynchronize(st));  // kt and hb are reused
                }
                CK(stage_solve(k, st));
                ++launch_count;
            }
            CK(launch_xupdate_slab<T>(pp, xpart.p, slab_xblocks(), st));
            for (int t = 0; t < 3; ++t) CK(launch_sum_partials(xpart.p, slab_xblocks(), 8, t, scal.p + t, st));
            launch_count += 4;
            CK(cudaMemcpyAsync(sums, scal.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (fn(user, sums, 3) != 0) {
                set_error("the allreduce function failed");
                return IFCTN_EINVAL;
            }
            ++ex_sweeps;
        }
        ifctn_status rs = check_flags();
        if (rs != IFCTN_OK) return rs;
        if (out) {
            memset(out, 0, sizeof(*out));
            out->sweeps_done = ex_sweeps;
            out->rel_change = sums[1] > 0 ? std::sqrt(sums[0]) / std::sqrt(sums[1]) : (sums[0] > 0 ? INFINITY : 0.0);
            out->objective = 0.5 * sums[2];
            out->rse = out->rmse = NAN;
            if (n == 0) out->rel_change = out->objective = NAN;
        }
        return IFCTN_OK;
    }

    ifctn_status wait_selftest(long long budget) override {
        CK(cudaMemsetAsync(bar.p, 0, sizeof(unsigned), st));
        CK(launch_wait_selftest(flags(), bar.p, budget, st));
        CK(cudaStreamSynchronize(st));
        return check_flags();
    }

    ifctn_status complete(void* out_X, ifctn_stats* out) override {
        ifctn_status rs = run(prob.max_sweeps, prob.tol, out);
        if (rs != IFCTN_OK) return rs;
        if (out_X) return get_x(out_X);
        return IFCTN_OK;
    }

    ifctn_status reconstruct(void* out) override {
        if (!out) {
            set_error("null output");
            return IFCTN_EINVAL;
        }
        T* dst = nullptr;
        CK(cudaMallocAsync(reinterpret_cast<void**>(&dst), sh.P * sizeof(T), st));
        CK(launch_reconstruct<T>(sh, W.p, dst, nullptr, xblocks, st));
        CK(cudaMemcpyAsync(out, dst, sh.P * sizeof(T), cudaMemcpyDefault, st));
        CK(cudaFreeAsync(dst, st));
        CK(cudaStreamSynchronize(st));
        return IFCTN_OK;
    }

    ifctn_status get_factors(double* out) override {
        if (!out) return IFCTN_EINVAL;
        CK(cudaMemcpyAsync(out, Gd.p, sh.gsize * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
        return IFCTN_OK;
    }

    ifctn_status set_factors(const double* in) override {
        if (!in) return IFCTN_EINVAL;
        CK(cudaMemcpyAsync(Gd.p, in, sh.gsize * sizeof(double), cudaMemcpyDefault, st));
        ifctn_status rs = refresh_factors();
        if (rs != IFCTN_OK) return rs;
        CK(cudaStreamSynchronize(st));
        return IFCTN_OK;
    }

    ifctn_status get_x(void* out) override {
        if (!out) return IFCTN_EINVAL;
        CK(cudaMemcpyAsync(out, X.p, sh.P * sizeof(T), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
        return IFCTN_OK;
    }

    ifctn_status set_x(const void* in) override {
        if (!in) return IFCTN_EINVAL;
        CK(cudaMemcpyAsync(X.p, in, sh.P * sizeof(T), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
        return IFCTN_OK;
    }

    ifctn_status set_truth(const void* xt, int lg) override {
        if (xt) {
            if (!Xt.p && alloc(Xt, sh.P) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation failed");
                return IFCTN_ENOMEM;
            }
            CK(cudaMemcpyAsync(Xt.p, xt, sh.P * sizeof(T), cudaMemcpyDefault, st));
            truth = true;
        }
        logm = lg != 0;
        CK(cudaStreamSynchronize(st));
        pp.Xt = (logm && truth) ? Xt.p : nullptr;
        return build_graph();
    }

    ifctn_status get_log(ifctn_stats* out, int max, int* n) override {
        int cnt = 0;
        CK(cudaMemcpyAsync(&cnt, counter(), sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const int avail = std::min(cnt, LOG_CAP);
        const int take = std::max(0, std::min(avail, max));
        std::vector<SweepStat> h(LOG_CAP);
        CK(cudaMemcpy(h.data(), log.p, LOG_CAP * sizeof(SweepStat), cudaMemcpyDeviceToHost));
        const int first = cnt - avail;
        for (int i = 0; i < take; ++i) {
            const SweepStat& r = h[(first + i) % LOG_CAP];
            out[i].sweeps_done = r.sweep;
            out[i].converged = r.converged;
            out[i].rel_change = r.rel_change;
            out[i].objective = r.objective;
            out[i].rse = r.rse;
            out[i].rmse = r.rmse;
        }
        if (n) *n = take;
        return IFCTN_OK;
    }

    ifctn_status mode_system(int k, double* Mout, double* Kout) override {
        if (k < 0 || k >= sh.N) {
            set_error("mode out of range");
            return IFCTN_EINVAL;
        }
        CK(cudaMemsetAsync(done(), 0, sizeof(int), st));
        CK(enqueue_mode_systems(k));
        const int Q = mode_q(sh, k);
        if (Mout) CK(cudaMemcpyAsync(Mout, Mk[k].p, static_cast<size_t>(sh.I[k]) * Q * sizeof(double),
                                     cudaMemcpyDefault, st));
        if (Kout) {
            if (sizeof(T) == sizeof(double)) {
                CK(cudaMemcpyAsync(Kout, Kk.p, static_cast<size_t>(Q) * Q * sizeof(double), cudaMemcpyDefault, st));
            } else {
                double* tmp = nullptr;
                CK(cudaMallocAsync(reinterpret_cast<void**>(&tmp), static_cast<size_t>(Q) * Q * sizeof(double), st));
                CK(launch_to_double(static_cast<long long>(Q) * Q, reinterpret_cast<const float*>(Kk.p), tmp, st));
                CK(cudaMemcpyAsync(Kout, tmp, static_cast<size_t>(Q) * Q * sizeof(double), cudaMemcpyDefault, st));
                CK(cudaFreeAsync(tmp, st));
            }
        }
        CK(cudaStreamSynchronize(st));
        return check_flags();
    }
};

template struct Engine<float>;
template struct Engine<double>;

namespace {

template <typename T>
ifctn_status make_engine(const ifctn_problem* prob, const void* obs, const uint8_t* mask, const double* init,
                         void* stream, bool tune_timing, int force_path, Engine<T>** out) {
    auto* e = new Engine<T>();
    e->tune_timing = tune_timing;
    e->force_path = force_path;
    const ifctn_status rs = e->init(prob, obs, mask, init, stream);
    if (rs != IFCTN_OK) {
        delete e;
        *out = nullptr;
        return rs;
    }
    *out = e;
    return IFCTN_OK;
}

// Cache key of the execution-path choice of a shape (see create_ctx).
std::string path_key(const Shape& sh, int sz) {
    std::string key = std::string("ifctn-tune-v1 ") + IFCTN_SOURCE_DIGEST + (sz == 4 ? " f32 " : " f64 ");
    key += "N" + std::to_string(sh.N);
    for (int m = 0; m < sh.N; ++m) key += "," + std::to_string(sh.I[m]);
    key += " R";
    for (int p2 = 0; p2 < sh.N; ++p2)
        for (int q = p2 + 1; q < sh.N; ++q) key += std::to_string(sh.R[p2][q]) + ".";
    key += " path sms" + std::to_string(num_sms());
    return key;
}

// The execution path of a tensor that fits the persistent launch's L2 rule:
// with a tuning cache (IFCTN_TUNE_CACHE), the cached choice for the shape, or,
// where the cache has none and timing is allowed, both paths are built, 10
// sweeps of each are timed from the same initial state after 10 warm-up
// ones, the faster context is kept (its state restored) and the choice is
// appended to the cache.  IFCTN_PATH overrides everything.
template <typename T>
ifctn_status create_tuned(const ifctn_problem* prob, const void* obs, const uint8_t* mask, const double* init,
                          void* stream, bool tune_timing, ifctn_ctx** out) {
    Shape sh;
    ifctn_status rs = build_shape(prob, sh);
    if (rs != IFCTN_OK) return rs;
    const int sz = static_cast<int>(sizeof(T));
    const char* cache = getenv("IFCTN_TUNE_CACHE");
    int force = 0;
    if (!getenv("IFCTN_PATH") && cache && *cache && !sh.wide && !choose_graph_only(sh, sz)) {
        const std::string key = path_key(sh, sz);
        if (FILE* f = fopen(cache, "r")) {
            char buf[1024];
            while (fgets(buf, sizeof(buf), f)) {
                const std::string ln(buf);
                if (ln.compare(0, key.size(), key) == 0 && ln.size() > key.size() && ln[key.size()] == ' ') {
                    if (ln.find(" path=graph") != std::string::npos) force = 1;
                    if (ln.find(" path=persistent") != std::string::npos) force = 2;
                }
            }
            fclose(f);
        }
        if (!force && tune_timing) {
            Engine<T>* a = nullptr;
            Engine<T>* g = nullptr;
            rs = make_engine<T>(prob, obs, mask, init, stream, true, 2, &a);
            if (rs != IFCTN_OK) return rs;
            rs = make_engine<T>(prob, obs, mask, init, stream, true, 1, &g);
            if (rs != IFCTN_OK) {
                delete a;
                return rs;
            }
            double ta = 0, tg = 0;
            rs = a->time_sweeps(10, &ta);
            if (rs == IFCTN_OK) rs = g->time_sweeps(10, &tg);
            if (rs != IFCTN_OK) {
                delete a;
                delete g;
                return rs;
            }
            // the size rule's choice (persistent) stays unless the graph beats it by 2 %
            const bool graph = tg <= 0.98 * ta;
            if (FILE* f = fopen(cache, "a")) {
                fprintf(f, "%s path=%s seconds_persistent=%.9g seconds_graph=%.9g\n", key.c_str(),
                        graph ? "graph" : "persistent", ta / 10, tg / 10);
                fclose(f);
            }
            if (graph) {
                delete a;
                *out = g;
            } else {
                delete g;
                *out = a;
            }
            return IFCTN_OK;
        }
    }
    Engine<T>* e = nullptr;
    rs = make_engine<T>(prob, obs, mask, init, stream, tune_timing, force, &e);
    if (rs != IFCTN_OK) return rs;
    *out = e;
    return IFCTN_OK;
}

}  // namespace

ifctn_status create_ctx(const ifctn_problem* prob, const void* obs, const uint8_t* mask, const double* init,
                        void* stream, ifctn_ctx** out, bool tune_timing) {
    if (!out || !prob) {
        set_error("null argument");
        return IFCTN_EINVAL;
    }
    *out = nullptr;
    if (prob->precision == IFCTN_FP64) return create_tuned<double>(prob, obs, mask, init, stream, tune_timing, out);
    return create_tuned<float>(prob, obs, mask, init, stream, tune_timing, out);
}

size_t ctx_device_bytes(const ifctn_ctx* c) { return c ? c->device_bytes() : 0; }
int ctx_batch_kind(const ifctn_ctx* c) { return c ? c->batch_kind() : 0; }

namespace {

// One cooperative launch that runs ns[i] sweeps of each persistent-path
// context ctxs[i] (all of the same dtype) on its own slice of the grid.  Every
// job gets at least one CTA and at most its own full-launch grid, the rest in
// proportion to its tensor size; the kernel and the per-job arithmetic are
// those of the job's own launch, whose results do not depend on the grid size.
template <typename T>
ifctn_status run_batch_t(ifctn_ctx* const* ctxs, const int* ns, int nj, cudaStream_t bst) {
    std::vector<Engine<T>*> es(nj);
    int smem = 0;
    double wsum = 0;
    for (int i = 0; i < nj; ++i) {
        es[i] = static_cast<Engine<T>*>(ctxs[i]);
        smem = std::max(smem, es[i]->psmem);
        wsum += static_cast<double>(es[i]->sh.P);
    }
    const int gmax = persistent_multi_max_grid<T>(smem);
    if (gmax < nj) {
        set_error("a batched launch cannot give every job a CTA");
        return IFCTN_ECUDA;
    }
    std::vector<int> nc(nj);
    int used = 0;
    for (int i = 0; i < nj; ++i) {
        const double share = static_cast<double>(es[i]->sh.P) / wsum;
        nc[i] = std::max(1, std::min(es[i]->pgrid, static_cast<int>(share * (gmax - nj)) + 1));
        used += nc[i];
    }
    while (used > gmax) {  // the +1 floors can overshoot by a few CTAs
        int big = 0;
        for (int i = 1; i < nj; ++i)
            if (nc[i] > nc[big]) big = i;
        --nc[big];
        --used;
    }
    std::vector<SweepParams<T>> hp(nj);
    int c0 = 0;
    for (int i = 0; i < nj; ++i) {
        ifctn_status rs = es[i]->batch_prepare(ns[i], bst, c0, nc[i], &hp[i]);
        if (rs != IFCTN_OK) return rs;
        c0 += nc[i];
    }
    SweepParams<T>* dp = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&dp), nj * sizeof(SweepParams<T>), bst));
    CK(cudaMemcpyAsync(dp, hp.data(), nj * sizeof(SweepParams<T>), cudaMemcpyHostToDevice, bst));
    const cudaError_t e = launch_persistent_multi<T>(dp, nj, c0, smem, bst);
    cudaFreeAsync(dp, bst);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("batched persistent launch failed: ") + cudaGetErrorString(e));
        return IFCTN_ECUDA;
    }
    // the host copy of the parameters must outlive the asynchronous upload
    CK(cudaStreamSynchronize(bst));
    return IFCTN_OK;
}

}  // namespace

ifctn_status ctx_run_batch(ifctn_ctx* const* ctxs, const int* nsweeps, int njobs, cudaStream_t bst) {
    if (njobs <= 0) return IFCTN_OK;
    const int kind = ctxs[0]->batch_kind();
    for (int i = 1; i < njobs; ++i)
        if (ctxs[i]->batch_kind() != kind) {
            set_error("a batched launch needs jobs of one dtype on the persistent path");
            return IFCTN_EINVAL;
        }
    if (kind == 4) return run_batch_t<float>(ctxs, nsweeps, njobs, bst);
    if (kind == 8) return run_batch_t<double>(ctxs, nsweeps, njobs, bst);
    set_error("a batched launch needs contexts on the persistent path");
    return IFCTN_EINVAL;
}
ifctn_status ctx_enqueue(ifctn_ctx* c, int n, double tol, bool reset) { return c->enqueue(n, tol, reset); }
void ctx_set_grid_cap(ifctn_ctx* c, int g) { c->set_grid_cap(g); }
cudaStream_t ctx_stream(ifctn_ctx* c) { return c->stream(); }

}  // namespace ifctn

extern "C" {

ifctn_status ifctn_create(const ifctn_problem* prob, const void* obs, const uint8_t* mask,
                          const double* init_factors, void* cuda_stream, ifctn_ctx** out) {
    g_last_error.clear();
    return create_ctx(prob, obs, mask, init_factors, cuda_stream, out, true);
}

#define IFCTN_CTX_CALL(ctx, expr)          \
    do {                                   \
        if (!(ctx)) {                      \
            set_error("null context");     \
            return IFCTN_EINVAL;           \
        }                                  \
        return (ctx)->expr;                \
    } while (0)

ifctn_status ifctn_sweep(ifctn_ctx* ctx, int32_t n, ifctn_stats* out) { IFCTN_CTX_CALL(ctx, sweep(n, out)); }
ifctn_status ifctn_complete(ifctn_ctx* ctx, void* out_X, ifctn_stats* out) {
    IFCTN_CTX_CALL(ctx, complete(out_X, out));
}
ifctn_status ifctn_reconstruct(ifctn_ctx* ctx, void* out) { IFCTN_CTX_CALL(ctx, reconstruct(out)); }
ifctn_status ifctn_get_factors(ifctn_ctx* ctx, double* out) { IFCTN_CTX_CALL(ctx, get_factors(out)); }
ifctn_status ifctn_set_factors(ifctn_ctx* ctx, const double* in) { IFCTN_CTX_CALL(ctx, set_factors(in)); }
ifctn_status ifctn_get_x(ifctn_ctx* ctx, void* out) { IFCTN_CTX_CALL(ctx, get_x(out)); }
ifctn_status ifctn_set_x(ifctn_ctx* ctx, const void* in) { IFCTN_CTX_CALL(ctx, set_x(in)); }
ifctn_status ifctn_set_truth(ifctn_ctx* ctx, const void* xt, int32_t log) { IFCTN_CTX_CALL(ctx, set_truth(xt, log)); }
ifctn_status ifctn_get_log(ifctn_ctx* ctx, ifctn_stats* out, int32_t max, int32_t* n) {
    IFCTN_CTX_CALL(ctx, get_log(out, max, n));
}
ifctn_status ifctn_mode_system(ifctn_ctx* ctx, int32_t k, double* Mk, double* Kk) {
    IFCTN_CTX_CALL(ctx, mode_system(k, Mk, Kk));
}
int32_t ifctn_kernels_per_sweep(const ifctn_ctx* ctx) { return ctx ? ctx->kernels_per_sweep() : 0; }
int64_t ifctn_launch_count(const ifctn_ctx* ctx) { return ctx ? ctx->launch_total() : 0; }
ifctn_status ifctn_phase_times(ifctn_ctx* ctx, double* out, int32_t max, int32_t* n) {
    IFCTN_CTX_CALL(ctx, phase_times(out, max, n));
}
ifctn_status ifctn_sweep_async(ifctn_ctx* ctx, int32_t n) {
    if (n < 0) {
        set_error("n must be >= 0");
        return IFCTN_EINVAL;
    }
    IFCTN_CTX_CALL(ctx, enqueue(n, 0.0, true));
}
ifctn_status ifctn_launch_stage(ifctn_ctx* ctx, int32_t stage, int32_t k) {
    IFCTN_CTX_CALL(ctx, launch_stage(stage, k));
}
ifctn_status ifctn_sweep_exchange(ifctn_ctx* ctx, int32_t n, ifctn_allreduce_fn allreduce, void* user,
                                  ifctn_stats* out) {
    IFCTN_CTX_CALL(ctx, sweep_exchange(n, allreduce, user, out));
}
ifctn_status ifctn_tune(ifctn_ctx* ctx, const char* cache_path, int32_t* timed) {
    int t = 0;
    if (!ctx) {
        set_error("null context");
        return IFCTN_EINVAL;
    }
    const ifctn_status rs = ctx->tune(cache_path, &t);
    if (timed) *timed = t;
    return rs;
}
int32_t ifctn_tune_choose(int32_t n, const double* seconds) {
    if (n <= 0 || !seconds) return -1;
    return ifctn::tune_choose(n, seconds);
}
ifctn_status ifctn_wait_selftest(ifctn_ctx* ctx, int64_t budget_cycles) {
    if (budget_cycles < 1000 || budget_cycles > ifctn::WAIT_BUDGET_CYCLES) {
        set_error("budget_cycles must be in 1000..4e9");
        return IFCTN_EINVAL;
    }
    IFCTN_CTX_CALL(ctx, wait_selftest(budget_cycles));
}
void ifctn_destroy(ifctn_ctx* ctx) { delete ctx; }
const char* ifctn_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
