// ifctn_server.cu -- continuous batching of completion jobs on one GPU.
//
// Jobs are queued in arrival order.  A scheduler thread admits the head of
// the queue as soon as a slot and enough of the device-memory budget are
// free, gives every resident job its own CUDA stream and sweep graph, and
// keeps a few sweeps of every resident job in flight so that the kernels of
// different jobs overlap on the device.  A finished job's tensor is copied to
// pinned host memory and its memory returns to the budget immediately, which
// admits the next queued job while the others keep running.  Each job runs
// exactly the kernels (same plans, same reduction order) it would run alone,
// so its result does not depend on what else is resident.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ifctn.h"
#include "ifctn_api_internal.h"
#include "ifctn_launch.h"

using namespace ifctn;
using Clock = std::chrono::steady_clock;

namespace {

enum JobState { QUEUED, RESIDENT, FINISHING, DONE, FAILED };

struct Job {
    uint64_t ticket = 0;
    ifctn_problem prob;
    size_t P = 0, esz = 0;
    void* obs = nullptr;       // pinned host copies of the inputs
    uint8_t* mask = nullptr;
    double* init = nullptr;
    void* result = nullptr;    // pinned host result
    ifctn_ctx* ctx = nullptr;
    cudaEvent_t ev = nullptr;
    int enqueued = 0;
    bool batch_pending = false;  // part of the shared launch in flight
    size_t bytes = 0;
    JobState state = QUEUED;
    ifctn_status err = IFCTN_OK;
    std::string msg;
    ifctn_stats stats;
    Clock::time_point t_submit, t_done;
};

size_t job_bytes_estimate(const Shape& s, size_t esz) {
    // X, the transient observation copy and mask bytes, the bitset, plus slack
    size_t b = static_cast<size_t>(s.P) * (2 * esz + 1) + static_cast<size_t>(s.P) / 8 + (8u << 20);
    if (s.wide) {  // ranks above 8: K_k (Q_k^2), M_k (FP64) and the chain buffers grow with Q_k
        size_t kmax = 0, chain = 0;
        for (int k = 0; k < s.N; ++k) {
            const size_t Q = static_cast<size_t>(mode_q(s, k));
            b += static_cast<size_t>(s.I[k]) * Q * 8;
            kmax = std::max(kmax, Q * Q);
            chain = std::max(chain, static_cast<size_t>(wide_v_elems(s, k)) + static_cast<size_t>(wide_t_elems(s, k)));
        }
        b += (kmax + chain) * esz;
    }
    return b;
}

void free_pinned(Job& j) {
    if (j.obs) cudaFreeHost(j.obs);
    if (j.mask) cudaFreeHost(j.mask);
    if (j.init) cudaFreeHost(j.init);
    j.obs = nullptr;
    j.mask = nullptr;
    j.init = nullptr;
}

}  // namespace

struct ifctn_server {
    size_t budget = 0;
    int max_slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::vector<std::shared_ptr<Job>> resident;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    std::map<uint64_t, double> latency;
    uint64_t next_ticket = 1;
    size_t in_use = 0;
    int64_t completed = 0, peak_resident = 0;
    int64_t batch_launches = 0, batched_jobs = 0;
    bool stop = false;
    std::thread worker;
    // jobs whose sweeps run as one persistent launch share one cooperative
    // launch per round, on this stream, each on its own slice of the grid
    cudaStream_t bst = nullptr;
    cudaEvent_t bev = nullptr;
    bool batch_inflight = false;
    std::vector<std::shared_ptr<Job>> batch_members;

    void run();
    void admit_locked_unlock(std::unique_lock<std::mutex>& lk);
};

void ifctn_server::run() {
    cudaSetDevice(device);
    const int kInflight = 4;  // sweeps kept queued per resident job
    const int kRound = 4;     // sweeps of every job in one shared persistent launch
    cudaStreamCreateWithFlags(&bst, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&bev, cudaEventDisableTiming);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        // 1. admission, in arrival order
        while (!queue.empty() && static_cast<int>(resident.size()) < max_slots &&
               in_use + queue.front()->bytes <= budget) {
            std::shared_ptr<Job> j = queue.front();
            queue.pop_front();
            in_use += j->bytes;
            lk.unlock();
            ifctn_ctx* c = nullptr;
            ifctn_status rs = create_ctx(&j->prob, j->obs, j->mask, j->init, nullptr, &c, false);
            if (rs == IFCTN_OK) rs = ctx_enqueue(c, 0, j->prob.tol, true);
            // a job of the shared launches runs on the server's stream: its own
            // stream's set-up must be complete first
            if (rs == IFCTN_OK && ctx_batch_kind(c) && cudaStreamSynchronize(ctx_stream(c)) != cudaSuccess)
                rs = IFCTN_ECUDA;
            if (rs == IFCTN_OK && cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess)
                rs = IFCTN_ECUDA;
            lk.lock();
            if (rs != IFCTN_OK) {
                j->err = rs;
                j->msg = ifctn_last_error();
                j->state = FAILED;
                if (c) {
                    lk.unlock();
                    ifctn_destroy(c);
                    lk.lock();
                }
                in_use -= j->bytes;
                j->t_done = Clock::now();
                free_pinned(*j);
                cv_done.notify_all();
                continue;
            }
            // reserve the larger of the estimate and the measured footprint
            const size_t real = std::max(ctx_device_bytes(c), j->bytes);
            in_use = in_use - j->bytes + real;
            j->bytes = real;
            j->ctx = c;
            j->state = RESIDENT;
            resident.push_back(j);
            peak_resident = std::max<int64_t>(peak_resident, static_cast<int64_t>(resident.size()));
        }
        if (resident.empty()) {
            cv_work.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        // 2. keep sweeps in flight for every resident job, round robin
        std::vector<std::shared_ptr<Job>> snap = resident;
        lk.unlock();
        bool progressed = false;
        // 2a. jobs on the persistent path: one shared cooperative launch per
        // round (kRound sweeps of each, one dtype per round)
        if (batch_inflight && cudaEventQuery(bev) == cudaSuccess) {
            batch_inflight = false;
            for (auto& j : batch_members) j->batch_pending = false;
            batch_members.clear();
            progressed = true;
        }
        if (!batch_inflight) {
            std::vector<std::shared_ptr<Job>> mem;
            std::vector<ifctn_ctx*> cs;
            std::vector<int> ns;
            int kind = 0;
            for (auto& j : snap) {
                if (j->state != RESIDENT || j->err != IFCTN_OK || j->enqueued >= j->prob.max_sweeps) continue;
                const int k = ctx_batch_kind(j->ctx);
                if (!k) continue;
                if (!kind) kind = k;
                if (k != kind) continue;
                mem.push_back(j);
                cs.push_back(j->ctx);
                ns.push_back(std::min(kRound, j->prob.max_sweeps - j->enqueued));
            }
            if (!mem.empty()) {
                ifctn_status rs = ctx_run_batch(cs.data(), ns.data(), static_cast<int>(cs.size()), bst);
                if (rs == IFCTN_OK && cudaEventRecord(bev, bst) != cudaSuccess) rs = IFCTN_ECUDA;
                for (size_t i = 0; i < mem.size(); ++i) {
                    mem[i]->enqueued += ns[i];
                    if (rs != IFCTN_OK) {
                        mem[i]->err = rs;
                        mem[i]->msg = ifctn_last_error();
                    } else {
                        mem[i]->batch_pending = true;
                    }
                }
                if (rs == IFCTN_OK) {
                    batch_members = mem;
                    batch_inflight = true;
                    ++batch_launches;
                    batched_jobs += static_cast<int64_t>(mem.size());
                }
                progressed = true;
            }
        }
        for (auto& j : snap) {
            if (j->state == RESIDENT) {
                const int total = j->prob.max_sweeps;
                const bool shared = ctx_batch_kind(j->ctx) != 0;
                if (shared && (j->batch_pending || (j->enqueued < total && j->err == IFCTN_OK))) continue;
                if (j->enqueued < total && !shared) {
                    // only top up when the previous batch has drained
                    if (j->enqueued == 0 || cudaEventQuery(j->ev) == cudaSuccess) {
                        const int n = std::min(kInflight, total - j->enqueued);
                        ifctn_status rs = ctx_enqueue(j->ctx, n, j->prob.tol, false);
                        if (rs == IFCTN_OK) cudaEventRecord(j->ev, ctx_stream(j->ctx));
                        j->enqueued += n;
                        progressed = true;
                        if (rs != IFCTN_OK) {
                            j->err = rs;
                            j->msg = ifctn_last_error();
                        }
                    }
                } else if (shared || cudaEventQuery(j->ev) == cudaSuccess || total == 0) {
                    // 3. result to pinned host memory
                    ifctn_status rs = j->err;
                    if (rs == IFCTN_OK) rs = ifctn_sweep(j->ctx, 0, &j->stats);
                    if (rs == IFCTN_OK) rs = ifctn_get_x(j->ctx, j->result);
                    if (rs != IFCTN_OK && j->msg.empty()) j->msg = ifctn_last_error();
                    j->err = rs;
                    j->stats.sweeps_done = std::max(j->stats.sweeps_done, 0);
                    ifctn_destroy(j->ctx);
                    j->ctx = nullptr;
                    cudaEventDestroy(j->ev);
                    j->ev = nullptr;
                    j->state = FINISHING;
                    progressed = true;
                }
            }
        }
        lk.lock();
        for (size_t i = 0; i < resident.size();) {
            auto& j = resident[i];
            if (j->state == FINISHING) {
                j->state = j->err == IFCTN_OK ? DONE : FAILED;
                j->t_done = Clock::now();
                in_use -= j->bytes;
                latency[j->ticket] = std::chrono::duration<double>(j->t_done - j->t_submit).count();
                ++completed;
                free_pinned(*j);
                resident.erase(resident.begin() + i);
                cv_done.notify_all();
            } else {
                ++i;
            }
        }
        if (!progressed) cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

extern "C" {

ifctn_status ifctn_server_create(size_t hbm_budget_bytes, int32_t max_slots, ifctn_server** out) {
    if (!out || max_slots < 1 || hbm_budget_bytes == 0) {
        set_error("invalid server arguments");
        return IFCTN_EINVAL;
    }
    auto* s = new ifctn_server();
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    cudaGetDevice(&s->device);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return IFCTN_OK;
}

ifctn_status ifctn_submit(ifctn_server* srv, const ifctn_problem* prob, const void* obs, const uint8_t* mask,
                          const double* init_factors, uint64_t* ticket) {
    if (!srv || !prob || !obs || !mask || !ticket) {
        set_error("null argument");
        return IFCTN_EINVAL;
    }
    Shape sh;
    ifctn_status rs = build_shape(prob, sh);
    if (rs != IFCTN_OK) return rs;
    auto j = std::make_shared<Job>();
    j->prob = *prob;
    j->P = static_cast<size_t>(sh.P);
    j->esz = prob->precision == IFCTN_FP64 ? 8 : 4;
    j->bytes = job_bytes_estimate(sh, j->esz);
    if (j->bytes > srv->budget) {
        set_error("job exceeds the server's device-memory budget");
        return IFCTN_ENOMEM;
    }
    if (cudaHostAlloc(&j->obs, j->P * j->esz, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&j->mask), j->P, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(&j->result, j->P * j->esz, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        free_pinned(*j);
        if (j->result) cudaFreeHost(j->result);
        set_error("pinned host allocation failed");
        return IFCTN_ENOMEM;
    }
    if (cudaMemcpy(j->obs, obs, j->P * j->esz, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(j->mask, mask, j->P, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        free_pinned(*j);
        cudaFreeHost(j->result);
        set_error("input copy failed");
        return IFCTN_ECUDA;
    }
    if (init_factors) {
        const size_t gb = static_cast<size_t>(sh.gsize) * sizeof(double);
        if (cudaHostAlloc(reinterpret_cast<void**>(&j->init), gb, cudaHostAllocDefault) != cudaSuccess ||
            cudaMemcpy(j->init, init_factors, gb, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            free_pinned(*j);
            cudaFreeHost(j->result);
            set_error("factor copy failed");
            return IFCTN_ECUDA;
        }
    }
    memset(&j->stats, 0, sizeof(j->stats));
    {
        std::lock_guard<std::mutex> g(srv->mu);
        j->ticket = srv->next_ticket++;
        j->t_submit = Clock::now();
        srv->jobs[j->ticket] = j;
        srv->queue.push_back(j);
        *ticket = j->ticket;
    }
    srv->cv_work.notify_all();
    return IFCTN_OK;
}

ifctn_status ifctn_poll(ifctn_server* srv, uint64_t ticket, void* out_X, ifctn_stats* out, int64_t timeout_us) {
    if (!srv) {
        set_error("null server");
        return IFCTN_EINVAL;
    }
    std::shared_ptr<Job> j;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->jobs.find(ticket);
        if (it == srv->jobs.end()) {
            set_error("unknown ticket");
            return IFCTN_ENOTFOUND;
        }
        j = it->second;
        auto ready = [&] { return j->state == DONE || j->state == FAILED; };
        if (!ready()) {
            if (timeout_us == 0) return IFCTN_ENOTREADY;
            if (timeout_us < 0)
                srv->cv_done.wait(lk, ready);
            else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
                return IFCTN_ETIMEOUT;
        }
        srv->jobs.erase(ticket);
    }
    ifctn_status rs = j->err;
    if (rs != IFCTN_OK) {
        set_error(j->msg);
    } else {
        if (out_X && cudaMemcpy(out_X, j->result, j->P * j->esz, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            set_error("result copy failed");
            rs = IFCTN_ECUDA;
        }
        if (out) *out = j->stats;
    }
    if (j->result) cudaFreeHost(j->result);
    j->result = nullptr;
    return rs;
}

ifctn_status ifctn_server_info_get(ifctn_server* srv, ifctn_server_info* out) {
    if (!srv || !out) return IFCTN_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    out->queued = static_cast<int64_t>(srv->queue.size());
    out->resident = static_cast<int64_t>(srv->resident.size());
    out->completed = srv->completed;
    out->bytes_in_use = static_cast<int64_t>(srv->in_use);
    out->peak_resident = srv->peak_resident;
    out->batch_launches = srv->batch_launches;
    out->batched_jobs = srv->batched_jobs;
    return IFCTN_OK;
}

ifctn_status ifctn_server_latency(ifctn_server* srv, uint64_t ticket, double* seconds) {
    if (!srv || !seconds) return IFCTN_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->latency.find(ticket);
    if (it == srv->latency.end()) return IFCTN_ENOTFOUND;
    *seconds = it->second;
    return IFCTN_OK;
}

void ifctn_server_destroy(ifctn_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    if (srv->bst) {
        cudaStreamSynchronize(srv->bst);
        cudaStreamDestroy(srv->bst);
    }
    if (srv->bev) cudaEventDestroy(srv->bev);
    for (auto& j : srv->resident) {
        if (j->ctx) ifctn_destroy(j->ctx);
        if (j->ev) cudaEventDestroy(j->ev);
        free_pinned(*j);
    }
    for (auto& kv : srv->jobs) {
        free_pinned(*kv.second);
        if (kv.second->result) cudaFreeHost(kv.second->result);
    }
    delete srv;
}

}  // extern "C"
