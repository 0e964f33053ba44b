// Continuous-batching request server.
//
// Requests (a circuit of n qubits in one precision) arrive through sv_server_submit and
// are fused on a small pool of host threads (Algorithm 2).  One GPU worker thread admits
// fused requests, cheapest estimated GPU work first with aging (a request's priority
// grows with its wait, so large ones are not starved), while the HBM they need fits the
// budget -- the memory
// model of Eq. 14, M = 2^n s + (2^k)^2 s + M_ws, checked against the budget instead of
// the paper's Eq. 15 query, and queuing instead of the paper's GPU->CPU fallback -- and
// while a slot is free.  Each slot has its own CUDA stream and workspace; a request's
// state comes from the stream-ordered allocator on that stream, so requests overlap on
// the device and new ones start as soon as memory and a slot free up.  A request runs
// sv_set_basis + every fused pass + the top-k search; its results come back through
// pinned host memory and an event, and its memory is released in stream order.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sv_internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    uint32_t n = 0;
    sv_dtype dtype = SV_C64;
    std::vector<svi::Gate> gates;      // sorted, unfused
    sv_circuit *circuit = nullptr;     // fused
    sv_status fuse_status = SV_OK;
    size_t cost = 0;
    double est_s = 0;                  // estimated GPU time: passes x bytes / pass rate
    double t_submit = 0, t_admit = 0, t_done = 0;
};

// Requests estimated below this run on the slot's high-priority stream, so that their
// kernels are scheduled ahead of long requests' as SMs free up.
constexpr double SHORT_REQUEST_S = 0.02;
// Seconds of estimated work that one second of waiting is worth in the admission order.
constexpr double AGING = 0.25;

struct Slot {
    sv_state state;                    // buf (and stream) re-pointed per request
    cudaStream_t s_hi = nullptr, s_lo = nullptr;   // high- and low-priority streams
    cudaEvent_t done = nullptr;
    double *host_p = nullptr;          // pinned 64 doubles
    unsigned long long *host_i = nullptr;
    Request *req = nullptr;
    sv_status launch_status = SV_OK;
};

}  // namespace

struct sv_server {
    sv_server_config cfg;
    clk::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;   // new submissions / fused requests / stop
    std::condition_variable cv_done;   // new results
    std::deque<Request *> to_fuse, ready;
    std::vector<sv_server_result> results;
    std::vector<Slot> slots;
    std::vector<std::thread> fusers;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    size_t in_use = 0;
    uint64_t submitted = 0, completed = 0;
    int device = 0, num_sms = 0;
    unsigned char *ws_block = nullptr;

    double now() const { return std::chrono::duration<double>(clk::now() - t0).count(); }
};

namespace {

size_t elem_bytes_s(sv_dtype d) { return d == SV_C64 ? 8 : 16; }

void fuser_loop(sv_server *S) {
    while (true) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv_work.wait(lock, [&] { return S->stop || !S->to_fuse.empty(); });
            if (S->stop && S->to_fuse.empty()) return;
            r = S->to_fuse.front();
            S->to_fuse.pop_front();
        }
        sv_circuit *c = new (std::nothrow) sv_circuit();
        if (!c) {
            r->fuse_status = SV_ERR_OOM;
        } else {
            c->n = r->n;
            // complex128 width-5 gates have no tensor-core pass: such requests are fused at
            // width <= 4 where the complex128 tensor-core kernel serves the state
            const uint32_t kf = (r->dtype == SV_C128 && r->n >= 11) ? std::min(S->cfg.max_k, 4u)
                                                                    : S->cfg.max_k;
            c->gates = svi::fuse_gates(r->gates, r->n, kf);
            r->gates.clear();
            r->gates.shrink_to_fit();
            r->circuit = c;
            uint32_t kmax = 1;
            for (const svi::Gate &g : c->gates) kmax = std::max(kmax, g.k);
            // Eq. 14: state + one resident gate matrix + the workspace
            r->cost = (elem_bytes_s(r->dtype) << r->n) + (size_t(1) << (2 * kmax)) * elem_bytes_s(r->dtype) +
                      svi::WS_BYTES;
            // GPU time: a read and a write of the state per pass at the measured pass rates
            // (complex64 about 5.5 TB/s, complex128 about 3 TB/s) plus a launch each
            const double rate = r->dtype == SV_C64 ? 5.5e12 : 3.0e12;
            r->est_s = (double)c->gates.size() * (2.0 * (double)(elem_bytes_s(r->dtype) << r->n) / rate + 2.5e-5);
        }
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->ready.push_back(r);
        }
        S->cv_work.notify_all();
    }
}

// Enqueue one admitted request on its slot (worker thread, no lock held).
sv_status start_request(sv_server *S, Slot &sl, Request *r) {
    sv_state &st = sl.state;
    st.stream = r->est_s < SHORT_REQUEST_S ? sl.s_hi : sl.s_lo;
    const size_t bytes = elem_bytes_s(r->dtype) << r->n;
    void *buf = nullptr;
    SV_CUDA(cudaMallocAsync(&buf, bytes, st.stream));
    st.n = r->n;
    st.dtype = r->dtype;
    st.buf = buf;
    st.cap = bytes;
    st.owned = false;
    sv_status s = sv_set_basis(&st, 0);
    (void)S;
    for (size_t i = 0; s == SV_OK && i < r->circuit->gates.size(); ++i)
        s = svi::launch_apply(&st, r->circuit->gates[i]);
    if (s == SV_OK) s = svi::enqueue_topk(&st, sl.host_p, sl.host_i);
    SV_CUDA(cudaFreeAsync(buf, st.stream));
    st.buf = nullptr;
    SV_CUDA(cudaEventRecord(sl.done, st.stream));
    (void)S;
    return s;
}

void finish(sv_server *S, Slot &sl, sv_status status) {
    Request *r = sl.req;
    sv_server_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = r->id;
    res.status = status;
    res.dtype_used = r->dtype;
    res.n = r->n;
    const uint64_t N = 1ull << r->n;
    res.k = (uint32_t)std::min<uint64_t>(S->cfg.topk, N);
    if (status == SV_OK)
        for (uint32_t j = 0; j < res.k; ++j) {
            res.idx[j] = sl.host_i[j];
            res.p[j] = sl.host_p[j];
        }
    res.t_submit = r->t_submit;
    res.t_admit = r->t_admit;
    res.t_done = S->now();
    res.passes = r->circuit ? r->circuit->gates.size() : 0;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->results.push_back(res);
        S->in_use -= r->cost;
        ++S->completed;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
    delete r->circuit;
    delete r;
    sl.req = nullptr;
}

void worker_loop(sv_server *S) {
    cudaSetDevice(S->device);
    while (true) {
        bool progressed = false;
        // completions
        for (Slot &sl : S->slots) {
            if (!sl.req) continue;
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) continue;
            sv_status st = sl.launch_status;
            if (e != cudaSuccess && st == SV_OK) st = SV_ERR_CUDA;
            if (st == SV_OK) {
                int err = 0;
                if (cudaMemcpy(&err, sl.state.ws + svi::WS_ERR, sizeof(int), cudaMemcpyDeviceToHost) ==
                        cudaSuccess && err) {
                    cudaMemset(sl.state.ws + svi::WS_ERR, 0, sizeof(int));
                    st = SV_ERR_TIMEOUT;
                }
            }
            finish(S, sl, st);
            progressed = true;
        }
        // admissions: failed or never-fitting requests first (reported at once), then the
        // request with the least estimated work minus AGING x its wait; if that one does
        // not fit the free memory, nothing else is admitted until it does
        while (true) {
            Request *r = nullptr;
            Slot *slot = nullptr;
            Request *rejected = nullptr;
            {
                std::lock_guard<std::mutex> lock(S->mu);
                if (S->ready.empty()) break;
                const double now = S->now();
                size_t best = S->ready.size();
                double best_key = 0.0;
                for (size_t i = 0; i < S->ready.size(); ++i) {
                    Request *q = S->ready[i];
                    if (q->fuse_status != SV_OK || q->cost > S->cfg.budget_bytes) {
                        best = i;
                        rejected = q;
                        break;
                    }
                    const double key = q->est_s - AGING * (now - q->t_submit);
                    if (best == S->ready.size() || key < best_key) {
                        best = i;
                        best_key = key;
                    }
                }
                Request *head = S->ready[best];
                if (rejected) {
                    // fusion failed or it can never fit: report it instead of queuing forever
                    S->ready.erase(S->ready.begin() + (std::ptrdiff_t)best);
                    head->t_admit = now;
                    S->in_use += head->cost;
                } else {
                    for (Slot &sl : S->slots)
                        if (!sl.req) {
                            slot = &sl;
                            break;
                        }
                    if (!slot || S->in_use + head->cost > S->cfg.budget_bytes) break;
                    S->ready.erase(S->ready.begin() + (std::ptrdiff_t)best);
                    r = head;
                    S->in_use += r->cost;
                    r->t_admit = now;
                    slot->req = r;
                }
            }
            if (rejected) {
                Slot tmp;
                tmp.req = rejected;
                finish(S, tmp, rejected->fuse_status != SV_OK ? rejected->fuse_status : SV_ERR_OOM);
            } else {
                slot->launch_status = start_request(S, *slot, r);
            }
            progressed = true;
        }
        {
            std::unique_lock<std::mutex> lock(S->mu);
            bool busy = false;
            for (Slot &sl : S->slots) busy |= sl.req != nullptr;
            if (S->stop && !busy && S->ready.empty() && S->to_fuse.empty()) return;
            if (!progressed) {
                if (busy) S->cv_work.wait_for(lock, std::chrono::microseconds(50));
                else S->cv_work.wait_for(lock, std::chrono::milliseconds(5));
            }
        }
    }
}

}  // namespace

using namespace svi;

extern "C" {

sv_status sv_server_create(const sv_server_config *cfg, sv_server **out) {
    clear_error();
    if (!out) return set_error(SV_ERR_ARG, "sv_server_create: null out");
    *out = nullptr;
    sv_server *S = new (std::nothrow) sv_server();
    if (!S) return set_error(SV_ERR_OOM, "sv_server_create: host allocation failed");
    std::memset(&S->cfg, 0, sizeof(S->cfg));
    if (cfg) S->cfg = *cfg;
    if (!S->cfg.budget_bytes) S->cfg.budget_bytes = size_t(150) << 30;
    if (!S->cfg.max_slots) S->cfg.max_slots = 16;
    if (S->cfg.max_slots > 256) S->cfg.max_slots = 256;
    if (!S->cfg.topk || S->cfg.topk > 64) S->cfg.topk = 64;
    if (!S->cfg.max_k) S->cfg.max_k = 5;
    if (S->cfg.max_k > SV_MAX_K) S->cfg.max_k = SV_MAX_K;
    if (!S->cfg.fuse_threads) S->cfg.fuse_threads = 4;
    S->t0 = clk::now();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, S->device);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&S->ws_block), WS_BYTES * S->cfg.max_slots);
    if (e == cudaSuccess) e = cudaMemset(S->ws_block, 0, WS_BYTES * S->cfg.max_slots);
    if (e == cudaSuccess) {
        // keep freed request memory in the stream-ordered pool up to the budget, so that
        // admissions do not go back to the driver for every request
        cudaMemPool_t pool;
        e = cudaDeviceGetDefaultMemPool(&pool, S->device);
        uint64_t thr = S->cfg.budget_bytes;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    S->slots.resize(S->cfg.max_slots);
    for (uint32_t i = 0; e == cudaSuccess && i < S->cfg.max_slots; ++i) {
        Slot &sl = S->slots[i];
        sl.state.device = S->device;
        sl.state.num_sms = S->num_sms;
        sl.state.ws = S->ws_block + WS_BYTES * i;
        int lo_prio = 0, hi_prio = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.s_hi, cudaStreamNonBlocking, hi_prio);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.s_lo, cudaStreamNonBlocking, lo_prio);
        sl.state.stream = sl.s_lo;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl.host_p), 64 * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMallocHost(reinterpret_cast<void **>(&sl.host_i), 64 * sizeof(unsigned long long));
    }
    if (e != cudaSuccess) {
        const std::string msg = std::string("sv_server_create: ") + cudaGetErrorString(e);
        sv_server_destroy(S);
        return set_error(SV_ERR_CUDA, msg);
    }
    for (uint32_t i = 0; i < S->cfg.fuse_threads; ++i) S->fusers.emplace_back(fuser_loop, S);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return SV_OK;
}

sv_status sv_server_submit(sv_server *S, uint32_t n, sv_dtype dtype, const sv_gate *gates, size_t ngates,
                           uint64_t *id) {
    clear_error();
    if (!S || (ngates && !gates)) return set_error(SV_ERR_ARG, "sv_server_submit: null argument");
    if (n < 1 || n > SV_MAX_QUBITS) return set_error(SV_ERR_ARG, "sv_server_submit: n must be 1..34");
    if (dtype != SV_C64 && dtype != SV_C128) return set_error(SV_ERR_ARG, "sv_server_submit: bad dtype");
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(SV_ERR_OOM, "sv_server_submit: host allocation failed");
    r->t_submit = S->now();
    r->n = n;
    r->dtype = dtype;
    r->gates.reserve(ngates);
    for (size_t i = 0; i < ngates; ++i) {
        const sv_gate &g = gates[i];
        bool ok = g.u && g.k >= 1 && g.k <= SV_MAX_K;
        uint64_t seen = 0;
        for (uint32_t j = 0; ok && j < g.k; ++j) {
            ok = g.targets[j] < n && !(seen & (1ull << g.targets[j]));
            seen |= 1ull << g.targets[j];
        }
        if (!ok) {
            delete r;
            return set_error(SV_ERR_ARG, "sv_server_submit: bad gate " + std::to_string(i));
        }
        r->gates.push_back(sorted_gate(g.k, g.targets, g.u));
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) {
            delete r;
            return set_error(SV_ERR_STATE, "sv_server_submit: server is shutting down");
        }
        r->id = S->next_id++;
        S->to_fuse.push_back(r);
        ++S->submitted;
        if (id) *id = r->id;
    }
    S->cv_work.notify_all();
    return SV_OK;
}

sv_status sv_server_poll(sv_server *S, sv_server_result *out, size_t cap, size_t *nout, int wait_ms) {
    clear_error();
    if (!S || !nout || (cap && !out)) return set_error(SV_ERR_ARG, "sv_server_poll: null argument");
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->results.empty() && wait_ms > 0)
        S->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !S->results.empty(); });
    const size_t m = std::min(cap, S->results.size());
    for (size_t i = 0; i < m; ++i) out[i] = S->results[i];
    S->results.erase(S->results.begin(), S->results.begin() + (long)m);
    *nout = m;
    return SV_OK;
}

sv_status sv_server_get_stats(sv_server *S, sv_server_stats *st) {
    clear_error();
    if (!S || !st) return set_error(SV_ERR_ARG, "sv_server_get_stats: null argument");
    std::lock_guard<std::mutex> lock(S->mu);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->queued = S->to_fuse.size() + S->ready.size();
    uint32_t active = 0;
    for (const Slot &sl : S->slots) active += sl.req != nullptr;
    st->active = active;
    st->in_use_bytes = S->in_use;
    st->budget_bytes = S->cfg.budget_bytes;
    st->now = S->now();
    return SV_OK;
}

sv_status sv_server_destroy(sv_server *S) {
    if (!S) return SV_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread &t : S->fusers)
        if (t.joinable()) t.join();
    if (S->worker.joinable()) S->worker.join();
    for (Slot &sl : S->slots) {
        for (cudaStream_t st : {sl.s_hi, sl.s_lo})
            if (st) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
            }
        sl.state.stream = nullptr;
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.host_p) cudaFreeHost(sl.host_p);
        if (sl.host_i) cudaFreeHost(sl.host_i);
    }
    for (Request *r : S->to_fuse) delete r;
    for (Request *r : S->ready) {
        delete r->circuit;
        delete r;
    }
    if (S->ws_block) cudaFree(S->ws_block);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    delete S;
    return SV_OK;
}

}  // extern "C"
