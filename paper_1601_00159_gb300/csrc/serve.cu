// Serving form: continuous batching of variable-size requests against one resident
// index (host runtime; every query runs in the batch path's kernels).
//
// Data path of a request: the client copies its arrays into a pinned ring (submit);
// the dispatcher thread coalesces ready requests, in arrival order and contiguous in
// the ring, into a batch of at most max_batch queries on a free device slot:
//   h2d stream:     ring -> slot inputs                          (event in)
//   compute stream: wait in; pi_execute_batch on the slot        (event done)
//   d2h stream:     wait done; slot results -> the ring          (event out)
// With several slots in flight, batch k+1's copy in and batch k's copy out overlap
// batch k's and k+1's kernels. The dispatcher polls the out events in dispatch order
// and stamps the requests complete; a client collects its results from the ring, which
// frees the space (collection is in submission order, so the ring is a FIFO).
// Only public entry points of the library touch the index, from the dispatcher thread.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t pos;       // ring position (monotone counter; physical index pos % R)
    uint32_t n;
    bool ready;         // inputs copied into the ring
    bool dispatched;
    bool done;
    int64_t t_arrive;   // ns
    int64_t t_done;
};

struct Slot {
    uint8_t* d_ops = nullptr;
    uint64_t* d_keys = nullptr;
    uint64_t* d_vals = nullptr;
    pi_result_t* d_res = nullptr;
    cudaEvent_t ev_in = nullptr, ev_done = nullptr, ev_out = nullptr;
    uint64_t first = 0;  // ticket of the batch's first request
    uint32_t nreq = 0;
    bool busy = false;
};

int map_err(cudaError_t e) {
    if (e == cudaSuccess) return PI_OK;
    return e == cudaErrorMemoryAllocation ? PI_ERR_OOM : PI_ERR_CUDA;
}

}  // namespace

struct pi_server {
    pi_index_t* idx = nullptr;
    int device = 0;
    uint32_t max_batch = 0, nslots = 0;
    uint64_t R = 0;  // ring capacity in queries
    uint8_t* r_ops = nullptr;
    uint64_t* r_keys = nullptr;
    uint64_t* r_vals = nullptr;
    pi_result_t* r_res = nullptr;
    std::vector<Slot> slots;
    std::deque<uint32_t> busy_order;  // slots in dispatch order
    cudaStream_t cs = nullptr, hs = nullptr, ds = nullptr;
    std::mutex mu;
    std::condition_variable cv_space, cv_work, cv_done;
    std::deque<Req> reqs;   // uncollected requests, ticket order; reqs[0] has ticket `first`
    uint64_t first = 1;     // ticket of reqs.front()
    uint64_t next_disp = 1; // ticket of the first request not yet dispatched
    uint64_t tail = 0;      // ring position after the newest request
    std::thread worker;
    bool stop = false;
    bool disp_idle = false;      // the dispatcher sleeps with nothing in flight
    uint32_t submit_waiters = 0; // collectors waiting for a ticket to be submitted
    int error = PI_OK;
    // statistics since the last reset
    std::vector<double> lat;
    uint64_t n_req = 0, n_q = 0, n_batches = 0;
    uint32_t inflight = 0, max_inflight = 0;

    Req& at(uint64_t ticket) { return reqs[(size_t)(ticket - first)]; }
};

namespace {

void run_dispatcher(pi_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false;
        // retire completed batches, oldest first
        while (!s->busy_order.empty()) {
            Slot& sl = s->slots[s->busy_order.front()];
            const cudaError_t q = cudaEventQuery(sl.ev_out);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess && s->error == PI_OK) s->error = map_err(q);
            const int64_t t = now_ns();
            for (uint32_t k = 0; k < sl.nreq; ++k) {
                Req& r = s->at(sl.first + k);
                r.done = true;
                r.t_done = t;
                s->lat.push_back((double)(t - r.t_arrive) * 1e-9);
                s->n_req++;
                s->n_q += r.n;
            }
            sl.busy = false;
            s->busy_order.pop_front();
            s->inflight--;
            progress = true;
            s->cv_done.notify_all();
        }
        // dispatch the ready requests into a free slot
        uint32_t free_slot = s->nslots;
        for (uint32_t i = 0; i < s->nslots; ++i)
            if (!s->slots[i].busy) {
                free_slot = i;
                break;
            }
        const uint64_t end_ticket = s->first + s->reqs.size();
        if (free_slot < s->nslots && s->next_disp < end_ticket && s->at(s->next_disp).ready && s->error == PI_OK) {
            const uint64_t t0 = s->next_disp;
            const uint64_t pos0 = s->at(t0).pos;
            uint64_t pos_end = pos0, t = t0;
            uint32_t n = 0;
            while (t < end_ticket) {
                const Req& r = s->at(t);
                if (!r.ready || r.pos != pos_end || n + r.n > s->max_batch) break;
                if ((pos0 % s->R) + (pos_end - pos0) + r.n > s->R) break;  // stays contiguous in the ring
                n += r.n;
                pos_end += r.n;
                ++t;
            }
            Slot& sl = s->slots[free_slot];
            sl.first = t0;
            sl.nreq = (uint32_t)(t - t0);
            sl.busy = true;
            for (uint64_t k = t0; k < t; ++k) s->at(k).dispatched = true;
            s->next_disp = t;
            s->busy_order.push_back(free_slot);
            s->inflight++;
            s->max_inflight = std::max(s->max_inflight, s->inflight);
            s->n_batches++;
            lk.unlock();
            const uint64_t p = pos0 % s->R;
            cudaError_t e = cudaMemcpyAsync(sl.d_ops, s->r_ops + p, n, cudaMemcpyHostToDevice, s->hs);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_keys, s->r_keys + p, (size_t)n * 8, cudaMemcpyHostToDevice, s->hs);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_vals, s->r_vals + p, (size_t)n * 8, cudaMemcpyHostToDevice, s->hs);
            if (e == cudaSuccess) e = cudaEventRecord(sl.ev_in, s->hs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cs, sl.ev_in, 0);
            int rc = e == cudaSuccess ? PI_OK : map_err(e);
            if (rc == PI_OK)
                rc = pi_execute_batch(s->idx, sl.d_ops, sl.d_keys, sl.d_vals, n, sl.d_res,
                                      reinterpret_cast<pi_stream_t>(s->cs));
            if (rc == PI_OK) {
                e = cudaEventRecord(sl.ev_done, s->cs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->ds, sl.ev_done, 0);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(s->r_res + p, sl.d_res, (size_t)n * sizeof(pi_result_t), cudaMemcpyDeviceToHost,
                                        s->ds);
                rc = map_err(e);
            }
            // the out event is recorded even after an error, so the batch still retires
            cudaEventRecord(sl.ev_out, s->ds);
            lk.lock();
            if (rc != PI_OK && s->error == PI_OK) s->error = rc;
            progress = true;
        }
        if (s->stop && s->busy_order.empty() && (s->next_disp >= s->first + s->reqs.size() || s->error != PI_OK))
            break;
        if (!progress) {
            if (s->busy_order.empty()) {
                s->disp_idle = true;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(1));
                s->disp_idle = false;
            } else {
                s->cv_work.wait_for(lk, std::chrono::microseconds(10));  // polling the GPU
            }
        }
    }
    s->cv_done.notify_all();
}

void free_server(pi_server* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    for (auto& sl : s->slots) {
        cudaFree(sl.d_ops);
        cudaFree(sl.d_keys);
        cudaFree(sl.d_vals);
        cudaFree(sl.d_res);
        if (sl.ev_in) cudaEventDestroy(sl.ev_in);
        if (sl.ev_done) cudaEventDestroy(sl.ev_done);
        if (sl.ev_out) cudaEventDestroy(sl.ev_out);
    }
    if (s->r_ops) cudaFreeHost(s->r_ops);
    if (s->r_keys) cudaFreeHost(s->r_keys);
    if (s->r_vals) cudaFreeHost(s->r_vals);
    if (s->r_res) cudaFreeHost(s->r_res);
    if (s->cs) cudaStreamDestroy(s->cs);
    if (s->hs) cudaStreamDestroy(s->hs);
    if (s->ds) cudaStreamDestroy(s->ds);
    delete s;
}

// Reserves ring space and tickets for count requests back to back (request k has
// sizes[k] queries): each request contiguous in the ring and off every physical slot of
// an uncollected request, i.e. the group's end <= R + the oldest uncollected position
// (anything is free when nothing is uncollected). Waits for space.
int reserve_group(pi_server* s, const uint32_t* sizes, uint32_t count, const int64_t* t_arrive, uint64_t* pos,
                  uint64_t* first_ticket) {
    if (!s || count == 0) return PI_ERR_INVALID_ARG;
    uint64_t total = 0;
    for (uint32_t k = 0; k < count; ++k) {
        if (sizes[k] == 0 || sizes[k] > s->max_batch) return PI_ERR_INVALID_ARG;
        total += sizes[k];
    }
    if (total > s->R) return PI_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->error != PI_OK) return s->error;
        uint64_t p = s->tail;
        for (uint32_t k = 0; k < count; ++k) {
            if (p % s->R + sizes[k] > s->R) p += s->R - p % s->R;
            pos[k] = p;
            p += sizes[k];
        }
        if (s->reqs.empty() || p <= s->reqs.front().pos + s->R) break;
        s->cv_space.wait(lk);
    }
    *first_ticket = s->first + s->reqs.size();
    for (uint32_t k = 0; k < count; ++k) s->reqs.push_back(Req{pos[k], sizes[k], false, false, false, t_arrive[k], 0});
    s->tail = pos[count - 1] + sizes[count - 1];
    return PI_OK;
}

// Copies reserved requests' queries (request k from offset offs[k] of the arrays) into
// the ring and hands them to the dispatcher.
void fill_group(pi_server* s, const uint8_t* ops, const uint64_t* keys, const uint64_t* vals, const uint32_t* sizes,
                const uint64_t* offs, uint32_t count, const uint64_t* pos, uint64_t first_ticket) {
    for (uint32_t k = 0; k < count; ++k) {
        const uint64_t p = pos[k] % s->R, o = offs[k], n = sizes[k];
        std::memcpy(s->r_ops + p, ops + o, n);
        std::memcpy(s->r_keys + p, keys + o, n * 8);
        std::memcpy(s->r_vals + p, vals + o, n * 8);
    }
    bool wake_disp, wake_coll;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint32_t k = 0; k < count; ++k) s->at(first_ticket + k).ready = true;
        wake_disp = s->disp_idle;
        wake_coll = s->submit_waiters > 0;
    }
    if (wake_disp) s->cv_work.notify_one();
    if (wake_coll) s->cv_done.notify_all();  // a collector waits for these tickets to exist
}

// Collects, in ticket order from `ticket` on (the oldest uncollected request), every
// request that is done, at most `limit`, waiting for the first one: request j's results
// go to results_out + offs[j] (results_out may be null) and its latency to lat_out[j]
// (may be null); their ring space is freed at once. One lock round per group instead
// of one per request. Returns how many were collected (>= 1), or a negative error code.
int64_t collect_group(pi_server* s, uint64_t ticket, uint32_t limit, pi_result_t* results_out, const uint64_t* offs,
                      double* lat_out) {
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket != s->first || limit == 0) return PI_ERR_INVALID_ARG;
    if (s->reqs.empty()) {  // the collector may run ahead of the submitter
        s->submit_waiters++;
        s->cv_done.wait(lk, [&] { return !s->reqs.empty() || s->error != PI_OK; });
        s->submit_waiters--;
    }
    if (s->reqs.empty()) return s->error != PI_OK ? s->error : PI_ERR_INVALID_ARG;
    s->cv_done.wait(lk, [&] { return s->reqs.front().done || s->error != PI_OK; });
    if (!s->reqs.front().done) return s->error;
    uint32_t k = 0;
    while (k < limit && k < s->reqs.size() && s->reqs[k].done) ++k;
    std::vector<Req> rs(s->reqs.begin(), s->reqs.begin() + k);
    lk.unlock();
    for (uint32_t j = 0; j < k; ++j) {
        const Req& r = rs[j];
        if (results_out)
            std::memcpy(results_out + offs[j], s->r_res + r.pos % s->R, (size_t)r.n * sizeof(pi_result_t));
        if (lat_out) lat_out[j] = (double)(r.t_done - r.t_arrive) * 1e-9;
    }
    lk.lock();
    s->reqs.erase(s->reqs.begin(), s->reqs.begin() + k);
    s->first += k;
    lk.unlock();
    s->cv_space.notify_all();
    return (int64_t)k;
}

double pct(std::vector<double>& v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = (size_t)std::min<double>((double)(v.size() - 1), q * (double)(v.size() - 1) + 0.5);
    std::nth_element(v.begin(), v.begin() + (long)k, v.end());
    return v[k];
}

}  // namespace

extern "C" {

pi_server_t* pi_server_create(pi_index_t* idx, const pi_server_config_t* cfg) {
    pi::set_last_error(PI_OK);
    pi_server_config_t c{};
    c.struct_size = sizeof(c);
    c.max_batch = 1u << 20;
    c.slots = 3;
    if (cfg) {
        if (cfg->struct_size != sizeof(pi_server_config_t)) {
            pi::set_last_error(PI_ERR_INVALID_ARG);
            return nullptr;
        }
        if (cfg->max_batch) c.max_batch = cfg->max_batch;
        if (cfg->slots) c.slots = cfg->slots;
        c.ring_queries = cfg->ring_queries;
    }
    if (!c.ring_queries) c.ring_queries = 8ull * c.max_batch;
    if (!idx || c.max_batch > PI_MAX_BATCH || c.slots < 2 || c.slots > 8 || c.ring_queries < c.max_batch) {
        pi::set_last_error(PI_ERR_INVALID_ARG);
        return nullptr;
    }
    pi_server* s = new (std::nothrow) pi_server();
    if (!s) {
        pi::set_last_error(PI_ERR_OOM);
        return nullptr;
    }
    cudaGetDevice(&s->device);
    s->idx = idx;
    s->max_batch = c.max_batch;
    s->nslots = c.slots;
    s->R = c.ring_queries;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMallocHost(reinterpret_cast<void**>(&s->r_ops), s->R)) != cudaSuccess) break;
        if ((e = cudaMallocHost(reinterpret_cast<void**>(&s->r_keys), s->R * 8)) != cudaSuccess) break;
        if ((e = cudaMallocHost(reinterpret_cast<void**>(&s->r_vals), s->R * 8)) != cudaSuccess) break;
        if ((e = cudaMallocHost(reinterpret_cast<void**>(&s->r_res), s->R * sizeof(pi_result_t))) != cudaSuccess) break;
        s->slots.resize(s->nslots);
        for (auto& sl : s->slots) {
            if ((e = cudaMalloc(reinterpret_cast<void**>(&sl.d_ops), s->max_batch)) != cudaSuccess) break;
            if ((e = cudaMalloc(reinterpret_cast<void**>(&sl.d_keys), (size_t)s->max_batch * 8)) != cudaSuccess) break;
            if ((e = cudaMalloc(reinterpret_cast<void**>(&sl.d_vals), (size_t)s->max_batch * 8)) != cudaSuccess) break;
            if ((e = cudaMalloc(reinterpret_cast<void**>(&sl.d_res), (size_t)s->max_batch * sizeof(pi_result_t))) !=
                cudaSuccess)
                break;
            if ((e = cudaEventCreateWithFlags(&sl.ev_in, cudaEventDisableTiming)) != cudaSuccess) break;
            if ((e = cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming)) != cudaSuccess) break;
            if ((e = cudaEventCreateWithFlags(&sl.ev_out, cudaEventDisableTiming)) != cudaSuccess) break;
        }
        if (e != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&s->hs, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&s->ds, cudaStreamNonBlocking)) != cudaSuccess) break;
        // the index's earlier work (on the legacy default stream or elsewhere) is done first
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) break;
        // the index's per-batch scratch, sized for the largest coalesced batch now: growing
        // it later synchronises and reallocates in the middle of the first bursts
        if (pi::reserve_batch(idx, s->max_batch, s->cs) != PI_OK) {
            e = cudaErrorMemoryAllocation;
            break;
        }
    } while (0);
    if (e != cudaSuccess) {
        pi::set_last_error(map_err(e));
        free_server(s);
        return nullptr;
    }
    try {
        s->worker = std::thread(run_dispatcher, s);
    } catch (...) {
        pi::set_last_error(PI_ERR_OOM);
        free_server(s);
        return nullptr;
    }
    return s;
}

int pi_server_submit(pi_server_t* s, const uint8_t* ops, const uint64_t* keys, const uint64_t* values, uint32_t n,
                     uint64_t* ticket_out) {
    if (!s || !ops || !keys || !values) return PI_ERR_INVALID_ARG;
    const uint64_t off = 0;
    const int64_t t = now_ns();
    uint64_t pos = 0, ticket = 0;
    const int rc = reserve_group(s, &n, 1, &t, &pos, &ticket);
    if (rc != PI_OK) return rc;
    fill_group(s, ops, keys, values, &n, &off, 1, &pos, ticket);
    if (ticket_out) *ticket_out = ticket;
    return PI_OK;
}

int pi_server_wait(pi_server_t* s, uint64_t ticket, pi_result_t* results_out, double* latency_s) {
    if (!s) return PI_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket != s->first) return PI_ERR_INVALID_ARG;  // not the oldest uncollected request
    // the request may not be submitted yet (a collector thread runs ahead of the submitter)
    if (s->reqs.empty()) {
        s->submit_waiters++;
        s->cv_done.wait(lk, [&] { return !s->reqs.empty() || s->error != PI_OK; });
        s->submit_waiters--;
    }
    if (s->reqs.empty()) return s->error;
    s->cv_done.wait(lk, [&] { return s->reqs.front().done || s->error != PI_OK; });
    Req r = s->reqs.front();
    if (!r.done) return s->error;
    lk.unlock();
    if (results_out) std::memcpy(results_out, s->r_res + r.pos % s->R, (size_t)r.n * sizeof(pi_result_t));
    if (latency_s) *latency_s = (double)(r.t_done - r.t_arrive) * 1e-9;
    lk.lock();
    s->reqs.pop_front();
    s->first++;
    lk.unlock();
    s->cv_space.notify_all();
    return s->error;
}

int pi_server_stats(pi_server_t* s, pi_server_stats_t* out, int reset) {
    if (!s || !out) return PI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->requests = s->n_req;
    out->queries = s->n_q;
    out->batches = s->n_batches;
    out->max_in_flight = s->max_inflight;
    std::vector<double> v = s->lat;
    out->p50_s = pct(v, 0.50);
    out->p99_s = pct(v, 0.99);
    out->max_s = v.empty() ? 0.0 : *std::max_element(v.begin(), v.end());
    out->mean_batch = s->n_batches ? (double)s->n_q / (double)s->n_batches : 0.0;
    if (reset) {
        s->lat.clear();
        s->n_req = s->n_q = s->n_batches = 0;
        s->max_inflight = s->inflight;
    }
    return s->error;
}

int pi_server_replay(pi_server_t* s, const uint8_t* ops, const uint64_t* keys, const uint64_t* values,
                     const uint32_t* sizes, const double* arrival_s, uint32_t nreq, pi_result_t* results_out,
                     double* latency_s_out) {
    if (!s || !ops || !keys || !values || !sizes || !arrival_s) return PI_ERR_INVALID_ARG;
    uint64_t first;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        first = s->first + s->reqs.size();
    }
    std::vector<uint64_t> offs(nreq + 1, 0);
    for (uint32_t i = 0; i < nreq; ++i) offs[i + 1] = offs[i] + sizes[i];
    std::atomic<int> rc_collect{PI_OK};
    std::thread collector([&] {
        uint32_t i = 0;
        while (i < nreq) {  // every finished request at once, in ticket order
            const int64_t k = collect_group(s, first + i, nreq - i, results_out, offs.data() + i,
                                            latency_s_out ? latency_s_out + i : nullptr);
            if (k <= 0) {
                const int rc = k < 0 ? (int)k : PI_ERR_INVALID_ARG;
                rc_collect = rc;
                std::lock_guard<std::mutex> lk(s->mu);  // release a submitter waiting for space
                if (s->error == PI_OK) s->error = rc;
                s->cv_space.notify_all();
                s->cv_done.notify_all();
                return;
            }
            i += (uint32_t)k;
        }
    });
    int rc = PI_OK;
    const int64_t t0 = now_ns();
    std::vector<int64_t> target(nreq);
    for (uint32_t i = 0; i < nreq; ++i) target[i] = t0 + (int64_t)(arrival_s[i] * 1e9);
    // Copy helpers: the main thread reserves groups in arrival order, the helpers copy
    // them into the ring (round robin), so submission is not bound by one memcpy stream.
    struct Job {
        uint32_t i, k;
        uint64_t ticket;
        std::vector<uint64_t> pos;
    };
    const uint32_t nhelp = std::max(1u, std::min(8u, std::thread::hardware_concurrency() / 2));
    std::vector<std::deque<Job>> jobs(nhelp);
    std::mutex jmu;
    std::condition_variable jcv;
    bool jdone = false;
    std::vector<std::thread> helpers;
    for (uint32_t h = 0; h < nhelp; ++h)
        helpers.emplace_back([&, h] {
            std::unique_lock<std::mutex> lk(jmu);
            while (true) {
                jcv.wait(lk, [&] { return jdone || !jobs[h].empty(); });
                if (jobs[h].empty()) return;
                Job jb = std::move(jobs[h].front());
                jobs[h].pop_front();
                lk.unlock();
                fill_group(s, ops, keys, values, sizes + jb.i, offs.data() + jb.i, jb.k, jb.pos.data(), jb.ticket);
                lk.lock();
            }
        });
    uint32_t i = 0, rr = 0;
    while (i < nreq && rc == PI_OK) {
        while (now_ns() < target[i]) {
            if (target[i] - now_ns() > 200000) std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        // every request already due goes in one group (bounded so the ring can hold it)
        const int64_t now = now_ns();
        uint32_t k = 1;
        uint64_t q = sizes[i];
        while (i + k < nreq && k < 1024 && target[i + k] <= now && q + sizes[i + k] <= s->R / 8) q += sizes[i + k++];
        Job jb{i, k, 0, std::vector<uint64_t>(k)};
        rc = reserve_group(s, sizes + i, k, target.data() + i, jb.pos.data(), &jb.ticket);
        if (rc == PI_OK && jb.ticket != first + i) rc = PI_ERR_INVALID_ARG;  // another client interleaved
        if (rc == PI_OK) {
            {
                std::lock_guard<std::mutex> lk(jmu);
                jobs[rr].push_back(std::move(jb));
            }
            jcv.notify_all();
            rr = (rr + 1) % nhelp;
        }
        i += k;
    }
    {
        std::lock_guard<std::mutex> lk(jmu);
        jdone = true;
    }
    jcv.notify_all();
    for (auto& t : helpers) t.join();
    if (rc != PI_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error == PI_OK) s->error = rc;
        s->cv_done.notify_all();
    }
    collector.join();
    return rc != PI_OK ? rc : rc_collect.load();
}

void pi_server_destroy(pi_server_t* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->cs);
    cudaStreamSynchronize(s->ds);
    free_server(s);
}

}  // extern "C"
