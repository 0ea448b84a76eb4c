// Re-plan serving with continuous batching on one GPU.
//
// A dispatcher thread admits queued requests in arrival order while a slot is
// free and the request's device footprint fits.  Every slot has a host thread
// of its own: it gives its request a context (and so its own stream), queues
// all of the request's column-generation rounds as CUDA graphs at once, waits
// for the event recorded after them, copies the results into the request's
// buffers and releases the context.  Plans run concurrently, each on its own
// stream, and a plan's host work (upload, device build, read-back) never waits
// behind another plan's: a request's latency is its own work plus its share of
// the GPU.  With solve_slots = n > 0 the admitted requests still create their
// contexts alongside the running plans, but queue their rounds in admission
// order, at most n plans' rounds on the GPU at a time (a plan's persistent
// master solve occupies every SM, so two plans' rounds interleave rather than
// overlap).  Submitters and pollers only touch the queue and the result table
// under the mutex.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dao_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t1) {
    return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2 };

struct Request {
    dao_request r{};
    int64_t footprint = 0;
    int64_t order = 0;           // admission order: the turn of its rounds on the GPU
    int state = REQ_QUEUED;
    Clock::time_point t_submit, t_admit, t_done;
    dao_result res{};
};

struct Slot {
    bool busy = false;           // a request is assigned and not yet retired
    bool pending = false;        // assigned, not yet picked up by the slot's thread
    int64_t id = -1;
    dao_ctx* ctx = nullptr;
    cudaEvent_t done = nullptr;
    Clock::time_point sim_end;
    Clock::time_point t_queued;  // the plan's rounds were queued
    std::condition_variable cv;  // a request was assigned, or the server stops
    std::thread th;
};

void set_msg(dao_result* r, const char* msg) {
    std::strncpy(r->error, msg ? msg : "", sizeof(r->error) - 1);
    r->error[sizeof(r->error) - 1] = '\0';
}

}  // namespace

struct dao_server {
    dao_server_options opt{};
    bool simulate = false;
    std::mutex mu;
    std::condition_variable cv_work;  // new request or shutdown
    std::condition_variable cv_done;  // a request finished
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Request> reqs;
    std::vector<Slot> slots;
    bool stop_slots = false;  // the slot threads leave once idle
    int64_t next_id = 1;
    bool stop = false;
    int64_t bytes_in_use = 0;
    int64_t capacity = 0;  // the most a single plan may ever hold
    // plans whose rounds are on the GPU (opt.solve_slots > 0 bounds them):
    // requests take their turn in admission order once their context exists
    std::mutex mu_solve;
    std::condition_variable cv_solve;
    int solves_on_gpu = 0;
    int64_t next_turn = 0;   // admission order of the next request to take its turn
    int64_t next_order = 0;  // admission counter
    dao_server_stats stats{};
    std::thread worker;

    bool fits(int64_t fp) {
        if (opt.hbm_budget_bytes > 0) return bytes_in_use + fp <= opt.hbm_budget_bytes;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return (int64_t)free_b - opt.hbm_reserve_bytes >= fp;
    }

    // Slot thread, without the lock: this request's turn to put its rounds on
    // the GPU (in admission order, while fewer than solve_slots plans' rounds
    // are there); every admitted request takes its turn, a failed one too.
    void take_turn(Request& q) {
        if (opt.solve_slots <= 0) return;
        std::unique_lock<std::mutex> l(mu_solve);
        cv_solve.wait(l, [&] { return next_turn == q.order && solves_on_gpu < opt.solve_slots; });
        ++next_turn;
        ++solves_on_gpu;
        cv_solve.notify_all();  // the next turn may already be free
    }
    void end_turn() {
        if (opt.solve_slots <= 0) return;
        {
            std::lock_guard<std::mutex> l(mu_solve);
            --solves_on_gpu;
        }
        cv_solve.notify_all();
    }

    // Slot thread, without the lock: create the plan, take the request's turn,
    // queue its rounds.
    void start(Slot& s, Request& q) {
        if (simulate) {
            const Clock::time_point t0 = Clock::now();
            take_turn(q);
            q.res.gpu_wait_ms = ms_since(t0, Clock::now());
            s.sim_end = Clock::now() + std::chrono::microseconds(
                                           (int64_t)std::llround(1e3 * opt.simulate_ms_per_aperture * q.r.n_apertures));
            return;
        }
        dao_options po = opt.plan_options;
        po.stream = nullptr;  // the context makes its own stream
        po.device = opt.device;
        po.use_graphs = 1;
        const Clock::time_point t0 = Clock::now();
        dao_status st = dao_create(&q.r.D, &q.r.geometry, &q.r.structures, &q.r.weights, q.r.prescriptions, &po,
                                   &s.ctx);
        const Clock::time_point t1 = Clock::now();
        q.res.create_ms = ms_since(t0, t1);
        take_turn(q);
        q.res.gpu_wait_ms = ms_since(t1, Clock::now());
        if (st == DAO_OK) {
            // blocking sync: the slot's thread sleeps in the driver while its plan runs
            // instead of polling, which would contend for the driver with the other
            // slots' host work
            if (!s.done &&
                cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming | cudaEventBlockingSync) != cudaSuccess) {
                cudaGetLastError();
                st = dao::set_error(DAO_ECUDA, "cudaEventCreate failed");
            }
        }
        if (st == DAO_OK) st = dao::solve_async_begin(s.ctx, q.r.n_apertures, s.done);
        s.t_queued = Clock::now();
        if (st != DAO_OK) {
            q.res.status = st;
            set_msg(&q.res, dao_last_error());
            if (s.ctx) dao_destroy(s.ctx);
            s.ctx = nullptr;
        }
    }

    // Slot thread, without the lock: until the plan's event has completed.
    void wait_plan(Slot& s) {
        if (simulate) {
            std::this_thread::sleep_until(s.sim_end);
            return;
        }
        if (s.ctx == nullptr) return;  // failed at start
        if (cudaEventSynchronize(s.done) != cudaSuccess) cudaGetLastError();  // surfaced by the read-back
    }

    // Slot thread, without the lock: results into the caller's buffers.
    void finish(Slot& s, Request& q) {
        if (simulate) {
            q.res.status = DAO_OK;
            q.res.n_apertures = q.r.n_apertures;
            q.res.objective = std::numeric_limits<double>::quiet_NaN();
            return;
        }
        if (s.ctx == nullptr) return;  // q.res already holds the error
        const Clock::time_point t0 = Clock::now();
        q.res.solve_ms = ms_since(s.t_queued, t0);
        dao_status result = DAO_OK;
        int32_t n = 0;
        dao_status st = dao::solve_async_end(s.ctx, q.r.n_apertures, &n, &result);
        double F = std::numeric_limits<double>::quiet_NaN();
        if (st == DAO_OK) st = dao_dose(s.ctx, q.r.dose_out, &F);
        if (st == DAO_OK && q.r.intensities_out) st = dao_intensities(s.ctx, q.r.intensities_out, nullptr);
        if (st == DAO_OK && (q.r.beams_out || q.r.leaves_out)) {
            std::vector<int32_t> beams(opt.plan_options.k_max > 0 ? opt.plan_options.k_max : 1);
            int32_t k = 0;
            st = dao_apertures(s.ctx, beams.data(), q.r.leaves_out, &k);
            if (st == DAO_OK && q.r.beams_out) std::memcpy(q.r.beams_out, beams.data(), sizeof(int32_t) * k);
        }
        q.res.status = st != DAO_OK ? st : result;
        if (st != DAO_OK || (result != DAO_OK && result != DAO_OPTIMAL && result != DAO_DUPLICATE))
            set_msg(&q.res, dao_last_error());
        q.res.n_apertures = n;
        q.res.objective = F;
        dao_destroy(s.ctx);
        s.ctx = nullptr;
        q.res.finish_ms = ms_since(t0, Clock::now());
    }

    // One slot's host thread: start, wait, finish and retire each request the
    // dispatcher assigns to it.
    void slot_main(Slot& s) {
        if (!simulate) cudaSetDevice(opt.device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            s.cv.wait(lk, [&] { return s.pending || stop_slots; });
            if (!s.pending) break;  // stopping, idle
            s.pending = false;
            Request& q = reqs[s.id];
            lk.unlock();
            start(s, q);
            wait_plan(s);
            end_turn();  // the plan's rounds have left the GPU
            finish(s, q);
            lk.lock();
            q.state = REQ_DONE;
            q.t_done = Clock::now();
            q.res.run_ms = ms_since(q.t_admit, q.t_done);
            q.res.latency_ms = ms_since(q.t_submit, q.t_done);
            const bool ok = q.res.status == DAO_OK || q.res.status == DAO_OPTIMAL || q.res.status == DAO_DUPLICATE;
            if (ok) ++stats.completed; else ++stats.failed;
            bytes_in_use -= q.footprint;
            s.busy = false;
            s.id = -1;
            --stats.active;
            cv_done.notify_all();
            cv_work.notify_all();  // a slot and memory are free again
        }
    }

    // The dispatcher: admission in arrival order.
    void run() {
        if (!simulate) cudaSetDevice(opt.device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            while (!queue.empty() && !stop) {
                Slot* free_slot = nullptr;
                for (Slot& s : slots)
                    if (!s.busy) {
                        free_slot = &s;
                        break;
                    }
                if (!free_slot) break;
                const int64_t id = queue.front();
                Request& q = reqs[id];
                if (q.footprint > capacity) {  // can never fit: reject instead of blocking the queue
                    queue.pop_front();
                    q.state = REQ_DONE;
                    q.t_admit = q.t_done = Clock::now();
                    q.res.status = DAO_ENOMEM;
                    set_msg(&q.res, ("footprint of " + std::to_string(q.footprint) +
                                     " bytes exceeds what the server can ever admit").c_str());
                    q.res.queue_ms = q.res.latency_ms = ms_since(q.t_submit, q.t_done);
                    ++stats.rejected;
                    cv_done.notify_all();
                    continue;
                }
                if (!fits(q.footprint)) break;  // wait for a running plan to retire
                queue.pop_front();
                q.state = REQ_RUNNING;
                q.order = next_order++;
                q.t_admit = Clock::now();
                q.res.queue_ms = ms_since(q.t_submit, q.t_admit);
                free_slot->busy = true;
                free_slot->pending = true;
                free_slot->id = id;
                bytes_in_use += q.footprint;
                ++stats.active;
                if (stats.active > stats.max_active) stats.max_active = stats.active;
                free_slot->cv.notify_one();
            }
            stats.queued = (int32_t)queue.size();
            stats.bytes_in_use = bytes_in_use;
            if (stop && stats.active == 0 && queue.empty()) break;
            // woken by a submission, a retired plan or shutdown; the timeout
            // re-reads the free device memory while requests wait for it
            cv_work.wait_for(lk, std::chrono::milliseconds(queue.empty() ? 50 : 1));
        }
        stop_slots = true;
        for (Slot& s : slots) s.cv.notify_all();
    }
};

extern "C" {

void dao_server_options_default(dao_server_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->max_slots = 8;
    opt->queue_capacity = 1024;
    opt->hbm_reserve_bytes = (int64_t)2 << 30;
    opt->hbm_budget_bytes = 0;
    opt->device = 0;
    opt->simulate_ms_per_aperture = 0.0;
    dao_options_default(&opt->plan_options);
    opt->prewarm_bytes = (int64_t)2 << 30;
}

int64_t dao_server_footprint(const dao_request* req, const dao_options* plan_options) {
    if (!req) return 0;
    dao_options po;
    dao_options_default(&po);
    if (plan_options) po = *plan_options;
    const int64_t V = req->D.n_voxels, N = req->D.n_beamlets, nnz = req->D.nnz, B = req->geometry.n_beams;
    const bool wide = po.precision == DAO_PREC_FP32;
    const int64_t pad = wide ? 4 : 8;
    const int64_t ld = (V + dao::MASTER_TILE - 1) / dao::MASTER_TILE * dao::MASTER_TILE;
    const int64_t d_bytes = (V + 1) * 4 + (nnz + V * (pad - 1)) * (wide ? 8 : 4);
    const int64_t t_bytes = (N + 1) * 4 + (nnz + N * (pad - 1)) * (wide ? 8 : 6) + (wide ? 0 : N * 4);
    const int64_t master = ld * 4 * (dao::KMAX + dao::KROW) + ld * 8 + V * 4 * 4;
    // temporaries of the device build, alive together until the transpose is placed
    const int64_t CH = std::max<int64_t>(256, (V * N / (16 << 20) + 31) / 32 * 32);
    const int64_t build = (V + 1) * 8 + nnz * 8 + V * 12 + ((V + CH - 1) / CH) * N * 4 + N * 8 +
                          (wide ? 0 : (nnz + N * (pad - 1)) * 4);
    const int64_t by_beams = B * (V + 1) * 4 + nnz * (wide ? 6 : 4);  // D by beams for the aperture column
    return d_bytes + t_bytes + (B + 1) * V * 4 + by_beams + V + master + N * 64 + build + ((int64_t)40 << 20);
}

dao_status dao_server_create(const dao_server_options* opt_in, dao_server** out) {
    if (!out) return dao::set_error(DAO_EINVAL, "null output pointer");
    *out = nullptr;
    dao_server_options opt;
    dao_server_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.max_slots < 1 || opt.queue_capacity < 1 || opt.hbm_reserve_bytes < 0 || opt.hbm_budget_bytes < 0 ||
        !(opt.simulate_ms_per_aperture >= 0.0) || opt.prewarm_bytes < 0 || opt.solve_slots < 0)
        return dao::set_error(DAO_EINVAL,
                              "max_slots, queue_capacity >= 1; reserve, budget, simulation time, solve_slots >= 0");
    const bool simulate = opt.simulate_ms_per_aperture > 0.0;
    if (simulate && opt.hbm_budget_bytes <= 0)
        return dao::set_error(DAO_EINVAL, "simulation needs hbm_budget_bytes > 0 as its device memory");
    int64_t capacity = opt.hbm_budget_bytes;
    if (!simulate) {
        cudaError_t e = cudaSetDevice(opt.device);
        size_t free_b = 0, total_b = 0;
        if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess)
            return dao::set_error(DAO_ECUDA, std::string("dao_server_create: ") + cudaGetErrorString(e));
        const int64_t dev_cap = (int64_t)total_b - opt.hbm_reserve_bytes;
        capacity = opt.hbm_budget_bytes > 0 ? std::min<int64_t>(opt.hbm_budget_bytes, dev_cap) : dev_cap;
        if (opt.prewarm_bytes > 0) {
            // the pool keeps freed memory mapped (up to its release threshold), and the
            // staging free list keeps page-locked blocks: both taken once, here
            cudaStream_t st = nullptr;
            void* p = nullptr;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            const size_t want = (size_t)std::min<int64_t>(opt.prewarm_bytes, std::max<int64_t>(capacity / 2, 0));
            if (e == cudaSuccess && want > 0 && dao::pool_alloc(&p, want, opt.device, st) == cudaSuccess)
                dao::pool_free(p, st);
            if (e == cudaSuccess) cudaStreamSynchronize(st);
            if (st) cudaStreamDestroy(st);
            cudaGetLastError();  // prewarming is best effort
            std::vector<std::pair<void*, size_t>> blocks;
            for (int i = 0; i < opt.max_slots + 2; ++i) {
                void* h = nullptr;
                size_t b = (size_t)64 << 10;
                if (dao::pinned_alloc(&h, &b) != cudaSuccess) {
                    cudaGetLastError();
                    break;
                }
                blocks.emplace_back(h, b);
            }
            for (auto& hb : blocks) dao::pinned_release(hb.first, hb.second);
        }
    }
    dao_server* s = new (std::nothrow) dao_server();
    if (!s) return dao::set_error(DAO_ENOMEM, "host allocation failed");
    s->opt = opt;
    s->simulate = simulate;
    s->capacity = capacity;
    s->slots = std::vector<Slot>(opt.max_slots);
    for (Slot& sl : s->slots) sl.th = std::thread([s, &sl] { s->slot_main(sl); });
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return DAO_OK;
}

dao_status dao_server_submit(dao_server* s, const dao_request* req, int64_t* id) {
    if (!s || !req || !id) return dao::set_error(DAO_EINVAL, "null argument");
    if (req->n_apertures < 0) return dao::set_error(DAO_EINVAL, "negative aperture count");
    Request q;
    q.r = *req;
    q.t_submit = Clock::now();
    q.footprint = dao_server_footprint(req, &s->opt.plan_options);
    // host-only validation up front: an invalid request finishes at once
    dao_options po = s->opt.plan_options;
    po.device = s->opt.device;
    const dao_status v = dao::check_inputs(&req->D, &req->geometry, &req->structures, &req->weights,
                                           req->prescriptions, &po);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return dao::set_error(DAO_ESTATE, "server is shutting down");
    if (v != DAO_OK) {
        q.state = REQ_DONE;
        q.t_admit = q.t_done = q.t_submit;
        q.res.status = v;
        set_msg(&q.res, dao_last_error());
        *id = s->next_id++;
        s->reqs.emplace(*id, q);
        ++s->stats.submitted;
        ++s->stats.failed;
        s->cv_done.notify_all();
        return DAO_OK;
    }
    if ((int)s->queue.size() >= s->opt.queue_capacity) return dao::set_error(DAO_EBUSY, "request queue is full");
    *id = s->next_id++;
    s->reqs.emplace(*id, q);
    s->queue.push_back(*id);
    ++s->stats.submitted;
    s->stats.queued = (int32_t)s->queue.size();
    s->cv_work.notify_all();
    return DAO_OK;
}

dao_status dao_server_poll(dao_server* s, int64_t id, dao_result* out) {
    if (!s) return dao::set_error(DAO_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return dao::set_error(DAO_EINVAL, "unknown request id " + std::to_string(id));
    if (it->second.state != REQ_DONE) return DAO_EBUSY;
    if (out) *out = it->second.res;
    s->reqs.erase(it);
    return DAO_OK;
}

dao_status dao_server_wait(dao_server* s, int64_t id, double timeout_ms, dao_result* out) {
    if (!s) return dao::set_error(DAO_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1e3));
    for (;;) {
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return dao::set_error(DAO_EINVAL, "unknown request id " + std::to_string(id));
        if (it->second.state == REQ_DONE) {
            if (out) *out = it->second.res;
            s->reqs.erase(it);
            return DAO_OK;
        }
        if (timeout_ms < 0) {
            s->cv_done.wait(lk);
        } else if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto jt = s->reqs.find(id);
            if (jt != s->reqs.end() && jt->second.state == REQ_DONE) continue;
            return dao::set_error(DAO_ETIMEOUT, "request " + std::to_string(id) + " still running");
        }
    }
}

dao_status dao_server_stats_get(dao_server* s, dao_server_stats* out) {
    if (!s || !out) return dao::set_error(DAO_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = (int32_t)s->queue.size();
    out->bytes_in_use = s->bytes_in_use;
    return DAO_OK;
}

void dao_server_destroy(dao_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (int64_t id : s->queue) {  // cancel what has not started
            Request& q = s->reqs[id];
            q.state = REQ_DONE;
            q.res.status = DAO_ESTATE;
            set_msg(&q.res, "server destroyed before the request started");
        }
        s->queue.clear();
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();  // the dispatcher waits for the running plans first
    for (Slot& sl : s->slots)
        if (sl.th.joinable()) sl.th.join();
    for (Slot& sl : s->slots) {
        if (sl.ctx) dao_destroy(sl.ctx);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    delete s;
}

}  // extern "C"
