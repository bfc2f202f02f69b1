// Continuous-batching likelihood server (fg21_serve_* of fg21.h).
//
// Many nested-sampling runs (Sec. 3: each run deletes a batch of live points
// and evolves slice-sampling chains, every chain step needing one likelihood)
// submit requests of P points against their own device-resident model.  A
// batcher thread packs pending requests of admitted runs into one persistent
// launch (one request never shares a work item with another) on one of up to
// `max_inflight` streams, so requests that arrive while earlier launches run
// are packed into the next launch as soon as a slot is free; a completer thread
// waits on each launch's event, copies results to the callers' buffers and
// wakes their tickets.  Runs are admitted while their resident bytes fit the
// memory budget; the others wait in arrival order.
#include <cstdio>
#include <nvtx3/nvToolsExt.h>
#include <nvtx3/nvToolsExtCudaRt.h>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fg21_internal.h"
#include "fg21_model.h"

using Clock = std::chrono::steady_clock;

namespace fg21 {
namespace {

enum class TState { Pending, Running, Done };

struct Ticket {
    int64_t id;
    int run;
    int64_t P;
    std::vector<double> params;
    double *out;
    TState state = TState::Pending;
    int status = FG21_OK;
    Clock::time_point t_submit, t_done;
};

struct Run {
    int id;
    fg21_model *m;
    size_t bytes;
    bool admitted = false;
    int running = 0;    // tickets of this run inside a launch
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Workspace ws;
    char *d_io = nullptr, *h_io = nullptr;
    size_t io_cap = 0;
    bool busy = false;
    std::vector<Ticket *> batch;
    std::vector<size_t> loff;      // logL offsets in h_io
    size_t status_off = 0;         // copy of the device status word in h_io
    int launch_rc = FG21_OK;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace fg21

struct fg21_server {
    fg21_serve_opts opts;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_slot;
    std::map<int, fg21::Run> runs;
    std::deque<int> admission;          // waiting run ids, in order
    size_t admitted_bytes = 0;
    std::deque<fg21::Ticket *> pending;
    std::unordered_map<int64_t, fg21::Ticket *> tickets;
    std::vector<fg21::Slot> slots;
    std::deque<int> inflight;           // slot indices in launch order
    std::thread batcher, completer;
    bool stop = false;
    int next_run = 1;
    int64_t next_ticket = 1;
    // statistics
    std::vector<double> lat_ms;
    int64_t requests_done = 0, points_done = 0, launches = 0;
    double macs_done = 0;
    Clock::time_point t_create;
};

namespace fg21 {
namespace {

void admit_waiting(fg21_server *s) {
    while (!s->admission.empty()) {
        auto it = s->runs.find(s->admission.front());
        if (it == s->runs.end()) {
            s->admission.pop_front();
            continue;
        }
        if (s->admitted_bytes + it->second.bytes > s->opts.mem_budget_bytes) break;
        it->second.admitted = true;
        s->admitted_bytes += it->second.bytes;
        s->admission.pop_front();
    }
}

// Build and enqueue one launch on slot k from the pending queue (lock held).
// Returns false if there was nothing launchable.
bool launch_batch(fg21_server *s, int k, std::unique_lock<std::mutex> &lk) {
    Slot &sl = s->slots[k];
    sl.batch.clear();
    int64_t pts = 0;
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        Ticket *t = *it;
        Run &r = s->runs.at(t->run);
        if (!r.admitted) {
            ++it;
            continue;
        }
        if (!sl.batch.empty() && pts + t->P > s->opts.max_batch_points) break;
        sl.batch.push_back(t);
        pts += t->P;
        it = s->pending.erase(it);
    }
    if (sl.batch.empty()) return false;
    for (Ticket *t : sl.batch) {
        t->state = TState::Running;
        s->runs.at(t->run).running++;
    }
    sl.busy = true;
    // I/O layout: params of each request, then logL of each request
    std::vector<size_t> poff(sl.batch.size());
    sl.loff.assign(sl.batch.size(), 0);
    size_t off = 0;
    for (size_t j = 0; j < sl.batch.size(); ++j) {
        poff[j] = off;
        off += align256(sizeof(double) * sl.batch[j]->params.size());
    }
    const size_t lbase = off;
    for (size_t j = 0; j < sl.batch.size(); ++j) {
        sl.loff[j] = off;
        off += align256(sizeof(double) * sl.batch[j]->P);
    }
    sl.status_off = off;
    off += 256;
    std::vector<ReqDesc> reqs;
    std::vector<std::pair<Ticket *, fg21_model *>> work;
    for (Ticket *t : sl.batch) work.emplace_back(t, s->runs.at(t->run).m);
    lk.unlock();   // staging and launch without the server lock
    // profiler range (NVTX; near free when no tool is attached)
    char label[96];
    std::snprintf(label, sizeof label, "fg21 serve launch: slot %d, %zu requests, %lld points", k, work.size(),
                  (long long)pts);
    nvtxRangePushA(label);
    int rc = FG21_OK;
    do {
        if (off > sl.io_cap) {
            if (sl.d_io) cudaFree(sl.d_io);
            if (sl.h_io) cudaFreeHost(sl.h_io);
            sl.d_io = sl.h_io = nullptr;
            sl.io_cap = 0;
            size_t want = off + off / 2;
            if (cudaMalloc((void **)&sl.d_io, want) != cudaSuccess ||
                cudaMallocHost((void **)&sl.h_io, want) != cudaSuccess) {
                cudaGetLastError();
                rc = FG21_E_NOMEM;
                break;
            }
            sl.io_cap = want;
        }
        for (size_t j = 0; j < work.size(); ++j) {
            Ticket *t = work[j].first;
            std::memcpy(sl.h_io + poff[j], t->params.data(), sizeof(double) * t->params.size());
            reqs.push_back(model_request(work[j].second, (const double *)(sl.d_io + poff[j]), t->P,
                                         (double *)(sl.d_io + sl.loff[j]), s->opts.precision));
        }
        if (cudaMemcpyAsync(sl.d_io, sl.h_io, lbase, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess) {
            rc = cuda_error(cudaGetLastError(), "serve H2D");
            break;
        }
        rc = enqueue_requests(sl.ws, reqs, s->opts.precision, sl.stream);
        if (rc) break;
        if (cudaMemcpyAsync(sl.h_io + lbase, sl.d_io + lbase, sl.status_off - lbase, cudaMemcpyDeviceToHost,
                            sl.stream) != cudaSuccess ||
            cudaMemcpyAsync(sl.h_io + sl.status_off, sl.ws.d_status, 32, cudaMemcpyDeviceToHost, sl.stream) !=
                cudaSuccess) {
            rc = cuda_error(cudaGetLastError(), "serve D2H");
            break;
        }
        if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) {
            rc = cuda_error(cudaGetLastError(), "serve event");
            break;
        }
    } while (0);
    nvtxRangePop();
    lk.lock();
    sl.launch_rc = rc;
    s->inflight.push_back(k);
    s->launches++;
    s->cv_work.notify_all();
    return true;
}

void batcher_main(fg21_server *s) {
    cudaSetDevice(s->opts.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_work.wait(lk, [s] {
            if (s->stop) return true;
            bool any = false;
            for (Ticket *t : s->pending)
                if (s->runs.at(t->run).admitted) { any = true; break; }
            return any;
        });
        if (s->stop) break;
        // give the batch a moment to fill, but only while earlier launches keep
        // the GPU busy: with every slot free, what is pending goes at once
        // (waiting then would only add latency), and the wait ends early when
        // the batch is full or the GPU falls idle
        auto gpu_busy = [s] {
            for (const Slot &sl : s->slots)
                if (sl.busy) return true;
            return false;
        };
        int64_t pts = 0;
        for (Ticket *t : s->pending) pts += t->P;
        if (pts < s->opts.max_batch_points && s->opts.max_wait_us > 0 && gpu_busy()) {
            s->cv_work.wait_for(lk, std::chrono::microseconds(s->opts.max_wait_us), [s, &gpu_busy] {
                if (s->stop) return true;
                int64_t q = 0;
                for (Ticket *t : s->pending) q += t->P;
                return q >= s->opts.max_batch_points || !gpu_busy();
            });
            if (s->stop) break;
        }
        // a free slot
        int k = -1;
        s->cv_slot.wait(lk, [s, &k] {
            if (s->stop) return true;
            for (size_t j = 0; j < s->slots.size(); ++j)
                if (!s->slots[j].busy) { k = (int)j; return true; }
            return false;
        });
        if (s->stop) break;
        launch_batch(s, k, lk);
    }
}

void completer_main(fg21_server *s) {
    cudaSetDevice(s->opts.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_work.wait(lk, [s] { return s->stop || !s->inflight.empty(); });
        if (s->inflight.empty() && s->stop) break;
        const int k = s->inflight.front();
        s->inflight.pop_front();
        Slot &sl = s->slots[k];
        lk.unlock();
        nvtxRangePushA("fg21 serve completion: wait for the launch, copy results");
        int rc = sl.launch_rc;
        if (rc == FG21_OK) {
            if (cudaEventSynchronize(sl.done) != cudaSuccess) {
                cudaGetLastError();
                rc = FG21_E_CUDA;
            } else {
                unsigned st = 0;
                std::memcpy(&st, sl.h_io + sl.status_off, sizeof st);
                if (st) rc = FG21_E_DEVICE;
            }
        }
        if (rc == FG21_OK)
            for (size_t j = 0; j < sl.batch.size(); ++j)
                std::memcpy(sl.batch[j]->out, sl.h_io + sl.loff[j], sizeof(double) * sl.batch[j]->P);
        const auto now = Clock::now();
        nvtxRangePop();
        lk.lock();
        for (Ticket *t : sl.batch) {
            t->state = TState::Done;
            t->status = rc;
            t->t_done = now;
            auto it = s->runs.find(t->run);
            if (it != s->runs.end()) {
                it->second.running--;
                s->macs_done += (double)it->second.m->N * it->second.m->F * it->second.m->T * t->P;
            }
            s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - t->t_submit).count());
            s->requests_done++;
            s->points_done += t->P;
        }
        sl.batch.clear();
        sl.busy = false;
        s->cv_done.notify_all();
        s->cv_slot.notify_all();
        s->cv_work.notify_all();   // a batcher filling a launch stops waiting once the GPU is idle
    }
}

int finish_ticket(fg21_server *s, Ticket *t) {
    int rc = t->status;
    s->tickets.erase(t->id);
    delete t;
    return rc;
}

}  // namespace
}  // namespace fg21

using namespace fg21;

extern "C" {

int fg21_serve_create(const fg21_serve_opts *opts, fg21_server **out) {
    if (!opts || !out) return set_error(FG21_E_ARG, "NULL opts/out");
    *out = nullptr;
    if (opts->max_batch_points < 1 || opts->max_inflight < 1 || opts->max_inflight > 8 || opts->max_wait_us < 0)
        return set_error(FG21_E_ARG, "bad serve options");
    if (opts->precision < 0 || opts->precision > 3) return set_error(FG21_E_ARG, "bad precision");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || opts->device < 0 || opts->device >= ndev) {
        cudaGetLastError();
        return set_error(FG21_E_CUDA, "device %d not available", opts->device);
    }
    fg21_server *s = new fg21_server();
    s->opts = *opts;
    s->t_create = Clock::now();
    s->slots.resize(opts->max_inflight);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(opts->device);
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            cudaSetDevice(prev);
            fg21_serve_destroy(s);
            return set_error(FG21_E_CUDA, "stream/event creation failed");
        }
        char name[48];
        std::snprintf(name, sizeof name, "fg21 serve slot %d", (int)(&sl - s->slots.data()));
        nvtxNameCudaStreamA(sl.stream, name);      // labels the slot's stream in a profiler trace
    }
    cudaSetDevice(prev);
    s->batcher = std::thread(batcher_main, s);
    s->completer = std::thread(completer_main, s);
    *out = s;
    return FG21_OK;
}

int fg21_serve_destroy(fg21_server *s) {
    if (!s) return FG21_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // cancel what never started; let launches in flight finish
        for (Ticket *t : s->pending) {
            t->state = TState::Done;
            t->status = FG21_E_CANCELLED;
        }
        s->pending.clear();
        s->cv_done.wait(lk, [s] {
            for (auto &sl : s->slots)
                if (sl.busy) return false;
            return true;
        });
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_slot.notify_all();
    }
    if (s->batcher.joinable()) s->batcher.join();
    if (s->completer.joinable()) s->completer.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->opts.device);
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        sl.ws.release();
        if (sl.d_io) cudaFree(sl.d_io);
        if (sl.h_io) cudaFreeHost(sl.h_io);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    cudaSetDevice(prev);
    for (auto &kv : s->tickets) delete kv.second;
    delete s;
    return FG21_OK;
}

int fg21_serve_register_run(fg21_server *s, fg21_model *m, int32_t *run_id) {
    if (!s || !m || !run_id) return set_error(FG21_E_ARG, "NULL argument");
    if (m->device != s->opts.device) return set_error(FG21_E_ARG, "model lives on another device");
    if ((s->opts.precision == FG21_PREC_FP16X3 || s->opts.precision == FG21_PREC_BF16X3) &&
        m->N > FG21_MAX_REGIONS_TC)
        return set_error(FG21_E_RANGE, "N = %d above the tensor-core limit", m->N);
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t bytes = m->resident_bytes;
    if (bytes > s->opts.mem_budget_bytes)
        return set_error(FG21_E_RANGE, "run needs %zu bytes, budget is %zu", bytes, s->opts.mem_budget_bytes);
    Run r;
    r.id = s->next_run++;
    r.m = m;
    r.bytes = bytes;
    s->runs[r.id] = r;
    *run_id = r.id;
    if (s->admission.empty() && s->admitted_bytes + bytes <= s->opts.mem_budget_bytes) {
        s->runs[r.id].admitted = true;
        s->admitted_bytes += bytes;
        return FG21_OK;
    }
    s->admission.push_back(r.id);
    return FG21_E_BUSY;
}

int fg21_serve_unregister_run(fg21_server *s, int32_t run_id) {
    if (!s) return set_error(FG21_E_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->runs.find(run_id);
    if (it == s->runs.end()) return set_error(FG21_E_NOTFOUND, "unknown run %d", run_id);
    for (auto p = s->pending.begin(); p != s->pending.end();) {
        if ((*p)->run == run_id) {
            (*p)->state = TState::Done;
            (*p)->status = FG21_E_CANCELLED;
            (*p)->t_done = Clock::now();
            p = s->pending.erase(p);
        } else {
            ++p;
        }
    }
    s->cv_done.notify_all();
    // launches holding this run's model must finish before the run goes away
    s->cv_done.wait(lk, [s, run_id] { return s->runs.at(run_id).running == 0; });
    if (s->runs.at(run_id).admitted) s->admitted_bytes -= s->runs.at(run_id).bytes;
    s->runs.erase(run_id);
    s->admission.erase(std::remove(s->admission.begin(), s->admission.end(), run_id), s->admission.end());
    admit_waiting(s);
    s->cv_work.notify_all();
    return FG21_OK;
}

int fg21_serve_submit(fg21_server *s, int32_t run_id, const double *params, int64_t P, double *logL_out,
                      fg21_ticket *ticket) {
    if (!s || !ticket || P < 1 || !params || !logL_out) return set_error(FG21_E_ARG, "bad submit arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->runs.find(run_id);
    if (it == s->runs.end()) return set_error(FG21_E_NOTFOUND, "unknown run %d", run_id);
    if (P > s->opts.max_batch_points)
        return set_error(FG21_E_RANGE, "request of %lld points above max_batch_points", (long long)P);
    Ticket *t = new Ticket();
    t->id = s->next_ticket++;
    t->run = run_id;
    t->P = P;
    t->params.assign(params, params + (size_t)P * it->second.m->n_params());
    t->out = logL_out;
    t->t_submit = Clock::now();
    s->tickets[t->id] = t;
    s->pending.push_back(t);
    *ticket = t->id;
    s->cv_work.notify_all();
    return FG21_OK;
}

int fg21_serve_wait(fg21_server *s, fg21_ticket tk, int32_t timeout_ms) {
    if (!s) return set_error(FG21_E_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(tk);
    if (it == s->tickets.end()) return set_error(FG21_E_NOTFOUND, "unknown ticket %lld", (long long)tk);
    Ticket *t = it->second;
    auto done = [t] { return t->state == TState::Done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        return set_error(FG21_E_TIMEOUT, "ticket %lld not done after %d ms", (long long)tk, timeout_ms);
    }
    return finish_ticket(s, t);
}

int fg21_serve_poll(fg21_server *s, fg21_ticket tk) {
    if (!s) return set_error(FG21_E_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(tk);
    if (it == s->tickets.end()) return set_error(FG21_E_NOTFOUND, "unknown ticket %lld", (long long)tk);
    if (it->second->state != TState::Done) return FG21_E_BUSY;
    return finish_ticket(s, it->second);
}

int fg21_serve_cancel(fg21_server *s, fg21_ticket tk) {
    if (!s) return set_error(FG21_E_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(tk);
    if (it == s->tickets.end()) return set_error(FG21_E_NOTFOUND, "unknown ticket %lld", (long long)tk);
    Ticket *t = it->second;
    if (t->state != TState::Pending) return set_error(FG21_E_STATE, "ticket already running or done");
    s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), t), s->pending.end());
    t->state = TState::Done;
    t->status = FG21_E_CANCELLED;
    t->t_done = Clock::now();
    s->cv_done.notify_all();
    return FG21_OK;
}

int fg21_serve_stats(fg21_server *s, fg21_stats *out) {
    if (!s || !out) return set_error(FG21_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    std::vector<double> v = s->lat_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto q = [&v](double f) { return v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.5);
        out->p99_ms = q(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
    }
    const double el = std::chrono::duration<double>(Clock::now() - s->t_create).count();
    out->evals_per_s = el > 0 ? s->points_done / el : 0;
    out->macs_per_s = el > 0 ? s->macs_done / el : 0;
    out->requests_done = s->requests_done;
    out->points_done = s->points_done;
    out->launches = s->launches;
    out->queue_depth = (int64_t)s->pending.size();
    out->admitted_bytes = s->admitted_bytes;
    for (auto &kv : s->runs) {
        if (kv.second.admitted) out->runs_admitted++;
        else out->runs_waiting++;
    }
    return FG21_OK;
}

}  // extern "C"
