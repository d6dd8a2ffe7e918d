// server.cu -- the request server of fdf.h: continuous batching of independent
// runs on one GPU.
//
// Once the metric is known every neutrino is independent (Sec. 2.1), and so is
// every run.  The server exploits that to keep the GPU busy with requests of
// uneven sizes: each admitted request gets its own context (carved from one
// arena allocated up front, so admission and release never call cudaMalloc or
// cudaFree, which would synchronise the device) and its own streams; a worker
// thread feeds every running request slices of leapfrog steps, at most two in
// flight, so kernels of different requests overlap on the device and a request
// that arrives while others run starts as soon as a slot and memory are free.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fdf_internal.cuh"

namespace fdf {
namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kArenaAlign = 2u << 20;   // ranges start on 2 MiB boundaries
constexpr int kMaxInFlight = 2;            // step slices enqueued ahead per request
constexpr int kFlagSlots = 4096;           // requests held at once (pinned flag words)
constexpr int kRing = 4;                   // merged pass launches in flight

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator of [0, size) with coalescing of freed ranges.
class Ranges {
public:
    void init(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    bool take(size_t bytes, size_t* off)
    {
        bytes = round_up(bytes ? bytes : 1, kArenaAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void give(size_t off, size_t bytes)
    {
        bytes = round_up(bytes ? bytes : 1, kArenaAlign);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Request {
    int64_t id = 0;
    fdf_params p{};
    std::vector<double> lnk, lna, T_psi, T_phi, dT, cdf_t, cdf_F;
    fdf_tables t{};
    size_t footprint = 0, off = 0;
    int status = FDF_REQ_QUEUED;
    int error = 0;
    std::string message;
    double t_submit = 0, t_admit = 0;
    std::atomic<double> t_done{0.0};
    // worker-owned from admission on
    bool started = false, finishing = false;
    int rank = 0;                // priority rank: 0 = the oldest running request (highest)
    fdf_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int issued = 0;
    std::deque<cudaEvent_t> inflight;
    cudaEvent_t done_ev = nullptr;
    cudaEvent_t pass_ev = nullptr;   // merged passes: the request's stream is ready for its pass
    bool merged = false;             // its passes go into the server's merged launches
    int slot = -1;
    int* hflag = nullptr;        // pinned copy of the sampling error flag (a slot of the server's pool)
    Clock::time_point origin;
};

}  // namespace
}  // namespace fdf

struct fdf_server {
    int device = 0;
    char* arena = nullptr;
    size_t budget = 0;
    int max_active = 1, slice = 1;
    fdf::Ranges ranges;
    fdf::Clock::time_point t0;
    std::mutex mu;
    std::condition_variable wake;      // the worker: new submissions, releases, stop
    std::condition_variable finished;  // clients: a request finished
    std::deque<fdf::Request*> queue;
    std::vector<fdf::Request*> running;
    std::deque<int64_t> done_ids;
    std::map<int64_t, std::unique_ptr<fdf::Request>> all;
    int64_t next_id = 1;
    int* flags = nullptr;              // pinned words, one per held request
    std::vector<int> free_slots;
    bool stop = false;
    std::thread worker;
    // merged passes (FDF_SERVER_MERGE_PASSES): one launch steps one pass of every running
    // request of the FP64-state form (per grid precision), from a ring of argument slots
    bool merge = false;
    cudaStream_t ms = nullptr;
    struct Slot {
        fdf::PushArgs* host = nullptr;   // pinned, kMaxMerge entries
        fdf::PushArgs* dev = nullptr;    // device, kMaxMerge entries
        cudaEvent_t done = nullptr;
        bool used = false;
    } ring[fdf::kRing];
    int next_slot = 0;
    int sm_count = 152;
    int64_t merged_launches = 0;

    double now() const { return std::chrono::duration<double>(fdf::Clock::now() - t0).count(); }
};

namespace fdf {
namespace {

void CUDART_CB stamp_done(void* arg)
{
    Request* r = static_cast<Request*>(arg);
    r->t_done.store(std::chrono::duration<double>(Clock::now() - r->origin).count());
}

void fail_request(fdf_server* S, Request* r, int code, const std::string& msg)
{
    std::lock_guard<std::mutex> lk(S->mu);
    r->status = FDF_REQ_FAILED;
    r->error = code;
    r->message = msg;
    r->t_done.store(S->now());
    S->done_ids.push_back(r->id);
    S->finished.notify_all();
}

// Wait for the work the request already enqueued (finite kernels, no device-side
// waits) and free its CUDA objects; its arena range and flag slot stay with it.
void teardown(Request* r)
{
    if (r->stream) cudaStreamSynchronize(r->stream);
    for (cudaEvent_t e : r->inflight) cudaEventDestroy(e);
    r->inflight.clear();
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    r->done_ev = nullptr;
    if (r->pass_ev) cudaEventDestroy(r->pass_ev);
    r->pass_ev = nullptr;
    if (r->ctx) fdf_destroy(r->ctx);
    r->ctx = nullptr;
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
}

// One scheduling move for a running request; returns true if it did something.
bool advance(fdf_server* S, Request* r)
{
    if (!r->started) {
        r->started = true;
        // Older requests get higher stream priorities, so the block scheduler serves
        // them first and younger ones fill the gaps: close to first-come-first-served
        // completion, with the overlap kept.  The level is fixed at admission.
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        const int levels = least - greatest + 1;
        const int prio = greatest + std::min(r->rank, levels - 1);
        cudaError_t e = cudaStreamCreateWithPriority(&r->stream, cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->pass_ev, cudaEventDisableTiming);
        r->merged = S->merge && form_of(r->p.precision) == kWide;
        if (e != cudaSuccess) {
            fail_request(S, r, FDF_ECUDA, std::string("server: ") + cudaGetErrorString(e));
            return true;
        }
        *r->hflag = 0;
        int rc = fdf_create(&r->p, &r->t, r->stream, S->arena + r->off, r->footprint, &r->ctx);
        if (!rc) rc = sample_enqueue(r->ctx);
        if (rc) fail_request(S, r, rc, fdf_last_error());
        return true;
    }
    bool did = false;
    while (!r->inflight.empty()) {
        const cudaError_t q = cudaEventQuery(r->inflight.front());
        if (q == cudaErrorNotReady) break;
        cudaEventDestroy(r->inflight.front());
        r->inflight.pop_front();
        if (q != cudaSuccess) {
            fail_request(S, r, FDF_ECUDA, std::string("server: ") + cudaGetErrorString(q));
            return true;
        }
        did = true;
    }
    if (!r->finishing) {
        if (r->merged) {
            // the worker's merged launches issue the passes of the slice begun here
            if (slice_active(r->ctx)) return did;
            if (r->issued < r->p.n_steps) {
                const int n = std::min(S->slice, r->p.n_steps - r->issued);
                int rc = slice_begin(r->ctx, n);
                if (rc) {
                    fail_request(S, r, rc, fdf_last_error());
                    return true;
                }
                r->issued += n;
                return true;
            }
        }
        if (!r->merged && r->issued < r->p.n_steps && (int)r->inflight.size() < kMaxInFlight) {
            const int n = std::min(S->slice, r->p.n_steps - r->issued);
            int rc = fdf_step(r->ctx, n);
            cudaEvent_t ev = nullptr;
            if (!rc && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventRecord(ev, r->stream) == cudaSuccess) {
                r->inflight.push_back(ev);
            } else if (!rc) {
                if (ev) cudaEventDestroy(ev);
                fail_request(S, r, FDF_ECUDA, "server: recording a slice event failed");
                return true;
            }
            if (rc) {
                fail_request(S, r, rc, fdf_last_error());
                return true;
            }
            r->issued += n;
            return true;
        }
        if (r->issued == r->p.n_steps) {
            // the deposit of every species, the sampling flag, the completion time
            // and the completion event, in stream order after the last slice
            int rc = deposit_enqueue(r->ctx, -1, FDF_Q_W_EPS, -1, ctx_deposit_grid(r->ctx));
            cudaError_t e = cudaSuccess;
            if (!rc) e = cudaMemcpyAsync(r->hflag, ctx_error_flag(r->ctx), sizeof(int), cudaMemcpyDeviceToHost,
                                         r->stream);
            if (!rc && e == cudaSuccess) e = cudaLaunchHostFunc(r->stream, stamp_done, r);
            if (!rc && e == cudaSuccess) e = cudaEventRecord(r->done_ev, r->stream);
            if (rc) fail_request(S, r, rc, fdf_last_error());
            else if (e != cudaSuccess) fail_request(S, r, FDF_ECUDA, std::string("server: ") + cudaGetErrorString(e));
            else r->finishing = true;
            return true;
        }
        return did;
    }
    const cudaError_t q = cudaEventQuery(r->done_ev);
    if (q == cudaErrorNotReady) return did;
    if (q != cudaSuccess) {
        fail_request(S, r, FDF_ECUDA, std::string("server: ") + cudaGetErrorString(q));
        return true;
    }
    for (cudaEvent_t ev : r->inflight) cudaEventDestroy(ev);
    r->inflight.clear();
    if (*r->hflag) {
        fail_request(S, r, FDF_EINVAL, "a direction could not be drawn in 64 attempts");
        return true;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    r->status = FDF_REQ_DONE;
    S->done_ids.push_back(r->id);
    S->finished.notify_all();
    return true;
}

// One merged launch: the next pass of each request of `group` (all of the FP64-state form
// with one grid precision, at most kMaxMerge), in one kernel on the server's stream.
// Each request's stream is ordered before it (its previous pass, re-sorts and field
// builds) and after it (the grids' release, the next re-sort).
void merged_tick(fdf_server* S, const std::vector<Request*>& group, int gprec)
{
    auto& slot = S->ring[S->next_slot];
    S->next_slot = (S->next_slot + 1) % kRing;
    if (slot.used) cudaEventSynchronize(slot.done);   // its pinned arguments are free again
    slot.used = true;
    MultiPass m{};
    std::vector<Request*> in;
    for (Request* r : group) {
        const int k = (int)in.size();
        int rc = slice_next(r->ctx, slot.host[k]);
        cudaError_t e = cudaSuccess;
        if (!rc) e = cudaEventRecord(r->pass_ev, r->stream);
        if (!rc && e == cudaSuccess) e = cudaStreamWaitEvent(S->ms, r->pass_ev, 0);
        if (rc || e != cudaSuccess) {
            fail_request(S, r, rc ? rc : FDF_ECUDA, rc ? fdf_last_error() : cudaGetErrorString(e));
            continue;
        }
        const ParticleState& st = ctx_state(r->ctx);
        m.seg[k] = MultiPass::Seg{m.total, slot.dev + k, st.xd, st.qd, st.q0f};
        m.total += slot.host[k].n;
        in.push_back(r);
    }
    m.nseg = (int)in.size();
    cudaError_t e = cudaSuccess;
    if (m.nseg) {
        e = cudaMemcpyAsync(slot.dev, slot.host, m.nseg * sizeof(PushArgs), cudaMemcpyHostToDevice, S->ms);
        if (e == cudaSuccess) e = launch_push_multi(S->ms, gprec, m, S->sm_count * 3);
        ++S->merged_launches;
    }
    cudaEventRecord(slot.done, S->ms);
    for (Request* r : in) {
        int rc = FDF_OK;
        cudaError_t w = e;
        if (w == cudaSuccess) w = cudaStreamWaitEvent(r->stream, slot.done, 0);
        if (w == cudaSuccess) rc = slice_done(r->ctx);
        if (w != cudaSuccess) fail_request(S, r, FDF_ECUDA, std::string("server: ") + cudaGetErrorString(w));
        else if (rc) fail_request(S, r, rc, fdf_last_error());
    }
}

// The merged launches of one round: every running request with a pass to issue, by grid
// precision, in groups of at most kMaxMerge.
bool merged_round(fdf_server* S, const std::vector<Request*>& run)
{
    bool did = false;
    for (int gprec : {FDF_PREC_F32, FDF_PREC_BF16}) {
        std::vector<Request*> group;
        for (Request* r : run)
            if (r->merged && r->ctx && r->status == FDF_REQ_RUNNING && !r->finishing && slice_active(r->ctx) &&
                grid_prec(r->p.precision) == gprec)
                group.push_back(r);
        for (size_t b = 0; b < group.size(); b += kMaxMerge) {
            std::vector<Request*> part(group.begin() + b, group.begin() + std::min(group.size(), b + kMaxMerge));
            merged_tick(S, part, gprec);
            did = true;
        }
    }
    return did;
}

void worker_loop(fdf_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->stop) break;
        // admission: first come, first served, while a slot and a free range exist
        while (!S->queue.empty() && (int)S->running.size() < S->max_active) {
            Request* r = S->queue.front();
            size_t off = 0;
            if (!S->ranges.take(r->footprint, &off)) break;
            S->queue.pop_front();
            r->off = off;
            // one level below the youngest running request (levels are fixed per stream)
            r->rank = 0;
            for (const Request* o : S->running) r->rank = std::max(r->rank, o->rank + 1);
            r->status = FDF_REQ_RUNNING;
            r->t_admit = S->now();
            S->running.push_back(r);
        }
        std::vector<Request*> run = S->running;
        lk.unlock();
        bool did = false;
        for (Request* r : run) did |= advance(S, r);
        if (S->merge) did |= merged_round(S, run);
        lk.lock();
        // finished requests leave the running set (they keep their memory until released)
        S->running.erase(std::remove_if(S->running.begin(), S->running.end(),
                                        [](Request* r) { return r->status != FDF_REQ_RUNNING; }),
                         S->running.end());
        if (!did) S->wake.wait_for(lk, std::chrono::microseconds(200));
    }
    std::vector<Request*> run = S->running;
    lk.unlock();
    for (Request* r : run) teardown(r);
}

Request* find(fdf_server* S, int64_t id)
{
    auto it = S->all.find(id);
    return it == S->all.end() ? nullptr : it->second.get();
}

}  // namespace
}  // namespace fdf

using namespace fdf;

extern "C" {

int fdf_server_create(size_t hbm_budget, int32_t max_active, int32_t slice_steps, fdf_server** out)
{
    return fdf_server_create_opts(hbm_budget, max_active, slice_steps, 0, out);
}

int fdf_server_create_opts(size_t hbm_budget, int32_t max_active, int32_t slice_steps, int32_t options,
                           fdf_server** out)
{
    if (!out) return set_error(FDF_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_active < 1 || slice_steps < 1 || hbm_budget < kArenaAlign)
        return set_error(FDF_EINVAL, "need max_active >= 1, slice_steps >= 1 and a budget of at least 2 MiB");
    if (options & ~FDF_SERVER_MERGE_PASSES) return set_error(FDF_EINVAL, "unknown server options");
    auto S = std::make_unique<fdf_server>();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) return set_error(FDF_ECUDA, cudaGetErrorString(e));
    S->budget = hbm_budget / kArenaAlign * kArenaAlign;
    e = cudaMalloc((void**)&S->arena, S->budget);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(FDF_ENOMEM, (std::string("server arena: ") + cudaGetErrorString(e)).c_str());
    }
    e = cudaHostAlloc((void**)&S->flags, kFlagSlots * sizeof(int), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaFree(S->arena);
        return set_error(FDF_ENOMEM, (std::string("server flags: ") + cudaGetErrorString(e)).c_str());
    }
    for (int i = kFlagSlots - 1; i >= 0; --i) S->free_slots.push_back(i);
    S->merge = (options & FDF_SERVER_MERGE_PASSES) != 0;
    if (S->merge) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device) == cudaSuccess && sms > 0)
            S->sm_count = sms;
        e = cudaStreamCreateWithFlags(&S->ms, cudaStreamNonBlocking);
        for (int i = 0; i < kRing && e == cudaSuccess; ++i) {
            e = cudaHostAlloc((void**)&S->ring[i].host, kMaxMerge * sizeof(PushArgs), cudaHostAllocDefault);
            if (e == cudaSuccess) e = cudaMalloc((void**)&S->ring[i].dev, kMaxMerge * sizeof(PushArgs));
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ring[i].done, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            for (auto& sl : S->ring) {
                if (sl.host) cudaFreeHost(sl.host);
                if (sl.dev) cudaFree(sl.dev);
                if (sl.done) cudaEventDestroy(sl.done);
            }
            if (S->ms) cudaStreamDestroy(S->ms);
            cudaFree(S->arena);
            cudaFreeHost(S->flags);
            return set_error(FDF_ENOMEM, (std::string("server merged passes: ") + cudaGetErrorString(e)).c_str());
        }
    }
    S->ranges.init(S->budget);
    S->max_active = max_active;
    S->slice = slice_steps;
    S->t0 = Clock::now();
    fdf_server* raw = S.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return FDF_OK;
}

int fdf_server_submit(fdf_server* S, const fdf_params* p, const fdf_tables* t, int64_t* id)
{
    if (!S || !p || !t || !id) return set_error(FDF_EINVAL, "NULL argument");
    size_t fp = 0;
    int rc = fdf_footprint(p, &fp);
    if (rc) return rc;
    if (round_up(fp, kArenaAlign) > S->budget)
        return set_error(FDF_ENOMEM, "the request's footprint exceeds the server's whole budget");
    if (!t->lnk || !t->lna || !t->T_psi || !t->T_phi || !t->dTphi_dlna || !t->cdf_t || !t->cdf_F || t->nk < 2 ||
        t->na < 2 || t->ncdf < 2)
        return set_error(FDF_EINVAL, "incomplete tables");
    auto r = std::make_unique<Request>();
    r->p = *p;
    const size_t nt = (size_t)t->nk * t->na;
    r->lnk.assign(t->lnk, t->lnk + t->nk);
    r->lna.assign(t->lna, t->lna + t->na);
    r->T_psi.assign(t->T_psi, t->T_psi + nt);
    r->T_phi.assign(t->T_phi, t->T_phi + nt);
    r->dT.assign(t->dTphi_dlna, t->dTphi_dlna + nt);
    r->cdf_t.assign(t->cdf_t, t->cdf_t + t->ncdf);
    r->cdf_F.assign(t->cdf_F, t->cdf_F + t->ncdf);
    r->t = fdf_tables{t->nk, t->na, r->lnk.data(), r->lna.data(), r->T_psi.data(), r->T_phi.data(), r->dT.data(),
                      t->ncdf, r->cdf_t.data(), r->cdf_F.data()};
    r->footprint = fp;
    r->origin = S->t0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->free_slots.empty()) return set_error(FDF_ENOMEM, "too many requests held (4096)");
        r->slot = S->free_slots.back();
        S->free_slots.pop_back();
        r->hflag = S->flags + r->slot;
        r->id = S->next_id++;
        r->t_submit = S->now();
        *id = r->id;
        S->queue.push_back(r.get());
        S->all[r->id] = std::move(r);
    }
    S->wake.notify_all();
    return FDF_OK;
}

int fdf_server_wait(fdf_server* S, int32_t timeout_ms, int64_t* id)
{
    if (!S || !id) return set_error(FDF_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return !S->done_ids.empty(); };
    if (timeout_ms < 0) S->finished.wait(lk, ready);
    else if (!S->finished.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return set_error(FDF_ETIMEOUT, "no request finished in time");
    *id = S->done_ids.front();
    S->done_ids.pop_front();
    return FDF_OK;
}

int fdf_server_info(fdf_server* S, int64_t id, fdf_request_info* info)
{
    if (!S || !info) return set_error(FDF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    Request* r = find(S, id);
    if (!r) return set_error(FDF_EINVAL, "unknown request id");
    std::memset(info, 0, sizeof(*info));
    info->id = r->id;
    info->status = r->status;
    info->error = r->error;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_done = r->status == FDF_REQ_DONE || r->status == FDF_REQ_FAILED ? r->t_done.load() : 0.0;
    info->footprint = r->footprint;
    info->particle_steps = (int64_t)r->p.n_species * r->p.n_part * r->p.n_steps;
    std::strncpy(info->message, r->message.c_str(), sizeof(info->message) - 1);
    return FDF_OK;
}

static Request* done_request(fdf_server* S, int64_t id, int* rc)
{
    std::lock_guard<std::mutex> lk(S->mu);
    Request* r = find(S, id);
    if (!r) *rc = set_error(FDF_EINVAL, "unknown request id");
    else if (r->status != FDF_REQ_DONE) *rc = set_error(FDF_ESTATE, "the request is not done");
    else *rc = FDF_OK;
    return *rc ? nullptr : r;
}

int fdf_server_get(fdf_server* S, int64_t id, int32_t species, double* x, double* q, double* w, int32_t on_device)
{
    if (!S) return set_error(FDF_EINVAL, "NULL server");
    int rc = 0;
    Request* r = done_request(S, id, &rc);
    if (!r) return rc;
    return fdf_get(r->ctx, species, x, q, w, on_device);
}

int fdf_server_deposit(fdf_server* S, int64_t id, double* out, int32_t on_device)
{
    if (!S || !out) return set_error(FDF_EINVAL, "NULL argument");
    int rc = 0;
    Request* r = done_request(S, id, &rc);
    if (!r) return rc;
    const size_t N = (size_t)r->p.n_grid;
    cudaError_t e = cudaMemcpyAsync(out, ctx_deposit_grid(r->ctx), N * N * N * 8,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return set_error(FDF_ECUDA, cudaGetErrorString(e));
    return FDF_OK;
}

int fdf_server_release(fdf_server* S, int64_t id)
{
    if (!S) return set_error(FDF_EINVAL, "NULL server");
    std::unique_ptr<Request> owned;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(id);
        if (it == S->all.end()) return set_error(FDF_EINVAL, "unknown request id");
        Request* r = it->second.get();
        if (r->status != FDF_REQ_DONE && r->status != FDF_REQ_FAILED)
            return set_error(FDF_ESTATE, "the request is still queued or running");
        owned = std::move(it->second);
        S->all.erase(it);
        S->done_ids.erase(std::remove(S->done_ids.begin(), S->done_ids.end(), id), S->done_ids.end());
    }
    // the worker no longer touches a finished request: free its CUDA objects, then
    // hand its range back so that a waiting request can be admitted
    const bool placed = owned->started;
    teardown(owned.get());
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (placed) S->ranges.give(owned->off, owned->footprint);
        S->free_slots.push_back(owned->slot);
    }
    S->wake.notify_all();
    return FDF_OK;
}

double fdf_server_clock(const fdf_server* S) { return S ? S->now() : 0.0; }

int fdf_server_merged_launches(const fdf_server* S, int64_t* launches)
{
    if (!S || !launches) return set_error(FDF_EINVAL, "NULL argument");
    *launches = S->merged_launches;
    return FDF_OK;
}

int fdf_server_load(fdf_server* S, int32_t* queued, int32_t* running, size_t* bytes_in_use)
{
    if (!S) return set_error(FDF_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int32_t)S->queue.size();
    if (running) *running = (int32_t)S->running.size();
    if (bytes_in_use) *bytes_in_use = S->ranges.used();
    return FDF_OK;
}

void fdf_server_destroy(fdf_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->wake.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->all) teardown(kv.second.get());
    S->all.clear();
    if (S->ms) cudaStreamSynchronize(S->ms);
    for (auto& sl : S->ring) {
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (S->ms) cudaStreamDestroy(S->ms);
    if (S->arena) cudaFree(S->arena);
    if (S->flags) cudaFreeHost(S->flags);
    delete S;
}

}  // extern "C"
