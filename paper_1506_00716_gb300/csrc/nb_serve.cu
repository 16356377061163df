// nb_serve.cu -- continuous-batching server (nb_server_*).
//
// One scheduler thread owns all CUDA work of a server.  It keeps up to two
// waves in flight, one per stream.  When a stream is free it admits the
// oldest pending requests whose estimated device footprint fits the budget
// (FIFO, at most max_wave) and launches them as one wave: systems are
// created, their inputs uploaded, and grid put, search, prune, forces,
// energies and the unsort run as one launch per stage over every system of
// the wave (the batch-aware kernels index systems by descriptor).  Results
// are copied to pinned host staging on the wave's stream and an event marks
// the end; when the event has completed the scheduler hands the results to
// the requests, frees the wave's device memory and wakes the waiters.  While
// one wave's force kernel runs, the next wave's upload, grid and search run
// on the other stream.
#include <algorithm>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nb_host.h"

using namespace nbgb;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    unsigned long long id = 0;
    int natoms = 0;
    double box[3] = {0, 0, 0};
    unsigned flags = 0;
    // inputs, copied at submission into one pinned block (the uploads are
    // then plain DMA): x y z q, types, and the symmetric exclusion CSR
    void* pin = nullptr;
    size_t pin_class = 0;
    const float* xq = nullptr;
    const int* type = nullptr;
    const int* ei = nullptr;
    const int* ea = nullptr;
    bool has_excl = false;
    size_t est_bytes = 0;
    // results
    std::vector<float> f;
    double energy[2] = {0, 0};
    double virial[9] = {0};
    long long npairs = 0;
    int wave_size = 0;
    nb_status status = NB_OK;
    std::string err;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;
    // a thread is inside nb_server_wait for this request (set and cleared
    // under the server's mutex); a second waiter is refused
    bool claimed = false;
};

// Growable pinned host buffer.
struct Pinned {
    void* p = nullptr;
    size_t bytes = 0;
    bool reserve(size_t n) {
        if (n <= bytes) return true;
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        size_t want = std::max(n, (size_t)1 << 20);
        if (cudaMallocHost(&p, want) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        bytes = want;
        return true;
    }
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
};

struct Wave {
    std::vector<Request*> reqs;
    std::vector<nb_sys*> systems;
    std::vector<size_t> f_off;
    Plan* plan = nullptr;
    size_t bytes = 0;
    unsigned flags = 0;
    int attempts = 0;
    double boost = 1.0;  // list capacity relative to the estimate
    bool busy = false;
};

// Pinned host blocks in power-of-two size classes, reused across requests so
// that steady-state serving allocates no pinned memory.
struct PinnedPool {
    std::mutex mu;
    std::unordered_map<size_t, std::vector<void*>> free_blocks;
    std::vector<void*> all;
    void* get(size_t bytes, size_t* cls) {
        size_t c = (size_t)1 << 16;
        while (c < bytes) c <<= 1;
        *cls = c;
        {
            std::lock_guard<std::mutex> lock(mu);
            auto& v = free_blocks[c];
            if (!v.empty()) {
                void* p = v.back();
                v.pop_back();
                return p;
            }
        }
        void* p = nullptr;
        if (cudaHostAlloc(&p, c, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        std::lock_guard<std::mutex> lock(mu);
        all.push_back(p);
        return p;
    }
    void put(void* p, size_t cls) {
        if (!p) return;
        std::lock_guard<std::mutex> lock(mu);
        free_blocks[cls].push_back(p);
    }
    ~PinnedPool() {
        for (void* p : all) cudaFreeHost(p);
    }
};

}  // namespace

struct nb_server {
    int device = 0;
    nb_ctx* ctxs[2] = {nullptr, nullptr};
    cudaStream_t streams[2] = {nullptr, nullptr};
    cudaEvent_t events[2] = {nullptr, nullptr};
    Pinned f_stage[2], res_stage[2], cnt_stage[2];
    Wave waves[2];
    nb_params p{};
    std::vector<float> c6, c12;
    nb_tuning tuning{32, 3, 0, 0};
    size_t budget = 0;
    int max_wave = 64;
    size_t in_use = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<unsigned long long, Request*> reqs;
    PinnedPool pinned;
    bool stop = false;
    unsigned long long next_id = 1;
    std::thread thread;
};

namespace {

// Called once the device no longer reads the request's pinned inputs.
void finish(nb_server* s, Request* r, nb_status st, const std::string& msg) {
    s->pinned.put(r->pin, r->pin_class);
    r->pin = nullptr;
    r->status = st;
    r->err = msg;
    r->t_done = Clock::now();
    r->done = true;
}

nb_status run_wave(nb_server* s, int k, double boost);

// Launch one wave on stream slot k (scheduler thread, lock not held).
void launch_wave(nb_server* s, int k, std::vector<Request*> reqs) {
    Wave& w = s->waves[k];
    w = Wave();
    nb_ctx* ctx = s->ctxs[k];
    auto fail_all = [&](nb_status code, const std::string& msg) {
        // uploads already enqueued still read the requests' pinned inputs
        cudaStreamSynchronize(s->streams[k]);
        for (nb_sys* y : w.systems) nb_sys_destroy(y);
        w.systems.clear();
        std::lock_guard<std::mutex> lock(s->mu);
        for (Request* r : reqs) finish(s, r, code, msg);
        s->in_use -= std::min(s->in_use, w.bytes);
        s->cv_done.notify_all();
    };
    size_t bytes = 0;
    unsigned flags = 0;
    for (Request* r : reqs) {
        bytes += r->est_bytes;
        flags |= r->flags;
    }
    w.bytes = bytes;
    w.flags = flags;
    for (Request* r : reqs) {
        nb_sys* y = nullptr;
        nb_status stt = nb_sys_create(ctx, &s->p, r->natoms, r->box, &y);
        if (stt == NB_OK && r->has_excl) stt = sys_upload_exclusions(y, r->ei, r->ea);
        if (stt == NB_OK) stt = stage_coords(y, r->xq, r->type);
        if (stt != NB_OK) {
            if (y) nb_sys_destroy(y);
            fail_all(stt, nb_last_error());
            return;
        }
        w.systems.push_back(y);
    }
    size_t tot_f = 0;
    for (Request* r : reqs) {
        w.f_off.push_back(tot_f);
        tot_f += (size_t)r->natoms * 3;
    }
    if (!s->f_stage[k].reserve(4 * tot_f) || !s->res_stage[k].reserve(8 * NRES * reqs.size()) ||
        !s->cnt_stage[k].reserve(4 * CNT_N)) {
        fail_all(NB_ERR_OOM, "pinned staging allocation failed");
        return;
    }
    w.reqs = std::move(reqs);
    nb_status stt = run_wave(s, k, 1.0);
    if (stt != NB_OK) {
        reqs = std::move(w.reqs);
        fail_all(stt, nb_last_error());
    }
}

// Create the wave's plan (list capacity = estimate x boost) and enqueue the
// whole path plus the result copies on the wave's stream.  The systems'
// inputs are already on the device, so a retry after a list overflow runs
// the same sequence again with a larger list.
nb_status run_wave(nb_server* s, int k, double boost) {
    Wave& w = s->waves[k];
    nb_ctx* ctx = s->ctxs[k];
    cudaStream_t st = s->streams[k];
    const unsigned flags = w.flags;
    nb_status stt = plan_create(ctx, w.systems.data(), (int)w.systems.size(), &w.plan, boost);
    if (stt != NB_OK) {
        w.plan = nullptr;
        return stt;
    }
    ++w.attempts;
    w.boost = boost;
    plan_set_geometry(w.plan);
    PlanLaunch pl = launch_of(w.plan);
    cudaError_t e = cudaMemsetAsync(w.plan->list.counters, 0, 4 * CNT_N, st);
    if (e == cudaSuccess) e = launch_grid_put(pl, st);
    if (e == cudaSuccess) e = launch_search(pl, st);
    if (e == cudaSuccess) e = launch_prune(pl, st);
    if (e == cudaSuccess) e = launch_prepare(pl, false, st);
    if (e == cudaSuccess) e = launch_forces(pl, flags, st);
    if (e == cudaSuccess && (flags & NB_F_ENERGY)) e = launch_energy(pl, st);
    if (e == cudaSuccess) e = launch_excl_corr(pl, flags, st);
    if (e == cudaSuccess) e = launch_finalize(pl, flags, st);
    float* hf = (float*)s->f_stage[k].p;
    double* hres = (double*)s->res_stage[k].p;
    for (size_t q = 0; q < w.reqs.size() && e == cudaSuccess; ++q) {
        nb_sys* y = w.systems[q];
        e = cudaMemcpyAsync(hf + w.f_off[q], y->h.f_out, 12 * (size_t)y->natoms, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hres + NRES * q, y->h.res, 8 * NRES, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->cnt_stage[k].p, w.plan->list.counters, 4 * CNT_N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->events[k], st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        plan_destroy(w.plan);
        w.plan = nullptr;
        return cuda_fail(e, "serving wave launch");
    }
    w.busy = true;
    return NB_OK;
}

// Hand a completed wave's results to its requests and free its memory.
void retire_wave(nb_server* s, int k) {
    Wave& w = s->waves[k];
    const int* cnt = (const int*)s->cnt_stage[k].p;
    const bool overflow = (cnt[CNT_OVERFLOW] & 3) != 0;
    if (overflow && w.attempts < 3) {
        // The list outgrew its estimate: the counters hold the sizes the
        // search wanted, so run the wave again with room for them.
        const double need = std::max((double)cnt[CNT_ITEMS] / std::max<long long>(1, w.plan->item_cap),
                                     (double)entries_needed(cnt, w.plan->tot_clcap) /
                                         std::max<long long>(1, w.plan->entry_cap));
        const double boost = w.boost * 1.25 * std::max(1.0, need) * (w.attempts == 1 ? 1.0 : 2.0);
        plan_destroy(w.plan);
        w.plan = nullptr;
        w.busy = false;
        if (run_wave(s, k, boost) == NB_OK) return;
    }
    const float* hf = (const float*)s->f_stage[k].p;
    const double* hres = (const double*)s->res_stage[k].p;
    for (size_t q = 0; q < w.reqs.size(); ++q) {
        Request* r = w.reqs[q];
        if (!overflow) {
            r->f.assign(hf + w.f_off[q], hf + w.f_off[q] + (size_t)r->natoms * 3);
            r->energy[0] = hres[NRES * q + 0];
            r->energy[1] = hres[NRES * q + 1];
            for (int c = 0; c < 9; ++c) r->virial[c] = hres[NRES * q + 2 + c];
            r->npairs = (long long)hres[NRES * q + 11];
        }
        r->wave_size = (int)w.reqs.size();
    }
    plan_destroy(w.plan);
    w.plan = nullptr;
    for (nb_sys* y : w.systems) nb_sys_destroy(y);
    w.systems.clear();
    std::lock_guard<std::mutex> lock(s->mu);
    for (Request* r : w.reqs) {
        if (overflow)
            finish(s, r, NB_ERR_CAPACITY, "the wave's pair list outgrew its estimate");
        else
            finish(s, r, NB_OK, "");
    }
    s->in_use -= std::min(s->in_use, w.bytes);
    w.reqs.clear();
    w.busy = false;
    s->cv_done.notify_all();
}

void scheduler(nb_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool did = false;
        for (int k = 0; k < 2; ++k) {
            if (s->waves[k].busy && cudaEventQuery(s->events[k]) == cudaSuccess) {
                retire_wave(s, k);
                did = true;
            }
        }
        for (int k = 0; k < 2; ++k) {
            if (s->waves[k].busy) continue;
            std::vector<Request*> take;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                while (!s->pending.empty() && (int)take.size() < s->max_wave) {
                    Request* r = s->pending.front();
                    if (s->budget && r->est_bytes > s->budget) {
                        s->pending.pop_front();
                        finish(s, r, NB_ERR_BUDGET, "request larger than the server's HBM budget");
                        s->cv_done.notify_all();
                        continue;
                    }
                    if (s->budget && s->in_use + r->est_bytes > s->budget) break;
                    s->pending.pop_front();
                    s->in_use += r->est_bytes;
                    r->t_admit = Clock::now();
                    take.push_back(r);
                }
            }
            if (!take.empty()) {
                launch_wave(s, k, std::move(take));
                did = true;
            }
        }
        if (did) continue;
        std::unique_lock<std::mutex> lock(s->mu);
        const bool busy = s->waves[0].busy || s->waves[1].busy;
        if (s->stop && s->pending.empty() && !busy) break;
        if (busy)
            s->cv_sched.wait_for(lock, std::chrono::microseconds(20));
        else
            s->cv_sched.wait_for(lock, std::chrono::milliseconds(5));
    }
}

}  // namespace

extern "C" {

nb_status nb_server_create(nb_ctx* ctx, const nb_params* params, size_t hbm_budget_bytes, int max_wave,
                           nb_server** out) {
    if (!ctx || !params || !out) return fail(NB_ERR_ARG, "ctx / params / out is NULL");
    if (max_wave < 1 || max_wave > 4096) return fail(NB_ERR_ARG, "max_wave must be in 1..4096");
    *out = nullptr;
    const double probe_box[3] = {1e3, 1e3, 1e3};
    size_t dummy = 0;
    nb_status st = nb_sys_footprint(params, 1, probe_box, &dummy);
    if (st != NB_OK) return st;
    nb_server* s = new nb_server();
    s->device = ctx->device;
    s->p = *params;
    int nt = params->ntypes;
    s->c6.assign(params->c6, params->c6 + nt * nt);
    s->c12.assign(params->c12, params->c12 + nt * nt);
    s->p.c6 = s->c6.data();
    s->p.c12 = s->c12.data();
    s->tuning = ctx->tuning;
    s->budget = hbm_budget_bytes;
    s->max_wave = max_wave;
    cudaError_t e = cudaSetDevice(s->device);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->events[k], cudaEventDisableTiming);
        if (e == cudaSuccess) {
            st = nb_ctx_create(s->device, s->streams[k], 0, &s->ctxs[k]);
            if (st != NB_OK) e = cudaErrorUnknown;
            else nb_ctx_set_tuning(s->ctxs[k], &s->tuning);
        }
    }
    if (e != cudaSuccess) {
        for (int k = 0; k < 2; ++k) {
            if (s->ctxs[k]) nb_ctx_destroy(s->ctxs[k]);
            if (s->events[k]) cudaEventDestroy(s->events[k]);
            if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
        }
        delete s;
        return cuda_fail(e, "nb_server_create");
    }
    s->thread = std::thread(scheduler, s);
    *out = s;
    return NB_OK;
}

nb_status nb_server_destroy(nb_server* s) {
    if (!s) return fail(NB_ERR_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->thread.joinable()) s->thread.join();
    for (int k = 0; k < 2; ++k) {
        if (s->ctxs[k]) nb_ctx_destroy(s->ctxs[k]);
        if (s->events[k]) cudaEventDestroy(s->events[k]);
        if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
    }
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return NB_OK;
}

nb_status nb_server_submit(nb_server* s, int natoms, const double box[3], const float* xq, const int* type,
                           const int* excl_index, const int* excl_atoms, unsigned flags,
                           unsigned long long* ticket) {
    if (!s || !ticket || !xq || !type) return fail(NB_ERR_ARG, "NULL argument");
    if (flags & ~(unsigned)(NB_F_ENERGY | NB_F_VIRIAL)) return fail(NB_ERR_ARG, "unknown flag bits");
    size_t est = 0;
    nb_status st = nb_sys_footprint(&s->p, natoms, box, &est);
    if (st != NB_OK) return st;
    // exclusions validated and symmetrised here, on the caller's thread
    std::vector<int> ei_v, ea_v;
    const int *pei = nullptr, *pea = nullptr;
    size_t n_ei = 0, n_ea = 0;
    if (excl_index) {
        st = excl_symmetrise(natoms, excl_index, excl_atoms, ei_v, ea_v, &pei, &pea);
        if (st != NB_OK) return st;
        n_ei = (size_t)natoms + 1;
        n_ea = (size_t)pei[natoms];
    }
    Request* r = new Request();
    r->natoms = natoms;
    for (int d = 0; d < 3; ++d) r->box[d] = box[d];
    r->flags = flags;
    const size_t n = (size_t)natoms;
    const size_t bytes = 16 * n + 4 * n + 4 * (n_ei + n_ea);
    char* b = (char*)s->pinned.get(bytes, &r->pin_class);
    if (!b) {
        delete r;
        return fail(NB_ERR_OOM, "pinned staging allocation failed");
    }
    r->pin = b;
    std::memcpy(b, xq, 16 * n);
    std::memcpy(b + 16 * n, type, 4 * n);
    r->xq = (const float*)b;
    r->type = (const int*)(b + 16 * n);
    if (excl_index) {
        int* e = (int*)(b + 20 * n);
        std::memcpy(e, pei, 4 * n_ei);
        if (n_ea) std::memcpy(e + n_ei, pea, 4 * n_ea);
        r->ei = e;
        r->ea = e + n_ei;
        r->has_excl = true;
    }
    r->est_bytes = est + 4 * (n_ei + n_ea + 1) + 4096;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            s->pinned.put(r->pin, r->pin_class);
            delete r;
            return fail(NB_ERR_STATE, "server is shutting down");
        }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->pending.push_back(r);
        *ticket = r->id;
    }
    s->cv_sched.notify_one();
    return NB_OK;
}

nb_status nb_server_wait(nb_server* s, unsigned long long ticket, long long timeout_us, float* f,
                         double* energy, double* virial, nb_request_stats* stats) {
    if (!s) return fail(NB_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(NB_ERR_ARG, "unknown or already collected ticket");
    Request* r = it->second;
    if (r->claimed) return fail(NB_ERR_ARG, "another thread is already waiting on this ticket");
    r->claimed = true;
    auto ready = [&] { return r->done; };
    if (timeout_us < 0) {
        s->cv_done.wait(lock, ready);
    } else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready)) {
        r->claimed = false;
        return fail(NB_ERR_TIMEOUT, "request not finished within the timeout");
    }
    // by key: submissions during the wait may have rehashed the map
    s->reqs.erase(ticket);
    lock.unlock();
    nb_status st = r->status;
    if (st == NB_OK) {
        if (f) std::copy(r->f.begin(), r->f.end(), f);
        if (energy) {
            energy[0] = r->energy[0];
            energy[1] = r->energy[1];
        }
        if (virial) std::copy(r->virial, r->virial + 9, virial);
    }
    if (stats) {
        stats->latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
        stats->queue_s = std::chrono::duration<double>(r->t_admit - r->t_submit).count();
        stats->n_pairs = r->npairs;
        stats->wave_size = r->wave_size;
    }
    std::string err = r->err;
    delete r;
    if (st != NB_OK) return fail(st, err);
    return NB_OK;
}

}  // extern "C"
