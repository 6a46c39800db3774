// Fit server: fits of different sizes are submitted as they arrive, admitted
// into device slots by HBM footprint, and advanced together (continuous
// batching): every tick replays one CUDA graph of K passes over all running
// fits [tile map -> constants -> NLL+grad -> state update], then the host
// retires the fits that ended, frees their memory and admits waiting ones.
//
// The paper fits one data set at a time from Python (Sec. 3-4); this is the
// serving form of the same path.  A fit in the server computes exactly what
// ipa_fit_batch computes for it alone: its likelihood segment and its state
// machine do not depend on the other fits, so results are bitwise equal.
//
// Memory: one event arena per column, sized by the HBM budget (40 bytes per
// event: t, cos thK, cos thmu, phi, w); a fit occupies a contiguous range,
// first fit in submission order (no overtaking, so no starvation).  Events are
// copied into host staging at submit, so the caller may free its buffers as
// soon as submit returns; they move to the device when the fit is admitted.
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fitcore.cuh"
#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr int kTickPasses = 4;   // passes per tick (one graph replay)

enum ReqState { kQueued = 0, kRunning = 1, kFinished = 2 };

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0;
    bool weighted = false;
    std::vector<double> cols[5];   // t, ck, cl, phi, w (host staging)
    Spec spec{};
    double theta0[kMaxP] = {};
    double theta[kMaxP] = {}, err[kMaxP] = {}, nll = 0.0;
    int32_t status = IPA_FIT_MAXITER, iters = 0, passes = 0;
    ipa_status error = IPA_OK;
    int state = kQueued;
    int slot = -1;
    int64_t off = 0;
};

__global__ void fill_kernel(double* p, int64_t n, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace
}  // namespace ipa

struct ipa_server {
    ipa_model model{};
    int P = 0, max_slots = 0, max_iter = 200, device = 0;
    double tol = 1e-8;
    int64_t arena_cap = 0;
    cudaStream_t stream = nullptr;
    double* arena[5] = {};
    ipa::Spec* d_specs = nullptr;
    ipa::State* d_states = nullptr;
    double* d_theta_eval = nullptr;
    double* d_res = nullptr;
    int* d_active = nullptr;
    int64_t* d_begin = nullptr;
    int64_t* d_end = nullptr;
    int* d_nact = nullptr;
    double *d_out_theta = nullptr, *d_out_err = nullptr, *d_out_nll = nullptr;
    int32_t *d_out_status = nullptr, *d_out_iters = nullptr, *d_out_passes = nullptr;
    // pinned mirrors
    int64_t *h_begin = nullptr, *h_end = nullptr;
    int* h_active = nullptr;
    double *h_out_theta = nullptr, *h_out_err = nullptr, *h_out_nll = nullptr;
    int32_t *h_out_status = nullptr, *h_out_iters = nullptr, *h_out_passes = nullptr;
    ipa::Scratch sc;               // the server's own likelihood scratch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // host state
    std::vector<ipa::Request*> slot_req;
    std::map<int64_t, int64_t> free_ranges;   // arena offset -> length
    std::deque<ipa::Request*> queue;
    std::unordered_map<uint64_t, ipa::Request*> reqs;
    uint64_t next_ticket = 1;
    int running = 0;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    ipa_status fatal = IPA_OK;
    char fatal_msg[256] = "";
    std::thread worker;
};

namespace ipa {
namespace {

int64_t arena_alloc(ipa_server* s, int64_t n) {
    if (n == 0) return 0;
    for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
        if (it->second >= n) {
            const int64_t off = it->first, len = it->second;
            s->free_ranges.erase(it);
            if (len > n) s->free_ranges[off + n] = len - n;
            return off;
        }
    }
    return -1;
}

void arena_free(ipa_server* s, int64_t off, int64_t n) {
    if (n == 0) return;
    auto next = s->free_ranges.lower_bound(off);
    int64_t o = off, l = n;
    if (next != s->free_ranges.end() && next->first == off + n) {
        l += next->second;
        next = s->free_ranges.erase(next);
    }
    if (next != s->free_ranges.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == o) {
            o = prev->first;
            l += prev->second;
            s->free_ranges.erase(prev);
        }
    }
    s->free_ranges[o] = l;
}

// Event columns kept in the arena besides the weights (arena[4]): t, then
// ck, cl, phi (4D) or the tag q in arena[1] (tagged model).
int arena_cols(int kind) { return kind == IPA_MODEL_ANGTIME4D ? 4 : (kind == IPA_MODEL_TAGGED1D ? 2 : 1); }

// One pass over every slot (inactive slots have no tiles and are skipped).
ipa_status server_pass(ipa_server* s) {
    const ModelDev m{s->model.kind, s->model.n_par, s->model.t_lo, s->model.t_hi};
    ipa_status q;
    if ((q = launch_seg_tiles(s->d_begin, s->d_end, s->d_active, s->max_slots, s->arena_cap, s->sc.seg_tiles,
                              s->stream)) != IPA_OK)
        return q;
    if ((q = launch_consts(m, s->d_theta_eval, s->max_slots, s->sc.consts, s->stream)) != IPA_OK) return q;
    const bool four = s->model.kind == IPA_MODEL_ANGTIME4D;
    const bool tag = s->model.kind == IPA_MODEL_TAGGED1D;
    const Cols cols{s->arena[0], four ? s->arena[1] : nullptr, four ? s->arena[2] : nullptr,
                    four ? s->arena[3] : nullptr, s->arena[4], nullptr, 0, tag ? s->arena[1] : nullptr};
    if ((q = launch_nll(m, true, cols, s->arena_cap, s->d_begin, s->d_end, s->sc.seg_tiles, s->max_slots,
                        s->sc.consts, &s->sc, s->d_res, s->stream)) != IPA_OK)
        return q;
    if ((q = cuda_fail(cudaMemsetAsync(s->d_nact, 0, sizeof(int), s->stream), "server count")) != IPA_OK) return q;
    const int fb = 128, fg = (s->max_slots + fb - 1) / fb;
    qn_kernel<<<fg, fb, 0, s->stream>>>(s->d_specs, 1, s->max_slots, s->d_begin, s->d_end, s->d_res, s->d_states,
                                        s->d_theta_eval, s->d_active, s->d_nact);
    return cuda_fail(cudaGetLastError(), "server step");
}

void worker_fail(ipa_server* s, ipa_status st) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = st;
    snprintf(s->fatal_msg, sizeof(s->fatal_msg), "%s", ipa_last_error());
    for (auto& kv : s->reqs) {
        if (kv.second->state != kFinished) {
            kv.second->state = kFinished;
            kv.second->error = st;
        }
    }
    s->cv.notify_all();
}

void worker_main(ipa_server* s) {
    cudaSetDevice(s->device);
    const int P = s->P;
    while (true) {
        std::vector<Request*> admitted;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop || s->fatal != IPA_OK) break;
            // an injected admission failure (IPA_FAULT_ADMIT) leaves every queued
            // request waiting, in order, for a later tick
            while (!s->queue.empty() && !fault(IPA_FAULT_ADMIT)) {
                Request* r = s->queue.front();
                int slot = -1;
                for (int i = 0; i < s->max_slots; ++i)
                    if (!s->slot_req[i]) {
                        slot = i;
                        break;
                    }
                if (slot < 0) break;
                const int64_t off = arena_alloc(s, r->n);
                if (off < 0) break;                    // wait for memory (first in, first served)
                s->queue.pop_front();
                r->slot = slot;
                r->off = off;
                r->state = kRunning;
                s->slot_req[slot] = r;
                s->running += 1;
                admitted.push_back(r);
            }
            if (admitted.empty() && s->running == 0) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        ipa_status st = IPA_OK;
        // upload admitted fits: events into the arena, spec and start point into the slot
        const int n_cols = arena_cols(s->model.kind);
        for (Request* r : admitted) {
            for (int c = 0; c < n_cols && st == IPA_OK; ++c) {
                if (r->n > 0)
                    st = cuda_fail(cudaMemcpyAsync(s->arena[c] + r->off, r->cols[c].data(), sizeof(double) * r->n,
                                                   cudaMemcpyHostToDevice, s->stream), "server upload");
            }
            if (st == IPA_OK && r->n > 0) {
                if (r->weighted) {
                    st = cuda_fail(cudaMemcpyAsync(s->arena[4] + r->off, r->cols[4].data(), sizeof(double) * r->n,
                                                   cudaMemcpyHostToDevice, s->stream), "server upload");
                } else {
                    fill_kernel<<<64, 256, 0, s->stream>>>(s->arena[4] + r->off, r->n, 1.0);
                    st = cuda_fail(cudaGetLastError(), "server weights");
                }
            }
            if (st == IPA_OK)
                st = cuda_fail(cudaMemcpyAsync(s->d_specs + r->slot, &r->spec, sizeof(Spec), cudaMemcpyHostToDevice,
                                               s->stream), "server spec");
            if (st == IPA_OK)
                st = cuda_fail(cudaMemcpyAsync(s->d_theta_eval + (size_t)r->slot * P, r->theta0, sizeof(double) * P,
                                               cudaMemcpyHostToDevice, s->stream), "server start");
            s->h_begin[r->slot] = r->off;
            s->h_end[r->slot] = r->off + r->n;
        }
        if (st == IPA_OK && !admitted.empty()) {
            st = cuda_fail(cudaMemcpyAsync(s->d_begin, s->h_begin, sizeof(int64_t) * s->max_slots,
                                           cudaMemcpyHostToDevice, s->stream), "server ranges");
            if (st == IPA_OK)
                st = cuda_fail(cudaMemcpyAsync(s->d_end, s->h_end, sizeof(int64_t) * s->max_slots,
                                               cudaMemcpyHostToDevice, s->stream), "server ranges");
            for (Request* r : admitted) {
                if (st != IPA_OK) break;
                init_kernel<<<1, 32, 0, s->stream>>>(s->d_specs + r->slot, 0, 1, s->d_theta_eval + (size_t)r->slot * P,
                                                     s->d_states + r->slot, s->d_theta_eval + (size_t)r->slot * P,
                                                     s->d_active + r->slot);
                st = cuda_fail(cudaGetLastError(), "server init");
            }
        }
        // staging copies must finish before the host buffers are released
        if (st == IPA_OK && !admitted.empty()) st = cuda_fail(cudaStreamSynchronize(s->stream), "server admit");
        for (Request* r : admitted)
            for (auto& c : r->cols) std::vector<double>().swap(c);
        // K passes over all running fits
        if (st == IPA_OK) st = cuda_fail(cudaGraphLaunch(s->exec, s->stream), "server tick");
        if (st == IPA_OK) {
            const int fb = 128, fg = (s->max_slots + fb - 1) / fb;
            final_kernel<<<fg, fb, 0, s->stream>>>(s->d_specs, 1, s->max_slots, s->d_states, s->d_out_theta,
                                                    s->d_out_err, s->d_out_nll, s->d_out_status, s->d_out_iters,
                                                    s->d_out_passes);
            st = cuda_fail(cudaGetLastError(), "server results");
        }
        struct Cp {
            void* h;
            const void* d;
            size_t b;
        };
        const Cp cps[] = {{s->h_active, s->d_active, sizeof(int) * s->max_slots},
                          {s->h_out_theta, s->d_out_theta, sizeof(double) * s->max_slots * P},
                          {s->h_out_err, s->d_out_err, sizeof(double) * s->max_slots * P},
                          {s->h_out_nll, s->d_out_nll, sizeof(double) * s->max_slots},
                          {s->h_out_status, s->d_out_status, sizeof(int32_t) * s->max_slots},
                          {s->h_out_iters, s->d_out_iters, sizeof(int32_t) * s->max_slots},
                          {s->h_out_passes, s->d_out_passes, sizeof(int32_t) * s->max_slots}};
        for (const Cp& c : cps) {
            if (st != IPA_OK) break;
            st = cuda_fail(cudaMemcpyAsync(c.h, c.d, c.b, cudaMemcpyDeviceToHost, s->stream), "server readback");
        }
        if (st == IPA_OK) st = cuda_fail(cudaStreamSynchronize(s->stream), "server tick sync");
        if (st != IPA_OK) {
            worker_fail(s, st);
            break;
        }
        // retire finished fits
        std::lock_guard<std::mutex> lk(s->mu);
        for (int i = 0; i < s->max_slots; ++i) {
            Request* r = s->slot_req[i];
            if (!r || s->h_active[i]) continue;
            for (int p = 0; p < P; ++p) {
                r->theta[p] = s->h_out_theta[(size_t)i * P + p];
                r->err[p] = s->h_out_err[(size_t)i * P + p];
            }
            r->nll = s->h_out_nll[i];
            r->status = s->h_out_status[i];
            r->iters = s->h_out_iters[i];
            r->passes = s->h_out_passes[i];
            r->state = kFinished;
            arena_free(s, r->off, r->n);
            s->slot_req[i] = nullptr;
            s->h_begin[i] = s->h_end[i] = 0;
            s->running -= 1;
        }
        s->cv.notify_all();
    }
}

template <class T>
ipa_status dalloc(T** p, size_t count, const char* what) {
    return device_alloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1), what);
}

template <class T>
ipa_status halloc(T** p, size_t count, const char* what) {
    ipa_status st = cuda_fail(cudaMallocHost(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1)), what);
    if (st == IPA_OK) memset(*p, 0, sizeof(T) * (count ? count : 1));
    return st;
}

void server_free(ipa_server* s) {
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    for (double* a : s->arena) cudaFree(a);
    void* dev[] = {s->d_specs, s->d_states, s->d_theta_eval, s->d_res, s->d_active, s->d_begin, s->d_end,
                   s->d_nact, s->d_out_theta, s->d_out_err, s->d_out_nll, s->d_out_status, s->d_out_iters,
                   s->d_out_passes, s->sc.partials, s->sc.counters, s->sc.gcount, s->sc.work, s->sc.seg_tiles,
                   s->sc.consts};
    for (void* p : dev) cudaFree(p);
    void* host[] = {s->h_begin, s->h_end, s->h_active, s->h_out_theta, s->h_out_err, s->h_out_nll,
                    s->h_out_status, s->h_out_iters, s->h_out_passes};
    for (void* p : host) cudaFreeHost(p);
    if (s->stream) cudaStreamDestroy(s->stream);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_server_create(const ipa_model* model, size_t hbm_budget_bytes, int32_t max_slots,
                                        int32_t max_iter, double tol, ipa_server** out) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if (model->kind == IPA_MODEL_PHIS || n_acc(model->kind, true) > kSmallAcc) {
        set_error("ipa_server_create: the phi_s model is not served (fit it with ipa_fit_batch)");
        return IPA_ERR_ARG;
    }
    if (!out || max_slots < 1 || max_slots > 65536 || max_iter < 1 || !(tol > 0.0)) {
        set_error("ipa_server_create: bad arguments");
        return IPA_ERR_ARG;
    }
    const int64_t cap = (int64_t)(hbm_budget_bytes / (5 * sizeof(double)));
    if (cap < kTile) {
        set_error("ipa_server_create: HBM budget below one tile of events");
        return IPA_ERR_ARG;
    }
    ipa_server* s = new ipa_server();
    s->model = *model;
    s->P = model->n_par;
    s->max_slots = max_slots;
    s->max_iter = max_iter;
    s->tol = tol;
    s->arena_cap = cap;
    cudaGetDevice(&s->device);
    const int P = s->P;
    const size_t S = (size_t)max_slots;
    const int n_cols = arena_cols(model->kind);
    st = cuda_fail(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "server stream");
    for (int c = 0; c < 5 && st == IPA_OK; ++c)
        if (c < n_cols || c == 4) st = dalloc(&s->arena[c], (size_t)cap, "server arena");
    if (st == IPA_OK) st = dalloc(&s->d_specs, S, "server specs");
    if (st == IPA_OK) st = dalloc(&s->d_states, S, "server states");
    if (st == IPA_OK) st = dalloc(&s->d_theta_eval, S * P, "server theta");
    if (st == IPA_OK) st = dalloc(&s->d_res, S * (1 + P), "server results");
    if (st == IPA_OK) st = dalloc(&s->d_active, S, "server mask");
    if (st == IPA_OK) st = dalloc(&s->d_begin, S, "server ranges");
    if (st == IPA_OK) st = dalloc(&s->d_end, S, "server ranges");
    if (st == IPA_OK) st = dalloc(&s->d_nact, 1, "server count");
    if (st == IPA_OK) st = dalloc(&s->d_out_theta, S * P, "server out");
    if (st == IPA_OK) st = dalloc(&s->d_out_err, S * P, "server out");
    if (st == IPA_OK) st = dalloc(&s->d_out_nll, S, "server out");
    if (st == IPA_OK) st = dalloc(&s->d_out_status, S, "server out");
    if (st == IPA_OK) st = dalloc(&s->d_out_iters, S, "server out");
    if (st == IPA_OK) st = dalloc(&s->d_out_passes, S, "server out");
    const size_t tiles = (size_t)(cap / kTile + max_slots + 1);
    if (st == IPA_OK) st = dalloc(&s->sc.partials, tiles * kSmallAcc, "server partials");
    if (st == IPA_OK) st = dalloc(&s->sc.counters, S + 1, "server counters");
    if (st == IPA_OK) st = dalloc(&s->sc.gcount, tiles, "server group counters");
    if (st == IPA_OK) st = dalloc(&s->sc.work, 2, "server work counters");
    if (st == IPA_OK) st = dalloc(&s->sc.seg_tiles, S + 1, "server tiles");
    if (st == IPA_OK) st = dalloc(&s->sc.consts, S, "server consts");
    s->sc.partials_cap = tiles * kSmallAcc;
    s->sc.seg_cap = S + 1;
    if (st == IPA_OK) st = halloc(&s->h_begin, S, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_end, S, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_active, S, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_out_theta, S * P, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_out_err, S * P, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_out_nll, S, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_out_status, S, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_out_iters, S, "server pinned");
    if (st == IPA_OK) st = halloc(&s->h_out_passes, S, "server pinned");
    // every slot table starts at zero: slots never given a fit hold an empty spec
    // (no parameters), which the state-machine kernels skip
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->d_specs, 0, sizeof(Spec) * S, s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->d_states, 0, sizeof(State) * S, s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->d_res, 0, sizeof(double) * S * (1 + P), s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->d_active, 0, sizeof(int) * S, s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->sc.counters, 0, sizeof(unsigned) * (S + 1), s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->sc.gcount, 0, sizeof(unsigned) * tiles, s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->sc.work, 0, 2 * sizeof(unsigned), s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->d_begin, 0, sizeof(int64_t) * S, s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->d_end, 0, sizeof(int64_t) * S, s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaMemsetAsync(s->d_theta_eval, 0, sizeof(double) * S * P, s->stream), "server init");
    if (st == IPA_OK) st = cuda_fail(cudaStreamSynchronize(s->stream), "server init");
    // capture the K-pass tick once; it reads the slot tables from device memory
    if (st == IPA_OK) {
        if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "server capture");
        } else {
            ipa_status q = IPA_OK;
            for (int k = 0; k < kTickPasses && q == IPA_OK; ++k) q = server_pass(s);
            const cudaError_t e = cudaStreamEndCapture(s->stream, &s->graph);
            if (q != IPA_OK) st = q;
            else if (e != cudaSuccess) st = cuda_fail(e, "server capture");
            else st = cuda_fail(cudaGraphInstantiate(&s->exec, s->graph, 0), "server graph");
        }
    }
    if (st != IPA_OK) {
        server_free(s);
        return st;
    }
    s->slot_req.assign(S, nullptr);
    s->free_ranges[0] = cap;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return IPA_OK;
}

extern "C" ipa_status ipa_serve_submit(ipa_server* s, const ipa_events* ev, const ipa_param* spec,
                                       uint64_t* ticket) {
    using namespace ipa;
    if (!s || !spec || !ticket) {
        set_error("ipa_serve_submit: NULL argument");
        return IPA_ERR_ARG;
    }
    // the events are copied, so any alignment is accepted
    if (!ev || ev->n < 0 ||
        (ev->n > 0 && (!ev->t || (s->model.kind == IPA_MODEL_ANGTIME4D && (!ev->ck || !ev->cl || !ev->phi)) ||
                       (s->model.kind == IPA_MODEL_TAGGED1D && !ev->q)))) {
        set_error("ipa_serve_submit: missing event columns or negative count");
        return IPA_ERR_ARG;
    }
    ipa_status st = IPA_OK;
    if (ev->n > s->arena_cap) {
        set_error("ipa_serve_submit: %lld events exceed the server's HBM budget of %lld events",
                  (long long)ev->n, (long long)s->arena_cap);
        return IPA_ERR_ARG;
    }
    if (fault(IPA_FAULT_SUBMIT)) {
        set_error("ipa_serve_submit: staging allocation failed (injected, IPA_FAULT_SUBMIT); the request was "
                  "not taken and may be submitted again");
        return IPA_ERR_OOM;
    }
    Request* r = new Request();
    if ((st = build_spec(&s->model, spec, s->max_iter, s->tol, &r->spec)) != IPA_OK) {
        delete r;
        return st;
    }
    for (int p = 0; p < s->P; ++p) r->theta0[p] = spec[p].value;
    r->n = ev->n;
    r->weighted = ev->w != nullptr;
    const double* src[5] = {ev->t, s->model.kind == IPA_MODEL_TAGGED1D ? ev->q : ev->ck, ev->cl, ev->phi, ev->w};
    const int n_cols = arena_cols(s->model.kind);
    for (int c = 0; c < 5; ++c) {
        if ((c >= n_cols && c != 4) || !src[c] || r->n == 0) continue;
        r->cols[c].resize((size_t)r->n);
        cudaPointerAttributes attr{};
        const bool on_device = cudaPointerGetAttributes(&attr, src[c]) == cudaSuccess &&
                               (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        if (on_device) {
            st = cuda_fail(cudaMemcpy(r->cols[c].data(), src[c], sizeof(double) * r->n, cudaMemcpyDeviceToHost),
                           "ipa_serve_submit: copy of the events");
        } else {
            memcpy(r->cols[c].data(), src[c], sizeof(double) * r->n);
        }
        if (st != IPA_OK) {
            delete r;
            return st;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != IPA_OK) {
        delete r;
        set_error("ipa_serve_submit: server stopped after an error: %s", s->fatal_msg);
        return s->fatal;
    }
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    s->cv.notify_all();
    return IPA_OK;
}

extern "C" ipa_status ipa_serve_poll(ipa_server* s, uint64_t ticket, double* theta_out, double* err_out,
                                     double* nll, int32_t* fit_status) {
    using namespace ipa;
    if (!s) {
        set_error("ipa_serve_poll: NULL server");
        return IPA_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("ipa_serve_poll: unknown ticket %llu", (unsigned long long)ticket);
        return IPA_ERR_ARG;
    }
    Request* r = it->second;
    if (r->state != kFinished) return IPA_PENDING;
    const ipa_status err = r->error;
    if (err == IPA_OK) {
        for (int p = 0; p < s->P; ++p) {
            if (theta_out) theta_out[p] = r->theta[p];
            if (err_out) err_out[p] = r->err[p];
        }
        if (nll) *nll = r->nll;
        if (fit_status) *fit_status = r->status;
    } else {
        set_error("ipa_serve_poll: %s", s->fatal_msg);
    }
    s->reqs.erase(it);
    delete r;
    return err;
}

extern "C" ipa_status ipa_server_destroy(ipa_server* s) {
    using namespace ipa;
    if (!s) return IPA_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->stream);
    server_free(s);
    return IPA_OK;
}
