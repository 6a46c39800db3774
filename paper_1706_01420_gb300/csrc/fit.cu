// ipa_fit_batch: many fits advanced together on the device (the per-fit
// state machine is in fitcore.cuh).  One CUDA graph launch runs the whole
// minimisation: a conditional WHILE node repeats K passes [tile map ->
// constants -> NLL+grad -> state update] until every fit is DONE, decided on
// the device; fits that are done drop out of the tile map, so stragglers do not
// pay for the whole batch.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "fitcore.cuh"
#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr int kGraphSteps = 8;     // passes per graph replay

// One library stream per device for the fitter (non-blocking, so it can be captured).
cudaStream_t fit_stream() {
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return nullptr;
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        set_error("could not create the fitter stream");
        return nullptr;
    }
    return streams[dev];
}

// Last kernel of the loop body: run the body again while any fit is active and
// fewer than max_rounds bodies have run.
__global__ void continue_kernel(cudaGraphConditionalHandle handle, const int* n_active, int* rounds,
                                int max_rounds) {
    const int r = ++(*rounds);
    cudaGraphSetConditional(handle, (*n_active > 0 && r < max_rounds) ? 1u : 0u);
}

// Per-device fit workspace, kept between calls (grow-only), with the graph of
// the last call: a graph reads only workspace and scratch buffers and the event
// columns, so consecutive fits of the same event set (one toy after another)
// reuse it without capturing again.
constexpr int kKeyPtrs = 25;
struct GraphKey {
    int kind = 0, n_par = 0, n_fits = 0, max_rounds = 0, spec_stride = 0, n_cat = 0, n_joint = 0;
    unsigned tune = 0;             // launch-geometry table version the graph was captured with
    double t_lo = 0.0, t_hi = 0.0;
    int64_t n = 0, fk_stride = 0;
    const void* ptr[kKeyPtrs] = {};
    bool operator==(const GraphKey& o) const {
        if (kind != o.kind || n_par != o.n_par || n_fits != o.n_fits || max_rounds != o.max_rounds ||
            spec_stride != o.spec_stride || n_cat != o.n_cat || n_joint != o.n_joint || tune != o.tune ||
            t_lo != o.t_lo || t_hi != o.t_hi || n != o.n || fk_stride != o.fk_stride)
            return false;
        for (int i = 0; i < kKeyPtrs; ++i)
            if (ptr[i] != o.ptr[i]) return false;
        return true;
    }
};

struct FitContext {
    std::mutex mu;
    int cap = 0;                   // fits the buffers hold
    State* states = nullptr;
    double* theta_eval = nullptr;
    double* res = nullptr;
    int* active = nullptr;
    int* nact = nullptr;           // kGraphSteps pass counts + the loop-body counter
    int* h_nact = nullptr;         // pinned copy of the pass counts (host-loop fallback)
    cudaEvent_t order = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool one_launch = false;
    bool have_key = false;
    GraphKey key;
};

FitContext* fit_context() {
    static FitContext ctx[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    return &ctx[dev];
}

void drop_graph(FitContext& c) {
    if (c.exec) cudaGraphExecDestroy(c.exec);
    if (c.graph) cudaGraphDestroy(c.graph);
    c.exec = nullptr;
    c.graph = nullptr;
    c.have_key = false;
}

ipa_status ensure_capacity(FitContext& c, int n_fits, int P) {
    if (!c.order) {
        ipa_status st = cuda_fail(cudaEventCreateWithFlags(&c.order, cudaEventDisableTiming), "fit event");
        if (st != IPA_OK) return st;
    }
    if (!c.nact) {
        ipa_status st = device_alloc((void**)&c.nact, sizeof(int) * (kGraphSteps + 1), "fit count");
        if (st == IPA_OK) st = cuda_fail(cudaMallocHost(&c.h_nact, sizeof(int) * kGraphSteps), "pinned count");
        if (st != IPA_OK) return st;
    }
    if (n_fits <= c.cap) return IPA_OK;
    int cap = c.cap ? c.cap : 64;
    while (cap < n_fits) cap *= 2;
    cudaDeviceSynchronize();
    drop_graph(c);
    cudaFree(c.states);
    cudaFree(c.theta_eval);
    cudaFree(c.res);
    cudaFree(c.active);
    c.states = nullptr;
    c.theta_eval = c.res = nullptr;
    c.active = nullptr;
    c.cap = 0;
    const size_t n = (size_t)cap;
    ipa_status st = device_alloc((void**)&c.states, sizeof(State) * n, "fit state");
    if (st == IPA_OK) st = device_alloc((void**)&c.theta_eval, sizeof(double) * n * kMaxP, "fit theta");
    if (st == IPA_OK) st = device_alloc((void**)&c.res, sizeof(double) * n * (1 + kMaxP), "fit results");
    if (st == IPA_OK) st = device_alloc((void**)&c.active, sizeof(int) * n, "fit mask");
    if (st == IPA_OK) c.cap = cap;
    (void)P;
    return st;
}

// ipa_fit_batch's specification and offsets in device memory (per device,
// grow-only; the mutex spans a whole call).
struct BatchArgs {
    std::mutex mu;
    Spec* spec = nullptr;
    int64_t* seg_off = nullptr;
    int cap = 0;
};

BatchArgs* batch_args_of_device() {
    static BatchArgs args[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    return &args[dev];
}

// Grow the arguments buffer to n_fits fits (the caller holds a.mu).
ipa_status batch_args_reserve(BatchArgs& a, int n_fits) {
    if (!a.spec && device_alloc((void**)&a.spec, sizeof(Spec), "fit spec") != IPA_OK) {
        a.spec = nullptr;
        set_error("fit spec allocation failed");
        return IPA_ERR_OOM;
    }
    if (n_fits <= a.cap) return IPA_OK;
    int cap = a.cap ? a.cap : 64;
    while (cap < n_fits) cap *= 2;
    cudaDeviceSynchronize();
    cudaFree(a.seg_off);
    a.seg_off = nullptr;
    a.cap = 0;
    ipa_status st = device_alloc((void**)&a.seg_off, sizeof(int64_t) * ((size_t)cap + 1), "fit offsets");
    if (st == IPA_OK) a.cap = cap;
    return st;
}

}  // namespace

ipa_status fit_run(const ipa_model* model, const ipa_events* ev, int n_fits, const int64_t* begin,
                   const int64_t* end, const Spec* specs, int spec_stride, int max_passes, int64_t tiles_bound,
                   double* theta_io_dev, double* err_out_dev, double* nll_out_dev, int32_t* fit_status_dev,
                   int32_t* iters_out_dev, int32_t* passes_out_dev, cudaStream_t user, const char* who,
                   const JointDev* joint) {
    // The fit runs on a library stream (capturable even when the caller passes the
    // legacy default stream), ordered after the caller's stream by an event.
    cudaStream_t s = fit_stream();
    FitContext* cp = fit_context();
    if (!s || !cp) return IPA_ERR_CUDA;
    FitContext& c = *cp;
    std::lock_guard<std::mutex> lk(c.mu);      // one fit call per device at a time
    ipa_status st;
    if ((st = ensure_capacity(c, n_fits, model->n_par)) != IPA_OK) return st;
    cudaEventRecord(c.order, user);
    cudaStreamWaitEvent(s, c.order, 0);

    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    Scratch* sc = nullptr;
    const int n_seg = joint ? n_fits * joint->n_cat : n_fits;
    if ((st = scratch_get(tiles_bound, n_seg + 1, &sc)) != IPA_OK) return st;
    int* n_active = c.nact;
    int* d_rounds = c.nact + kGraphSteps;
    const int max_rounds = (max_passes + kGraphSteps - 1) / kGraphSteps + 2;
    auto done = [&](ipa_status r) -> ipa_status {
        cudaStreamSynchronize(s);
        return r;
    };

    const int fb = 128, fg = (n_fits + fb - 1) / fb;
    init_kernel<<<fg, fb, 0, s>>>(specs, spec_stride, n_fits, theta_io_dev, c.states, c.theta_eval, c.active);
    if ((st = cuda_fail(cudaGetLastError(), "fit init")) != IPA_OK) return done(st);

    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride, ev->q};
    // one pass = tile map, constants, segmented NLL+grad, state update
    // (a joint fit: the categories' parameters from the joint ones, the NLL and
    // gradient per category, their sums per fit)
    auto pass = [&](int k) -> ipa_status {
        ipa_status q;
        if (joint) {
            if ((q = launch_joint_scatter(*joint, n_fits, c.theta_eval, c.active, s)) != IPA_OK) return q;
            if ((q = launch_seg_tiles(joint->seg_begin, joint->seg_end, joint->seg_active, n_seg, ev->n,
                                      sc->seg_tiles, s)) != IPA_OK)
                return q;
            if ((q = launch_consts(m, joint->theta_seg, n_seg, sc->consts, s)) != IPA_OK) return q;
            if ((q = launch_nll(m, true, cols, ev->n, joint->seg_begin, joint->seg_end, sc->seg_tiles, n_seg,
                                sc->consts, sc, joint->res_seg, s)) != IPA_OK)
                return q;
            if ((q = launch_joint_gather(*joint, n_fits, c.active, c.res, s)) != IPA_OK) return q;
        } else {
            if ((q = launch_seg_tiles(begin, end, c.active, n_fits, ev->n, sc->seg_tiles, s)) != IPA_OK)
                return q;
            if ((q = launch_consts(m, c.theta_eval, n_fits, sc->consts, s)) != IPA_OK) return q;
            if ((q = launch_nll(m, true, cols, ev->n, begin, end, sc->seg_tiles, n_fits, sc->consts, sc, c.res,
                                s)) != IPA_OK)
                return q;
        }
        if ((q = cuda_fail(cudaMemsetAsync(n_active + k, 0, sizeof(int), s), "fit count reset")) != IPA_OK)
            return q;
        qn_kernel<<<fg, fb, 0, s>>>(specs, spec_stride, n_fits, begin, end, c.res, c.states, c.theta_eval,
                                    c.active, n_active + k);
        return cuda_fail(cudaGetLastError(), "fit step");
    };

    GraphKey key;
    key.kind = m.kind;
    key.n_par = m.n_par;
    key.n_fits = n_fits;
    key.max_rounds = max_rounds;
    key.spec_stride = spec_stride;
    key.t_lo = m.t_lo;
    key.t_hi = m.t_hi;
    key.n = ev->n;
    key.fk_stride = ev->fk_stride;
    key.tune = tune_epoch();
    key.n_cat = joint ? joint->n_cat : 0;
    key.n_joint = joint ? joint->n_joint : 0;
    const void* ptrs[kKeyPtrs] = {ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->q, sc->partials, sc->counters,
                                  sc->gcount, sc->work, sc->seg_tiles, sc->consts, c.states, begin, end, specs,
                                  (const void*)s,
                                  joint ? (const void*)joint->map : nullptr,
                                  joint ? (const void*)joint->value : nullptr,
                                  joint ? (const void*)joint->seg_begin : nullptr,
                                  joint ? (const void*)joint->seg_end : nullptr,
                                  joint ? (const void*)joint->theta_seg : nullptr,
                                  joint ? (const void*)joint->res_seg : nullptr,
                                  joint ? (const void*)joint->seg_active : nullptr};
    for (int i = 0; i < kKeyPtrs; ++i) key.ptr[i] = ptrs[i];
    if (!(c.have_key && c.key == key)) {
        // Preferred: the whole minimisation as ONE graph launch.  A conditional
        // WHILE node repeats a body of kGraphSteps passes; the last kernel of the
        // body keeps the loop going while any fit is active and fewer than
        // max_rounds bodies have run (so the loop always ends).
        drop_graph(c);
        cudaGraphConditionalHandle handle;
        cudaGraphNodeParams np = {};
        cudaGraphNode_t cnode;
        bool ok = cudaGraphCreate(&c.graph, 0) == cudaSuccess &&
                  cudaGraphConditionalHandleCreate(&handle, c.graph, 1u, cudaGraphCondAssignDefault) == cudaSuccess;
        if (ok) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = handle;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            ok = cudaGraphAddNode(&cnode, c.graph, nullptr, nullptr, 0, &np) == cudaSuccess;
        }
        if (ok && cudaStreamBeginCaptureToGraph(s, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            ipa_status q = IPA_OK;
            for (int k = 0; k < kGraphSteps && q == IPA_OK; ++k) q = pass(k);
            if (q == IPA_OK) {
                continue_kernel<<<1, 1, 0, s>>>(handle, n_active + kGraphSteps - 1, d_rounds, max_rounds);
                q = cuda_fail(cudaGetLastError(), "fit loop condition");
            }
            cudaGraph_t body = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &body);
            ok = q == IPA_OK && e == cudaSuccess && cudaGraphInstantiate(&c.exec, c.graph, 0) == cudaSuccess;
        } else {
            ok = false;
        }
        c.one_launch = ok;
        if (!ok) {
            // Fallback: a graph of kGraphSteps passes replayed from the host
            cudaGetLastError();
            drop_graph(c);
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                ipa_status q = IPA_OK;
                for (int k = 0; k < kGraphSteps && q == IPA_OK; ++k) q = pass(k);
                const cudaError_t e = cudaStreamEndCapture(s, &c.graph);
                if (!(q == IPA_OK && e == cudaSuccess && cudaGraphInstantiate(&c.exec, c.graph, 0) == cudaSuccess)) {
                    cudaGetLastError();
                    drop_graph(c);
                }
            } else {
                cudaGetLastError();
            }
        }
        if (c.exec) {
            c.key = key;
            c.have_key = true;
        }
    }
    if (c.one_launch && c.exec) {
        st = cuda_fail(cudaMemsetAsync(d_rounds, 0, sizeof(int), s), "fit loop counter");
        if (st == IPA_OK) st = cuda_fail(cudaGraphLaunch(c.exec, s), "fit graph launch");
    } else {
        for (int round = 0; round < max_rounds && st == IPA_OK; ++round) {
            if (c.exec) {
                st = cuda_fail(cudaGraphLaunch(c.exec, s), "fit graph launch");
            } else {
                for (int k = 0; k < kGraphSteps && st == IPA_OK; ++k) st = pass(k);
            }
            if (st != IPA_OK) break;
            st = cuda_fail(cudaMemcpyAsync(c.h_nact, n_active, sizeof(int) * kGraphSteps, cudaMemcpyDeviceToHost, s),
                           "fit count copy");
            if (st == IPA_OK) st = cuda_fail(cudaStreamSynchronize(s), "fit sync");
            if (st == IPA_OK && c.h_nact[kGraphSteps - 1] == 0) break;
        }
    }
    if (st != IPA_OK) return done(st);
    final_kernel<<<fg, fb, 0, s>>>(specs, spec_stride, n_fits, c.states, theta_io_dev, err_out_dev, nll_out_dev,
                                   fit_status_dev, iters_out_dev, passes_out_dev);
    st = cuda_fail(cudaGetLastError(), "fit final");
    st = done(st);
    if (st == IPA_OK) st = cuda_fail(cudaGetLastError(), "fit final sync");
    trace("{\"call\": \"%s\", \"n_fits\": %d, \"events\": %lld, \"loop\": \"%s\"}", who, n_fits,
          (long long)ev->n, c.one_launch && c.exec ? "device" : "host");
    // later work on the caller's stream sees the results: the call is blocking
    return st;
}

// ---- stepwise fits: the minimiser's state in memory the caller owns ----
// Layout of a state buffer of n fits with P parameters (offsets rounded up to
// 256 bytes): the n x P points to evaluate next, the Spec, n States, n
// activity flags.  Everything a fit's future depends on is in the buffer, so a
// copy taken between passes resumes the fits bit for bit.
namespace {
size_t round256(size_t b) { return (b + 255) / 256 * 256; }
struct StepLayout {
    size_t spec, states, active, total;
};
StepLayout step_layout(int n_fits, int n_par) {
    StepLayout l;
    l.spec = round256((size_t)n_fits * n_par * sizeof(double));
    l.states = l.spec + round256(sizeof(Spec));
    l.active = l.states + round256((size_t)n_fits * sizeof(State));
    l.total = l.active + round256((size_t)n_fits * sizeof(int));
    return l;
}
ipa_status step_args(const ipa_model* model, int n_fits, const void* state_dev) {
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if (n_fits < 1 || !state_dev || (reinterpret_cast<uintptr_t>(state_dev) & 255u)) {
        set_error("stepwise fit: n_fits >= 1 and a 256-byte aligned state buffer required");
        return IPA_ERR_ARG;
    }
    return IPA_OK;
}
}  // namespace
}  // namespace ipa

extern "C" uint64_t ipa_fit_state_bytes(int32_t n_fits, int32_t n_par) {
    if (n_fits < 1 || n_par < 1 || n_par > ipa::kMaxP) return 0;
    return ipa::step_layout(n_fits, n_par).total;
}

extern "C" ipa_status ipa_fit_begin(const ipa_model* model, const ipa_param* spec, int32_t n_fits,
                                    const double* theta0_dev, int32_t max_iter, double tol, void* state_dev,
                                    void* stream) {
    using namespace ipa;
    ipa_status st = step_args(model, n_fits, state_dev);
    if (st != IPA_OK) return st;
    if (!spec || !theta0_dev || max_iter < 1 || !(tol > 0.0)) {
        set_error("ipa_fit_begin: bad arguments");
        return IPA_ERR_ARG;
    }
    Spec sp{};
    if ((st = build_spec(model, spec, max_iter, tol, &sp)) != IPA_OK) return st;
    const StepLayout l = step_layout(n_fits, model->n_par);
    unsigned char* base = static_cast<unsigned char*>(state_dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a pageable source: the copy is staged before cudaMemcpyAsync returns
    if ((st = cuda_fail(cudaMemcpyAsync(base + l.spec, &sp, sizeof(Spec), cudaMemcpyHostToDevice, s),
                        "fit spec copy")) != IPA_OK)
        return st;
    const int fb = 128, fg = (n_fits + fb - 1) / fb;
    init_kernel<<<fg, fb, 0, s>>>(reinterpret_cast<const Spec*>(base + l.spec), 0, n_fits, theta0_dev,
                                  reinterpret_cast<State*>(base + l.states), reinterpret_cast<double*>(base),
                                  reinterpret_cast<int*>(base + l.active));
    return cuda_fail(cudaGetLastError(), "fit init");
}

extern "C" ipa_status ipa_fit_advance(const ipa_model* model, int32_t n_fits, const double* results_dev,
                                      void* state_dev, int32_t* n_active_dev, void* stream) {
    using namespace ipa;
    ipa_status st = step_args(model, n_fits, state_dev);
    if (st != IPA_OK) return st;
    if (!results_dev || !n_active_dev) {
        set_error("ipa_fit_advance: results and n_active are required");
        return IPA_ERR_ARG;
    }
    const StepLayout l = step_layout(n_fits, model->n_par);
    unsigned char* base = static_cast<unsigned char*>(state_dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = cuda_fail(cudaMemsetAsync(n_active_dev, 0, sizeof(int32_t), s), "fit count reset")) != IPA_OK)
        return st;
    const int fb = 128, fg = (n_fits + fb - 1) / fb;
    qn_kernel<<<fg, fb, 0, s>>>(reinterpret_cast<const Spec*>(base + l.spec), 0, n_fits, nullptr, nullptr,
                                results_dev, reinterpret_cast<State*>(base + l.states),
                                reinterpret_cast<double*>(base), reinterpret_cast<int*>(base + l.active),
                                n_active_dev);
    return cuda_fail(cudaGetLastError(), "fit step");
}

extern "C" ipa_status ipa_fit_end(const ipa_model* model, int32_t n_fits, const void* state_dev,
                                  double* theta_out_dev, double* err_out_dev, double* nll_out_dev,
                                  int32_t* fit_status_dev, int32_t* iters_out_dev, int32_t* passes_out_dev,
                                  void* stream) {
    using namespace ipa;
    ipa_status st = step_args(model, n_fits, state_dev);
    if (st != IPA_OK) return st;
    if (!theta_out_dev) {
        set_error("ipa_fit_end: theta_out is required");
        return IPA_ERR_ARG;
    }
    const StepLayout l = step_layout(n_fits, model->n_par);
    const unsigned char* base = static_cast<const unsigned char*>(state_dev);
    const int fb = 128, fg = (n_fits + fb - 1) / fb;
    final_kernel<<<fg, fb, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const Spec*>(base + l.spec), 0, n_fits, reinterpret_cast<const State*>(base + l.states),
        theta_out_dev, err_out_dev, nll_out_dev, fit_status_dev, iters_out_dev, passes_out_dev);
    return cuda_fail(cudaGetLastError(), "fit final");
}

extern "C" ipa_status ipa_fit_batch(const ipa_model* model, const ipa_events* ev,
                                    const int64_t* seg_off_dev, int32_t n_fits, const ipa_param* spec,
                                    double* theta_io_dev, double* err_out_dev, double* nll_out_dev,
                                    int32_t* fit_status_dev, int32_t* iters_out_dev,
                                    int32_t* passes_out_dev, int32_t max_iter, double tol, void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if (n_fits < 1 || !seg_off_dev || !spec || !theta_io_dev || max_iter < 1 || !(tol > 0.0)) {
        set_error("ipa_fit_batch: bad arguments");
        return IPA_ERR_ARG;
    }
    Spec sp{};
    if ((st = build_spec(model, spec, max_iter, tol, &sp)) != IPA_OK) return st;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    BatchArgs* ap = batch_args_of_device();
    if (!ap) return IPA_ERR_CUDA;
    BatchArgs& a = *ap;
    std::lock_guard<std::mutex> lk(a.mu);
    if ((st = batch_args_reserve(a, n_fits)) != IPA_OK) return st;
    // the specification and the offsets, in library buffers ordered on the caller's stream
    if ((st = cuda_fail(cudaMemcpyAsync(a.spec, &sp, sizeof(Spec), cudaMemcpyHostToDevice, user),
                        "fit spec copy")) != IPA_OK)
        return st;
    if ((st = cuda_fail(cudaMemcpyAsync(a.seg_off, seg_off_dev, sizeof(int64_t) * (n_fits + 1),
                                        cudaMemcpyDeviceToDevice, user), "fit offsets copy")) != IPA_OK)
        return st;
    st = fit_run(model, ev, n_fits, a.seg_off, a.seg_off + 1, a.spec, 0, sp.max_passes,
                 (ev->n + kTile - 1) / kTile + n_fits, theta_io_dev, err_out_dev, nll_out_dev, fit_status_dev,
                 iters_out_dev, passes_out_dev, user, "ipa_fit_batch");
    return st;
}
