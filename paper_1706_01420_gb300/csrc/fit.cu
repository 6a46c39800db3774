// ipa_fit_batch: many fits advanced together on the device (the per-fit
// state machine is in fitcore.cuh).  The host replays a CUDA graph of K passes
// [tile map -> constants -> NLL+grad -> state update] until every fit is DONE;
// fits that are done drop out of the tile map, so stragglers do not pay for
// the whole batch.
#include <math.h>
#include <string.h>

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

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace
}  // namespace ipa

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

    // The fit runs on a library stream (capturable even when the caller passes the
    // legacy default stream), ordered after the caller's stream by an event.
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t s = fit_stream();
    if (!s) return IPA_ERR_CUDA;
    cudaEvent_t ev_in = nullptr;
    if ((st = cuda_fail(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming), "fit event")) != IPA_OK)
        return st;
    cudaEventRecord(ev_in, user);
    cudaStreamWaitEvent(s, ev_in, 0);
    cudaEventDestroy(ev_in);

    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    const int P = model->n_par;
    Scratch* sc = nullptr;
    if ((st = scratch_get((ev->n + kTile - 1) / kTile + n_fits, n_fits + 1, &sc)) != IPA_OK) return st;

    DevBuf b_spec, b_state, b_eval, b_res, b_active, b_nact;
    if ((st = cuda_fail(cudaMalloc(&b_spec.p, sizeof(Spec)), "fit spec")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_state.p, sizeof(State) * (size_t)n_fits), "fit state")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_eval.p, sizeof(double) * (size_t)n_fits * P), "fit theta")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_res.p, sizeof(double) * (size_t)n_fits * (1 + P)), "fit results")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_active.p, sizeof(int) * (size_t)n_fits), "fit mask")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_nact.p, sizeof(int) * kGraphSteps), "fit count")) != IPA_OK) return st;
    Spec* d_spec = static_cast<Spec*>(b_spec.p);
    State* states = static_cast<State*>(b_state.p);
    double* theta_eval = static_cast<double*>(b_eval.p);
    double* res = static_cast<double*>(b_res.p);
    int* active = static_cast<int*>(b_active.p);
    int* n_active = static_cast<int*>(b_nact.p);
    int* h_nact = nullptr;
    if ((st = cuda_fail(cudaMallocHost(&h_nact, sizeof(int) * kGraphSteps), "pinned count")) != IPA_OK) return st;

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // every exit waits for the library stream before the buffers are freed
    auto done = [&](ipa_status r) -> ipa_status {
        cudaStreamSynchronize(s);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFreeHost(h_nact);
        return r;
    };

    const int fb = 128, fg = (n_fits + fb - 1) / fb;
    if ((st = cuda_fail(cudaMemcpyAsync(d_spec, &sp, sizeof(Spec), cudaMemcpyHostToDevice, s), "fit spec copy")) != IPA_OK)
        return done(st);
    init_kernel<<<fg, fb, 0, s>>>(d_spec, 0, n_fits, theta_io_dev, states, theta_eval, active);
    if ((st = cuda_fail(cudaGetLastError(), "fit init")) != IPA_OK) return done(st);

    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride};
    // one pass = tile map, constants, segmented NLL+grad, state update
    auto pass = [&](int k) -> ipa_status {
        ipa_status q;
        if ((q = launch_seg_tiles(seg_off_dev, seg_off_dev + 1, active, n_fits, ev->n, sc->seg_tiles, s)) != IPA_OK)
            return q;
        if ((q = launch_consts(m, theta_eval, n_fits, sc->consts, s)) != IPA_OK) return q;
        if ((q = launch_nll(m, true, cols, ev->n, seg_off_dev, seg_off_dev + 1, sc->seg_tiles, n_fits,
                            sc->consts, sc, res, s)) != IPA_OK)
            return q;
        if ((q = cuda_fail(cudaMemsetAsync(n_active + k, 0, sizeof(int), s), "fit count reset")) != IPA_OK)
            return q;
        qn_kernel<<<fg, fb, 0, s>>>(d_spec, 0, n_fits, seg_off_dev, seg_off_dev + 1, res, states, theta_eval,
                                    active, n_active + k);
        return cuda_fail(cudaGetLastError(), "fit step");
    };

    // capture kGraphSteps passes once, replay until every fit is done
    bool use_graph = false;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        ipa_status q = IPA_OK;
        for (int k = 0; k < kGraphSteps && q == IPA_OK; ++k) q = pass(k);
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        use_graph = q == IPA_OK && e == cudaSuccess &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (!use_graph) cudaGetLastError();
    } else {
        cudaGetLastError();
    }
    const int max_rounds = (sp.max_passes + kGraphSteps - 1) / kGraphSteps + 2;
    for (int round = 0; round < max_rounds && st == IPA_OK; ++round) {
        if (use_graph) {
            st = cuda_fail(cudaGraphLaunch(exec, s), "fit graph launch");
        } else {
            for (int k = 0; k < kGraphSteps && st == IPA_OK; ++k) st = pass(k);
        }
        if (st != IPA_OK) break;
        st = cuda_fail(cudaMemcpyAsync(h_nact, n_active, sizeof(int) * kGraphSteps, cudaMemcpyDeviceToHost, s),
                       "fit count copy");
        if (st == IPA_OK) st = cuda_fail(cudaStreamSynchronize(s), "fit sync");
        if (st == IPA_OK && h_nact[kGraphSteps - 1] == 0) break;
    }
    if (st != IPA_OK) return done(st);
    final_kernel<<<fg, fb, 0, s>>>(d_spec, 0, n_fits, states, theta_io_dev, err_out_dev, nll_out_dev,
                                   fit_status_dev, iters_out_dev, passes_out_dev);
    st = cuda_fail(cudaGetLastError(), "fit final");
    st = done(st);
    if (st == IPA_OK) st = cuda_fail(cudaGetLastError(), "fit final sync");
    // later work on the caller's stream sees the results: the call is blocking
    return st;
}
