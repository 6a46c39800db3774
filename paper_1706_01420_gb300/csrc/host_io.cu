// ipa_nll_grad_host: the NLL and gradient of events that sit in host memory.
// Page-locked columns are read by the kernel in place (the device's mapping
// of the host allocation): the transfer overlaps the event pass with no
// staging.  Pageable columns are copied into library staging buffers, chunk by chunk, on
// four copy streams (the columns spread over them, so several copy engines
// share the link) while the likelihood kernel runs, on the caller's stream,
// over the chunks already on the device; the chunks' results are then summed
// in chunk order.  A chunk holds at least 2^20 events: one pass of the kernel
// over fewer events takes about as long as over one full wave of tiles
// (1.2e6 events on 152 SMs), so smaller chunks would cost more kernel time
// than the overlap saves.
#include <mutex>

#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr int kMaxChunks = 16;
constexpr int64_t kMinChunk = (int64_t)1 << 20;   // events per chunk, at least
constexpr int kCols = 6;                          // t, ck, cl, phi, w, q
constexpr int kCopyStreams = 4;

struct HostStage {
    std::mutex mu;
    double* col[kCols] = {};
    int64_t cap = 0;                   // events each column holds
    double* part = nullptr;            // kMaxChunks x (1 + IPA_MAX_PAR) chunk results
    cudaStream_t copy[kCopyStreams] = {};
    cudaEvent_t start = nullptr;
    cudaEvent_t ready[kMaxChunks][kCopyStreams] = {};
};

HostStage* host_stage() {
    static HostStage st[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    return &st[dev];
}

ipa_status stage_reserve(HostStage& h, int64_t n) {
    ipa_status st = IPA_OK;
    if (!h.copy[0]) {
        for (int q = 0; q < kCopyStreams && st == IPA_OK; ++q)
            st = cuda_fail(cudaStreamCreateWithFlags(&h.copy[q], cudaStreamNonBlocking), "host copy stream");
        if (st == IPA_OK) st = cuda_fail(cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming), "host event");
        for (int c = 0; c < kMaxChunks && st == IPA_OK; ++c)
            for (int q = 0; q < kCopyStreams && st == IPA_OK; ++q)
                st = cuda_fail(cudaEventCreateWithFlags(&h.ready[c][q], cudaEventDisableTiming), "host event");
        if (st == IPA_OK)
            st = device_alloc((void**)&h.part, sizeof(double) * kMaxChunks * (1 + IPA_MAX_PAR), "chunk results");
        if (st != IPA_OK) return st;
    }
    if (n <= h.cap) return IPA_OK;
    int64_t cap = h.cap ? h.cap : kMinChunk;
    while (cap < n) cap *= 2;
    cudaDeviceSynchronize();           // a kernel of an earlier call may still read the old buffers
    for (int k = 0; k < kCols; ++k) {
        cudaFree(h.col[k]);
        h.col[k] = nullptr;
    }
    h.cap = 0;
    for (int k = 0; k < kCols; ++k)
        if ((st = device_alloc((void**)&h.col[k], sizeof(double) * cap, "host staging")) != IPA_OK) return st;
    h.cap = cap;
    return IPA_OK;
}

// out[j] = sum over chunks c = 0, 1, ... of part[c][j] (one thread per output)
__global__ void chunk_sum_kernel(const double* __restrict__ part, int n_chunks, int stride, int n_out,
                                 double* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= n_out) return;
    double v = 0.0;
    for (int c = 0; c < n_chunks; ++c) v += part[c * stride + j];
    out[j] = v;
}

// Chunks of a call over n events: k = clamp(floor(n / 2^20), 1, 16) pieces
// of ceil(ceil(n / k) / 512) * 512 events (whole tiles), the last one shorter.
int64_t host_chunk_events(int64_t n, int* n_chunks) {
    int k = (int)(n / kMinChunk);
    k = k < 1 ? 1 : (k > kMaxChunks ? kMaxChunks : k);
    const int64_t per = (n + k - 1) / k;
    const int64_t chunk = (per + kTile - 1) / kTile * kTile;
    *n_chunks = (int)((n + chunk - 1) / chunk);
    return chunk;
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_nll_grad_host(const ipa_model* model, const ipa_events* host_ev, const double* theta_dev,
                                        double* out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, host_ev)) != IPA_OK) return st;
    if (!theta_dev || !out_dev) {
        set_error("ipa_nll_grad_host: theta and out must be device pointers");
        return IPA_ERR_ARG;
    }
    if (host_ev->fk) {
        set_error("ipa_nll_grad_host: a cached angular basis is a device array; use ipa_nll_grad");
        return IPA_ERR_ARG;
    }
    const int64_t n = host_ev->n;
    if (n == 0) return ipa_nll_grad(model, host_ev, theta_dev, out_dev, stream);
    // page-locked columns: the kernel reads them where they are (through the
    // device's mapping of the host allocation), so the transfer runs inside
    // the event pass and nothing is staged
    {
        const double* src0[kCols] = {host_ev->t, host_ev->ck, host_ev->cl, host_ev->phi, host_ev->w, host_ev->q};
        double* mapped[kCols] = {};
        bool all_pinned = true;
        for (int k = 0; k < kCols && all_pinned; ++k) {
            if (!src0[k]) continue;
            cudaPointerAttributes a{};
            void* dp = nullptr;
            all_pinned = cudaPointerGetAttributes(&a, src0[k]) == cudaSuccess && a.type == cudaMemoryTypeHost &&
                         cudaHostGetDevicePointer(&dp, const_cast<double*>(src0[k]), 0) == cudaSuccess;
            mapped[k] = static_cast<double*>(dp);
        }
        cudaGetLastError();            // a pageable column leaves an error behind: clear it
        if (all_pinned) {
            ipa_events dev_ev = *host_ev;
            dev_ev.t = mapped[0];
            dev_ev.ck = mapped[1];
            dev_ev.cl = mapped[2];
            dev_ev.phi = mapped[3];
            dev_ev.w = mapped[4];
            dev_ev.q = mapped[5];
            return ipa_nll_grad(model, &dev_ev, theta_dev, out_dev, stream);
        }
    }
    HostStage* hp = host_stage();
    if (!hp) return IPA_ERR_CUDA;
    HostStage& h = *hp;
    std::lock_guard<std::mutex> lk(h.mu);
    if ((st = stage_reserve(h, n)) != IPA_OK) return st;
    int n_chunks = 1;
    const int64_t chunk = host_chunk_events(n, &n_chunks);
    Scratch* sc = nullptr;
    if ((st = scratch_get((chunk + kTile - 1) / kTile + 1, 2, &sc)) != IPA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double* src[kCols] = {host_ev->t, host_ev->ck, host_ev->cl, host_ev->phi, host_ev->w, host_ev->q};
    // the copies start after the caller's earlier work (which may still read the staging buffers)
    if ((st = cuda_fail(cudaEventRecord(h.start, s), "host order")) != IPA_OK) return st;
    for (int q = 0; q < kCopyStreams; ++q)
        if ((st = cuda_fail(cudaStreamWaitEvent(h.copy[q], h.start, 0), "host order")) != IPA_OK) return st;
    for (int c = 0; c < n_chunks; ++c) {
        const int64_t off = (int64_t)c * chunk, len = (n - off < chunk) ? n - off : chunk;
        int q = 0;
        for (int k = 0; k < kCols; ++k) {
            if (!src[k]) continue;
            st = cuda_fail(cudaMemcpyAsync(h.col[k] + off, src[k] + off, sizeof(double) * len,
                                           cudaMemcpyHostToDevice, h.copy[q]), "host column copy");
            if (st != IPA_OK) return st;
            q = (q + 1) % kCopyStreams;
        }
        for (int r = 0; r < kCopyStreams; ++r)
            if ((st = cuda_fail(cudaEventRecord(h.ready[c][r], h.copy[r]), "host chunk event")) != IPA_OK) return st;
    }
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_consts(m, theta_dev, 1, sc->consts, s)) != IPA_OK) return st;
    const int stride = 1 + model->n_par;
    for (int c = 0; c < n_chunks; ++c) {
        const int64_t off = (int64_t)c * chunk, len = (n - off < chunk) ? n - off : chunk;
        for (int r = 0; r < kCopyStreams; ++r)
            if ((st = cuda_fail(cudaStreamWaitEvent(s, h.ready[c][r], 0), "host chunk wait")) != IPA_OK) return st;
        auto at = [&](int k) -> const double* { return src[k] ? h.col[k] + off : nullptr; };
        const Cols cols{at(0), at(1), at(2), at(3), at(4), nullptr, 0, at(5)};
        if ((st = launch_nll(m, true, cols, len, nullptr, nullptr, nullptr, 1, sc->consts, sc, h.part + c * stride,
                             s)) != IPA_OK)
            return st;
    }
    chunk_sum_kernel<<<1, 64, 0, s>>>(h.part, n_chunks, stride, stride, out_dev);
    return cuda_fail(cudaGetLastError(), "chunk sum");
}
