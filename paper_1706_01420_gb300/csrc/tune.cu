// Launch-geometry autotuner of the likelihood kernel.
//
// The kernel's summation order is fixed by its 512-event tiles and 32-tile
// groups, so the block size, the number of resident warps per SM and the
// number of tiles a warp takes at once change only the speed, never a result.
// ipa_autotune times every candidate geometry on the caller's own events and
// keeps the fastest for that kernel variant (model, gradient or not, cached
// angular basis or not, one segment or many) and size class (the tile count
// rounded down to a power of two).  Launches of a size class nobody tuned use
// the built-in default: single-warp blocks with as many resident warps per SM
// as there are tiles per SM, which spreads small launches evenly over the SMs.
#include <math.h>

#include <map>
#include <mutex>
#include <vector>

#include "ipa_internal.cuh"

namespace ipa {
namespace {

std::mutex g_tune_mu;
std::map<uint64_t, LaunchCfg> g_table[64];   // per device ordinal
unsigned g_epoch = 1;

int size_class(int64_t tiles) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << (b + 1)) <= tiles) ++b;
    return b;
}

uint64_t table_key(int kind, bool grad, bool cached, bool segmented, int64_t tiles) {
    return (uint64_t)kind << 16 | (uint64_t)grad << 10 | (uint64_t)cached << 9 | (uint64_t)segmented << 8 |
           (uint64_t)size_class(tiles);
}

int device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev & 63;
}

bool valid(const LaunchCfg& c) {
    const int w = c.warps_per_block;
    const int k = c.tiles_per_take;
    return (w == 1 || w == 2 || w == 4 || w == 8) && c.warps_per_sm >= 0 && c.warps_per_sm <= 64 &&
           (k == 1 || k == 2 || k == 4);
}

LaunchCfg from_public(const ipa_launch_config& p) {
    return LaunchCfg{p.warps_per_block, p.warps_per_sm, p.tiles_per_take};
}

void to_public(const LaunchCfg& c, float ms, ipa_launch_config* p) {
    p->warps_per_block = c.warps_per_block;
    p->warps_per_sm = c.warps_per_sm;
    p->tiles_per_take = c.tiles_per_take;
    p->ms = ms;
}

}  // namespace

int64_t launch_grid(const LaunchCfg& cfg, int W, int K, int per_sm, int64_t tiles, bool single) {
    const int64_t sms = sm_count();
    const int64_t units = (tiles + K - 1) / K;
    int64_t want = cfg.warps_per_sm > 0 ? cfg.warps_per_sm : (units + sms - 1) / sms;
    if (want > (int64_t)per_sm * W) want = (int64_t)per_sm * W;
    if (want < 1) want = 1;
    int64_t grid = sms * ((want + W - 1) / W);
    if (single) {
        const int64_t need = (units + W - 1) / W;   // blocks beyond this find no tile
        grid = need < grid ? need : grid;
    }
    return grid < 1 ? 1 : grid;
}

LaunchCfg launch_cfg(int kind, bool grad, bool cached, bool segmented, int64_t tiles) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto& t = g_table[device()];
    auto it = t.find(table_key(kind, grad, cached, segmented, tiles));
    if (it != t.end()) return it->second;
    return LaunchCfg{1, 0, 1};
}

unsigned tune_epoch() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_epoch;
}

}  // namespace ipa

using namespace ipa;

namespace {

ipa_status config_args(const ipa_model* model, int64_t n_events, int32_t n_seg, ipa_launch_config* cfg) {
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if (n_events < 0 || n_seg < 1 || !cfg) {
        set_error("launch config: n_events >= 0, n_seg >= 1 and a config pointer required");
        return IPA_ERR_ARG;
    }
    return IPA_OK;
}

}  // namespace

extern "C" ipa_status ipa_launch_config_get(const ipa_model* model, int64_t n_events, int32_t n_seg, int32_t grad,
                                            int32_t cached, ipa_launch_config* cfg) {
    ipa_status st = config_args(model, n_events, n_seg, cfg);
    if (st != IPA_OK) return st;
    const bool c = cached && model->kind == IPA_MODEL_ANGTIME4D;
    to_public(launch_cfg(model->kind, grad != 0, c, n_seg > 1, tile_estimate(n_events, n_seg)), 0.0f, cfg);
    return IPA_OK;
}

extern "C" ipa_status ipa_launch_config_set(const ipa_model* model, int64_t n_events, int32_t n_seg, int32_t grad,
                                            int32_t cached, const ipa_launch_config* cfg) {
    ipa_status st = config_args(model, n_events, n_seg, const_cast<ipa_launch_config*>(cfg));
    if (st != IPA_OK) return st;
    const LaunchCfg c = from_public(*cfg);
    if (!valid(c)) {
        set_error("launch config: warps_per_block in {1,2,4,8}, warps_per_sm in [0, 64], tiles_per_take in {1,2,4}");
        return IPA_ERR_ARG;
    }
    const bool ca = cached && model->kind == IPA_MODEL_ANGTIME4D;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table[device()][table_key(model->kind, grad != 0, ca, n_seg > 1, tile_estimate(n_events, n_seg))] = c;
    ++g_epoch;
    return IPA_OK;
}

extern "C" ipa_status ipa_autotune(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                                   int32_t n_seg, const double* theta_dev, int32_t grad,
                                   ipa_launch_config* picked, void* stream) {
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if (!theta_dev || n_seg < 1 || (!seg_off_dev && n_seg != 1)) {
        set_error("ipa_autotune: theta required; n_seg >= 1 (offsets required for n_seg > 1)");
        return IPA_ERR_ARG;
    }
    if (ev->n == 0) {
        set_error("ipa_autotune: no events to time");
        return IPA_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((st = cuda_fail(cudaStreamIsCapturing(s, &cap), "stream query")) != IPA_OK) return st;
    if (cap != cudaStreamCaptureStatusNone) {
        set_error("ipa_autotune: the stream is being captured (tuning times launches and synchronises)");
        return IPA_ERR_BUSY;
    }
    const int64_t tiles = tile_estimate(ev->n, n_seg);
    Scratch* sc = nullptr;
    if ((st = scratch_get(tiles + n_seg, n_seg + 1, &sc)) != IPA_OK) return st;
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    const bool g = grad != 0;
    const int stride = g ? 1 + model->n_par : 1;
    double* out = nullptr;
    if ((st = device_alloc((void**)&out, sizeof(double) * (size_t)n_seg * stride, "tuner output")) != IPA_OK)
        return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride, ev->q};
    const int64_t* b = seg_off_dev;
    const int64_t* e = seg_off_dev ? seg_off_dev + 1 : nullptr;
    st = launch_consts(m, theta_dev, n_seg, sc->consts, s);
    if (st == IPA_OK && seg_off_dev) st = launch_seg_tiles(b, e, nullptr, n_seg, ev->n, sc->seg_tiles, s);

    // time one candidate: mean of `reps` back-to-back launches
    auto time_cfg = [&](const LaunchCfg& c, int reps, float* ms) -> ipa_status {
        ipa_status q = launch_nll(m, g, cols, ev->n, b, e, sc->seg_tiles, n_seg, sc->consts, sc, out, s, &c);
        if (q != IPA_OK) return q;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && q == IPA_OK; ++r)
            q = launch_nll(m, g, cols, ev->n, b, e, sc->seg_tiles, n_seg, sc->consts, sc, out, s, &c);
        cudaEventRecord(e1, s);
        if (q != IPA_OK) return q;
        if ((q = cuda_fail(cudaEventSynchronize(e1), "tuner timing")) != IPA_OK) return q;
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
        return IPA_OK;
    };

    std::vector<LaunchCfg> cands;
    for (int w : {1, 2, 4, 8})
        for (int wps : {0, 64})
            for (int k : {1, 2, 4}) cands.push_back(LaunchCfg{w, wps, k});
    LaunchCfg best = cands[0];
    float best_ms = INFINITY;
    int reps = 3;
    for (size_t i = 0; i < cands.size() && st == IPA_OK; ++i) {
        float ms = 0.0f;
        if (i == 0) {
            // size the repetitions from a first timing: about 5 ms per candidate
            if ((st = time_cfg(cands[0], 1, &ms)) != IPA_OK) break;
            reps = ms > 0.0f ? (int)ceilf(5.0f / ms) : 50;
            reps = reps < 3 ? 3 : (reps > 50 ? 50 : reps);
        }
        if ((st = time_cfg(cands[i], reps, &ms)) != IPA_OK) break;
        trace("{\"call\":\"ipa_autotune\",\"n\":%lld,\"n_seg\":%d,\"grad\":%d,\"warps_per_block\":%d,"
              "\"warps_per_sm\":%d,\"tiles_per_take\":%d,\"ms\":%.6f}",
              (long long)ev->n, n_seg, (int)g, cands[i].warps_per_block, cands[i].warps_per_sm,
              cands[i].tiles_per_take, ms);
        if (ms < best_ms) {
            best_ms = ms;
            best = cands[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(out);
    if (st != IPA_OK) return st;
    {
        const bool ca = ev->fk != nullptr && model->kind == IPA_MODEL_ANGTIME4D;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_table[device()][table_key(model->kind, g, ca, n_seg > 1, tiles)] = best;
        ++g_epoch;
    }
    if (picked) to_public(best, best_ms, picked);
    return IPA_OK;
}
