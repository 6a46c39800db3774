// Host runtime: argument checks, thread-local error text, per-device scratch.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "ipa_internal.cuh"

namespace ipa {

namespace {
// Host-side fault injection mask (ipa_fault_inject; IPA_FAULT at load).
uint32_t fault_from_env() {
    const char* v = getenv("IPA_FAULT");
    if (!v) return 0;
    uint32_t m = 0;
    if (strstr(v, "alloc")) m |= IPA_FAULT_ALLOC;
    if (strstr(v, "submit")) m |= IPA_FAULT_SUBMIT;
    if (strstr(v, "admit")) m |= IPA_FAULT_ADMIT;
    return m;
}
std::atomic<uint32_t> g_fault{fault_from_env()};
thread_local char g_err[512] = "";
std::mutex g_mu;
std::vector<Scratch> g_scratch;   // indexed by device ordinal
std::vector<int> g_sms;
}  // namespace

// IPA_TRACE=<path>: one JSON line per traced call, appended to <path> (the
// variable is read at every call, so it can be set or changed at run time).
void trace(const char* fmt, ...) {
    static std::mutex mu;
    static FILE* f = nullptr;
    static char open_path[1024] = "";
    const char* path = getenv("IPA_TRACE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lk(mu);
    if (!f || strncmp(path, open_path, sizeof(open_path)) != 0) {
        if (f) fclose(f);
        f = fopen(path, "a");
        snprintf(open_path, sizeof(open_path), "%s", path);
    }
    if (!f) return;
    va_list ap;
    va_start(ap, fmt);
    vfprintf(f, fmt, ap);
    va_end(ap);
    fputc('\n', f);
    fflush(f);
}

bool fault(uint32_t bit) { return (g_fault.load(std::memory_order_relaxed) & bit) != 0; }

ipa_status device_alloc(void** p, size_t bytes, const char* what) {
    if (fault(IPA_FAULT_ALLOC)) {
        set_error("%s: allocation of %zu bytes failed (injected, IPA_FAULT_ALLOC)", what, bytes);
        return IPA_ERR_OOM;
    }
    return cuda_fail(cudaMalloc(p, bytes), what);
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ipa_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return IPA_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? IPA_ERR_OOM : IPA_ERR_CUDA;
}

ipa_status check_model(const ipa_model* m) {
    if (!m) {
        set_error("model is NULL");
        return IPA_ERR_ARG;
    }
    if (m->kind != IPA_MODEL_TIME1D && m->kind != IPA_MODEL_ANGTIME4D && m->kind != IPA_MODEL_TAGGED1D &&
        m->kind != IPA_MODEL_PHIS) {
        set_error("unknown model kind %d", m->kind);
        return IPA_ERR_ARG;
    }
    const int want = npar_of(m->kind);
    if (m->n_par != want) {
        set_error("model n_par %d, expected %d (use ipa_model_init)", m->n_par, want);
        return IPA_ERR_ARG;
    }
    if (!(m->t_lo < m->t_hi)) {
        set_error("empty decay-time range [%g, %g]", m->t_lo, m->t_hi);
        return IPA_ERR_ARG;
    }
    return IPA_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

ipa_status check_events(const ipa_model* m, const ipa_events* ev) {
    if (!ev) {
        set_error("events are NULL");
        return IPA_ERR_ARG;
    }
    if (ev->n < 0) {
        set_error("negative event count %lld", (long long)ev->n);
        return IPA_ERR_ARG;
    }
    if (ev->n == 0) return IPA_OK;
    const bool tag = m->kind == IPA_MODEL_TAGGED1D;
    const double* need[5] = {ev->t, tag ? ev->q : ev->ck, ev->cl, ev->phi, ev->q};
    const int n_need = m->kind == IPA_MODEL_PHIS ? 5 : (m->kind == IPA_MODEL_ANGTIME4D ? 4 : (tag ? 2 : 1));
    const char* names[5] = {"t", tag ? "q" : "ck", "cl", "phi", "q"};
    for (int i = 0; i < n_need; ++i) {
        if (!need[i]) {
            set_error("event column %s is NULL", names[i]);
            return IPA_ERR_ARG;
        }
        if (!aligned16(need[i])) {
            set_error("event column %s is not 16-byte aligned", names[i]);
            return IPA_ERR_ARG;
        }
    }
    if (ev->w && !aligned16(ev->w)) {
        set_error("weight column is not 16-byte aligned");
        return IPA_ERR_ARG;
    }
    if (ev->fk) {
        if (m->kind != IPA_MODEL_ANGTIME4D && m->kind != IPA_MODEL_PHIS) {
            set_error("an angular basis was given for a model without angles");
            return IPA_ERR_ARG;
        }
        if (!aligned16(ev->fk) || ev->fk_stride < ev->n || (ev->fk_stride & 1)) {
            set_error("angular basis: 16-byte aligned, even stride >= n required");
            return IPA_ERR_ARG;
        }
    }
    return IPA_OK;
}

int sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_sms.size() <= dev) g_sms.resize(dev + 1, 0);
    if (g_sms[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = v > 0 ? v : 1;
    }
    return g_sms[dev];
}

// Grow-only scratch.  Growing frees the old buffers after a device
// synchronisation (a kernel of an earlier call may still read them).
ipa_status scratch_get(int64_t tiles, int64_t segs, Scratch** out) {
    int dev = 0;
    ipa_status st = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != IPA_OK) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_scratch.size() <= dev) g_scratch.resize(dev + 1);
    Scratch& s = g_scratch[dev];
    const size_t need_p = (size_t)(tiles < 1 ? 1 : tiles) * kMaxAcc;
    const size_t need_s = (size_t)(segs < 2 ? 2 : segs);
    if (need_p > s.partials_cap) {
        size_t cap = s.partials_cap ? s.partials_cap : (size_t)1 << 16;
        while (cap < need_p) cap *= 2;
        if (s.partials) {
            cudaDeviceSynchronize();
            cudaFree(s.partials);
            cudaFree(s.gcount);
            s.partials = nullptr;
            s.gcount = nullptr;
            s.partials_cap = 0;
        }
        if ((st = device_alloc((void**)&s.partials, cap * sizeof(double), "scratch partials")) != IPA_OK)
            return st;
        // one group counter per tile; zero between calls (kernels reset what they use)
        const size_t n_tiles = cap / kMaxAcc + 1;
        if ((st = device_alloc((void**)&s.gcount, n_tiles * sizeof(unsigned), "scratch group counters")) != IPA_OK) {
            cudaFree(s.partials);
            s.partials = nullptr;
            return st;
        }
        if ((st = cuda_fail(cudaMemset(s.gcount, 0, n_tiles * sizeof(unsigned)), "scratch memset")) != IPA_OK)
            return st;
        if ((st = cuda_fail(cudaDeviceSynchronize(), "scratch init")) != IPA_OK) return st;
        s.partials_cap = cap;
    }
    if (!s.work) {
        if ((st = device_alloc((void**)&s.work, 2 * sizeof(unsigned), "scratch work counters")) != IPA_OK) return st;
        if ((st = cuda_fail(cudaMemset(s.work, 0, 2 * sizeof(unsigned)), "scratch memset")) != IPA_OK) return st;
        if ((st = cuda_fail(cudaDeviceSynchronize(), "scratch init")) != IPA_OK) return st;
    }
    if (need_s > s.seg_cap) {
        size_t cap = s.seg_cap ? s.seg_cap : 64;
        while (cap < need_s) cap *= 2;
        if (s.counters) {
            cudaDeviceSynchronize();
            cudaFree(s.counters);
            cudaFree(s.seg_tiles);
            cudaFree(s.consts);
            s.counters = nullptr;
            s.seg_tiles = nullptr;
            s.consts = nullptr;
            s.seg_cap = 0;
        }
        if ((st = device_alloc((void**)&s.counters, cap * sizeof(unsigned), "scratch counters")) != IPA_OK)
            return st;
        if ((st = device_alloc((void**)&s.seg_tiles, (cap + 1) * sizeof(int64_t), "scratch tiles")) != IPA_OK ||
            (st = device_alloc((void**)&s.consts, cap * sizeof(Consts), "scratch consts")) != IPA_OK) {
            cudaFree(s.counters);
            cudaFree(s.seg_tiles);
            s.counters = nullptr;
            s.seg_tiles = nullptr;
            return st;
        }
        // counters must be zero between calls; kernels reset what they use
        if ((st = cuda_fail(cudaMemset(s.counters, 0, cap * sizeof(unsigned)), "scratch memset")) != IPA_OK)
            return st;
        if ((st = cuda_fail(cudaDeviceSynchronize(), "scratch init")) != IPA_OK) return st;
        s.seg_cap = cap;
    }
    *out = &s;
    return IPA_OK;
}

// Device bytes of the scratch held on device `dev` (the buffers scratch_get allocates).
uint64_t scratch_bytes(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= (int)g_scratch.size()) return 0;
    const Scratch& s = g_scratch[dev];
    uint64_t b = 0;
    if (s.partials) b += s.partials_cap * sizeof(double) + (s.partials_cap / kMaxAcc + 1) * sizeof(unsigned);
    if (s.work) b += 2 * sizeof(unsigned);
    if (s.counters) b += s.seg_cap * (sizeof(unsigned) + sizeof(Consts)) + (s.seg_cap + 1) * sizeof(int64_t);
    return b;
}

}  // namespace ipa

extern "C" ipa_status ipa_model_init(ipa_model* m, int32_t kind, double t_lo, double t_hi) {
    if (!m) {
        ipa::set_error("model is NULL");
        return IPA_ERR_ARG;
    }
    if (kind != IPA_MODEL_TIME1D && kind != IPA_MODEL_ANGTIME4D && kind != IPA_MODEL_TAGGED1D &&
        kind != IPA_MODEL_PHIS) {
        ipa::set_error("unknown model kind %d", kind);
        return IPA_ERR_ARG;
    }
    if (!(t_lo < t_hi)) {
        ipa::set_error("empty decay-time range [%g, %g]", t_lo, t_hi);
        return IPA_ERR_ARG;
    }
    m->kind = kind;
    m->n_par = ipa::npar_of(kind);
    m->t_lo = t_lo;
    m->t_hi = t_hi;
    return IPA_OK;
}

extern "C" ipa_status ipa_reserve(int64_t max_events, int32_t max_segments) {
    if (max_events < 0 || max_segments < 1) {
        ipa::set_error("ipa_reserve: bad sizes");
        return IPA_ERR_ARG;
    }
    ipa::Scratch* sc = nullptr;
    return ipa::scratch_get((max_events + ipa::kTile - 1) / ipa::kTile + max_segments,
                            (int64_t)max_segments + 1, &sc);
}

extern "C" ipa_status ipa_scratch_bytes(uint64_t* bytes) {
    if (!bytes) {
        ipa::set_error("ipa_scratch_bytes: bytes is NULL");
        return IPA_ERR_ARG;
    }
    int dev = 0;
    ipa_status st = ipa::cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != IPA_OK) return st;
    *bytes = ipa::scratch_bytes(dev);
    return IPA_OK;
}

extern "C" uint32_t ipa_fault_inject(uint32_t mask) {
    return ipa::g_fault.exchange(mask & (IPA_FAULT_ALLOC | IPA_FAULT_SUBMIT | IPA_FAULT_ADMIT));
}

extern "C" const char* ipa_last_error(void) { return ipa::g_err; }

extern "C" const char* ipa_version(void) { return "ipanema-gb300 0.1 (sm_103a)"; }
