// ipa_nll_grad_noalloc: the NLL + gradient pass of ipa_nll_grad with its
// scratch (tile partials, completion and group counters and the parameter constants)
// in a fixed array compiled into this library instead of memory the library
// allocates.  It exists for callers that cannot allocate device memory when
// they call: code that must not trigger an allocation (and the device
// synchronisation that freeing or growing a buffer implies) inside a
// latency-critical loop, and hosts whose framework allocator has already
// reserved the GPU's memory so that a cudaMalloc from a plugin fails.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (about 2 MB) until the process exits.  Host code may not
// use its name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress while that device is current, and
// later calls reuse it.  That first call should therefore come before any
// stream capture.  The address belongs to the device's current CUDA context:
// each call compares the context's unique id with the one the address was
// looked up in and looks it up again after a device reset (a new primary
// context reloads the library's device code, and the array with it).  All calls share the one array and it keeps the previous
// call's contents: the completion, group and work counters are cleared on the stream
// before every launch, and calls that overlap on the GPU (different streams, or
// different host threads without ordering) race on the array.
#include <cuda.h>

#include <mutex>

#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr int64_t kNoAllocMaxEvents = IPA_NOALLOC_MAX_EVENTS;
constexpr int64_t kNoAllocMaxTiles = kNoAllocMaxEvents / kTile + 1;
constexpr size_t kConstsBytes = 1024;     // one Consts record, padded
constexpr size_t kCounterBytes = 256;     // completion counter and the two work counters, padded
constexpr size_t kGroupBytes = ((size_t)kNoAllocMaxTiles * sizeof(unsigned) + 255) / 256 * 256;  // group counters
constexpr size_t kPartialsBytes = (size_t)kNoAllocMaxTiles * kSmallAcc * sizeof(double);
static_assert(sizeof(Consts) <= kConstsBytes, "Consts must fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kConstsBytes + kCounterBytes + kGroupBytes + kPartialsBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (cuCtxGetId, reached
// through the runtime's driver entry points, so that the library needs no
// link-time dependency on the driver library); 0 when it cannot be read.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the array on the current device: looked up once per
// device and context.  A thread whose context is not yet current reads id 0
// and looks the address up (which makes the context current); the id read
// after the lookup is the one kept.
ipa_status noalloc_base(unsigned char** base) {
    int dev = 0;
    ipa_status st = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != IPA_OK) return st;
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("ipa_nll_grad_noalloc: device ordinal %d not supported", dev);
        return IPA_ERR_ARG;
    }
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev] || ctx == 0 || g_noalloc_ctx[dev] != ctx) {
        void* p = nullptr;
        if ((st = cuda_fail(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress")) != IPA_OK)
            return st;
        g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
        g_noalloc_ctx[dev] = current_context_id();
    }
    *base = g_noalloc_addr[dev];
    return IPA_OK;
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_nll_grad_noalloc(const ipa_model* model, const ipa_events* ev,
                                           const double* theta_dev, double* out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if (!theta_dev || !out_dev) {
        set_error("theta and out must be device pointers");
        return IPA_ERR_ARG;
    }
    if (n_acc(model->kind, true) > kSmallAcc) {
        set_error("ipa_nll_grad_noalloc: the phi_s model needs more scratch per tile than the fixed "
                  "array holds (use ipa_nll_grad)");
        return IPA_ERR_ARG;
    }
    if (ev->n > kNoAllocMaxEvents) {
        set_error("ipa_nll_grad_noalloc: %lld events exceed the fixed scratch of %lld events "
                  "(use ipa_nll_grad)", (long long)ev->n, (long long)kNoAllocMaxEvents);
        return IPA_ERR_ARG;
    }
    unsigned char* base = nullptr;
    if ((st = noalloc_base(&base)) != IPA_OK) return st;
    Scratch sc;
    sc.consts = reinterpret_cast<Consts*>(base);
    sc.counters = reinterpret_cast<unsigned*>(base + kConstsBytes);
    sc.work = sc.counters + 1;
    sc.gcount = reinterpret_cast<unsigned*>(base + kConstsBytes + kCounterBytes);
    sc.partials = reinterpret_cast<double*>(base + kConstsBytes + kCounterBytes + kGroupBytes);
    sc.partials_cap = (size_t)kNoAllocMaxTiles * kSmallAcc;
    sc.seg_cap = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = cuda_fail(cudaMemsetAsync(sc.counters, 0, 3 * sizeof(unsigned), s), "counter clear")) != IPA_OK)
        return st;
    // group counters sit at each group's first tile: tiles 0, 32, 64, ...
    const int64_t used = (ev->n + kTile - 1) / kTile;
    if (used > 0 &&
        (st = cuda_fail(cudaMemsetAsync(sc.gcount, 0, (size_t)used * sizeof(unsigned), s), "counter clear")) != IPA_OK)
        return st;
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_consts(m, theta_dev, 1, sc.consts, s)) != IPA_OK) return st;
    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride, ev->q};
    return launch_nll(m, true, cols, ev->n, nullptr, nullptr, nullptr, 1, sc.consts, &sc, out_dev, s);
}
