// Internal declarations shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ipanema.h"

namespace ipa {

// Events per reduction tile.  Lane l of the warp that owns a tile adds events
// l, l+32, ... of the tile in order; the warp reduces its lanes with a fixed
// butterfly into one partial per tile, each group of kGroupTiles tiles is
// reduced (lane l holding tile l of the group) into one group partial, and a
// segment's group partials are added in a fixed order.  This order depends
// only on the segment's events, not on the launch geometry (block size, grid,
// tiles taken at once), so tuning the geometry never changes a result.
#ifndef IPA_TILE_EVENTS
#define IPA_TILE_EVENTS 512
#endif
constexpr int kTile = IPA_TILE_EVENTS;
constexpr int kGroupTiles = 32;
constexpr int kBlock = 256;   // threads per block of the generator and helper kernels

// Parameters of a model kind.
__host__ __device__ constexpr int npar_of(int kind) {
    return kind == IPA_MODEL_TIME1D ? IPA_NPAR_1D
           : kind == IPA_MODEL_TAGGED1D ? IPA_NPAR_TAGGED
           : kind == IPA_MODEL_PHIS ? IPA_NPAR_PHIS : IPA_NPAR_4D;
}

// Number of FP64 accumulators per tile.
//   NLL only:      L = sum w log P
//   1D + grad:     L, Q = sum w/P, S = sum (w/P) T, D_Gamma, D_sigma, D_mu
//   4D + grad:     L, Q, S_1..S_10 = sum (w/P) T f_k, D_Gamma, D_sigma, D_mu
//   tagged + grad: 13 (tagged.cu);  phi_s + grad: 47 (phis.cu)
__host__ __device__ constexpr int n_acc(int kind, bool grad) {
    return !grad ? 1
                 : (kind == IPA_MODEL_TIME1D ? 6
                    : kind == IPA_MODEL_TAGGED1D ? 13 : kind == IPA_MODEL_PHIS ? 47 : 15);
}
// Doubles per tile that the partials buffers of the library scratch hold (the
// largest n_acc); the server's and the no-allocation scratch hold
// kSmallAcc per tile and serve only the models that need no more.
constexpr int kMaxAcc = 47;
constexpr int kSmallAcc = 15;

// Parameter-derived constants of one fit (step a1 of the hot path), computed
// once per call on the device from theta and read by every event tile.
struct Consts {
    double Gamma, sigma, mu, fb;
    double c_exp;     // Gamma^2 sigma^2 / 2
    double Gs2;       // Gamma sigma^2
    double k_z;       // 1 / (sqrt2 sigma)   (erfc argument scale)
    double k_g;       // 1 / (2 sigma^2)     (Gaussian exponent scale)
    double cG;        // 1 / (sqrt(2 pi) sigma)
    double s2;        // sigma^2
    double G2s;       // Gamma^2 sigma
    double Gsig;      // Gamma sigma
    double inv_s;     // 1 / sigma
    double cs;        // (1 - f_b) / (I_T I_Omega)
    double cb;        // f_b / V
    double inv_ITIO;  // 1 / (I_T I_Omega)
    double inv_V;     // 1 / V
    double dlnIT[3];  // (dI_T / dtheta_j) / I_T for Gamma, sigma, mu
    double h[10];     // amplitude coefficients h_k (4D), h[0] = 1 for 1D
    double dh[10][6]; // dh_k / d(A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S)
    double MT;        // time envelope: max of g(t - mu) on [t_lo, t_hi] (upper bound)
    double MO;        // angular envelope: sum |h_k| max|f_k|
    double IT;        // I_T
    double pad_;
};
constexpr int kConstsDoubles = sizeof(Consts) / sizeof(double);
static_assert(sizeof(Consts) % 16 == 0, "Consts must be a multiple of 16 bytes");

// Model description passed by value to kernels.
struct ModelDev {
    int kind;
    int n_par;
    double t_lo, t_hi;
};

struct Cols {
    const double *t, *ck, *cl, *phi, *w;
    const double* fk = nullptr;   // cached angular basis (10 columns) or nullptr
    int64_t fk_stride = 0;
    const double* q = nullptr;    // flavour tag (tagged model)
};

// ---- host-side helpers (runtime.cu) ----
void set_error(const char* fmt, ...);
// Append one line to the IPA_TRACE file (if the variable is set).
void trace(const char* fmt, ...);
ipa_status cuda_fail(cudaError_t e, const char* what);
// Host-side fault injection (ipa_fault_inject): whether `bit` is set.
bool fault(uint32_t bit);
// cudaMalloc, or IPA_ERR_OOM without calling it while IPA_FAULT_ALLOC is set.
ipa_status device_alloc(void** p, size_t bytes, const char* what);
ipa_status check_model(const ipa_model* m);
ipa_status check_events(const ipa_model* m, const ipa_events* ev);

// Per-device scratch shared by the likelihood, generator and fitter kernels.
struct Scratch {
    double* partials = nullptr;     // tiles * n_acc doubles
    size_t partials_cap = 0;        // doubles
    unsigned* counters = nullptr;   // one per segment, zero between calls
    unsigned* gcount = nullptr;     // one per tile (used at a group's first tile), zero between calls
    unsigned* work = nullptr;       // [tiles taken, warps finished], zero between calls
    int64_t* seg_tiles = nullptr;   // n_seg + 1 prefix of tiles per segment
    Consts* consts = nullptr;       // one per segment
    size_t seg_cap = 0;             // segments
};
// Ensure the current device's scratch holds `tiles` tiles of 15 accumulators
// (and their group counters) and `segs` segments.  May synchronise the device
// when it grows.
ipa_status scratch_get(int64_t tiles, int64_t segs, Scratch** out);
// Device bytes that scratch_get has allocated on device `dev`.
uint64_t scratch_bytes(int dev);

// ---- kernels launched across translation units ----
// consts.cu: theta (n_seg x n_par) -> Consts[n_seg]
ipa_status launch_consts(const ModelDev& m, const double* theta, int n_seg, Consts* out,
                         cudaStream_t s);
// tagged.cu: the same for the tagged model (a TagConsts record in each slot)
ipa_status launch_tag_consts(const ModelDev& m, const double* theta, int n_seg, Consts* out, cudaStream_t s);

// Launch geometry of the likelihood kernel (tune.cu picks it; no result
// depends on it).
struct LaunchCfg {
    int warps_per_block;   // 1, 2, 4 or 8
    int warps_per_sm;      // resident warps wanted per SM; 0 = ceil(work units / SMs)
    int tiles_per_take;    // tiles a warp takes from the work counter at once: 1, 2 or 4
};
// Host estimate of a launch's tile count (selects the size class only): exact
// for one segment, ceil(n / kTile) + n_seg / 2 for several.
inline int64_t tile_estimate(int64_t n, int n_seg) {
    return (n + kTile - 1) / kTile + (n_seg > 1 ? n_seg / 2 : 0);
}
// Configuration for a launch over about `tiles` tiles (table entry of the
// autotuner for this kernel variant and size, else the built-in default).
LaunchCfg launch_cfg(int kind, bool grad, bool cached, bool segmented, int64_t tiles);
// Blocks of a likelihood launch: cfg's resident warps per SM (or one tile take
// per warp, ceil(takes / SMs)) in blocks of W warps, capped by `per_sm` resident
// blocks per SM, and for one segment by the blocks that find a tile (tiles
// taken K at a time).
int64_t launch_grid(const LaunchCfg& cfg, int W, int K, int per_sm, int64_t tiles, bool single);
// Incremented whenever a table entry changes (cached CUDA graphs that hold a
// likelihood launch compare it to know when to re-capture).
unsigned tune_epoch();

// nll.cu: NLL(+grad) over precomputed consts; out: (1 + n_par) per segment (1 without
// the gradient).  With seg_begin == nullptr there is one segment [0, n).  Otherwise
// segment s is events [seg_begin[s], seg_end[s]) and seg_tiles must hold the device
// prefix of its tiles (launch_seg_tiles).  The geometry is launch_cfg's for
// tile_estimate(n, n_seg) tiles and n_seg > 1, unless `cfg` forces one.
ipa_status launch_nll(const ModelDev& m, bool grad, const Cols& cols, int64_t n,
                      const int64_t* seg_begin, const int64_t* seg_end, const int64_t* seg_tiles, int n_seg,
                      const Consts* consts, Scratch* sc, double* out, cudaStream_t s,
                      const LaunchCfg* cfg = nullptr);
// phis.cu: constants and launch_nll of the phi_s model
ipa_status launch_phis_consts(const ModelDev& m, const double* theta, int n_seg, Consts* out, cudaStream_t s);
ipa_status launch_phis_nll(const ModelDev& m, bool grad, const Cols& cols, int64_t n,
                           const int64_t* seg_begin, const int64_t* seg_end, const int64_t* seg_tiles, int n_seg,
                           const Consts* consts, Scratch* sc, double* out, cudaStream_t s, const LaunchCfg* cfg);
// tagged.cu: launch_nll for the tagged model
ipa_status launch_tag_nll(const ModelDev& m, bool grad, const Cols& cols, int64_t n,
                          const int64_t* seg_begin, const int64_t* seg_end, const int64_t* seg_tiles, int n_seg,
                          const Consts* consts, Scratch* sc, double* out, cudaStream_t s, const LaunchCfg* cfg);
// toygen.cu / tagged.cu: the tagged model's generator over consts[0]
ipa_status launch_tag_toygen(const ModelDev& m, const Consts* consts, uint64_t seed, int n_toys,
                             const int64_t* n_sig, const int64_t* n_bkg, const int64_t* offsets,
                             const ipa_event_buffers* out, cudaStream_t s);
// phis.cu: the phi_s model's generator (a PhisConsts record in consts[0])
ipa_status launch_phis_toygen(const ModelDev& m, const Consts* consts, uint64_t seed, int n_toys,
                              const int64_t* n_sig, const int64_t* n_bkg, const int64_t* offsets,
                              const ipa_event_buffers* out, cudaStream_t s);
// nll.cu: seg_tiles[s] = sum_{r<s} ceil(size_r / kTile), s = 0..n_seg, with the
// ranges clamped to [0, n]; segments with active[r] == 0 get no tiles (active may
// be NULL).
ipa_status launch_seg_tiles(const int64_t* seg_begin, const int64_t* seg_end, const int* active, int n_seg,
                            int64_t n, int64_t* seg_tiles, cudaStream_t s);

// tagged.cu / phis.cu: the last reduction level and the gradient contraction
// over gathered group partials (ipa_nll_grad_combine), one warp.
ipa_status launch_tag_combine(const double* groups, int64_t n_groups, const Consts* consts, int n_par, double* out,
                              cudaStream_t s);
ipa_status launch_phis_combine(const double* groups, int64_t n_groups, bool cached, const Consts* consts, int n_par,
                               double* out, cudaStream_t s);

// Number of SMs of the current device (cached).
int sm_count();

}  // namespace ipa
