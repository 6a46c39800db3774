// Hot-path step a8: batched minimisation (Sec. 3-4: MIGRAD to the minimum,
// HESSE for the errors), all fits advancing together on the device.
//
// Every fit is a small state machine advanced by one thread of `qn_kernel`
// after each segmented NLL+gradient pass over all active fits:
//
//   INIT   first evaluation at the start point; H^-1 = diag(step^2).
//   LS     BFGS line search: Armijo backtracking along d = -H^-1 g (projected
//          onto the limits); on acceptance the BFGS update of H^-1 (skipped when
//          y.s <= 0), with Shanno-Phua scaling before the first update.  When
//          the Newton decrement sqrt(g.H^-1.g) (the step in units of the
//          parameter errors) drops below kSwitch, the fit moves to HESS.
//   HESS   the Hessian by central finite differences of the analytic gradient,
//          two gradient passes per free parameter (one-sided near a limit).
//   NEWTON Newton steps with that Hessian until the decrement is below `tol`.
//   DONE   errors = sqrt(diag H^-1), i.e. Delta NLL = 1/2 (Sec. 3).
//
// The host replays a CUDA graph of K passes [tile map -> constants -> NLL+grad
// -> state update] until every fit is DONE; fits that are done drop out of the
// tile map, so stragglers do not pay for the whole batch.
#include <math.h>
#include <string.h>

#include <vector>

#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr int kMaxP = 10;          // parameters of the largest model
constexpr double kSwitch = 1e-3;   // BFGS -> finite-difference Newton (decrement, sigma units)
constexpr double kRehess = 2e-3;   // Newton moved further than this (sigma units): Hessian again
constexpr int kGraphSteps = 8;     // passes per graph replay
enum Phase { kInit = 0, kLS = 1, kHess = 2, kNewton = 3, kDone = 4 };

struct Spec {
    int n_par, n_free;
    int free_idx[kMaxP];
    double lo[kMaxP], hi[kMaxP], step[kMaxP];
    double tol;
    int max_iter, max_passes;
};

struct State {
    double theta[kMaxP];      // current point (all parameters)
    double g[kMaxP];          // gradient at theta (free components)
    double Hinv[kMaxP * kMaxP];
    double H[kMaxP * kMaxP];  // finite-difference Hessian (rows filled during HESS)
    double d[kMaxP];          // search direction (free components)
    double s_prev[kMaxP];     // step of the current trial (free components)
    double h[kMaxP];          // finite-difference steps
    double ga[kMaxP];         // gradient at the first stencil point of the current column
    double theta_h[kMaxP];    // point where H was taken (free components)
    double f, gd, alpha;
    int phase, iter, passes, hess_j, newton, status, scaled, onesided, rehess;
};

__device__ inline double clampd(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

// Cholesky solve of the n x n SPD matrix A (row-major, leading dim kMaxP):
// writes A^-1 into inv.  Returns false if A is not positive definite.
__device__ bool spd_inverse(const double* A, int n, double* inv) {
    double L[kMaxP * kMaxP];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * kMaxP + j];
            for (int k = 0; k < j; ++k) s -= L[i * kMaxP + k] * L[j * kMaxP + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * kMaxP + i] = sqrt(s);
            } else {
                L[i * kMaxP + j] = s / L[j * kMaxP + j];
            }
        }
    }
    // inv = L^-T L^-1, column by column
    for (int c = 0; c < n; ++c) {
        double y[kMaxP];
        for (int i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * kMaxP + k] * y[k];
            y[i] = s / L[i * kMaxP + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < n; ++k) s -= L[k * kMaxP + i] * inv[k * kMaxP + c];
            inv[i * kMaxP + c] = s / L[i * kMaxP + i];
        }
    }
    return true;
}

__device__ inline bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return false;
    return true;
}

// Set theta_eval = theta + alpha d (projected) and remember the step.
__device__ void set_trial(const Spec& sp, State& S, double alpha, double* theta_eval) {
    for (int p = 0; p < sp.n_par; ++p) theta_eval[p] = S.theta[p];
    for (int a = 0; a < sp.n_free; ++a) {
        const int p = sp.free_idx[a];
        const double v = clampd(S.theta[p] + alpha * S.d[a], sp.lo[p], sp.hi[p]);
        theta_eval[p] = v;
        S.s_prev[a] = v - S.theta[p];
    }
}

// Stencil point of Hessian column j/2: central (+h, -h), or one-sided (+h, +2h)
// when theta - h would leave the limits.
__device__ void set_hess_point(const Spec& sp, State& S, double* theta_eval) {
    for (int p = 0; p < sp.n_par; ++p) theta_eval[p] = S.theta[p];
    const int a = S.hess_j >> 1, second = S.hess_j & 1;
    const int p = sp.free_idx[a];
    const double h = S.h[a];
    double x;
    if (!S.onesided) x = second ? S.theta[p] - h : S.theta[p] + h;
    else x = second ? S.theta[p] + 2.0 * h : S.theta[p] + h;
    theta_eval[p] = x;
}

__device__ void start_hess(const Spec& sp, State& S, double* theta_eval) {
    S.phase = kHess;
    S.hess_j = 0;
    for (int a = 0; a < sp.n_free; ++a) S.theta_h[a] = S.theta[sp.free_idx[a]];
    for (int a = 0; a < sp.n_free; ++a) {
        const int p = sp.free_idx[a];
        double h = 2e-3 * sqrt(fmax(S.Hinv[a * kMaxP + a], 0.0));
        const double floor_h = 1e-7 * (fabs(S.theta[p]) + 1e-3);
        if (!(h > floor_h)) h = floor_h;
        const double room = sp.hi[p] - sp.lo[p];
        if (h > 0.05 * room) h = 0.05 * room;
        S.h[a] = h;
    }
    {
        const int p = sp.free_idx[0];
        S.onesided = (S.theta[p] - S.h[0] < sp.lo[p]) ? 1 : 0;
    }
    set_hess_point(sp, S, theta_eval);
}

__device__ void finish(const Spec& sp, State& S, int status) {
    S.phase = kDone;
    if (status == IPA_FIT_CONVERGED) {
        for (int a = 0; a < sp.n_free; ++a) {
            const int p = sp.free_idx[a];
            const double tol_lim = 1e-9 * (sp.hi[p] - sp.lo[p]);
            if (S.theta[p] <= sp.lo[p] + tol_lim || S.theta[p] >= sp.hi[p] - tol_lim)
                status = IPA_FIT_AT_LIMIT;
        }
    }
    S.status = status;
}

// New BFGS direction from (theta, g, Hinv); start a line search or switch to HESS.
__device__ void new_direction(const Spec& sp, State& S, double* theta_eval) {
    const int n = sp.n_free;
    double gd = 0.0;
    for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s -= S.Hinv[a * kMaxP + b] * S.g[b];
        S.d[a] = s;
        gd += S.g[a] * s;
    }
    if (!(gd < 0.0)) {   // lost positive definiteness: restart from the diagonal
        for (int a = 0; a < n * kMaxP; ++a) S.Hinv[a] = 0.0;
        gd = 0.0;
        for (int a = 0; a < n; ++a) {
            const double s2 = sp.step[sp.free_idx[a]] * sp.step[sp.free_idx[a]];
            S.Hinv[a * kMaxP + a] = s2;
            S.d[a] = -s2 * S.g[a];
            gd += S.g[a] * S.d[a];
        }
        S.scaled = 0;
    }
    const double dec = sqrt(fmax(0.0, -gd));
    if (dec < kSwitch || S.iter >= sp.max_iter) {
        start_hess(sp, S, theta_eval);
        return;
    }
    S.phase = kLS;
    S.alpha = 1.0;
    set_trial(sp, S, 1.0, theta_eval);
}

__device__ void newton_step(const Spec& sp, State& S, double* theta_eval) {
    const int n = sp.n_free;
    double gd = 0.0;
    for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s -= S.Hinv[a * kMaxP + b] * S.g[b];
        S.d[a] = s;
        gd += S.g[a] * s;
    }
    const double dec = sqrt(fmax(0.0, -gd));
    if (dec < sp.tol) {
        // errors come from H: take it again if Newton moved away from where it was taken
        double disp2 = 0.0;
        for (int a = 0; a < n; ++a) {
            const double da = S.theta[sp.free_idx[a]] - S.theta_h[a];
            for (int b = 0; b < n; ++b) {
                const double db = S.theta[sp.free_idx[b]] - S.theta_h[b];
                disp2 += da * 0.5 * (S.H[a * kMaxP + b] + S.H[b * kMaxP + a]) * db;
            }
        }
        if (!S.rehess && disp2 > kRehess * kRehess) {
            S.rehess = 1;
            start_hess(sp, S, theta_eval);
            return;
        }
        finish(sp, S, IPA_FIT_CONVERGED);
        return;
    }
    if (S.newton >= 8 || S.iter >= sp.max_iter) {
        finish(sp, S, IPA_FIT_MAXITER);
        return;
    }
    S.phase = kNewton;
    S.alpha = 1.0;
    S.gd = gd;
    set_trial(sp, S, 1.0, theta_eval);
}

__global__ void qn_kernel(Spec sp, int n_fits, const int64_t* __restrict__ seg_off,
                          const double* __restrict__ res, State* __restrict__ states,
                          double* __restrict__ theta_eval_all, int* __restrict__ active,
                          int* __restrict__ n_active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fits) return;
    if (!active[i]) return;
    State& S = states[i];
    const int n = sp.n_free, P = sp.n_par;
    const double* r = res + (size_t)i * (1 + P);
    double* theta_eval = theta_eval_all + (size_t)i * P;
    const double fe = r[0];
    double ge[kMaxP];
    for (int a = 0; a < n; ++a) ge[a] = r[1 + sp.free_idx[a]];
    const bool ok = isfinite(fe) && finite_all(ge, n);
    S.passes += 1;

    switch (S.phase) {
    case kInit: {
        if (seg_off[i + 1] <= seg_off[i]) {
            S.f = 0.0;
            finish(sp, S, IPA_FIT_EMPTY);
            break;
        }
        if (!ok) {
            S.f = fe;
            finish(sp, S, IPA_FIT_BAD_PDF);
            break;
        }
        S.f = fe;
        for (int a = 0; a < n; ++a) S.g[a] = ge[a];
        for (int a = 0; a < kMaxP * kMaxP; ++a) S.Hinv[a] = 0.0;
        for (int a = 0; a < n; ++a) {
            const double st = sp.step[sp.free_idx[a]];
            S.Hinv[a * kMaxP + a] = st * st;
        }
        new_direction(sp, S, theta_eval);
        break;
    }
    case kLS: {
        double gs = 0.0;
        for (int a = 0; a < n; ++a) gs += S.g[a] * S.s_prev[a];
        if (ok && fe <= S.f + 1e-4 * gs) {
            double y[kMaxP], s[kMaxP], ys = 0.0, yy = 0.0;
            for (int a = 0; a < n; ++a) {
                y[a] = ge[a] - S.g[a];
                s[a] = S.s_prev[a];
                ys += y[a] * s[a];
                yy += y[a] * y[a];
            }
            if (ys > 1e-300) {
                if (!S.scaled) {   // Shanno-Phua: scale the initial matrix by y.s / y.H.y
                    double yHy = 0.0;
                    for (int a = 0; a < n; ++a)
                        for (int b = 0; b < n; ++b) yHy += y[a] * S.Hinv[a * kMaxP + b] * y[b];
                    if (yHy > 0.0) {
                        const double sc = ys / yHy;
                        for (int a = 0; a < n * kMaxP; ++a) S.Hinv[a] *= sc;
                    }
                    S.scaled = 1;
                }
                // H+ = (I - rho s y^T) H (I - rho y s^T) + rho s s^T
                const double rho = 1.0 / ys;
                double Hy[kMaxP], yHy = 0.0;
                for (int a = 0; a < n; ++a) {
                    double v = 0.0;
                    for (int b = 0; b < n; ++b) v += S.Hinv[a * kMaxP + b] * y[b];
                    Hy[a] = v;
                    yHy += y[a] * v;
                }
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b)
                        S.Hinv[a * kMaxP + b] += -rho * (Hy[a] * s[b] + s[a] * Hy[b]) +
                                                 (rho * rho * yHy + rho) * s[a] * s[b];
            }
            for (int a = 0; a < n; ++a) {
                S.theta[sp.free_idx[a]] += s[a];
                S.g[a] = ge[a];
            }
            S.f = fe;
            S.iter += 1;
            new_direction(sp, S, theta_eval);
        } else {
            S.alpha *= 0.25;
            if (S.alpha < 1e-8) {
                start_hess(sp, S, theta_eval);   // no progress along d: polish with Newton
            } else {
                set_trial(sp, S, S.alpha, theta_eval);
            }
        }
        break;
    }
    case kHess: {
        if (!ok) {
            finish(sp, S, IPA_FIT_BAD_PDF);
            break;
        }
        const int a = S.hess_j >> 1;
        if ((S.hess_j & 1) == 0) {
            for (int b = 0; b < n; ++b) S.ga[b] = ge[b];
        } else {
            const double h = S.h[a];
            for (int b = 0; b < n; ++b) {
                S.H[a * kMaxP + b] = S.onesided ? (-3.0 * S.g[b] + 4.0 * S.ga[b] - ge[b]) / (2.0 * h)
                                                : (S.ga[b] - ge[b]) / (2.0 * h);
            }
        }
        S.hess_j += 1;
        if (S.hess_j < 2 * n) {
            if ((S.hess_j & 1) == 0) {
                const int p = sp.free_idx[S.hess_j >> 1];
                S.onesided = (S.theta[p] - S.h[S.hess_j >> 1] < sp.lo[p]) ? 1 : 0;
            }
            set_hess_point(sp, S, theta_eval);
            break;
        }
        // symmetrise, invert (shifting if not positive definite), then Newton
        double Hs[kMaxP * kMaxP];
        for (int x = 0; x < n; ++x)
            for (int z = 0; z < n; ++z)
                Hs[x * kMaxP + z] = 0.5 * (S.H[x * kMaxP + z] + S.H[z * kMaxP + x]);
        double inv[kMaxP * kMaxP];
        bool pd = spd_inverse(Hs, n, inv);
        double shift = 0.0;
        double dmax = 0.0;
        for (int x = 0; x < n; ++x) dmax = fmax(dmax, fabs(Hs[x * kMaxP + x]));
        for (int k = 0; k < 40 && !pd; ++k) {
            shift = shift == 0.0 ? 1e-10 * dmax : shift * 4.0;
            double Ht[kMaxP * kMaxP];
            for (int x = 0; x < n * kMaxP; ++x) Ht[x] = Hs[x];
            for (int x = 0; x < n; ++x) Ht[x * kMaxP + x] += shift;
            pd = spd_inverse(Ht, n, inv);
        }
        if (!pd) {
            finish(sp, S, IPA_FIT_BAD_PDF);
            break;
        }
        for (int x = 0; x < n * kMaxP; ++x) S.Hinv[x] = inv[x];
        S.newton = 0;
        newton_step(sp, S, theta_eval);   // f and g at theta are those of the last accepted step
        break;
    }
    case kNewton: {
        double gs = 0.0;
        for (int a = 0; a < n; ++a) gs += S.g[a] * S.s_prev[a];
        // accept a decrease, or an increase within rounding of the NLL near the minimum
        if (ok && (fe <= S.f + 1e-4 * gs || fe <= S.f + 1e-13 * fabs(S.f))) {
            for (int a = 0; a < n; ++a) {
                S.theta[sp.free_idx[a]] += S.s_prev[a];
                S.g[a] = ge[a];
            }
            S.f = fe;
            S.newton += 1;
            S.iter += 1;
            newton_step(sp, S, theta_eval);
        } else {
            S.alpha *= 0.5;
            if (S.alpha < 1e-6) {
                finish(sp, S, IPA_FIT_CONVERGED);   // at the rounding floor of the NLL
            } else {
                set_trial(sp, S, S.alpha, theta_eval);
            }
        }
        break;
    }
    default:
        break;
    }
    if (S.phase != kDone && S.passes >= sp.max_passes) finish(sp, S, IPA_FIT_MAXITER);
    if (S.phase == kDone) {
        active[i] = 0;
        for (int p = 0; p < P; ++p) theta_eval[p] = S.theta[p];
    } else {
        atomicAdd(n_active, 1);
    }
}

__global__ void init_kernel(Spec sp, int n_fits, const double* __restrict__ theta_io,
                            State* __restrict__ states, double* __restrict__ theta_eval,
                            int* __restrict__ active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fits) return;
    State& S = states[i];
    for (int p = 0; p < sp.n_par; ++p) {
        double v = theta_io[(size_t)i * sp.n_par + p];
        bool is_free = false;
        for (int a = 0; a < sp.n_free; ++a) is_free |= sp.free_idx[a] == p;
        if (is_free) v = clampd(v, sp.lo[p], sp.hi[p]);
        S.theta[p] = v;
        theta_eval[(size_t)i * sp.n_par + p] = v;
    }
    S.phase = kInit;
    S.iter = S.passes = S.hess_j = S.newton = 0;
    S.status = IPA_FIT_MAXITER;
    S.scaled = 0;
    S.onesided = 0;
    S.rehess = 0;
    S.f = 0.0;
    active[i] = 1;
}

__global__ void final_kernel(Spec sp, int n_fits, const State* __restrict__ states,
                             double* __restrict__ theta_io, double* __restrict__ err,
                             double* __restrict__ nll, int32_t* __restrict__ status,
                             int32_t* __restrict__ iters, int32_t* __restrict__ passes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fits) return;
    const State& S = states[i];
    for (int p = 0; p < sp.n_par; ++p) {
        theta_io[(size_t)i * sp.n_par + p] = S.theta[p];
        if (err) err[(size_t)i * sp.n_par + p] = 0.0;
    }
    if (err) {
        for (int a = 0; a < sp.n_free; ++a)
            err[(size_t)i * sp.n_par + sp.free_idx[a]] = sqrt(fmax(S.Hinv[a * kMaxP + a], 0.0));
    }
    if (nll) nll[i] = S.f;
    if (status) status[i] = S.phase == kDone ? S.status : IPA_FIT_MAXITER;
    if (iters) iters[i] = S.iter;
    if (passes) passes[i] = S.passes;
}

// Active-masked tile map: inactive fits get no tiles.
__global__ void masked_tiles_kernel(const int64_t* __restrict__ seg_off, const int* __restrict__ active,
                                    int n_seg, int64_t n, int64_t* __restrict__ seg_tiles) {
    __shared__ int64_t run[1024];
    const int nt = blockDim.x;
    const int per = (n_seg + nt - 1) / nt;
    const int b = threadIdx.x * per;
    const int e = min(n_seg, b + per);
    auto tiles = [&](int s) -> int64_t {
        if (!active[s]) return 0;
        int64_t lo = seg_off[s], hi = seg_off[s + 1];
        lo = lo < 0 ? 0 : (lo > n ? n : lo);
        hi = hi < lo ? lo : (hi > n ? n : hi);
        return (hi - lo + kTile - 1) / kTile;
    };
    int64_t sum = 0;
    for (int s = b; s < e; ++s) sum += tiles(s);
    run[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        const int64_t v = threadIdx.x >= d ? run[threadIdx.x - d] : 0;
        __syncthreads();
        run[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t acc = threadIdx.x ? run[threadIdx.x - 1] : 0;
    for (int s = b; s < e; ++s) {
        seg_tiles[s] = acc;
        acc += tiles(s);
    }
    if (threadIdx.x == nt - 1) seg_tiles[n_seg] = run[nt - 1];
}

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
    sp.n_par = model->n_par;
    sp.tol = tol;
    sp.max_iter = max_iter;
    for (int p = 0; p < sp.n_par; ++p) {
        if (!(spec[p].lo <= spec[p].value && spec[p].value <= spec[p].hi) && !spec[p].fixed) {
            set_error("ipa_fit_batch: start value of parameter %d outside its limits", p);
            return IPA_ERR_ARG;
        }
        sp.lo[p] = spec[p].lo;
        sp.hi[p] = spec[p].hi;
        double step = spec[p].step;
        if (!(step > 0.0)) step = (isfinite(spec[p].hi - spec[p].lo) && spec[p].hi > spec[p].lo)
                                      ? 0.1 * (spec[p].hi - spec[p].lo) : 0.1 * (fabs(spec[p].value) + 1.0);
        sp.step[p] = step;
        if (!spec[p].fixed) sp.free_idx[sp.n_free++] = p;
    }
    if (sp.n_free == 0) {
        set_error("ipa_fit_batch: no free parameter");
        return IPA_ERR_ARG;
    }
    sp.max_passes = 6 * max_iter + 4 * sp.n_free + 40;

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

    DevBuf b_state, b_eval, b_res, b_active, b_nact;
    if ((st = cuda_fail(cudaMalloc(&b_state.p, sizeof(State) * (size_t)n_fits), "fit state")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_eval.p, sizeof(double) * (size_t)n_fits * P), "fit theta")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_res.p, sizeof(double) * (size_t)n_fits * (1 + P)), "fit results")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_active.p, sizeof(int) * (size_t)n_fits), "fit mask")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMalloc(&b_nact.p, sizeof(int) * kGraphSteps), "fit count")) != IPA_OK) return st;
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
    init_kernel<<<fg, fb, 0, s>>>(sp, n_fits, theta_io_dev, states, theta_eval, active);
    if ((st = cuda_fail(cudaGetLastError(), "fit init")) != IPA_OK) return done(st);

    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w};
    // one pass = tile map, constants, segmented NLL+grad, state update
    auto pass = [&](int k) -> ipa_status {
        ipa_status q;
        masked_tiles_kernel<<<1, 1024, 0, s>>>(seg_off_dev, active, n_fits, ev->n, sc->seg_tiles);
        if ((q = cuda_fail(cudaGetLastError(), "fit tile map")) != IPA_OK) return q;
        if ((q = launch_consts(m, theta_eval, n_fits, sc->consts, s)) != IPA_OK) return q;
        if ((q = launch_nll(m, true, cols, ev->n, seg_off_dev, sc->seg_tiles, n_fits, sc->consts, sc,
                            res, s)) != IPA_OK)
            return q;
        if ((q = cuda_fail(cudaMemsetAsync(n_active + k, 0, sizeof(int), s), "fit count reset")) != IPA_OK)
            return q;
        qn_kernel<<<fg, fb, 0, s>>>(sp, n_fits, seg_off_dev, res, states, theta_eval, active, n_active + k);
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
    final_kernel<<<fg, fb, 0, s>>>(sp, n_fits, states, theta_io_dev, err_out_dev, nll_out_dev,
                                   fit_status_dev, iters_out_dev, passes_out_dev);
    st = cuda_fail(cudaGetLastError(), "fit final");
    st = done(st);
    if (st == IPA_OK) st = cuda_fail(cudaGetLastError(), "fit final sync");
    // later work on the caller's stream sees the results: the call is blocking
    return st;
}
