// Hot-path step a8 (shared by the batch fitter and the fit server): batched minimisation (Sec. 3-4: MIGRAD to the minimum,
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
#pragma once

#include <math.h>

#include "ipa_internal.cuh"

namespace ipa {

constexpr int kMaxP = 32;          // parameters of a fit (IPA_MAX_PAR; joint fits over categories)
constexpr double kSwitch = 1e-3;   // BFGS -> finite-difference Newton (decrement, sigma units)
constexpr double kRehess = 2e-3;   // Newton moved further than this (sigma units): Hessian again
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
    double H[kMaxP * kMaxP];  // finite-difference Hessian (rows filled during HESS, then symmetrised)
    double W[kMaxP * kMaxP];  // Cholesky factor (work space of spd_inverse)
    double d[kMaxP];          // search direction (free components)
    double s_prev[kMaxP];     // step of the current trial (free components)
    double h[kMaxP];          // finite-difference steps
    double ga[kMaxP];         // gradient at the first stencil point of the current column
    double theta_h[kMaxP];    // point where H was taken (free components)
    double f, gd, alpha;
    int phase, iter, passes, hess_j, newton, status, scaled, onesided, rehess;
};

// A simultaneous fit over categories (ipa_fit_joint): category c of fit i is
// segment i * n_cat + c; category c evaluates the model at theta_c[p] =
// theta_J[map[c][p]] (map >= 0) or value[c][p].  Device arrays; theta_seg,
// res_seg and seg_active are work buffers of n_fits * n_cat segments.
struct JointDev {
    int n_cat = 0, n_model = 0, n_joint = 0;
    const int32_t* map = nullptr;       // n_cat x n_model
    const double* value = nullptr;      // n_cat x n_model
    const int64_t* seg_begin = nullptr; // n_fits * n_cat
    const int64_t* seg_end = nullptr;
    double* theta_seg = nullptr;        // n_fits * n_cat x n_model
    double* res_seg = nullptr;          // n_fits * n_cat x (1 + n_model)
    int* seg_active = nullptr;          // n_fits * n_cat
    bool grad = true;                   // false: NLL only (res_seg and the sums one double per entry)
};

// joint.cu: theta_seg (and seg_active = active[fit], or 1 without a mask) from
// the joint parameters theta_joint (n_fits x n_joint); res_joint (n_fits x
// (1 + n_joint)) from res_seg in the fixed order (c ascending, p ascending),
// for the active fits (every fit without a mask).
ipa_status launch_joint_scatter(const JointDev& j, int n_fits, const double* theta_joint, const int* active,
                                cudaStream_t s);
ipa_status launch_joint_gather(const JointDev& j, int n_fits, const int* active, double* res_joint,
                               cudaStream_t s);
// joint.cu: host checks of a category map (IPA_ERR_ARG with the reason).
ipa_status check_joint(const ipa_model* m, const ipa_joint* j, int n_fits);

// fit.cu: run n_fits fits to the end.  Fit i minimises the NLL of events
// [begin[i], end[i]) with specs[i * spec_stride] (device arrays the caller
// keeps unchanged until the call returns; ranges may overlap, e.g. several
// fits of the same events with different fixed parameters), starting at
// theta_io[i] (n_par values, device) and writing the result back there;
// err, nll, status, iters, passes as in ipa_fit_batch (device, may be NULL).
// tiles_bound >= the sum over fits of their 512-event tiles.  Ordered after
// the caller's `stream`; blocks until the fits end.  `who` names the call in
// the IPA_TRACE record.  With `joint`, fit i is a simultaneous fit over its
// categories (its parameters the joint ones; [begin[i], end[i]) then only
// decides whether the fit is empty) and tiles_bound covers all the segments.
ipa_status fit_run(const ipa_model* model, const ipa_events* ev, int n_fits, const int64_t* begin,
                   const int64_t* end, const Spec* specs, int spec_stride, int max_passes, int64_t tiles_bound,
                   double* theta_io, double* err, double* nll, int32_t* status, int32_t* iters, int32_t* passes,
                   cudaStream_t stream, const char* who, const JointDev* joint = nullptr);

namespace {

__device__ inline double clampd(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

// A specification the kernels may index with (slots that were never given a
// fit hold zeros: no parameters, nothing to do).
__device__ inline bool spec_ok(const Spec& sp) {
    if (sp.n_par < 1 || sp.n_par > kMaxP || sp.n_free < 1 || sp.n_free > sp.n_par) return false;
    for (int a = 0; a < sp.n_free; ++a)
        if (sp.free_idx[a] < 0 || sp.free_idx[a] >= sp.n_par) return false;
    return true;
}

// Cholesky solve of the n x n SPD matrix A + shift I (row-major, leading dim
// kMaxP): writes (A + shift I)^-1 into inv, with the factor in L (n x kMaxP,
// work space the caller provides, so that no kMaxP^2 array sits in local
// memory).  Returns false if the matrix is not positive definite.
__device__ bool spd_inverse(const double* A, int n, double shift, double* inv, double* L) {
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = i == j ? A[i * kMaxP + j] + shift : A[i * kMaxP + j];
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

// Advance fit i by one pass: res holds (NLL, gradient) at theta_eval of fit i.
// Fit i uses specs[i * spec_stride] and events [seg_begin[i], seg_end[i])
// (seg_begin NULL: the caller evaluated the points itself, no fit is empty).
__global__ void qn_kernel(const Spec* __restrict__ specs, int spec_stride, int n_fits,
                          const int64_t* __restrict__ seg_begin, const int64_t* __restrict__ seg_end,
                          const double* __restrict__ res, State* __restrict__ states,
                          double* __restrict__ theta_eval_all, int* __restrict__ active,
                          int* __restrict__ n_active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fits) return;
    if (!active[i]) return;
    const Spec& sp = specs[(size_t)i * spec_stride];
    if (!spec_ok(sp)) return;
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
        if (seg_begin && seg_end[i] <= seg_begin[i]) {
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
        // symmetrise in place, invert (shifting the diagonal if not positive
        // definite) into Hinv, then Newton
        for (int x = 0; x < n; ++x)
            for (int z = x + 1; z < n; ++z) {
                const double v = 0.5 * (S.H[x * kMaxP + z] + S.H[z * kMaxP + x]);
                S.H[x * kMaxP + z] = v;
                S.H[z * kMaxP + x] = v;
            }
        bool pd = spd_inverse(S.H, n, 0.0, S.Hinv, S.W);
        double shift = 0.0;
        double dmax = 0.0;
        for (int x = 0; x < n; ++x) dmax = fmax(dmax, fabs(S.H[x * kMaxP + x]));
        for (int k = 0; k < 40 && !pd; ++k) {
            shift = shift == 0.0 ? 1e-10 * dmax : shift * 4.0;
            pd = spd_inverse(S.H, n, shift, S.Hinv, S.W);
        }
        if (!pd) {
            finish(sp, S, IPA_FIT_BAD_PDF);
            break;
        }
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

// Start fit i at theta_io[i] (free parameters clamped into their limits).
__global__ void init_kernel(const Spec* __restrict__ specs, int spec_stride, int n_fits,
                            const double* __restrict__ theta_io, State* __restrict__ states,
                            double* __restrict__ theta_eval, int* __restrict__ active) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fits) return;
    const Spec& sp = specs[(size_t)i * spec_stride];
    if (!spec_ok(sp)) return;
    State& S = states[i];
    // every field starts at zero: fits that end before their first Hessian
    // (empty, non-physical) report zero errors
    double* raw = reinterpret_cast<double*>(&S);
    for (size_t k = 0; k < sizeof(State) / sizeof(double); ++k) raw[k] = 0.0;
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

// Results of fit i: theta, errors sqrt(diag H^-1) (0 for fixed parameters),
// NLL, status, iterations, passes; NULL outputs are skipped.
__global__ void final_kernel(const Spec* __restrict__ specs, int spec_stride, int n_fits,
                             const State* __restrict__ states, double* __restrict__ theta_io,
                             double* __restrict__ err, double* __restrict__ nll,
                             int32_t* __restrict__ status, int32_t* __restrict__ iters,
                             int32_t* __restrict__ passes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fits) return;
    const Spec& sp = specs[(size_t)i * spec_stride];
    if (!spec_ok(sp)) return;
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

// Host: the minimiser specification from the parameter array (Parameter /
// Free of App. B): limits, steps (0 -> a tenth of the range, or of |value|+1),
// the free-parameter list, tolerance and budgets.  n_par: the parameters of a
// fit (0: the model's; a joint fit's n_joint otherwise).
inline ipa_status build_spec(const ipa_model* model, const ipa_param* spec, int max_iter, double tol,
                             Spec* out, int n_par = 0) {
    Spec sp{};
    sp.n_par = n_par > 0 ? n_par : model->n_par;
    sp.tol = tol;
    sp.max_iter = max_iter;
    for (int p = 0; p < sp.n_par; ++p) {
        if (!(spec[p].lo <= spec[p].value && spec[p].value <= spec[p].hi) && !spec[p].fixed) {
            set_error("start value of parameter %d outside its limits", p);
            return IPA_ERR_ARG;
        }
        sp.lo[p] = spec[p].lo;
        sp.hi[p] = spec[p].hi;
        double step = spec[p].step;
        if (!(step > 0.0))
            step = (isfinite(spec[p].hi - spec[p].lo) && spec[p].hi > spec[p].lo)
                       ? 0.1 * (spec[p].hi - spec[p].lo) : 0.1 * (fabs(spec[p].value) + 1.0);
        sp.step[p] = step;
        if (!spec[p].fixed) sp.free_idx[sp.n_free++] = p;
    }
    if (sp.n_free == 0) {
        set_error("no free parameter");
        return IPA_ERR_ARG;
    }
    sp.max_passes = 6 * max_iter + 4 * sp.n_free + 40;
    *out = sp;
    return IPA_OK;
}

}  // namespace
}  // namespace ipa
