// Error analysis after the fit, on the device: HESSE (the covariance and the
// correlation matrix from the Hessian of the NLL) and MINOS (the profile-
// likelihood interval of each parameter).  Sec. 3 and Sec. 4 report the
// MIGRAD minimum, the HESSE errors and the correlation matrix of each fit; the
// MINOS interval is where the NLL, minimised over every other free parameter,
// rises by `up` (1/2 for the FCN = -log L) above the minimum.
//
// Both are batched the way the fitter is: the unit of work is a "virtual
// segment", an event range with its own parameters, and many virtual segments
// may cover the same events.
//   HESSE: per fit, 1 + 2 n_free segments over the fit's events (the centre
//   and the two stencil points of each free parameter) in one segmented
//   NLL+gradient launch; the Hessian by central differences of the analytic
//   gradient (one-sided at a limit), twice: steps of 1e-3 of the parameter
//   step, then 2e-3 of the errors that gives (the fitter's own rule).
//   MINOS: per fit, scanned parameter and side, a probe: a constrained fit with
//   the parameter fixed at x.  All probes of all fits are fitted together by
//   the batched minimiser (fit_run), then every probe moves x by a secant step
//   on s(x) = sqrt(2 (NLL_profile(x) - NLL_min)) toward sqrt(2 up), until
//   |NLL_profile - NLL_min - up| < tol.  A round costs one batched fit of all
//   probes; converged probes drop out (empty event ranges).
#include <math.h>
#include <string.h>

#include <mutex>

#include "fitcore.cuh"
#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr int kHesseBlock = 128;

// Stencil of free parameter a of a fit at theta with step h: one-sided (+h,
// +2h) when theta - h leaves the lower limit, central (+h, -h) otherwise.
__device__ inline bool hesse_onesided(const Spec& sp, const double* theta, const double* h, int a) {
    const int p = sp.free_idx[a];
    return theta[p] - h[a] < sp.lo[p];
}

// Virtual segment v = f (1 + 2 n_free) + k of fit f: k = 0 the centre, k = 1 + 2a
// and 2 + 2a the two stencil points of free parameter a.
__global__ void hesse_points_kernel(const Spec* __restrict__ spp, int n_fits, const int64_t* __restrict__ seg_off,
                                    const double* __restrict__ theta, const double* __restrict__ h,
                                    int64_t* __restrict__ vbegin, int64_t* __restrict__ vend,
                                    double* __restrict__ vtheta) {
    const Spec& sp = *spp;
    const int nv = 1 + 2 * sp.n_free, P = sp.n_par;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_fits * nv) return;
    const int f = v / nv, k = v % nv;
    const double* th = theta + (size_t)f * P;
    double* out = vtheta + (size_t)v * P;
    for (int p = 0; p < P; ++p) out[p] = th[p];
    if (k > 0) {
        const int a = (k - 1) >> 1, second = (k - 1) & 1;
        const double* hf = h + (size_t)f * kMaxP;
        const int p = sp.free_idx[a];
        const bool one = hesse_onesided(sp, th, hf, a);
        out[p] = one ? th[p] + (second ? 2.0 : 1.0) * hf[a] : th[p] + (second ? -hf[a] : hf[a]);
    }
    if (seg_off) {      // (simultaneous fits take their categories' ranges instead)
        vbegin[v] = seg_off[f];
        vend[v] = seg_off[f + 1];
    }
}

__global__ void hesse_first_steps_kernel(const Spec* __restrict__ spp, int n_fits, double* __restrict__ h) {
    const Spec& sp = *spp;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_fits) return;
    for (int a = 0; a < sp.n_free; ++a) h[(size_t)f * kMaxP + a] = 1e-3 * sp.step[sp.free_idx[a]];
}

// Simultaneous fits: category c of virtual point v (of fit v / nv) reads the
// events of that fit's category c.
__global__ void hesse_joint_ranges_kernel(const int64_t* __restrict__ seg_off, int n_v, int nv, int n_cat,
                                          int64_t* __restrict__ jbegin, int64_t* __restrict__ jend) {
    const int64_t vs = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vs >= (int64_t)n_v * n_cat) return;
    const int64_t v = vs / n_cat, c = vs - v * n_cat, f = v / nv;
    jbegin[vs] = seg_off[f * n_cat + c];
    jend[vs] = seg_off[f * n_cat + c + 1];
}

// The Hessian of fit f from its virtual segments' gradients; stage 0 sets the
// steps of stage 1 from the errors, stage 1 writes the outputs.
// work: 3 kMaxP^2 doubles per fit (inverse, Cholesky factor, Hessian).
__global__ void hesse_assemble_kernel(const Spec* __restrict__ spp, int n_fits, const double* __restrict__ theta,
                                      double* __restrict__ h, const double* __restrict__ vres, int stage,
                                      double* __restrict__ work, double* __restrict__ cov,
                                      double* __restrict__ corr, double* __restrict__ err,
                                      int32_t* __restrict__ status) {
    const Spec& sp = *spp;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_fits) return;
    const int n = sp.n_free, P = sp.n_par, nv = 1 + 2 * n;
    const double* th = theta + (size_t)f * P;
    double* hf = h + (size_t)f * kMaxP;
    const double* rc = vres + (size_t)f * nv * (1 + P);
    double* H = work + (size_t)n_fits * 2 * kMaxP * kMaxP + (size_t)f * kMaxP * kMaxP;
    bool finite = true;
    for (int a = 0; a < n; ++a) {
        const double* r1 = rc + (size_t)(1 + 2 * a) * (1 + P);
        const double* r2 = rc + (size_t)(2 + 2 * a) * (1 + P);
        const bool one = hesse_onesided(sp, th, hf, a);
        for (int b = 0; b < n; ++b) {
            const int q = 1 + sp.free_idx[b];
            H[a * kMaxP + b] = one ? (-3.0 * rc[q] + 4.0 * r1[q] - r2[q]) / (2.0 * hf[a])
                                   : (r1[q] - r2[q]) / (2.0 * hf[a]);
            finite &= isfinite(H[a * kMaxP + b]);
        }
    }
    double* Hs = H;                                   // symmetrised in place
    double* inv = work + (size_t)f * 2 * kMaxP * kMaxP;
    double* L = inv + kMaxP * kMaxP;
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            const double v = 0.5 * (H[a * kMaxP + b] + H[b * kMaxP + a]);
            H[a * kMaxP + b] = v;
            H[b * kMaxP + a] = v;
        }
    bool pd = finite && spd_inverse(Hs, n, 0.0, inv, L);
    int st = 0;
    if (finite && !pd) {
        // not positive definite: shift the diagonal until it is (status 1)
        double dmax = 0.0, shift = 0.0;
        for (int a = 0; a < n; ++a) dmax = fmax(dmax, fabs(Hs[a * kMaxP + a]));
        for (int k = 0; k < 40 && !pd; ++k) {
            shift = shift == 0.0 ? 1e-10 * dmax : shift * 4.0;
            pd = spd_inverse(Hs, n, shift, inv, L);
        }
        st = 1;
    }
    if (!pd) st = 3;
    if (stage == 0) {
        for (int a = 0; a < n; ++a) {
            const int p = sp.free_idx[a];
            double hn = pd ? 2e-3 * sqrt(fmax(inv[a * kMaxP + a], 0.0)) : hf[a];
            const double floor_h = 1e-7 * (fabs(th[p]) + 1e-3);
            if (!(hn > floor_h)) hn = floor_h;
            const double room = sp.hi[p] - sp.lo[p];
            if (hn > 0.05 * room) hn = 0.05 * room;
            hf[a] = hn;
        }
        return;
    }
    double* C = cov + (size_t)f * P * P;
    for (int x = 0; x < P * P; ++x) C[x] = 0.0;
    if (corr) for (int x = 0; x < P * P; ++x) corr[(size_t)f * P * P + x] = 0.0;
    if (err) for (int p = 0; p < P; ++p) err[(size_t)f * P + p] = 0.0;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int a = 0; a < n; ++a) {
        const int p = sp.free_idx[a];
        for (int b = 0; b < n; ++b) C[p * P + sp.free_idx[b]] = pd ? inv[a * kMaxP + b] : nan;
    }
    for (int a = 0; a < n; ++a) {
        const int p = sp.free_idx[a];
        const double sa = sqrt(fmax(C[p * P + p], 0.0));
        if (err) err[(size_t)f * P + p] = pd ? sa : nan;
        if (corr) {
            for (int b = 0; b < n; ++b) {
                const int q = sp.free_idx[b];
                const double sb = sqrt(fmax(C[q * P + q], 0.0));
                corr[(size_t)f * P * P + p * P + q] = pd ? C[p * P + q] / (sa * sb) : nan;
            }
        }
    }
    if (status) status[f] = st;
}

// ---- MINOS ----

struct Probe {
    double x, s;          // current abscissa and s(x) = sqrt(2 dNLL) (valid after a round)
    double xp, sp;        // previous point
    double result;        // the interval end (valid when done)
    int round, done, status, have_prev;
};

// Probe p = (f * n_scan + k) * 2 + side of fit f, scanned parameter scan[k].
__device__ inline void probe_ids(int p, int n_scan, int* f, int* k, int* side) {
    *side = p & 1;
    *k = (p >> 1) % n_scan;
    *f = (p >> 1) / n_scan;
}

__global__ void minos_init_kernel(const Spec* __restrict__ spp, const int* __restrict__ scan, int n_scan,
                                  int n_probes, const double* __restrict__ theta_min, const double* __restrict__ cov,
                                  Probe* __restrict__ probes) {
    const Spec& sp = *spp;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_probes) return;
    int f, k, side;
    probe_ids(p, n_scan, &f, &k, &side);
    const int j = scan[k], P = sp.n_par;
    const double c = theta_min[(size_t)f * P + j];
    const double sj = sqrt(fmax(cov[(size_t)f * P * P + j * P + j], 0.0));
    Probe q{};
    q.x = fmin(fmax(c + (side ? sj : -sj), sp.lo[j]), sp.hi[j]);
    q.status = IPA_MINOS_MAXROUNDS;
    if (!(sj > 0.0) || !isfinite(sj)) {
        q.done = 1;
        q.status = IPA_MINOS_FIT_FAILED;
        q.result = c;
    }
    probes[p] = q;
}

// The constrained fits of this round: the spec without the scanned parameter,
// the start point theta_min + C[., j] / C_jj (x - theta_min_j) (the
// conditional mean of the Gaussian approximation, clamped into the limits),
// the fit's event range, or an empty range for a probe that is done.
__global__ void minos_prepare_kernel(const Spec* __restrict__ spp, const int* __restrict__ scan, int n_scan,
                                     int n_probes, const int64_t* __restrict__ seg_off, int n_cat,
                                     const double* __restrict__ theta_min, const double* __restrict__ cov,
                                     const Probe* __restrict__ probes, Spec* __restrict__ pspecs,
                                     int64_t* __restrict__ pbegin, int64_t* __restrict__ pend,
                                     double* __restrict__ ptheta, int64_t* __restrict__ jbegin,
                                     int64_t* __restrict__ jend) {
    const Spec& sp = *spp;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_probes) return;
    int f, k, side;
    probe_ids(p, n_scan, &f, &k, &side);
    const int j = scan[k], P = sp.n_par;
    const Probe& q = probes[p];
    Spec cs = sp;
    cs.n_free = 0;
    for (int a = 0; a < sp.n_free; ++a)
        if (sp.free_idx[a] != j) cs.free_idx[cs.n_free++] = sp.free_idx[a];
    for (int a = cs.n_free; a < kMaxP; ++a) cs.free_idx[a] = 0;
    cs.max_passes = 6 * sp.max_iter + 4 * cs.n_free + 40;
    pspecs[p] = cs;
    const double* tm = theta_min + (size_t)f * P;
    const double* C = cov + (size_t)f * P * P;
    double* th = ptheta + (size_t)p * P;
    const double cjj = C[j * P + j];
    for (int r = 0; r < P; ++r) {
        double v = tm[r];
        if (r != j && cjj > 0.0 && isfinite(cjj)) v += C[r * P + j] / cjj * (q.x - tm[j]);
        th[r] = fmin(fmax(v, sp.lo[r]), sp.hi[r]);
    }
    th[j] = q.x;
    // the fit's events (simultaneous fits: all its categories, and each
    // category's range for the category pass)
    pbegin[p] = q.done ? 0 : seg_off[(int64_t)f * n_cat];
    pend[p] = q.done ? 0 : seg_off[(int64_t)(f + 1) * n_cat];
    if (jbegin) {
        for (int c = 0; c < n_cat; ++c) {
            jbegin[(int64_t)p * n_cat + c] = q.done ? 0 : seg_off[(int64_t)f * n_cat + c];
            jend[(int64_t)p * n_cat + c] = q.done ? 0 : seg_off[(int64_t)f * n_cat + c + 1];
        }
    }
}

// Move every probe that is not done: with d = NLL_profile(x) - NLL_min and
// s = sqrt(2 d), converged when |d - up| < tol; otherwise a secant step on s
// toward T = sqrt(2 up) (through the previous point, or through the minimum
// where s = 0 on the first round or when the secant points the wrong way),
// the distance from the minimum kept within [1/4, 4] times the current one.
__global__ void minos_update_kernel(const Spec* __restrict__ spp, const int* __restrict__ scan, int n_scan,
                                    int n_probes, const double* __restrict__ theta_min,
                                    const double* __restrict__ nll_min, const double* __restrict__ pnll,
                                    const int32_t* __restrict__ pstatus, double up, double tol, int max_rounds,
                                    Probe* __restrict__ probes, int* __restrict__ n_open) {
    const Spec& sp = *spp;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_probes) return;
    Probe& q = probes[p];
    if (q.done) return;
    int f, k, side;
    probe_ids(p, n_scan, &f, &k, &side);
    const int j = scan[k], P = sp.n_par;
    const double c = theta_min[(size_t)f * P + j];
    const double limit = side ? sp.hi[j] : sp.lo[j];
    const double d = pnll[p] - nll_min[f];
    q.round += 1;
    const int fs = pstatus ? pstatus[p] : IPA_FIT_CONVERGED;
    if (!isfinite(d) || fs == IPA_FIT_BAD_PDF || fs == IPA_FIT_EMPTY) {
        q.done = 1;
        q.status = IPA_MINOS_FIT_FAILED;
        q.result = q.x;
        return;
    }
    if (d < -tol) {           // a lower NLL than the minimum: the fit was not at the minimum
        q.done = 1;
        q.status = IPA_MINOS_NEW_MINIMUM;
        q.result = q.x;
        return;
    }
    if (fabs(d - up) < tol) {
        q.done = 1;
        q.status = IPA_MINOS_OK;
        q.result = q.x;
        return;
    }
    if (d < up && q.x == limit) {  // the profile stays below the threshold up to the limit
        q.done = 1;
        q.status = IPA_MINOS_AT_LIMIT;
        q.result = q.x;
        return;
    }
    if (q.round >= max_rounds) {
        q.done = 1;
        q.status = IPA_MINOS_MAXROUNDS;
        q.result = q.x;
        return;
    }
    const double T = sqrt(2.0 * up);
    const double s = sqrt(2.0 * fmax(d, 0.0));
    const double dist = q.x - c;
    double xn;
    bool secant = false;
    if (q.have_prev && s != q.sp) {
        xn = q.x + (T - s) * (q.x - q.xp) / (s - q.sp);
        secant = (xn - c) * dist > 0.0;
    }
    if (!secant) xn = s > 0.0 ? c + dist * (T / s) : c + 2.0 * dist;
    double dn = xn - c;
    if (fabs(dn) > 4.0 * fabs(dist)) dn = 4.0 * dist;
    if (fabs(dn) < 0.25 * fabs(dist)) dn = 0.25 * dist;
    q.xp = q.x;
    q.sp = s;
    q.have_prev = 1;
    q.x = fmin(fmax(c + dn, sp.lo[j]), sp.hi[j]);
    atomicAdd(n_open, 1);
}

__global__ void minos_final_kernel(const Spec* __restrict__ spp, const int* __restrict__ scan, int n_scan,
                                   int n_fits, const double* __restrict__ theta_min,
                                   const Probe* __restrict__ probes, double* __restrict__ lo_out,
                                   double* __restrict__ hi_out, int32_t* __restrict__ status_out) {
    const Spec& sp = *spp;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_fits) return;
    const int P = sp.n_par;
    for (int r = 0; r < P; ++r) {
        lo_out[(size_t)f * P + r] = 0.0;
        hi_out[(size_t)f * P + r] = 0.0;
        if (status_out) status_out[((size_t)f * P + r) * 2] = status_out[((size_t)f * P + r) * 2 + 1] =
                            IPA_MINOS_NOT_SCANNED;
    }
    for (int k = 0; k < n_scan; ++k) {
        const int j = scan[k];
        const double c = theta_min[(size_t)f * P + j];
        for (int side = 0; side < 2; ++side) {
            const Probe& q = probes[(f * n_scan + k) * 2 + side];
            (side ? hi_out : lo_out)[(size_t)f * P + j] = q.result - c;
            if (status_out) status_out[((size_t)f * P + j) * 2 + side] = q.status;
        }
    }
}

// Per-device buffers of HESSE and MINOS (grow-only; one call at a time).
struct ProfileContext {
    std::mutex mu;
    Spec* spec = nullptr;
    int* scan = nullptr;
    int* n_open = nullptr;
    int* h_open = nullptr;
    // HESSE
    double* h = nullptr;
    double* hwork = nullptr;        // 3 kMaxP^2 per fit (hesse_assemble_kernel)
    int64_t *vbegin = nullptr, *vend = nullptr;
    double *vtheta = nullptr, *vres = nullptr;
    size_t cap_fit = 0, cap_v = 0;
    // HESSE of simultaneous fits: the categories of every virtual point
    int32_t* jmap = nullptr;
    double* jvalue = nullptr;
    int64_t *jbegin = nullptr, *jend = nullptr;
    double *jtheta = nullptr, *jres = nullptr;
    int* jactive = nullptr;
    size_t cap_jmap = 0, cap_jseg = 0;
    // MINOS
    Probe* probes = nullptr;
    Spec* pspecs = nullptr;
    int64_t *pbegin = nullptr, *pend = nullptr;
    double *ptheta = nullptr, *pnll = nullptr;
    int32_t* pstatus = nullptr;
    size_t cap_p = 0;
};

ProfileContext* profile_context() {
    static ProfileContext ctx[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    return &ctx[dev];
}

template <typename T>
ipa_status grow(T** p, size_t n, const char* what) {
    cudaFree(*p);
    *p = nullptr;
    return device_alloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1), what);
}

ipa_status profile_basics(ProfileContext& c) {
    ipa_status st = IPA_OK;
    if (!c.spec) st = device_alloc((void**)&c.spec, sizeof(Spec), "profile spec");
    if (st == IPA_OK && !c.scan) st = device_alloc((void**)&c.scan, sizeof(int) * kMaxP, "profile scan list");
    if (st == IPA_OK && !c.n_open) st = device_alloc((void**)&c.n_open, sizeof(int), "profile counter");
    if (st == IPA_OK && !c.h_open) st = cuda_fail(cudaMallocHost(&c.h_open, sizeof(int)), "profile counter");
    return st;
}

ipa_status hesse_reserve(ProfileContext& c, size_t n_fits, size_t n_v, int P) {
    ipa_status st = IPA_OK;
    if (n_fits > c.cap_fit) {
        cudaDeviceSynchronize();
        st = grow(&c.h, n_fits * kMaxP, "hesse steps");
        if (st == IPA_OK) st = grow(&c.hwork, n_fits * 3 * kMaxP * kMaxP, "hesse work");
        if (st == IPA_OK) c.cap_fit = n_fits;
    }
    if (st == IPA_OK && n_v > c.cap_v) {
        cudaDeviceSynchronize();
        c.cap_v = 0;
        st = grow(&c.vbegin, n_v, "hesse segments");
        if (st == IPA_OK) st = grow(&c.vend, n_v, "hesse segments");
        if (st == IPA_OK) st = grow(&c.vtheta, n_v * kMaxP, "hesse points");
        if (st == IPA_OK) st = grow(&c.vres, n_v * (1 + kMaxP), "hesse gradients");
        if (st == IPA_OK) c.cap_v = n_v;
    }
    (void)P;
    return st;
}

ipa_status joint_reserve(ProfileContext& c, size_t map_n, size_t n_seg) {
    ipa_status st = IPA_OK;
    if (map_n > c.cap_jmap) {
        cudaDeviceSynchronize();
        c.cap_jmap = 0;
        st = grow(&c.jmap, map_n, "hesse joint map");
        if (st == IPA_OK) st = grow(&c.jvalue, map_n, "hesse joint values");
        if (st == IPA_OK) c.cap_jmap = map_n;
    }
    if (st == IPA_OK && n_seg > c.cap_jseg) {
        cudaDeviceSynchronize();
        c.cap_jseg = 0;
        st = grow(&c.jbegin, n_seg, "hesse joint segments");
        if (st == IPA_OK) st = grow(&c.jend, n_seg, "hesse joint segments");
        if (st == IPA_OK) st = grow(&c.jtheta, n_seg * kMaxP, "hesse joint category points");
        if (st == IPA_OK) st = grow(&c.jres, n_seg * (1 + kMaxP), "hesse joint category results");
        if (st == IPA_OK) st = grow(&c.jactive, n_seg, "hesse joint category mask");
        if (st == IPA_OK) c.cap_jseg = n_seg;
    }
    return st;
}

ipa_status minos_reserve(ProfileContext& c, size_t n_p) {
    if (n_p <= c.cap_p) return IPA_OK;
    cudaDeviceSynchronize();
    c.cap_p = 0;
    ipa_status st = grow(&c.probes, n_p, "minos probes");
    if (st == IPA_OK) st = grow(&c.pspecs, n_p, "minos specs");
    if (st == IPA_OK) st = grow(&c.pbegin, n_p, "minos segments");
    if (st == IPA_OK) st = grow(&c.pend, n_p, "minos segments");
    if (st == IPA_OK) st = grow(&c.ptheta, n_p * kMaxP, "minos points");
    if (st == IPA_OK) st = grow(&c.pnll, n_p * (1 + kMaxP), "minos results");
    if (st == IPA_OK) st = grow(&c.pstatus, n_p, "minos statuses");
    if (st == IPA_OK) c.cap_p = n_p;
    return st;
}

ipa_status check_common(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off, int n_fits,
                        const ipa_param* spec, const char* who) {
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if (n_fits < 1 || !seg_off || !spec) {
        set_error("%s: bad arguments", who);
        return IPA_ERR_ARG;
    }
    return IPA_OK;
}

// One segmented NLL(+gradient) launch over n_v virtual segments.
ipa_status virtual_pass(const ipa_model* model, const ipa_events* ev, int n_v, const int64_t* vbegin,
                        const int64_t* vend, const double* vtheta, int64_t tiles_bound, bool grad, double* out,
                        cudaStream_t s) {
    Scratch* sc = nullptr;
    ipa_status st = scratch_get(tiles_bound, n_v + 1, &sc);
    if (st != IPA_OK) return st;
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_seg_tiles(vbegin, vend, nullptr, n_v, ev->n, sc->seg_tiles, s)) != IPA_OK) return st;
    if ((st = launch_consts(m, vtheta, n_v, sc->consts, s)) != IPA_OK) return st;
    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride, ev->q};
    return launch_nll(m, grad, cols, ev->n, vbegin, vend, sc->seg_tiles, n_v, sc->consts, sc, out, s);
}

// The same for n_v points of simultaneous fits: every point's categories
// (theta_J -> theta_c, NLL+gradient per category, fixed-order sums per point).
ipa_status virtual_pass_joint(const ipa_model* model, const ipa_events* ev, const JointDev& jd, int n_v,
                              const double* vtheta, int64_t tiles_bound, double* out, cudaStream_t s) {
    const int n_seg = n_v * jd.n_cat;
    Scratch* sc = nullptr;
    ipa_status st = scratch_get(tiles_bound, n_seg + 1, &sc);
    if (st != IPA_OK) return st;
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_joint_scatter(jd, n_v, vtheta, nullptr, s)) != IPA_OK) return st;
    if ((st = launch_seg_tiles(jd.seg_begin, jd.seg_end, nullptr, n_seg, ev->n, sc->seg_tiles, s)) != IPA_OK)
        return st;
    if ((st = launch_consts(m, jd.theta_seg, n_seg, sc->consts, s)) != IPA_OK) return st;
    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride, ev->q};
    if ((st = launch_nll(m, jd.grad, cols, ev->n, jd.seg_begin, jd.seg_end, sc->seg_tiles, n_seg, sc->consts, sc,
                         jd.res_seg, s)) != IPA_OK)
        return st;
    return launch_joint_gather(jd, n_v, nullptr, out, s);
}

}  // namespace
}  // namespace ipa

namespace ipa {
namespace {

// HESSE of n_fits fits (joint: simultaneous fits over categories, P = n_joint).
ipa_status hesse_run(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev, int32_t n_fits,
                     const Spec& sp, const double* theta_dev, double* cov_out_dev, double* corr_out_dev,
                     double* err_out_dev, int32_t* status_out_dev, cudaStream_t s, const ipa_joint* joint,
                     const char* who) {
    ProfileContext* cp = profile_context();
    if (!cp) return IPA_ERR_CUDA;
    ProfileContext& c = *cp;
    std::lock_guard<std::mutex> lk(c.mu);
    const int nv = 1 + 2 * sp.n_free;
    const size_t n_v = (size_t)n_fits * nv;
    const int n_cat = joint ? joint->n_cat : 1;
    ipa_status st;
    if (n_v * (size_t)n_cat > (size_t)1 << 30) {
        set_error("%s: %zu virtual segments, more than 2^30", who, n_v * (size_t)n_cat);
        return IPA_ERR_ARG;
    }
    if ((st = profile_basics(c)) != IPA_OK) return st;
    if ((st = hesse_reserve(c, (size_t)n_fits, n_v, model->n_par)) != IPA_OK) return st;
    if (joint && (st = joint_reserve(c, (size_t)n_cat * model->n_par, n_v * n_cat)) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMemcpyAsync(c.spec, &sp, sizeof(Spec), cudaMemcpyHostToDevice, s), "hesse spec copy")) !=
        IPA_OK)
        return st;
    JointDev jd;
    if (joint) {
        const size_t mn = (size_t)n_cat * model->n_par;
        st = cuda_fail(cudaMemcpyAsync(c.jmap, joint->map, mn * sizeof(int32_t), cudaMemcpyHostToDevice, s),
                       "hesse joint map copy");
        if (st == IPA_OK)
            st = joint->value ? cuda_fail(cudaMemcpyAsync(c.jvalue, joint->value, mn * sizeof(double),
                                                          cudaMemcpyHostToDevice, s), "hesse joint values copy")
                              : cuda_fail(cudaMemsetAsync(c.jvalue, 0, mn * sizeof(double), s), "hesse joint values");
        if (st != IPA_OK) return st;
        const int64_t nj = (int64_t)n_v * n_cat;
        hesse_joint_ranges_kernel<<<(unsigned)((nj + kHesseBlock - 1) / kHesseBlock), kHesseBlock, 0, s>>>(
            seg_off_dev, (int)n_v, nv, n_cat, c.jbegin, c.jend);
        if ((st = cuda_fail(cudaGetLastError(), "hesse joint ranges")) != IPA_OK) return st;
        jd.n_cat = n_cat;
        jd.n_model = model->n_par;
        jd.n_joint = joint->n_joint;
        jd.map = c.jmap;
        jd.value = c.jvalue;
        jd.seg_begin = c.jbegin;
        jd.seg_end = c.jend;
        jd.theta_seg = c.jtheta;
        jd.res_seg = c.jres;
        jd.seg_active = c.jactive;
    }
    const int64_t tiles = (int64_t)nv * ((ev->n + kTile - 1) / kTile + (int64_t)n_fits * n_cat);
    const int gf = (n_fits + kHesseBlock - 1) / kHesseBlock, gv = (int)((n_v + kHesseBlock - 1) / kHesseBlock);
    hesse_first_steps_kernel<<<gf, kHesseBlock, 0, s>>>(c.spec, n_fits, c.h);
    // (joint: the points' event ranges are the categories', set above; the
    // per-fit ranges the points kernel writes are not used)
    const int64_t* fit_off = seg_off_dev;
    for (int stage = 0; stage < 2 && st == IPA_OK; ++stage) {
        hesse_points_kernel<<<gv, kHesseBlock, 0, s>>>(c.spec, n_fits, joint ? nullptr : fit_off, theta_dev, c.h,
                                                       c.vbegin, c.vend, c.vtheta);
        if ((st = cuda_fail(cudaGetLastError(), "hesse points")) != IPA_OK) break;
        if (joint) {
            st = virtual_pass_joint(model, ev, jd, (int)n_v, c.vtheta, tiles, c.vres, s);
        } else {
            st = virtual_pass(model, ev, (int)n_v, c.vbegin, c.vend, c.vtheta, tiles, true, c.vres, s);
        }
        if (st != IPA_OK) break;
        hesse_assemble_kernel<<<gf, kHesseBlock, 0, s>>>(c.spec, n_fits, theta_dev, c.h, c.vres, stage, c.hwork,
                                                         cov_out_dev, corr_out_dev, err_out_dev, status_out_dev);
        st = cuda_fail(cudaGetLastError(), "hesse assemble");
    }
    // blocking: the library buffers are reused by the next call
    ipa_status sy = cuda_fail(cudaStreamSynchronize(s), "hesse sync");
    trace("{\"call\": \"%s\", \"n_fits\": %d, \"events\": %lld, \"segments\": %lld}", who, n_fits,
          (long long)ev->n, (long long)(n_v * n_cat));
    return st != IPA_OK ? st : sy;
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_hesse(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                                int32_t n_fits, const ipa_param* spec, const double* theta_dev, double* cov_out_dev,
                                double* corr_out_dev, double* err_out_dev, int32_t* status_out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_common(model, ev, seg_off_dev, n_fits, spec, "ipa_hesse");
    if (st != IPA_OK) return st;
    if (!theta_dev || !cov_out_dev) {
        set_error("ipa_hesse: theta and the covariance output are required");
        return IPA_ERR_ARG;
    }
    Spec sp{};
    if ((st = build_spec(model, spec, 1, 1.0, &sp)) != IPA_OK) return st;
    return hesse_run(model, ev, seg_off_dev, n_fits, sp, theta_dev, cov_out_dev, corr_out_dev, err_out_dev,
                     status_out_dev, static_cast<cudaStream_t>(stream), nullptr, "ipa_hesse");
}

extern "C" ipa_status ipa_hesse_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                                      int32_t n_fits, const ipa_joint* joint, const ipa_param* spec,
                                      const double* theta_dev, double* cov_out_dev, double* corr_out_dev,
                                      double* err_out_dev, int32_t* status_out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_common(model, ev, seg_off_dev, n_fits, spec, "ipa_hesse_joint");
    if (st != IPA_OK) return st;
    if ((st = check_joint(model, joint, n_fits)) != IPA_OK) return st;
    if (!theta_dev || !cov_out_dev) {
        set_error("ipa_hesse_joint: theta and the covariance output are required");
        return IPA_ERR_ARG;
    }
    Spec sp{};
    if ((st = build_spec(model, spec, 1, 1.0, &sp, joint->n_joint)) != IPA_OK) return st;
    return hesse_run(model, ev, seg_off_dev, n_fits, sp, theta_dev, cov_out_dev, corr_out_dev, err_out_dev,
                     status_out_dev, static_cast<cudaStream_t>(stream), joint, "ipa_hesse_joint");
}

namespace ipa {
namespace {

ipa_status minos_run(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev, int32_t n_fits,
                     const ipa_param* spec, const Spec& sp, int n_par, const double* theta_min_dev,
                     const double* nll_min_dev, const double* cov_dev, const int32_t* scan, double up, double tol,
                     int32_t max_rounds, int32_t max_iter, double* lo_out_dev, double* hi_out_dev,
                     int32_t* status_out_dev, cudaStream_t s, const ipa_joint* joint, const char* who) {
    ipa_status st = IPA_OK;
    int list[kMaxP], n_scan = 0;
    for (int p = 0; p < n_par; ++p) {
        if (!scan[p]) continue;
        if (spec[p].fixed) {
            set_error("%s: parameter %d is fixed and cannot be scanned", who, p);
            return IPA_ERR_ARG;
        }
        list[n_scan++] = p;
    }
    if (n_scan == 0) {
        // nothing to scan: zero intervals, every status "not scanned"
        ProfileContext* cp0 = profile_context();
        if (!cp0) return IPA_ERR_CUDA;
        std::lock_guard<std::mutex> lk0(cp0->mu);
        if ((st = profile_basics(*cp0)) != IPA_OK) return st;
        if ((st = cuda_fail(cudaMemcpyAsync(cp0->spec, &sp, sizeof(Spec), cudaMemcpyHostToDevice, s), "minos spec")) !=
            IPA_OK)
            return st;
        minos_final_kernel<<<(n_fits + 127) / 128, 128, 0, s>>>(cp0->spec, cp0->scan, 0, n_fits, theta_min_dev,
                                                                nullptr, lo_out_dev, hi_out_dev, status_out_dev);
        st = cuda_fail(cudaGetLastError(), "minos final");
        ipa_status sy = cuda_fail(cudaStreamSynchronize(s), "minos sync");
        return st != IPA_OK ? st : sy;
    }
    ProfileContext* cp = profile_context();
    if (!cp) return IPA_ERR_CUDA;
    ProfileContext& c = *cp;
    std::lock_guard<std::mutex> lk(c.mu);
    const int n_cat = joint ? joint->n_cat : 1;
    if ((size_t)n_fits * n_scan * 2 * (size_t)n_cat > (size_t)1 << 30) {
        set_error("%s: too many profile fits (n_fits x scanned parameters x 2 x categories > 2^30)", who);
        return IPA_ERR_ARG;
    }
    const int n_probes = n_fits * n_scan * 2;
    if ((st = profile_basics(c)) != IPA_OK) return st;
    if ((st = minos_reserve(c, (size_t)n_probes)) != IPA_OK) return st;
    if (joint && (st = joint_reserve(c, (size_t)n_cat * model->n_par, (size_t)n_probes * n_cat)) != IPA_OK)
        return st;
    if ((st = cuda_fail(cudaMemcpyAsync(c.spec, &sp, sizeof(Spec), cudaMemcpyHostToDevice, s), "minos spec")) != IPA_OK)
        return st;
    if ((st = cuda_fail(cudaMemcpyAsync(c.scan, list, sizeof(int) * n_scan, cudaMemcpyHostToDevice, s),
                        "minos scan list")) != IPA_OK)
        return st;
    JointDev jd;
    if (joint) {
        const size_t mn = (size_t)n_cat * model->n_par;
        st = cuda_fail(cudaMemcpyAsync(c.jmap, joint->map, mn * sizeof(int32_t), cudaMemcpyHostToDevice, s),
                       "minos joint map copy");
        if (st == IPA_OK)
            st = joint->value ? cuda_fail(cudaMemcpyAsync(c.jvalue, joint->value, mn * sizeof(double),
                                                          cudaMemcpyHostToDevice, s), "minos joint values copy")
                              : cuda_fail(cudaMemsetAsync(c.jvalue, 0, mn * sizeof(double), s), "minos joint values");
        if (st != IPA_OK) return st;
        jd.n_cat = n_cat;
        jd.n_model = model->n_par;
        jd.n_joint = joint->n_joint;
        jd.map = c.jmap;
        jd.value = c.jvalue;
        jd.seg_begin = c.jbegin;
        jd.seg_end = c.jend;
        jd.theta_seg = c.jtheta;
        jd.res_seg = c.jres;
        jd.seg_active = c.jactive;
    }
    const int gp = (n_probes + 127) / 128;
    minos_init_kernel<<<gp, 128, 0, s>>>(c.spec, c.scan, n_scan, n_probes, theta_min_dev, cov_dev, c.probes);
    if ((st = cuda_fail(cudaGetLastError(), "minos init")) != IPA_OK) return st;
    const int64_t tiles = (int64_t)n_scan * 2 * ((ev->n + kTile - 1) / kTile + (int64_t)n_fits * n_cat);
    const bool only_free = sp.n_free == 1;   // the profile is the NLL itself
    const int max_passes = 6 * max_iter + 4 * sp.n_free + 40;
    int rounds = 0;
    for (; rounds < max_rounds && st == IPA_OK; ++rounds) {
        minos_prepare_kernel<<<gp, 128, 0, s>>>(c.spec, c.scan, n_scan, n_probes, seg_off_dev, n_cat, theta_min_dev,
                                                cov_dev, c.probes, c.pspecs, c.pbegin, c.pend, c.ptheta,
                                                joint ? c.jbegin : nullptr, joint ? c.jend : nullptr);
        if ((st = cuda_fail(cudaGetLastError(), "minos prepare")) != IPA_OK) break;
        if (only_free && joint) {
            jd.grad = false;
            st = virtual_pass_joint(model, ev, jd, n_probes, c.ptheta, tiles, c.pnll, s);
        } else if (only_free) {
            st = virtual_pass(model, ev, n_probes, c.pbegin, c.pend, c.ptheta, tiles, false, c.pnll, s);
        } else {
            jd.grad = true;
            st = fit_run(model, ev, n_probes, c.pbegin, c.pend, c.pspecs, 1, max_passes, tiles, c.ptheta, nullptr,
                         c.pnll, c.pstatus, nullptr, nullptr, s, joint ? "ipa_minos_joint constrained fits"
                                                                       : "ipa_minos constrained fits",
                         joint ? &jd : nullptr);
        }
        if (st != IPA_OK) break;
        if ((st = cuda_fail(cudaMemsetAsync(c.n_open, 0, sizeof(int), s), "minos counter")) != IPA_OK) break;
        minos_update_kernel<<<gp, 128, 0, s>>>(c.spec, c.scan, n_scan, n_probes, theta_min_dev, nll_min_dev, c.pnll,
                                               only_free ? nullptr : c.pstatus, up, tol, max_rounds, c.probes,
                                               c.n_open);
        if ((st = cuda_fail(cudaGetLastError(), "minos update")) != IPA_OK) break;
        if ((st = cuda_fail(cudaMemcpyAsync(c.h_open, c.n_open, sizeof(int), cudaMemcpyDeviceToHost, s),
                            "minos counter copy")) != IPA_OK)
            break;
        if ((st = cuda_fail(cudaStreamSynchronize(s), "minos sync")) != IPA_OK) break;
        if (*c.h_open == 0) {
            ++rounds;
            break;
        }
    }
    if (st == IPA_OK) {
        minos_final_kernel<<<(n_fits + 127) / 128, 128, 0, s>>>(c.spec, c.scan, n_scan, n_fits, theta_min_dev,
                                                                c.probes, lo_out_dev, hi_out_dev, status_out_dev);
        st = cuda_fail(cudaGetLastError(), "minos final");
    }
    ipa_status sy = cuda_fail(cudaStreamSynchronize(s), "minos sync");
    trace("{\"call\": \"%s\", \"n_fits\": %d, \"probes\": %d, \"rounds\": %d}", who, n_fits, n_probes, rounds);
    return st != IPA_OK ? st : sy;
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_minos(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                                int32_t n_fits, const ipa_param* spec, const double* theta_min_dev,
                                const double* nll_min_dev, const double* cov_dev, const int32_t* scan, double up,
                                double tol, int32_t max_rounds, int32_t max_iter, double fit_tol, double* lo_out_dev,
                                double* hi_out_dev, int32_t* status_out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_common(model, ev, seg_off_dev, n_fits, spec, "ipa_minos");
    if (st != IPA_OK) return st;
    if (!theta_min_dev || !nll_min_dev || !cov_dev || !scan || !lo_out_dev || !hi_out_dev || !(up > 0.0) ||
        !(tol > 0.0) || max_rounds < 1 || max_iter < 1 || !(fit_tol > 0.0)) {
        set_error("ipa_minos: bad arguments");
        return IPA_ERR_ARG;
    }
    Spec sp{};
    if ((st = build_spec(model, spec, max_iter, fit_tol, &sp)) != IPA_OK) return st;
    return minos_run(model, ev, seg_off_dev, n_fits, spec, sp, model->n_par, theta_min_dev, nll_min_dev, cov_dev,
                     scan, up, tol, max_rounds, max_iter, lo_out_dev, hi_out_dev, status_out_dev,
                     static_cast<cudaStream_t>(stream), nullptr, "ipa_minos");
}

extern "C" ipa_status ipa_minos_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                                      int32_t n_fits, const ipa_joint* joint, const ipa_param* spec,
                                      const double* theta_min_dev, const double* nll_min_dev, const double* cov_dev,
                                      const int32_t* scan, double up, double tol, int32_t max_rounds,
                                      int32_t max_iter, double fit_tol, double* lo_out_dev, double* hi_out_dev,
                                      int32_t* status_out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_common(model, ev, seg_off_dev, n_fits, spec, "ipa_minos_joint");
    if (st != IPA_OK) return st;
    if ((st = check_joint(model, joint, n_fits)) != IPA_OK) return st;
    if (!theta_min_dev || !nll_min_dev || !cov_dev || !scan || !lo_out_dev || !hi_out_dev || !(up > 0.0) ||
        !(tol > 0.0) || max_rounds < 1 || max_iter < 1 || !(fit_tol > 0.0)) {
        set_error("ipa_minos_joint: bad arguments");
        return IPA_ERR_ARG;
    }
    Spec sp{};
    if ((st = build_spec(model, spec, max_iter, fit_tol, &sp, joint->n_joint)) != IPA_OK) return st;
    return minos_run(model, ev, seg_off_dev, n_fits, spec, sp, joint->n_joint, theta_min_dev, nll_min_dev, cov_dev,
                     scan, up, tol, max_rounds, max_iter, lo_out_dev, hi_out_dev, status_out_dev,
                     static_cast<cudaStream_t>(stream), joint, "ipa_minos_joint");
}
