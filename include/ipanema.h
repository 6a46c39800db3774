/*
 * ipanema.h -- C ABI of the GB300 unbinned-likelihood library.
 *
 * The library evaluates, on one GPU, the per-event normalised PDF of an
 * unbinned maximum-likelihood fit (Ipanema-beta, arXiv:1706.01420), takes
 * -w log P per event and reduces it deterministically in FP64 to the negative
 * log-likelihood (NLL) and its gradient; it generates pseudo-experiments by
 * accept-reject and fits many of them at once.
 *
 * Paper passages (section numbers of arXiv:1706.01420):
 *   Sec. 3 (Example 1)  event-parallel PDF kernel, analytic normalisation,
 *                       log of the signal/background mixture, sum of logs,
 *                       FCN = -log L with errors at Delta FCN = 1/2, MIGRAD/HESSE;
 *   Sec. 4 (Example 2)  decay-time x helicity-angle fit of Bs -> J/psi K K:
 *                       P wave (3 polarisations) + S wave; Parameter/Free with
 *                       limits, Cat (per-category event array);
 *   Sec. 7 (Example 5)  toy generation by accept-reject with a counter-based
 *                       generator, Poisson-fluctuated counts drawn on the host;
 *   App. A-C            ParamBox, Parameter and Cat classes.
 *
 * Model (the paper prints no formula; this is the reading the library uses):
 *   g(tau)  = 1/2 exp(-Gamma tau + Gamma^2 sigma^2 / 2) erfc((Gamma sigma^2 - tau)/(sqrt2 sigma)),
 *             tau = t - mu: exp(-Gamma t) convolved with a Gaussian of width sigma;
 *   I_T     = int_{t_lo}^{t_hi} g(t - mu) dt (closed form);
 *   A(Omega)= sum_{k=1..10} h_k f_k(cos thK, cos thmu, phi)   (4D model only),
 *             I_Omega = 16 pi / 9;
 *   P       = (1 - f_b) g/I_T [A/I_Omega] + f_b / V,   V = volume of the box;
 *   NLL     = -sum_e w_e log P_e   (w_e = 1 when no weight column is given).
 *
 * Conventions for every call:
 *   - Event columns, theta and outputs are DEVICE pointers (cudaMalloc'd or torch
 *     CUDA tensors) unless a parameter says "host".  The caller owns them; the
 *     library never frees or keeps them after the call returns.
 *   - Event columns are contiguous FP64 structure-of-arrays and must be 16-byte
 *     aligned (vectorised loads); a misaligned column gives IPA_ERR_ARG.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream: results are valid once the stream reaches
 *     them.  Calls on the same stream are ordered; calls that share library
 *     scratch (see ipa_reserve) must not run concurrently on different streams.
 *   - Errors are returned as a status and never abort the process; the text
 *     of the last error of the calling thread is ipa_last_error().
 *   - Non-physical parameters (sigma <= 0, Gamma <= 0, fractions outside [0,1])
 *     are not rejected on the host (theta lives on the device); they produce
 *     NaN results, which the fitter reports as IPA_FIT_BAD_PDF.
 *   - The library keeps per-device state between calls (scratch, streams,
 *     captured graphs, fitter workspace).  It belongs to the device's current
 *     context: a device reset (cudaDeviceReset) between calls is not supported,
 *     except by ipa_nll_grad_noalloc, which looks its array up again in a new
 *     context.
 */
#ifndef IPANEMA_H
#define IPANEMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IPA_OK = 0,
    IPA_ERR_ARG = -1,      /* invalid argument (null, size, alignment, model kind) */
    IPA_ERR_OOM = -2,      /* a device allocation failed */
    IPA_ERR_CUDA = -3,     /* a CUDA runtime call failed; see ipa_last_error() */
    IPA_ERR_TIMEOUT = -4,  /* a bounded wait ran out */
    IPA_ERR_BUSY = -5,     /* no free slot / budget (server admission) */
    IPA_PENDING = 1        /* the request is still running (server poll) */
} ipa_status;

typedef enum {
    IPA_MODEL_TIME1D = 1,     /* decay time only: P(t)                              */
    IPA_MODEL_ANGTIME4D = 2,  /* decay time x helicity angles: P(t, ck, cl, phi)    */
    IPA_MODEL_TAGGED1D = 3,   /* flavour-tagged decay time with B_s oscillation: P(t, q) */
    IPA_MODEL_PHIS = 4        /* time-dependent angular model with tagging: P(t, ck, cl, phi, q) */
} ipa_model_kind;

/* The full time-dependent angular model (Sec. 4, the phi_s fit of
 * B_s -> J/psi K K: P wave and S wave, Gamma_L and Gamma_H, flavour-tagged
 * Dm oscillation, the CP phase; Sec. 2 for the convolution of the
 * oscillation with the resolution).  The paper prints no formula; this
 * library evolves the transversity amplitudes of the 4D model in time:
 * A_i(t) = A_i [g+(t) + eta_i lambda g-(t)] for a B_s at t = 0 and
 * A_i [g-(t) + eta_i lambda g+(t)] for a anti-B_s, eta = (+1, +1, -1, -1) for
 * (0, para, perp, S), lambda = e^{-i phi_s}; the ten angular terms are the
 * bilinears of the 4D model with A_i -> A_i(t), whose products of g+- are
 * sums of e^{-Gamma_L t}, e^{-Gamma_H t} and e^{-Gamma t} e^{i Dm t}, each
 * convolved with the Gaussian resolution; a tag q = +-1 with mistag omega
 * mixes the two initial flavours; normalised over t, the angles and both
 * tags, plus a flat background f_b; the three S-P interference terms carry a
 * factor C_SP (the overlap of the S- and P-wave lineshapes in a m(KK)
 * category, usually held at its computed value).  Parameters: the ten of the
 * 4D model, then DG, Dm, phi_s, omega, C_SP and the tag-normalisation
 * selector Q (IPA_PHIS_DG .. IPA_PHIS_QNORM).  With Q = 0 the PDF is
 * normalised over t, the angles and both tags; with Q = +1 or -1 over the one
 * tag (a category holding the events of one flavour, as in a simultaneous fit
 * over m(KK) bins times B flavours, Sec. 4 Example 2): the events of such a
 * segment must all carry that tag.  Events carry t, ck, cl, phi and q. */

/* The tagged model (Sec. 4, the B_s -> J/psi phi example, whose time-dependent
 * fit has the oscillation frequency Dm_s, the widths Gamma and DG and the
 * CP-violating phase as parameters; Sec. 2 and the symbolic-programming
 * section for the Faddeeva function that the oscillating terms convolved with
 * the Gaussian resolution need).  The paper prints no formula; this library
 * takes the tagged decay rate of a CP-even final state with |lambda| = 1,
 *   S(t, q) = e^{-Gamma t} [cosh(DG t / 2) - cos(phi_s) sinh(DG t / 2)
 *                          + q (1 - 2 omega) sin(phi_s) sin(Dm t)],  t >= 0,
 * convolved with a Gaussian (sigma, offset mu).  With Gamma_H,L = Gamma -+ DG/2
 * and g(tau; z) = int_0^inf e^{-z u} G(tau - u) du (complex z),
 *   S = (1 - c)/2 g(tau; Gamma_H) + (1 + c)/2 g(tau; Gamma_L)
 *       + q (1 - 2 omega) s Im g(tau; Gamma - i Dm),   c, s = cos, sin phi_s,
 * normalised over [t_lo, t_hi] and both tags by N = (1 - c) I(Gamma_H) +
 * (1 + c) I(Gamma_L), and P(t, q) = (1 - f_b) S / N + f_b / (2 (t_hi - t_lo)).
 * Parameters: Gamma, sigma, mu, f_b, DG, Dm, phi_s, omega (IPA_GAMMA ..
 * IPA_OMEGA).  Events carry t and q = +1.0 or -1.0. */

/* Parameter indices (theta layout).  1D uses the first 4, 4D the first 10,
 * the tagged model the first 4 and its own 4 to 7, the phi_s model the ten
 * of the 4D model and 10 to 15. */
enum {
    IPA_GAMMA = 0,   /* decay width Gamma [1/ps]                   */
    IPA_SIGMA = 1,   /* Gaussian time resolution sigma [ps]        */
    IPA_MU = 2,      /* resolution offset mu [ps]                  */
    IPA_FB = 3,      /* flat background fraction f_b               */
    IPA_A0SQ = 4,    /* |A_0|^2 (P-wave fraction, before 1 - F_S)  */
    IPA_APESQ = 5,   /* |A_perp|^2; |A_par|^2 = 1 - |A_0|^2 - |A_perp|^2 */
    IPA_DPA = 6,     /* strong phase delta_par [rad]               */
    IPA_DPE = 7,     /* strong phase delta_perp [rad]              */
    IPA_FS = 8,      /* S-wave fraction F_S                        */
    IPA_DS = 9,      /* S-wave phase delta_S [rad]; delta_0 = 0    */
    IPA_DG = 4,      /* tagged: width difference DG = Gamma_L - Gamma_H [1/ps] */
    IPA_DM = 5,      /* tagged: mass difference Dm_s [1/ps]        */
    IPA_PHIS = 6,    /* tagged: CP-violating phase phi_s [rad]     */
    IPA_OMEGA = 7,   /* tagged: mistag probability omega           */
    IPA_PHIS_DG = 10,    /* phi_s model: DG = Gamma_L - Gamma_H [1/ps]  */
    IPA_PHIS_DM = 11,    /* phi_s model: Dm_s [1/ps]                    */
    IPA_PHIS_PHIS = 12,  /* phi_s model: phi_s [rad]                    */
    IPA_PHIS_OMEGA = 13, /* phi_s model: mistag probability omega       */
    IPA_PHIS_CSP = 14,   /* phi_s model: C_SP factor of the three S-P interference terms */
    IPA_PHIS_QNORM = 15, /* phi_s model: normalisation over both tags (0) or over the tag
                            +1 (> 0) or -1 (< 0) alone; a selector, held fixed (gradient 0) */
    IPA_NPAR_1D = 4,
    IPA_NPAR_4D = 10,
    IPA_NPAR_TAGGED = 8,
    IPA_NPAR_PHIS = 16,
    IPA_MAX_PAR = 32     /* parameters of a fit (a joint fit over categories included) */
};

/* One fit parameter (Parameter / Free of App. B): start value, limits, step,
 * and whether it is held constant (fixed != 0). */
typedef struct {
    double value, lo, hi, step;
    int32_t fixed;
    int32_t _pad;
} ipa_param;

/* An event set (Cat of App. C): n events as FP64 SoA device columns.
 * t is required; ck, cl, phi are required for the 4D model and ignored
 * otherwise; q (the flavour tag, +1.0 or -1.0) is required for the tagged
 * and the phi_s models and ignored otherwise; w may be NULL (unit weights).
 * The phi_s model needs t, ck, cl, phi and q.  Every column is
 * 16-byte aligned.  fk may be NULL, or hold the angular basis of these events
 * written by ipa_angular_basis (10 columns of fk_stride doubles); 4D
 * likelihood and fit calls then read it instead of evaluating the angular
 * functions. */
typedef struct {
    int64_t n;
    const double *t, *ck, *cl, *phi, *w;
    const double* fk;
    int64_t fk_stride;
    const double* q;
} ipa_events;

/* Writable event columns for the generator; `capacity` is the number of
 * events each non-NULL column can hold (q: the tagged model's tag). */
typedef struct {
    int64_t capacity;
    double *t, *ck, *cl, *phi;
    double* q;
} ipa_event_buffers;

/* The model: its kind, number of parameters and the decay-time range. */
typedef struct {
    int32_t kind;      /* ipa_model_kind */
    int32_t n_par;     /* IPA_NPAR_1D, _4D, _TAGGED or _PHIS (set by ipa_model_init) */
    double t_lo, t_hi; /* decay-time range [ps], t_lo < t_hi */
} ipa_model;

/* Per-fit status written by ipa_fit_batch. */
enum {
    IPA_FIT_CONVERGED = 0,  /* Newton decrement (step in sigma units) below tol  */
    IPA_FIT_MAXITER = 1,    /* max_iter reached                                  */
    IPA_FIT_AT_LIMIT = 2,   /* converged with a free parameter on a limit        */
    IPA_FIT_BAD_PDF = 3,    /* NaN/inf NLL or gradient (non-physical parameters) */
    IPA_FIT_EMPTY = 4       /* the fit has no events                             */
};

/* Fill *m for `kind` on [t_lo, t_hi].  IPA_ERR_ARG for an unknown kind or an
 * empty range. */
ipa_status ipa_model_init(ipa_model* m, int32_t kind, double t_lo, double t_hi);

/* NLL = -sum_e w_e log P_e (Sec. 3: per-event PDF, log of the mixture, sum of
 * logs; Sec. 4: the 4D and the tagged model).  theta_dev: n_par doubles (device).
 * out_dev: 1 double (device).  The sum is a fixed-order FP64 tree over
 * 512-event tiles: the result does not depend on launch geometry.  n = 0
 * gives 0.  Uses library scratch (ipa_reserve). */
ipa_status ipa_nll(const ipa_model* model, const ipa_events* ev, const double* theta_dev,
                   double* out_dev, void* stream);

/* NLL and its analytic gradient in one event pass (Sec. 3 / App. B: analytic
 * gradients handed to the minimiser).  out_dev: 1 + n_par doubles (device):
 * out[0] = NLL, out[1 + j] = dNLL/dtheta_j for every j (free or not). */
ipa_status ipa_nll_grad(const ipa_model* model, const ipa_events* ev, const double* theta_dev,
                        double* out_dev, void* stream);

/* ipa_nll_grad for events in HOST memory (the columns of *host_ev are host
 * pointers, 16-byte aligned).  Page-locked columns (cudaHostAlloc or
 * registered) are read by the kernel in place through the device's mapping
 * of the allocation, so the transfer runs inside the event pass: out_dev is
 * bitwise ipa_nll_grad of the same events.  Pageable columns are split into
 * k = clamp(floor(n / 2^20), 1, 16) chunks of ceil(ceil(n / k) / 512) * 512
 * events (the last one shorter), copied into library staging buffers on four
 * library copy streams while the likelihood kernel runs, on `stream`, over the
 * chunks already on the device: out_dev (device, 1 + n_par doubles) = the sum,
 * in chunk order, of ipa_nll_grad over each chunk (bitwise).  The host columns must stay unchanged until the work on
 * `stream` completes.  No cached angular basis (IPA_ERR_ARG).  The staging
 * buffers grow to n events per column (library memory, kept). */
ipa_status ipa_nll_grad_host(const ipa_model* model, const ipa_events* host_ev, const double* theta_dev,
                             double* out_dev, void* stream);

/* Same as ipa_nll_grad for n_seg event segments packed back to back in one
 * set of columns: segment s is events [seg_off[s], seg_off[s+1]) and uses
 * theta_dev + s*n_par; out_dev receives (1 + n_par) doubles per segment.
 * seg_off_dev: n_seg + 1 int64 (device), non-decreasing, within [0, ev->n]
 * (offsets live on the device and are not checked on the host; values outside
 * [0, ev->n] are clamped into it).  Each segment's result is bitwise the result of ipa_nll_grad on
 * that segment alone; an empty segment gives NLL = 0 and a zero gradient. */
ipa_status ipa_nll_grad_segmented(const ipa_model* model, const ipa_events* ev,
                                  const int64_t* seg_off_dev, int32_t n_seg,
                                  const double* theta_dev, double* out_dev, void* stream);

/* Angular basis of an event set (hot-path step a3, data-only; Sec. 4 and the
 * symbolic-programming section): fk_dev[k * stride + e] = f_{k+1}(ck[e], cl[e],
 * phi[e]) for k = 0..9, e < ev->n.  stride >= ev->n and even; fk_dev 16-byte
 * aligned (device, 10 * stride doubles, caller-owned).  Computed once per event
 * set, it replaces the sine, cosine, square root and ten products of every
 * later likelihood pass by 80 bytes of reads.  4D model only. */
ipa_status ipa_angular_basis(const ipa_model* model, const ipa_events* ev, double* fk_dev, int64_t stride,
                             void* stream);

/* Accept-reject pseudo-experiments (Sec. 7).  Toy k holds n_sig[k] signal
 * events then n_bkg[k] background events, written at event offset
 * offsets[k] of each output column (offsets[k] + n_sig[k] + n_bkg[k] <=
 * out->capacity).  Signal candidate j of toy k uses Philox-4x32-10 with key =
 * (seed lo32, seed hi32) and counters (j lo32, j hi32, k, c) for c = 0,1,2;
 * the toy keeps the first n_sig[k] accepted candidates in increasing j.
 * Background event i uses counters (i lo32, i hi32, k, 4) and (.., 5).
 * Tagged model: candidate j draws (t, u) from call 0 and the tag from the
 * first uniform u_q of call 1 (q = +1 if u_q <= 1/2, else -1) and is kept iff
 * u M_S < S(t - mu, q), M_S = (1 - c)/2 M(Gamma_H) + (1 + c)/2 M(Gamma_L) +
 * |(1 - 2 omega) s| M(Gamma) with M(x) = min(1, e^{-x (t_lo - mu) + x^2
 * sigma^2 / 2}); background event i takes t and q from call 4; out->t and
 * out->q are written.
 * phi_s model: the proposal is piecewise uniform in t over 64 equal bins
 * (left edges e_i = t_lo + i w) with weights B_i = (m(Gamma_L) + m(Gamma_H) +
 * 2 m(Gamma)) sum_k max|f_k| |b_k| r_k, m(x) = min(1, e^{-x (e_i - mu) + x^2
 * sigma^2 / 2}) (|b_k| the magnitude of the term's amplitude product, r_k =
 * |C_SP| for the S-P terms, else 1), a bound of the rate on the bin.
 * Candidate j draws (u_bin, u) from call 0, (ck, cl) from call 1, (phi, u_pos)
 * from call 2 and u_q from call 3; its bin is the first i with u_bin C_64 <=
 * C_{i+1} (C the running sums of B), t = min(e_i + u_pos w, t_hi); its tag is
 * the one the normalisation selector names (theta[IPA_PHIS_QNORM] = +-1),
 * else +1 if u_q <= 1/2 and -1 otherwise; it is kept iff u B_i < rate(t,
 * Omega, q).  Background event i: t, ck from call 4, cl, phi from call 5,
 * u_q from call 6.  All five columns are written.
 * Candidates are built with IEEE-exact operations only, so a stream is
 * reproducible bit for bit.  n_sig, n_bkg, offsets: n_toys int64 each
 * (device).  For 1D only out->t is written.  A toy with a negative count or
 * a range outside [0, capacity) is skipped (its slots are left untouched).
 * Parameters for which nothing can be accepted (non-finite envelope), or a
 * toy that exhausts its candidate budget (65536 n_sig + 2^22 candidates),
 * leave NaN in the unfilled signal slots. */
ipa_status ipa_toygen(const ipa_model* model, const double* theta_dev, uint64_t seed,
                      int32_t n_toys, const int64_t* n_sig_dev, const int64_t* n_bkg_dev,
                      const int64_t* offsets_dev, const ipa_event_buffers* out, void* stream);

/* Fit n_fits event segments at once (Sec. 3-4: MIGRAD minimisation and HESSE
 * errors).  Segments as in ipa_nll_grad_segmented.  spec (host): n_par
 * parameters (start value, limits, fixed flag), shared by all fits; the start
 * values are read from theta_io_dev (n_fits x n_par, device) and the fitted
 * values written back there.  Outputs (device): err_out_dev n_fits x n_par
 * (sqrt of the inverse-Hessian diagonal, 0 for fixed parameters), nll_out_dev
 * n_fits, fit_status_dev n_fits (IPA_FIT_*), iters_out_dev n_fits (minimiser
 * iterations; may be NULL), passes_out_dev n_fits (NLL+gradient passes over
 * the fit's events, including line-search trials and the Hessian; may be NULL).  Stops each fit when its Newton decrement is below tol or after
 * max_iter iterations.  Blocks the calling thread until all fits end. */
ipa_status ipa_fit_batch(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                         int32_t n_fits, const ipa_param* spec, double* theta_io_dev,
                         double* err_out_dev, double* nll_out_dev, int32_t* fit_status_dev,
                         int32_t* iters_out_dev, int32_t* passes_out_dev, int32_t max_iter, double tol,
                         void* stream);

/* ---- stepwise fits: the minimiser of ipa_fit_batch driven one pass at a time ----
 * Sec. 3 hands Minuit an FCN that the GPU evaluates; here the caller evaluates
 * the NLL and gradient (ipa_nll_grad_segmented, or the event-sharded
 * ipa_nll_grad_shard + ipa_nll_grad_combine over several GPUs) and the library
 * advances every fit's quasi-Newton state machine on the device (the same
 * kernels as ipa_fit_batch: BFGS line search, finite-difference Hessian,
 * Newton steps; given the same evaluations the fits follow the same path).
 * The state of n_fits fits lives in one device buffer the caller owns
 * (ipa_fit_state_bytes bytes, 256-byte aligned).  Its first n_fits x n_par
 * doubles are the points the fits want evaluated next (row i: fit i); the rest
 * holds the specification and each fit's minimiser state as plain data, so a
 * copy of the buffer taken between two passes resumes the fits bit for bit
 * (the analogue of the ParamBox fit summary the paper saves, App. B).  The
 * calls are asynchronous on `stream` and allocate nothing. */
uint64_t ipa_fit_state_bytes(int32_t n_fits, int32_t n_par);   /* 0 for bad sizes */

/* Start n_fits fits at theta0_dev (n_fits x n_par, device), with the limits,
 * steps and fixed flags of spec (host, n_par entries; start values are taken
 * from theta0_dev) and the tolerance and budget of ipa_fit_batch.  Writes the
 * state and the first points to evaluate. */
ipa_status ipa_fit_begin(const ipa_model* model, const ipa_param* spec, int32_t n_fits, const double* theta0_dev,
                         int32_t max_iter, double tol, void* state_dev, void* stream);

/* One pass: results_dev (n_fits x (1 + n_par), device) holds the NLL and
 * gradient at each fit's current point (the first rows of the state).  Every
 * fit still running takes its step and writes its next point; *n_active_dev
 * (device int32) receives the number of fits still running (0: all done).
 * Rows of finished fits are not read. */
ipa_status ipa_fit_advance(const ipa_model* model, int32_t n_fits, const double* results_dev, void* state_dev,
                           int32_t* n_active_dev, void* stream);

/* The fits' results from their state, as ipa_fit_batch writes them (theta_out
 * n_fits x n_par; the other outputs may be NULL). */
ipa_status ipa_fit_end(const ipa_model* model, int32_t n_fits, const void* state_dev, double* theta_out_dev,
                       double* err_out_dev, double* nll_out_dev, int32_t* fit_status_dev, int32_t* iters_out_dev,
                       int32_t* passes_out_dev, void* stream);

/* ---- event-sharded likelihood over several GPUs (one process per GPU) ----
 * The NLL and its gradient are sums over events (Sec. 3: the PDF is evaluated
 * one thread per event and the log-likelihoods are summed).  Rank r of W holds
 * the contiguous events [a_r, b_r) of the fit, with every a_r a multiple of
 * IPA_SHARD_EVENTS (16384 events: one group of 32 tiles of the kernel's fixed
 * reduction tree).  Each rank calls ipa_nll_grad_shard on its events; the
 * ranks all-gather the group partials in rank order (ceil((b_r - a_r) /
 * IPA_SHARD_EVENTS) rows of ipa_shard_width doubles per rank); every rank then
 * calls ipa_nll_grad_combine on the gathered rows.  The combine runs the last,
 * fixed-order level of the reduction and the gradient contraction, so every
 * rank obtains exactly the bits that ipa_nll_grad gives for all events on one
 * GPU, whatever the number of ranks.  Exchanged per pass: 8 x width bytes per
 * 16384 events (120 doubles per 1.3e5 events for the 4D model). */
#define IPA_SHARD_EVENTS 16384

/* Doubles per group partial for this model (15 for 4D, 6 for 1D, 13 tagged,
 * 47 phi_s). */
ipa_status ipa_shard_width(const ipa_model* model, int32_t* width);

/* ipa_nll_grad over this rank's events (out_dev: 1 + n_par doubles, this
 * shard's own NLL and gradient), plus its group partials into groups_dev
 * (device, ceil(n / IPA_SHARD_EVENTS) x ipa_shard_width doubles; not written
 * for n = 0). */
ipa_status ipa_nll_grad_shard(const ipa_model* model, const ipa_events* ev, const double* theta_dev,
                              double* out_dev, double* groups_dev, void* stream);

/* NLL and gradient (out_dev, 1 + n_par doubles) from n_groups gathered group
 * partials (groups_dev, device, in event order), at theta_dev; cached: the
 * shards used a cached angular basis (ev->fk).  n_groups = 0 gives zeros. */
ipa_status ipa_nll_grad_combine(const ipa_model* model, const double* theta_dev, const double* groups_dev,
                                int64_t n_groups, int32_t cached, double* out_dev, void* stream);

/* A simultaneous fit over categories (Sec. 4, Example 2: one -2 log L summed
 * over 12 categories, six m(KK) bins times two B flavours, that share most
 * parameters while the S-wave parameters are per bin and C_SP is a constant of
 * each bin; App. B: the Cat and ParamBox classes).  Every fit has n_cat
 * categories; category c of fit i is the event segment i * n_cat + c of
 * seg_off_dev (n_fits * n_cat + 1 int64 offsets, device, as in
 * ipa_nll_grad_segmented).  A fit has n_joint parameters theta_J
 * (1 <= n_joint <= IPA_MAX_PAR); category c evaluates the model at
 *   theta_c[p] = theta_J[map[c * n_par + p]]   where map[...] >= 0,
 *   theta_c[p] = value[c * n_par + p]           where map[...] == -1,
 * and the fit's NLL is sum_c NLL_c(theta_c), its gradient
 * dNLL/dtheta_J[j] = sum over (c, p) with map = j of dNLL_c/dtheta_c[p], both
 * summed in a fixed order (c ascending, then p ascending), so results do not
 * depend on the launch geometry.  map and value are host arrays of
 * n_cat x n_par (the model's n_par), read during the call.  IPA_ERR_ARG when
 * an entry of map is outside [-1, n_joint) or a joint parameter is used by no
 * category. */
typedef struct ipa_joint {
    int32_t n_cat;          /* categories per fit (>= 1) */
    int32_t n_joint;        /* parameters of a fit */
    const int32_t* map;     /* host, n_cat x n_par: joint index or -1 */
    const double* value;    /* host, n_cat x n_par: the constant where map is -1 (may be NULL if none is) */
} ipa_joint;

/* The joint NLL and gradient of n_fits simultaneous fits at theta_dev
 * (n_fits x n_joint, device): out_dev (device) receives 1 + n_joint doubles per
 * fit (NLL, then dNLL/dtheta_J).  Each category's NLL and gradient is
 * bitwise that of ipa_nll_grad_segmented at its theta_c. */
ipa_status ipa_nll_grad_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                              int32_t n_fits, const ipa_joint* joint, const double* theta_dev, double* out_dev,
                              void* stream);

/* Fit n_fits simultaneous fits at once: ipa_fit_batch's minimiser over the
 * joint parameters.  spec (host): n_joint parameters (start value, limits,
 * step, fixed flag); theta_io_dev n_fits x n_joint (start values in, fitted
 * values out); err_out_dev n_fits x n_joint; the other outputs as in
 * ipa_fit_batch (IPA_FIT_EMPTY when all of a fit's categories are empty). */
ipa_status ipa_fit_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                         int32_t n_fits, const ipa_joint* joint, const ipa_param* spec, double* theta_io_dev,
                         double* err_out_dev, double* nll_out_dev, int32_t* fit_status_dev,
                         int32_t* iters_out_dev, int32_t* passes_out_dev, int32_t max_iter, double tol,
                         void* stream);

/* HESSE on the device (Sec. 3-4: the errors and the correlation matrix that
 * follow each MIGRAD minimum, Figs. 2 and 4).  For each fit, the Hessian of
 * the NLL over the free parameters at theta_dev (n_fits x n_par, device; the
 * minima from ipa_fit_batch, or any point) by central differences of the
 * analytic gradient (one-sided, +h and +2h, where theta - h would leave the
 * lower limit), in two batched passes: steps of 1e-3 of each parameter's step,
 * then 2e-3 of the errors that gives.  Outputs (device, n_fits blocks,
 * row-major): cov_out_dev n_par x n_par = H^-1 (zero rows and columns for fixed
 * parameters); corr_out_dev n_par x n_par correlations (may be NULL);
 * err_out_dev n_par = sqrt(diag) (may be NULL); status_out_dev (may be NULL):
 * 0 positive definite, 1 made positive definite by a diagonal shift, 3 not
 * finite (outputs NaN).  Segments and spec (host: limits, steps, the fixed
 * flags; values unused) as in ipa_fit_batch.  Blocks until done. */
ipa_status ipa_hesse(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev, int32_t n_fits,
                     const ipa_param* spec, const double* theta_dev, double* cov_out_dev, double* corr_out_dev,
                     double* err_out_dev, int32_t* status_out_dev, void* stream);

/* HESSE of simultaneous fits (Sec. 4, Example 2: the covariance and
 * correlation matrix of the twelve-category fit): ipa_hesse over the joint
 * parameters, each virtual point evaluated as in ipa_nll_grad_joint.
 * Segments, joint map and spec (n_joint parameters) as in ipa_fit_joint;
 * theta_dev n_fits x n_joint; outputs as in ipa_hesse with n_par = n_joint. */
ipa_status ipa_hesse_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                           int32_t n_fits, const ipa_joint* joint, const ipa_param* spec, const double* theta_dev,
                           double* cov_out_dev, double* corr_out_dev, double* err_out_dev,
                           int32_t* status_out_dev, void* stream);

/* MINOS status of one side of one parameter's interval. */
enum {
    IPA_MINOS_OK = 0,            /* |NLL_profile - NLL_min - up| < tol                   */
    IPA_MINOS_MAXROUNDS = 1,     /* max_rounds reached; the last point is reported       */
    IPA_MINOS_AT_LIMIT = 2,      /* the profile stays below the threshold up to the limit */
    IPA_MINOS_FIT_FAILED = 3,    /* a constrained fit failed, or no HESSE error to start  */
    IPA_MINOS_NEW_MINIMUM = 4,   /* a constrained fit went below NLL_min - tol           */
    IPA_MINOS_NOT_SCANNED = 5
};

/* MINOS profile-likelihood intervals on the device.  For each fit and each
 * parameter p with scan[p] != 0 (host, n_par flags; p must be free), the
 * points x_lo < theta_p < x_hi where the NLL minimised over every other free
 * parameter with theta_p fixed at x rises by `up` (0.5 for 1 sigma) above
 * nll_min_dev[f].  theta_min_dev (n_fits x n_par), nll_min_dev (n_fits) and
 * cov_dev (n_fits x n_par x n_par, from ipa_hesse) describe the minima
 * (device).  All fits, parameters and sides advance together: each round is
 * one batched constrained fit (the minimiser of ipa_fit_batch with max_iter
 * and fit_tol) per open probe, started at the conditional mean of the
 * Gaussian approximation, then a secant step on sqrt(2 (NLL_profile -
 * NLL_min)); a probe ends when |NLL_profile - NLL_min - up| < tol or after
 * max_rounds rounds.  Outputs (device): lo_out_dev, hi_out_dev (n_fits x
 * n_par): x_lo - theta_p (negative) and x_hi - theta_p, 0 where not scanned;
 * status_out_dev (n_fits x n_par x 2: lower, upper; may be NULL):
 * IPA_MINOS_*.  Blocks until done. */
ipa_status ipa_minos(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev, int32_t n_fits,
                     const ipa_param* spec, const double* theta_min_dev, const double* nll_min_dev,
                     const double* cov_dev, const int32_t* scan, double up, double tol, int32_t max_rounds,
                     int32_t max_iter, double fit_tol, double* lo_out_dev, double* hi_out_dev,
                     int32_t* status_out_dev, void* stream);

/* MINOS of simultaneous fits: ipa_minos over the joint parameters, every
 * constrained fit a simultaneous fit over the fit's categories (as in
 * ipa_fit_joint).  Segments, joint map and spec (n_joint parameters) as in
 * ipa_fit_joint; theta_min_dev n_fits x n_joint, cov_dev n_fits x n_joint x
 * n_joint (ipa_hesse_joint), scan n_joint flags; outputs as in ipa_minos with
 * n_par = n_joint. */
ipa_status ipa_minos_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                           int32_t n_fits, const ipa_joint* joint, const ipa_param* spec,
                           const double* theta_min_dev, const double* nll_min_dev, const double* cov_dev,
                           const int32_t* scan, double up, double tol, int32_t max_rounds, int32_t max_iter,
                           double fit_tol, double* lo_out_dev, double* hi_out_dev, int32_t* status_out_dev,
                           void* stream);

/* ---- binned workloads (Example 4 "CLs" and the toolkit's generateBinned and
 * Gaussian smearing) ----
 *
 * Poisson pseudo-experiments of a histogram (generateBinned): counts_out_dev
 * [k * n_bins + i] ~ Poisson(lambda_dev[i]) for toy toy0 + k, k < n_toys
 * (int32, device, caller-owned; lambda_dev n_bins doubles, device).  Bin i of
 * toy k under `hypothesis` h (0 or 1) inverts the Poisson CDF with uniforms
 * from Philox-4x32-10, key = (seed lo32, seed hi32), counter (i lo32, i hi32,
 * k, 8 + 2^16 h + m/2) for piece m of a mean split into ceil(lambda / 400)
 * equal pieces above 400; every step is a correctly rounded IEEE operation,
 * so the counts are reproducible bit for bit.  lambda <= 0 gives 0.
 * The CDF of each bin is tabulated once per call (the recurrence depends only
 * on the mean), so a draw is one Philox block and a few comparisons.
 * IPA_ERR_ARG for negative sizes, a hypothesis other than 0 or 1, or NULL
 * arrays.  Synchronises `stream` once (to size the tables), then runs
 * asynchronously on it. */
ipa_status ipa_binned_generate(const double* lambda_dev, int64_t n_bins, uint64_t seed, int32_t hypothesis,
                               int32_t toy0, int32_t n_toys, int32_t* counts_out_dev, void* stream);

/* Gaussian smearing of a histogram (the binned resolution convolution):
 * out_i = sum_{|d| <= R} K_d hist_{i-d}, R = ceil(8 sigma / bin_width), bins
 * outside the histogram contributing nothing, K_d = exp(-(d bin_width)^2 /
 * (2 sigma^2)) normalised to unit sum.  hist_dev, out_dev: n_bins doubles
 * (device, distinct).  IPA_ERR_ARG for non-positive width or sigma, sigma
 * above 1.25e6 bins, or aliased arrays.  Asynchronous on `stream`. */
ipa_status ipa_binned_smear(const double* hist_dev, int64_t n_bins, double bin_width, double sigma, double* out_dev,
                            void* stream);

/* CL_b, CL_s+b and CL_s of a binned search (Example 4; the modified
 * frequentist method of its references): with expected signal s_dev and
 * background b_dev per bin (n_bins doubles each, device, b > 0 in every bin)
 * and the observed counts data_dev (n_bins int32, device), the statistic
 * X = sum_i n_i ln(1 + s_i / b_i) (the data-dependent part of -2 ln Q,
 * Q = L(s+b) / L(b)) of n_toys toys under the background-only (h = 0, mean
 * b) and the signal-plus-background hypothesis (h = 1, mean s + b), drawn as
 * in ipa_binned_generate with toys 0..n_toys-1, gives CL_b = P_b(X <= X_obs),
 * CL_s+b = P_s+b(X <= X_obs), CL_s = CL_s+b / CL_b (NaN when CL_b = 0).
 * Outputs (device): cl_out_dev[3] = (CL_b, CL_s+b, CL_s); counts_out_dev[2]
 * the toy counts behind them (may be NULL); x_out_dev (2 n_toys + 1: X of the
 * b toys, of the s+b toys, X_obs; may be NULL).  Toys are drawn on the fly,
 * one block per toy: nothing of size n_toys x n_bins is stored.  Synchronises
 * `stream` twice (to size the CDF tables), then runs asynchronously on it. */
ipa_status ipa_cls(const double* s_dev, const double* b_dev, int64_t n_bins, const int32_t* data_dev, int32_t n_toys,
                   uint64_t seed, double* cl_out_dev, int64_t* counts_out_dev, double* x_out_dev, void* stream);

/* Fit server (continuous batching).  Fits of different sizes are submitted
 * as they arrive; each is admitted into a device slot when a slot and a
 * contiguous range of the event arena (the HBM budget, 40 bytes per event) are
 * free, in submission order; all admitted fits advance together, four passes
 * per tick, with the state machine of ipa_fit_batch, so a fit's result is
 * bitwise the one ipa_fit_batch gives for it alone.  The paper fits one data
 * set at a time (Sec. 3-4); this is the serving form of the same path. */
typedef struct ipa_server ipa_server;

/* Create a server on the current device: event arena of hbm_budget_bytes,
 * max_slots concurrent fits, minimiser budget and tolerance as in
 * ipa_fit_batch.  Starts one host worker thread.  *out owns device memory
 * until ipa_server_destroy. */
ipa_status ipa_server_create(const ipa_model* model, size_t hbm_budget_bytes, int32_t max_slots,
                             int32_t max_iter, double tol, ipa_server** out);

/* Submit one fit: ev (columns in host or device memory, any alignment; w may
 * be NULL) and spec (host, n_par parameters: start value, limits, step, fixed).
 * The events are copied before the call returns, so the caller may free them.
 * *ticket identifies the fit.  IPA_ERR_ARG if ev->n exceeds the arena. */
ipa_status ipa_serve_submit(ipa_server* server, const ipa_events* ev, const ipa_param* spec,
                            uint64_t* ticket);

/* Poll a fit: IPA_PENDING while it waits or runs; IPA_OK once finished, with
 * theta_out and err_out (host, n_par each), *nll and *fit_status (IPA_FIT_*)
 * written (NULL outputs are skipped) and the ticket released; IPA_ERR_ARG for
 * an unknown ticket; the server's error status if it stopped on a CUDA error. */
ipa_status ipa_serve_poll(ipa_server* server, uint64_t ticket, double* theta_out, double* err_out,
                          double* nll, int32_t* fit_status);

/* Stop the worker, drop unfinished fits and free the server's memory. */
ipa_status ipa_server_destroy(ipa_server* server);

/* Largest event count accepted by ipa_nll_grad_noalloc (2^23). */
#define IPA_NOALLOC_MAX_EVENTS 8388608

/* ipa_nll_grad without any device allocation.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory at call
 * time -- a host framework whose allocator already reserved the GPU, or a
 * latency-critical loop that must not pay for an allocation and the device
 * synchronisation that growing library scratch implies.  Same arguments and
 * results as ipa_nll_grad.  Its scratch is one fixed array compiled into the
 * library (~2 MB, held on every GPU that loads the library until exit), so
 * ev->n may not exceed IPA_NOALLOC_MAX_EVENTS (IPA_ERR_ARG otherwise).  The
 * first call on each device looks the array's address up (cudaGetSymbolAddress)
 * with that device current; make it before any stream capture.  The array is
 * shared by all calls and keeps the last call's contents; calls that overlap
 * on the GPU race on it. */
ipa_status ipa_nll_grad_noalloc(const ipa_model* model, const ipa_events* ev, const double* theta_dev,
                                double* out_dev, void* stream);

/* Host-side fault injection for tests of the error paths (the paper has no
 * counterpart).  Sets the mask and returns the previous one; nothing is ever
 * injected on the device.
 *   IPA_FAULT_ALLOC   every device allocation the library makes (scratch,
 *                     fitter workspace, server memory) fails with IPA_ERR_OOM
 *                     without calling cudaMalloc; state already allocated is
 *                     kept, and calls succeed again once the bit is cleared;
 *   IPA_FAULT_SUBMIT  ipa_serve_submit returns IPA_ERR_OOM before it takes the
 *                     request (as if its staging allocation failed); the caller
 *                     still holds the events and may submit them again;
 *   IPA_FAULT_ADMIT   the fit server admits no queued fit: queued requests
 *                     keep their place and are admitted once the bit is cleared.
 * The environment variable IPA_FAULT ("alloc", "submit", "admit", comma
 * separated) sets the mask when the library is loaded. */
#define IPA_FAULT_ALLOC 1u
#define IPA_FAULT_SUBMIT 2u
#define IPA_FAULT_ADMIT 4u
uint32_t ipa_fault_inject(uint32_t mask);

/* Grow the library's device scratch on the current device to hold one call
 * over `max_events` events in up to `max_segments` segments, so that later
 * calls allocate nothing (needed before CUDA-graph capture).  Calls allocate
 * on demand otherwise. */
ipa_status ipa_reserve(int64_t max_events, int32_t max_segments);

/* Bytes of device memory that the library's per-device scratch (the buffers
 * that ipa_reserve grows and that ipa_nll, ipa_nll_grad, the segmented, joint
 * and fitting calls use) holds on the current device; 0 before the first such
 * call.  A diagnostic with no counterpart in the paper: it lets a caller check
 * that a sequence of calls (for example ipa_nll_grad_noalloc alone) allocated
 * no scratch.  IPA_ERR_ARG if bytes is NULL. */
ipa_status ipa_scratch_bytes(uint64_t* bytes);

/* ---- launch geometry and its autotuner (the paper has no counterpart: its
 * kernels use one thread per event and a host-side sum, Sec. 3) ----
 *
 * The likelihood kernel adds each segment's events in an order fixed by
 * 512-event tiles and groups of 32 tiles, so the geometry below changes the
 * speed of ipa_nll, ipa_nll_grad, ipa_nll_grad_segmented, ipa_fit_batch and the
 * server, never a result (bit for bit).  A geometry is kept per device, kernel
 * variant (model kind, gradient or not, cached angular basis or not, one
 * segment or several) and size class (tile count rounded down to a power of
 * two).  Untuned classes use single-warp blocks with ceil(tiles / SMs)
 * resident warps per SM. */
typedef struct {
    int32_t warps_per_block;   /* 1, 2, 4 or 8 */
    int32_t warps_per_sm;      /* resident warps wanted per SM (capped by occupancy);
                                  0 = one per tile-take per SM, ceil(takes / SMs) */
    int32_t tiles_per_take;    /* 512-event tiles a warp takes from the work counter at once: 1, 2 or 4 */
    float ms;                  /* ipa_autotune: measured time per launch of the pick; 0 otherwise */
} ipa_launch_config;

/* Time every geometry (block size 1/2/4/8 warps x {ceil(takes/SMs), occupancy}
 * warps per SM x 1/2/4 tiles per take) on these events and parameters and
 * keep the fastest for their variant and size class.  seg_off_dev (device,
 * n_seg + 1 offsets) may be NULL for one segment; theta_dev holds n_seg x
 * n_par parameters; grad selects the NLL+gradient (1) or NLL-only (0) kernel;
 * a cached basis in ev->fk selects the cached variant.  Blocking (synchronises
 * the stream; about 24 x 5 ms); IPA_ERR_BUSY if the stream is being captured,
 * IPA_ERR_ARG for no events.  `picked` (host, may be NULL) receives the pick
 * with its time.  Graphs the fitter cached before the call are re-captured. */
ipa_status ipa_autotune(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev, int32_t n_seg,
                        const double* theta_dev, int32_t grad, ipa_launch_config* picked, void* stream);

/* Geometry that a launch over n_events events in n_seg segments would use
 * (host output), and explicit setting of a class's geometry (IPA_ERR_ARG for
 * values outside the ranges above). */
ipa_status ipa_launch_config_get(const ipa_model* model, int64_t n_events, int32_t n_seg, int32_t grad,
                                 int32_t cached, ipa_launch_config* cfg);
ipa_status ipa_launch_config_set(const ipa_model* model, int64_t n_events, int32_t n_seg, int32_t grad,
                                 int32_t cached, const ipa_launch_config* cfg);

/* FP64 roofline calibration on the current device (blocking, ~1 s).
 * results (host, 15 doubles): [0] DFMA per clock per SM, [1] DFMA per second
 * for the whole GPU, [2..7] cost of one CUDA exp, erfc, log, sincos, sqrt and
 * reciprocal in DFMA issue slots, [8] SM clock during the DFMA run [MHz],
 * [9..12] cost of the library's own table-driven exp, log, sincos and erfcx,
 * [13..14] time of the library's integer-pipe exp and sincos run alone, in
 * DFMA slots (they use no FP64 instruction; in the likelihood kernel they
 * overlap the FP64 work). */
ipa_status ipa_calibrate_fp64(double* results, void* stream);

/* The library's own FP64 elementary functions, evaluated elementwise: test
 * support with no counterpart in the paper (the likelihood kernel calls these
 * functions; their accuracy is tested against the CPU's libm).
 *   IPA_MATH_EXP    table-driven exp (library exp above 709)
 *   IPA_MATH_LOG    table-driven log (library log for zero, negative,
 *                   subnormal, infinite and NaN arguments)
 *   IPA_MATH_SIN,
 *   IPA_MATH_COS    integer-pipe sincos for |x| < 1024 (the angles and the
 *                   oscillation phase), table-driven above, library sincos
 *                   for |x| >= 1e5
 *   IPA_MATH_ERFCX  piecewise polynomial on [0, 6.25], library erfcx above
 *   IPA_MATH_RCP    1/x from an FP32 seed and one FP64 Newton step
 * x_dev, y_dev: device arrays of n doubles (caller-owned).  IPA_ERR_ARG for an
 * unknown fn or NULL arrays with n > 0.  Asynchronous on `stream`. */
enum { IPA_MATH_EXP = 0, IPA_MATH_LOG = 1, IPA_MATH_SIN = 2, IPA_MATH_COS = 3, IPA_MATH_ERFCX = 4,
       IPA_MATH_RCP = 5 };
ipa_status ipa_math_eval(int32_t fn, const double* x_dev, double* y_dev, int64_t n, void* stream);

/* The Faddeeva function w(z) = exp(-z^2) erfc(-i z) as the tagged model's
 * kernels evaluate it (Sec. 2 and the symbolic-programming section: the
 * oscillating decay-time terms convolved with the Gaussian resolution need
 * it): for Im z >= 0 Weideman's rational approximation with N = 40 terms
 * (SIAM J. Numer. Anal. 31 (1994) 1497), relative error below 1e-15; for
 * Im z < 0 the reflection w(z) = 2 exp(-z^2) - w(-z), which overflows where
 * exp(-z^2) does.  Test support: z_dev and w_dev hold n complex numbers as
 * (re, im) pairs of doubles (device, caller-owned).  IPA_ERR_ARG for NULL
 * arrays with n > 0.  Asynchronous on `stream`. */
ipa_status ipa_faddeeva(const double* z_dev, double* w_dev, int64_t n, void* stream);

/* Text of the calling thread's last error ("" if none). */
const char* ipa_last_error(void);

/* Library version string. */
const char* ipa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IPANEMA_H */
