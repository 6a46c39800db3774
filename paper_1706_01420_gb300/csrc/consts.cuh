// Step a1 of the hot path: parameter-derived constants, computed on the device
// from theta once per call, so that theta can stay in device memory and calls
// can be captured in CUDA graphs.  Two layouts share every arithmetic step
// (so they give bit-identical records): one thread per fit when many fits are
// evaluated at once, one four-warp block per fit when latency matters.
//
// Time part (Sec. 3, analytic normalisation): with F(tau) = [Phi(tau/sigma) -
// g(tau)] / Gamma, dF/dtau = g, the normalisation is I_T = F(t_hi - mu) -
// F(t_lo - mu).  Its derivatives: dF/dGamma = -(F + dg/dGamma) / Gamma,
// dF/dsigma = (-(tau/sigma) G(tau) - dg/dsigma) / Gamma, dF/dmu = -g(tau),
// where dg/dGamma = (Gamma sigma^2 - tau) g - sigma^2 G and
// dg/dsigma = Gamma^2 sigma g - (Gamma sigma + tau/sigma) G.
//
// Angular part (Sec. 4, P wave + S wave): amplitude magnitudes
// |A_0|^2 = (1-F_S) A0sq, |A_perp|^2 = (1-F_S) Apesq,
// |A_par|^2 = (1-F_S)(1 - A0sq - Apesq), |A_S|^2 = F_S, delta_0 = 0, and the
// ten coefficients h_k of the helicity-basis angular functions.
#pragma once

#include <math.h>

#include "ipa_internal.cuh"

namespace ipa {

namespace cdetail {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2Pi = 0.39894228040143267794;
constexpr double kPi = 3.14159265358979323846;

__device__ inline double conv_g(double tau, double Gamma, double sigma) {
    const double z = (Gamma * sigma * sigma - tau) / (kSqrt2 * sigma);
    return 0.5 * exp(-Gamma * tau + 0.5 * Gamma * Gamma * sigma * sigma) * erfc(z);
}

__device__ inline double gauss(double tau, double sigma) {
    const double x = tau / sigma;
    return kInvSqrt2Pi / sigma * exp(-0.5 * x * x);
}

// Normal CDF Phi(tau / sigma).
__device__ inline double edge_phi(double tau, double sigma) {
    return 0.5 * erfc(-tau / (kSqrt2 * sigma));
}

// F(tau) and its derivatives (Gamma, sigma, mu) at one edge of the range from
// g(tau), the Gaussian G(tau) and Phi(tau / sigma).
__device__ inline void edge_combine(double tau, double Gamma, double sigma, double g, double G, double Phi,
                                    double* F, double* dF) {
    const double dg_dG = (Gamma * sigma * sigma - tau) * g - sigma * sigma * G;
    const double dg_ds = Gamma * Gamma * sigma * g - (Gamma * sigma + tau / sigma) * G;
    *F = (Phi - g) / Gamma;
    dF[0] = -(*F + dg_dG) / Gamma;
    dF[1] = (-(tau / sigma) * G - dg_ds) / Gamma;
    dF[2] = -g;
}

// F(tau) and its derivatives (Gamma, sigma, mu) at one edge of the range.
__device__ inline void edge(double tau, double Gamma, double sigma, double* F, double* dF) {
    edge_combine(tau, Gamma, sigma, conv_g(tau, Gamma, sigma), gauss(tau, sigma), edge_phi(tau, sigma), F, dF);
}


// The transcendental inputs of the angular coefficients.
struct AngPieces {
    double sn[6], cs[6];   // sin/cos of (dpe - dpa), dpa, dpe, (dpa - dS), (dpe - dS), dS
    double rt[5];          // sqrt of x0, xa, xe, F, s
};

__device__ inline double ang_arg(int i, double dpa, double dpe, double dS) {
    switch (i) {
    case 0: return dpe - dpa;
    case 1: return dpa;
    case 2: return dpe;
    case 3: return dpa - dS;
    case 4: return dpe - dS;
    default: return dS;
    }
}

__device__ inline double sqrt_arg(int i, double x0, double xa, double xe, double F, double s) {
    switch (i) {
    case 0: return x0;
    case 1: return xa;
    case 2: return xe;
    case 3: return F;
    default: return s;
    }
}

// h_k and dh_k / d(A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S) for row k.
__device__ inline void h_row(int k, const AngPieces& a, double x0, double xe, double xa, double s, double F,
                             double* h, double* d) {
    const double s4 = a.sn[0], c4 = a.cs[0], s5 = a.sn[1], c5 = a.cs[1], s6 = a.sn[2], c6 = a.cs[2];
    const double s8 = a.sn[3], c8 = a.cs[3], s9 = a.sn[4], c9 = a.cs[4], s10 = a.sn[5], c10 = a.cs[5];
    const double r0 = a.rt[0], ra = a.rt[1], re = a.rt[2], rF = a.rt[3], rs = a.rt[4];
    const double rFs = rF * rs;
    const double dFs = (1.0 - 2.0 * F) / (2.0 * rFs);
    for (int j = 0; j < 6; ++j) d[j] = 0.0;
    switch (k) {
    case 0: *h = s * x0; d[0] = s; d[4] = -x0; break;
    case 1: *h = s * xa; d[0] = -s; d[1] = -s; d[4] = -xa; break;
    case 2: *h = s * xe; d[1] = s; d[4] = -xe; break;
    case 3:
        *h = s * ra * re * s4;
        d[0] = s * (-xe) / (2.0 * ra * re) * s4;
        d[1] = s * (xa - xe) / (2.0 * ra * re) * s4;
        d[2] = -s * ra * re * c4;
        d[3] = s * ra * re * c4;
        d[4] = -ra * re * s4;
        break;
    case 4:
        *h = s * r0 * ra * c5;
        d[0] = s * (xa - x0) / (2.0 * r0 * ra) * c5;
        d[1] = s * (-x0) / (2.0 * r0 * ra) * c5;
        d[2] = -s * r0 * ra * s5;
        d[4] = -r0 * ra * c5;
        break;
    case 5:
        *h = s * r0 * re * s6;
        d[0] = s * xe / (2.0 * r0 * re) * s6;
        d[1] = s * x0 / (2.0 * r0 * re) * s6;
        d[3] = s * r0 * re * c6;
        d[4] = -r0 * re * s6;
        break;
    case 6: *h = F; d[4] = 1.0; break;
    case 7:
        *h = rFs * ra * c8;
        d[0] = -rFs / (2.0 * ra) * c8;
        d[1] = -rFs / (2.0 * ra) * c8;
        d[2] = -rFs * ra * s8;
        d[4] = dFs * ra * c8;
        d[5] = rFs * ra * s8;
        break;
    case 8:
        *h = rFs * re * s9;
        d[1] = rFs / (2.0 * re) * s9;
        d[3] = rFs * re * c9;
        d[4] = dFs * re * s9;
        d[5] = -rFs * re * c9;
        break;
    default:
        *h = rFs * r0 * c10;
        d[0] = rFs / (2.0 * r0) * c10;
        d[4] = dFs * r0 * c10;
        d[5] = -rFs * r0 * s10;
        break;
    }
}

// max |f_k| over the angular box
__device__ inline double basis_max(int k) {
    switch (k) {
    case 0: return 1.0;
    case 1: case 2: case 3: return 0.5;
    case 4: case 5: return kSqrt2 / 4.0;
    case 6: return 1.0 / 3.0;
    case 7: case 8: return 0.40824829046386301637;
    default: return 1.15470053837925152902;
    }
}

__device__ inline double time_envelope(const ModelDev& m, double Gamma, double sigma, double mu) {
    return fmin(1.0, exp(-Gamma * (m.t_lo - mu) + 0.5 * Gamma * Gamma * sigma * sigma));
}

// The divisions of the record that need only theta and the model:
// k_z, k_g, cG, inv_s, cb, inv_V (numerator and denominator of item i).
__device__ inline void scalar_quotient(int i, const ModelDev& m, const double* th, double* num, double* den) {
    const double sigma = th[IPA_SIGMA], fb = th[IPA_FB];
    const bool four = m.kind == IPA_MODEL_ANGTIME4D;
    const double span = m.t_hi - m.t_lo;
    const double V = four ? span * 8.0 * kPi : span;
    switch (i) {
    case 0: *num = 1.0; *den = kSqrt2 * sigma; break;
    case 1: *num = 1.0; *den = 2.0 * sigma * sigma; break;
    case 2: *num = kInvSqrt2Pi; *den = sigma; break;
    case 3: *num = 1.0; *den = sigma; break;
    case 4: *num = fb; *den = V; break;
    default: *num = 1.0; *den = V; break;
    }
}
constexpr int kScalarQuotients = 6;

// The divisions by I_T: dlnIT[0..2], cs, inv_ITIO (numerator, denominator).
__device__ inline void it_quotient(int i, const ModelDev& m, const double* th, double IT, const double* dIT,
                                   double* num, double* den) {
    const double fb = th[IPA_FB];
    const double IO = m.kind == IPA_MODEL_ANGTIME4D ? 16.0 * kPi / 9.0 : 1.0;
    if (i < 3) {
        *num = dIT[i];
        *den = IT;
    } else {
        *num = i == 3 ? 1.0 - fb : 1.0;
        *den = IT * IO;
    }
}
constexpr int kItQuotients = 5;

// Whether theta lies in the model's domain: Gamma > 0, sigma > 0, f_b in
// [0, 1] and (4D) F_S, |A_0|^2, |A_perp|^2 and |A_par|^2 = 1 - |A_0|^2 -
// |A_perp|^2 in [0, 1] (false for NaN).  Outside, the PDF is not a density.
__device__ inline bool in_domain(const double* th, bool four) {
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], fb = th[IPA_FB];
    bool ok = Gamma > 0.0 && sigma > 0.0 && fb >= 0.0 && fb <= 1.0;
    if (four) {
        const double x0 = th[IPA_A0SQ], xe = th[IPA_APESQ], F = th[IPA_FS];
        ok = ok && F >= 0.0 && F <= 1.0 && x0 >= 0.0 && xe >= 0.0 && x0 + xe <= 1.0;
    }
    return ok;
}

// Scalars of the record without a division, and the quotients q[] of
// scalar_quotient (q[0..5]) and it_quotient (q[6..10]).  For theta outside the
// domain cs and cb are NaN, so that every P, the NLL and the gradient are NaN
// (the fitter reports such a point as IPA_FIT_BAD_PDF).
__device__ inline void write_plain_scalars(const double* th, double IT, double MT, double MO, bool four,
                                           const double* q, Consts* c) {
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU], fb = th[IPA_FB];
    const bool ok = in_domain(th, four);
    c->Gamma = Gamma;
    c->sigma = sigma;
    c->mu = mu;
    c->fb = fb;
    c->c_exp = 0.5 * Gamma * Gamma * sigma * sigma;
    c->Gs2 = Gamma * sigma * sigma;
    c->k_z = q[0];
    c->k_g = q[1];
    c->cG = q[2];
    c->s2 = sigma * sigma;
    c->G2s = Gamma * Gamma * sigma;
    c->Gsig = Gamma * sigma;
    c->inv_s = q[3];
    c->IT = IT;
    for (int j = 0; j < 3; ++j) c->dlnIT[j] = q[6 + j];
    c->MT = MT;
    c->MO = four ? MO : 1.0;
    c->cs = ok ? q[9] : NAN;
    c->cb = ok ? q[4] : NAN;
    c->inv_ITIO = q[10];
    c->inv_V = q[5];
    c->pad_ = 0.0;
}

// Scalars of the record from I_T pieces and the envelopes.
__device__ inline void write_scalars(const ModelDev& m, const double* th, double Fh, double Fl,
                                     const double* dIT, double MT, double MO, Consts* c) {
    const double IT = Fh - Fl;
    double q[kScalarQuotients + kItQuotients];
    for (int i = 0; i < kScalarQuotients; ++i) {
        double a, b;
        scalar_quotient(i, m, th, &a, &b);
        q[i] = a / b;
    }
    for (int i = 0; i < kItQuotients; ++i) {
        double a, b;
        it_quotient(i, m, th, IT, dIT, &a, &b);
        q[kScalarQuotients + i] = a / b;
    }
    write_plain_scalars(th, IT, MT, MO, m.kind == IPA_MODEL_ANGTIME4D, q, c);
}

struct AmpParams {
    double x0, xe, xa, s, F, dpa, dpe, dS;
};

__device__ inline AmpParams amp_params(const ModelDev& m, const double* th) {
    AmpParams p{};
    if (m.kind == IPA_MODEL_ANGTIME4D) {
        p.x0 = th[IPA_A0SQ];
        p.xe = th[IPA_APESQ];
        p.dpa = th[IPA_DPA];
        p.dpe = th[IPA_DPE];
        p.F = th[IPA_FS];
        p.dS = th[IPA_DS];
    }
    p.xa = 1.0 - p.x0 - p.xe;
    p.s = 1.0 - p.F;
    return p;
}

}  // namespace cdetail

// One thread computes one Consts record: used when many fits are evaluated at
// once (batched fits, the server), where lanes of a warp hold different fits
// and every FP64 instruction does useful work in all of them.
__device__ inline void compute_consts_thread(const ModelDev& m, const double* th, Consts* c) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU];
    double Fh, Fl, dFh[3], dFl[3];
    edge(m.t_hi - mu, Gamma, sigma, &Fh, dFh);
    edge(m.t_lo - mu, Gamma, sigma, &Fl, dFl);
    double dIT[3];
    for (int j = 0; j < 3; ++j) dIT[j] = dFh[j] - dFl[j];
    const double MT = time_envelope(m, Gamma, sigma, mu);
    const AmpParams p = amp_params(m, th);
    double MO = 0.0;
    if (m.kind == IPA_MODEL_ANGTIME4D) {
        AngPieces a;
        for (int i = 0; i < 6; ++i) sincos(ang_arg(i, p.dpa, p.dpe, p.dS), &a.sn[i], &a.cs[i]);
        for (int i = 0; i < 5; ++i) a.rt[i] = sqrt(sqrt_arg(i, p.x0, p.xa, p.xe, p.F, p.s));
        for (int k = 0; k < 10; ++k) {
            double h, d[6];
            h_row(k, a, p.x0, p.xe, p.xa, p.s, p.F, &h, d);
            c->h[k] = h;
            for (int j = 0; j < 6; ++j) c->dh[k][j] = d[j];
            MO = k ? MO + fabs(h) * basis_max(k) : fabs(h) * basis_max(k);
        }
    } else {
        for (int k = 0; k < 10; ++k) {
            c->h[k] = k == 0 ? 1.0 : 0.0;
            for (int j = 0; j < 6; ++j) c->dh[k][j] = 0.0;
        }
    }
    write_scalars(m, th, Fh, Fl, dIT, MT, MO, c);
}

// Exchange buffer of compute_consts_block.
struct ConstsBlockScratch {
    double g[2], G[2], Phi[2];     // edge 0: t_hi, edge 1: t_lo
    double F[2], dF[2][3];
    double MT, MO;
    cdetail::AngPieces a;
    double q[cdetail::kScalarQuotients + cdetail::kItQuotients];
    double h[10], d[10][6];
};

// One block of 128 threads (four warps, one per SM sub-partition) computes one
// Consts record: a single fit, where latency matters.  On this GPU a warp's
// FP64 instruction occupies its sub-partition's FP64 unit for tens of cycles
// whatever the active lanes, so the record's independent pieces go to
// different warps and, within a warp, to lanes running the same code:
//   phase 1  warp 0: g at both edges (exp, erfc); warp 1: Phi at both edges
//            (erfc); warp 2: the Gaussian at both edges and the envelope M_T;
//            warp 3: six sine/cosine pairs, five square roots and the six
//            divisions that need theta only;
//   phase 2  warp 0: F and its derivatives at both edges; warps 1-3: the ten
//            rows of h and dh (at most two rows with divisions per warp);
//   phase 3  warp 0: the five divisions by I_T; warp 1: M_Omega.
// Every value comes from the same expression as in compute_consts_thread, so
// both give the same bits (this file is compiled without FMA contraction).
__device__ inline void compute_consts_block(const ModelDev& m, const double* th, Consts* c,
                                            ConstsBlockScratch* S) {
    using namespace cdetail;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU];
    const bool four = m.kind == IPA_MODEL_ANGTIME4D;
    const AmpParams p = amp_params(m, th);
    const double tau_e = (lane == 0 ? m.t_hi : m.t_lo) - mu;
    if (w == 0) {
        if (lane < 2) S->g[lane] = conv_g(tau_e, Gamma, sigma);
    } else if (w == 1) {
        if (lane < 2) S->Phi[lane] = edge_phi(tau_e, sigma);
    } else if (w == 2) {
        if (lane < 2) S->G[lane] = gauss(tau_e, sigma);
        else if (lane == 2) S->MT = time_envelope(m, Gamma, sigma, mu);
    } else if (w == 3) {
        if (lane < 6) {
            if (four) sincos(ang_arg(lane, p.dpa, p.dpe, p.dS), &S->a.sn[lane], &S->a.cs[lane]);
        } else if (lane < 11) {
            if (four) S->a.rt[lane - 6] = sqrt(sqrt_arg(lane - 6, p.x0, p.xa, p.xe, p.F, p.s));
        } else if (lane < 11 + kScalarQuotients) {
            double num, den;
            scalar_quotient(lane - 11, m, th, &num, &den);
            S->q[lane - 11] = num / den;
        }
    }
    __syncthreads();
    // rows of h: warp 1 -> 0, 3, 4; warp 2 -> 1, 5, 7; warp 3 -> 2, 6, 8, 9
    int k = -1;
    if (w == 0) {
        if (lane < 2) edge_combine(tau_e, Gamma, sigma, S->g[lane], S->G[lane], S->Phi[lane], &S->F[lane], S->dF[lane]);
    } else if (w == 1) {
        k = lane == 0 ? 0 : (lane == 1 ? 3 : (lane == 2 ? 4 : -1));
    } else if (w == 2) {
        k = lane == 0 ? 1 : (lane == 1 ? 5 : (lane == 2 ? 7 : -1));
    } else if (w == 3) {
        k = lane == 0 ? 2 : (lane == 1 ? 6 : (lane == 2 ? 8 : (lane == 3 ? 9 : -1)));
    }
    if (k >= 0) {
        double h = k == 0 ? 1.0 : 0.0, d[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (four) h_row(k, S->a, p.x0, p.xe, p.xa, p.s, p.F, &h, d);
        S->h[k] = h;
        for (int j = 0; j < 6; ++j) S->d[k][j] = d[j];
    }
    __syncthreads();
    const double IT = S->F[0] - S->F[1];
    if (w == 0 && lane < kItQuotients) {
        double dIT[3];
        for (int j = 0; j < 3; ++j) dIT[j] = S->dF[0][j] - S->dF[1][j];
        double num, den;
        it_quotient(lane, m, th, IT, dIT, &num, &den);
        S->q[kScalarQuotients + lane] = num / den;
    } else if (w == 1 && lane == 0) {
        double MO = 0.0;
        if (four)
            for (int r = 0; r < 10; ++r)
                MO = r ? MO + fabs(S->h[r]) * basis_max(r) : fabs(S->h[r]) * basis_max(r);
        S->MO = MO;
    }
    __syncthreads();
    if (threadIdx.x == 0) write_plain_scalars(th, IT, S->MT, S->MO, four, S->q, c);
    if (threadIdx.x < 60) c->dh[threadIdx.x / 6][threadIdx.x % 6] = S->d[threadIdx.x / 6][threadIdx.x % 6];
    if (threadIdx.x >= 64 && threadIdx.x < 74) c->h[threadIdx.x - 64] = S->h[threadIdx.x - 64];
}

}  // namespace ipa
