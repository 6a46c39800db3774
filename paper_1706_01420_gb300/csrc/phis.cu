// Hot path of the full time-dependent angular model with tagging (the phi_s
// fit of Sec. 4; formulas in ipanema.h): constants, the likelihood with its
// fused gradient, and the deterministic reduction.
//
// Coefficient form.  Each angular term k is a bilinear b_k = conj(A_i) A_j of
// transversity amplitudes with CP eigenvalues eta_i, eta_j; with the time
// evolution its tag-mixed rate is a combination of four convolved time
// functions, G = (g_L, g_H, q Re g_c, q Im g_c) (g_c = g(tau; Gamma - i Dm)):
//   rate(t, Omega, q) = sum_k f_k sum_j C_kj G_j,
// where, with c, s = cos, sin phi_s and D = 1 - 2 omega, for
//   eta_i = eta_j = eta:   part(b) (1 + eta c)/2, part(b) (1 - eta c)/2, 0, D eta s part(b),
//   eta_i = -eta_j, eta = eta_j, real part:
//       eta s Im b / 2, -eta s Im b / 2, D Re b, -D eta c Im b,
//   imaginary part:
//       -eta s Re b / 2, eta s Re b / 2, D Im b, D eta c Re b
// (part = Re or Im as the term takes; the products of g+- are written out
// in ipanema.h).  Per event: the ten f'_k (integer pipe), the four time
// functions (as in tagged.cu), F_j = sum_k Cq_kj f'_k, P = sum_j F_j G_j + cb.
//
// Gradient.  Amplitude, phase and mistag parameters act only through C: the
// pass accumulates S_kj = sum_e r f'_k G_j (40 sums) and the segment's finalise
// contracts them with dC/dtheta.  The five time parameters act through the G_j:
// each event adds r sum_j F_j dG_j/dtheta (5 sums, the derivatives written out
// from dg/dz = (z sigma^2 - tau) g - sigma^2 G, dg/dsigma = z^2 sigma g -
// (z sigma + tau/sigma) G, dg/dtau = -z g + G).  With Q = sum r: 47 sums.
#include <math.h>

#include "angular.cuh"
#include "consts.cuh"
#include "faddeeva.cuh"
#include "fp64_math.cuh"
#include "int_math.cuh"
#include "ipa_internal.cuh"
#include "philox.cuh"
#include "phis_consts.cuh"
#include "tagged.cuh"
#include "tile_reduce.cuh"

namespace ipa {
namespace {

constexpr int kPerLane = kTile / 32;
constexpr int kSub = 4;
constexpr int kMaxWarps = 8;
constexpr int kTeam = kPerLane / kSub;   // warps that share a tile: each takes kSub of a lane's events
constexpr int kNA = 47;          // accumulators with the gradient (n_acc of the phi_s model)
static_assert(kNA == n_acc(IPA_MODEL_PHIS, true) && kNA <= kMaxAcc, "the scratch must hold the accumulators");
constexpr int kS = 2;            // first S_kj
constexpr int kT = 42;           // first time-parameter sum (Gamma, sigma, mu, DG, Dm)
__device__ const double kEta[4] = {1.0, 1.0, -1.0, -1.0};

// (i, j, imaginary part?) of the ten bilinears conj(A_i) A_j (0, para, perp, S)
__device__ const int kPairI[10] = {0, 1, 2, 1, 0, 0, 3, 3, 3, 3};
__device__ const int kPairJ[10] = {0, 1, 2, 2, 1, 2, 3, 1, 2, 0};
__device__ const int kPairIm[10] = {0, 0, 0, 1, 0, 1, 0, 0, 1, 0};

// Row factor: C_SP for the S-P interference terms, 1 otherwise.
__device__ __forceinline__ double row_scale(const PhisConsts& c, int k) { return k >= 7 ? c.csp : 1.0; }

// Row k of C from part(b) pieces: pr = Re b, pi = Im b.  Every entry is a
// product of part(b), one of (one, c, s) and of wu (untagged entries) or wt
// (tagged entries, D), so that with (one, c, s) = (1, cos, sin phi_s) and
// (wu, wt) = (1, D) it is C itself, with (0, -sin, cos) its derivative in
// phi_s, and with (wu, wt) = (0, -2) its derivative in omega.
__device__ inline void c_row(int k, double pr, double pi, double one, double c, double s, double wu, double wt,
                             double* out) {
    const double ei = kEta[kPairI[k]], ej = kEta[kPairJ[k]];
    if (ei == ej) {
        const double p = kPairIm[k] ? pi : pr;
        out[0] = wu * 0.5 * p * (one + ej * c);
        out[1] = wu * 0.5 * p * (one - ej * c);
        out[2] = 0.0;
        out[3] = wt * ej * s * p;
    } else if (!kPairIm[k]) {
        out[0] = wu * 0.5 * ej * s * pi;
        out[1] = -wu * 0.5 * ej * s * pi;
        out[2] = wt * one * pr;
        out[3] = -wt * ej * c * pi;
    } else {
        out[0] = -wu * 0.5 * ej * s * pr;
        out[1] = wu * 0.5 * ej * s * pr;
        out[2] = wt * one * pi;
        out[3] = wt * ej * c * pr;
    }
}

// d b_k / d(A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S), parameter a: b_k =
// m e^{i psi} with the magnitude m a product of square roots and the phase psi
// a difference of strong phases.
__device__ inline void b_deriv(const PhisConsts& c, int k, int a, double* dr, double* di) {
    const double sF = c.rs * c.rs;
    double dm = 0.0, dpsi = 0.0, m = 0.0, cp = 1.0, sp = 0.0;
    const double r0 = c.r0, ra = c.ra, re = c.re, rF = c.rF, rs = c.rs;
    const double rFs = rF * rs, dFs = (1.0 - 2.0 * c.F) / (2.0 * rFs);
    switch (k) {
    case 0: m = sF * c.x0; dm = a == 0 ? sF : (a == 4 ? -c.x0 : 0.0); break;
    case 1: m = sF * c.xa; dm = (a == 0 || a == 1) ? -sF : (a == 4 ? -c.xa : 0.0); break;
    case 2: m = sF * c.xe; dm = a == 1 ? sF : (a == 4 ? -c.xe : 0.0); break;
    case 3:   // para, perp: psi = dpe - dpa
        m = sF * ra * re;
        dm = a == 0 ? sF * (-c.xe) / (2.0 * ra * re)
           : a == 1 ? sF * (c.xa - c.xe) / (2.0 * ra * re)
           : a == 4 ? -ra * re : 0.0;
        dpsi = a == 2 ? -1.0 : (a == 3 ? 1.0 : 0.0);
        cp = c.cw[0]; sp = c.sw[0];
        break;
    case 4:   // 0, para: psi = dpa
        m = sF * r0 * ra;
        dm = a == 0 ? sF * (c.xa - c.x0) / (2.0 * r0 * ra)
           : a == 1 ? sF * (-c.x0) / (2.0 * r0 * ra)
           : a == 4 ? -r0 * ra : 0.0;
        dpsi = a == 2 ? 1.0 : 0.0;
        cp = c.cw[1]; sp = c.sw[1];
        break;
    case 5:   // 0, perp: psi = dpe
        m = sF * r0 * re;
        dm = a == 0 ? sF * c.xe / (2.0 * r0 * re)
           : a == 1 ? sF * c.x0 / (2.0 * r0 * re)
           : a == 4 ? -r0 * re : 0.0;
        dpsi = a == 3 ? 1.0 : 0.0;
        cp = c.cw[2]; sp = c.sw[2];
        break;
    case 6: m = c.F; dm = a == 4 ? 1.0 : 0.0; break;
    case 7:   // S, para: psi = dpa - dS
        m = rFs * ra;
        dm = (a == 0 || a == 1) ? -rFs / (2.0 * ra) : (a == 4 ? dFs * ra : 0.0);
        dpsi = a == 2 ? 1.0 : (a == 5 ? -1.0 : 0.0);
        cp = c.cw[3]; sp = c.sw[3];
        break;
    case 8:   // S, perp: psi = dpe - dS
        m = rFs * re;
        dm = a == 1 ? rFs / (2.0 * re) : (a == 4 ? dFs * re : 0.0);
        dpsi = a == 3 ? 1.0 : (a == 5 ? -1.0 : 0.0);
        cp = c.cw[4]; sp = c.sw[4];
        break;
    default:  // S, 0: psi = -dS
        m = rFs * r0;
        dm = a == 0 ? rFs / (2.0 * r0) : (a == 4 ? dFs * r0 : 0.0);
        dpsi = a == 5 ? -1.0 : 0.0;
        cp = c.cw[5]; sp = -c.sw[5];
        break;
    }
    *dr = dm * cp - m * dpsi * sp;
    *di = dm * sp + m * dpsi * cp;
}

// Per-warp copy: the record and Cq_kj = (cs / 2) C_kj c_k (the basis factor c_k
// for the unscaled f'_k, 1 for a cached basis; 1/2 for the doubled G).
struct PhisWarp {
    PhisConsts c;
    double cq[40];
};

// One event: log term and, with GRAD, the 45 sums.  G2 = 2 G (doubled as in tagged.cu).
template <bool GRAD, bool WEIGHTED>
__device__ __forceinline__ void phis_event(const PhisWarp& pw, const MathTables* mt, double t, double q, double w,
                                           const double* f, const TagSlow& sl, double* acc, double* prod,
                                           int* esum) {
    const PhisConsts& c = pw.c;
    const double tau = t - c.mu;
    const double E2H = exp_int(fma(-c.GH, tau, c.cH2), mt);
    const double E2L = exp_int(fma(-c.GL, tau, c.cL2), mt);
    const double E2C = exp_int(fma(-c.Gamma, tau, c.cC2), mt);
    double sn, cn;
    sincos_int_wide(fma(c.Dm, tau, -c.ph0), mt, &sn, &cn);
    const long long bH = __double_as_longlong(sl.xH), bL = __double_as_longlong(sl.xL);
    const long long bG = __double_as_longlong(sl.gx);
    const double T2H = bH < 0 ? -sl.xH : E2H - sl.xH;
    const double T2L = bL < 0 ? -sl.xL : E2L - sl.xL;
    const double Cr = bG < 0 ? sl.wr : fma(E2C, cn, -sl.wr);
    const double Ci = bG < 0 ? sl.wi : fma(E2C, sn, -sl.wi);
    const double gx = __longlong_as_double(bG & 0x7FFFFFFFFFFFFFFFll);
    const double G2[4] = {T2L, T2H, q * Cr, q * Ci};
    double Fw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double v = pw.cq[j] * f[0];
#pragma unroll
        for (int k = 1; k < 10; ++k) v = fma(pw.cq[4 * k + j], f[k], v);
        Fw[j] = v;
    }
    const double P = fma(Fw[0], G2[0], fma(Fw[1], G2[1], fma(Fw[2], G2[2], fma(Fw[3], G2[3], c.cb))));
    if (WEIGHTED && __double_as_longlong(w) != 0x3FF0000000000000ll)
        acc[0] = fma(w, log_fast(P, mt), acc[0]);
    else
        log_mul(P, prod, esum);
    if (!GRAD) return;
    const double r = WEIGHTED ? w * rcp_newton(P) : rcp_newton(P);
    acc[1] += r;
    double rG[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) rG[j] = r * G2[j];
#pragma unroll
    for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[kS + 4 * k + j] = fma(f[k], rG[j], acc[kS + 4 * k + j]);
    // derivatives of the doubled time functions; G2g = 2 G (the Gaussian density)
    const double G2g = 2.0 * c.cG * gx;
    const double s2 = c.s2, sg = c.sigma, its = tau * c.inv_s;
    const double dL_G = fma(c.GL * s2 - tau, T2L, -s2 * G2g);
    const double dH_G = fma(c.GH * s2 - tau, T2H, -s2 * G2g);
    const double dL_s = fma(c.GL * c.GL * sg, T2L, -(c.GL * sg + its) * G2g);
    const double dH_s = fma(c.GH * c.GH * sg, T2H, -(c.GH * sg + its) * G2g);
    const double dL_t = fma(-c.GL, T2L, G2g);
    const double dH_t = fma(-c.GH, T2H, G2g);
    // complex: z = Gamma - i Dm
    const double a0 = c.Gamma * s2 - tau, dms2 = c.Dm * s2;
    const double zr = fma(a0, Cr, fma(dms2, Ci, -s2 * G2g));       // Re d(2g_c)/dz
    const double zi = fma(a0, Ci, -dms2 * Cr);                      // Im d(2g_c)/dz
    const double g2 = (c.Gamma - c.Dm) * (c.Gamma + c.Dm), gd2 = 2.0 * c.Gamma * c.Dm;
    const double sr = fma(sg, fma(g2, Cr, gd2 * Ci), -(c.Gamma * sg + its) * G2g);   // Re d/dsigma
    const double si = fma(sg, fma(g2, Ci, -gd2 * Cr), c.Dm * sg * G2g);               // Im d/dsigma
    const double tr = -fma(c.Gamma, Cr, c.Dm * Ci) + G2g;                               // Re d/dtau
    const double ti = -fma(c.Gamma, Ci, -c.Dm * Cr);                                    // Im d/dtau
    const double qF2 = q * Fw[2], qF3 = q * Fw[3];
    const double dG = fma(Fw[0], dL_G, fma(Fw[1], dH_G, fma(qF2, zr, qF3 * zi)));
    const double dS = fma(Fw[0], dL_s, fma(Fw[1], dH_s, fma(qF2, sr, qF3 * si)));
    const double dT = -fma(Fw[0], dL_t, fma(Fw[1], dH_t, fma(qF2, tr, qF3 * ti)));
    const double dDG = 0.5 * fma(Fw[0], dL_G, -Fw[1] * dH_G);
    const double dDm = fma(qF2, zi, -qF3 * zr);                     // d/dDm = -i d/dz
    acc[kT + 0] = fma(r, dG, acc[kT + 0]);
    acc[kT + 1] = fma(r, dS, acc[kT + 1]);
    acc[kT + 2] = fma(r, dT, acc[kT + 2]);
    acc[kT + 3] = fma(r, dDG, acc[kT + 3]);
    acc[kT + 4] = fma(r, dDm, acc[kT + 4]);
}

// NLL and gradient of one segment (every lane holds acc; lane j writes
// component j).  With S2_kj = c_k S_kj (the scaled basis), SR = sum r rate =
// (1/2) sum_kj C_kj S2_kj, the time sums D_t = cs sum r d rate / d theta_t:
//   time parameters:            -D_t + cs dlnN_t SR,
//   f_b:                        SR / N - Q / V,
//   amplitudes, phi_s, omega, C_SP:  -(cs/2) sum_kj dC_kj/dtheta S2_kj + cs dlnN SR
// (C rows 7, 8, 9 carry C_SP).
template <bool GRAD, bool CACHED>
__device__ __forceinline__ void phis_finalize(const PhisConsts& c, const double* acc, int n_par, double* out, int lane) {
    if (lane == 0) out[0] = -acc[0];
    if (!GRAD) return;
    // (loops unrolled: acc stays in registers)
    double SR = 0.0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        double row[4];
        c_row(k, c.br[k], c.bi[k], 1.0, c.c, c.s, 1.0, c.D, row);
        const double sc = row_scale(c, k) * (CACHED ? 1.0 : kBasisScale[k]);
#pragma unroll
        for (int j = 0; j < 4; ++j) SR = fma(row[j], sc * acc[kS + 4 * k + j], SR);
    }
    SR *= 0.5;
    const double csSR = c.cs * SR;
    if (lane >= IPA_NPAR_PHIS) {
        for (int j = lane; j < n_par; j += 32) out[1 + j] = 0.0;
        return;
    }
    double v;
    if (lane == IPA_FB) {
        v = fma(SR, c.inv_N, -acc[1] * c.inv_V);
    } else if (lane == IPA_PHIS_QNORM) {
        v = 0.0;
    } else if (lane < 3 || lane == IPA_PHIS_DG || lane == IPA_PHIS_DM) {
        // register operands only (an index computed from the lane would put acc in local memory)
        const double Dt = lane == 0 ? acc[kT] : lane == 1 ? acc[kT + 1] : lane == 2 ? acc[kT + 2]
                        : lane == IPA_PHIS_DG ? acc[kT + 3] : acc[kT + 4];
        v = fma(c.dlnN[lane], csSR, -Dt);
    } else {
        double dsum = 0.0;
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            double row[4];
            double rs = row_scale(c, k);
            if (lane == IPA_PHIS_PHIS) {
                c_row(k, c.br[k], c.bi[k], 0.0, -c.s, c.c, 1.0, c.D, row);
            } else if (lane == IPA_PHIS_OMEGA) {
                c_row(k, c.br[k], c.bi[k], 1.0, c.c, c.s, 0.0, -2.0, row);
            } else if (lane == IPA_PHIS_CSP) {
                c_row(k, c.br[k], c.bi[k], 1.0, c.c, c.s, 1.0, c.D, row);
                rs = k >= 7 ? 1.0 : 0.0;
            } else {
                double dr, di;
                b_deriv(c, k, lane - IPA_A0SQ, &dr, &di);
                c_row(k, dr, di, 1.0, c.c, c.s, 1.0, c.D, row);
            }
            const double sc = rs * (CACHED ? 1.0 : kBasisScale[k]);
#pragma unroll
            for (int j = 0; j < 4; ++j) dsum = fma(row[j], sc * acc[kS + 4 * k + j], dsum);
        }
        v = fma(c.dlnN[lane], csSR, -0.5 * c.cs * dsum);
    }
    out[1 + lane] = v;
    for (int j = IPA_NPAR_PHIS + lane; j < n_par; j += 32) out[1 + j] = 0.0;
}

template <bool GRAD, bool WEIGHTED, bool CACHED>
__global__ void __launch_bounds__(32 * kTeam, 1)
phis_kernel(Cols cols, int64_t n, const int64_t* __restrict__ seg_begin, const int64_t* __restrict__ seg_end,
            const int64_t* __restrict__ seg_tiles, int n_seg, const Consts* __restrict__ consts,
            double* __restrict__ partials, unsigned* __restrict__ counters, unsigned* __restrict__ gcount,
            unsigned* __restrict__ work, double* __restrict__ out, int n_par, int per_take) {
    constexpr int NA = GRAD ? kNA : 1;
    const int out_stride = GRAD ? 1 + n_par : 1;
    __shared__ MathTables mt;
    __shared__ int64_t s_take;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n_wib = kTeam;
    TagSlow* const sbuf = reinterpret_cast<TagSlow*>(dyn_smem) + wib * (kSub * 32);
    PhisWarp& pw = reinterpret_cast<PhisWarp*>(dyn_smem + (size_t)n_wib * kSub * 32 * sizeof(TagSlow))[wib];
    double* const xbuf = reinterpret_cast<double*>(dyn_smem + (size_t)n_wib * (kSub * 32 * sizeof(TagSlow) +
                                                                               sizeof(PhisWarp)));
    double* const xtot = xbuf + (size_t)kTeam * NA * 32;

    load_math_tables(&mt);
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const bool single = seg_begin == nullptr;
    const int64_t total = single ? (n + kTile - 1) / kTile : __ldg(seg_tiles + n_seg);
    if (blockIdx.x == 0) {
        for (int s = threadIdx.x; s < n_seg; s += blockDim.x) {
            const bool empty = single ? (n == 0) : (__ldg(seg_tiles + s + 1) == __ldg(seg_tiles + s));
            if (empty)
                for (int j = 0; j < out_stride; ++j) out[(size_t)s * out_stride + j] = 0.0;
        }
    }

    int cur = -1;
    while (true) {
        // the team (the block's four warps) takes tiles together
        if (threadIdx.x == 0) s_take = (int64_t)atomicAdd(work, 1u) * per_take;
        __syncthreads();
        const int64_t first = s_take;
        __syncthreads();
        if (first >= total) break;
        const int64_t stop = first + per_take < total ? first + per_take : total;
        for (int64_t tile = first; tile < stop; ++tile) {
            int seg = 0;
            int64_t t0 = 0, t1 = total, ev0 = 0, ev1 = n;
            if (!single) {
                seg = find_segment(seg_tiles, n_seg, tile);
                t0 = __ldg(seg_tiles + seg);
                t1 = __ldg(seg_tiles + seg + 1);
                ev0 = clamp_off(__ldg(seg_begin + seg), n);
                ev1 = clamp_off(__ldg(seg_end + seg), n);
                if (ev1 < ev0) ev1 = ev0;
            }
            if (seg != cur) {
                __syncwarp();
                const double* src = reinterpret_cast<const double*>(consts + seg);
                double* dst = reinterpret_cast<double*>(&pw.c);
                for (int i = lane; i < kPhisDoubles; i += 32) dst[i] = __ldg(src + i);
                __syncwarp();
                if (lane < 10) {
                    double row[4];
                    c_row(lane, pw.c.br[lane], pw.c.bi[lane], 1.0, pw.c.c, pw.c.s, 1.0, pw.c.D, row);
                    const double sc = 0.5 * pw.c.cs * row_scale(pw.c, lane) * (CACHED ? 1.0 : kBasisScale[lane]);
                    for (int j = 0; j < 4; ++j) pw.cq[4 * lane + j] = sc * row[j];
                }
                __syncwarp();
                cur = seg;
            }

            double acc[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) acc[a] = 0.0;
            double prod = 1.0;
            int esum = 0;
            const int64_t tbase = ev0 + (tile - t0) * kTile;
            const unsigned below = (1u << lane) - 1u;
            // warp w of the team takes events [4 w, 4 w + 4) of each lane's 16
            {
                const int i0 = wib * kSub;
                unsigned m0, m1, m2, m3;
                {
                    unsigned mk[kSub];
#pragma unroll
                    for (int k = 0; k < kSub; ++k) {
                        const int64_t e = tbase + lane + 32 * (i0 + k);
                        const bool slow = e < ev1 && !greater(__ldg(cols.t + e), pw.c.tcut);
                        mk[k] = __ballot_sync(0xffffffffu, slow);
                    }
                    m0 = mk[0];
                    m1 = mk[1];
                    m2 = mk[2];
                    m3 = mk[3];
                }
                const int p1 = __popc(m0), p2 = p1 + __popc(m1), p3 = p2 + __popc(m2);
                const int n_slow = p3 + __popc(m3);
                for (int j = lane; j < n_slow; j += 32) {
                    const int k = (j >= p1) + (j >= p2) + (j >= p3);
                    const unsigned m = k == 0 ? m0 : (k == 1 ? m1 : (k == 2 ? m2 : m3));
                    const int before = k == 0 ? 0 : (k == 1 ? p1 : (k == 2 ? p2 : p3));
                    const int64_t e = tbase + nth_set(m, j - before) + 32 * (i0 + k);
                    sbuf[j] = tag_slow(pw.c, __ldg(cols.t + e) - pw.c.mu, &mt);
                }
                __syncwarp();
#pragma unroll 1
                for (int k = 0; k < kSub; ++k) {
                    const int64_t e = tbase + lane + 32 * (i0 + k);
                    if (e < ev1) {
                        const unsigned m = k == 0 ? m0 : (k == 1 ? m1 : (k == 2 ? m2 : m3));
                        const int before = k == 0 ? 0 : (k == 1 ? p1 : (k == 2 ? p2 : p3));
                        TagSlow sl = {0.0, 0.0, 0.0, 0.0, 0.0};
                        if ((m >> lane) & 1u) sl = sbuf[before + __popc(m & below)];
                        const double w = WEIGHTED ? __ldg(cols.w + e) : 1.0;
                        double f[10];
                        if (CACHED) {
#pragma unroll
                            for (int kk = 0; kk < 10; ++kk) f[kk] = __ldg(cols.fk + kk * cols.fk_stride + e);
                        } else {
                            basis_unscaled(__ldg(cols.ck + e), __ldg(cols.cl + e), __ldg(cols.phi + e), &mt, f);
                        }
                        phis_event<GRAD, WEIGHTED>(pw, &mt, __ldg(cols.t + e), __ldg(cols.q + e), w, f, sl, acc,
                                                   &prod, &esum);
                    }
                }
                __syncwarp();
            }
            acc[0] += log_of(prod, esum, &mt);
            // every warp's sums to shared memory; warp w then reduces accumulators
            // w, w + 4, ...: the team's four values lane by lane in warp order, then
            // the xor butterfly over the lanes (the reduction work spread over the
            // four sub-partitions); warp 0 commits the tile
#pragma unroll
            for (int a = 0; a < NA; ++a) xbuf[(wib * NA + a) * 32 + lane] = acc[a];
            __syncthreads();
            for (int a = wib; a < NA; a += kTeam) {
                double v = xbuf[a * 32 + lane];
                for (int w = 1; w < kTeam; ++w) v += xbuf[(w * NA + a) * 32 + lane];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) xtot[a] = v;
            }
            __syncthreads();
            if (wib == 0) {
#pragma unroll
                for (int a = 0; a < NA; ++a) acc[a] = xtot[a];
                if (tile_commit_wide<NA>(lane, tile, t0, t1, seg, partials, gcount, counters, acc)) {
                    phis_finalize<GRAD, CACHED>(pw.c, acc, n_par, out + (size_t)seg * out_stride, lane);
                    if (lane == 0) counters[seg] = 0u;
                }
            }
            __syncthreads();
        }
    }
    work_done(work, lane);
}

template <bool GRAD, bool WEIGHTED, bool CACHED>
ipa_status launch_phis_t(const Cols& cols, int64_t n, const int64_t* seg_begin, const int64_t* seg_end,
                         const int64_t* seg_tiles, int n_seg, const Consts* consts, Scratch* sc, double* out,
                         int n_par, cudaStream_t st, const LaunchCfg* force) {
    const bool single = seg_begin == nullptr;
    const int64_t tiles = tile_estimate(n, n_seg);
    if (GRAD && single && sc->partials_cap < (size_t)((n + kTile - 1) / kTile) * kNA) {
        set_error("phi_s likelihood: the scratch holds too few accumulators per tile");
        return IPA_ERR_ARG;
    }
    const LaunchCfg cfg = force ? *force : launch_cfg(IPA_MODEL_PHIS, GRAD, CACHED, n_seg > 1, tiles);
    // one block = one team of four warps sharing each tile (the geometry's
    // warps per block does not apply; its tiles per take and resident blocks do)
    const int W = kTeam;
    const int K = cfg.tiles_per_take >= 1 ? cfg.tiles_per_take : 1;
    const size_t per_warp = sizeof(PhisWarp) + kSub * 32 * sizeof(TagSlow);
    constexpr int NA = GRAD ? kNA : 1;
    const size_t smem = (size_t)W * per_warp + ((size_t)kTeam * NA * 32 + NA) * sizeof(double);
    auto kern = phis_kernel<GRAD, WEIGHTED, CACHED>;
    static bool attr[64] = {};
    static int occ[64][kMaxWarps + 1] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr[dev & 63]) {
        ipa_status q = cuda_fail(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                 "phi_s kernel attribute");
        if (q != IPA_OK) return q;
        attr[dev & 63] = true;
    }
    int& per_sm = occ[dev & 63][W];
    if (per_sm == 0) {
        int v = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, 32 * W, smem);
        per_sm = e == cudaSuccess && v >= 1 ? v : 1;
    }
    const int64_t grid = launch_grid(cfg, W, K, per_sm, tiles, single);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(32u * W);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = la;
    lc.numAttrs = 1;
    return cuda_fail(cudaLaunchKernelEx(&lc, kern, cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts,
                                        sc->partials, sc->counters, sc->gcount, sc->work, out, n_par, K),
                     "phi_s likelihood kernel launch");
}

template <bool GRAD, bool CACHED>
ipa_status launch_phis_w(const Cols& cols, int64_t n, const int64_t* seg_begin, const int64_t* seg_end,
                         const int64_t* seg_tiles, int n_seg, const Consts* consts, Scratch* sc, double* out,
                         int n_par, cudaStream_t st, const LaunchCfg* cfg) {
    if (cols.w)
        return launch_phis_t<GRAD, true, CACHED>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out,
                                                 n_par, st, cfg);
    return launch_phis_t<GRAD, false, CACHED>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, n_par,
                                              st, cfg);
}

// ---- generator (Sec. 7, Example 5: accept-reject with counter-based draws) ----

constexpr int kGenBins = 64;    // decay-time bins of the generator's envelope

// The envelope, piecewise constant in t: bin i = [e_i, e_i + w), e_i = t_lo +
// i w, w = (t_hi - t_lo) / 64, bound B_i >= rate there.  Every observed
// bilinear is at most |b_k| (gL + gH + 2 |gc|) and a convolved exponential
// g(tau; x) decreases in tau and is at most min(1, e^{-x tau + x^2 sigma^2 /
// 2}), taken at the left edge: B_i = (m(Gamma_L) + m(Gamma_H) + 2 m(Gamma))
// sum_k max|f_k| |b_k| r_k (r_k = |C_SP| for the S-P terms).  C: running sums of
// B in order (C_0 = 0), the proposal's cumulative weights.  One thread.
__device__ void phis_envelope_bins(const PhisConsts& c, const ModelDev& m, double w, double* B, double* C) {
    using namespace cdetail;
    const double sF = 1.0 - c.F, rFs = c.rF * c.rs;
    const double mag[10] = {sF * c.x0, sF * c.xa, sF * c.xe, sF * c.ra * c.re, sF * c.r0 * c.ra, sF * c.r0 * c.re,
                            c.F, rFs * c.ra, rFs * c.re, rFs * c.r0};
    double ang = 0.0;
    for (int k = 0; k < 10; ++k) ang += basis_max(k) * mag[k] * (k >= 7 ? fabs(c.csp) : 1.0);
    C[0] = 0.0;
    for (int i = 0; i < kGenBins; ++i) {
        const double e = __dadd_rn(m.t_lo, __dmul_rn((double)i, w)) - c.mu;
        const double ML = fmin(1.0, exp(-c.GL * e + 0.5 * c.GL * c.GL * c.s2));
        const double MH = fmin(1.0, exp(-c.GH * e + 0.5 * c.GH * c.GH * c.s2));
        const double MG = fmin(1.0, exp(-c.Gamma * e + 0.5 * c.Gamma * c.Gamma * c.s2));
        B[i] = (ML + MH + 2.0 * MG) * ang;
        C[i + 1] = __dadd_rn(C[i], B[i]);
    }
}

// rate(t, Omega, q) = sum_k f_k r_k sum_j C_kj G_j, G = (gL, gH, q Re gc, q Im gc),
// with the exact convolutions (library exp, erfcx, the Faddeeva function).
__device__ double phis_rate_exact(const PhisConsts& c, const MathTables* mt, double t, double ck, double cl,
                                  double phi, double q) {
    const double tau = t - c.mu;
    double cr, ci;
    conv2_complex(c, tau, &cr, &ci);
    const double G[4] = {0.5 * conv2_real(c, tau, c.GL, c.uL0), 0.5 * conv2_real(c, tau, c.GH, c.uH0),
                         0.5 * q * cr, 0.5 * q * ci};
    double f[10];
    basis_unscaled(ck, cl, phi, mt, f);
    double r = 0.0;
    for (int k = 0; k < 10; ++k) {
        double row[4];
        c_row(k, c.br[k], c.bi[k], 1.0, c.c, c.s, 1.0, c.D, row);
        const double e = row[0] * G[0] + row[1] * G[1] + row[2] * G[2] + row[3] * G[3];
        r += kBasisScale[k] * f[k] * row_scale(c, k) * e;
    }
    return r;
}

constexpr int kGenPerThread = 16;              // candidates per thread per chunk (bits of a mask)
constexpr int kGenChunk = kBlock * kGenPerThread;

// Signal candidate j of toy k: Philox calls (j, k, 0): u_bin, u_acc; (j, k, 1):
// ck, cl; (j, k, 2): phi, u_pos; (j, k, 3): u_q.  Its bin is the first i with
// u_bin C_64 <= C_{i+1} (the proposal is piecewise uniform with weights B_i),
// t = min(e_i + u_pos w, t_hi); the tag is the selected one (Q = +-1) or +1 for
// u_q <= 1/2, else -1; kept iff u_acc B_i < rate.  The toy takes the first
// n_sig kept candidates in increasing j.  Background event i: (i, k, 4): t,
// ck; (i, k, 5): cl, phi; (i, k, 6): u_q.  One block per toy.
__global__ void __launch_bounds__(kBlock)
phis_toygen_kernel(ModelDev m, const Consts* __restrict__ consts, uint32_t k0, uint32_t k1, int n_toys,
                   const int64_t* __restrict__ n_sig, const int64_t* __restrict__ n_bkg,
                   const int64_t* __restrict__ offsets, int64_t capacity, double* __restrict__ ot,
                   double* __restrict__ ock, double* __restrict__ ocl, double* __restrict__ ophi,
                   double* __restrict__ oq) {
    __shared__ __align__(16) PhisConsts c;
    __shared__ MathTables mt;
    __shared__ int warp_sums[kBlock / 32];
    __shared__ double B[kGenBins], C[kGenBins + 1];
    {
        const double* src = reinterpret_cast<const double*>(consts);
        double* dst = reinterpret_cast<double*>(&c);
        for (int i = threadIdx.x; i < kPhisDoubles; i += blockDim.x) dst[i] = src[i];
    }
    load_math_tables(&mt);
    const double span = __dsub_rn(m.t_hi, m.t_lo);
    const double w = __ddiv_rn(span, (double)kGenBins);
    __syncthreads();
    if (threadIdx.x == 0) phis_envelope_bins(c, m, w, B, C);
    __syncthreads();
    const double total = C[kGenBins];
    // the first bin i with target <= C[i + 1] (C non-decreasing: binary search)
    auto bin_of = [&](double u) {
        const double target = __dmul_rn(u, total);
        int lo = 0, hi = kGenBins - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (target <= C[mid + 1]) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    auto t_of = [&](int b, double u) {
        return fmin(__dadd_rn(__dadd_rn(m.t_lo, __dmul_rn((double)b, w)), __dmul_rn(u, w)), m.t_hi);
    };
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const double Q = c.qsel;
    auto tag = [&](double u) { return Q != 0.0 ? Q : (u <= 0.5 ? 1.0 : -1.0); };
    auto angles = [&](const U4& b, const U4& d, double* ck, double* cl, double* ph) {
        *ck = __dsub_rn(__dmul_rn(2.0, u01(b.x, b.y)), 1.0);
        *cl = __dsub_rn(__dmul_rn(2.0, u01(b.z, b.w)), 1.0);
        *ph = __dmul_rn(cdetail::kPi, __dsub_rn(__dmul_rn(2.0, u01(d.x, d.y)), 1.0));
    };
    for (int toy = blockIdx.x; toy < n_toys; toy += gridDim.x) {
        const int64_t ns = n_sig[toy], nb = n_bkg[toy], off = offsets[toy];
        if (ns < 0 || nb < 0 || off < 0 || off + ns + nb > capacity) continue;   // skipped
        const bool usable = isfinite(total) && total > 0.0 && isfinite(c.N) && c.N > 0.0;
        const uint64_t budget = usable ? (uint64_t)ns * 65536ull + (1ull << 22) : 0ull;
        int64_t got = 0;
        for (uint64_t j0 = 0; got < ns && j0 < budget; j0 += kGenChunk) {
            const uint64_t jt = j0 + (uint64_t)threadIdx.x * kGenPerThread;
            unsigned mask = 0;
#pragma unroll 1
            for (int i = 0; i < kGenPerThread; ++i) {
                const uint64_t j = jt + i;
                const U4 a = draw(j, (uint32_t)toy, 0u, k0, k1);
                const U4 b = draw(j, (uint32_t)toy, 1u, k0, k1);
                const U4 d = draw(j, (uint32_t)toy, 2u, k0, k1);
                const double uq = Q != 0.0 ? 0.0 : u01(draw(j, (uint32_t)toy, 3u, k0, k1).x,
                                                       draw(j, (uint32_t)toy, 3u, k0, k1).y);
                const int bin = bin_of(u01(a.x, a.y));
                const double t = t_of(bin, u01(d.z, d.w));
                double ck, cl, ph;
                angles(b, d, &ck, &cl, &ph);
                if (__dmul_rn(u01(a.z, a.w), B[bin]) < phis_rate_exact(c, &mt, t, ck, cl, ph, tag(uq)))
                    mask |= 1u << i;
            }
            int total;
            const int before = block_exclusive_scan(__popc(mask), warp_sums, &total);
            int rank = 0;
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1u;
                const int64_t pos = got + before + rank;
                ++rank;
                if (pos >= ns) break;
                const uint64_t j = jt + i;
                const U4 a = draw(j, (uint32_t)toy, 0u, k0, k1);
                const U4 b = draw(j, (uint32_t)toy, 1u, k0, k1);
                const U4 d = draw(j, (uint32_t)toy, 2u, k0, k1);
                const U4 e = draw(j, (uint32_t)toy, 3u, k0, k1);
                double ck, cl, ph;
                angles(b, d, &ck, &cl, &ph);
                ot[off + pos] = t_of(bin_of(u01(a.x, a.y)), u01(d.z, d.w));
                ock[off + pos] = ck;
                ocl[off + pos] = cl;
                ophi[off + pos] = ph;
                oq[off + pos] = tag(u01(e.x, e.y));
            }
            got += total;
        }
        for (int64_t pos = got + threadIdx.x; pos < ns; pos += blockDim.x)
            ot[off + pos] = ock[off + pos] = ocl[off + pos] = ophi[off + pos] = oq[off + pos] = nan;
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
            const U4 a = draw((uint64_t)i, (uint32_t)toy, 4u, k0, k1);
            const U4 b = draw((uint64_t)i, (uint32_t)toy, 5u, k0, k1);
            const U4 e = draw((uint64_t)i, (uint32_t)toy, 6u, k0, k1);
            const int64_t pos = off + ns + i;
            ot[pos] = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
            ock[pos] = __dsub_rn(__dmul_rn(2.0, u01(a.z, a.w)), 1.0);
            ocl[pos] = __dsub_rn(__dmul_rn(2.0, u01(b.x, b.y)), 1.0);
            ophi[pos] = __dmul_rn(cdetail::kPi, __dsub_rn(__dmul_rn(2.0, u01(b.z, b.w)), 1.0));
            oq[pos] = tag(u01(e.x, e.y));
        }
    }
}

}  // namespace

ipa_status launch_phis_toygen(const ModelDev& m, const Consts* consts, uint64_t seed, int n_toys,
                              const int64_t* n_sig, const int64_t* n_bkg, const int64_t* offsets,
                              const ipa_event_buffers* out, cudaStream_t s) {
    phis_toygen_kernel<<<n_toys, kBlock, 0, s>>>(m, consts, (uint32_t)seed, (uint32_t)(seed >> 32), n_toys, n_sig,
                                                 n_bkg, offsets, out->capacity, out->t, out->ck, out->cl, out->phi,
                                                 out->q);
    return cuda_fail(cudaGetLastError(), "phi_s toygen kernel launch");
}


namespace {
// ipa_nll_grad_combine for the phi_s model: the kernel's last reduction level
// (the wide form) over gathered group partials, then phis_finalize (one warp).
template <bool CACHED>
__global__ void phis_combine_kernel(const double* __restrict__ groups, int64_t n_groups,
                                    const Consts* __restrict__ consts, int n_par, double* __restrict__ out) {
    constexpr int NA = n_acc(IPA_MODEL_PHIS, true);
    const int lane = threadIdx.x & 31;
    if (n_groups == 0) {
        for (int j = lane; j < 1 + n_par; j += 32) out[j] = 0.0;
        return;
    }
    double acc[NA];
    reduce_partials_wide<NA>(groups, 0, n_groups, 1, acc);
    phis_finalize<true, CACHED>(*reinterpret_cast<const PhisConsts*>(consts), acc, n_par, out, lane);
}
}  // namespace

ipa_status launch_phis_combine(const double* groups, int64_t n_groups, bool cached, const Consts* consts, int n_par,
                               double* out, cudaStream_t s) {
    if (cached)
        phis_combine_kernel<true><<<1, 32, 0, s>>>(groups, n_groups, consts, n_par, out);
    else
        phis_combine_kernel<false><<<1, 32, 0, s>>>(groups, n_groups, consts, n_par, out);
    return cuda_fail(cudaGetLastError(), "phi_s combine kernel launch");
}

ipa_status launch_phis_nll(const ModelDev& m, bool grad, const Cols& cols, int64_t n,
                           const int64_t* seg_begin, const int64_t* seg_end, const int64_t* seg_tiles, int n_seg,
                           const Consts* consts, Scratch* sc, double* out, cudaStream_t st, const LaunchCfg* cfg) {
    const int P = m.n_par;
    if (cols.fk)
        return grad ? launch_phis_w<true, true>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg)
                    : launch_phis_w<false, true>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg);
    return grad ? launch_phis_w<true, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg)
                : launch_phis_w<false, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg);
}

}  // namespace ipa
