// Hot path of the flavour-tagged model (model formulas in tagged.cuh): the
// parameter constants, the likelihood with its fused gradient and the
// deterministic reduction, and the Faddeeva test entry point.
//
// Per event (tau = t - mu) the PDF needs 2 g for the two real rates Gamma_H,
// Gamma_L and for the complex rate Gamma - i Dm.  For t > tcut every erfc
// term is below 1e-17 of its exponential and
//   2 gH = exp(-Gamma_H tau + Gamma_H^2 sigma^2/2 + ln2),  2 gL likewise,
//   2 g  = exp(-Gamma tau + (Gamma^2 - Dm^2) sigma^2/2 + ln2) e^{i (Dm tau - Gamma Dm sigma^2)}:
// three exponentials and one sine/cosine pair, all on the integer pipe.  Events
// with t <= tcut (up to about six resolution widths past the peak) also need
// the Gaussian, two erfcx and one Faddeeva function; as in the 4D kernel they
// are listed by ballot and evaluated 32 to a pass into the warp's buffer, so
// the FP64 pipe does not run the long branch for lanes that discard it.
//
// Gradient.  With r = w / P, P = cs S + cb, every derivative is a contraction
// of 12 per-event sums with parameter-only factors (tag_finalize): the sums of
// r 2gH, r tau 2gH, r 2gL, r tau 2gL, r q 2Re g, r q tau 2Re g, r q 2Im g,
// r q tau 2Im g, r Gx, r tau Gx, r q Gx and r, so the event pass carries 13
// accumulators for 8 parameters.
#include <math.h>

#include "faddeeva.cuh"
#include "fp64_math.cuh"
#include "int_math.cuh"
#include "ipa_internal.cuh"
#include "tagged.cuh"
#include "tile_reduce.cuh"

namespace ipa {
namespace {

constexpr int kPerLane = kTile / 32;
constexpr int kSub = 4;
static_assert(kPerLane % kSub == 0, "events per lane must be a multiple of kSub");
constexpr int kMaxWarps = 8;

// One event: w log P into acc[0] (or, for w = 1 exactly, P into the lane's
// log product) and the 12 adjoint sums into acc[1..12].
template <bool GRAD, bool WEIGHTED>
__device__ __forceinline__ void tag_event(const TagConsts& c, const MathTables* mt, double t, double q, double w,
                                          const TagSlow& sl, double* acc, double* prod, int* esum) {
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
    const double P = fma(c.qH, T2H, fma(c.qL, T2L, fma(q * c.qD, Ci, c.cb)));
    if (WEIGHTED && __double_as_longlong(w) != 0x3FF0000000000000ll)
        acc[0] = fma(w, log_fast(P, mt), acc[0]);
    else
        log_mul(P, prod, esum);
    if (GRAD) {
        const double r = WEIGHTED ? w * rcp_newton(P) : rcp_newton(P);
        acc[1] += r;
        const double rH = r * T2H, rL = r * T2L;
        acc[2] += rH;
        acc[3] = fma(rH, tau, acc[3]);
        acc[4] += rL;
        acc[5] = fma(rL, tau, acc[5]);
        const double rq = q * r;
        const double rr = rq * Cr, ri = rq * Ci;
        acc[6] += rr;
        acc[7] = fma(rr, tau, acc[7]);
        acc[8] += ri;
        acc[9] = fma(ri, tau, acc[9]);
        const double rG = r * gx;
        acc[10] += rG;
        acc[11] = fma(rG, tau, acc[11]);
        acc[12] = fma(rq, gx, acc[12]);
    }
}

// NLL and gradient of one segment from its reduced sums (every lane holds
// acc; lane j writes component j).  With RH = sum r gH, TH = sum r tau gH (and
// L likewise), Rr + i Ri = sum r q g, Tr + i Ti = sum r q tau g (complex rate),
// RG = sum r G, TG = sum r tau G, RqG = sum r q G, Q = sum r and
// SR = sum r S = aH RH + aL RL + Ds Ri:
//   dNLL/dtheta_j = cs (dlnN_j SR - sum r dS/dtheta_j)  (j != f_b),
//   dNLL/df_b     = SR / N - Q / (2 (t_hi - t_lo)),
// where sum r dS/dtheta_j follows from dg/dz = (z sigma^2 - tau) g - sigma^2 G,
// dg/dsigma = z^2 sigma g - (z sigma + tau/sigma) G, dg/dtau = -z g + G,
// dz/dDm = -i, and the derivatives of aH, aL, Ds in phi_s and omega.
template <bool GRAD>
__device__ void tag_finalize(const TagConsts& c, const double* acc, int n_par, double* out, int lane) {
    if (lane == 0) out[0] = -acc[0];
    if (!GRAD) return;
    const double Q = acc[1];
    const double RH = 0.5 * acc[2], TH = 0.5 * acc[3], RL = 0.5 * acc[4], TL = 0.5 * acc[5];
    const double Rr = 0.5 * acc[6], Tr = 0.5 * acc[7], Ri = 0.5 * acc[8], Ti = 0.5 * acc[9];
    const double RG = c.cG * acc[10], TG = c.cG * acc[11], RqG = c.cG * acc[12];
    const double SR = c.aH * RH + c.aL * RL + c.Ds * Ri;
    const double s2 = c.s2, sg = c.sigma;
    double dS = 0.0;
    if (lane == 0) {          // Gamma
        dS = c.aH * (c.GH * s2 * RH - TH - s2 * RG) + c.aL * (c.GL * s2 * RL - TL - s2 * RG) +
             c.Ds * (c.Gamma * s2 * Ri - Ti - c.Dm * s2 * Rr);
    } else if (lane == 1) {   // sigma
        dS = c.aH * (c.GH * c.GH * sg * RH - c.GH * sg * RG - TG * c.inv_s) +
             c.aL * (c.GL * c.GL * sg * RL - c.GL * sg * RG - TG * c.inv_s) +
             c.Ds * (sg * ((c.Gamma - c.Dm) * (c.Gamma + c.Dm) * Ri - 2.0 * c.Gamma * c.Dm * Rr) + c.Dm * sg * RqG);
    } else if (lane == 2) {   // mu
        dS = c.aH * (c.GH * RH - RG) + c.aL * (c.GL * RL - RG) + c.Ds * (c.Gamma * Ri - c.Dm * Rr);
    } else if (lane == 4) {   // DG
        dS = -0.5 * c.aH * (c.GH * s2 * RH - TH - s2 * RG) + 0.5 * c.aL * (c.GL * s2 * RL - TL - s2 * RG);
    } else if (lane == 5) {   // Dm
        dS = -c.Ds * (c.Gamma * s2 * Rr - Tr + c.Dm * s2 * Ri - s2 * RqG);
    } else if (lane == 6) {   // phi_s
        dS = 0.5 * c.s * (RH - RL) + c.D * c.c * Ri;
    } else if (lane == 7) {   // omega
        dS = -2.0 * c.s * Ri;
    }
    if (lane == IPA_FB) out[1 + IPA_FB] = fma(SR, c.inv_N, -Q * c.inv_V2);
    else if (lane < IPA_NPAR_TAGGED) out[1 + lane] = c.cs * fma(c.dlnN[lane], SR, -dS);
    for (int j = IPA_NPAR_TAGGED + lane; j < n_par; j += 32) out[1 + j] = 0.0;
}

template <bool GRAD, bool WEIGHTED>
__global__ void __launch_bounds__(32 * kMaxWarps, 2)
tag_kernel(Cols cols, int64_t n, const int64_t* __restrict__ seg_begin, const int64_t* __restrict__ seg_end,
           const int64_t* __restrict__ seg_tiles, int n_seg, const Consts* __restrict__ consts,
           double* __restrict__ partials, unsigned* __restrict__ counters, unsigned* __restrict__ gcount,
           unsigned* __restrict__ work, double* __restrict__ out, int n_par, int per_take) {
    constexpr int NA = GRAD ? 13 : 1;
    const int out_stride = GRAD ? 1 + n_par : 1;
    __shared__ MathTables mt;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n_wib = blockDim.x >> 5;
    TagSlow* const sbuf = reinterpret_cast<TagSlow*>(dyn_smem) + wib * (kSub * 32);
    TagConsts& tc = reinterpret_cast<TagConsts*>(dyn_smem + (size_t)n_wib * kSub * 32 * sizeof(TagSlow))[wib];

    load_math_tables(&mt);
    __syncthreads();
    // a programmatic dependent of the constants kernel: wait for its results
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
        unsigned taken = 0;
        if (lane == 0) taken = atomicAdd(work, 1u);
        const int64_t first = (int64_t)__shfl_sync(0xffffffffu, taken, 0) * per_take;
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
                double* dst = reinterpret_cast<double*>(&tc);
                for (int i = lane; i < kTagConstsDoubles; i += 32) dst[i] = __ldg(src + i);
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
#pragma unroll 1
            for (int i0 = 0; i0 < kPerLane; i0 += kSub) {
                unsigned m0, m1, m2, m3;
                {
                    unsigned mk[kSub];
#pragma unroll
                    for (int k = 0; k < kSub; ++k) {
                        const int64_t e = tbase + lane + 32 * (i0 + k);
                        const bool slow = e < ev1 && !greater(__ldg(cols.t + e), tc.tcut);
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
                    sbuf[j] = tag_slow(tc, __ldg(cols.t + e) - tc.mu, &mt);
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
                        tag_event<GRAD, WEIGHTED>(tc, &mt, __ldg(cols.t + e), __ldg(cols.q + e), w, sl, acc, &prod,
                                                  &esum);
                    }
                }
                __syncwarp();
            }
            acc[0] += log_of(prod, esum, &mt);
            const double share = warp_butterfly<NA>(acc, lane);
            if (!tile_commit<NA>(share, lane, tile, t0, t1, seg, partials, gcount, counters, acc)) continue;
            tag_finalize<GRAD>(tc, acc, n_par, out + (size_t)seg * out_stride, lane);
            if (lane == 0) counters[seg] = 0u;
        }
    }
    work_done(work, lane);
}

template <bool GRAD, bool WEIGHTED>
ipa_status launch_tag_t(const Cols& cols, int64_t n, const int64_t* seg_begin, const int64_t* seg_end,
                        const int64_t* seg_tiles, int n_seg, const Consts* consts, Scratch* sc, double* out,
                        int n_par, cudaStream_t st, const LaunchCfg* force) {
    const bool single = seg_begin == nullptr;
    const int64_t tiles = tile_estimate(n, n_seg);
    const LaunchCfg cfg = force ? *force : launch_cfg(IPA_MODEL_TAGGED1D, GRAD, false, n_seg > 1, tiles);
    const int W = cfg.warps_per_block >= 1 && cfg.warps_per_block <= kMaxWarps ? cfg.warps_per_block : 1;
    const int K = cfg.tiles_per_take >= 1 ? cfg.tiles_per_take : 1;
    const size_t smem = (size_t)W * (sizeof(TagConsts) + kSub * 32 * sizeof(TagSlow));
    auto kern = tag_kernel<GRAD, WEIGHTED>;
    // dynamic shared memory above the default limit (8 warps: 44 KB besides
    // the static tables) needs the opt-in, once per device
    static bool attr[64] = {};
    static int occ[64][kMaxWarps + 1] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr[dev & 63]) {
        ipa_status q = cuda_fail(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)(kMaxWarps * (sizeof(TagConsts) + kSub * 32 * sizeof(TagSlow)))),
                                 "tagged kernel attribute");
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
                     "tagged likelihood kernel launch");
}

__global__ void faddeeva_kernel(const double* __restrict__ z, double* __restrict__ w, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double wr, wi;
        faddeeva(z[2 * i], z[2 * i + 1], &wr, &wi);
        w[2 * i] = wr;
        w[2 * i + 1] = wi;
    }
}

}  // namespace

namespace {
// ipa_nll_grad_combine for the tagged model: the kernel's last reduction level
// over gathered group partials, then tag_finalize (one warp).
__global__ void tag_combine_kernel(const double* __restrict__ groups, int64_t n_groups,
                                   const Consts* __restrict__ consts, int n_par, double* __restrict__ out) {
    constexpr int NA = n_acc(IPA_MODEL_TAGGED1D, true);
    const int lane = threadIdx.x & 31;
    if (n_groups == 0) {
        for (int j = lane; j < 1 + n_par; j += 32) out[j] = 0.0;
        return;
    }
    double acc[NA];
    gather_butterfly<NA>(reduce_partials<NA>(groups, 0, n_groups, 1, lane), acc);
    tag_finalize<true>(*reinterpret_cast<const TagConsts*>(consts), acc, n_par, out, lane);
}
}  // namespace

ipa_status launch_tag_combine(const double* groups, int64_t n_groups, const Consts* consts, int n_par, double* out,
                              cudaStream_t s) {
    tag_combine_kernel<<<1, 32, 0, s>>>(groups, n_groups, consts, n_par, out);
    return cuda_fail(cudaGetLastError(), "tagged combine kernel launch");
}

ipa_status launch_tag_nll(const ModelDev& m, bool grad, const Cols& cols, int64_t n,
                          const int64_t* seg_begin, const int64_t* seg_end, const int64_t* seg_tiles, int n_seg,
                          const Consts* consts, Scratch* sc, double* out, cudaStream_t st, const LaunchCfg* cfg) {
    const int P = m.n_par;
    if (cols.w)
        return grad ? launch_tag_t<true, true>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg)
                    : launch_tag_t<false, true>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg);
    return grad ? launch_tag_t<true, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg)
                : launch_tag_t<false, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg);
}

}  // namespace ipa

extern "C" ipa_status ipa_faddeeva(const double* z_dev, double* w_dev, int64_t n, void* stream) {
    using namespace ipa;
    if (n < 0 || (n > 0 && (!z_dev || !w_dev))) {
        set_error("ipa_faddeeva: bad arguments");
        return IPA_ERR_ARG;
    }
    if (n == 0) return IPA_OK;
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 4096 ? blocks : 4096);
    faddeeva_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(z_dev, w_dev, n);
    return cuda_fail(cudaGetLastError(), "faddeeva kernel launch");
}
