// Hot-path steps a2-a6: per-event normalised PDF, -w log P, fused analytic
// adjoint and the deterministic FP64 reduction, for one fit or for many
// segments (fits) packed back to back.
//
// Sec. 3 of the paper evaluates the PDF with one thread per event, takes the
// log of the signal/background mixture in a second launch and sums the logs
// on the host.  Here one kernel does all of it: each 256-thread block walks
// 512-event tiles (two events per thread, one 16-byte load per column),
// keeps FP64 accumulators in registers, reduces them with a fixed tree, and
// the block that finishes the last tile of a segment reduces that segment's
// tile partials in fixed order and writes its NLL and gradient.
//
// Gradient (fused adjoint).  With r = w/P, every derivative of the NLL is a
// contraction of a few per-event sums with parameter-only factors:
//   S_k = sum r T f_k,  D_j = sum r A dT/dtheta_j (j = Gamma, sigma, mu),
//   Q = sum r,          SH = sum_k h_k S_k = sum r T A,
//   dNLL/dtime_j = -cs D_j + cs (dI_T/dtheta_j / I_T) SH,
//   dNLL/df_b    = SH / (I_T I_Omega) - Q / V,
//   dNLL/dang_j  = -cs sum_k (dh_k/dtheta_j) S_k,   cs = (1 - f_b)/(I_T I_Omega),
// so the event pass carries 15 accumulators (4D) instead of one per
// parameter and the angular derivatives cost nothing per event.
#include <math.h>

#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double k2OverSqrt6 = 0.81649658092772603273;
constexpr double k2OverSqrt3 = 1.15470053837925152902;

// f_k(cos thK, cos thmu, phi), k = 1..10 (Sec. 4, helicity basis).
__device__ __forceinline__ void angular_basis(double ck, double cl, double phi, double f[10]) {
    const double sk2 = fma(-ck, ck, 1.0);
    const double sl2 = fma(-cl, cl, 1.0);
    const double sk = sqrt(sk2), sl = sqrt(sl2);
    double sp, cp;
    sincos(phi, &sp, &cp);
    f[0] = ck * ck * sl2;
    f[1] = 0.5 * sk2 * (1.0 - sl2 * cp * cp);
    f[2] = 0.5 * sk2 * (1.0 - sl2 * sp * sp);
    f[3] = sk2 * sl2 * sp * cp;
    const double a = sk * ck * sl * cl;
    f[4] = kSqrt2 * a * cp;
    f[5] = -kSqrt2 * a * sp;
    f[6] = sl2 * (1.0 / 3.0);
    const double b = sk * sl * cl;
    f[7] = k2OverSqrt6 * b * cp;
    f[8] = -k2OverSqrt6 * b * sp;
    f[9] = k2OverSqrt3 * ck * sl2;
}

// One event: accumulate w log P (and the adjoint sums).
template <int KIND, bool GRAD>
__device__ __forceinline__ void event(const Consts& c, double t, double ck, double cl, double phi,
                                      double w, double* acc) {
    const double tau = t - c.mu;
    const double E = exp(fma(-c.Gamma, tau, c.c_exp));
    const double z = (c.Gs2 - tau) * c.k_z;
    const double T = 0.5 * E * erfc(z);
    double A = 1.0;
    double f[10];
    if (KIND == IPA_MODEL_ANGTIME4D) {
        angular_basis(ck, cl, phi, f);
        A = 0.0;
#pragma unroll
        for (int k = 0; k < 10; ++k) A = fma(c.h[k], f[k], A);
    }
    const double P = fma(c.cs * T, A, c.cb);
    acc[0] = fma(w, log(P), acc[0]);
    if (GRAD) {
        const double r = w / P;
        acc[1] += r;
        const double rT = r * T;
        constexpr int kD = KIND == IPA_MODEL_ANGTIME4D ? 12 : 3;
        if (KIND == IPA_MODEL_ANGTIME4D) {
#pragma unroll
            for (int k = 0; k < 10; ++k) acc[2 + k] = fma(rT, f[k], acc[2 + k]);
        } else {
            acc[2] += rT;
        }
        const double G = c.cG * exp(-(tau * tau) * c.k_g);
        const double rA = r * A;
        const double dTG = fma(c.Gs2 - tau, T, -c.s2 * G);
        const double dTs = fma(c.G2s, T, -fma(tau, c.inv_s, c.Gsig) * G);
        const double dTm = fma(c.Gamma, T, -G);
        acc[kD + 0] = fma(rA, dTG, acc[kD + 0]);
        acc[kD + 1] = fma(rA, dTs, acc[kD + 1]);
        acc[kD + 2] = fma(rA, dTm, acc[kD + 2]);
    }
}

// Fixed reduction tree over the 256 slots of a block: at each level slot s
// adds slot s + half (half = 128, 64, 32 through shared memory, then 16..1
// by warp shuffles).  The result is in thread 0.
template <int NA>
__device__ __forceinline__ void block_tree(double* acc, double (*red)[kSlots / 2]) {
    const int s = threadIdx.x;
#pragma unroll
    for (int half = kSlots / 2; half >= 32; half >>= 1) {
        if (s >= half && s < 2 * half) {
#pragma unroll
            for (int a = 0; a < NA; ++a) red[a][s - half] = acc[a];
        }
        __syncthreads();
        if (s < half) {
#pragma unroll
            for (int a = 0; a < NA; ++a) acc[a] += red[a][s];
        }
        __syncthreads();
    }
    if (s < 32) {
#pragma unroll
        for (int half = 16; half >= 1; half >>= 1) {
#pragma unroll
            for (int a = 0; a < NA; ++a) acc[a] += __shfl_down_sync(0xffffffffu, acc[a], half);
        }
    }
}

__device__ __forceinline__ int64_t clamp_off(int64_t v, int64_t n) {
    return v < 0 ? 0 : (v > n ? n : v);
}

// Segment s covers tiles [seg_tiles[s], seg_tiles[s+1]); find s for `tile`.
__device__ __forceinline__ int find_segment(const int64_t* seg_tiles, int n_seg, int64_t tile) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(seg_tiles + mid) <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Write NLL (and gradient) of one segment from its reduced accumulators.
template <int KIND, bool GRAD>
__device__ void finalize(const Consts& c, const double* acc, int n_par, double* out) {
    out[0] = -acc[0];
    if (!GRAD) return;
    const double Q = acc[1];
    double SH;
    constexpr int kD = KIND == IPA_MODEL_ANGTIME4D ? 12 : 3;
    if (KIND == IPA_MODEL_ANGTIME4D) {
        SH = 0.0;
        for (int k = 0; k < 10; ++k) SH = fma(c.h[k], acc[2 + k], SH);
    } else {
        SH = acc[2];
    }
    for (int j = 0; j < 3; ++j) out[1 + j] = c.cs * fma(c.dlnIT[j], SH, -acc[kD + j]);
    out[1 + IPA_FB] = fma(SH, c.inv_ITIO, -Q * c.inv_V);
    if (KIND == IPA_MODEL_ANGTIME4D) {
        for (int j = 0; j < 6; ++j) {
            double s = 0.0;
            for (int k = 0; k < 10; ++k) s = fma(c.dh[k][j], acc[2 + k], s);
            out[1 + IPA_A0SQ + j] = -c.cs * s;
        }
    }
    for (int j = (KIND == IPA_MODEL_ANGTIME4D ? IPA_NPAR_4D : IPA_NPAR_1D); j < n_par; ++j)
        out[1 + j] = 0.0;
}

template <int KIND, bool GRAD>
__global__ void __launch_bounds__(kBlock)
nll_kernel(Cols cols, int64_t n, const int64_t* __restrict__ seg_off,
           const int64_t* __restrict__ seg_tiles, int n_seg, const Consts* __restrict__ consts,
           double* __restrict__ partials, unsigned* __restrict__ counters,
           double* __restrict__ out, int n_par) {
    constexpr int NA = n_acc(KIND, GRAD);
    const int out_stride = GRAD ? 1 + n_par : 1;
    __shared__ double red[NA][kSlots / 2];
    __shared__ __align__(16) Consts sc;
    __shared__ int s_last;

    const bool single = seg_off == nullptr;
    const int64_t total = single ? (n + kTile - 1) / kTile : __ldg(seg_tiles + n_seg);

    // empty segments have no tile to finalise them: block 0 writes their zeros
    if (blockIdx.x == 0) {
        for (int s = threadIdx.x; s < n_seg; s += blockDim.x) {
            const bool empty = single ? (n == 0) : (__ldg(seg_tiles + s + 1) == __ldg(seg_tiles + s));
            if (empty) {
                for (int j = 0; j < out_stride; ++j) out[(size_t)s * out_stride + j] = 0.0;
            }
        }
    }

    int cur = -1;
    for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int seg = 0;
        int64_t t0 = 0, t1 = total, ev0 = 0, ev1 = n;
        if (!single) {
            seg = find_segment(seg_tiles, n_seg, tile);
            t0 = __ldg(seg_tiles + seg);
            t1 = __ldg(seg_tiles + seg + 1);
            ev0 = clamp_off(__ldg(seg_off + seg), n);
            ev1 = clamp_off(__ldg(seg_off + seg + 1), n);
            if (ev1 < ev0) ev1 = ev0;
        }
        if (seg != cur) {
            __syncthreads();
            const double* src = reinterpret_cast<const double*>(consts + seg);
            double* dst = reinterpret_cast<double*>(&sc);
            for (int i = threadIdx.x; i < kConstsDoubles; i += blockDim.x) dst[i] = __ldg(src + i);
            __syncthreads();
            cur = seg;
        }

        double acc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] = 0.0;

        const int64_t i0 = ev0 + (tile - t0) * kTile + 2 * threadIdx.x;
        if (i0 + 1 < ev1 && (ev0 & 1) == 0) {
            const double2 t2 = __ldg(reinterpret_cast<const double2*>(cols.t + i0));
            double2 w2 = make_double2(1.0, 1.0);
            if (cols.w) w2 = __ldg(reinterpret_cast<const double2*>(cols.w + i0));
            if (KIND == IPA_MODEL_ANGTIME4D) {
                const double2 k2 = __ldg(reinterpret_cast<const double2*>(cols.ck + i0));
                const double2 l2 = __ldg(reinterpret_cast<const double2*>(cols.cl + i0));
                const double2 p2 = __ldg(reinterpret_cast<const double2*>(cols.phi + i0));
                event<KIND, GRAD>(sc, t2.x, k2.x, l2.x, p2.x, w2.x, acc);
                event<KIND, GRAD>(sc, t2.y, k2.y, l2.y, p2.y, w2.y, acc);
            } else {
                event<KIND, GRAD>(sc, t2.x, 0.0, 0.0, 0.0, w2.x, acc);
                event<KIND, GRAD>(sc, t2.y, 0.0, 0.0, 0.0, w2.y, acc);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int64_t i = i0 + e;
                if (i < ev1) {
                    const double w = cols.w ? __ldg(cols.w + i) : 1.0;
                    if (KIND == IPA_MODEL_ANGTIME4D)
                        event<KIND, GRAD>(sc, __ldg(cols.t + i), __ldg(cols.ck + i),
                                          __ldg(cols.cl + i), __ldg(cols.phi + i), w, acc);
                    else
                        event<KIND, GRAD>(sc, __ldg(cols.t + i), 0.0, 0.0, 0.0, w, acc);
                }
            }
        }

        block_tree<NA>(acc, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int a = 0; a < NA; ++a) partials[tile * NA + a] = acc[a];
            __threadfence();
            const unsigned done = atomicAdd(counters + seg, 1u) + 1u;
            s_last = (done == (unsigned)(t1 - t0));
        }
        __syncthreads();
        if (s_last) {
            // this block wrote the segment's last tile: reduce its partials
            __threadfence();
#pragma unroll
            for (int a = 0; a < NA; ++a) acc[a] = 0.0;
            for (int64_t tt = t0 + threadIdx.x; tt < t1; tt += kSlots) {
#pragma unroll
                for (int a = 0; a < NA; ++a) acc[a] += __ldcg(partials + tt * NA + a);
            }
            block_tree<NA>(acc, red);
            if (threadIdx.x == 0) {
                finalize<KIND, GRAD>(sc, acc, n_par, out + (size_t)seg * out_stride);
                counters[seg] = 0u;
            }
        }
        __syncthreads();
    }
}

// seg_tiles[s] = sum_{r<s} ceil(size_r / kTile), one block, sequential per thread
// over a contiguous run of segments, then a block scan of the run totals.
__global__ void seg_tiles_kernel(const int64_t* __restrict__ seg_off, int n_seg, int64_t n,
                                 int64_t* __restrict__ seg_tiles) {
    __shared__ int64_t run[1024];
    const int nt = blockDim.x;
    const int per = (n_seg + nt - 1) / nt;
    const int b = threadIdx.x * per;
    const int e = min(n_seg, b + per);
    int64_t sum = 0;
    for (int s = b; s < e; ++s) {
        const int64_t lo = clamp_off(seg_off[s], n);
        int64_t hi = clamp_off(seg_off[s + 1], n);
        if (hi < lo) hi = lo;
        sum += (hi - lo + kTile - 1) / kTile;
    }
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
        const int64_t lo = clamp_off(seg_off[s], n);
        int64_t hi = clamp_off(seg_off[s + 1], n);
        if (hi < lo) hi = lo;
        acc += (hi - lo + kTile - 1) / kTile;
    }
    if (threadIdx.x == nt - 1) seg_tiles[n_seg] = run[nt - 1];
}

template <int KIND, bool GRAD>
ipa_status launch_t(const Cols& cols, int64_t n, const int64_t* seg_off, const int64_t* seg_tiles,
                    int n_seg, const Consts* consts, Scratch* sc, double* out, int n_par,
                    cudaStream_t st) {
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, nll_kernel<KIND, GRAD>, kBlock, 0);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    }
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (seg_off == nullptr) {
        const int64_t tiles = (n + kTile - 1) / kTile;
        grid = tiles < grid ? tiles : grid;
    }
    if (grid < 1) grid = 1;
    nll_kernel<KIND, GRAD><<<(unsigned)grid, kBlock, 0, st>>>(
        cols, n, seg_off, seg_tiles, n_seg, consts, sc->partials, sc->counters, out, n_par);
    return cuda_fail(cudaGetLastError(), "likelihood kernel launch");
}

}  // namespace

ipa_status launch_seg_tiles(const int64_t* seg_off, int n_seg, int64_t n, int64_t* seg_tiles,
                            cudaStream_t st) {
    seg_tiles_kernel<<<1, 1024, 0, st>>>(seg_off, n_seg, n, seg_tiles);
    return cuda_fail(cudaGetLastError(), "segment tiling kernel launch");
}

ipa_status launch_nll(const ModelDev& m, bool grad, const Cols& cols, int64_t n,
                      const int64_t* seg_off, const int64_t* seg_tiles, int n_seg,
                      const Consts* consts, Scratch* sc, double* out, cudaStream_t st) {
    if (m.kind == IPA_MODEL_TIME1D)
        return grad ? launch_t<IPA_MODEL_TIME1D, true>(cols, n, seg_off, seg_tiles, n_seg, consts, sc, out, m.n_par, st)
                    : launch_t<IPA_MODEL_TIME1D, false>(cols, n, seg_off, seg_tiles, n_seg, consts, sc, out, m.n_par, st);
    return grad ? launch_t<IPA_MODEL_ANGTIME4D, true>(cols, n, seg_off, seg_tiles, n_seg, consts, sc, out, m.n_par, st)
                : launch_t<IPA_MODEL_ANGTIME4D, false>(cols, n, seg_off, seg_tiles, n_seg, consts, sc, out, m.n_par, st);
}

namespace {

ipa_status run(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off, int n_seg,
               const double* theta, double* out, bool grad, void* stream) {
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if (!theta || !out) {
        set_error("theta and out must be device pointers");
        return IPA_ERR_ARG;
    }
    if (n_seg < 1) {
        set_error("n_seg must be >= 1");
        return IPA_ERR_ARG;
    }
    if (seg_off == nullptr && n_seg != 1) {
        set_error("segment offsets are required for n_seg > 1");
        return IPA_ERR_ARG;
    }
    const int64_t tiles = (ev->n + kTile - 1) / kTile + n_seg;
    Scratch* sc = nullptr;
    if ((st = scratch_get(tiles, n_seg + 1, &sc)) != IPA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_consts(m, theta, n_seg, sc->consts, s)) != IPA_OK) return st;
    if (seg_off) {
        if ((st = launch_seg_tiles(seg_off, n_seg, ev->n, sc->seg_tiles, s)) != IPA_OK) return st;
    }
    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w};
    return launch_nll(m, grad, cols, ev->n, seg_off, seg_off ? sc->seg_tiles : nullptr, n_seg,
                      sc->consts, sc, out, s);
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_nll(const ipa_model* model, const ipa_events* ev, const double* theta_dev,
                              double* out_dev, void* stream) {
    return ipa::run(model, ev, nullptr, 1, theta_dev, out_dev, false, stream);
}

extern "C" ipa_status ipa_nll_grad(const ipa_model* model, const ipa_events* ev,
                                   const double* theta_dev, double* out_dev, void* stream) {
    return ipa::run(model, ev, nullptr, 1, theta_dev, out_dev, true, stream);
}

extern "C" ipa_status ipa_nll_grad_segmented(const ipa_model* model, const ipa_events* ev,
                                             const int64_t* seg_off_dev, int32_t n_seg,
                                             const double* theta_dev, double* out_dev,
                                             void* stream) {
    if (!seg_off_dev) {
        ipa::set_error("seg_off_dev must not be NULL");
        return IPA_ERR_ARG;
    }
    return ipa::run(model, ev, seg_off_dev, n_seg, theta_dev, out_dev, true, stream);
}
