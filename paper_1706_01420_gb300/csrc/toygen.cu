// Hot-path step a7: pseudo-experiment generation by accept-reject (Sec. 7).
//
// Sec. 7 of the paper draws curand uniforms per thread and keeps the events
// that pass an accept-reject test, with the event counts drawn on the host.
// Here the generator is Philox-4x32-10 (Salmon et al., SC'11) written out in
// this file, addressed by counters so that every candidate of every toy is a
// pure function of (seed, toy, candidate index):
//   key     = (seed lo32, seed hi32)
//   signal candidate j of toy k:  counters (j lo32, j hi32, k, c), c = 0, 1, 2
//     c = 0 -> (t = t_lo + u (t_hi - t_lo), u_t)
//     c = 1 -> (cos thK = 2u - 1, cos thmu = 2u - 1)
//     c = 2 -> (phi = pi (2u - 1), u_a)
//     kept iff u_t M_T < g(t - mu)  and (4D)  u_a M_Omega < A(Omega);
//   background event i of toy k:  counters (i lo32, i hi32, k, 4) -> (t, ck),
//                                 (.., 5) -> (cl, phi), always kept.
// Each 64-bit uniform is u = (((a << 32) | b) >> 11) + 1) 2^-53 from two
// 32-bit words, in (0, 1].  Candidates are built with correctly rounded
// multiplies and adds only (no contraction into FMA), so the event values are
// reproducible bit for bit on any IEEE machine.  A toy keeps its first n_sig
// accepted candidates in increasing j: one block per toy walks candidate
// chunks, and a block-wide exclusive scan orders the accepted ones.
//
// Decisions first run in FP32 (this GPU's FP32 rate is 64 times its FP64
// rate): each test is evaluated with a per-candidate bound on its FP32 error,
// built from the documented accuracy of expf, erfcf, sincosf and sqrtf and
// the rounding of every input, and is decided in FP32 only when the uniform
// lies outside that band around the threshold.  Inside the band (about one
// candidate in 10^4), or wherever the bound is not established (a uniform or
// cosine near the end of its range, an exponent near over- or underflow), the
// FP64 test decides.  A decision is therefore always the FP64 test's; the
// FP32 pass only avoids evaluating it on clear cases.  Accepted candidates
// are regenerated from their counters and written with the exact FP64 values.
#include <math.h>

#include "consts.cuh"
#include "ipa_internal.cuh"
#include "philox.cuh"
#include "tagged.cuh"

namespace ipa {
namespace {

constexpr int kPerThread = 16;             // candidates per thread per chunk (bits of a mask)
constexpr int kChunk = kBlock * kPerThread;
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double k2OverSqrt6 = 0.81649658092772603273;
constexpr double k2OverSqrt3 = 1.15470053837925152902;


// A(Omega) = sum_k h_k f_k, evaluated as the oracle's definition (Sec. 4).
__device__ __forceinline__ double angular_pdf(const Consts& c, double ck, double cl, double phi) {
    const double sk = sqrt(1.0 - ck * ck), sl = sqrt(1.0 - cl * cl);
    double sp, cp;
    sincos(phi, &sp, &cp);
    double f[10];
    f[0] = ck * ck * sl * sl;
    f[1] = 0.5 * sk * sk * (1.0 - sl * sl * cp * cp);
    f[2] = 0.5 * sk * sk * (1.0 - sl * sl * sp * sp);
    f[3] = sk * sk * sl * sl * sp * cp;
    f[4] = kSqrt2 * sk * ck * sl * cl * cp;
    f[5] = -kSqrt2 * sk * ck * sl * cl * sp;
    f[6] = sl * sl / 3.0;
    f[7] = k2OverSqrt6 * sk * sl * cl * cp;
    f[8] = -k2OverSqrt6 * sk * sl * cl * sp;
    f[9] = k2OverSqrt3 * ck * sl * sl;
    double A = 0.0;
#pragma unroll
    for (int k = 0; k < 10; ++k) A += c.h[k] * f[k];
    return A;
}

__device__ __forceinline__ double time_pdf(const Consts& c, double t) {
    const double tau = t - c.mu;
    const double z = (c.Gs2 - tau) * c.k_z;
    return 0.5 * exp(-c.Gamma * tau + c.c_exp) * erfc(z);
}

// ---- FP32 decision filter ----
// Single-precision copies of what the tests read (set once per block).
struct Filter32 {
    float d;          // t_lo - mu
    float span;       // t_hi - t_lo
    float Gamma, c_exp, Gs2, k_z;
    float MT, MO;
    float h[10];
    float bandA;      // absolute band of the angular test: 3e-4 M_Omega
};

constexpr float kTwoM32 = 2.3283064365386963e-10f;   // 2^-32

// u ~ a 2^-32 from the high word of a uniform: |u32 - u| <= 2^-24 u + 2^-31.
__device__ __forceinline__ float u32of(uint32_t hi) { return __uint2float_rn(hi) * kTwoM32; }

// +1: u_t M_T < g(t - mu) for sure; -1: not; 0: undecided (FP64 decides).
// Error bound per candidate (2^-22 ~ 2.4e-7 covers one float rounding with
// a factor 2 to spare): tau = d + u span carries
//   dtau <= 2^-22 (span + |tau| + |d|);
// the exponent a = -Gamma tau + c carries da <= |Gamma| dtau + 2^-21 (|Gamma tau| + |c|);
// expf adds 2 ulp; z = (Gamma sigma^2 - tau) k_z carries dz <= k_z (dtau + 2^-22
// |Gamma sigma^2|) + 2^-21 |z|; erfcf adds 4 ulp and the argument error enters
// through |erfc'(z)| / erfc(z) <= z + sqrt(z^2 + 2) (z >= 0; Abramowitz and
// Stegun 7.1.13) or <= 2/sqrt(pi) (z < 0, where erfc >= 1).
__device__ __forceinline__ int time_filter(const Filter32& f, uint32_t t_hi_word, uint32_t acc_hi_word) {
    const float tau = fmaf(u32of(t_hi_word), f.span, f.d);
    const float dtau = 2.384185791015625e-07f * (f.span + fabsf(tau) + fabsf(f.d));
    const float gt = f.Gamma * tau;
    const float arg = f.c_exp - gt;
    const float z = (f.Gs2 - tau) * f.k_z;
    if (!(fabsf(arg) <= 80.0f) || !(z <= 8.0f)) return 0;
    const float da = fabsf(f.Gamma) * dtau + 4.76837158203125e-07f * (fabsf(gt) + fabsf(f.c_exp));
    const float dz = f.k_z * (dtau + 2.384185791015625e-07f * fabsf(f.Gs2)) + 4.76837158203125e-07f * fabsf(z);
    const float sens = z > 0.0f ? z + sqrtf(fmaf(z, z, 2.0f)) : 1.2f;
    const float rel = 2.0f * (1.01f * da + 1.1f * sens * dz + 2.0e-6f) + 4.0e-6f;
    if (!(rel <= 1.0e-3f)) return 0;
    const float g = 0.5f * expf(arg) * erfcf(z);
    if (!(g >= 1.0e-30f) || !isfinite(g)) return 0;
    const float lhs = u32of(acc_hi_word) * f.MT;
    const float dl = lhs * 4.76837158203125e-07f + f.MT * 9.5367431640625e-07f;
    if (lhs + dl < g * (1.0f - rel)) return 1;
    if (lhs - dl > g * (1.0f + rel)) return -1;
    return 0;
}

// +1 / -1 / 0 for u_a M_Omega < A(Omega), from the words of calls 1 and 2.
// The cosines carry errors below 2.5e-7 and phi below 1.2e-6.  With sin^2 >=
// 1e-2 for both polar angles, the sines (square roots of 1 - c^2, whose error
// is below 4.2e-7) carry errors below 2.2e-6 and the sine and cosine of phi
// below 1.4e-6, so every f_k (constant factor included) is within 1e-5 and
// |A32 - A| <= 1e-5 sum|h_k| + 6e-7 M_Omega <= 3.2e-5 M_Omega (each max|f_k|
// >= 1/3, so sum|h_k| <= 3 M_Omega): the band of 3e-4 M_Omega leaves a factor
// 9 to spare.
__device__ __forceinline__ int angle_filter(const Filter32& f, const U4& b, const U4& e) {
    const float ck = fmaf(2.0f, u32of(b.x), -1.0f);
    const float cl = fmaf(2.0f, u32of(b.z), -1.0f);
    const float sk2 = fmaf(-ck, ck, 1.0f), sl2 = fmaf(-cl, cl, 1.0f);
    if (!(sk2 >= 1.0e-2f) || !(sl2 >= 1.0e-2f)) return 0;
    const float phi = 3.14159265358979323846f * fmaf(2.0f, u32of(e.x), -1.0f);
    float sp, cp;
    sincosf(phi, &sp, &cp);
    const float sk = sqrtf(sk2), sl = sqrtf(sl2);
    const float fk[10] = {ck * ck * sl2,
                          0.5f * sk2 * (1.0f - sl2 * cp * cp),
                          0.5f * sk2 * (1.0f - sl2 * sp * sp),
                          sk2 * sl2 * sp * cp,
                          1.41421356f * sk * ck * sl * cl * cp,
                          -1.41421356f * sk * ck * sl * cl * sp,
                          sl2 * (1.0f / 3.0f),
                          0.81649658f * sk * sl * cl * cp,
                          -0.81649658f * sk * sl * cl * sp,
                          1.15470054f * ck * sl2};
    float A = 0.0f;
#pragma unroll
    for (int k = 0; k < 10; ++k) A = fmaf(f.h[k], fk[k], A);
    const float lhs = u32of(e.z) * f.MO;
    const float dl = f.MO * 9.5367431640625e-07f;
    if (lhs + dl < A - f.bandA) return 1;
    if (lhs - dl > A + f.bandA) return -1;
    return 0;
}


template <int KIND>
__global__ void __launch_bounds__(kBlock)
toygen_kernel(ModelDev m, const Consts* __restrict__ consts, uint32_t k0, uint32_t k1, int n_toys,
              const int64_t* __restrict__ n_sig, const int64_t* __restrict__ n_bkg,
              const int64_t* __restrict__ offsets, int64_t capacity, double* __restrict__ ot,
              double* __restrict__ ock, double* __restrict__ ocl, double* __restrict__ ophi) {
    __shared__ __align__(16) Consts c;
    __shared__ Filter32 f32;
    __shared__ int warp_sums[kBlock / 32];
    {
        const double* src = reinterpret_cast<const double*>(consts);
        double* dst = reinterpret_cast<double*>(&c);
        for (int i = threadIdx.x; i < kConstsDoubles; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const double span = __dsub_rn(m.t_hi, m.t_lo);
    if (threadIdx.x == 0) {
        f32.d = (float)(m.t_lo - c.mu);
        f32.span = (float)span;
        f32.Gamma = (float)c.Gamma;
        f32.c_exp = (float)c.c_exp;
        f32.Gs2 = (float)c.Gs2;
        f32.k_z = (float)c.k_z;
        f32.MT = (float)c.MT;
        f32.MO = (float)c.MO;
        for (int k = 0; k < 10; ++k) f32.h[k] = (float)c.h[k];
        f32.bandA = (float)(3.0e-4 * c.MO);
    }
    __syncthreads();
    for (int toy = blockIdx.x; toy < n_toys; toy += gridDim.x) {
        const int64_t ns = n_sig[toy], nb = n_bkg[toy], off = offsets[toy];
        if (ns < 0 || nb < 0 || off < 0 || off + ns + nb > capacity) continue;   // skipped
        // signal: chunks of kChunk candidates, candidate j = j0 + threadIdx.x * kPerThread + i.
        // Non-finite or non-positive envelopes (non-physical theta) accept nothing: the
        // signal slots are then filled with NaN instead of searching forever, and so
        // is whatever remains when the candidate budget runs out.
        const bool usable = isfinite(c.MT) && c.MT > 0.0 && isfinite(c.MO) && c.MO > 0.0 &&
                            isfinite(c.IT) && c.IT > 0.0;
        const uint64_t budget = usable ? (uint64_t)ns * 65536ull + (1ull << 22) : 0ull;
        int64_t got = 0;
        uint64_t j0 = 0;
        for (; got < ns && j0 < budget; j0 += kChunk) {
            const uint64_t jt = j0 + (uint64_t)threadIdx.x * kPerThread;
            unsigned mask = 0;
#pragma unroll 1
            for (int i = 0; i < kPerThread; ++i) {
                const uint64_t j = jt + i;
                const U4 a = draw(j, (uint32_t)toy, 0u, k0, k1);
                int d = time_filter(f32, a.x, a.z);
                if (d == 0) {
                    const double t = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
                    d = __dmul_rn(u01(a.z, a.w), c.MT) < time_pdf(c, t) ? 1 : -1;
                }
                if (KIND == IPA_MODEL_ANGTIME4D && d > 0) {
                    const U4 b = draw(j, (uint32_t)toy, 1u, k0, k1);
                    const U4 e = draw(j, (uint32_t)toy, 2u, k0, k1);
                    d = angle_filter(f32, b, e);
                    if (d == 0) {
                        const double ck = __dsub_rn(__dmul_rn(2.0, u01(b.x, b.y)), 1.0);
                        const double cl = __dsub_rn(__dmul_rn(2.0, u01(b.z, b.w)), 1.0);
                        const double phi = __dmul_rn(kPi, __dsub_rn(__dmul_rn(2.0, u01(e.x, e.y)), 1.0));
                        d = __dmul_rn(u01(e.z, e.w), c.MO) < angular_pdf(c, ck, cl, phi) ? 1 : -1;
                    }
                }
                if (d > 0) mask |= 1u << i;
            }
            int total;
            const int before = block_exclusive_scan(__popc(mask), warp_sums, &total);
            int rank = 0;
            // accepted candidates are regenerated from their counters (exact FP64 values)
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1u;
                const int64_t pos = got + before + rank;
                ++rank;
                if (pos >= ns) break;
                const uint64_t j = jt + i;
                const U4 a = draw(j, (uint32_t)toy, 0u, k0, k1);
                ot[off + pos] = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
                if (KIND == IPA_MODEL_ANGTIME4D) {
                    const U4 b = draw(j, (uint32_t)toy, 1u, k0, k1);
                    const U4 e = draw(j, (uint32_t)toy, 2u, k0, k1);
                    ock[off + pos] = __dsub_rn(__dmul_rn(2.0, u01(b.x, b.y)), 1.0);
                    ocl[off + pos] = __dsub_rn(__dmul_rn(2.0, u01(b.z, b.w)), 1.0);
                    ophi[off + pos] = __dmul_rn(kPi, __dsub_rn(__dmul_rn(2.0, u01(e.x, e.y)), 1.0));
                }
            }
            got += total;
        }
        for (int64_t pos = got + threadIdx.x; pos < ns; pos += blockDim.x) {
            ot[off + pos] = __longlong_as_double(0x7ff8000000000000ll);
            if (KIND == IPA_MODEL_ANGTIME4D)
                ock[off + pos] = ocl[off + pos] = ophi[off + pos] = __longlong_as_double(0x7ff8000000000000ll);
        }
        // background: uniform in the box, always kept
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
            const U4 a = draw((uint64_t)i, (uint32_t)toy, 4u, k0, k1);
            const int64_t pos = off + ns + i;
            ot[pos] = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
            if (KIND == IPA_MODEL_ANGTIME4D) {
                const U4 b = draw((uint64_t)i, (uint32_t)toy, 5u, k0, k1);
                ock[pos] = __dsub_rn(__dmul_rn(2.0, u01(a.z, a.w)), 1.0);
                ocl[pos] = __dsub_rn(__dmul_rn(2.0, u01(b.x, b.y)), 1.0);
                ophi[pos] = __dmul_rn(kPi, __dsub_rn(__dmul_rn(2.0, u01(b.z, b.w)), 1.0));
            }
        }
    }
}

// The tagged model: candidate j of toy k takes (t, u) from call 0 and the tag
// from the first uniform of call 1 (q = +1 if u_q <= 1/2, else -1), and is
// kept iff u M_S < S(t - mu, q), S evaluated in FP64 with the exact forms of
// tagged.cuh (no filter: the FP64 test runs for every candidate).  Background
// event i takes t and q from call 4.
__global__ void __launch_bounds__(kBlock)
toygen_tag_kernel(ModelDev m, const Consts* __restrict__ consts, uint32_t k0, uint32_t k1, int n_toys,
                  const int64_t* __restrict__ n_sig, const int64_t* __restrict__ n_bkg,
                  const int64_t* __restrict__ offsets, int64_t capacity, double* __restrict__ ot,
                  double* __restrict__ oq) {
    __shared__ __align__(16) TagConsts c;
    __shared__ int warp_sums[kBlock / 32];
    {
        const double* src = reinterpret_cast<const double*>(consts);
        double* dst = reinterpret_cast<double*>(&c);
        for (int i = threadIdx.x; i < kTagConstsDoubles; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const double span = __dsub_rn(m.t_hi, m.t_lo);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int toy = blockIdx.x; toy < n_toys; toy += gridDim.x) {
        const int64_t ns = n_sig[toy], nb = n_bkg[toy], off = offsets[toy];
        if (ns < 0 || nb < 0 || off < 0 || off + ns + nb > capacity) continue;   // skipped
        const bool usable = isfinite(c.MS) && c.MS > 0.0 && isfinite(c.N) && c.N > 0.0;
        const uint64_t budget = usable ? (uint64_t)ns * 65536ull + (1ull << 22) : 0ull;
        int64_t got = 0;
        uint64_t j0 = 0;
        for (; got < ns && j0 < budget; j0 += kChunk) {
            const uint64_t jt = j0 + (uint64_t)threadIdx.x * kPerThread;
            unsigned mask = 0;
#pragma unroll 1
            for (int i = 0; i < kPerThread; ++i) {
                const uint64_t j = jt + i;
                const U4 a = draw(j, (uint32_t)toy, 0u, k0, k1);
                const U4 b = draw(j, (uint32_t)toy, 1u, k0, k1);
                const double t = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
                const double q = u01(b.x, b.y) <= 0.5 ? 1.0 : -1.0;
                if (__dmul_rn(u01(a.z, a.w), c.MS) < tag_signal(c, t, q)) mask |= 1u << i;
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
                ot[off + pos] = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
                oq[off + pos] = u01(b.x, b.y) <= 0.5 ? 1.0 : -1.0;
            }
            got += total;
        }
        for (int64_t pos = got + threadIdx.x; pos < ns; pos += blockDim.x) ot[off + pos] = oq[off + pos] = nan;
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
            const U4 a = draw((uint64_t)i, (uint32_t)toy, 4u, k0, k1);
            const int64_t pos = off + ns + i;
            ot[pos] = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
            oq[pos] = u01(a.z, a.w) <= 0.5 ? 1.0 : -1.0;
        }
    }
}

}  // namespace

ipa_status launch_tag_toygen(const ModelDev& m, const Consts* consts, uint64_t seed, int n_toys,
                             const int64_t* n_sig, const int64_t* n_bkg, const int64_t* offsets,
                             const ipa_event_buffers* out, cudaStream_t s) {
    toygen_tag_kernel<<<n_toys, kBlock, 0, s>>>(m, consts, (uint32_t)seed, (uint32_t)(seed >> 32), n_toys, n_sig,
                                                n_bkg, offsets, out->capacity, out->t, out->q);
    return cuda_fail(cudaGetLastError(), "tagged toygen kernel launch");
}

}  // namespace ipa

extern "C" ipa_status ipa_toygen(const ipa_model* model, const double* theta_dev, uint64_t seed,
                                 int32_t n_toys, const int64_t* n_sig_dev, const int64_t* n_bkg_dev,
                                 const int64_t* offsets_dev, const ipa_event_buffers* out,
                                 void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if (n_toys < 0 || !out || !theta_dev) {
        set_error("ipa_toygen: bad arguments");
        return IPA_ERR_ARG;
    }
    if (n_toys == 0) return IPA_OK;
    if (!n_sig_dev || !n_bkg_dev || !offsets_dev || !out->t || out->capacity < 0) {
        set_error("ipa_toygen: NULL count, offset or output column");
        return IPA_ERR_ARG;
    }
    const bool four = model->kind == IPA_MODEL_ANGTIME4D;
    if (four && (!out->ck || !out->cl || !out->phi)) {
        set_error("ipa_toygen: the 4D model needs ck, cl and phi output columns");
        return IPA_ERR_ARG;
    }
    const bool phis = model->kind == IPA_MODEL_PHIS;
    if (phis && (!out->ck || !out->cl || !out->phi || !out->q)) {
        set_error("ipa_toygen: the phi_s model needs ck, cl, phi and q output columns");
        return IPA_ERR_ARG;
    }
    const bool tag = model->kind == IPA_MODEL_TAGGED1D;
    if (tag && !out->q) {
        set_error("ipa_toygen: the tagged model needs a q output column");
        return IPA_ERR_ARG;
    }
    Scratch* sc = nullptr;
    if ((st = scratch_get(1, 2, &sc)) != IPA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_consts(m, theta_dev, 1, sc->consts, s)) != IPA_OK) return st;
    if (tag) return launch_tag_toygen(m, sc->consts, seed, n_toys, n_sig_dev, n_bkg_dev, offsets_dev, out, s);
    if (phis) return launch_phis_toygen(m, sc->consts, seed, n_toys, n_sig_dev, n_bkg_dev, offsets_dev, out, s);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int grid = n_toys;
    if (four)
        toygen_kernel<IPA_MODEL_ANGTIME4D><<<grid, kBlock, 0, s>>>(
            m, sc->consts, k0, k1, n_toys, n_sig_dev, n_bkg_dev, offsets_dev, out->capacity, out->t,
            out->ck, out->cl, out->phi);
    else
        toygen_kernel<IPA_MODEL_TIME1D><<<grid, kBlock, 0, s>>>(
            m, sc->consts, k0, k1, n_toys, n_sig_dev, n_bkg_dev, offsets_dev, out->capacity, out->t,
            nullptr, nullptr, nullptr);
    return cuda_fail(cudaGetLastError(), "toygen kernel launch");
}
