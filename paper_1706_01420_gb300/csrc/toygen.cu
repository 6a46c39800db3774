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
#include <math.h>

#include "consts.cuh"
#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
constexpr int kPerThread = 4;              // candidates per thread per chunk
constexpr int kChunk = kBlock * kPerThread;
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double k2OverSqrt6 = 0.81649658092772603273;
constexpr double k2OverSqrt3 = 1.15470053837925152902;

struct U4 {
    uint32_t x, y, z, w;
};

// Philox-4x32 with 10 rounds.  Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
// c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key bumped by (W0, W1) between rounds.
__device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += kW0;
            k1 += kW1;
        }
        const uint32_t lo0 = kM0 * c.x, hi0 = __umulhi(kM0, c.x);
        const uint32_t lo1 = kM1 * c.z, hi1 = __umulhi(kM1, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
    const unsigned long long v = ((((unsigned long long)a) << 32) | b) >> 11;
    return __dmul_rn(__ull2double_rn(v + 1ull), 0x1p-53);
}

__device__ __forceinline__ U4 draw(uint64_t idx, uint32_t toy, uint32_t call, uint32_t k0, uint32_t k1) {
    return philox(U4{(uint32_t)idx, (uint32_t)(idx >> 32), toy, call}, k0, k1);
}

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

// Exclusive scan of one int per thread over the block; returns the prefix and
// writes the block total to *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < kBlock / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < kBlock / 32) warp_sums[lane] = s;   // inclusive warp prefix
    }
    __syncthreads();
    const int before = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[kBlock / 32 - 1];
    __syncthreads();
    return before + x - v;
}

template <int KIND>
__global__ void __launch_bounds__(kBlock)
toygen_kernel(ModelDev m, const Consts* __restrict__ consts, uint32_t k0, uint32_t k1, int n_toys,
              const int64_t* __restrict__ n_sig, const int64_t* __restrict__ n_bkg,
              const int64_t* __restrict__ offsets, int64_t capacity, double* __restrict__ ot,
              double* __restrict__ ock, double* __restrict__ ocl, double* __restrict__ ophi) {
    __shared__ __align__(16) Consts c;
    __shared__ int warp_sums[kBlock / 32];
    {
        const double* src = reinterpret_cast<const double*>(consts);
        double* dst = reinterpret_cast<double*>(&c);
        for (int i = threadIdx.x; i < kConstsDoubles; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const double span = __dsub_rn(m.t_hi, m.t_lo);
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
            double vt[kPerThread], vk[kPerThread], vl[kPerThread], vp[kPerThread];
            unsigned mask = 0;
#pragma unroll
            for (int i = 0; i < kPerThread; ++i) {
                const uint64_t j = j0 + (uint64_t)threadIdx.x * kPerThread + i;
                const U4 a = draw(j, (uint32_t)toy, 0u, k0, k1);
                const double t = __dadd_rn(m.t_lo, __dmul_rn(u01(a.x, a.y), span));
                vt[i] = t;
                bool keep = __dmul_rn(u01(a.z, a.w), c.MT) < time_pdf(c, t);
                if (KIND == IPA_MODEL_ANGTIME4D && keep) {
                    const U4 b = draw(j, (uint32_t)toy, 1u, k0, k1);
                    const U4 d = draw(j, (uint32_t)toy, 2u, k0, k1);
                    vk[i] = __dsub_rn(__dmul_rn(2.0, u01(b.x, b.y)), 1.0);
                    vl[i] = __dsub_rn(__dmul_rn(2.0, u01(b.z, b.w)), 1.0);
                    vp[i] = __dmul_rn(kPi, __dsub_rn(__dmul_rn(2.0, u01(d.x, d.y)), 1.0));
                    keep = __dmul_rn(u01(d.z, d.w), c.MO) < angular_pdf(c, vk[i], vl[i], vp[i]);
                }
                if (keep) mask |= 1u << i;
            }
            int total;
            const int before = block_exclusive_scan(__popc(mask), warp_sums, &total);
            int rank = 0;
#pragma unroll
            for (int i = 0; i < kPerThread; ++i) {
                if (mask & (1u << i)) {
                    const int64_t pos = got + before + rank;
                    ++rank;
                    if (pos < ns) {
                        ot[off + pos] = vt[i];
                        if (KIND == IPA_MODEL_ANGTIME4D) {
                            ock[off + pos] = vk[i];
                            ocl[off + pos] = vl[i];
                            ophi[off + pos] = vp[i];
                        }
                    }
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

}  // namespace
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
    Scratch* sc = nullptr;
    if ((st = scratch_get(1, 2, &sc)) != IPA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_consts(m, theta_dev, 1, sc->consts, s)) != IPA_OK) return st;
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
