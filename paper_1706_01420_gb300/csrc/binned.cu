// Binned workloads (Example 4, CLs, and the toolkit's generateBinned and
// Gaussian smearing): Poisson pseudo-experiments of a histogram, the smearing
// of a histogram by a Gaussian, and CL_b, CL_s+b, CL_s from toys.
//
// Poisson counts.  Bin i of toy k under hypothesis h is Poisson(lambda_i) by
// inversion of the CDF with one uniform per piece from Philox-4x32-10
// (philox.cuh): counter (i lo32, i hi32, k, 8 + 2^16 h + m/2), words 2 (m mod 2)
// and 2 (m mod 2) + 1; a mean above 400 is split into M = ceil(lambda/400)
// pieces of lambda/M (Poisson counts add).  Piece of mean nu, uniform u:
//   n = 0, p = exp(-nu), F = p;  while u > F and p > 0 and n < cap:
//   n += 1, p = (p nu) / n, F += p;   cap = floor(nu + 40 sqrt(nu) + 100).
// Every step is a correctly rounded IEEE operation (no contraction), so the
// counts are reproducible bit for bit.
//
// CLs.  With w_i = ln(1 + s_i / b_i), X = sum_i n_i w_i (the data-dependent part
// of -2 ln Q, Q = L(s+b) / L(b)); CL_s+b = P_s+b(X <= X_obs), CL_b =
// P_b(X <= X_obs), CL_s = CL_s+b / CL_b over n_toys toys per hypothesis.  One
// block per toy draws its bins on the fly (no histogram is stored) and adds
// n_i w_i in a fixed order (thread-strided partial sums, then a fixed tree).
#include <math.h>

#include "ipa_internal.cuh"
#include "philox.cuh"

namespace ipa {
namespace {

constexpr double kPiece = 400.0;
constexpr int kBinBlock = 256;
constexpr uint32_t kBinnedCall = 8u;

__device__ __forceinline__ uint32_t binned_call(int hyp, int m) {
    return kBinnedCall + ((uint32_t)hyp << 16) + (uint32_t)(m >> 1);
}

// One piece: inversion with its exp(-nu) given.
__device__ __forceinline__ int poisson_piece(double nu, double p0, double u) {
    int n = 0;
    double p = p0, F = p0;
    const double cap = floor(__dadd_rn(__dadd_rn(nu, __dmul_rn(40.0, sqrt(nu))), 100.0));
    while (u > F && p > 0.0 && (double)n < cap) {
        n += 1;
        p = __ddiv_rn(__dmul_rn(p, nu), (double)n);
        F = __dadd_rn(F, p);
    }
    return n;
}

// Pieces of a bin mean: M, nu = lambda / M and exp(-nu).
struct BinMean {
    double nu, p0;
    int M;
};

__device__ __forceinline__ BinMean bin_mean(double lam) {
    BinMean b;
    if (!(lam > 0.0)) {
        b.M = 0;
        b.nu = 0.0;
        b.p0 = 1.0;
        return b;
    }
    const double Md = ceil(lam / kPiece);
    b.M = Md < 1.0 ? 1 : (int)Md;
    b.nu = __ddiv_rn(lam, (double)b.M);
    b.p0 = exp(-b.nu);
    return b;
}

__device__ __forceinline__ int poisson_bin(const BinMean& bm, uint64_t i, uint32_t toy, int hyp, uint32_t k0,
                                           uint32_t k1) {
    int n = 0;
    for (int m = 0; m < bm.M; ++m) {
        const U4 r = draw(i, toy, binned_call(hyp, m), k0, k1);
        const double u = (m & 1) ? u01(r.z, r.w) : u01(r.x, r.y);
        n += poisson_piece(bm.nu, bm.p0, u);
    }
    return n;
}

__global__ void __launch_bounds__(kBinBlock)
generate_kernel(const double* __restrict__ lam, int64_t n_bins, uint32_t k0, uint32_t k1, int hyp, int toy0,
                int n_toys, int32_t* __restrict__ counts) {
    const int64_t total = n_bins * (int64_t)n_toys;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = x / n_bins, i = x - k * n_bins;
        const BinMean bm = bin_mean(__ldg(lam + i));
        counts[x] = poisson_bin(bm, (uint64_t)i, (uint32_t)(toy0 + k), hyp, k0, k1);
    }
}

// Discrete Gaussian kernel K_d (|d| <= R), normalised to unit sum (one block).
__global__ void smear_weights_kernel(int R, double width, double sigma, double* __restrict__ K) {
    __shared__ double part[kBinBlock];
    const int n = 2 * R + 1;
    const double c = 1.0 / (2.0 * sigma * sigma);
    double acc = 0.0;
    for (int d = threadIdx.x; d < n; d += blockDim.x) {
        const double x = (d - R) * width;
        const double v = exp(-(x * x) * c);
        K[d] = v;
        acc += v;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    const double inv = 1.0 / part[0];
    for (int d = threadIdx.x; d < n; d += blockDim.x) K[d] *= inv;
}

// out_i = sum_{|d| <= R} K_d h_{i-d}, bins outside the histogram contributing nothing.
__global__ void __launch_bounds__(kBinBlock)
smear_kernel(const double* __restrict__ h, int64_t n_bins, int R, const double* __restrict__ K,
             double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bins; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j0 = i - R < 0 ? 0 : i - R;
        const int64_t j1 = i + R >= n_bins ? n_bins - 1 : i + R;
        double acc = 0.0;
        for (int64_t j = j0; j <= j1; ++j) acc = fma(__ldg(K + (i - j + R)), __ldg(h + j), acc);
        out[i] = acc;
    }
}

// Per bin: w_i and the pieces of both hypotheses' means.
__global__ void cls_prepare_kernel(const double* __restrict__ s, const double* __restrict__ b, int64_t n_bins,
                                   double* __restrict__ w, BinMean* __restrict__ mb, BinMean* __restrict__ msb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bins; i += (int64_t)gridDim.x * blockDim.x) {
        const double si = __ldg(s + i), bi = __ldg(b + i);
        w[i] = log1p(si / bi);
        mb[i] = bin_mean(bi);
        msb[i] = bin_mean(si + bi);
    }
}

// Fixed-order block sum (every thread gets the total).
__device__ __forceinline__ double block_sum(double v, double* part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
    __syncthreads();
    return t;
}

// X of toy k under hypothesis h (blocks stride over toys); toy index -1: the data.
__global__ void __launch_bounds__(kBinBlock)
cls_toys_kernel(const BinMean* __restrict__ mean, const double* __restrict__ w, int64_t n_bins, uint32_t k0,
                uint32_t k1, int hyp, int n_toys, const int32_t* __restrict__ data, double* __restrict__ x_out) {
    __shared__ double part[kBinBlock / 32];
    const int first = data ? 0 : blockIdx.x;
    const int stride = data ? 1 : gridDim.x;
    const int last = data ? 1 : n_toys;
    for (int k = first; k < last; k += stride) {
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n_bins; i += blockDim.x) {
            const int n = data ? __ldg(data + i) : poisson_bin(mean[i], (uint64_t)i, (uint32_t)k, hyp, k0, k1);
            if (n) acc = fma((double)n, __ldg(w + i), acc);
        }
        const double X = block_sum(acc, part);
        if (threadIdx.x == 0) x_out[data ? 0 : k] = X;
    }
}

// counts[0] = #{k: X_b[k] <= X_obs}, counts[1] = #{k: X_sb[k] <= X_obs}; then the CLs.
__global__ void cls_count_kernel(const double* __restrict__ xb, const double* __restrict__ xsb,
                                 const double* __restrict__ xobs, int n_toys, unsigned long long* __restrict__ cnt) {
    const double xo = *xobs;
    unsigned long long a = 0, c = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_toys; k += gridDim.x * blockDim.x) {
        a += xb[k] <= xo;
        c += xsb[k] <= xo;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(cnt, a);
        atomicAdd(cnt + 1, c);
    }
}

__global__ void cls_final_kernel(const unsigned long long* __restrict__ cnt, int n_toys, double* __restrict__ cl,
                                 int64_t* __restrict__ counts) {
    const double nb = (double)cnt[0], nsb = (double)cnt[1];
    const double clb = nb / n_toys, clsb = nsb / n_toys;
    cl[0] = clb;
    cl[1] = clsb;
    cl[2] = cnt[0] ? clsb / clb : __longlong_as_double(0x7ff8000000000000ll);
    if (counts) {
        counts[0] = (int64_t)cnt[0];
        counts[1] = (int64_t)cnt[1];
    }
}

int grid_for(int64_t work) {
    const int64_t g = (work + kBinBlock - 1) / kBinBlock;
    const int64_t cap = (int64_t)sm_count() * 16;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_binned_generate(const double* lambda_dev, int64_t n_bins, uint64_t seed, int32_t hypothesis,
                                          int32_t toy0, int32_t n_toys, int32_t* counts_out_dev, void* stream) {
    using namespace ipa;
    if (n_bins < 0 || n_toys < 0 || toy0 < 0 || hypothesis < 0 || hypothesis > 1 ||
        (n_bins > 0 && n_toys > 0 && (!lambda_dev || !counts_out_dev))) {
        set_error("ipa_binned_generate: bad arguments");
        return IPA_ERR_ARG;
    }
    if (n_bins == 0 || n_toys == 0) return IPA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    generate_kernel<<<grid_for(n_bins * n_toys), kBinBlock, 0, s>>>(lambda_dev, n_bins, (uint32_t)seed,
                                                                    (uint32_t)(seed >> 32), hypothesis, toy0, n_toys,
                                                                    counts_out_dev);
    return cuda_fail(cudaGetLastError(), "binned generator launch");
}

extern "C" ipa_status ipa_binned_smear(const double* hist_dev, int64_t n_bins, double bin_width, double sigma,
                                       double* out_dev, void* stream) {
    using namespace ipa;
    if (n_bins < 0 || !(bin_width > 0.0) || !(sigma > 0.0) || (n_bins > 0 && (!hist_dev || !out_dev)) ||
        hist_dev == out_dev) {
        set_error("ipa_binned_smear: bad arguments (positive width and sigma, distinct arrays)");
        return IPA_ERR_ARG;
    }
    const double Rd = ceil(8.0 * sigma / bin_width);
    if (!(Rd <= 1e7)) {
        set_error("ipa_binned_smear: sigma spans more than 1e7 / 8 bins");
        return IPA_ERR_ARG;
    }
    if (n_bins == 0) return IPA_OK;
    const int R = (int)Rd;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* K = nullptr;
    ipa_status st = cuda_fail(cudaMallocAsync(&K, sizeof(double) * (2 * (size_t)R + 1), s), "smearing kernel alloc");
    if (st != IPA_OK) return st;
    smear_weights_kernel<<<1, kBinBlock, 0, s>>>(R, bin_width, sigma, K);
    smear_kernel<<<grid_for(n_bins), kBinBlock, 0, s>>>(hist_dev, n_bins, R, K, out_dev);
    st = cuda_fail(cudaGetLastError(), "smearing launch");
    cudaFreeAsync(K, s);
    return st;
}

extern "C" ipa_status ipa_cls(const double* s_dev, const double* b_dev, int64_t n_bins, const int32_t* data_dev,
                              int32_t n_toys, uint64_t seed, double* cl_out_dev, int64_t* counts_out_dev,
                              double* x_out_dev, void* stream) {
    using namespace ipa;
    if (n_bins < 1 || n_toys < 1 || !s_dev || !b_dev || !data_dev || !cl_out_dev) {
        set_error("ipa_cls: bad arguments");
        return IPA_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nb = (size_t)n_bins, nt = (size_t)n_toys;
    // per bin: w, two BinMeans; per toy: X under b and s+b, X_obs; two counters
    const size_t bytes = nb * (sizeof(double) + 2 * sizeof(BinMean)) + (x_out_dev ? 0 : (2 * nt + 1) * sizeof(double)) +
                         2 * sizeof(unsigned long long) + 64;
    unsigned char* buf = nullptr;
    ipa_status st = cuda_fail(cudaMallocAsync((void**)&buf, bytes, s), "cls scratch alloc");
    if (st != IPA_OK) return st;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(buf);
    double* w = reinterpret_cast<double*>(buf + 16);
    BinMean* mb = reinterpret_cast<BinMean*>(w + nb);
    BinMean* msb = mb + nb;
    double* x = x_out_dev ? x_out_dev : reinterpret_cast<double*>(msb + nb);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s);
    cls_prepare_kernel<<<grid_for(n_bins), kBinBlock, 0, s>>>(s_dev, b_dev, n_bins, w, mb, msb);
    const int gt = n_toys < sm_count() * 8 ? n_toys : sm_count() * 8;
    cls_toys_kernel<<<gt, kBinBlock, 0, s>>>(mb, w, n_bins, k0, k1, 0, n_toys, nullptr, x);
    cls_toys_kernel<<<gt, kBinBlock, 0, s>>>(msb, w, n_bins, k0, k1, 1, n_toys, nullptr, x + nt);
    cls_toys_kernel<<<1, kBinBlock, 0, s>>>(mb, w, n_bins, k0, k1, 0, 1, data_dev, x + 2 * nt);
    cls_count_kernel<<<grid_for(n_toys), kBinBlock, 0, s>>>(x, x + nt, x + 2 * nt, n_toys, cnt);
    cls_final_kernel<<<1, 1, 0, s>>>(cnt, n_toys, cl_out_dev, counts_out_dev);
    st = cuda_fail(cudaGetLastError(), "cls launch");
    cudaFreeAsync(buf, s);
    return st;
}
