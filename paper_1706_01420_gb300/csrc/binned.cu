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
// counts are reproducible bit for bit.  The recurrence depends only on the
// bin's mean, so it runs once per bin and call into a CDF table (BinTable);
// a draw is then one Philox block and a few comparisons.
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

// The inversion of one bin, tabulated once per call and shared by every toy:
// with nu = lambda / M, p_0 = exp(-nu), cap = floor(nu + 40 sqrt(nu) + 100), the
// recurrence p_n = (p_{n-1} nu) / n, F_n = F_{n-1} + p_n (each step correctly
// rounded) gives the CDF values F_0, F_1, ...  A draw with uniform u is the
// first n with u <= F_n, or `stop` (the n where the recurrence ends, p = 0 or
// n = cap) when u exceeds them all.  The table keeps F_0 .. F_{len-1}, up to
// the point past the mode where adding p_n no longer changes F (after that no
// u changes the outcome before `stop`), so a draw compares u with the same
// values in the same order as the plain sequential loop, and the counts are
// those of that loop bit for bit.
struct BinTable {
    int64_t off;    // first entry in the flat CDF array
    double nu;      // mean of one piece
    int M;          // pieces (0 for a non-positive mean)
    int len;        // entries F_0 .. F_{len-1}
    int stop;       // the draw when u > F_{len-1}
    int pad_;
};

// Run the recurrence of one bin: entries and stop index; with F != nullptr
// also write the entries.
__device__ inline void bin_recurrence(double lam, BinTable* t, double* F) {
    if (!(lam > 0.0)) {
        t->M = 0;
        t->nu = 0.0;
        t->len = 0;
        t->stop = 0;
        return;
    }
    const double Md = ceil(lam / kPiece);
    const int M = Md < 1.0 ? 1 : (int)Md;
    const double nu = __ddiv_rn(lam, (double)M);
    const double cap = floor(__dadd_rn(__dadd_rn(nu, __dmul_rn(40.0, sqrt(nu))), 100.0));
    double p = exp(-nu), f = p;
    int n = 0, len = 1;
    bool settled = false;
    if (F) F[0] = f;
    // u <= 1 < any F would end the loop anyway; u > F runs it to p = 0 or n = cap
    while (p > 0.0 && (double)n < cap) {
        n += 1;
        p = __ddiv_rn(__dmul_rn(p, nu), (double)n);
        const double g = __dadd_rn(f, p);
        if (!settled) {
            if (g == f && (double)n > nu) {
                settled = true;
            } else {
                if (F) F[len] = g;
                ++len;
            }
        }
        f = g;
    }
    t->M = M;
    t->nu = nu;
    t->len = len;
    t->stop = n;
}

__device__ __forceinline__ int table_draw(const BinTable& t, const double* __restrict__ F, double u) {
    const double* f = F + t.off;
    int j = 0;
    while (j < t.len && u > __ldg(f + j)) ++j;
    return j < t.len ? j : t.stop;
}

__device__ __forceinline__ int poisson_bin(const BinTable& t, const double* __restrict__ F, uint64_t i, uint32_t toy,
                                           int hyp, uint32_t k0, uint32_t k1) {
    int n = 0;
    for (int m = 0; m < t.M; ++m) {
        const U4 r = draw(i, toy, binned_call(hyp, m), k0, k1);
        const double u = (m & 1) ? u01(r.z, r.w) : u01(r.x, r.y);
        n += table_draw(t, F, u);
    }
    return n;
}

__global__ void table_size_kernel(const double* __restrict__ lam, const double* __restrict__ add, int64_t n_bins,
                                  BinTable* __restrict__ tab) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bins; i += (int64_t)gridDim.x * blockDim.x) {
        const double l = add ? __ldg(lam + i) + __ldg(add + i) : __ldg(lam + i);
        BinTable t{};
        bin_recurrence(l, &t, nullptr);
        tab[i] = t;
    }
}

// off[i] = sum_{r<i} len_r (one block: a sequential run per thread, then a
// block scan of the run totals); *total = the sum.
__global__ void table_offsets_kernel(BinTable* __restrict__ tab, int64_t n_bins, int64_t* __restrict__ total) {
    __shared__ int64_t run[1024];
    const int nt = blockDim.x;
    const int64_t per = (n_bins + nt - 1) / nt;
    const int64_t b = threadIdx.x * per;
    const int64_t e = b + per < n_bins ? b + per : n_bins;
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += tab[i].len;
    run[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        const int64_t v = threadIdx.x >= d ? run[threadIdx.x - d] : 0;
        __syncthreads();
        run[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t acc = threadIdx.x ? run[threadIdx.x - 1] : 0;
    for (int64_t i = b; i < e; ++i) {
        tab[i].off = acc;
        acc += tab[i].len;
    }
    if (threadIdx.x == nt - 1) *total = run[nt - 1];
}

__global__ void table_fill_kernel(const double* __restrict__ lam, const double* __restrict__ add, int64_t n_bins,
                                  const BinTable* __restrict__ tab, double* __restrict__ F) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bins; i += (int64_t)gridDim.x * blockDim.x) {
        const double l = add ? __ldg(lam + i) + __ldg(add + i) : __ldg(lam + i);
        BinTable t{};
        bin_recurrence(l, &t, F + tab[i].off);
    }
}

__global__ void __launch_bounds__(kBinBlock)
generate_kernel(const BinTable* __restrict__ tab, const double* __restrict__ F, int64_t n_bins, uint32_t k0,
                uint32_t k1, int hyp, int toy0, int n_toys, int32_t* __restrict__ counts) {
    const int64_t total = n_bins * (int64_t)n_toys;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = x / n_bins, i = x - k * n_bins;
        counts[x] = poisson_bin(tab[i], F, (uint64_t)i, (uint32_t)(toy0 + k), hyp, k0, k1);
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

// w_i = ln(1 + s_i / b_i).
__global__ void cls_weights_kernel(const double* __restrict__ s, const double* __restrict__ b, int64_t n_bins,
                                   double* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bins; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = log1p(__ldg(s + i) / __ldg(b + i));
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
cls_toys_kernel(const BinTable* __restrict__ tab, const double* __restrict__ F, const double* __restrict__ w,
                int64_t n_bins, uint32_t k0, uint32_t k1, int hyp, int n_toys, const int32_t* __restrict__ data,
                double* __restrict__ x_out) {
    __shared__ double part[kBinBlock / 32];
    const int first = data ? 0 : blockIdx.x;
    const int stride = data ? 1 : gridDim.x;
    const int last = data ? 1 : n_toys;
    for (int k = first; k < last; k += stride) {
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n_bins; i += blockDim.x) {
            const int n = data ? __ldg(data + i) : poisson_bin(tab[i], F, (uint64_t)i, (uint32_t)k, hyp, k0, k1);
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

// The CDF tables of the bin means lam (+ add, if given), in stream-ordered
// allocations the caller frees with cudaFreeAsync.  Synchronises the stream
// once (the size of the flat table).
ipa_status build_tables(const double* lam, const double* add, int64_t n_bins, cudaStream_t s, BinTable** tab,
                        double** F, int64_t* scratch_total, int64_t* host_total);

int grid_for(int64_t work) {
    const int64_t g = (work + kBinBlock - 1) / kBinBlock;
    const int64_t cap = (int64_t)sm_count() * 16;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

ipa_status build_tables(const double* lam, const double* add, int64_t n_bins, cudaStream_t s, BinTable** tab,
                        double** F, int64_t* scratch_total, int64_t* host_total) {
    *tab = nullptr;
    *F = nullptr;
    ipa_status st = cuda_fail(cudaMallocAsync((void**)tab, sizeof(BinTable) * (size_t)n_bins, s), "binned tables");
    if (st != IPA_OK) return st;
    table_size_kernel<<<grid_for(n_bins), kBinBlock, 0, s>>>(lam, add, n_bins, *tab);
    table_offsets_kernel<<<1, 1024, 0, s>>>(*tab, n_bins, scratch_total);
    if ((st = cuda_fail(cudaMemcpyAsync(host_total, scratch_total, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                        "binned table size")) != IPA_OK)
        return st;
    if ((st = cuda_fail(cudaStreamSynchronize(s), "binned table size")) != IPA_OK) return st;
    if ((st = cuda_fail(cudaMallocAsync((void**)F, sizeof(double) * (size_t)(*host_total > 0 ? *host_total : 1), s),
                        "binned tables")) != IPA_OK)
        return st;
    table_fill_kernel<<<grid_for(n_bins), kBinBlock, 0, s>>>(lam, add, n_bins, *tab, *F);
    return cuda_fail(cudaGetLastError(), "binned table launch");
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
    int64_t* total = nullptr;
    ipa_status st = cuda_fail(cudaMallocAsync((void**)&total, sizeof(int64_t), s), "binned scratch");
    if (st != IPA_OK) return st;
    BinTable* tab = nullptr;
    double* F = nullptr;
    int64_t h_total = 0;
    st = build_tables(lambda_dev, nullptr, n_bins, s, &tab, &F, total, &h_total);
    if (st == IPA_OK) {
        generate_kernel<<<grid_for(n_bins * n_toys), kBinBlock, 0, s>>>(tab, F, n_bins, (uint32_t)seed,
                                                                        (uint32_t)(seed >> 32), hypothesis, toy0,
                                                                        n_toys, counts_out_dev);
        st = cuda_fail(cudaGetLastError(), "binned generator launch");
    }
    if (F) cudaFreeAsync(F, s);
    if (tab) cudaFreeAsync(tab, s);
    cudaFreeAsync(total, s);
    return st;
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
    // two counters, the table size, w per bin, X per toy (unless the caller keeps them)
    const size_t bytes = 32 + nb * sizeof(double) + (x_out_dev ? 0 : (2 * nt + 1) * sizeof(double));
    unsigned char* buf = nullptr;
    ipa_status st = cuda_fail(cudaMallocAsync((void**)&buf, bytes, s), "cls scratch alloc");
    if (st != IPA_OK) return st;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(buf);
    int64_t* total = reinterpret_cast<int64_t*>(buf + 16);
    double* w = reinterpret_cast<double*>(buf + 32);
    double* x = x_out_dev ? x_out_dev : w + nb;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    BinTable *tb = nullptr, *tsb = nullptr;
    double *Fb = nullptr, *Fsb = nullptr;
    int64_t h_total = 0;
    st = build_tables(b_dev, nullptr, n_bins, s, &tb, &Fb, total, &h_total);
    if (st == IPA_OK) st = build_tables(s_dev, b_dev, n_bins, s, &tsb, &Fsb, total, &h_total);
    if (st == IPA_OK) {
        cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s);
        cls_weights_kernel<<<grid_for(n_bins), kBinBlock, 0, s>>>(s_dev, b_dev, n_bins, w);
        const int gt = n_toys < sm_count() * 8 ? n_toys : sm_count() * 8;
        cls_toys_kernel<<<gt, kBinBlock, 0, s>>>(tb, Fb, w, n_bins, k0, k1, 0, n_toys, nullptr, x);
        cls_toys_kernel<<<gt, kBinBlock, 0, s>>>(tsb, Fsb, w, n_bins, k0, k1, 1, n_toys, nullptr, x + nt);
        cls_toys_kernel<<<1, kBinBlock, 0, s>>>(tb, Fb, w, n_bins, k0, k1, 0, 1, data_dev, x + 2 * nt);
        cls_count_kernel<<<grid_for(n_toys), kBinBlock, 0, s>>>(x, x + nt, x + 2 * nt, n_toys, cnt);
        cls_final_kernel<<<1, 1, 0, s>>>(cnt, n_toys, cl_out_dev, counts_out_dev);
        st = cuda_fail(cudaGetLastError(), "cls launch");
    }
    if (Fb) cudaFreeAsync(Fb, s);
    if (tb) cudaFreeAsync(tb, s);
    if (Fsb) cudaFreeAsync(Fsb, s);
    if (tsb) cudaFreeAsync(tsb, s);
    cudaFreeAsync(buf, s);
    return st;
}
