// FP64 roofline calibration: the DFMA issue rate of this GPU and the cost of
// the FP64 math functions the likelihood kernels call, in DFMA slots.
//
// Each kernel runs 8 independent dependency chains per thread at full
// occupancy (one 256-thread block per SM x 8), so it measures throughput, not
// latency.  clock64() gives cycles per SM, cudaEvent gives seconds; their
// ratio is the SM clock during the run.
#include <math.h>

#include "fp64_math.cuh"
#include "int_math.cuh"
#include "ipa_internal.cuh"

namespace ipa {
namespace {

constexpr int kCalBlocksPerSm = 8;
constexpr int kCalThreads = 256;

template <int OP>
__global__ void __launch_bounds__(kCalThreads)
calib_kernel(const double* __restrict__ in, double* __restrict__ out, int iters,
             long long* __restrict__ cycles) {
    __shared__ MathTables mt;
    if (OP >= 7) {
        load_math_tables(&mt);
        __syncthreads();
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = in[i] + 0.125 * k;
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (OP == 0) x[k] = fma(x[k], 0.9999999, 1e-7);
            if (OP == 1) x[k] = exp(x[k]) * 1e-3;           // stays near 1e-3
            if (OP == 2) x[k] = erfc(x[k]);                 // stays in [0, 1]
            if (OP == 3) x[k] = log(x[k] + 2.0);            // stays near 1.15
            if (OP == 4) {
                double s, c;
                sincos(x[k], &s, &c);
                x[k] = s + c;                               // stays in [-1.5, 1.5]
            }
            if (OP == 5) x[k] = sqrt(x[k] + 1.0);           // tends to 1.618
            if (OP == 6) x[k] = 1.0 / (x[k] + 1.5);         // stays in (0.3, 0.7)
            // the library's own table-driven functions (fp64_math.cuh)
            if (OP == 7) x[k] = exp_fast(x[k], &mt) * 1e-3;
            if (OP == 8) x[k] = log_fast(x[k] + 2.0, &mt);
            if (OP == 9) {
                double s, c;
                sincos_fast(x[k], &mt, &s, &c);
                x[k] = s + c;
            }
            if (OP == 10) x[k] = erfcx_poly(x[k], &mt) - 0.25;  // stays in [0, 1]
            // the integer-pipe functions (int_math.cuh): their time alone, in DFMA
            // slots (in the likelihood kernel it overlaps the FP64 work)
            if (OP == 11) x[k] = exp_int(x[k], &mt) * 1e-3;
            if (OP == 12) {
                double s, c;
                sincos_int(x[k], &mt, &s, &c);
                x[k] = s + c;
            }
        }
    }
    const long long c1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[i] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

template <int OP>
ipa_status run_one(const double* in, double* out, long long* cyc, int blocks, int iters,
                   cudaStream_t s, double* sec, double* cycles_per_block) {
    ipa_status st;
    calib_kernel<OP><<<blocks, kCalThreads, 0, s>>>(in, out, iters, cyc);   // warm-up
    if ((st = cuda_fail(cudaGetLastError(), "calibration launch")) != IPA_OK) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    calib_kernel<OP><<<blocks, kCalThreads, 0, s>>>(in, out, iters, cyc);
    cudaEventRecord(e1, s);
    st = cuda_fail(cudaEventSynchronize(e1), "calibration run");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != IPA_OK) return st;
    long long h[4096];
    const int nb = blocks < 4096 ? blocks : 4096;
    if ((st = cuda_fail(cudaMemcpy(h, cyc, sizeof(long long) * nb, cudaMemcpyDeviceToHost), "calibration copy")) != IPA_OK)
        return st;
    double mx = 0.0;
    for (int b = 0; b < nb; ++b) mx = h[b] > mx ? (double)h[b] : mx;
    *sec = ms * 1e-3;
    *cycles_per_block = mx;
    return IPA_OK;
}

}  // namespace
}  // namespace ipa

// results (host, 15 doubles):
//   [0] DFMA per clock per SM, [1] DFMA per second (whole GPU),
//   [2..7] cost in DFMA slots of the library exp, erfc, log, sincos, sqrt, 1/x,
//   [8] SM clock during the DFMA run [MHz],
//   [9..12] cost of this library's exp_fast, log_fast, sincos_fast, erfcx_poly,
//   [13..14] time of exp_int and sincos_int alone, in DFMA slots.
extern "C" ipa_status ipa_calibrate_fp64(double* results, void* stream) {
    using namespace ipa;
    if (!results) {
        set_error("ipa_calibrate_fp64: results is NULL");
        return IPA_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = sm_count();
    const int blocks = sms * kCalBlocksPerSm;
    const int n = blocks * kCalThreads;
    double *in = nullptr, *out = nullptr;
    long long* cyc = nullptr;
    ipa_status st;
    if ((st = device_alloc((void**)&in, sizeof(double) * n, "calibration alloc")) != IPA_OK) return st;
    if ((st = device_alloc((void**)&out, sizeof(double) * n, "calibration alloc")) != IPA_OK) {
        cudaFree(in);
        return st;
    }
    if ((st = device_alloc((void**)&cyc, sizeof(long long) * blocks, "calibration alloc")) != IPA_OK) {
        cudaFree(in);
        cudaFree(out);
        return st;
    }
    cudaMemsetAsync(in, 0, sizeof(double) * n, s);
    double sec[13], cpb[13];
    const int iters[13] = {4096, 256, 128, 256, 256, 512, 512, 256, 256, 256, 256, 256, 256};
    st = run_one<0>(in, out, cyc, blocks, iters[0], s, &sec[0], &cpb[0]);
    if (st == IPA_OK) st = run_one<1>(in, out, cyc, blocks, iters[1], s, &sec[1], &cpb[1]);
    if (st == IPA_OK) st = run_one<2>(in, out, cyc, blocks, iters[2], s, &sec[2], &cpb[2]);
    if (st == IPA_OK) st = run_one<3>(in, out, cyc, blocks, iters[3], s, &sec[3], &cpb[3]);
    if (st == IPA_OK) st = run_one<4>(in, out, cyc, blocks, iters[4], s, &sec[4], &cpb[4]);
    if (st == IPA_OK) st = run_one<5>(in, out, cyc, blocks, iters[5], s, &sec[5], &cpb[5]);
    if (st == IPA_OK) st = run_one<6>(in, out, cyc, blocks, iters[6], s, &sec[6], &cpb[6]);
    if (st == IPA_OK) st = run_one<7>(in, out, cyc, blocks, iters[7], s, &sec[7], &cpb[7]);
    if (st == IPA_OK) st = run_one<8>(in, out, cyc, blocks, iters[8], s, &sec[8], &cpb[8]);
    if (st == IPA_OK) st = run_one<9>(in, out, cyc, blocks, iters[9], s, &sec[9], &cpb[9]);
    if (st == IPA_OK) st = run_one<10>(in, out, cyc, blocks, iters[10], s, &sec[10], &cpb[10]);
    if (st == IPA_OK) st = run_one<11>(in, out, cyc, blocks, iters[11], s, &sec[11], &cpb[11]);
    if (st == IPA_OK) st = run_one<12>(in, out, cyc, blocks, iters[12], s, &sec[12], &cpb[12]);
    cudaFree(in);
    cudaFree(out);
    cudaFree(cyc);
    if (st != IPA_OK) return st;
    // ops per SM in the DFMA run: blocks/SM * threads * iters * 8 chains
    const double ops_per_sm = (double)kCalBlocksPerSm * kCalThreads * iters[0] * 8.0;
    results[0] = ops_per_sm / cpb[0];
    results[1] = ops_per_sm * sms / sec[0];
    const double dfma_time_per_op = sec[0] / (ops_per_sm * sms);
    // each loop body adds one FP64 operation besides the call, except erfc
    const double extra[13] = {0.0, 1.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0};
    for (int f = 1; f < 13; ++f) {
        const double calls = (double)blocks * kCalThreads * iters[f] * 8.0;
        const double cost = (sec[f] / calls) / dfma_time_per_op - extra[f];
        results[f < 7 ? 1 + f : 2 + f] = cost;
    }
    results[8] = cpb[0] / sec[0] * 1e-6;
    return IPA_OK;
}

namespace ipa {
namespace {

// The library's own FP64 functions, one element per thread.
__global__ void math_eval_kernel(int fn, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    __shared__ MathTables mt;
    load_math_tables(&mt);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        double r;
        switch (fn) {
        case IPA_MATH_EXP: r = exp_int(v, &mt); break;
        case IPA_MATH_LOG: r = log_fast(v, &mt); break;
        case IPA_MATH_SIN: { double s, c; sincos_int_wide(v, &mt, &s, &c); r = s; break; }
        case IPA_MATH_COS: { double s, c; sincos_int_wide(v, &mt, &s, &c); r = c; break; }
        case IPA_MATH_ERFCX: r = erfcx_fast(v, &mt); break;
        default: r = rcp_newton(v); break;
        }
        y[i] = r;
    }
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_math_eval(int32_t fn, const double* x_dev, double* y_dev, int64_t n, void* stream) {
    using namespace ipa;
    if (fn < IPA_MATH_EXP || fn > IPA_MATH_RCP || n < 0 || (n > 0 && (!x_dev || !y_dev))) {
        set_error("ipa_math_eval: bad arguments");
        return IPA_ERR_ARG;
    }
    if (n == 0) return IPA_OK;
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 4096 ? blocks : 4096);
    math_eval_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(fn, x_dev, y_dev, n);
    return cuda_fail(cudaGetLastError(), "math eval kernel launch");
}
