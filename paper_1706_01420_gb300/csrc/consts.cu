// Step a1 of the hot path: theta -> the Consts record read by every event
// tile (see consts.cuh for the formulas): one six-warp block per fit for a
// few fits, one thread per fit for many; the same for the tagged model's
// record (tagged.cuh) and the phi_s model's (phis_consts.cuh).  This file is compiled without FMA contraction, so
// both layouts of a record give the same bits.
#include "consts.cuh"
#include "phis_consts.cuh"
#include "tagged.cuh"

namespace ipa {

namespace {
// One block of six warps per fit (few fits: latency).
__global__ void __launch_bounds__(kConstsBlock) consts_block_kernel(ModelDev m, const double* __restrict__ theta,
                                                                    Consts* __restrict__ out) {
    __shared__ ConstsBlockScratch S;
    // the likelihood kernel that follows may start now (it waits for this
    // kernel's results before reading them)
    asm volatile("griddepcontrol.launch_dependents;");
    const int s = blockIdx.x;
    compute_consts_block(m, theta + (size_t)s * m.n_par, out + s, &S);
}

// One thread per fit (many fits: throughput).
__global__ void consts_thread_kernel(ModelDev m, const double* __restrict__ theta, int n_seg,
                                     Consts* __restrict__ out) {
    __shared__ MathTables mt;
    asm volatile("griddepcontrol.launch_dependents;");
    cdetail::load_consts_tables(&mt);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_seg) compute_consts_thread(m, theta + (size_t)s * m.n_par, &mt, out + s);
}
// The tagged model's record: one thread per segment.
__global__ void tag_consts_kernel(ModelDev m, const double* __restrict__ theta, int n_seg, Consts* __restrict__ out) {
    __shared__ MathTables mt;
    asm volatile("griddepcontrol.launch_dependents;");
    cdetail::load_consts_tables(&mt);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_seg) tag_consts_thread(m, theta + (size_t)s * m.n_par, &mt, reinterpret_cast<TagConsts*>(out + s));
}

// The tagged model's record: one block of eight warps per segment.
__global__ void __launch_bounds__(kTagConstsBlock) tag_consts_block_kernel(ModelDev m, const double* __restrict__ theta,
                                                                           Consts* __restrict__ out) {
    __shared__ TagBlockScratch S;
    asm volatile("griddepcontrol.launch_dependents;");
    tag_consts_block(m, theta + (size_t)blockIdx.x * m.n_par, reinterpret_cast<TagConsts*>(out + blockIdx.x), &S);
}
// The phi_s model's record: one thread per segment.
__global__ void phis_consts_kernel(ModelDev m, const double* __restrict__ theta, int n_seg, Consts* __restrict__ out) {
    __shared__ MathTables mt;
    asm volatile("griddepcontrol.launch_dependents;");
    cdetail::load_consts_tables(&mt);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_seg) phis_consts_thread(m, theta + (size_t)s * m.n_par, &mt, reinterpret_cast<PhisConsts*>(out + s));
}

// The phi_s model's record: one block of eight warps per segment.
__global__ void __launch_bounds__(kPhisConstsBlock) phis_consts_block_kernel(ModelDev m,
                                                                             const double* __restrict__ theta,
                                                                             Consts* __restrict__ out) {
    __shared__ PhisBlockScratch S;
    asm volatile("griddepcontrol.launch_dependents;");
    phis_consts_block(m, theta + (size_t)blockIdx.x * m.n_par, reinterpret_cast<PhisConsts*>(out + blockIdx.x), &S);
}
}  // namespace

ipa_status launch_phis_consts(const ModelDev& m, const double* theta, int n_seg, Consts* out, cudaStream_t st) {
    if (n_seg <= 0) return IPA_OK;
    if (n_seg < 64)
        phis_consts_block_kernel<<<n_seg, kPhisConstsBlock, 0, st>>>(m, theta, out);
    else
        phis_consts_kernel<<<(n_seg + 63) / 64, 64, 0, st>>>(m, theta, n_seg, out);
    return cuda_fail(cudaGetLastError(), "phi_s consts kernel launch");
}

ipa_status launch_tag_consts(const ModelDev& m, const double* theta, int n_seg, Consts* out, cudaStream_t st) {
    if (n_seg <= 0) return IPA_OK;
    if (n_seg < 64)
        tag_consts_block_kernel<<<n_seg, kTagConstsBlock, 0, st>>>(m, theta, out);
    else
        tag_consts_kernel<<<(n_seg + 63) / 64, 64, 0, st>>>(m, theta, n_seg, out);
    return cuda_fail(cudaGetLastError(), "tagged consts kernel launch");
}

ipa_status launch_consts(const ModelDev& m, const double* theta, int n_seg, Consts* out,
                         cudaStream_t st) {
    if (n_seg <= 0) return IPA_OK;
    if (m.kind == IPA_MODEL_TAGGED1D) return launch_tag_consts(m, theta, n_seg, out, st);
    if (m.kind == IPA_MODEL_PHIS) return launch_phis_consts(m, theta, n_seg, out, st);
    if (n_seg >= 64) {
        consts_thread_kernel<<<(n_seg + 63) / 64, 64, 0, st>>>(m, theta, n_seg, out);
        return cuda_fail(cudaGetLastError(), "consts kernel launch");
    }
    consts_block_kernel<<<n_seg, kConstsBlock, 0, st>>>(m, theta, out);
    return cuda_fail(cudaGetLastError(), "consts kernel launch");
}

}  // namespace ipa
