// Simultaneous fits over categories (Sec. 4, Example 2: one -2 log L summed
// over twelve categories that share most parameters, with per-bin S-wave
// parameters and a per-bin constant C_SP; App. B: Cat and ParamBox).
//
// A category is an event segment with its own parameter vector theta_c, built
// from the fit's joint parameters by a fixed map (joint index or constant).
// One pass: scatter theta_J -> theta_c for every segment, the per-segment
// constants and NLL+gradient (the kernels of ipa_nll_grad_segmented), then the
// gather: NLL_J = sum_c NLL_c and dNLL_J/dtheta_J[j] = sum over (c, p) mapped
// to j of dNLL_c/dtheta_c[p], in a fixed order (c ascending, then p).
#include <string.h>

#include <mutex>
#include <vector>

#include "fitcore.cuh"
#include "ipa_internal.cuh"

namespace ipa {
namespace {

__global__ void joint_scatter_kernel(JointDev j, int n_fits, const double* __restrict__ theta_joint,
                                     const int* __restrict__ active) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_seg = (int64_t)n_fits * j.n_cat;
    if (idx >= n_seg * j.n_model) return;
    const int64_t s = idx / j.n_model;
    const int p = (int)(idx - s * j.n_model);
    const int64_t i = s / j.n_cat;
    const int c = (int)(s - i * j.n_cat);
    const int a = active ? active[i] : 1;
    if (p == 0) j.seg_active[s] = a;
    if (!a) return;
    const int q = j.map[c * j.n_model + p];
    j.theta_seg[s * j.n_model + p] = q >= 0 ? theta_joint[i * j.n_joint + q] : j.value[c * j.n_model + p];
}

// One thread per (fit, output): output 0 is the NLL, sum over c of NLL_c;
// output 1 + q the sum over (c, p) with map[c][p] = q of dNLL_c/dtheta_c[p],
// both in the order c ascending, then p ascending.  Without the gradient, one
// thread per fit.
__global__ void joint_gather_kernel(JointDev j, int n_fits, const int* __restrict__ active,
                                    double* __restrict__ res_joint) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n_out = j.grad ? 1 + j.n_joint : 1;
    if (idx >= (int64_t)n_fits * n_out) return;
    const int64_t i = idx / n_out;
    const int o = (int)(idx - i * n_out);
    if (active && !active[i]) return;
    const int stride = j.grad ? 1 + j.n_model : 1;
    const double* r = j.res_seg + i * j.n_cat * stride;
    double v = 0.0;
    if (o == 0) {
        for (int c = 0; c < j.n_cat; ++c) v += r[c * stride];
    } else {
        const int q = o - 1;
        for (int c = 0; c < j.n_cat; ++c)
            for (int p = 0; p < j.n_model; ++p)
                if (j.map[c * j.n_model + p] == q) v += r[c * stride + 1 + p];
    }
    res_joint[i * n_out + o] = v;
}

// fit i: the event range of its categories (decides IPA_FIT_EMPTY)
__global__ void joint_fit_range_kernel(const int64_t* __restrict__ seg_off, int n_fits, int n_cat,
                                       int64_t* __restrict__ fit_begin, int64_t* __restrict__ fit_end) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fits) return;
    fit_begin[i] = seg_off[(int64_t)i * n_cat];
    fit_end[i] = seg_off[(int64_t)(i + 1) * n_cat];
}

// Per-device joint buffers (grow-only; the mutex spans a call).  One set for
// ipa_nll_grad_joint and one for ipa_fit_joint.
struct JointArgs {
    std::mutex mu;
    int32_t* map = nullptr;
    double* value = nullptr;
    size_t map_cap = 0;             // entries of map and value
    int64_t* seg_off = nullptr;     // n_seg + 1 (fits: a copy of the caller's offsets)
    int64_t* fit_begin = nullptr;   // n_fits each
    int64_t* fit_end = nullptr;
    double* theta_seg = nullptr;    // n_seg x n_model
    double* res_seg = nullptr;      // n_seg x (1 + n_model)
    int* seg_active = nullptr;      // n_seg
    Spec* spec = nullptr;
    size_t seg_cap = 0, fit_cap = 0;
};

JointArgs* joint_args(int which) {
    static JointArgs args[2][64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    return &args[which][dev];
}

template <typename T>
ipa_status grow(T** p, size_t have, size_t need, const char* what) {
    if (need <= have && *p) return IPA_OK;
    if (*p) {
        cudaDeviceSynchronize();
        cudaFree(*p);
        *p = nullptr;
    }
    return device_alloc(reinterpret_cast<void**>(p), sizeof(T) * (need ? need : 1), what);
}

size_t round_up(size_t need, size_t cap) {
    size_t c = cap ? cap : 64;
    while (c < need) c *= 2;
    return c;
}

ipa_status reserve(JointArgs& a, size_t map_n, size_t n_seg, size_t n_fits) {
    ipa_status st = IPA_OK;
    if (map_n > a.map_cap || !a.map) {
        const size_t cap = round_up(map_n, a.map_cap);
        if ((st = grow(&a.map, 0, cap, "joint map")) != IPA_OK) return st;
        if ((st = grow(&a.value, 0, cap, "joint values")) != IPA_OK) return st;
        a.map_cap = cap;
    }
    if (n_seg > a.seg_cap || !a.seg_off) {
        const size_t cap = round_up(n_seg, a.seg_cap);
        if ((st = grow(&a.seg_off, 0, cap + 1, "joint offsets")) != IPA_OK) return st;
        if ((st = grow(&a.theta_seg, 0, cap * kMaxP, "joint category parameters")) != IPA_OK) return st;
        if ((st = grow(&a.res_seg, 0, cap * (1 + kMaxP), "joint category results")) != IPA_OK) return st;
        if ((st = grow(&a.seg_active, 0, cap, "joint category mask")) != IPA_OK) return st;
        a.seg_cap = cap;
    }
    if (n_fits > a.fit_cap || !a.fit_begin) {
        const size_t cap = round_up(n_fits, a.fit_cap);
        if ((st = grow(&a.fit_begin, 0, cap, "joint fit ranges")) != IPA_OK) return st;
        if ((st = grow(&a.fit_end, 0, cap, "joint fit ranges")) != IPA_OK) return st;
        a.fit_cap = cap;
    }
    if (!a.spec) st = device_alloc((void**)&a.spec, sizeof(Spec), "joint fit spec");
    return st;
}

// Host checks of the map; IPA_ERR_ARG with the reason.
ipa_status check_joint_map(const ipa_model* m, const ipa_joint* j, int n_fits) {
    if (!j || j->n_cat < 1 || j->n_joint < 1 || j->n_joint > kMaxP || !j->map) {
        set_error("joint: need n_cat >= 1, 1 <= n_joint <= %d and a map", kMaxP);
        return IPA_ERR_ARG;
    }
    if (n_fits < 1 || (int64_t)n_fits * j->n_cat > (int64_t)1 << 30) {
        set_error("joint: bad number of fits %d", n_fits);
        return IPA_ERR_ARG;
    }
    std::vector<int> used(j->n_joint, 0);
    const int64_t n_map = (int64_t)j->n_cat * m->n_par;
    for (int64_t k = 0; k < n_map; ++k) {
        const int q = j->map[k];
        if (q < -1 || q >= j->n_joint) {
            set_error("joint: map entry %lld (category %lld, parameter %lld) is %d, outside [-1, %d)", (long long)k,
                      (long long)(k / m->n_par), (long long)(k % m->n_par), q, j->n_joint);
            return IPA_ERR_ARG;
        }
        if (q == -1 && !j->value) {
            set_error("joint: map entry %lld is a constant but no values were given", (long long)k);
            return IPA_ERR_ARG;
        }
        if (q >= 0) used[q] = 1;
    }
    for (int q = 0; q < j->n_joint; ++q)
        if (!used[q]) {
            set_error("joint: joint parameter %d is used by no category", q);
            return IPA_ERR_ARG;
        }
    return IPA_OK;
}

// Copy the map and values into the library buffers, ordered on stream s.
ipa_status upload(JointArgs& a, const ipa_model* m, const ipa_joint* j, cudaStream_t s) {
    const size_t n = (size_t)j->n_cat * m->n_par;
    ipa_status st = cuda_fail(cudaMemcpyAsync(a.map, j->map, n * sizeof(int32_t), cudaMemcpyHostToDevice, s),
                              "joint map copy");
    if (st != IPA_OK) return st;
    if (j->value) {
        st = cuda_fail(cudaMemcpyAsync(a.value, j->value, n * sizeof(double), cudaMemcpyHostToDevice, s),
                       "joint values copy");
    } else {
        st = cuda_fail(cudaMemsetAsync(a.value, 0, n * sizeof(double), s), "joint values reset");
    }
    return st;
}

JointDev joint_dev(JointArgs& a, const ipa_model* m, const ipa_joint* j, const int64_t* seg_off) {
    JointDev d;
    d.n_cat = j->n_cat;
    d.n_model = m->n_par;
    d.n_joint = j->n_joint;
    d.map = a.map;
    d.value = a.value;
    d.seg_begin = seg_off;
    d.seg_end = seg_off + 1;
    d.theta_seg = a.theta_seg;
    d.res_seg = a.res_seg;
    d.seg_active = a.seg_active;
    return d;
}

}  // namespace

ipa_status check_joint(const ipa_model* m, const ipa_joint* j, int n_fits) { return check_joint_map(m, j, n_fits); }

ipa_status launch_joint_scatter(const JointDev& j, int n_fits, const double* theta_joint, const int* active,
                                cudaStream_t s) {
    const int64_t n = (int64_t)n_fits * j.n_cat * j.n_model;
    const int b = 256;
    joint_scatter_kernel<<<(unsigned)((n + b - 1) / b), b, 0, s>>>(j, n_fits, theta_joint, active);
    return cuda_fail(cudaGetLastError(), "joint scatter");
}

ipa_status launch_joint_gather(const JointDev& j, int n_fits, const int* active, double* res_joint,
                               cudaStream_t s) {
    const int b = 128;
    const int64_t n = (int64_t)n_fits * (j.grad ? 1 + j.n_joint : 1);
    joint_gather_kernel<<<(unsigned)((n + b - 1) / b), b, 0, s>>>(j, n_fits, active, res_joint);
    return cuda_fail(cudaGetLastError(), "joint gather");
}

}  // namespace ipa

extern "C" ipa_status ipa_nll_grad_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                                         int32_t n_fits, const ipa_joint* joint, const double* theta_dev,
                                         double* out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if ((st = check_joint(model, joint, n_fits)) != IPA_OK) return st;
    if (!seg_off_dev || !theta_dev || !out_dev) {
        set_error("ipa_nll_grad_joint: NULL device pointer");
        return IPA_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    JointArgs* ap = joint_args(0);
    if (!ap) return IPA_ERR_CUDA;
    JointArgs& a = *ap;
    std::lock_guard<std::mutex> lk(a.mu);
    const int n_seg = n_fits * joint->n_cat;
    if ((st = reserve(a, (size_t)joint->n_cat * model->n_par, n_seg, n_fits)) != IPA_OK) return st;
    if ((st = upload(a, model, joint, s)) != IPA_OK) return st;
    Scratch* sc = nullptr;
    if ((st = scratch_get((ev->n + kTile - 1) / kTile + n_seg, n_seg + 1, &sc)) != IPA_OK) return st;
    const JointDev jd = joint_dev(a, model, joint, seg_off_dev);
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride, ev->q};
    if ((st = launch_joint_scatter(jd, n_fits, theta_dev, nullptr, s)) != IPA_OK) return st;
    if ((st = launch_seg_tiles(jd.seg_begin, jd.seg_end, nullptr, n_seg, ev->n, sc->seg_tiles, s)) != IPA_OK)
        return st;
    if ((st = launch_consts(m, jd.theta_seg, n_seg, sc->consts, s)) != IPA_OK) return st;
    if ((st = launch_nll(m, true, cols, ev->n, jd.seg_begin, jd.seg_end, sc->seg_tiles, n_seg, sc->consts, sc,
                         jd.res_seg, s)) != IPA_OK)
        return st;
    return launch_joint_gather(jd, n_fits, nullptr, out_dev, s);
}

extern "C" ipa_status ipa_fit_joint(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off_dev,
                                    int32_t n_fits, const ipa_joint* joint, const ipa_param* spec,
                                    double* theta_io_dev, double* err_out_dev, double* nll_out_dev,
                                    int32_t* fit_status_dev, int32_t* iters_out_dev, int32_t* passes_out_dev,
                                    int32_t max_iter, double tol, void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if ((st = check_joint(model, joint, n_fits)) != IPA_OK) return st;
    if (!seg_off_dev || !spec || !theta_io_dev || max_iter < 1 || !(tol > 0.0)) {
        set_error("ipa_fit_joint: bad arguments");
        return IPA_ERR_ARG;
    }
    Spec sp{};
    if ((st = build_spec(model, spec, max_iter, tol, &sp, joint->n_joint)) != IPA_OK) return st;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    JointArgs* ap = joint_args(1);
    if (!ap) return IPA_ERR_CUDA;
    JointArgs& a = *ap;
    std::lock_guard<std::mutex> lk(a.mu);
    const int n_seg = n_fits * joint->n_cat;
    if ((st = reserve(a, (size_t)joint->n_cat * model->n_par, n_seg, n_fits)) != IPA_OK) return st;
    if ((st = upload(a, model, joint, user)) != IPA_OK) return st;
    // the specification and the offsets in library buffers (stable addresses
    // let consecutive calls reuse the captured graph)
    if ((st = cuda_fail(cudaMemcpyAsync(a.spec, &sp, sizeof(Spec), cudaMemcpyHostToDevice, user),
                        "joint spec copy")) != IPA_OK)
        return st;
    if ((st = cuda_fail(cudaMemcpyAsync(a.seg_off, seg_off_dev, sizeof(int64_t) * ((size_t)n_seg + 1),
                                        cudaMemcpyDeviceToDevice, user), "joint offsets copy")) != IPA_OK)
        return st;
    joint_fit_range_kernel<<<(n_fits + 127) / 128, 128, 0, user>>>(a.seg_off, n_fits, joint->n_cat, a.fit_begin,
                                                                   a.fit_end);
    if ((st = cuda_fail(cudaGetLastError(), "joint fit ranges")) != IPA_OK) return st;
    const JointDev jd = joint_dev(a, model, joint, a.seg_off);
    return fit_run(model, ev, n_fits, a.fit_begin, a.fit_end, a.spec, 0, sp.max_passes,
                   (ev->n + kTile - 1) / kTile + n_seg, theta_io_dev, err_out_dev, nll_out_dev, fit_status_dev,
                   iters_out_dev, passes_out_dev, user, "ipa_fit_joint", &jd);
}
