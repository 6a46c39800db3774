"""The autograd binding: backward equals the fused analytic gradient, matches
finite differences, and a torch optimiser driving it reaches the minimum that
ipa_fit_batch finds."""
import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH1 = np.array([0.66, 0.045, 0.0, 0.1])


@pytest.fixture(scope="module")
def env():
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api, autograd
    return G, torch, api, autograd


def test_backward_is_the_fused_gradient(env):
    G, torch, api, autograd = env
    cols = synth.events_4d(20000, 3, weighted=True)
    ev = G.to_dev(cols)
    m = api.model_4d()
    th = torch.tensor([0.66, 0.045, 0.002, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3], dtype=torch.float64,
                      device="cuda", requires_grad=True)
    f = autograd.nll(m, ev, th)
    (3.0 * f).backward()
    ref = api.ipa_nll_grad(m, ev, th.detach())
    assert float(f) == float(ref[0])
    assert torch.equal(th.grad, 3.0 * ref[1:])
    # against finite differences of the forward itself
    for j in (0, 4, 9):
        h = 1e-5 * max(abs(float(th[j])), 0.05)
        tp, tm = th.detach().clone(), th.detach().clone()
        tp[j] += h
        tm[j] -= h
        fd = (float(autograd.nll(m, ev, tp)) - float(autograd.nll(m, ev, tm))) / (2 * h)
        assert abs(fd - float(ref[1 + j])) <= 1e-6 * abs(float(ref[1 + j])) + 1e-4


def test_torch_optimiser_reaches_the_fit_minimum(env):
    G, torch, api, autograd = env
    t = synth.events_1d(50000, 4, t_lo=0.0)
    ev = G.to_dev({"t": t})
    m = api.model_1d(0.0, 15.0)
    # reference: the library's fitter (Gamma, sigma, f_b free; mu fixed)
    lo, hi = [0.3, 0.01, -0.1, 0.0], [1.5, 0.2, 0.1, 0.5]
    step = [0.01, 0.003, 0.002, 0.005]
    params = [api.Param(float(TH1[i]), lo[i], hi[i], step[i], fixed=(i == 2)) for i in range(4)]
    off = torch.tensor([0, t.size], dtype=torch.int64, device="cuda")
    r = api.ipa_fit_batch(m, ev, off, params, torch.tensor(TH1[None, :], device="cuda"), tol=1e-9)
    ref = r["theta"][0].cpu().numpy()
    err = r["err"][0].cpu().numpy()
    # torch L-BFGS on the free parameters, in units of their errors
    free = torch.tensor([0, 1, 3], device="cuda")
    scale = torch.tensor(err[[0, 1, 3]], device="cuda")
    x = torch.zeros(3, dtype=torch.float64, device="cuda", requires_grad=True)
    base = torch.tensor(TH1, device="cuda")

    def theta_of(x):
        th = base.clone()
        th[free] = base[free] + x * scale
        return th

    opt = torch.optim.LBFGS([x], lr=1.0, max_iter=200, tolerance_grad=1e-12, tolerance_change=1e-15,
                            line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        f = autograd.nll(m, ev, theta_of(x))
        f.backward()
        return f

    opt.step(closure)
    got = theta_of(x).detach().cpu().numpy()
    assert np.all(np.abs(got[[0, 1, 3]] - ref[[0, 1, 3]]) < 1e-4 * err[[0, 1, 3]])


def test_joint_backward_is_the_joint_gradient(env):
    """Two simultaneous fits of three 1D categories (Gamma shared, f_b per
    category): backward of a weighted sum of the fits' NLLs is each fit's joint
    gradient times its weight, and a torch optimiser on the joint NLL reaches
    ipa_fit_joint's minimum."""
    G, torch, api, autograd = env
    m = api.model_1d(0.3, 15.0)
    jmap = [[0, -1, -1, 1], [0, -1, -1, 2], [0, -1, -1, 3]]
    value = [[0.0, 0.045, 0.0, 0.0], [0.0, 0.05, 0.0, 0.0], [0.0, 0.04, 0.0, 0.0]]
    joint = api.Joint(jmap, value)
    cats = [synth.events_1d(3000 + 500 * c, 40 + c) for c in range(6)]
    ev = G.to_dev({"t": np.concatenate(cats)})
    off = torch.tensor(np.concatenate([[0], np.cumsum([c.size for c in cats])]), dtype=torch.int64, device="cuda")
    th = torch.tensor([[0.66, 0.1, 0.12, 0.08], [0.6, 0.09, 0.1, 0.11]], dtype=torch.float64, device="cuda",
                      requires_grad=True)
    f = autograd.nll_joint(m, ev, off, joint, th)
    (f * torch.tensor([2.0, -1.0], dtype=torch.float64, device="cuda")).sum().backward()
    ref = api.ipa_nll_grad_joint(m, ev, off, joint, th.detach())
    assert torch.equal(f.detach(), ref[:, 0])
    assert torch.equal(th.grad[0], 2.0 * ref[0, 1:]) and torch.equal(th.grad[1], -1.0 * ref[1, 1:])
    # an optimiser on fit 0 (in units of the errors, one L-BFGS call) reaches the
    # joint fit's minimum
    sub = off[:4].contiguous()
    start = torch.tensor([0.7, 0.12, 0.12, 0.12], dtype=torch.float64, device="cuda")
    params = [api.Param(v, 0.0, 2.0, 0.01) for v in (0.7, 0.12, 0.12, 0.12)]
    r = api.ipa_fit_joint(m, ev, sub, joint, params, start[None, :].clone(), max_iter=300, tol=1e-10)
    ref, err = r["theta"][0], r["err"][0]
    x = torch.zeros(4, dtype=torch.float64, device="cuda", requires_grad=True)
    opt = torch.optim.LBFGS([x], lr=1.0, max_iter=300, tolerance_grad=1e-12, tolerance_change=1e-15,
                            line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        v = autograd.nll_joint(m, ev, sub, joint, (start + x * err)[None, :]).sum()
        v.backward()
        return v

    opt.step(closure)
    got = (start + x.detach() * err)
    assert torch.all((got - ref).abs() < 1e-4 * err), (got, ref)
