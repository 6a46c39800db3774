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
