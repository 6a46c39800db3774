"""ipa_nll_grad_noalloc: the NLL + gradient call that allocates no device memory.

Some callers cannot allocate when they call into the library: a host
framework whose allocator has already reserved the GPU, or a latency-critical
loop that must not pay for an allocation.  For them the library keeps the
scratch of this one call in a fixed array compiled into it.  These tests call
it through the C ABI and check its output against ipa_nll_grad, the entry point
that uses allocated scratch, within the tolerances of the other parity tests,
on two calls in a row (of different sizes, so stale contents of the shared
array would show).  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


def _check_close(O, G, m_o, cols, th, got, ref):
    logl, _ = O.nll_grad_terms(m_o, cols, th)
    labs = math.fsum(np.abs(logl))
    scale = G.grad_scale(O, m_o, cols, th)
    G.assert_nll_grad_close(got, float(ref[0]), np.asarray(ref[1:]), scale, labs)


def test_noalloc_matches_allocating_call_twice(env):
    O, G, torch, api = env
    m = api.model_4d(0.0, 15.0)
    m_o = O.Model("4d", 0.0, 15.0)
    th = torch.tensor(TH4, device="cuda")
    out = torch.empty(11, dtype=torch.float64, device="cuda")
    for n, seed, weighted in ((300_000, 31, True), (4097, 32, False)):
        cols = synth.events_4d(n, seed, weighted=weighted)
        ev = G.to_dev(cols)
        got = api.ipa_nll_grad_noalloc(m, ev, th, out).cpu().numpy().copy()
        ref = api.ipa_nll_grad(m, ev, th).cpu().numpy()
        _check_close(O, G, m_o, cols, TH4, got, ref)


def test_noalloc_rejects_oversized_input(env):
    O, G, torch, api = env
    from paper_1706_01420_gb300 import _capi as C
    n = C.IPA_NOALLOC_MAX_EVENTS + 1
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    with pytest.raises(api.IpaError, match="exceed the fixed scratch"):
        api.ipa_nll_grad_noalloc(api.model_1d(), {"t": t}, torch.tensor(TH4[:4], device="cuda"), out)
    # the limit itself is accepted (1D model, one column)
    lib = C.load()
    m = api.model_1d(0.3, 15.0)
    e = api.ipa_events({"t": t[:-1]})
    th1 = torch.tensor([0.66, 0.045, 0.0, 0.1], device="cuda")
    assert lib.ipa_nll_grad_noalloc(ctypes.byref(m), ctypes.byref(e), th1.data_ptr(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream) == C.IPA_OK
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))
