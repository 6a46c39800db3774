"""ipa_nll_grad_noalloc: the NLL + gradient call that allocates no device memory.

Some callers cannot allocate when they call into the library: a host
framework whose allocator has already reserved the GPU, or a latency-critical
loop that must not pay for an allocation and the device synchronisation that
growing a buffer implies.  For them the library keeps the scratch of this one
call in a fixed array compiled into it.  These tests call it through the C ABI
and check, on two calls in a row of different sizes (so stale contents of the
shared array would show):

* its output against the CPU oracle, within the tolerances of the other parity
  tests, for the 4D model (weighted and not), the tagged model and the 1D
  model, and bitwise against ipa_nll_grad (the same kernels with allocated
  scratch);
* an empty event set, the largest accepted size and the refusals (too many
  events, the phi_s model whose tiles need more scratch than the array holds);
* in a fresh process, that the call run first allocates no library scratch at
  all (ipa_scratch_bytes stays 0) and still matches the oracle.

This file is collected last on purpose.
"""
import ctypes
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
TH1 = np.array([0.66, 0.045, 0.0, 0.1])
THT = np.array([0.66, 0.045, 0.0, 0.1, 0.085, 17.77, 0.8, 0.3])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


def _noalloc_and_plain(torch, api, m, cols, th):
    from tests import gpu_common as G
    ev = G.to_dev(cols)
    theta = torch.tensor(th, device="cuda")
    out = torch.empty(1 + m.n_par, dtype=torch.float64, device="cuda")
    got = api.ipa_nll_grad_noalloc(m, ev, theta, out).cpu().numpy().copy()
    ref = api.ipa_nll_grad(m, ev, theta).cpu().numpy()
    return got, ref


def test_noalloc_4d_matches_oracle_twice(env):
    O, G, torch, api = env
    m, m_o = api.model_4d(0.0, 15.0), O.Model("4d", 0.0, 15.0)
    for n, seed, weighted in ((300_000, 31, True), (4097, 32, False)):
        cols = synth.events_4d(n, seed, weighted=weighted)
        got, plain = _noalloc_and_plain(torch, api, m, cols, TH4)
        f_ref, g_ref = O.nll_grad(m_o, cols, TH4)
        logl, _ = O.nll_grad_terms(m_o, cols, TH4)
        G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale(O, m_o, cols, TH4), math.fsum(np.abs(logl)))
        assert np.array_equal(got, plain), (n, got - plain)


def test_noalloc_tagged_and_1d_match_oracle(env):
    O, G, torch, api = env
    from oracle import tagged as T
    m_t, mo_t = api.model_tagged(0.0, 15.0), O.Model("tag", 0.0, 15.0)
    for n, seed, weighted in ((20_000, 41, True), (1537, 42, False)):
        cols = synth.events_tagged(n, seed, weighted=weighted)
        got, plain = _noalloc_and_plain(torch, api, m_t, cols, THT)
        f_ref, g_ref = T.nll_grad(mo_t, cols, THT)
        logl, _ = T.nll_grad_terms(mo_t, cols, THT)
        G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale_tagged(O, T, mo_t, cols, THT),
                                math.fsum(np.abs(logl)))
        assert np.array_equal(got, plain)
    m_1, mo_1 = api.model_1d(0.3, 15.0), O.Model("1d", 0.3, 15.0)
    cols = {"t": synth.events_1d(100_000, 43)}
    got, plain = _noalloc_and_plain(torch, api, m_1, cols, TH1)
    f_ref, g_ref = O.nll_grad(mo_1, cols, TH1)
    logl, _ = O.nll_grad_terms(mo_1, cols, TH1)
    G.assert_nll_grad_close(got, f_ref, g_ref, G.grad_scale(O, mo_1, cols, TH1), math.fsum(np.abs(logl)))
    assert np.array_equal(got, plain)


def test_noalloc_empty_input_gives_zeros(env):
    O, G, torch, api = env
    m = api.model_4d(0.0, 15.0)
    empty = {k: torch.empty(0, dtype=torch.float64, device="cuda") for k in ("t", "ck", "cl", "phi")}
    out = torch.full((11,), 7.0, dtype=torch.float64, device="cuda")
    got = api.ipa_nll_grad_noalloc(m, empty, torch.tensor(TH4, device="cuda"), out).cpu().numpy()
    assert np.array_equal(got, np.zeros(11))


def test_noalloc_rejects_oversized_input_and_the_phis_model(env):
    O, G, torch, api = env
    from paper_1706_01420_gb300 import _capi as C
    n = C.IPA_NOALLOC_MAX_EVENTS + 1
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    with pytest.raises(api.IpaError, match="exceed the fixed scratch"):
        api.ipa_nll_grad_noalloc(api.model_1d(), {"t": t}, torch.tensor(TH1, device="cuda"), out)
    # the limit itself is accepted (1D model, one column)
    lib = C.load()
    m = api.model_1d(0.3, 15.0)
    e = api.ipa_events({"t": t[:-1]})
    th1 = torch.tensor(TH1, device="cuda")
    assert lib.ipa_nll_grad_noalloc(ctypes.byref(m), ctypes.byref(e), th1.data_ptr(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream) == C.IPA_OK
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))
    # the phi_s model keeps 47 sums per tile; the array holds 15
    cols = synth.events_phis(1000, 44)
    ev = G.to_dev(cols)
    out17 = torch.empty(17, dtype=torch.float64, device="cuda")
    with pytest.raises(api.IpaError, match="needs more scratch"):
        api.ipa_nll_grad_noalloc(api.model_phis(0.0, 15.0), ev, torch.zeros(16, dtype=torch.float64, device="cuda"),
                                 out17)


FRESH = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1706_01420_gb300 import api, synth
from oracle import ipa_oracle as O
TH4 = np.array(json.loads(sys.argv[2]))
cols = synth.events_4d(20_000, 51, weighted=True)
ev = {k: torch.tensor(v, device="cuda") for k, v in cols.items()}
m = api.model_4d(0.0, 15.0)
th = torch.tensor(TH4, device="cuda")
out = torch.empty(11, dtype=torch.float64, device="cuda")
first = api.ipa_nll_grad_noalloc(m, ev, th, out).cpu().numpy().tolist()
second = api.ipa_nll_grad_noalloc(m, ev, th, out).cpu().numpy().tolist()
scratch_after_noalloc = api.ipa_scratch_bytes()
plain = api.ipa_nll_grad(m, ev, th).cpu().numpy().tolist()
f_ref, g_ref = O.nll_grad(O.Model("4d", 0.0, 15.0), cols, TH4)
print(json.dumps({"first": first, "second": second, "plain": plain, "scratch_after_noalloc": scratch_after_noalloc,
                  "scratch_after_plain": api.ipa_scratch_bytes(), "f_ref": f_ref, "g_ref": list(g_ref)}))
"""


def test_noalloc_first_call_in_a_fresh_process_allocates_no_scratch(env):
    """A new process whose first library call is ipa_nll_grad_noalloc: the
    library's allocating scratch stays at 0 bytes through two calls, the
    results match the oracle and equal ipa_nll_grad's, which then does
    allocate scratch (so the query sees allocations)."""
    O, G, torch, api = env
    r = subprocess.run([sys.executable, "-c", FRESH, ROOT, json.dumps(TH4.tolist())], capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["scratch_after_noalloc"] == 0
    assert d["scratch_after_plain"] > 0
    assert d["first"] == d["second"] == d["plain"]
    got = np.array(d["first"])
    assert abs(got[0] - d["f_ref"]) <= 1e-12 * abs(d["f_ref"])
    g_ref = np.array(d["g_ref"])
    assert np.all(np.abs(got[1:] - g_ref) <= 1e-8 * (np.abs(g_ref) + np.abs(g_ref).max()))
