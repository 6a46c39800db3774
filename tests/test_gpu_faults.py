"""Failure handling with host-side fault injection (ipa_fault_inject): no
fault, trap or hang is ever made on the device.

* a failed device allocation (IPA_FAULT_ALLOC) returns IPA_ERR_OOM and leaves
  the library usable: the same call succeeds once the fault is cleared, with
  the result of a process that never saw the fault;
* a submit whose staging fails (IPA_FAULT_SUBMIT) is refused with IPA_ERR_OOM
  and the caller's events are untouched: submitting them again gives the fit
  of a server that never failed;
* while the server cannot admit (IPA_FAULT_ADMIT), queued fits keep their
  place and stay pending; once the fault is cleared they are admitted in order
  and give the same fits.
"""
import json
import os
import subprocess
import sys
import time

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
LO4 = np.array([0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2])
HI4 = np.array([1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2])
STEP4 = np.array([0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2])


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    yield oracle, G, torch, api
    api.ipa_fault_inject(0)


FRESH = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1706_01420_gb300 import api, synth
from paper_1706_01420_gb300 import _capi as C
TH4 = np.array(json.loads(sys.argv[2]))
cols = synth.events_4d(30_000, 81)
ev = {k: torch.tensor(v, device="cuda") for k, v in cols.items()}
m = api.model_4d(0.0, 15.0)
th = torch.tensor(TH4, device="cuda")
res = {"mask_at_load": api.ipa_fault_inject(C.IPA_FAULT_ALLOC)}
try:
    api.ipa_nll_grad(m, ev, th)
    res["first"] = "ok"
except api.IpaError as e:
    res["first"] = str(e)
res["scratch_after_fault"] = api.ipa_scratch_bytes()
api.ipa_fault_inject(0)
res["second"] = api.ipa_nll_grad(m, ev, th).cpu().numpy().tolist()
print(json.dumps(res))
"""

CLEAN = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1706_01420_gb300 import api, synth
TH4 = np.array(json.loads(sys.argv[2]))
cols = synth.events_4d(30_000, 81)
ev = {k: torch.tensor(v, device="cuda") for k, v in cols.items()}
print(json.dumps(api.ipa_nll_grad(api.model_4d(0.0, 15.0), ev, torch.tensor(TH4, device="cuda")).cpu().numpy().tolist()))
"""


def test_alloc_fault_returns_oom_and_recovers(env):
    """In a fresh process started with IPA_FAULT=alloc: the first call cannot
    allocate its scratch and returns IPA_ERR_OOM; after clearing the mask the
    same call returns the bits of a process that never saw the fault."""
    O, G, torch, api = env
    env_v = dict(os.environ, IPA_FAULT="alloc")
    r = subprocess.run([sys.executable, "-c", FRESH, ROOT, json.dumps(TH4.tolist())], capture_output=True,
                       text=True, timeout=600, cwd=ROOT, env=env_v)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["mask_at_load"] == 1
    assert "IPA_ERR_OOM" in d["first"] and "injected" in d["first"]
    assert d["scratch_after_fault"] == 0
    env_c = {k: v for k, v in os.environ.items() if k != "IPA_FAULT"}
    c = subprocess.run([sys.executable, "-c", CLEAN, ROOT, json.dumps(TH4.tolist())], capture_output=True,
                       text=True, timeout=600, cwd=ROOT, env=env_c)
    assert c.returncode == 0, c.stderr[-3000:]
    assert d["second"] == json.loads(c.stdout.strip().splitlines()[-1])


def _params(api):
    return [api.Param(float(TH4[i]), float(LO4[i]), float(HI4[i]), float(STEP4[i])) for i in range(10)]


def _requests(O, n_req, seed):
    m_o = O.Model("4d", 0.0, 15.0)
    return [O.toy_one(m_o, TH4, seed, k, 4500 + 300 * k, 500) for k in range(n_req)]


def _reference_fits(torch, api, m, reqs, params):
    out = []
    for ev in reqs:
        d = {k: torch.tensor(v, device="cuda") for k, v in ev.items()}
        n = ev["t"].size
        r = api.ipa_fit_batch(m, d, torch.tensor([0, n], dtype=torch.int64, device="cuda"), params,
                              torch.tensor(TH4[None, :], device="cuda"), max_iter=200, tol=1e-8)
        out.append({"theta": r["theta"][0].cpu().numpy(), "nll": float(r["nll"][0]), "status": int(r["status"][0])})
    return out


def _wait(api, srv, tickets, timeout_s=120):
    res, t0 = {}, time.time()
    while len(res) < len(tickets):
        for i, tk in enumerate(tickets):
            if i not in res:
                r = api.ipa_serve_poll(srv, tk, 10)
                if r is not None:
                    res[i] = r
        assert time.time() - t0 < timeout_s, "server did not finish"
        time.sleep(0.002)
    return [res[i] for i in range(len(tickets))]


def test_submit_fault_refuses_and_resubmission_fits(env):
    O, G, torch, api = env
    from paper_1706_01420_gb300 import _capi as C
    m = api.model_4d(0.0, 15.0)
    params = _params(api)
    reqs = _requests(O, 3, 82)
    ref = _reference_fits(torch, api, m, reqs, params)
    srv = api.ipa_server_create(m, 1 << 30, max_slots=8, max_iter=200, tol=1e-8)
    try:
        api.ipa_fault_inject(C.IPA_FAULT_SUBMIT)
        with pytest.raises(api.IpaError, match="IPA_ERR_OOM"):
            api.ipa_serve_submit(srv, reqs[0], params)
        api.ipa_fault_inject(0)
        tickets = [api.ipa_serve_submit(srv, ev, params) for ev in reqs]
        got = _wait(api, srv, tickets)
    finally:
        api.ipa_fault_inject(0)
        api.ipa_server_destroy(srv)
    for g, r in zip(got, ref):
        assert g["status"] == r["status"] == 0
        assert np.array_equal(g["theta"], r["theta"]) and g["nll"] == r["nll"]


def test_admission_fault_keeps_requests_queued(env):
    O, G, torch, api = env
    from paper_1706_01420_gb300 import _capi as C
    m = api.model_4d(0.0, 15.0)
    params = _params(api)
    reqs = _requests(O, 4, 83)
    ref = _reference_fits(torch, api, m, reqs, params)
    srv = api.ipa_server_create(m, 1 << 30, max_slots=8, max_iter=200, tol=1e-8)
    try:
        api.ipa_fault_inject(C.IPA_FAULT_ADMIT)
        tickets = [api.ipa_serve_submit(srv, ev, params) for ev in reqs]
        time.sleep(0.5)
        assert all(api.ipa_serve_poll(srv, tk, 10) is None for tk in tickets)
        api.ipa_fault_inject(0)
        got = _wait(api, srv, tickets)
    finally:
        api.ipa_fault_inject(0)
        api.ipa_server_destroy(srv)
    for g, r in zip(got, ref):
        assert g["status"] == r["status"] == 0
        assert np.array_equal(g["theta"], r["theta"]) and g["nll"] == r["nll"]
