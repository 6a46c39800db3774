"""Fit server (continuous batching): every fit's result, taken from the mix,
is bitwise the result of ipa_fit_batch on that fit alone; fits wait for HBM
when the arena is full and all complete; bad requests are refused."""
import time

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
LO4 = [0.3, 0.01, -0.1, 0.0, 0.2, 0.05, 0.0, 0.0, 0.0, -3.2]
HI4 = [1.5, 0.2, 0.1, 0.5, 0.8, 0.5, 6.3, 6.3, 0.5, 3.2]
STEP4 = [0.01, 0.003, 0.002, 0.005, 0.005, 0.006, 0.1, 0.1, 0.01, 0.2]


@pytest.fixture(scope="module")
def env():
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return G, torch, api


def _pool(torch, api, n_toys=40, per=25000, seed=3):
    m = api.model_4d(0.0, 15.0)
    d64 = lambda a: torch.tensor(a, dtype=torch.int64, device="cuda")
    n_bkg = np.full(n_toys, per // 10, dtype=np.int64)
    n_sig = np.full(n_toys, per, dtype=np.int64) - n_bkg
    off = np.arange(n_toys, dtype=np.int64) * per
    cols = {k: torch.empty(n_toys * per, dtype=torch.float64, device="cuda") for k in ("t", "ck", "cl", "phi")}
    api.ipa_toygen(m, torch.tensor(TH4, device="cuda"), seed, d64(n_sig), d64(n_bkg), d64(off), cols)
    torch.cuda.synchronize()
    host = {k: v.cpu().numpy() for k, v in cols.items()}
    host["w"] = synth.weights(n_toys * per, seed)
    return host


def _params(api, start):
    return [api.Param(float(start[i]), LO4[i], HI4[i], STEP4[i]) for i in range(10)]


def _solo(G, torch, api, m, ev, params, start):
    dev = {k: torch.tensor(v, device="cuda") for k, v in ev.items()}
    n = len(ev["t"])
    off = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    r = api.ipa_fit_batch(m, dev, off, params, torch.tensor(start[None, :], device="cuda"), max_iter=200, tol=1e-8)
    torch.cuda.synchronize()
    return {"theta": r["theta"][0].cpu().numpy(), "err": r["err"][0].cpu().numpy(),
            "nll": float(r["nll"][0]), "status": int(r["status"][0])}


def _wait(api, srv, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = api.ipa_serve_poll(srv, t, 10)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "server did not finish in time"
        time.sleep(0.002)
    return out


def test_results_in_the_mix_equal_solo_fits(env):
    G, torch, api = env
    pool = _pool(torch, api)
    m = api.model_4d(0.0, 15.0)
    rng = np.random.default_rng(1)
    sizes = [0, 1000, 20000, 3000, 150000, 50000, 700, 90000, 12000, 250000]
    # arena for ~300k events: admission has to wait for memory part of the time
    srv = api.ipa_server_create(m, 300_000 * 40, max_slots=4)
    try:
        reqs, tickets = [], []
        for i, n in enumerate(sizes):
            a = int(rng.integers(0, len(pool["t"]) - n))
            ev = {k: np.ascontiguousarray(v[a:a + n]) for k, v in pool.items()}
            if i % 3 == 1:
                ev.pop("w")
            start = TH4 * (1 + 0.01 * rng.normal(size=10))
            start[2] = 0.001
            reqs.append((ev, start))
            tickets.append(api.ipa_serve_submit(srv, ev, _params(api, start)))
            if i % 4 == 0:
                time.sleep(0.01)           # arrivals spread while others run
        got = _wait(api, srv, tickets)
    finally:
        api.ipa_server_destroy(srv)
    for (ev, start), t in zip(reqs, tickets):
        solo = _solo(G, torch, api, m, ev, _params(api, start), start)
        r = got[t]
        assert r["status"] == solo["status"]
        assert np.array_equal(r["theta"], solo["theta"])
        assert np.array_equal(r["err"], solo["err"])
        assert r["nll"] == solo["nll"]
    assert got[tickets[0]]["status"] == 4                        # the empty fit


def test_refuses_bad_requests(env):
    G, torch, api = env
    m = api.model_4d(0.0, 15.0)
    srv = api.ipa_server_create(m, 10_000 * 40, max_slots=2)
    try:
        big = {k: np.zeros(20_000) for k in ("t", "ck", "cl", "phi")}
        with pytest.raises(api.IpaError, match="HBM budget"):
            api.ipa_serve_submit(srv, big, _params(api, TH4))
        with pytest.raises(api.IpaError, match="unknown ticket"):
            api.ipa_serve_poll(srv, 12345, 10)
        bad = _params(api, TH4)
        bad[0].value = 5.0                                            # outside its limits
        with pytest.raises(api.IpaError, match="outside its limits"):
            api.ipa_serve_submit(srv, {k: np.zeros(10) for k in ("t", "ck", "cl", "phi")}, bad)
    finally:
        api.ipa_server_destroy(srv)


def test_device_inputs_and_destroy_with_pending_fits(env):
    G, torch, api = env
    pool = _pool(torch, api, n_toys=8, per=20000, seed=4)
    m = api.model_4d(0.0, 15.0)
    srv = api.ipa_server_create(m, 200_000 * 40, max_slots=2)
    try:
        dev = {k: torch.tensor(v[:30000], device="cuda") for k, v in pool.items()}
        t = api.ipa_serve_submit(srv, dev, _params(api, TH4))
        del dev
        torch.cuda.empty_cache()
        r = _wait(api, srv, [t])[t]
        assert r["status"] in (0, 2)
        for _ in range(3):          # left running: destroy must stop cleanly
            api.ipa_serve_submit(srv, {k: np.ascontiguousarray(v[:100000]) for k, v in pool.items()},
                                 _params(api, TH4))
    finally:
        api.ipa_server_destroy(srv)
