"""GPU toy generation: Philox streams bit-exact against the oracle.

* the oracle's Philox-4x32-10 block function equals cuRAND's device function
  curand_Philox4x32_10 for random (counter, key) pairs, all four counter words;
* ipa_toygen output equals the oracle's toys bit for bit (1D and 4D, small
  toys, ragged counts, empty toys);
* the 4096-toy batch of Poisson(2e4) sizes: sampled toys bit-exact, every toy
  fully written, per-toy background counts exact;
* parameter regimes where the generator's FP32 decision filter hands many
  candidates to the FP64 test (decay times below the resolution offset, where
  the erfc argument is large and positive; narrow and wide resolutions; large
  exponents) still give the oracle's toys bit for bit.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1706_01420_gb300 import synth

pytestmark = pytest.mark.gpu

TH1 = np.array([0.66, 0.045, 0.0, 0.1])
TH4 = np.array([0.66, 0.045, 0.0, 0.1, 0.52, 0.25, 3.2, 3.1, 0.04, 0.3])
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def env(oracle):
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import api
    return oracle, G, torch, api


def _gen(env, kind, th, seed, n_sig, n_bkg, pad=0, t_range=None):
    O, G, torch, api = env
    n_sig = np.asarray(n_sig, dtype=np.int64)
    n_bkg = np.asarray(n_bkg, dtype=np.int64)
    sizes = n_sig + n_bkg + pad
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    total = int(sizes.sum())
    if t_range is None:
        t_range = (0.3, 15.0) if kind == "1d" else (0.0, 15.0)
    m = api.model_1d(*t_range) if kind == "1d" else api.model_4d(*t_range)
    keys = ("t",) if kind == "1d" else ("t", "ck", "cl", "phi")
    out = {k: torch.full((max(total, 1),), -7.0, dtype=torch.float64, device="cuda") for k in keys}
    d = lambda a: torch.tensor(a, dtype=torch.int64, device="cuda")
    api.ipa_toygen(m, torch.tensor(th, device="cuda"), seed, d(n_sig), d(n_bkg), d(off), out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, off


def test_philox_block_matches_curand_device(env, tmp_path):
    O, G, torch, api = env
    so = tmp_path / "libcurandref.so"
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", "-o", str(so), os.path.join(HERE, "helpers", "curand_philox.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(str(so))
    rng = np.random.default_rng(123)
    n = 10000
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:10] = 0
    ctr[10:20] = 0xFFFFFFFF
    c_d = torch.tensor(ctr.view(np.int32), device="cuda")
    k_d = torch.tensor(key.view(np.int32), device="cuda")
    o_d = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    assert lib.philox_ref(ctypes.c_void_p(c_d.data_ptr()), ctypes.c_void_p(k_d.data_ptr()),
                          ctypes.c_void_p(o_d.data_ptr()), n) == 0
    ref = o_d.cpu().numpy().view(np.uint32).astype(np.uint64)
    c64, k64 = ctr.astype(np.uint64), key.astype(np.uint64)
    mine = np.stack(O.philox4x32_10(c64[:, 0], c64[:, 1], c64[:, 2], c64[:, 3], k64[:, 0], k64[:, 1]), axis=1)
    np.testing.assert_array_equal(mine, ref)


@pytest.mark.parametrize("kind", ["1d", "4d"])
def test_toys_bit_exact_small(env, kind):
    O = env[0]
    th = TH1 if kind == "1d" else TH4
    n_sig = [0, 1, 2, 1023, 1024, 1025, 3000, 17]
    n_bkg = [0, 0, 5, 100, 0, 1, 333, 2]
    got, off = _gen(env, kind, th, 99, n_sig, n_bkg, pad=3)
    m = O.Model(kind, 0.3 if kind == "1d" else 0.0, 15.0)
    for k in range(len(n_sig)):
        ref = O.toy_one(m, th, 99, k, n_sig[k], n_bkg[k])
        n = n_sig[k] + n_bkg[k]
        for col, v in ref.items():
            np.testing.assert_array_equal(got[col][off[k]:off[k] + n], v, err_msg=f"toy {k} {col}")
            # the padding after each toy is untouched
            assert np.all(got[col][off[k] + n:off[k] + n + 3] == -7.0)


def test_toys_off_truth_and_other_seed(env):
    O = env[0]
    th = TH4.copy()
    th[:4] = [1.1, 0.07, 0.02, 0.25]
    th[4:] = [0.3, 0.4, 1.0, -2.0, 0.3, 2.0]
    got, off = _gen(env, "4d", th, 2**63 + 12345, [4000, 500], [10, 0])
    m = O.Model("4d", 0.0, 15.0)
    for k, (s, b) in enumerate([(4000, 10), (500, 0)]):
        ref = O.toy_one(m, th, 2**63 + 12345, k, s, b)
        for col, v in ref.items():
            np.testing.assert_array_equal(got[col][off[k]:off[k] + s + b], v)


def test_config3_batch_sampled(env):
    """4096 toys, sizes Poisson(2e4) split by Binomial(f_b): every slot written,
    toys 0, 1, 2048 and 4095 bit-exact against the oracle."""
    O = env[0]
    n_sig, n_bkg = synth.toy_sizes(4096, 2e4, TH4[3], seed=0)
    got, off = _gen(env, "4d", TH4, 0, n_sig, n_bkg)
    for col in got.values():
        assert np.all(np.isfinite(col)) and not np.any(col == -7.0)
    m = O.Model("4d", 0.0, 15.0)
    for k in (0, 1, 2048, 4095):
        ref = O.toy_one(m, TH4, 0, k, int(n_sig[k]), int(n_bkg[k]))
        n = int(n_sig[k] + n_bkg[k])
        for col, v in ref.items():
            np.testing.assert_array_equal(got[col][off[k]:off[k] + n], v, err_msg=f"toy {k} {col}")


def test_non_physical_theta_terminates_with_nan(env):
    th = TH1.copy()
    th[1] = float("nan")
    got, off = _gen(env, "1d", th, 1, [50], [4])
    assert np.all(np.isnan(got["t"][:50]))
    assert np.all(np.isfinite(got["t"][50:54]))


@pytest.mark.parametrize("kind,t_range,th", [
    ("1d", (-1.0, 15.0), [2.0, 0.01, 0.05, 0.2]),            # tau < 0: erfc argument up to ~75
    ("1d", (0.0, 40.0), [0.3, 0.005, 0.0, 0.05]),            # narrow resolution, exponent up to 12
    ("1d", (-0.2, 3.0), [4.0, 0.3, 0.1, 0.0]),               # wide resolution, steep decay
    ("4d", (-0.5, 8.0), [1.5, 0.2, -0.1, 0.3, 0.45, 0.3, 2.5, -1.0, 0.2, 1.5]),
])
def test_toys_bit_exact_in_filter_edge_regimes(env, kind, t_range, th):
    O = env[0]
    th = np.asarray(th, dtype=np.float64)
    n_sig, n_bkg = [2500, 700], [3, 0]
    got, off = _gen(env, kind, th, 4242, n_sig, n_bkg, t_range=t_range)
    m = O.Model(kind, *t_range)
    for k in range(2):
        ref = O.toy_one(m, th, 4242, k, n_sig[k], n_bkg[k])
        n = n_sig[k] + n_bkg[k]
        for col, v in ref.items():
            np.testing.assert_array_equal(got[col][off[k]:off[k] + n], v, err_msg=f"toy {k} {col}")
