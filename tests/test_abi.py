"""CPU-side checks of the C ABI: the library builds, loads and exports every
function declared in include/ipanema.h, and rejects bad arguments on the host
without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1706_01420_gb300 import _capi, build
    build.build()
    return _capi.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ipanema.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ipa_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("ipa_nll", "ipa_nll_grad", "ipa_nll_grad_segmented", "ipa_toygen", "ipa_fit_batch"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1706_01420_gb300 import _capi
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _capi.PROTOTYPES, f"{name} missing from the Python binding"


def test_model_init_and_host_argument_checks(lib):
    from paper_1706_01420_gb300 import _capi as C
    m = C.ipa_model()
    assert lib.ipa_model_init(ctypes.byref(m), C.IPA_MODEL_ANGTIME4D, 0.0, 15.0) == C.IPA_OK
    assert (m.kind, m.n_par, m.t_lo, m.t_hi) == (2, 10, 0.0, 15.0)
    assert lib.ipa_model_init(ctypes.byref(m), 7, 0.0, 15.0) == C.IPA_ERR_ARG
    assert lib.ipa_model_init(ctypes.byref(m), 1, 2.0, 1.0) == C.IPA_ERR_ARG
    assert b"range" in lib.ipa_last_error()
    lib.ipa_model_init(ctypes.byref(m), C.IPA_MODEL_ANGTIME4D, 0.0, 15.0)
    ev = C.ipa_events()
    ev.n = 10
    ev.t = 16                      # never dereferenced: rejected on the host
    assert lib.ipa_nll(ctypes.byref(m), ctypes.byref(ev), 16, 16, None) == C.IPA_ERR_ARG   # ck NULL
    ev.ck, ev.cl, ev.phi = 32, 48, 8                                                      # phi misaligned
    assert lib.ipa_nll(ctypes.byref(m), ctypes.byref(ev), 16, 16, None) == C.IPA_ERR_ARG
    assert b"aligned" in lib.ipa_last_error()
    ev.n = -1
    assert lib.ipa_nll_grad(ctypes.byref(m), ctypes.byref(ev), 16, 16, None) == C.IPA_ERR_ARG
    assert lib.ipa_nll(None, ctypes.byref(ev), 16, 16, None) == C.IPA_ERR_ARG
    bad = C.ipa_model(kind=2, n_par=4, t_lo=0.0, t_hi=1.0)
    assert lib.ipa_nll(ctypes.byref(bad), ctypes.byref(ev), 16, 16, None) == C.IPA_ERR_ARG
    assert lib.ipa_reserve(-1, 1) == C.IPA_ERR_ARG
    assert lib.ipa_scratch_bytes(None) == C.IPA_ERR_ARG
    assert lib.ipa_version().startswith(b"ipanema")


def test_joint_map_host_checks(lib):
    """ipa_nll_grad_joint and ipa_fit_joint reject a bad category map on the host."""
    import numpy as np
    from paper_1706_01420_gb300 import _capi as C
    m = C.ipa_model()
    lib.ipa_model_init(ctypes.byref(m), C.IPA_MODEL_TIME1D, 0.0, 15.0)
    ev = C.ipa_events()
    ev.n = 10
    ev.t = 16                      # never dereferenced: rejected on the host

    def call(jmap, value=None, n_joint=None, n_fits=1):
        jm = np.ascontiguousarray(np.asarray(jmap, dtype=np.int32))
        j = C.ipa_joint()
        j.n_cat = jm.shape[0]
        j.n_joint = int(jm.max()) + 1 if n_joint is None else n_joint
        j.map = jm.ctypes.data
        v = None if value is None else np.ascontiguousarray(np.asarray(value, dtype=np.float64))
        j.value = None if v is None else v.ctypes.data
        return lib.ipa_nll_grad_joint(ctypes.byref(m), ctypes.byref(ev), 16, n_fits, ctypes.byref(j), 16, 16,
                                      None)

    assert call([[0, 1, 2, 4]]) == C.IPA_ERR_ARG                       # joint parameter 3 unused
    assert b"used by no category" in lib.ipa_last_error()
    assert call([[0, 1, 2, -2]]) == C.IPA_ERR_ARG                      # below -1
    assert call([[0, 1, 2, 3]], n_joint=3) == C.IPA_ERR_ARG            # above n_joint
    assert call([[0, 1, -1, 2]]) == C.IPA_ERR_ARG                      # a constant without values
    assert b"no values" in lib.ipa_last_error()
    assert call([[0] * 4], n_joint=33) == C.IPA_ERR_ARG                # more than IPA_MAX_PAR
    assert call([[0, 1, 2, 3]], n_fits=0) == C.IPA_ERR_ARG
    spec = (C.ipa_param * 4)()
    jm = np.array([[0, 1, 2, 3], [0, 1, 2, 5]], dtype=np.int32)
    j = C.ipa_joint(n_cat=2, n_joint=6, map=jm.ctypes.data, value=None)
    assert lib.ipa_fit_joint(ctypes.byref(m), ctypes.byref(ev), 16, 1, ctypes.byref(j), spec, 16, None, None,
                             None, None, None, 10, 1e-9, None) == C.IPA_ERR_ARG   # joint parameter 4 unused
    assert lib.ipa_hesse_joint(ctypes.byref(m), ctypes.byref(ev), 16, 1, ctypes.byref(j), spec, 16, 16, None,
                               None, None, None) == C.IPA_ERR_ARG
    flags = (ctypes.c_int32 * 6)(1, 0, 0, 0, 0, 0)
    assert lib.ipa_minos_joint(ctypes.byref(m), ctypes.byref(ev), 16, 1, ctypes.byref(j), spec, 16, 16, 16, flags,
                               0.5, 1e-7, 10, 100, 1e-9, 16, 16, None, None) == C.IPA_ERR_ARG
    assert b"used by no category" in lib.ipa_last_error()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1706_01420_gb300 import _capi
    saved = _capi._lib
    _capi._lib = None
    try:
        with pytest.raises(ImportError, match="no CPU fallback"):
            _capi.load(str(tmp_path / "missing.so"))
    finally:
        _capi._lib = saved


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1706_01420_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "ipa_oracle" not in text, f


def test_launch_config_table_host_logic(lib):
    """Setting and reading back a launch geometry is host-only bookkeeping:
    the value set for a size class is returned for every size of that class,
    classes are kept apart, and out-of-range geometries are refused."""
    from paper_1706_01420_gb300 import _capi as C
    m = C.ipa_model()
    lib.ipa_model_init(ctypes.byref(m), C.IPA_MODEL_ANGTIME4D, 0.0, 15.0)
    default = C.ipa_launch_config()
    assert lib.ipa_launch_config_get(ctypes.byref(m), 123_456_789, 1, 1, 0, ctypes.byref(default)) == C.IPA_OK
    assert (default.warps_per_block, default.warps_per_sm, default.tiles_per_take) == (1, 0, 1)
    cfg = C.ipa_launch_config(4, 12, 2, 0.0)
    # 3e6 events = 5860 tiles: class [4096, 8192) tiles
    assert lib.ipa_launch_config_set(ctypes.byref(m), 3_000_000, 1, 1, 0, ctypes.byref(cfg)) == C.IPA_OK
    for n in (4096 * 512, 3_000_000, 8191 * 512):
        got = C.ipa_launch_config()
        assert lib.ipa_launch_config_get(ctypes.byref(m), n, 1, 1, 0, ctypes.byref(got)) == C.IPA_OK
        assert (got.warps_per_block, got.warps_per_sm, got.tiles_per_take) == (4, 12, 2), n
    for other in ((8192 * 512, 1, 1, 0), (3_000_000, 1, 0, 0), (3_000_000, 1, 1, 1), (3_000_000, 64, 1, 0)):
        got = C.ipa_launch_config()
        lib.ipa_launch_config_get(ctypes.byref(m), other[0], other[1], other[2], other[3], ctypes.byref(got))
        assert (got.warps_per_block, got.warps_per_sm, got.tiles_per_take) == (1, 0, 1), other
    for bad in ((3, 0, 1), (0, 0, 1), (16, 0, 1), (1, -1, 1), (1, 65, 1), (1, 0, 3), (1, 0, 0)):
        c = C.ipa_launch_config(*bad, 0.0)
        assert lib.ipa_launch_config_set(ctypes.byref(m), 1000, 1, 1, 0, ctypes.byref(c)) == C.IPA_ERR_ARG
    assert lib.ipa_launch_config_get(ctypes.byref(m), -1, 1, 1, 0, ctypes.byref(cfg)) == C.IPA_ERR_ARG
    assert lib.ipa_launch_config_get(ctypes.byref(m), 10, 0, 1, 0, ctypes.byref(cfg)) == C.IPA_ERR_ARG
    lib.ipa_launch_config_set(ctypes.byref(m), 3_000_000, 1, 1, 0, ctypes.byref(default))   # leave the default


def test_fault_mask_set_and_read_back(lib):
    """ipa_fault_inject returns the previous mask and keeps only the known bits;
    IPA_FAULT in the environment sets the mask when the library loads (checked in
    a fresh process).  No GPU is needed: nothing is injected on a device."""
    import subprocess
    import sys
    from paper_1706_01420_gb300 import _capi as C
    old = lib.ipa_fault_inject(C.IPA_FAULT_SUBMIT | 64)
    assert lib.ipa_fault_inject(0) == C.IPA_FAULT_SUBMIT
    lib.ipa_fault_inject(old)
    code = ("import sys; sys.path.insert(0, %r); from paper_1706_01420_gb300 import _capi as C; "
            "print(C.load().ipa_fault_inject(0))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120,
                       env=dict(os.environ, IPA_FAULT="admit,alloc"))
    assert r.returncode == 0, r.stderr
    assert int(r.stdout.strip()) == C.IPA_FAULT_ALLOC | C.IPA_FAULT_ADMIT
