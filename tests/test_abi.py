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
    assert lib.ipa_version().startswith(b"ipanema")


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
