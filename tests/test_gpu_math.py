"""Accuracy of the library's own FP64 elementary functions (the table-driven
exp, log, sincos and erfcx the likelihood kernel calls, and the Newton
reciprocal of its adjoint sums), evaluated on the GPU through ipa_math_eval,
against the CPU's libm (numpy) and scipy.special.erfcx.

Bounds are stated in units of the double spacing at the reference value
(ulp) or relative to it; the kernel's NLL tolerance (1e-12 relative) needs
about 1e-13 per event, the gradient's (1e-9) far less."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from tests import gpu_common as G
    G.need_gpu()
    import torch
    from paper_1706_01420_gb300 import _capi as C, api
    return torch, api, C


def _eval(env, fn, x):
    torch, api, C = env
    y = api.ipa_math_eval(fn, torch.tensor(x, device="cuda"))
    return y.cpu().numpy()


def _ulps(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_exp(env):
    C = env[2]
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-700, 700, 200000), rng.uniform(-1, 1, 100000),
                        [0.0, -0.0, 1e-300, -1e-300, 709.7, -707.0, -706.9]])
    got = _eval(env, C.IPA_MATH_EXP, x)
    ref = np.exp(x)
    assert _ulps(got, ref).max() <= 2.0
    # flush to zero below -707: exp(-707) ~ 9e-308, nothing in the kernel needs less
    assert _eval(env, C.IPA_MATH_EXP, np.array([-710.0, -1e5]))[0] == 0.0


def test_log(env):
    C = env[2]
    rng = np.random.default_rng(2)
    x = np.concatenate([np.exp(rng.uniform(-690, 690, 200000)), rng.uniform(1e-4, 65536.0, 100000),
                        1.0 + rng.uniform(-1e-3, 1e-3, 50000), [1.0, 2.0, 0.5]])
    got = _eval(env, C.IPA_MATH_LOG, x)
    ref = np.log(x)
    # near x = 1 the result is small: bound by ulps of the result or 2^-53 absolute
    err = np.abs(got - ref)
    assert np.all(err <= np.maximum(2.0 * np.spacing(np.abs(ref)), 2.0 ** -53)), err.max()
    assert got[-3] == 0.0
    special = _eval(env, C.IPA_MATH_LOG, np.array([0.0, -1.0, np.inf, np.nan, 5e-324]))
    assert special[0] == -np.inf and np.isnan(special[1]) and special[2] == np.inf and np.isnan(special[3])
    assert special[4] == np.log(5e-324)


@pytest.mark.parametrize("which", ["sin", "cos"])
def test_sincos(env, which):
    C = env[2]
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-np.pi, np.pi, 300000), rng.uniform(-1e4, 1e4, 50000),
                        [0.0, np.pi, -np.pi, np.pi / 2, 1e-300]])
    fn = C.IPA_MATH_SIN if which == "sin" else C.IPA_MATH_COS
    got = _eval(env, fn, x)
    ref = np.sin(x) if which == "sin" else np.cos(x)
    # absolute: the angular functions are bounded by 1 and enter as products
    assert np.abs(got - ref).max() <= 2.5e-16 * (1.0 + np.abs(x).max() * 2.0 ** -40)


def test_erfcx(env):
    C = env[2]
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(0.0, 6.25, 300000), rng.uniform(6.25, 1e3, 20000),
                        [0.0, 0.25, 6.25, 6.2500001]])
    got = _eval(env, C.IPA_MATH_ERFCX, x)
    ref = special.erfcx(x)
    # the piecewise fit reaches about 1e-15 relative (a few ulp)
    assert (np.abs(got - ref) / ref).max() <= 1.5e-15


def test_newton_reciprocal(env):
    C = env[2]
    rng = np.random.default_rng(5)
    x = np.concatenate([np.exp(rng.uniform(-85, 85, 200000)), -np.exp(rng.uniform(-85, 85, 20000)),
                        rng.uniform(1e-4, 20.0, 100000)])
    got = _eval(env, C.IPA_MATH_RCP, x)
    assert (np.abs(got * x - 1.0)).max() <= 1e-13
    edge = np.array([0.0, np.inf, 1e-300, 1e300, 2.0 ** -126, 2.0 ** 126])
    with np.errstate(divide="ignore"):
        ref = 1.0 / edge
    assert np.array_equal(_eval(env, C.IPA_MATH_RCP, edge), ref)
