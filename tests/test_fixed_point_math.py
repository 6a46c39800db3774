"""CPU checks of the integer-pipe exp and sin/cos (int_math.cuh): the generated
fixed-point tables and constants equal their exact values rounded once, and a
step-by-step integer emulation of the two algorithms (Python integers with the
64-bit wrap-around and 64x64->128-bit high products of the CUDA code) meets the
accuracy stated in int_math.cuh against 50-digit mpmath.  The GPU results of
the same functions are checked against libm in tests/test_gpu_math.py."""
import math
import os
import re
import struct

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50
TABLES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1706_01420_gb300",
                      "csrc", "fp64_tables.cuh")
M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def tab():
    src = open(TABLES).read()

    def const(name):
        return int(re.search(name + r" = (-?\d+)u?ll", src).group(1))

    def arr(name):
        body = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
        return [int(x.strip().rstrip("l").rstrip("u")) for x in body.split(",") if x.strip()]

    names = ["kTwoOverPiQ64", "kPiOver32Q64", "kSinC3Q64", "kSinC5Q64", "kSinC7Q64", "kSinC9Q64", "kCosC2Q64",
             "kCosC4Q64", "kCosC6Q64", "kCosC8Q64", "kInvLn2x64Q56", "kLn2d64Q128Hi", "kLn2d64Q128Lo",
             "kExpC2Q63", "kExpC3Q63", "kExpC4Q63", "kExpC5Q63", "kExpC6Q63", "k32OverPiQ59",
             "kPiOver32Q128Hi", "kPiOver32Q128Lo"]
    t = {n: const(n) for n in names}
    t["S"], t["C"], t["E"] = arr("kSinQ62"), arr("kCosQ62"), arr("kExp2Q62")
    return t


def _q(x, bits):
    return int(mp.nint(mp.mpf(x) * mp.power(2, bits)))


def test_tables_are_exact_values_rounded_once(tab):
    assert tab["kTwoOverPiQ64"] == _q(2 / mp.pi, 64) and tab["kPiOver32Q64"] == _q(mp.pi / 32, 64)
    assert tab["kInvLn2x64Q56"] == _q(64 / mp.log(2), 56)
    assert (tab["kLn2d64Q128Hi"] << 64) + tab["kLn2d64Q128Lo"] == _q(mp.log(2) / 64, 128)
    assert (tab["kPiOver32Q128Hi"] << 64) + tab["kPiOver32Q128Lo"] == _q(mp.pi / 32, 128)
    assert tab["k32OverPiQ59"] == _q(32 / mp.pi, 59)
    for n, k in ((3, "kSinC3Q64"), (5, "kSinC5Q64"), (7, "kSinC7Q64"), (9, "kSinC9Q64"), (2, "kCosC2Q64"),
                 (4, "kCosC4Q64"), (6, "kCosC6Q64"), (8, "kCosC8Q64")):
        assert tab[k] == _q(1 / mp.factorial(n), 64)
    for n in range(2, 7):
        assert tab[f"kExpC{n}Q63"] == _q(1 / mp.factorial(n), 63)
    assert tab["S"] == [_q(mp.sin(j * mp.pi / 32), 62) for j in range(65)]
    assert tab["C"] == [_q(mp.cos(j * mp.pi / 32), 62) for j in range(65)]
    assert tab["E"] == [_q(mp.power(2, mp.mpf(j) / 64), 62) for j in range(64)]


def _s64(x):
    x &= M64
    return x - (1 << 64) if x >> 63 else x


def _umulhi(a, b):
    return ((a & M64) * (b & M64)) >> 64


def _mulhi(a, b):
    return (_s64(a) * _s64(b)) >> 64


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _q62_to_double(v, e2):
    if v == 0:
        return 0.0
    sign = 1 << 63 if v < 0 else 0
    a = -v if v < 0 else v
    lz = 64 - a.bit_length()
    a = (a << lz) & M64
    m, rem = a >> 11, a & 0x7FF
    m += 1 if (rem > 0x400 or (rem == 0x400 and (m & 1))) else 0
    return struct.unpack("<d", struct.pack("<Q", (sign | (((1 - lz + e2 + 1022) << 52) + m)) & M64))[0]


def _sincos(t, phi):
    b = _bits(phi)
    E = ((b >> 52) & 0x7FF) - 1023
    M = (b & 0xFFFFFFFFFFFFF) | (1 << 52)
    sh = E + 9
    X = (M << sh) & M64 if sh >= 0 else (M >> -sh if sh > -64 else 0)
    U = _umulhi(X, t["kTwoOverPiQ64"])
    k = (U + (1 << 56)) >> 57
    rq = _s64(U - (k << 57))
    ra = -rq if rq < 0 else rq
    r = _umulhi((ra << 7) & M64, t["kPiOver32Q64"])
    z = _umulhi(r, r)
    p = t["kSinC9Q64"]
    for c in ("kSinC7Q64", "kSinC5Q64", "kSinC3Q64"):
        p = (t[c] - _umulhi(z, p)) & M64
    sr = _s64(r - _umulhi(r, _umulhi(z, p)))
    q = t["kCosC8Q64"]
    for c in ("kCosC6Q64", "kCosC4Q64", "kCosC2Q64"):
        q = (t[c] - _umulhi(z, q)) & M64
    cm = _s64(_umulhi(z, q))
    srs = -sr if rq < 0 else sr
    Sk, Ck = t["S"][k], t["C"][k]
    sd = _q62_to_double(_s64(Sk - _mulhi(Sk, cm) + _mulhi(Ck, srs)), 0)
    return (-sd if b >> 63 else sd), _q62_to_double(_s64(Ck - _mulhi(Ck, cm) - _mulhi(Sk, srs)), 0)


def _sincos_wide(t, phi):
    """sincos_int_wide: |phi| < 1024 in Q53, k = round(|phi| 32/pi), r in Q64 with
    pi/32 to 128 bits, then the same polynomials and table (entry k mod 64)."""
    b = _bits(phi)
    E = ((b >> 52) & 0x7FF) - 1023
    M = (b & 0xFFFFFFFFFFFFF) | (1 << 52)
    sh = E + 1
    A = (M << sh) & M64 if sh >= 0 else (M >> -sh if sh > -64 else 0)
    k = (_umulhi(A, t["k32OverPiQ59"]) + (1 << 47)) >> 48
    kl = k * t["kPiOver32Q128Hi"] + ((k * t["kPiOver32Q128Lo"]) >> 64)
    r = _s64((A << 11) - kl)
    ra = -r if r < 0 else r
    z = _umulhi(ra, ra)
    p = t["kSinC9Q64"]
    for c in ("kSinC7Q64", "kSinC5Q64", "kSinC3Q64"):
        p = (t[c] - _umulhi(z, p)) & M64
    sr = _s64(ra - _umulhi(ra, _umulhi(z, p)))
    q = t["kCosC8Q64"]
    for c in ("kCosC6Q64", "kCosC4Q64", "kCosC2Q64"):
        q = (t[c] - _umulhi(z, q)) & M64
    cm = _s64(_umulhi(z, q))
    srs = -sr if r < 0 else sr
    Sk, Ck = t["S"][k & 63], t["C"][k & 63]
    sd = _q62_to_double(_s64(Sk - _mulhi(Sk, cm) + _mulhi(Ck, srs)), 0)
    return (-sd if b >> 63 else sd), _q62_to_double(_s64(Ck - _mulhi(Ck, cm) - _mulhi(Sk, srs)), 0)


def test_wide_sincos_emulation_accuracy(tab):
    """Phases up to 1024 (Dm t of the tagged model reaches a few hundred)."""
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-1023.9, 1023.9, 3000), rng.uniform(-4, 4, 500),
                         [0.0, 1e-300, 0.5, 1023.99, -1023.99, 100 * np.pi, 201.0625, 266.55]])
    worst = 0.0
    with mp.workdps(60):
        for x in xs:
            s, c = _sincos_wide(tab, float(x))
            worst = max(worst, abs(float(mp.mpf(s) - mp.sin(mp.mpf(float(x))))),
                        abs(float(mp.mpf(c) - mp.cos(mp.mpf(float(x))))))
    assert worst <= 6e-17, worst


def _exp(t, a):
    b = _bits(a)
    E = ((b >> 52) & 0x7FF) - 1023
    neg = b >> 63
    M = (b & 0xFFFFFFFFFFFFF) | (1 << 52)
    sh = E + 1
    A = (M << sh) & M64 if sh >= 0 else (M >> -sh if sh > -64 else 0)
    k = (_umulhi(A, t["kInvLn2x64Q56"]) + (1 << 44)) >> 45
    kl = k * t["kLn2d64Q128Hi"] + ((k * t["kLn2d64Q128Lo"]) >> 64)
    r = _s64((A << 11) - kl)
    rs, ks = (-r, -k) if neg else (r, k)
    v = t["kExpC6Q63"]
    for c in ("kExpC5Q63", "kExpC4Q63", "kExpC3Q63", "kExpC2Q63"):
        v = _s64(t[c] + _mulhi(rs, v))
    pm = _s64(rs + _s64(_mulhi(_mulhi(rs, v), rs) << 1))
    T = t["E"][ks & 63]
    return _q62_to_double(_s64(T + _mulhi(T, pm)), ks >> 6)


def test_sincos_emulation_accuracy(tab):
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-np.pi, np.pi, 4000), rng.uniform(-3.999, 3.999, 1000),
                         [0.0, -0.0, 1e-300, np.pi, -np.pi, np.pi / 2, 3.999, 1e-10, -1e-17]])
    worst = 0.0
    for x in xs:
        s, c = _sincos(tab, float(x))
        worst = max(worst, abs(float(mp.mpf(s) - mp.sin(mp.mpf(float(x))))),
                    abs(float(mp.mpf(c) - mp.cos(mp.mpf(float(x))))))
    # a few 2^-62 before the final rounding, half an ulp of 1 after it
    assert worst <= 6e-17, worst


def test_exp_emulation_accuracy(tab):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(-704.9, 708.9, 4000), rng.uniform(-1, 1, 1000), rng.uniform(-1e-3, 1e-3, 500),
                         [0.0, -0.0, 1e-300, -704.99, 708.99, 0.5, -0.5, 1.0]])
    worst = 0.0
    for x in xs:
        ref = mp.exp(mp.mpf(float(x)))
        worst = max(worst, abs(float((mp.mpf(_exp(tab, float(x))) - ref) / math.ulp(float(ref)))))
    assert worst <= 1.5, worst


def _to_q62(x):
    b = _bits(x)
    sh = ((b >> 52) & 0x7FF) - 1023 + 10
    M = (b & 0xFFFFFFFFFFFFF) | (1 << 52)
    v = (M << sh) & M64 if sh >= 0 else (M >> -sh if sh > -64 else 0)
    return -v if b >> 63 else v


def _mq(a, b):
    return _s64(_mulhi(a, b) << 2)


def _sqrt_q124(X):
    """sqrt_q124 with the FP32 seed taken as the float32-rounded 1/sqrt (the GPU's
    rsqrtf differs in the last bits; the two Newton steps remove the difference)."""
    if X <= 0:
        return 0
    lead = X.bit_length() - 1
    s = (124 - lead) & ~1
    Xn = X << s
    top = lead + s
    xf = np.float32((Xn >> (top - 23)) / 2.0 ** 23 * 2.0 ** (top - 124))
    y0 = float(np.float32(1.0) / np.sqrt(xf))
    ye = math.floor(math.log2(y0))
    Y0 = int(round(y0 * 2 ** 23 / 2 ** ye)) << (39 + ye)
    Q = _mq(Xn >> 62, Y0)
    for _ in range(2):
        R = Xn - Q * Q
        Q += _s64(_mulhi(R >> 62, Y0) << 1)
    return Q >> (s >> 1)


def _one_minus_sq(x):
    return ((1 << 124) - x * x) >> 62


def _basis_q62(t, ck, cl, phi):
    b = _bits(phi)
    sp, cp = _sincos_q62(t, b)
    if b >> 63:
        sp = -sp
    CK, CL = _to_q62(ck), _to_q62(cl)
    one = 1 << 62
    sk2, sl2 = _one_minus_sq(CK), _one_minus_sq(CL)
    ck2, cl2 = one - sk2, one - sl2
    cp2 = _mq(cp, cp)
    q = _sqrt_q124(sk2 * sl2)
    sksl2 = (sk2 * sl2) >> 62
    slcp2 = _mq(sl2, cp2)
    a = _mq(q, _mq(CK, CL))
    bq = _mq(q, CL)
    return [_mq(ck2, sl2), _mq(sk2, one - slcp2), _mq(sk2, slcp2 + cl2), _mq(sksl2, _mq(sp, cp)), _mq(a, cp),
            _mq(a, sp), sl2, _mq(bq, cp), _mq(bq, sp), _mq(CK, sl2)]


def _sincos_q62(t, b):
    E = ((b >> 52) & 0x7FF) - 1023
    M = (b & 0xFFFFFFFFFFFFF) | (1 << 52)
    sh = E + 9
    X = (M << sh) & M64 if sh >= 0 else (M >> -sh if sh > -64 else 0)
    U = _umulhi(X, t["kTwoOverPiQ64"])
    k = (U + (1 << 56)) >> 57
    rq = _s64(U - (k << 57))
    ra = -rq if rq < 0 else rq
    r = _umulhi((ra << 7) & M64, t["kPiOver32Q64"])
    z = _umulhi(r, r)
    p = t["kSinC9Q64"]
    for c in ("kSinC7Q64", "kSinC5Q64", "kSinC3Q64"):
        p = (t[c] - _umulhi(z, p)) & M64
    sr = _s64(r - _umulhi(r, _umulhi(z, p)))
    q = t["kCosC8Q64"]
    for c in ("kCosC6Q64", "kCosC4Q64", "kCosC2Q64"):
        q = (t[c] - _umulhi(z, q)) & M64
    cm = _s64(_umulhi(z, q))
    srs = -sr if rq < 0 else sr
    Sk, Ck = t["S"][k], t["C"][k]
    return _s64(Sk - _mulhi(Sk, cm) + _mulhi(Ck, srs)), _s64(Ck - _mulhi(Ck, cm) - _mulhi(Sk, srs))


def test_sqrt_emulation_accuracy():
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.uniform(0, 1, 3000), np.exp(rng.uniform(-40, 0, 1000)), [1.0, 0.25, 0.5, 1e-18]])
    for x in xs:
        X = _to_q62(float(x)) << 62
        got = mp.mpf(_sqrt_q124(X)) / mp.power(2, 62)
        ref = mp.sqrt(mp.mpf(X) / mp.power(2, 124))
        assert abs(float(got - ref)) <= 2.0 ** -61 + 2.0 ** -59 * float(ref), x


def test_angular_basis_emulation_accuracy(tab):
    """The fixed-point f'_k against the 50-digit formulas for angles basis_q62_ok
    accepts: absolute error a few 2^-60 (the angular functions are bounded by 1),
    and relative error below 1e-13 for every product not smaller than 1e-4."""
    rng = np.random.default_rng(3)
    n = 2000
    lim = 1.0 - 2.0 ** -17       # basis_q62_ok: the FP64 basis takes |cos| beyond this
    cks = np.concatenate([rng.uniform(-1, 1, n), [0.0, lim * 0.999999, -lim * 0.999999, 0.3]])
    cls = np.concatenate([rng.uniform(-1, 1, n), [0.5, -lim * 0.999999, lim * 0.999999, 0.0]])
    phs = np.concatenate([rng.uniform(-np.pi, np.pi, n), [0.0, np.pi, -np.pi, 3.99]])
    worst = 0.0
    for ck, cl, ph in zip(cks, cls, phs):
        if not (abs(ck) < lim and abs(cl) < lim):
            continue
        F = [mp.mpf(v) / mp.power(2, 62) for v in _basis_q62(tab, float(ck), float(cl), float(ph))]
        c, l, p = mp.mpf(float(ck)), mp.mpf(float(cl)), mp.mpf(float(ph))
        sk2, sl2, cp, sp = 1 - c * c, 1 - l * l, mp.cos(p), mp.sin(p)
        q = mp.sqrt(sk2 * sl2)
        ref = [c * c * sl2, sk2 * (1 - sl2 * cp * cp), sk2 * (sl2 * cp * cp + l * l), sk2 * sl2 * sp * cp,
               q * c * l * cp, q * c * l * sp, sl2, q * l * cp, q * l * sp, c * sl2]
        worst = max(worst, max(abs(float(a - b)) for a, b in zip(F, ref)))
        for a, b in zip(F, ref):
            if abs(b) >= 1e-4:
                assert abs(float((a - b) / b)) <= 1e-13
    assert worst <= 2.0 ** -56, worst


def test_amplitude_sum_emulation(tab):
    """A = sum_k (h_k c_k) f'_k from Q62 coefficients and products, accumulated
    in Q60 from the 64-bit high products and read back with exponent +2, as the
    likelihood kernel does: within a few 2^-60 of the 50-digit sum before the
    final rounding to double (half an ulp)."""
    rng = np.random.default_rng(4)
    c = [1.0, 0.5, 0.5, 1.0, math.sqrt(2), -math.sqrt(2), 1.0 / 3, 2 / math.sqrt(6), -2 / math.sqrt(6),
         2 / math.sqrt(3)]
    for _ in range(300):
        h = rng.uniform(-1, 1, 10)
        hc = [float(h[k] * c[k]) for k in range(10)]
        ck, cl, ph = rng.uniform(-0.99, 0.99), rng.uniform(-0.99, 0.99), rng.uniform(-np.pi, np.pi)
        F = _basis_q62(tab, ck, cl, ph)
        Af = sum(_mulhi(_to_q62(hc[k]), F[k]) for k in range(10))
        got = _q62_to_double(_s64(Af), 2)
        ref = mp.fsum(mp.mpf(hc[k]) * mp.mpf(F[k]) / mp.power(2, 62) for k in range(10))
        assert abs(float(mp.mpf(got) - ref)) <= 2.0 ** -57 + 2.0 ** -53 * abs(float(ref))
