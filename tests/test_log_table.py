"""The FP64 logarithm of the heatbath (log_u01 in su3_device.cuh), checked on
the CPU against the mathematics: its table (su3_log_table.cuh) holds log F_j
and 1/F_j, F_j = 1 + j/64, each the double nearest the exact value; and the
algorithm -- the same integer and floating-point steps as the device code,
with every fma rounded once -- is within two ulp of the result (2^-52
absolute near zero) of the exact logarithm of the uniforms the heatbath
draws, (x + 1/2) 2^-52.
"""
import os
import re
import struct
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "..", "paper_0904_1179_gb300", "csrc", "su3_log_table.cuh")


def load_table():
    text = open(TABLE).read()
    out = {}
    for name in ("kLogF", "kInvF"):
        body = re.search(name + r"\[65\] = \{(.*?)\};", text, re.S).group(1)
        vals = [float.fromhex(v) for v in re.findall(r"(-?0x[0-9a-fp.+-]+),", body)]
        assert len(vals) == 65
        out[name] = vals
    return out["kLogF"], out["kInvF"]


def nearest_double(x):
    """The double nearest the mpmath number x (ties impossible here)."""
    d = float(x)
    cands = [d, np.nextafter(d, -np.inf), np.nextafter(d, np.inf)]
    return min(cands, key=lambda c: abs(mpmath.mpf(c) - x))


def test_table_is_correctly_rounded():
    mpmath.mp.dps = 40
    log_f, inv_f = load_table()
    for j in range(65):
        F = mpmath.mpf(64 + j) / 64
        assert log_f[j] == nearest_double(mpmath.log(F)), j
        assert inv_f[j] == nearest_double(1 / F), j


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def d2ll(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def ll2d(x):
    return struct.unpack("<d", struct.pack("<q", x))[0]


def log_u01(u, log_f, inv_f):
    b = d2ll(u)
    e = (b >> 52) - 1023
    mb = b & 0x000FFFFFFFFFFFFF
    m = ll2d(mb | 0x3FF0000000000000)
    j = (mb + (1 << 45)) >> 46
    F = ll2d(0x3FF0000000000000 + (j << 46))
    r = (m - F) * inv_f[j]
    p = 1.0 / 7.0
    for c in (-1.0 / 6.0, 1.0 / 5.0, -1.0 / 4.0, 1.0 / 3.0, -0.5, 1.0):
        p = fma(p, r, c)
    ed = ll2d(0x4330000000000000 + (e + 1024)) - 4503599627371520.0
    assert ed == e
    return fma(ed, float.fromhex("0x1.62e42fefa39efp-1"), log_f[j]) + r * p


def test_log_u01_error_bound():
    mpmath.mp.dps = 40
    log_f, inv_f = load_table()
    rng = np.random.default_rng(3)
    xs = [int(v) for v in rng.integers(0, 1 << 52, size=4000, dtype=np.int64)]
    # the ends of the range, both sides of every power of two, the table's ends
    xs += [0, 1, (1 << 52) - 1, (1 << 51) - 1, 1 << 51, (1 << 50) - 1, 1 << 50, 1 << 46, (1 << 52) - (1 << 45)]
    xs += [(1 << k) - 1 for k in range(1, 52)] + [1 << k for k in range(52)]
    worst = 0.0
    for x in xs:
        u = (x + 0.5) * 2.0 ** -52
        exact = mpmath.log(mpmath.mpf(2 * x + 1) / mpmath.mpf(2) ** 53)
        err = float(abs(mpmath.mpf(log_u01(u, log_f, inv_f)) - exact))
        # two ulp of the result, and 2^-52 absolute where the result is near 0
        worst = max(worst, err / (2 * np.spacing(abs(float(exact))) + 2.0 ** -52))
    assert worst <= 1.0, worst
