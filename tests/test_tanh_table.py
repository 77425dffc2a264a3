"""The FP64 tanh table of the double-precision kernels, checked on the CPU.

The device routine evaluates tanh(k/16 + d) = sum_n a_n d^n (|d| <= 1/32)
from the coefficient table in csrc/tanh_table.inc.  Here the polynomial
with the stored coefficients is evaluated exactly (rational arithmetic) at
random doubles and compared with tanh in 50-digit arithmetic (mpmath): the
only errors left are the Taylor truncation and the rounding of the
coefficients (at most 0.77 ulp), so the polynomial's value, rounded once,
is within 1.3 ulp of tanh everywhere.  (The C library's tanh is itself up
to about 2 ulp off, so it only serves as a looser second check.)  A
dropped term, a wrong sign in the derivative recurrence or a shifted
interval centre fails by many ulps.
"""
import math
import os
import random
import re
from fractions import Fraction

import numpy as np

INC = os.path.join(os.path.dirname(__file__), "..", "paper_2005_00223_gb300", "csrc", "tanh_table.inc")


def _table():
    text = open(INC).read()
    deg = int(re.search(r"kTanhDeg = (\d+)", text).group(1))
    nk = int(re.search(r"kTanhK = (\d+)", text).group(1))
    body = text[text.index("{") + 1:text.rindex("}")]
    vals = [float.fromhex(v.strip()) for v in body.split(",") if v.strip()]
    assert len(vals) == (deg + 1) * nk
    return deg, nk, np.array(vals).reshape(deg + 1, nk)


def _ulp_dist(a, b):
    ia = np.array([a]).view(np.int64)[0]
    ib = np.array([b]).view(np.int64)[0]
    return abs(int(ia) - int(ib))


def test_table_shape_and_closed_forms():
    deg, nk, t = _table()
    assert deg == 10 and nk == 257
    # k = 0: the odd Taylor series of tanh at 0: x - x^3/3 + 2x^5/15 - 17x^7/315 + 62x^9/2835
    np.testing.assert_allclose(t[:, 0], [0, 1, 0, -1 / 3, 0, 2 / 15, 0, -17 / 315, 0, 62 / 2835, 0],
                               rtol=1e-15, atol=1e-300)
    for k in (1, 16, 100, 256):
        c = k / 16
        th = math.tanh(c)
        assert t[0, k] == th
        w = 1.0 / math.cosh(c) ** 2              # 1 - tanh^2 without cancellation
        assert abs(t[1, k] - w) <= 1e-15 * w
        assert abs(t[2, k] + th * w) <= 1e-15 * th * w
        assert abs(t[3, k] - w * (3 * th * th - 1) / 3) <= 1e-14 * w


def test_polynomial_within_one_ulp_of_tanh():
    deg, nk, t = _table()
    rng = random.Random(7)
    xs = [rng.uniform(0, 16) for _ in range(3000)] + [rng.uniform(0, 0.5) for _ in range(1000)]
    xs += [k / 16 + s / 32 for k in range(0, 256, 5) for s in (-1, 1) if k / 16 + s / 32 >= 0]
    xs += [1e-300, 1e-20, 1e-8, 0.03124, 15.96]
    try:
        import mpmath as mp
        mp.mp.dps = 50
    except ImportError:
        mp = None
    worst_true, worst_libm = 0.0, 0
    for x in xs:
        k = int(round(x * 16))
        d = x - k / 16                        # exact in double
        assert abs(d) <= 1 / 32 + 1e-18
        fd = Fraction(d)
        y = Fraction(0)
        for n in range(deg, -1, -1):
            y = y * fd + Fraction(t[n, k])
        yf = float(y)
        worst_libm = max(worst_libm, _ulp_dist(yf, math.tanh(x)))
        if mp is not None:
            ex = mp.tanh(mp.mpf(x))
            worst_true = max(worst_true, float(abs(mp.mpf(yf) - ex)) / math.ulp(float(ex)))
    assert worst_libm <= 3, worst_libm
    assert worst_true <= 1.3, worst_true
