"""Writes tanh_table.inc: Taylor coefficients of tanh for the FP64 kernels.

tanh on [0, 16) is split into intervals of width h = 1/16 centred at
c_k = k h (k = 0..256); on each, tanh(c_k + d) = sum_{n=0}^{10} a_n(c_k) d^n
for |d| <= h/2.  The coefficients follow from the derivatives of tanh:
with t = tanh(c) and w = 1 - t^2, tanh^(n)(c) = w Q_n(t) for n >= 1, where
Q_1 = 1 and Q_{n+1}(t) = -2 t Q_n(t) + (1 - t^2) Q_n'(t) (differentiate
w Q_n with w' = -2 t w).  So a_0 = t and a_n = w Q_n(t) / n!.  They are
evaluated in 60-digit arithmetic (mpmath) and rounded to the nearest double.

The truncation error of degree 10 on |d| <= 1/32 is below 1e-19 relative;
with the rounding of the coefficients the polynomial, evaluated exactly,
is within 0.77 ulp of tanh (checked at 12 points per interval by this
script with --check).  The table is stored coefficient-major,
T[n * 257 + k], so that neighboring intervals share cache lines.

Run: python gen_tanh_table.py [--check] > tanh_table.inc
"""
import sys

import mpmath as mp

mp.mp.dps = 60
DEG = 10
NK = 257
H = mp.mpf(1) / 16


def q_polys(deg):
    """Integer coefficient lists (ascending powers of t) of Q_1..Q_deg."""
    qs = [None, [1]]
    for n in range(1, deg):
        q = qs[n]
        nxt = [0] * (len(q) + 1)
        for p, c in enumerate(q):          # -2 t Q_n
            nxt[p + 1] += -2 * c
        for p in range(1, len(q)):         # (1 - t^2) Q_n'
            c = p * q[p]
            nxt[p - 1] += c
            nxt[p + 1] -= c
        while len(nxt) > 1 and nxt[-1] == 0:
            nxt.pop()
        qs.append(nxt)
    return qs


def coefficients(c, qs):
    t = mp.tanh(c)
    w = 1 - t * t
    out = [t]
    for n in range(1, DEG + 1):
        qv = mp.mpf(0)
        for p in reversed(range(len(qs[n]))):
            qv = qv * t + qs[n][p]
        out.append(w * qv / mp.factorial(n))
    return out


def main():
    qs = q_polys(DEG)
    table = [[0.0] * NK for _ in range(DEG + 1)]
    for k in range(NK):
        for n, a in enumerate(coefficients(k * H, qs)):
            table[n][k] = float(a)
    if "--check" in sys.argv:
        import math
        worst = 0.0
        for k in range(NK):
            lo = 0.0 if k == 0 else -1.0 / 32
            for j in range(12):
                d = lo + (1.0 / 32 - lo) * j / 11
                x = k * H + mp.mpf(d)
                y = sum(mp.mpf(table[n][k]) * mp.mpf(d) ** n for n in range(DEG + 1))
                ex = mp.tanh(x)
                if ex != 0:
                    worst = max(worst, float(abs(y - ex)) / math.ulp(float(ex)))
        print(f"max error {worst:.3f} ulp", file=sys.stderr)
    print("// Generated by gen_tanh_table.py: Taylor coefficients a_n(c_k) of tanh,")
    print(f"// c_k = k/16, n = 0..{DEG}, k = 0..{NK - 1}, stored at [n * {NK} + k].")
    print(f"constexpr int kTanhDeg = {DEG};")
    print(f"constexpr int kTanhK = {NK};")
    print(f"static __device__ const double kTanhTab[{(DEG + 1) * NK}] = {{")
    for n in range(DEG + 1):
        row = table[n]
        for k0 in range(0, NK, 4):
            print("    " + ", ".join(float.hex(v) for v in row[k0:k0 + 4]) + ",")
    print("};")


if __name__ == "__main__":
    main()
