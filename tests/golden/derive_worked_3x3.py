"""Derivation of tests/golden/worked_3x3.json from the definitions alone.

The paper prints no numeric example, so the fixture's values come from this
derivation: window sums by direct enumeration of the clipped W x W window
(Sec. 2, the window set S), the population variance V = n*S2 - S1^2, the local
mean m = S1/n and standard deviation s = sqrt(V)/n, the Sauvola threshold of
Eq. 4 and the Niblack rule t = m + k*s, and the decision of Eq. 3 (0 if f < t,
else 255).  Every step is exact: rationals (fractions.Fraction) for m and the
thresholds' rational parts, and a 60-digit decimal square root for s.  Nothing
here imports or calls the oracle.

Run it to print the JSON (python tests/golden/derive_worked_3x3.py); the test
test_worked_example_derivation_matches_fixture re-derives every value and
compares it with the stored file.
"""
import json
import os
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60

IMAGE = [[10, 20, 30], [40, 50, 60], [70, 80, 90]]
W = 3
K_SAUVOLA, R = Fraction(1, 2), Fraction(128)
K_NIBLACK = Fraction(-1, 5)
PIXELS = [(1, 1), (0, 0), (2, 1)]


def window(y, x):
    """The clipped window around (y, x): r_lo = W // 2 pixels before, W - 1 - r_lo after."""
    r_lo = W // 2
    r_hi = W - 1 - r_lo
    h, w = len(IMAGE), len(IMAGE[0])
    return [IMAGE[j][i] for j in range(max(0, y - r_lo), min(h - 1, y + r_hi) + 1)
            for i in range(max(0, x - r_lo), min(w - 1, x + r_hi) + 1)]


def dec(q: Fraction) -> Decimal:
    return Decimal(q.numerator) / Decimal(q.denominator)


def derive():
    out = []
    for y, x in PIXELS:
        vals = window(y, x)
        n, S1, S2 = len(vals), sum(vals), sum(v * v for v in vals)
        V = n * S2 - S1 * S1
        m = Fraction(S1, n)
        s = Decimal(V).sqrt() / n                                   # exact to 60 digits
        t_sau = dec(m * (1 - K_SAUVOLA)) + dec(m * K_SAUVOLA / R) * s  # m (1 + k (s/R - 1))
        t_nib = dec(m) + dec(K_NIBLACK) * s
        f = IMAGE[y][x]
        out.append({"y": y, "x": x, "n": n, "S1": S1, "S2": S2, "V": V, "m": float(m), "s": float(s),
                    "t_sauvola": float(t_sau), "g_sauvola": 0 if Decimal(f) < t_sau else 255,
                    "t_niblack": float(t_nib), "g_niblack": 0 if Decimal(f) < t_nib else 255})
    return out


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    g = json.load(open(os.path.join(here, "worked_3x3.json")))
    g["pixels"] = derive()
    print(json.dumps(g, indent=2))
