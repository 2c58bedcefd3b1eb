"""The fp32 error bounds behind the Niblack margin stages, checked on the CPU.

The fused kernel decides a pixel with an fp32 filter and re-decides it exactly
only when the filter lands inside a proven margin.  These tests emulate, with
numpy float32 arithmetic (each operation rounded to nearest, as on the device),
two of those fp32 evaluations and compare them with exact rational arithmetic
on random and extreme windows:

  - the unclipped-window Niblack filter nd = RN(S1 RN(1/n) + RN(RN(k/n) sq - f)),
    sq = sqrt.approx(V) with its worst relative error e = 2^-21 either way, must
    stay within the bound u (766 + 2.01 |k| s) + |k| s (e + 2.02 u) of t - f
    (the interior margin, half of E_int without the 1e-6);
  - the unclipped-window Sauvola filter nd = RN(S1 RN(omkn + kRn2 sq) - f) must
    stay within the host's Sauvola bound (half of its margin E without the 1e-6);
  - the per-pixel-n filters of border warps, constants from the table of
    correctly rounded 1/j and 1/j^2, must stay within the host's general bounds;
  - the single-pixel filters (whole-set constants, or a per-pixel n through
    rcp.approx) of the reduced-set kernel and of the margin re-evaluation must
    stay within the general margins;
  - the double-float stage's f - t must stay within the host's double_float_error;
  - the refinement D = RN(RN(n f - S1) - RN(RN(k) r)), r = RN(sqrt(RN(V))), must
    have the sign of X = n (f - t) and |X| / n > 1e-9 whenever
    |D| > 4.5 u |k| r + 1.01 n 1e-9.

Niblack t = m + k s with m = S1 / n, s = sqrt(V) / n, V = n S2 - S1^2 (Eq. 3 and
the Niblack rule); the exact X uses integer arithmetic and a 60-digit root."""
from decimal import Decimal, getcontext

import numpy as np
import pytest

import paper_1210_3165_gb300 as bnz

getcontext().prec = 60
U = 2.0 ** -24
E_SQRT = 2.0 ** -21
F32 = np.float32


def rn(x):
    return F32(x)


def v_to_float(V):
    # high word exact, low word rounded, one more rounding in the fused add (as on the device)
    hi, lo = V >> 32, V & 0xFFFFFFFF
    return rn(float(rn(hi)) * 4294967296.0 + float(rn(lo)))


def windows(rng, count):
    """(n, f, S1, S2) of random windows: W x W of random gray levels, plus near-flat and extreme ones."""
    out = []
    for i in range(count):
        W = int(rng.choice([3, 4, 15, 31, 61, 101, 255]))
        n = W * W
        kind = i % 4
        if kind == 0:
            g = rng.integers(0, 256, n)
        elif kind == 1:
            g = np.clip(rng.normal(rng.integers(0, 256), 3, n).round(), 0, 255).astype(np.int64)
        elif kind == 2:
            g = np.full(n, rng.integers(0, 256)); g[rng.integers(0, n)] = rng.integers(0, 256)
        else:
            g = rng.choice([0, 255], n)
        S1, S2 = int(g.sum()), int((g.astype(np.int64) ** 2).sum())
        out.append((n, int(rng.integers(0, 256)), S1, S2))
    return out


def exact_t_minus_f(n, f, S1, S2, k):
    V = n * S2 - S1 * S1
    s = Decimal(V).sqrt() / n
    return Decimal(S1) / n + Decimal(k) * s - f, s, V


def test_interior_niblack_filter_bound():
    rng = np.random.default_rng(5)
    for k in (-0.2, -0.5, 0.3, -1.5, 150.0):
        kn, invn_cache = None, {}
        for n, f, S1, S2 in windows(rng, 600):
            invn = rn(1.0 / n)
            kn = rn(k / n)
            tf, s, V = exact_t_minus_f(n, f, S1, S2, k)
            for d in (-E_SQRT, 0.0, E_SQRT):
                sq = rn(float(np.sqrt(np.float64(v_to_float(V)))) * (1.0 + d))
                y = rn(float(kn) * float(sq) - f)          # fma: one rounding
                nd = rn(float(S1) * float(invn) + float(y))  # fma: one rounding
                ks = abs(k) * float(s)
                bound = U * (766 + 2.01 * ks) + ks * (E_SQRT + 2.02 * U)
                assert abs(Decimal(float(nd)) - tf) <= Decimal(bound), (k, n, f, S1, S2, d)


def test_niblack_refinement_decides_correctly():
    rng = np.random.default_rng(9)
    tau = 1e-9
    decided = 0
    for k in (-0.2, -0.5, 0.3, -150.0):
        kf = rn(k)
        for n, f, S1, S2 in windows(rng, 600) + near_tie_windows(rng, k, 60):
            tf, s, V = exact_t_minus_f(n, f, S1, S2, k)
            X = -tf * n                                   # n (f - t)
            A = rn(n * f - S1)
            assert float(A) == n * f - S1                 # exact below 2^24
            r = rn(np.sqrt(np.float64(v_to_float(V))))    # correctly rounded root of the rounded V
            D = rn(float(A) - float(rn(float(kf) * float(r))))
            bnd = rn(float(rn(4.5 * U * abs(k))) * float(r) + float(rn(1.01 * tau)) * n)
            if abs(float(D)) > float(bnd):
                decided += 1
                assert (float(D) > 0) == (X > 0) and abs(X) / n > Decimal(tau), (k, n, f, S1, S2)
    assert decided > 1000


def sauvola_em(k, R):
    """Half the fp32 margin E of Sauvola before its 1e-6 (the host's bound, m <= 255, s <= 127.5)."""
    m, smax, ak = 255.0, 127.5, abs(k)
    T = m * (abs(1 - k) + ak * smax / R)
    return 6 * U * m * abs(1 - k) + m * ak * (smax / R) * (12 * U + E_SQRT) + U * T + U * (255 + T)


def test_interior_sauvola_filter_bound():
    """nd = RN(S1 RN(omkn + kRn2 sq) - f) with omkn = RN((1-k)/n), kRn2 = RN(k/(R n^2)) stays within the
    host's Sauvola bound of t - f = m (1 + k (s/R - 1)) - f."""
    rng = np.random.default_rng(11)
    for k, R in ((0.5, 128.0), (0.34, 128.0), (0.2, 64.0), (-3.0, 128.0), (20.0, 128.0), (0.5, 2.0)):
        em = sauvola_em(k, R)
        for n, f, S1, S2 in windows(rng, 400):
            omkn, kRn2 = rn((1 - k) / n), rn(k / (R * n * n))
            V = n * S2 - S1 * S1
            s = Decimal(V).sqrt() / n
            m = Decimal(S1) / n
            tf = m * (1 + Decimal(k) * (s / Decimal(R) - 1)) - f
            for d in (-E_SQRT, 0.0, E_SQRT):
                sq = rn(float(np.sqrt(np.float64(v_to_float(V)))) * (1.0 + d))
                x = rn(float(kRn2) * float(sq) + float(omkn))
                nd = rn(float(S1) * float(x) - f)
                assert abs(Decimal(float(nd)) - tf) <= Decimal(em), (k, R, n, f, S1, S2, d)


def niblack_em(k):
    """Half the fp32 margin E of Niblack before its 1e-6 (the host's general bound)."""
    m, smax, ak = 255.0, 127.5, abs(k)
    return 4 * U * m + U * 510 + ak * smax * (7 * U + E_SQRT) + U * (510 + ak * smax)


def clipped_windows(rng, count):
    """(nr, nc, f, S1, S2) of windows clipped at the page border: nr x nc pixels, nr, nc in 1..W."""
    out = []
    for i in range(count):
        W = int(rng.choice([3, 15, 31, 101, 255]))
        nr, nc = int(rng.integers(1, W + 1)), int(rng.integers(1, W + 1))
        g = rng.integers(0, 256, nr * nc) if i % 2 else np.clip(
            rng.normal(rng.integers(0, 256), 4, nr * nc).round(), 0, 255).astype(np.int64)
        out.append((nr, nc, int(rng.integers(0, 256)), int(g.sum()), int((g.astype(np.int64) ** 2).sum())))
    return out


def test_border_filter_bounds():
    """The per-pixel-n filters of warps at the page border (constants from the table of correctly rounded
    1/j and 1/j^2: c0 = RN(RN(a RN(1/nr)) RN(1/nc)), c1 likewise) stay within the host's general bounds."""
    rng = np.random.default_rng(13)
    for rule, k, R in (("sauvola", 0.5, 128.0), ("sauvola", -3.0, 128.0), ("sauvola", 0.5, 2.0),
                       ("niblack", -0.2, 1.0), ("niblack", 0.3, 1.0), ("niblack", -150.0, 1.0)):
        em = sauvola_em(k, R) if rule == "sauvola" else niblack_em(k)
        for nr, nc, f, S1, S2 in clipped_windows(rng, 400):
            n = nr * nc
            tr = (rn(1.0 / nr), rn(1.0 / (nr * nr)))
            tc = (rn(1.0 / nc), rn(1.0 / (nc * nc)))
            V = n * S2 - S1 * S1
            s = Decimal(V).sqrt() / n
            m = Decimal(S1) / n
            if rule == "sauvola":
                r0, r1 = rn(float(rn(1 - k)) * float(tr[0])), rn(float(rn(k / R)) * float(tr[1]))
                c0, c1 = rn(float(r0) * float(tc[0])), rn(float(r1) * float(tc[1]))
                tf = m * (1 + Decimal(k) * (s / Decimal(R) - 1)) - f
            else:
                r0, r1 = tr[0], rn(float(rn(k)) * float(tr[0]))
                c0, c1 = rn(float(r0) * float(tc[0])), rn(float(r1) * float(tc[0]))
                tf = m + Decimal(k) * s - f
            for d in (-E_SQRT, 0.0, E_SQRT):
                q = rn(float(np.sqrt(np.float64(v_to_float(V)))) * (1.0 + d))
                if rule == "sauvola":
                    nd = rn(float(S1) * float(rn(float(c1) * float(q) + float(c0))) - f)
                else:
                    nd = rn(float(S1) * float(c0) + float(rn(float(c1) * float(q) - f)))
                assert abs(Decimal(float(nd)) - tf) <= Decimal(em), (rule, k, R, nr, nc, f, S1, S2, d)


def fp64_definition_error(k):
    """The host's bound on the fp64 definition's own error, Niblack (w = 2^-53 per operation)."""
    return 8.0 * 2.0 ** -53 * (255.0 + abs(k) * 127.5)


def interior_niblack_margin(k):
    """The interior Niblack margin E_int: the fast filter's rounding before its last operation is at most
    u (510 + 1.01 |k| s) + |k| s (e + 2.02 u), s <= 127.5; the last rounding keeps the sign."""
    ks = abs(k) * 127.5
    em = U * (510 + 1.01 * ks) + ks * (E_SQRT + 2.02 * U)
    return 2 * em + 1e-6 + 2 * fp64_definition_error(k)


def sauvola_fp64_error(k, R):
    return 16.0 * 2.0 ** -53 * (255.0 + 255.0 * abs(1 - k) + 255.0 * abs(k) * (127.5 / R + 1.0))


@pytest.mark.parametrize("rule,k,R", [("niblack", -0.2, 1.0), ("niblack", 0.3, 1.0), ("niblack", -150.0, 1.0),
                                      ("niblack", 1e6, 1.0), ("sauvola", 0.5, 128.0), ("sauvola", 20.0, 128.0),
                                      ("sauvola", 0.5, 1e-3)])
def test_library_margins_are_these_bounds(rule, k, R):
    """The margins the library computes for a launch (bnz_decision_margins, host code) are the bounds these
    tests check: E = 2 em + 1e-6 + 2 (fp64 error) with the general em of each rule, E_int the interior
    Niblack margin (E for Sauvola), each rounded once to fp32."""
    E, Ei, _ = bnz.bnz_decision_margins(rule, k, R)
    if rule == "niblack":
        want_E = 2 * niblack_em(k) + 1e-6 + 2 * fp64_definition_error(k)
        want_Ei = min(interior_niblack_margin(k), float(np.float32(want_E)))
    else:
        want_E = 2 * sauvola_em(k, R) + 1e-6 + 2 * sauvola_fp64_error(k, R)
        want_Ei = want_E
    assert abs(E - want_E) <= 2e-7 * want_E and abs(Ei - want_Ei) <= 2e-7 * want_Ei, (E, want_E, Ei, want_Ei)


def near_tie_windows(rng, k, count):
    """Windows whose Niblack threshold lies within 3e-4 of an integer gray level f (the hard cases)."""
    out = []
    for _ in range(20):
        if len(out) >= count:
            break
        W = int(rng.choice([3, 4, 5, 7]))
        g = rng.integers(0, 256, (20000, W * W)).astype(np.int64)
        n = W * W
        S1, S2 = g.sum(1), (g * g).sum(1)
        t = S1 / n + k * np.sqrt(np.maximum(n * S2 - S1 * S1, 0)) / n
        f = np.clip(np.round(t), 0, 255)
        for i in np.nonzero(np.abs(t - f) < 3e-4)[0][: count - len(out)]:
            out.append((n, int(f[i]), int(S1[i]), int(S2[i])))
    return out


def test_interior_niblack_decision_rule():
    """Outside E_int the fast filter's sign is the sign of t - f and |t - f| is no tie (> 1e-9): on random
    windows and on windows whose threshold lies within 3e-4 of the pixel's level."""
    rng = np.random.default_rng(17)
    near = 0
    for k in (-0.2, -0.5, 0.3, -1.5, 150.0):
        Ei = bnz.bnz_decision_margins("niblack", k)[1]   # the library's margin, as a launch uses it
        for n, f, S1, S2 in windows(rng, 300) + near_tie_windows(rng, k, 60):
            invn, kn = rn(1.0 / n), rn(k / n)
            tf, s, V = exact_t_minus_f(n, f, S1, S2, k)
            for d in (-E_SQRT, 0.0, E_SQRT):
                sq = rn(float(np.sqrt(np.float64(v_to_float(V)))) * (1.0 + d))
                y = rn(float(kn) * float(sq) - f)
                nd = rn(float(S1) * float(invn) + float(y))
                if abs(float(nd)) >= Ei:
                    assert (float(nd) > 0) == (tf > 0) and abs(tf) > Decimal(1e-9), (k, n, f, S1, S2, d)
                else:
                    near += 1
    assert near > 0


# ---- the double-float stage (pairs of fp32 words), emulated operation by operation ----

def add(a, b):
    return rn(float(a) + float(b))


def sub(a, b):
    return rn(float(a) - float(b))


def mul(a, b):
    return rn(float(a) * float(b))


def fma(a, b, c):
    return rn(float(a) * float(b) + float(c))  # the product of two fp32 is exact in fp64


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def fast_two_sum(a, b):
    s = add(a, b)
    return s, sub(b, sub(s, a))


def df_add(a, b):
    s = two_sum(a[0], b[0])
    return fast_two_sum(s[0], add(s[1], add(a[1], b[1])))


def df_mul(a, b):
    p = mul(a[0], b[0])
    e = fma(a[0], b[0], -p)
    e = fma(a[0], b[1], fma(a[1], b[0], e))
    return fast_two_sum(p, e)


def df_div_int(x, nf):
    q = rn(np.float32(x[0]) / np.float32(nf))
    r = fma(-q, nf, x[0])
    return fast_two_sum(q, rn(np.float32(add(r, x[1])) / np.float32(nf)))


def df_sqrt_v(V):
    h, lo = V >> 32, V & 0xFFFFFFFF
    a = two_sum(mul(rn(h), 4294967296.0), mul(rn(lo >> 16), 65536.0))
    v = fast_two_sum(a[0], add(a[1], rn(lo & 0xFFFF)))
    if v[0] == 0:
        return F32(0), F32(0)
    sh = rn(np.sqrt(np.float32(v[0])))
    p = mul(sh, sh)
    pe = fma(sh, sh, -p)
    r = add(sub(sub(v[0], p), pe), v[1])
    return fast_two_sum(sh, rn(np.float32(r) / np.float32(mul(2.0, sh))))


def split(x):
    hi = rn(x)
    return hi, rn(x - float(hi))


def double_float_error(rule, k, R):
    u2, m, s, ak = 2.0 ** -48, 255.0, 127.5, abs(k)
    if rule == "sauvola":
        et = 12 * u2 * m * abs(1 - k) + 24 * u2 * m * s * ak / R
        T = m * abs(1 - k) + m * s * ak / R
    else:
        et = 4 * u2 * m + 17 * u2 * ak * s
        T = m + ak * s
    return 2 * (et + 3 * u2 * (255 + T))


@pytest.mark.parametrize("rule,k,R", [("sauvola", 0.5, 128.0), ("sauvola", 0.34, 128.0), ("sauvola", 20.0, 128.0),
                                      ("sauvola", 0.5, 0.5), ("niblack", -0.2, 1.0), ("niblack", -150.0, 1.0)])
def test_double_float_stage_bound(rule, k, R):
    """The second stage's f - t (double-float: pairs of fp32 with error-free sums and products, correctly
    rounded division and root) stays within the host's double_float_error of the exact f - t; the
    library's cut Tdf covers that bound, the fp64 definition's error and the 1e-9 tie width."""
    rng = np.random.default_rng(23)
    dfe = double_float_error(rule, k, R)
    Tdf = bnz.bnz_decision_margins(rule, k, R)[2]
    assert Tdf >= 1e-9 + dfe
    kd, c1, c2 = split(k), split(1 - k), split(k / R)
    for n, f, S1, S2 in windows(rng, 200) + (near_tie_windows(rng, k, 40) if rule == "niblack" else []):
        V = n * S2 - S1 * S1
        nf = rn(n)
        m = df_div_int((rn(S1), F32(0)), nf)
        sd = df_div_int(df_sqrt_v(V), nf)
        if rule == "sauvola":
            t = df_add(df_mul(m, c1), df_mul(df_mul(m, sd), c2))
            s_ex = Decimal(V).sqrt() / n
            t_ex = Decimal(S1) / n * (1 + Decimal(k) * (s_ex / Decimal(R) - 1))
        else:
            t = df_add(m, df_mul(kd, sd))
            t_ex = Decimal(S1) / n + Decimal(k) * Decimal(V).sqrt() / n
        d = df_add((rn(f), F32(0)), (-t[0], -t[1]))
        dv = Decimal(float(d[0])) + Decimal(float(d[1]))
        assert abs(dv - (f - t_ex)) <= Decimal(dfe), (rule, k, R, n, f, S1, S2)


def test_integer_ranges_of_the_window_sums():
    """The kernel's integer widths: S1 = sum f < 2^24 for every W <= 255 (exact in fp32 and int32),
    S2 = sum f^2 < 2^32, n f - S1 within (-2^24, 2^24); the variance numerator V = n S2 - S1^2 <= n^2 255^2 / 4
    fits 32 bits exactly up to W = 22 (the kernel's 32-bit path) and needs 64 bits from W = 23 on, and
    stays below 2^48 (the conversion to fp32 from two 32-bit words) for W <= 255."""
    W = 255
    n = W * W
    assert n * 255 < 2 ** 24 and n * 255 * 255 < 2 ** 32
    vmax = lambda W: (W * W) ** 2 * 255 ** 2 // 4
    assert vmax(22) < 2 ** 32 <= vmax(23)
    assert vmax(255) < 2 ** 48
    # the bound is reached: half the window 0, half 255 (n even) gives V = n^2 255^2 / 4
    n = 22 * 22
    S1, S2 = (n // 2) * 255, (n // 2) * 255 * 255
    assert n * S2 - S1 * S1 == vmax(22)


E_RCP = 2.0 ** -22


def set_windows(rng, count):
    """(n, f, S1, S2) over point sets of the reduced-set sizes (2W-1, 4W-3, 4W-4, 6W-9) with random levels."""
    out = []
    for i in range(count):
        W = int(rng.choice([3, 15, 31, 101, 255]))
        n = int(rng.choice([2 * W - 1, 4 * W - 3, 4 * W - 4, max(6 * W - 9, 1)]))
        g = rng.integers(0, 256, n) if i % 2 else np.clip(
            rng.normal(rng.integers(0, 256), 4, n).round(), 0, 255).astype(np.int64)
        out.append((n, int(rng.integers(0, 256)), int(g.sum()), int((g.astype(np.int64) ** 2).sum())))
    return out


@pytest.mark.parametrize("rule,k,R", [("sauvola", 0.5, 128.0), ("sauvola", -3.0, 128.0), ("sauvola", 0.5, 2.0),
                                      ("niblack", -0.2, 1.0), ("niblack", 0.3, 1.0), ("niblack", -150.0, 1.0)])
def test_general_filters_bound(rule, k, R):
    """The single-pixel filters of the reduced-set kernel and of the margin re-evaluation: d = f - t with the
    whole-set constants (host-rounded for n) or with a per-pixel n through rcp.approx (worst relative error
    2^-22 either way), sqrt.approx at its worst error either way, stay within half the library's general
    margin E less its 1e-6 and the fp64 definition's share."""
    rng = np.random.default_rng(29)
    E = bnz.bnz_decision_margins(rule, k, R)[0]
    fp64e = sauvola_fp64_error(k, R) if rule == "sauvola" else fp64_definition_error(k)
    em = (E - 1e-6) / 2 - fp64e
    kf, omk, kR = rn(k), rn(1 - k), rn(k / R)
    for n, f, S1, S2 in set_windows(rng, 300):
        V = n * S2 - S1 * S1
        s_ex = Decimal(V).sqrt() / n
        m_ex = Decimal(S1) / n
        if rule == "sauvola":
            t_ex = m_ex * (1 + Decimal(k) * (s_ex / Decimal(R) - 1))
        else:
            t_ex = m_ex + Decimal(k) * s_ex
        ff, S1f = rn(f), rn(S1)
        for ds in (-E_SQRT, E_SQRT):
            sq = rn(float(np.sqrt(np.float64(v_to_float(V)))) * (1.0 + ds))
            # whole set: constants rounded once on the host
            if rule == "sauvola":
                d_whole = fma(-S1f, fma(rn(k / (R * n * n)), sq, rn((1 - k) / n)), ff)
            else:
                d_whole = fma(-rn(k / n), sq, fma(-rn(1.0 / n), S1f, ff))
            ds_ = [d_whole]
            for dr in (-E_RCP, E_RCP):
                invn = rn(rn(1.0 / n) * (1.0 + dr))
                if rule == "sauvola":
                    ds_.append(fma(-S1f, fma(mul(mul(kR, invn), invn), sq, mul(omk, invn)), ff))
                else:
                    ds_.append(fma(-mul(kf, invn), sq, fma(-invn, S1f, ff)))
            for d in ds_:
                assert abs(Decimal(float(d)) - (f - t_ex)) <= Decimal(em), (rule, k, R, n, f, S1, S2, ds)
