"""Pins for the CPU oracle: brute force, library routines, exact arithmetic,
closed forms and invariants -- each a check that does not re-run the
oracle's own formula.  (CPU only.)
"""
import json
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_img(rng, h, w):
    return rng.integers(0, 256, (h, w), dtype=np.uint8)


# ---------------------------------------------------------------------------
# window sums (Sec. 2): two oracle paths, a brute-force loop and a library box filter
# ---------------------------------------------------------------------------

SHAPES = [(1, 1), (1, 7), (7, 1), (2, 3), (5, 5), (8, 13), (13, 8), (17, 23)]


@pytest.mark.parametrize("h,w", SHAPES)
def test_naive_equals_sliding_all_windows(h, w):
    rng = np.random.default_rng(h * 100 + w)
    f = _rand_img(rng, h, w)
    for W in range(1, 2 * max(h, w) + 2):
        a = oracle.window_sums(f, W, oracle.NAIVE)
        b = oracle.window_sums(f, W, oracle.SLIDING)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y, err_msg=f"W={W}")


def _brute_sums(f, W):
    """Independent pure-Python window loop (Sec. 2 window set, clipped)."""
    h, w = f.shape
    lo = W // 2
    hi = W - 1 - lo
    n = np.zeros((h, w), np.int64)
    s1 = np.zeros((h, w), np.int64)
    s2 = np.zeros((h, w), np.int64)
    for y in range(h):
        for x in range(w):
            vals = [int(f[yy, xx]) for yy in range(y - lo, y + hi + 1) for xx in range(x - lo, x + hi + 1)
                    if 0 <= yy < h and 0 <= xx < w]
            n[y, x] = len(vals)
            s1[y, x] = sum(vals)
            s2[y, x] = sum(v * v for v in vals)
    return n, s1, s2


@pytest.mark.parametrize("W", [1, 2, 3, 4, 5, 8, 9, 17])
def test_sums_brute_force_tiny(W):
    rng = np.random.default_rng(W)
    f = _rand_img(rng, 7, 9)
    ref = _brute_sums(f, W)
    for method in (oracle.NAIVE, oracle.SLIDING):
        got = oracle.window_sums(f, W, method)
        for x, y in zip(got, ref):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("W", [1, 2, 6, 15, 16, 31])
def test_sums_match_scipy_box_filter(W):
    """Clipped window sums = zero-padded correlation with a W x W box (origin W//2)."""
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(100 + W)
    f = _rand_img(rng, 40, 57).astype(np.int64)
    box = np.ones((W, W), np.int64)
    n_ref = nd.correlate(np.ones_like(f), box, mode="constant", cval=0)
    s1_ref = nd.correlate(f, box, mode="constant", cval=0)
    s2_ref = nd.correlate(f * f, box, mode="constant", cval=0)
    n, s1, s2 = oracle.window_sums(f.astype(np.uint8), W)
    np.testing.assert_array_equal(n, n_ref)
    np.testing.assert_array_equal(s1, s1_ref)
    np.testing.assert_array_equal(s2, s2_ref)


def test_integral_images_match_cumsum_and_window_sums():
    rng = np.random.default_rng(7)
    f = _rand_img(rng, 33, 41)
    I1, I2 = oracle.integral(f)
    f64 = f.astype(np.int64)
    ref1 = np.zeros((34, 42), np.int64)
    ref2 = np.zeros((34, 42), np.int64)
    ref1[1:, 1:] = f64.cumsum(0).cumsum(1)
    ref2[1:, 1:] = (f64 * f64).cumsum(0).cumsum(1)
    np.testing.assert_array_equal(I1, ref1)
    np.testing.assert_array_equal(I2, ref2)
    # four-corner lookups of the integral images give the clipped window sums
    W = 7
    lo, hi = W // 2, W - 1 - W // 2
    n, s1, s2 = oracle.window_sums(f, W)
    for y in range(33):
        for x in range(41):
            y0, y1 = max(0, y - lo), min(32, y + hi) + 1
            x0, x1 = max(0, x - lo), min(40, x + hi) + 1
            assert I1[y1, x1] - I1[y0, x1] - I1[y1, x0] + I1[y0, x0] == s1[y, x]
            assert I2[y1, x1] - I2[y0, x1] - I2[y1, x0] + I2[y0, x0] == s2[y, x]
            assert (y1 - y0) * (x1 - x0) == n[y, x]


# ---------------------------------------------------------------------------
# threshold and decision (Eq. 3, Eq. 4, Niblack) against exact arithmetic
# ---------------------------------------------------------------------------

def _exact_sign(f, n, s1, s2, rule, k, R):
    """Sign of f - t with exact rationals; t irrational only through sqrt(V)."""
    k = Fraction(k)
    R = Fraction(R)
    V = n * s2 - s1 * s1
    m = Fraction(s1, n)
    if rule == oracle.SAUVOLA:
        A = f - m * (1 - k)            # f - t = A - B sqrt(V)
        B = m * k / (R * n)
    else:
        A = f - m
        B = k / n
    # sign(A - B sqrt(V))
    if B == 0 or V == 0:
        return (A > 0) - (A < 0)
    if B > 0:
        if A <= 0:
            return -1
        d = A * A - B * B * V
        return (d > 0) - (d < 0)
    # B < 0: A - B sqrt(V) = A + |B| sqrt(V)
    if A >= 0:
        return 1
    d = B * B * V - A * A
    return (d > 0) - (d < 0)


def _exact_t(n, s1, s2, rule, k, R):
    getcontext().prec = 60
    V = n * s2 - s1 * s1
    m = Decimal(s1) / Decimal(n)
    s = Decimal(V).sqrt() / Decimal(n)
    k = Decimal(k)
    R = Decimal(R)
    if rule == oracle.SAUVOLA:
        return m * (1 + k * (s / R - 1))
    return m + k * s


@pytest.mark.parametrize("rule,k,R", [(oracle.SAUVOLA, 0.5, 128.0), (oracle.SAUVOLA, 0.34, 128.0),
                                      (oracle.SAUVOLA, 0.2, 64.0), (oracle.NIBLACK, -0.2, 128.0),
                                      (oracle.NIBLACK, 0.3, 128.0)])
def test_decision_matches_exact_rational(rule, k, R):
    rng = np.random.default_rng(11)
    for trial in range(6):
        f = _rand_img(rng, 6, 8)
        if trial % 2:
            f = (f // 64 * 64).astype(np.uint8)   # few distinct values: many near-ties
        W = [3, 4, 5, 7, 2, 9][trial]
        mask, ties = oracle.binarize(f, W, rule, k, R, method=oracle.NAIVE)
        n, s1, s2 = _brute_sums(f, W)
        tie_count = 0
        for y in range(6):
            for x in range(8):
                args = (int(n[y, x]), int(s1[y, x]), int(s2[y, x]))
                t = oracle.threshold_value(*args, rule, k, R)
                te = _exact_t(*args, rule, k, R)
                # fp64 threshold within a few ulps of the exact value
                assert abs(Decimal(t) - te) <= Decimal(8) * Decimal(2) ** -52 * max(Decimal(1), abs(te))
                is_tie = abs(int(f[y, x]) - t) < 1e-9
                tie_count += is_tie
                if not is_tie:
                    sgn = _exact_sign(int(f[y, x]), *args, rule, k, R)
                    assert mask[y, x] == (0 if sgn < 0 else 255)
        assert ties == tie_count


def test_worked_example_golden():
    g = json.load(open(os.path.join(GOLDEN, "worked_3x3.json")))
    img = np.array(g["image"], np.uint8)
    W = g["W"]
    n, s1, s2 = oracle.window_sums(img, W)
    ms, _ = oracle.sauvola(img, W, g["sauvola"]["k"], g["sauvola"]["R"])
    mn, _ = oracle.niblack(img, W, g["niblack"]["k"])
    for p in g["pixels"]:
        y, x = p["y"], p["x"]
        assert (n[y, x], s1[y, x], s2[y, x]) == (p["n"], p["S1"], p["S2"])
        assert n[y, x] * s2[y, x] - s1[y, x] ** 2 == p["V"]
        ts = oracle.threshold_value(n[y, x], s1[y, x], s2[y, x], oracle.SAUVOLA,
                                    g["sauvola"]["k"], g["sauvola"]["R"])
        tn = oracle.threshold_value(n[y, x], s1[y, x], s2[y, x], oracle.NIBLACK, g["niblack"]["k"], 1.0)
        assert ts == pytest.approx(p["t_sauvola"], abs=1e-12)
        assert tn == pytest.approx(p["t_niblack"], abs=1e-12)
        assert ms[y, x] == p["g_sauvola"] and mn[y, x] == p["g_niblack"]


def test_worked_example_derivation_matches_fixture():
    """Every number of the worked example is re-derived from the definitions with exact arithmetic
    (tests/golden/derive_worked_3x3.py: rationals and a 60-digit square root, no oracle call)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("derive_worked_3x3", os.path.join(GOLDEN, "derive_worked_3x3.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    g = json.load(open(os.path.join(GOLDEN, "worked_3x3.json")))
    assert g["image"] == mod.IMAGE and g["W"] == mod.W
    derived = mod.derive()
    assert len(derived) == len(g["pixels"])
    for p, q in zip(g["pixels"], derived):
        for key, v in p.items():
            if isinstance(v, float):
                assert v == pytest.approx(q[key], abs=1e-12), key
            else:
                assert v == q[key], key


# ---------------------------------------------------------------------------
# closed forms and special cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("c", [0, 1, 37, 128, 255])
def test_constant_image(c):
    f = np.full((11, 14), c, np.uint8)
    for W in (1, 4, 5, 15, 40):
        n, s1, s2 = oracle.window_sums(f, W)
        np.testing.assert_array_equal(s1, n * c)
        np.testing.assert_array_equal(s2, n * c * c)
        # Sauvola: s = 0, t = c (1 - k) exactly
        for k in (0.2, 0.5):
            t = oracle.threshold_value(int(n[5, 5]), int(s1[5, 5]), int(s2[5, 5]), oracle.SAUVOLA, k, 128.0)
            assert t == c * (1.0 - k)
            m, ties = oracle.sauvola(f, W, k, 128.0)
            assert (m == 255).all()
            assert ties == (f.size if c == 0 else 0)
        # Niblack: t = c, every pixel an exact tie resolved to 255 (strict < in Eq. 3)
        m, ties = oracle.niblack(f, W, -0.2)
        assert (m == 255).all() and ties == f.size


@pytest.mark.parametrize("a,b", [(30, 200), (200, 30), (0, 255), (90, 91)])
def test_step_edge_closed_form(a, b):
    W = 9
    f = np.full((30, 40), b, np.uint8)
    f[:, :20] = a
    n, s1, s2 = oracle.window_sums(f, W)
    y = 15
    for x in range(16, 25):
        p = max(0, min(W, 20 - (x - 4)))            # columns of value a in the window
        assert n[y, x] == W * W
        assert s1[y, x] == W * (p * a + (W - p) * b)
        m = (p * a + (W - p) * b) / W
        s = abs(a - b) * math.sqrt(p * (W - p)) / W
        for rule, k in ((oracle.SAUVOLA, 0.5), (oracle.NIBLACK, -0.2)):
            t = oracle.threshold_value(int(n[y, x]), int(s1[y, x]), int(s2[y, x]), rule, k, 128.0)
            ref = m * (1 + k * (s / 128.0 - 1)) if rule == oracle.SAUVOLA else m + k * s
            assert t == pytest.approx(ref, rel=1e-13, abs=1e-12)


def test_impulse():
    f = np.zeros((12, 15), np.uint8)
    f[5, 7] = 200
    W = 5
    n, s1, s2 = oracle.window_sums(f, W)
    for y in range(12):
        for x in range(15):
            inside = abs(y - 5) <= 2 and abs(x - 7) <= 2
            assert s1[y, x] == (200 if inside else 0)
            assert s2[y, x] == (40000 if inside else 0)
            ny = min(11, y + 2) - max(0, y - 2) + 1
            nx = min(14, x + 2) - max(0, x - 2) + 1
            assert n[y, x] == ny * nx


def test_k_zero_is_mean_threshold():
    """k = 0: both rules reduce to the local-mean threshold f < S1/n (integer test n f < S1)."""
    rng = np.random.default_rng(3)
    f = _rand_img(rng, 25, 31)
    for W in (3, 8, 15):
        n, s1, _ = oracle.window_sums(f, W)
        ref = np.where(f.astype(np.int64) * n < s1, 0, 255)
        for rule in (oracle.SAUVOLA, oracle.NIBLACK):
            m, _ = oracle.binarize(f, W, rule, 0.0, 128.0)
            np.testing.assert_array_equal(m, ref)


def test_s_equals_R_gives_mean():
    """When s = R, Eq. 4 gives t = m for every k."""
    for a, b in ((10, 50), (200, 100), (0, 254)):
        f = np.array([[a, b]], np.uint8)
        R = abs(a - b) / 2.0                      # two-pixel window: s = |a - b| / 2 exactly
        for k in (0.1, 0.5, 0.9):
            t = oracle.threshold_value(2, a + b, a * a + b * b, oracle.SAUVOLA, k, R)
            assert t == (a + b) / 2.0
            m, _ = oracle.sauvola(f, 3, k, R)
            np.testing.assert_array_equal(m[0], [0 if v < (a + b) / 2 else 255 for v in (a, b)])


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W", [3, 7, 15])
def test_flip_transpose_invariance(W):
    f = synth.page(48, 64, 9)
    for rule, k in ((oracle.SAUVOLA, 0.5), (oracle.NIBLACK, -0.2)):
        m, _ = oracle.binarize(f, W, rule, k, 128.0)
        for op in (np.fliplr, np.flipud, np.transpose):
            m2, _ = oracle.binarize(op(f).copy(), W, rule, k, 128.0)
            np.testing.assert_array_equal(op(m), m2)


def test_additive_constant_niblack():
    rng = np.random.default_rng(5)
    f = rng.integers(20, 200, (30, 30), dtype=np.uint8)
    c = 40
    W = 7
    n, s1, s2 = oracle.window_sums(f, W)
    n2, s12, s22 = oracle.window_sums(f + c, W)
    np.testing.assert_array_equal(s12, s1 + n * c)
    np.testing.assert_array_equal(s22, s2 + 2 * c * s1 + n * c * c)
    np.testing.assert_array_equal(n * s2 - s1 * s1, n2 * s22 - s12 * s12)
    m1, _ = oracle.niblack(f, W, -0.2)
    m2, _ = oracle.niblack(f + c, W, -0.2)
    diff = np.argwhere(m1 != m2)
    for y, x in diff:    # only exact or near ties may flip
        _, tie, t = oracle.pixel(f, W, oracle.NIBLACK, -0.2, 128.0, y, x)
        assert abs(int(f[y, x]) - t) < 1e-9


# ---------------------------------------------------------------------------
# gray conversion (Eq. 1), packing, pipeline plumbing
# ---------------------------------------------------------------------------

def test_gray_conversion():
    rng = np.random.default_rng(1)
    rgb = rng.integers(0, 256, (300, 400, 3), dtype=np.uint8)
    g = oracle.gray(rgb).astype(np.float64)
    r, gg, b = (rgb[..., i].astype(np.float64) for i in range(3))
    exact = 0.299 * r + 0.587 * gg + 0.114 * b
    assert np.abs(g - exact).max() <= 0.5 + 1e-9     # nearest integer
    away = np.abs((exact % 1.0) - 0.5) > 1e-6
    np.testing.assert_array_equal(g[away], np.floor(exact + 0.5)[away])
    # gray input r = g = b = v maps to v (weights sum to 1)
    v = np.arange(256, dtype=np.uint8)
    np.testing.assert_array_equal(oracle.gray(np.stack([v, v, v], -1)[None])[0], v)
    # exact half-way values round up: 299r+587g+114b = 1000 q + 500
    assert oracle.gray(np.array([[[0, 0, 0]]], np.uint8))[0, 0] == 0
    # 299*1 + 587*0 + 114*... find a triple whose exact value ends in .5
    found = False
    for rr in range(256):
        for bb in range(256):
            if (299 * rr + 114 * bb) % 1000 == 500:
                q = (299 * rr + 114 * bb - 500) // 1000
                assert oracle.gray(np.array([[[rr, 0, bb]]], np.uint8))[0, 0] == q + 1
                found = True
                break
        if found:
            break
    assert found


def test_pack_matches_numpy_packbits():
    rng = np.random.default_rng(2)
    for w in (1, 7, 8, 9, 37):
        m = np.where(rng.random((5, w)) < 0.5, 0, 255).astype(np.uint8)
        ref = np.packbits(m == 255, axis=1, bitorder="little")
        np.testing.assert_array_equal(oracle.pack(m), ref)


def test_threads_and_pixel_queries_agree():
    p = synth.page(97, 131, 4, synth.STAINS, 3)
    for W in (4, 15):
        m1, t1 = oracle.sauvola(p, W, threads=1)
        m4, t4 = oracle.sauvola(p, W, threads=4)
        mn, tn = oracle.sauvola(p, W, method=oracle.NAIVE, threads=3)
        np.testing.assert_array_equal(m1, m4)
        np.testing.assert_array_equal(m1, mn)
        assert t1 == t4 == tn
        rng = np.random.default_rng(W)
        for _ in range(40):
            y, x = int(rng.integers(0, 97)), int(rng.integers(0, 131))
            assert oracle.pixel(p, W, oracle.SAUVOLA, 0.5, 128.0, y, x)[0] == m1[y, x]


def test_plausible_mistakes_are_caught():
    """Plant typical mistakes in a copy of the threshold rule and check a pin fails."""
    g = json.load(open(os.path.join(GOLDEN, "worked_3x3.json")))
    p = g["pixels"][0]
    n, S1, S2 = p["n"], p["S1"], p["S2"]
    m = S1 / n
    s_pop = math.sqrt(n * S2 - S1 * S1) / n
    s_sample = math.sqrt((n * S2 - S1 * S1) / (n * (n - 1)))       # wrong: sample std
    good = m * (1 + 0.5 * (s_pop / 128 - 1))
    assert good == pytest.approx(p["t_sauvola"], abs=1e-12)
    assert m * (1 + 0.5 * (s_sample / 128 - 1)) != pytest.approx(p["t_sauvola"], abs=1e-6)
    assert m * (1 - 0.5 * (s_pop / 128 - 1)) != pytest.approx(p["t_sauvola"], abs=1e-6)  # sign
