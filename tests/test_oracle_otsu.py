"""Pins for the oracle's global threshold (Eq. 2 with Otsu's T): exact rational
arithmetic, the between-class variance recomputed from the pixels themselves,
closed forms and invariants.  (CPU only.)"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def exact_best(hist):
    """Every T in [1, 255] whose exact between-class variance w0 w1 (mu0 - mu1)^2 is the largest."""
    hist = [int(v) for v in hist]
    N = sum(hist)
    best, ts = None, []
    for t in range(1, 256):
        n0 = sum(hist[:t])
        n1 = N - n0
        if n0 == 0 or n1 == 0:
            continue
        mu0 = Fraction(sum(i * hist[i] for i in range(t)), n0)
        mu1 = Fraction(sum(i * hist[i] for i in range(t, 256)), n1)
        v = Fraction(n0, N) * Fraction(n1, N) * (mu0 - mu1) ** 2
        if best is None or v > best:
            best, ts = v, [t]
        elif v == best:
            ts.append(t)
    return best, ts


@pytest.mark.parametrize("seed", range(12))
def test_threshold_is_the_exact_argmax(seed):
    rng = np.random.default_rng(seed)
    # sparse and dense histograms, with and without empty bins at the ends
    hist = np.zeros(256, np.uint64)
    lo, hi = sorted(rng.integers(0, 256, 2))
    k = int(rng.integers(2, 40))
    levels = rng.integers(lo, hi + 1, k)
    np.add.at(hist, levels, rng.integers(1, 10_000, k).astype(np.uint64))
    T, q = oracle.otsu_threshold(hist)
    best, ts = exact_best(hist)
    if best is None:
        assert T == 0
        return
    # the fp64 criterion may tie or reorder candidates within its rounding; otherwise the exact
    # argmax, and the smallest of several exact maxima
    qmax = q[T]
    near = [t for t in range(1, 256) if q[t] >= qmax * (1 - 1e-12)]
    assert ts[0] == T or ts[0] in near


def test_between_class_variance_from_the_pixels():
    # the criterion recomputed from the pixel lists (class 0: f < T, Eq. 2), not from the histogram
    rng = np.random.default_rng(7)
    for _ in range(6):
        img = synth.page(40, 57, int(rng.integers(1, 1000)))
        T, q = oracle.otsu_threshold(oracle.histogram(img))
        f = img.astype(np.float64).ravel()
        var = np.full(256, -1.0)
        for t in range(1, 256):
            c0, c1 = f[f < t], f[f >= t]
            if len(c0) and len(c1):
                var[t] = len(c0) / len(f) * len(c1) / len(f) * (c0.mean() - c1.mean()) ** 2
        assert var[T] == pytest.approx(var.max(), rel=1e-12)
        assert np.all(var[:T] < var.max() * (1 - 1e-12)) or T == int(np.argmax(var))


@pytest.mark.parametrize("a,b", [(0, 255), (10, 200), (99, 100), (3, 4)])
def test_two_levels(a, b):
    img = np.full((20, 30), a, np.uint8)
    img[:, 7:] = b
    mask, T = oracle.otsu(img)
    assert T == a + 1                       # the smallest threshold that separates the two levels
    assert np.all(mask[:, :7] == 0) and np.all(mask[:, 7:] == 255)


@pytest.mark.parametrize("c", [0, 1, 128, 255])
def test_one_level_page(c):
    mask, T = oracle.otsu(np.full((9, 11), c, np.uint8))
    assert T == 0 and np.all(mask == 255)


def test_offset_invariance():
    img = synth.page(64, 80, 3)
    img = (img // 2).astype(np.uint8)       # room for an offset without clipping
    _, T = oracle.otsu(img)
    _, T2 = oracle.otsu(img + 40)
    assert T > 0 and T2 == T + 40


def test_rgb_histogram_is_the_gray_histogram_and_mask_is_eq2():
    img = synth.page(50, 70, 9, synth.STAINS, 3)
    g = oracle.gray(img)
    assert np.array_equal(oracle.histogram(img), np.bincount(g.ravel(), minlength=256).astype(np.uint64))
    mask, T = oracle.otsu(img)
    assert np.array_equal(mask, np.where(g < T, 0, 255).astype(np.uint8))
    packed, T2 = oracle.otsu(img, packed=True)
    assert T2 == T and np.array_equal(packed, np.packbits(mask == 255, axis=1, bitorder="little"))


def test_plausible_mistakes_are_caught():
    """Planted in a copy of the criterion: each changes the chosen T on a page where the pins hold."""
    hist = np.bincount(synth.page(64, 64, 5).ravel(), minlength=256)
    best, ts = exact_best(hist)
    N, S = int(hist.sum()), int((np.arange(256) * hist).sum())

    def argmax(crit):
        vals = [(crit(t), t) for t in range(1, 256)]
        return max(vals, key=lambda v: (v[0], -v[1]))[1]

    def parts(t, upto):
        n0 = int(hist[:upto].sum())
        s0 = int((np.arange(upto) * hist[:upto]).sum())
        return n0, s0

    def good(t):
        n0, s0 = parts(t, t)
        n1 = N - n0
        return Fraction((N * s0 - S * n0) ** 2, n0 * n1) if n0 and n1 else -1

    def inclusive_split(t):                 # class 0 = [0, t] instead of [0, t-1]
        n0, s0 = parts(t, t + 1)
        n1 = N - n0
        return Fraction((N * s0 - S * n0) ** 2, n0 * n1) if n0 and n1 else -1

    def no_class_weights(t):                # (mu0 - mu1)^2 alone
        n0, s0 = parts(t, t)
        n1 = N - n0
        return (Fraction(s0, n0) - Fraction(S - s0, n1)) ** 2 if n0 and n1 else -1

    assert argmax(good) == ts[0]
    assert argmax(inclusive_split) != ts[0]
    assert argmax(no_class_weights) != ts[0]
