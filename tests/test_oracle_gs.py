"""Pins of the reduced-set oracle (Sec. 2, Eq. 5) and of the Eq. 6 confusion
counts.  The structures are this project's proposals (the paper's Fig. 1 is
not available), so nothing here ties them to the paper's drawings; what is
pinned is that the oracle computes the stated sets and statistics:

* the sums equal a brute-force enumeration written differently (each
  structure as a union of line segments through the window, built as Python
  coordinate sets and clipped to the image);
* the whole-window structure (S' = S) reduces Eq. 5 to Eq. 4, so the mask and
  the tie count equal the exact oracle's;
* closed forms on ramps, constants and at the image corner;
* transpose symmetry for odd W;
* the F-measure of Eq. 6 on hand-counted masks and against a library F1.
"""
import numpy as np
import pytest

import oracle

ALL_GS = list(range(1, 7))


def lines(gs, W):
    """Each structure as line segments through the window: ('row', dy), ('col', dx), ('diag',), ('anti',)."""
    lo, hi = -(W // 2), W - 1 - W // 2
    cross = [("row", 0), ("col", 0)]
    diag = [("diag",), ("anti",)]
    frame = [("row", lo), ("row", hi), ("col", lo), ("col", hi)]
    return {1: cross, 2: diag, 3: cross + diag, 4: frame, 5: frame + cross, 6: frame + diag}[gs]


def brute_set(gs, W, y, x, h, w):
    lo, hi = -(W // 2), W - 1 - W // 2
    pts = set()
    for ln in lines(gs, W):
        for d in range(lo, hi + 1):
            if ln[0] == "row":
                pts.add((y + ln[1], x + d))
            elif ln[0] == "col":
                pts.add((y + d, x + ln[1]))
            elif ln[0] == "diag":
                pts.add((y + d, x + d))
            elif lo <= -d <= hi:  # anti-diagonal: dx = -dy, both inside the window
                pts.add((y + d, x - d))
    return {(a, b) for a, b in pts if 0 <= a < h and 0 <= b < w}


@pytest.mark.parametrize("W", [3, 4, 5, 6, 9])
@pytest.mark.parametrize("gs", ALL_GS)
def test_sums_equal_brute_force_sets(gs, W):
    rng = np.random.default_rng(100 + 10 * gs + W)
    f = rng.integers(0, 256, (11, 13), dtype=np.uint8)
    n, s1, s2 = oracle.gs_sums(f, W, gs)
    h, w = f.shape
    for y in range(h):
        for x in range(w):
            pts = brute_set(gs, W, y, x, h, w)
            vals = [int(f[a, b]) for a, b in pts]
            assert (n[y, x], s1[y, x], s2[y, x]) == (len(vals), sum(vals), sum(v * v for v in vals)), (y, x)


@pytest.mark.parametrize("W", [3, 6, 15])
def test_offsets_are_the_structures(W):
    """Offsets listed by the oracle = the brute-force set at an interior pixel, and the sizes are O(W)."""
    c = 2 * W
    for gs in ALL_GS:
        want = {(a - c, b - c) for a, b in brute_set(gs, W, c, c, 4 * W, 4 * W)}
        got = oracle.gs_offsets(gs, W)
        assert len(got) == len(set(got)) and set(got) == want
        assert len(got) <= 6 * W
    assert len(oracle.gs_offsets(oracle.GS_FULL, W)) == W * W


@pytest.mark.parametrize("W", [5, 7, 15])
def test_sizes_odd_closed_form(W):
    # frame (4W-4) meets the cross in 4 points and the diagonals in the 4 corners
    sizes = {g: len(oracle.gs_offsets(g, W)) for g in ALL_GS}
    assert sizes == {1: 2 * W - 1, 2: 2 * W - 1, 3: 4 * W - 3, 4: 4 * W - 4, 5: 6 * W - 9, 6: 6 * W - 9}
    # W = 3: the cross and diagonal arms end on the frame, so frame + either is the whole window
    assert {g: len(oracle.gs_offsets(g, 3)) for g in ALL_GS} == {1: 5, 2: 5, 3: 9, 4: 8, 5: 9, 6: 9}


@pytest.mark.parametrize("rule,k,R", [(oracle.SAUVOLA, 0.5, 128.0), (oracle.SAUVOLA, 0.2, 64.0),
                                      (oracle.NIBLACK, -0.2, 128.0)])
@pytest.mark.parametrize("W", [5, 8])
def test_whole_window_is_eq4(rule, k, R, W):
    """S' = S: m' = m, s' = s and Eq. 5 is Eq. 4 -- same mask and ties as the exact oracle."""
    import synth
    img = synth.page(60, 70, 9, synth.STAINS, 3)
    img[10:20, 10:30] = 120  # flat patch: ties of the definition
    want, wt = oracle.binarize(img, W, rule, k, R, method=oracle.NAIVE)
    got, gt = oracle.gs_binarize(img, W, oracle.GS_FULL, rule, k, R)
    np.testing.assert_array_equal(got, want)
    assert gt == wt
    f = oracle.gray(img)
    for a, b in zip(oracle.gs_sums(f, W, oracle.GS_FULL), oracle.window_sums(f, W, oracle.NAIVE)):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("W", [5, 9, 21])
def test_ramp_closed_forms(W):
    """f = c + x at interior pixels (odd W = 2r+1, Q = sum of d^2 over |d| <= r = r(r+1)(2r+1)/3):
    cross S2 = (2W-1) v^2 + Q; diagonals (2W-1) v^2 + 2Q;
    frame S1 = (4W-4) v, S2 = 2 (W v^2 + Q) + (W-2) ((v-r)^2 + (v+r)^2)."""
    r = W // 2
    Q = r * (r + 1) * (2 * r + 1) // 3
    h, w = 2 * W + 5, 3 * W
    c = 7
    f = (c + np.arange(w))[None, :].repeat(h, 0).astype(np.uint8)
    sums = {g: oracle.gs_sums(f, W, g) for g in (1, 2, 4)}
    for y in range(r, h - r):
        for x in range(r, w - r):
            v = c + x
            assert tuple(a[y, x] for a in sums[1]) == (2 * W - 1, (2 * W - 1) * v, (2 * W - 1) * v * v + Q)
            assert tuple(a[y, x] for a in sums[2]) == (2 * W - 1, (2 * W - 1) * v, (2 * W - 1) * v * v + 2 * Q)
            s2 = 2 * (W * v * v + Q) + (W - 2) * ((v - r) ** 2 + (v + r) ** 2)
            assert tuple(a[y, x] for a in sums[4]) == (4 * W - 4, (4 * W - 4) * v, s2)


@pytest.mark.parametrize("W", [5, 11])
def test_corner_counts(W):
    """At pixel (0, 0), odd W = 2r+1: cross 2r+1, diagonals r+1 (the anti-diagonal keeps only the centre),
    frame 2r+1 (bottom row r+1, right column r+1, one shared corner)."""
    r = W // 2
    f = np.full((2 * W, 2 * W), 50, np.uint8)
    n = {g: oracle.gs_sums(f, W, g)[0][0, 0] for g in (1, 2, 4)}
    assert n == {1: 2 * r + 1, 2: r + 1, 4: 2 * r + 1}


@pytest.mark.parametrize("gs", ALL_GS)
def test_constant_image(gs):
    """A constant c: S1' = c n', S2' = c^2 n' at every pixel, so s' = 0, t' = c (1 - k) and every pixel is
    background for k > 0."""
    c = 93
    src = np.full((23, 31), c, np.uint8)
    n, s1, s2 = oracle.gs_sums(src, 7, gs)
    np.testing.assert_array_equal(s1, c * n)
    np.testing.assert_array_equal(s2, c * c * n)
    assert n.min() >= 1
    mask, ties = oracle.gs_binarize(src, 7, gs, oracle.SAUVOLA, 0.5, 128.0)
    assert (mask == 255).all() and ties == 0


@pytest.mark.parametrize("gs", ALL_GS)
def test_transpose_symmetry_odd_W(gs):
    rng = np.random.default_rng(gs)
    f = rng.integers(0, 256, (17, 26), dtype=np.uint8)
    a = oracle.gs_sums(f, 7, gs)
    b = oracle.gs_sums(np.ascontiguousarray(f.T), 7, gs)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y.T)


def test_band_helper_matches_whole_page():
    import synth
    img = synth.page(90, 64, 4, synth.DOC, 1)
    whole, _ = oracle.gs_binarize(img, 15, oracle.GS_STAR, oracle.SAUVOLA, 0.5, 128.0)
    for y0, y1 in ((0, 10), (30, 47), (80, 90)):
        np.testing.assert_array_equal(
            oracle.gs_binarize_rows(img, 15, oracle.GS_STAR, oracle.SAUVOLA, 0.5, 128.0, y0, y1), whole[y0:y1])


def test_confusion_hand_counts():
    # mask ink = 0, reference ink = 1
    mask = np.array([[0, 0, 255], [0, 255, 255]], np.uint8)
    ref = np.array([[1, 0, 1], [1, 0, 0]], np.uint8)
    # (0,0) TP, (0,1) FP, (0,2) FN, (1,0) TP, (1,1) TN, (1,2) TN
    assert oracle.confusion(mask, ref) == (2, 1, 1, 2)
    fm, rec, prec = oracle.fmeasure((2, 1, 1, 2))
    assert rec == pytest.approx(2 / 3) and prec == pytest.approx(2 / 3) and fm == pytest.approx(2 / 3)
    assert oracle.fmeasure(oracle.confusion(mask, (mask == 0).astype(np.uint8)))[0] == 1.0
    assert oracle.fmeasure((0, 5, 5, 0)) == (0.0, 0.0, 0.0)


def test_fmeasure_equals_library_f1():
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(3)
    mask = np.where(rng.random((40, 50)) < 0.3, 0, 255).astype(np.uint8)
    ref = (rng.random((40, 50)) < 0.25).astype(np.uint8)
    fm, _, _ = oracle.fmeasure(oracle.confusion(mask, ref))
    assert fm == pytest.approx(skm.f1_score(ref.ravel(), (mask == 0).ravel().astype(np.uint8)), abs=1e-12)
