"""GPU parity of the reduced-set rule (Sec. 2, Eq. 5) and of the Eq. 6 counts.

The structures are this library's proposals (the paper's Fig. 1 is not
available); the kernel must reproduce the oracle's definition of them bit for
bit: the same mask and the same tie count on pages that span several strips
(256 columns) with a ragged tail and several row segments, for odd and even W
up to the maximum, both rules, gray and RGB, degenerate sizes, extreme k and R,
and sampled bands of a full 4096^2 page."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GS = list(range(1, 7))


@pytest.fixture(scope="module")
def bnz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1210_3165_gb300 as b
    b.load()
    return b


def run(bnz, img, W, gs, rule, k, R):
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = bnz.gs_binarize(bnz.to_device_pitched(img), W, gs, rule, k, R, d_stats=st)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


def check(bnz, img, W, gs, rule="sauvola", k=None, R=128.0):
    rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
    if k is None:
        k = 0.5 if rule == "sauvola" else -0.2
    ref, ties = oracle.gs_binarize(img, W, gs, rid, k, R)
    got, st = run(bnz, img, W, gs, rule, k, R)
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError(f"gs={gs} W={W} {rule}: {len(bad)} mismatches, first at {tuple(bad[0])}")
    assert st[1] == ties, (st, ties)
    return st


def page(h, w, seed, ch):
    img = synth.page(h, w, seed, synth.STAINS if ch == 3 else synth.DOC, ch)
    img[h // 3:h // 3 + 20, w // 4:w // 4 + 60] = 140  # flat patch: ties of the definition
    return img


@pytest.mark.parametrize("gs", GS)
@pytest.mark.parametrize("W,ch,rule", [(3, 1, "sauvola"), (4, 3, "niblack"), (31, 3, "sauvola"),
                                       (62, 1, "niblack"), (101, 3, "sauvola")])
def test_matches_oracle(bnz, gs, W, ch, rule):
    check(bnz, page(300, 1100, 10 * gs + W, ch), W, gs, rule)


@pytest.mark.parametrize("gs", [1, 4, 5, 6])
def test_max_window(bnz, gs):
    check(bnz, page(520, 700, 77 + gs, 3), 255, gs)


@pytest.mark.parametrize("h,w", [(1, 1), (1, 300), (300, 1), (5, 7), (40, 257), (257, 40)])
@pytest.mark.parametrize("gs", [3, 5, 6])
def test_degenerate_sizes(bnz, h, w, gs):
    img = synth.page(h, w, h * 1000 + w, synth.DOC, 1)
    check(bnz, img, 101, gs)
    check(bnz, img, 5, gs, "niblack")


@pytest.mark.parametrize("gs", [2, 5])
@pytest.mark.parametrize("rule,k,R", [("sauvola", 20.0, 128.0), ("sauvola", 0.5, 1e-3), ("sauvola", -3.0, 2.0),
                                      ("niblack", 1e6, 1.0), ("niblack", -150.0, 1.0)])
def test_extreme_parameters(bnz, gs, rule, k, R):
    """Wide fp32 margins: many pixels take the exact path, the masks must stay the oracle's."""
    check(bnz, page(256, 600, 5, 3), 15, gs, rule, k, R)


def test_constant_page(bnz):
    img = np.full((300, 700), 93, np.uint8)
    for gs in GS:
        got, st = run(bnz, img, 31, gs, "sauvola", 0.5, 128.0)
        assert (got == 255).all() and st[1] == 0


def test_full_page_sampled_bands(bnz):
    """4096^2 RGB, the launch shape of the bench: bands at the top, across segment boundaries and at the bottom
    equal the oracle's rows (computed on the band that holds their windows)."""
    img = synth.page(4096, 4096, 21, synth.STAINS, 3)
    for gs, W in ((3, 61), (5, 101), (2, 15)):
        got, _ = run(bnz, img, W, gs, "sauvola", 0.5, 128.0)
        for y0, y1 in ((0, 24), (1000, 1090), (2040, 2080), (4070, 4096)):
            ref = oracle.gs_binarize_rows(img, W, gs, oracle.SAUVOLA, 0.5, 128.0, y0, y1)
            assert np.array_equal(got[y0:y1], ref), (gs, W, y0, int((got[y0:y1] != ref).sum()))


def test_confusion_counts(bnz):
    img, gt = synth.page(700, 900, 3, synth.STAINS, 3, ground_truth=True)
    ref_mask, _ = oracle.gs_binarize(img, 31, 3, oracle.SAUVOLA, 0.5, 128.0)
    exact, _ = oracle.binarize(img, 31, oracle.SAUVOLA, 0.5, 128.0, threads=os.cpu_count() or 4)
    d_mask = bnz.to_device_pitched(ref_mask)
    fm, rec, prec, counts = bnz.fmeasure(d_mask, bnz.to_device_pitched(gt), 0, 1)
    want = oracle.confusion(ref_mask, gt, 0, 1)
    assert counts == want
    assert (fm, rec, prec) == oracle.fmeasure(want)
    fm2, _, _, counts2 = bnz.fmeasure(d_mask, bnz.to_device_pitched(exact), 0, 0)
    assert counts2 == oracle.confusion(ref_mask, exact, 0, 0)
    assert 0.0 < fm2 <= 1.0


def test_unaligned_crop(bnz):
    """Any source alignment and pitch: a crop at an odd offset of a larger RGB canvas."""
    canvas = synth.page(400, 900, 8, synth.STAINS, 3)
    d = torch.from_numpy(canvas).cuda()
    crop = d[7:307, 13:613]
    ref, ties = oracle.gs_binarize(np.ascontiguousarray(canvas[7:307, 13:613]), 25, 5, oracle.SAUVOLA, 0.5, 128.0)
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = bnz.gs_binarize(crop, 25, 5, "sauvola", 0.5, 128.0, d_stats=st)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref) and st[1].item() == ties
