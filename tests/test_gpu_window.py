"""Out-of-core binarization (bnz_binarize_window): a host page streams through
a small device window of row bands with read-only halos; the mask must equal
the oracle's bit for bit whatever the band height, including bands shorter
than the halo, even W, both rules and gray or RGB."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NTHREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def bnz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1210_3165_gb300 as b
    b.load()
    return b


def slot_bytes(B, W, w, ch):
    sp = (w * ch + 15) // 16 * 16
    dp = (w + 15) // 16 * 16
    return (B + W - 1) * sp + (B + W // 2) * dp


@pytest.mark.parametrize("h,w,ch,W,rule,k,B", [
    (3000, 1800, 3, 31, "sauvola", 0.5, 100),    # 30 bands
    (2500, 700, 1, 101, "niblack", -0.2, 8),     # bands of 8 rows under a 100-row halo
    (1200, 999, 3, 20, "sauvola", 0.34, 57),     # even W (the paper's 20 x 20), ragged last band
    (777, 1500, 1, 15, "sauvola", 0.5, 5000),    # window larger than the page: one band
])
def test_window_matches_oracle(bnz, h, w, ch, W, rule, k, B):
    img = synth.page(h, w, h + w + W, synth.STAINS if ch == 3 else synth.DOC, ch)
    rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
    ref, _ = oracle.binarize(img, W, rid, k, 128.0, threads=NTHREADS)
    got = bnz.binarize_window(img, W, rule, k, 128.0, window_bytes=3 * slot_bytes(min(B, h), W, w, ch))
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError(f"{len(bad)} mismatches, first at {tuple(bad[0])}")


def test_window_equals_host_call(bnz):
    img = synth.page(2048, 1024, 5, synth.STAINS, 3)
    a = bnz.binarize_window(img, 61, "sauvola", 0.5, 128.0, window_bytes=3 * slot_bytes(64, 61, 1024, 3))
    b = bnz.bnz_sauvola(img, 61, 0.5, 128.0)
    assert np.array_equal(a, b)


def test_window_too_small(bnz):
    img = synth.page(100, 100, 1, synth.DOC, 1)
    with pytest.raises(bnz.BnzError, match="too small"):
        bnz.binarize_window(img, 31, window_bytes=3 * slot_bytes(7, 31, 100, 1))


def test_large_page_host_call_streams_through_slots(bnz):
    """A page of 256 MiB or more (with its mask) goes through the band slots in bnz_sauvola: oracle-exact."""
    img = synth.page(16384, 8192, 3, synth.VIGNETTE, 1)    # 128 MiB page + 128 MiB mask
    ref, _ = oracle.binarize(img, 101, oracle.SAUVOLA, 0.34, 128.0, threads=NTHREADS)
    got = bnz.bnz_sauvola(img, 101, 0.34, 128.0)
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError(f"{len(bad)} mismatches, first at {tuple(bad[0])}")
