"""Integral-image comparison variant (int64 summed-area tables): tables and
masks against the CPU oracle, and masks against the fused kernel."""
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


def integral_mask(bnz, img, W, rule, k, R=128.0, packed=False):
    d = bnz.to_device_pitched(img)
    h, w = img.shape[:2]
    scratch = bnz.alloc_scratch(bnz.bnz_integral_scratch_bytes(h, w))
    out = bnz.alloc_pitched(h, (w + 7) // 8 if packed else w)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    rid = bnz.BNZ_SAUVOLA if rule == "sauvola" else bnz.BNZ_NIBLACK
    bnz.bnz_binarize_integral_dev(d, W, rid, k, R, out, scratch, packed=packed, d_stats=stats)
    torch.cuda.synchronize()
    return out.cpu().numpy(), stats.cpu().numpy()


@pytest.mark.parametrize("h,w,ch", [(1, 1, 1), (7, 300, 1), (300, 7, 3), (257, 513, 1), (600, 1100, 3)])
def test_tables_match_oracle(bnz, h, w, ch):
    img = synth.page(h, w, h * 7 + w, synth.STAINS if ch == 3 else synth.DOC, ch)
    d = bnz.to_device_pitched(img)
    scratch = bnz.alloc_scratch(bnz.bnz_integral_scratch_bytes(h, w))
    I1, I2 = bnz.bnz_integral_images_dev(d, scratch)
    torch.cuda.synchronize()
    R1, R2 = oracle.integral(oracle.gray(img))
    np.testing.assert_array_equal(I1.cpu().numpy(), R1)
    np.testing.assert_array_equal(I2.cpu().numpy(), R2)


@pytest.mark.parametrize("W", [1, 4, 15, 31, 101, 255])
@pytest.mark.parametrize("ch", [1, 3])
def test_masks_match_oracle_and_fused(bnz, W, ch):
    img = synth.page(531, 777, W * 3 + ch, synth.STAINS if ch == 3 else synth.VIGNETTE, ch)
    for rule, k in (("sauvola", 0.5), ("niblack", -0.2)):
        rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
        ref, ties = oracle.binarize(img, W, rid, k, 128.0, threads=NTHREADS)
        got, st = integral_mask(bnz, img, W, rule, k)
        np.testing.assert_array_equal(got, ref)
        assert st[1] == ties
        fused = bnz.binarize(bnz.to_device_pitched(img), W, rule, k).cpu().numpy()
        np.testing.assert_array_equal(got, fused)
    got, _ = integral_mask(bnz, img, W, "sauvola", 0.5, packed=True)
    np.testing.assert_array_equal(got, oracle.pack(oracle.sauvola(img, W, threads=NTHREADS)[0]))


def test_config_16384_gray_w101_int64(bnz):
    """Sums of f over the page exceed 2^32: the tables must be int64."""
    img = synth.page(16384, 16384, 3, synth.VIGNETTE, 1)
    ref, ties = oracle.binarize(img, 101, oracle.SAUVOLA, 0.34, 128.0, threads=NTHREADS)
    got, st = integral_mask(bnz, img, 101, "sauvola", 0.34)
    np.testing.assert_array_equal(got, ref)
    assert st[1] == ties


def test_scratch_too_small_rejected(bnz):
    img = synth.page(64, 64, 1)
    d = bnz.to_device_pitched(img)
    out = bnz.alloc_pitched(64, 64)
    small = bnz.alloc_scratch(bnz.bnz_integral_scratch_bytes(64, 64) - 64)
    with pytest.raises(bnz.BnzError) as e:
        bnz.bnz_binarize_integral_dev(d, 15, bnz.BNZ_SAUVOLA, 0.5, 128.0, out, small)
    assert e.value.status == bnz.BNZ_EINVAL
