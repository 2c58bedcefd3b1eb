"""GPU parity of the global threshold (Eq. 2 with Otsu's T): the histogram,
T and the mask equal the CPU oracle's exactly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bnz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1210_3165_gb300 as b
    b.load()
    return b


def check_otsu(bnz, img, packed=False):
    ref, T_ref = oracle.otsu(img, packed=packed)
    d = bnz.to_device_pitched(img)
    out, T, hist = bnz.otsu(d, packed=packed)
    torch.cuda.synchronize()
    assert int(T.item()) == T_ref
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), oracle.histogram(img))
    got = out.cpu().numpy()
    assert np.array_equal(got, ref), f"{int(np.sum(got != ref))} mismatches (T={T_ref})"
    return T_ref


def test_config_512_gray(bnz):
    assert 0 < check_otsu(bnz, synth.page(512, 512, 1)) < 256


def test_4096_rgb_page(bnz):
    check_otsu(bnz, synth.page(4096, 4096, 2, synth.STAINS, 3))


@pytest.mark.parametrize("h,w,ch", [(1, 1, 1), (1, 1, 3), (7, 300, 3), (300, 7, 1), (333, 1111, 3),
                                    (517, 1029, 1), (129, 2049, 3)])
def test_small_and_ragged(bnz, h, w, ch):
    check_otsu(bnz, synth.page(h, w, 5 + h + w, synth.STAINS if ch == 3 else synth.DOC, ch))


@pytest.mark.parametrize("packed", [False, True])
def test_packed(bnz, packed):
    check_otsu(bnz, synth.page(700, 901, 23, synth.STAINS, 3), packed=packed)


def test_one_level_and_two_levels(bnz):
    assert check_otsu(bnz, np.full((64, 80), 77, np.uint8)) == 0
    img = np.full((64, 80), 30, np.uint8)
    img[:, 33:] = 220
    assert check_otsu(bnz, img) == 31


def test_16384_gray_full(bnz):
    # 2^28 pixels, the largest page the call takes
    check_otsu(bnz, synth.page(16384, 16384, 3, synth.VIGNETTE, 1))


def test_too_many_pixels_rejected(bnz):
    d = torch.zeros((16385, 16384), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(d)
    scratch = torch.zeros(bnz.BNZ_OTSU_SCRATCH_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="2\\^28"):
        bnz.bnz_otsu_dev(d, out, scratch)
