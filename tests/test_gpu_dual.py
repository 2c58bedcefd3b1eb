"""GPU parity of the two-rule kernel: one pass over the window sums, the
Sauvola (Eq. 4) and the Niblack mask, each equal bit for bit to the CPU
oracle's, with each rule's ties counted in its own counter."""
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


def check_dual(bnz, img, W, ks=0.5, R=128.0, kn=-0.2, packed=False):
    ref_s, ties_s = oracle.binarize(img, W, oracle.SAUVOLA, ks, R, threads=NTHREADS, packed=packed)
    ref_n, ties_n = oracle.binarize(img, W, oracle.NIBLACK, kn, 128.0, threads=NTHREADS, packed=packed)
    d = bnz.to_device_pitched(img)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    out_s, out_n = bnz.binarize_dual(d, W, ks, R, kn, packed=packed, d_stats=stats)
    torch.cuda.synchronize()
    st = stats.cpu().numpy()
    assert st[2] == 0, "device wait timed out"
    for name, got, ref in (("sauvola", out_s.cpu().numpy(), ref_s), ("niblack", out_n.cpu().numpy(), ref_n)):
        if not np.array_equal(got, ref):
            bad = np.argwhere(got != ref)
            raise AssertionError(f"{name}: {len(bad)} mismatches (W={W} packed={packed}), first at {bad[0]}")
    assert st[1] == ties_s and st[3] == ties_n


def test_config_512_gray(bnz):
    check_dual(bnz, synth.page(512, 512, 1), 15)


@pytest.mark.parametrize("W", [15, 31, 61, 101])
def test_4096_rgb_crop_all_windows(bnz, W):
    # the page workload's rule pair at each of its windows, on a 1024-row crop
    img = synth.page(4096, 4096, 2, synth.STAINS, 3)[:1024]
    check_dual(bnz, np.ascontiguousarray(img), W)


@pytest.mark.parametrize("h,w,ch,W", [(1, 1, 1, 1), (7, 300, 3, 5), (300, 7, 1, 9), (333, 1111, 3, 21),
                                      (517, 1029, 1, 4), (600, 700, 1, 255), (129, 2049, 3, 45)])
def test_small_ragged_even_and_large_windows(bnz, h, w, ch, W):
    img = synth.page(h, w, 7 + h + w, synth.STAINS if ch == 3 else synth.DOC, ch)
    check_dual(bnz, img, W)


@pytest.mark.parametrize("packed", [False, True])
def test_packed_and_other_parameters(bnz, packed):
    img = synth.page(700, 900, 23, synth.STAINS, 3)
    check_dual(bnz, img, 31, ks=0.2, R=64.0, kn=0.3, packed=packed)


def test_constant_page_ties(bnz):
    # s = 0 everywhere: Sauvola t = c (1 - k), Niblack t = c; with k_niblack = 0 every pixel is a tie there
    img = np.full((300, 520), 100, np.uint8)
    check_dual(bnz, img, 15, ks=0.0, kn=0.0)


def test_same_as_single_rule_kernels(bnz):
    img = synth.page(1000, 1300, 31, synth.STAINS, 3)
    d = bnz.to_device_pitched(img)
    out_s, out_n = bnz.binarize_dual(d, 45, 0.4, 100.0, -0.3)
    one_s = bnz.binarize(d, 45, "sauvola", 0.4, 100.0)
    one_n = bnz.binarize(d, 45, "niblack", -0.3)
    torch.cuda.synchronize()
    assert torch.equal(out_s, one_s) and torch.equal(out_n, one_n)


def test_overlapping_masks_rejected(bnz):
    img = synth.page(64, 64, 1)
    d = bnz.to_device_pitched(img)
    out = bnz.alloc_pitched(64, 64, d.device)
    with pytest.raises(RuntimeError, match="overlap"):
        bnz.bnz_dual_dev(d, 15, 0.5, 128.0, -0.2, out, out)
