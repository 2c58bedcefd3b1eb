"""Every output equals the fp64 decision of the definition for every accepted
threshold parameter, not only for the usual ones: Sauvola with a small R
(large k/R) or a large |k|, Niblack with a large |k|.  There the fp32 margin
and the double-float stage's error bound grow with |k| and k/R, so more
pixels take the exact path; the masks and the tie counts must still equal the
oracle's.  Run through the fused kernel, the two-rule kernel and the
integral-image path on a page of more than a megapixel that also holds flat
patches (ties of the definition)."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NTHREADS = os.cpu_count() or 4

SAUVOLA_PARAMS = [(0.5, 2.0), (0.5, 0.5), (20.0, 128.0), (-3.0, 128.0), (0.5, 1e-3), (1e6, 1e-6)]
NIBLACK_PARAMS = [-150.0, 50.0, 1e6]


@pytest.fixture(scope="module")
def bnz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1210_3165_gb300 as b
    b.load()
    return b


@pytest.fixture(scope="module")
def page():
    img = synth.page(1024, 1100, 31, synth.STAINS, 3)
    img[100:180, 200:420] = 77           # flat patches: s = 0 there, t a multiple of m
    img[600:700, 50:300] = (10, 200, 90)
    return img


def stats_tensor():
    return torch.zeros(4, dtype=torch.int64, device="cuda")


def assert_same(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {tuple(bad[0])}")


@pytest.mark.parametrize("k,R", SAUVOLA_PARAMS)
def test_sauvola_fused(bnz, page, k, R):
    ref, ties = oracle.binarize(page, 31, oracle.SAUVOLA, k, R, threads=NTHREADS)
    st = stats_tensor()
    got = bnz.binarize(bnz.to_device_pitched(page), 31, "sauvola", k, R, d_stats=st).cpu().numpy()
    s = st.cpu().numpy()
    assert_same(got, ref, f"sauvola k={k} R={R}")
    assert s[2] == 0 and s[1] == ties


@pytest.mark.parametrize("k", NIBLACK_PARAMS)
def test_niblack_fused(bnz, page, k):
    ref, ties = oracle.binarize(page, 31, oracle.NIBLACK, k, 128.0, threads=NTHREADS)
    st = stats_tensor()
    got = bnz.binarize(bnz.to_device_pitched(page), 31, "niblack", k, d_stats=st).cpu().numpy()
    s = st.cpu().numpy()
    assert_same(got, ref, f"niblack k={k}")
    assert s[2] == 0 and s[1] == ties


@pytest.mark.parametrize("ks,R,kn", [(0.5, 0.5, -150.0), (20.0, 128.0, 50.0), (-3.0, 2.0, 1e6)])
def test_dual(bnz, page, ks, R, kn):
    ref_s, ties_s = oracle.binarize(page, 15, oracle.SAUVOLA, ks, R, threads=NTHREADS)
    ref_n, ties_n = oracle.binarize(page, 15, oracle.NIBLACK, kn, 128.0, threads=NTHREADS)
    st = stats_tensor()
    out_s, out_n = bnz.binarize_dual(bnz.to_device_pitched(page), 15, ks, R, kn, d_stats=st)
    s = st.cpu().numpy()
    assert_same(out_s.cpu().numpy(), ref_s, "dual sauvola")
    assert_same(out_n.cpu().numpy(), ref_n, "dual niblack")
    assert s[2] == 0 and s[1] == ties_s and s[3] == ties_n


@pytest.mark.parametrize("rule,k,R", [("sauvola", 0.5, 0.5), ("sauvola", 20.0, 128.0), ("niblack", -150.0, 1.0)])
def test_integral(bnz, page, rule, k, R):
    rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
    ref, ties = oracle.binarize(page, 61, rid, k, R, threads=NTHREADS)
    h, w = page.shape[:2]
    scratch = bnz.alloc_scratch(bnz.bnz_integral_scratch_bytes(h, w))
    out = bnz.alloc_pitched(h, w)
    st = stats_tensor()
    bid = bnz.BNZ_SAUVOLA if rule == "sauvola" else bnz.BNZ_NIBLACK
    bnz.bnz_binarize_integral_dev(bnz.to_device_pitched(page), 61, bid, k, R, out, scratch, d_stats=st)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert_same(out.cpu().numpy(), ref, f"integral {rule} k={k} R={R}")
    assert s[1] == ties


def test_many_pixels_take_the_exact_path(bnz, page):
    """With k/R = 1000 the fp32 margin is wide: the exact path runs for a large share of the page, and the
    result is still the oracle's (this is where a sign decided on too small a margin would show)."""
    ref, ties = oracle.binarize(page, 15, oracle.SAUVOLA, 0.5, 5e-4, threads=NTHREADS)
    st = stats_tensor()
    got = bnz.binarize(bnz.to_device_pitched(page), 15, "sauvola", 0.5, 5e-4, d_stats=st).cpu().numpy()
    s = st.cpu().numpy()
    assert_same(got, ref, "sauvola k/R=1000")
    assert s[1] == ties and s[0] > page.shape[0] * page.shape[1] // 100


@pytest.mark.parametrize("k", [-0.2, -0.5, 0.3])
@pytest.mark.parametrize("W", [15, 61])
def test_niblack_margin_pixels(bnz, k, W):
    """The usual Niblack settings leave a few pixels in 10^5 inside the fp32 margin; those take the tighter
    fp32 evaluation of n (f - t), then the double-float and fp64 stages, in the fused kernel (the interior
    margin for warps whose windows lie inside the page, the general one at the borders) and in the
    two-rule kernel.  Masks and tie counts equal the oracle's, and the margin path did run."""
    img = synth.page(1200, 1300, 7 + W, synth.STAINS, 3)
    img[300:340, 400:700] = 140           # a flat patch: ties of the definition
    ref, ties = oracle.binarize(img, W, oracle.NIBLACK, k, 1.0, threads=NTHREADS)
    st = stats_tensor()
    d = bnz.to_device_pitched(img)
    got = bnz.binarize(d, W, "niblack", k, d_stats=st).cpu().numpy()
    s = st.cpu().numpy()
    assert_same(got, ref, f"niblack W={W} k={k}")
    assert s[1] == ties and s[2] == 0 and s[0] > 0
    ref_s, _ = oracle.binarize(img, W, oracle.SAUVOLA, 0.5, 128.0, threads=NTHREADS)
    st2 = stats_tensor()
    out_s, out_n = bnz.binarize_dual(d, W, 0.5, 128.0, k, d_stats=st2)
    assert_same(out_n.cpu().numpy(), ref, f"dual niblack W={W} k={k}")
    assert_same(out_s.cpu().numpy(), ref_s, f"dual sauvola W={W}")
    assert int(st2[3].item()) == ties
