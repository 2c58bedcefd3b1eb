"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element
by element, on seeded synthetic pages.  Window sums are exact integers, so
the masks must match bit for bit; tie counts must match the oracle's."""
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


def run_gpu(bnz, img, W, rule, k, R=128.0, packed=False, tile=None):
    d = bnz.to_device_pitched(img)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = bnz.binarize(d, W, rule, k, R, packed=packed, tile=tile, d_stats=stats)
    torch.cuda.synchronize()
    st = stats.cpu().numpy()
    assert st[2] == 0, "device wait timed out"
    return out.cpu().numpy(), int(st[0]), int(st[1])


def check(bnz, img, W, rule, k, R=128.0, packed=False, tile=None):
    rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
    ref, ties = oracle.binarize(img, W, rid, k, R, threads=NTHREADS, packed=packed)
    got, nfb, nties = run_gpu(bnz, img, W, rule, k, R, packed, tile)
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        y, x = bad[0]
        raise AssertionError(f"{len(bad)} mismatches (W={W} {rule} packed={packed}); first at {y},{x}: "
                             f"gpu={got[y, x]} oracle={ref[y, x]}")
    assert nties == ties
    return nfb


def test_config_512_gray_sauvola(bnz):
    img = synth.page(512, 512, 1)
    check(bnz, img, 15, "sauvola", 0.5)


SHAPES = [(1, 1), (1, 37), (37, 1), (5, 7), (17, 300), (300, 17), (129, 257), (263, 531)]


@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("ch", [1, 3])
def test_small_and_ragged_shapes(bnz, h, w, ch):
    rng = np.random.default_rng(h * 1000 + w + ch)
    img = synth.page(h, w, h + w, synth.STAINS if ch == 3 else synth.DOC, ch)
    for W in (1, 2, 3, 8, 15, 64, 101):
        rule = "sauvola" if rng.random() < 0.5 else "niblack"
        k = 0.5 if rule == "sauvola" else -0.2
        check(bnz, img, W, rule, k, packed=bool(rng.random() < 0.3))


@pytest.mark.parametrize("W", [15, 31, 61, 101])
@pytest.mark.parametrize("ch", [1, 3])
def test_multi_tile_ragged_tail(bnz, W, ch):
    img = synth.page(1031, 2063, 77 + W, synth.STAINS if ch == 3 else synth.VIGNETTE, ch)
    check(bnz, img, W, "sauvola", 0.5)
    check(bnz, img, W, "niblack", -0.2, packed=True)


@pytest.mark.parametrize("W", [15, 31, 61, 101])
def test_config_4096_rgb_full(bnz, W):
    img = synth.page(4096, 4096, 2, synth.STAINS, 3)
    check(bnz, img, W, "sauvola", 0.5)
    check(bnz, img, W, "niblack", -0.2)


def test_config_16384_gray_w101_full(bnz):
    img = synth.page(16384, 16384, 3, synth.VIGNETTE, 1)
    nfb = check(bnz, img, 101, "sauvola", 0.34)
    assert nfb < img.size * 1e-3


def test_large_and_even_windows(bnz):
    img = synth.page(700, 900, 5, synth.DOC, 1)
    for W in (128, 200, 254, 255):
        check(bnz, img, W, "sauvola", 0.5)
    rgb = synth.page(300, 1100, 6, synth.STAINS, 3)
    check(bnz, rgb, 255, "niblack", -0.2, packed=True)


def test_window_larger_than_image(bnz):
    img = synth.page(40, 60, 8)
    for W in (81, 121, 255):
        check(bnz, img, W, "sauvola", 0.5)
        check(bnz, img, W, "niblack", 0.3)


def test_constant_image_ties(bnz):
    for c in (0, 77, 255):
        img = np.full((300, 700), c, np.uint8)
        got, _, nties = run_gpu(bnz, img, 31, "niblack", -0.2)
        assert (got == 255).all() and nties == img.size     # t = c exactly: every pixel a tie
        got, _, nties = run_gpu(bnz, img, 31, "sauvola", 0.5)
        assert (got == 255).all() and nties == (img.size if c == 0 else 0)


def test_other_parameters(bnz):
    img = synth.page(613, 811, 9, synth.STAINS, 3)
    for k, R in ((0.0, 128.0), (0.2, 64.0), (0.9, 255.0), (1.5, 30.0), (-0.3, 128.0)):
        check(bnz, img, 25, "sauvola", k, R)
    for k in (0.0, -1.0, 0.7):
        check(bnz, img, 25, "niblack", k)


def test_explicit_tile_shapes_agree(bnz):
    img = synth.page(900, 1500, 10, synth.DOC, 1)
    for tw in (0, 128, 256, 512):
        for chunk in (0, 8):
            for th in (0, 7, 50):
                tile = bnz.bnz_tile(tw, th, chunk, 0)
                check(bnz, img, 45, "sauvola", 0.5, tile=tile)


def test_host_pointer_api(bnz):
    img = synth.page(333, 444, 11, synth.STAINS, 3)
    ref, _ = oracle.sauvola(img, 21, 0.5, 128.0)
    np.testing.assert_array_equal(bnz.bnz_sauvola(img, 21, 0.5, 128.0), ref)
    ref, _ = oracle.niblack(img, 21, -0.2)
    np.testing.assert_array_equal(bnz.bnz_niblack(img, 21, -0.2), ref)


@pytest.mark.parametrize("h,w,ch,W,rule", [
    (1030, 1100, 3, 101, "sauvola"),   # bands of 515, 258, 257 rows; windows reach 50 rows past each
    (1031, 1024, 1, 15, "niblack"),    # 516, 258, 129, 128: odd heights
    (2050, 700, 1, 61, "sauvola"),     # 1025, 513, 256, 256: narrow page (2 strips)
    (1300, 1000, 3, 4, "niblack"),     # 650, 325, 163, 162: even window (r_lo = 2, r_hi = 1)
    (1100, 1000, 1, 255, "sauvola"),   # 550, 550: the largest window, 127 rows past each band
])
def test_host_pointer_api_row_bands(bnz, h, w, ch, W, rule):
    # pages of a megapixel and more go through the host API in row bands, each band's
    # upload, kernel and download on their own streams
    assert len(bnz.host_bands(h, w, W)) > 2                       # the case really runs in bands
    img = synth.page(h, w, 17, synth.STAINS if ch == 3 else synth.DOC, ch)
    if rule == "sauvola":
        ref, _ = oracle.sauvola(img, W, 0.5, 128.0, threads=NTHREADS)
        got = bnz.bnz_sauvola(img, W, 0.5, 128.0)
    else:
        ref, _ = oracle.niblack(img, W, -0.2, threads=NTHREADS)
        got = bnz.bnz_niblack(img, W, -0.2)
    assert not np.any(got != ref), f"{int(np.sum(got != ref))} mismatches"
    # twice in a row: the second call reuses the buffers, streams and events
    again = bnz.bnz_sauvola(img, W, 0.5, 128.0) if rule == "sauvola" else bnz.bnz_niblack(img, W, -0.2)
    np.testing.assert_array_equal(again, ref)


def test_unaligned_pitch_rejected(bnz):
    t = torch.zeros((10, 33), dtype=torch.uint8, device="cuda")[:, :30]   # pitch 33
    out = torch.zeros((10, 30), dtype=torch.uint8, device="cuda")
    with pytest.raises(bnz.BnzError) as e:
        bnz.bnz_sauvola_dev(t, 5, 0.5, 128.0, out)
    assert e.value.status == bnz.BNZ_EINVAL


def test_stream_async_and_repeatable(bnz):
    img = synth.page(1200, 1600, 12, synth.DOC, 1)
    d = bnz.to_device_pitched(img)
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for _ in range(3):
            outs.append(bnz.binarize(d, 31, "sauvola", 0.5, stream=s))
    s.synchronize()
    ref, _ = oracle.sauvola(img, 31, threads=NTHREADS)
    for o in outs:
        np.testing.assert_array_equal(o.cpu().numpy(), ref)


def test_sqrt_approx_error_within_margin_assumption(bnz):
    """The fp32 margin assumes sqrt.approx.f32 has relative error <= 2^-21 on [1, 2^48): V = n*S2 - S1^2
    stays below n^2 * 127.5^2 < 2^46 for W <= 255."""
    import ctypes
    err = ctypes.c_double(0.0)
    rc = bnz.load().bnz_selftest_sqrt_approx(1.0, float(2 ** 48), ctypes.byref(err))
    assert rc == 0, bnz.bnz_last_error()
    assert 0.0 < err.value <= 2.0 ** -21, err.value


def test_rcp_approx_error_within_margin_assumption(bnz):
    """Clipped windows use rcp.approx.f32 for 1/n; the margin assumes <= 2^-22 on n = 1..65025."""
    import ctypes
    err = ctypes.c_double(0.0)
    rc = bnz.load().bnz_selftest_rcp_approx(1, 65026, ctypes.byref(err))
    assert rc == 0, bnz.bnz_last_error()
    assert 0.0 < err.value <= 2.0 ** -22, err.value


def test_bounded_wait_gives_up_and_context_stays_usable(bnz):
    """A wait on a barrier phase that nothing completes gives up after its limit and reports it; the
    context then still runs the fused kernel correctly.  (The failure is made by never arriving: no
    trap, no bad address, no endless loop.)"""
    import ctypes
    lib = bnz.load()
    limit = 2_000_000  # SM cycles, about 1 ms
    to, cyc = ctypes.c_int(-1), ctypes.c_longlong(-1)
    rc = lib.bnz_selftest_wait_timeout(limit, 0, ctypes.byref(to), ctypes.byref(cyc))
    assert rc == 0, bnz.bnz_last_error()
    assert to.value == 1
    assert limit < cyc.value < limit + 1_000_000  # gives up soon after the limit (suspends <= 20 us per try)
    rc = lib.bnz_selftest_wait_timeout(limit, 1, ctypes.byref(to), ctypes.byref(cyc))
    assert rc == 0 and to.value == 0 and 0 <= cyc.value < limit
    img = synth.page(300, 257, 21, synth.DOC, 1)
    check(bnz, img, 15, "sauvola", 0.5)


def test_gray_conversion_exhaustive(bnz):
    """Eq. 1 as the fused kernel's producers compute it (byte dot products and a multiply-high by the
    reciprocal of 1000), over every one of the 2^24 (r, g, b) triples, equals the oracle's integer rule;
    a ragged tail of 3 pixels goes through the one-pixel form."""
    import ctypes
    i = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(i >> 16) & 255, (i >> 8) & 255, i & 255], axis=-1).astype(np.uint8).reshape(4096, 4096, 3)
    ref = oracle.gray(rgb).reshape(-1)
    d_rgb = torch.from_numpy(rgb.reshape(-1)).cuda()
    for npix in (1 << 24, (1 << 24) - 1):
        d_gray = torch.zeros(npix, dtype=torch.uint8, device="cuda")
        rc = bnz.load().bnz_selftest_gray(ctypes.c_void_p(d_rgb.data_ptr()), npix, ctypes.c_void_p(d_gray.data_ptr()),
                                          None)
        assert rc == 0, bnz.bnz_last_error()
        torch.cuda.synchronize()
        got = d_gray.cpu().numpy()
        bad = np.flatnonzero(got != ref[:npix])
        assert bad.size == 0, f"{bad.size} triples differ, first {rgb.reshape(-1, 3)[bad[0]]}"


@pytest.mark.parametrize("ch,W,rule", [(3, 31, "sauvola"), (1, 101, "niblack")])
def test_fused_kernel_abort_path(bnz, ch, W, rule):
    """The fused kernel's own waits made to give up (self-test entry: a wait gives up unless its copy has
    already landed, while the final drain of copies in flight keeps its normal limit): the call reports
    BNZ_ETIMEOUT and the timed-out CTAs in the counters; the context stays usable, and the next normal launch on
    the same buffers is bit-exact.  Nothing traps, faults or waits forever."""
    import ctypes
    img = synth.page(1500, 2100, 41, synth.STAINS if ch == 3 else synth.DOC, ch)
    d = bnz.to_device_pitched(img)
    out = bnz.alloc_pitched(img.shape[0], img.shape[1])
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    k = 0.5 if rule == "sauvola" else -0.2
    rid = bnz.BNZ_SAUVOLA if rule == "sauvola" else bnz.BNZ_NIBLACK
    s = torch.cuda.current_stream()
    rc = bnz.load().bnz_selftest_fused_timeout(d.data_ptr(), d.stride(0), img.shape[0], img.shape[1], ch, W, rid,
                                               k, 128.0, out.data_ptr(), out.stride(0), ctypes.c_void_p(s.cuda_stream),
                                               stats.data_ptr())
    assert rc == bnz.BNZ_ETIMEOUT, (rc, bnz.bnz_last_error())
    assert int(stats[2]) > 0
    check(bnz, img, W, rule, k)


@pytest.mark.parametrize("h,w,ch", [(2050, 1100, 3), (700, 900, 1)])
def test_host_one_page_several_settings(bnz, h, w, ch):
    """bnz_binarize_runs: one upload of the page, every setting's mask equal to the oracle's (and to the
    one-setting host calls); the larger page goes in row bands."""
    img = synth.page(h, w, 61, synth.STAINS if ch == 3 else synth.DOC, ch)
    runs = [(15, "sauvola", 0.5, 128.0), (101, "niblack", -0.2, 128.0), (31, "sauvola", 0.3, 64.0),
            (4, "niblack", 0.1, 1.0)]
    masks = bnz.binarize_runs(img, runs)
    for (W, rule, k, R), got in zip(runs, masks):
        rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
        ref, _ = oracle.binarize(img, W, rid, k, R, threads=NTHREADS)
        assert not np.any(got != ref), f"{rule} W={W}: {int(np.sum(got != ref))} mismatches"
    again = bnz.binarize_runs(img, runs[:1])
    np.testing.assert_array_equal(again[0], masks[0])


@pytest.mark.parametrize("ew", [16, 24, 40])
@pytest.mark.parametrize("w", [1100, 1500, 2200])
def test_edge_weight_split(bnz, ew, w):
    """Whole CTAs per strip, the edge strips weighted: every split covers every row once (oracle-exact)."""
    img = synth.page(700, w, ew + w, synth.STAINS, 3)
    ref, _ = oracle.binarize(img, 31, oracle.SAUVOLA, 0.5, 128.0, threads=os.cpu_count() or 4)
    for tile in (bnz.bnz_tile(0, 0, 0, ew), bnz.bnz_tile(256, 40, 0, ew)):
        got = bnz.binarize(bnz.to_device_pitched(img), 31, "sauvola", 0.5, 128.0, tile=tile).cpu().numpy()
        assert np.array_equal(got, ref)
