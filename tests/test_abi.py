"""The C ABI library loads, exports every function include/bnz.h declares, and
rejects bad arguments / reports a missing GPU without computing anything (CPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1210_3165_gb300 as bnz
from paper_1210_3165_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bnz_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return bnz.load()


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "bnz_sauvola" in names and "bnz_niblack" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string(lib):
    assert bnz.bnz_version() >= 100
    assert isinstance(bnz.bnz_last_error(), str)


@pytest.mark.parametrize("args,fragment", [
    (dict(W=0), "window size"),
    (dict(W=256), "window size"),
    (dict(R=0.0), "R must be"),
    (dict(k=float("nan")), "k must be finite"),
    (dict(k=1.0e6 * (1 + 1e-12)), "|k| <="),      # past the range where every constant stays finite
    (dict(k=-2.0e6), "|k| <="),
    (dict(R=0.9e-6), "R must be"),
    (dict(channels=2), "channels"),
    (dict(h=0), "height and width"),
])
def test_argument_errors(lib, args, fragment):
    a = dict(h=8, w=9, channels=1, W=3, k=0.5, R=128.0)
    a.update(args)
    src = np.zeros(max(a["h"], 1) * a["w"] * 3, np.uint8)
    dst = np.zeros(max(a["h"], 1) * a["w"], np.uint8)
    rc = lib.bnz_sauvola(src.ctypes.data, a["h"], a["w"], a["channels"], a["W"], a["k"], a["R"],
                         dst.ctypes.data)
    assert rc == bnz.BNZ_EINVAL
    assert fragment in bnz.bnz_last_error()


def test_parameter_range_limits_accepted(lib):
    """The ends of the accepted range pass the argument checks (no GPU here: the call then reports that
    there is no device, not a bad argument)."""
    src = np.zeros(64, np.uint8)
    dst = np.zeros(64, np.uint8)
    for k, R in ((1.0e6, 1.0e-6), (-1.0e6, 1.0e-6), (0.5, 1.0e300)):
        rc = lib.bnz_sauvola(src.ctypes.data, 8, 8, 1, 3, k, R, dst.ctypes.data)
        assert rc != bnz.BNZ_EINVAL, bnz.bnz_last_error()


def test_null_pointer_rejected(lib):
    rc = lib.bnz_niblack(None, 4, 4, 1, 3, -0.2, None)
    assert rc == bnz.BNZ_EINVAL


def test_no_gpu_means_no_result():
    """Without a CUDA device the library reports BNZ_ENODEV: there is no CPU path."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = bnz.load()
    src = np.full((16, 16), 100, np.uint8)
    dst = np.zeros((16, 16), np.uint8)
    rc = lib.bnz_sauvola(src.ctypes.data, 16, 16, 1, 5, 0.5, 128.0, dst.ctypes.data)
    assert rc == bnz.BNZ_ENODEV
    assert (dst == 0).all()
    with pytest.raises(bnz.BnzError):
        bnz.bnz_sauvola(src, 5)


def test_native_server_needs_a_device_and_checks_its_config():
    import ctypes
    import torch
    lib = bnz.load()
    h = ctypes.c_void_p(None)
    bad = bnz.bnz_server_config(1 << 10, 16, 2, 1, 0)  # budget below 1 MiB
    assert lib.bnz_server_create(ctypes.byref(bad), ctypes.byref(h)) == bnz.BNZ_EINVAL and not h.value
    bad = bnz.bnz_server_config(1 << 30, 16, 9, 1, 0)  # too many compute streams
    assert lib.bnz_server_create(ctypes.byref(bad), ctypes.byref(h)) == bnz.BNZ_EINVAL
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ok = bnz.bnz_server_config(1 << 30, 16, 2, 1, 0)
    assert lib.bnz_server_create(ctypes.byref(ok), ctypes.byref(h)) == bnz.BNZ_ENODEV and not h.value


def _aligned(buf):
    return (buf.ctypes.data + 15) & ~15


def test_dual_and_otsu_argument_checks(lib):
    # the checks run before any device work, so host addresses stand in for device buffers
    buf = np.zeros(8192, np.uint8)
    a = _aligned(buf)
    nan = float("nan")
    rc = lib.bnz_dual_dev(a, 16, 8, 16, 1, 5, 0.5, 128.0, -0.2, a + 1024, a + 1024 + 8, 16, 0, None, None)
    assert rc == bnz.BNZ_EINVAL and "overlap" in bnz.bnz_last_error()
    rc = lib.bnz_dual_dev(a, 16, 8, 16, 1, 5, 0.5, 128.0, nan, a + 1024, a + 2048, 16, 0, None, None)
    assert rc == bnz.BNZ_EINVAL and "k must be finite" in bnz.bnz_last_error()
    rc = lib.bnz_dual_dev(a, 16, 8, 16, 1, 5, 0.5, 128.0, -0.2, a + 1024, None, 16, 0, None, None)
    assert rc == bnz.BNZ_EINVAL and "null" in bnz.bnz_last_error()
    rc = lib.bnz_dual_dev(a, 16, 8, 16, 1, 256, 0.5, 128.0, -0.2, a + 1024, a + 2048, 16, 0, None, None)
    assert rc == bnz.BNZ_EINVAL and "window size" in bnz.bnz_last_error()
    rc = lib.bnz_otsu_dev(a, 16384, 16385, 16384, 1, a, 16384, 0, a, None)
    assert rc == bnz.BNZ_EINVAL and "2^28" in bnz.bnz_last_error()
    rc = lib.bnz_otsu_dev(a, 16, 8, 16, 1, a + 1024, 16, 0, a + 2049, None)
    assert rc == bnz.BNZ_EINVAL and "d_scratch" in bnz.bnz_last_error()
    rc = lib.bnz_otsu_dev(a + 1, 16, 8, 16, 1, a + 1024, 16, 0, a + 2048, None)
    assert rc == bnz.BNZ_EINVAL and "16-byte aligned" in bnz.bnz_last_error()
    rc = lib.bnz_otsu_dev(a, 16, 8, 16, 2, a + 1024, 16, 0, a + 2048, None)
    assert rc == bnz.BNZ_EINVAL and "channels" in bnz.bnz_last_error()


def test_dual_and_otsu_need_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = bnz.load()
    buf = np.zeros(8192, np.uint8)
    a = _aligned(buf)
    assert lib.bnz_dual_dev(a, 16, 8, 16, 1, 5, 0.5, 128.0, -0.2, a + 1024, a + 2048, 16, 0, None,
                            None) == bnz.BNZ_ENODEV
    assert lib.bnz_otsu_dev(a, 16, 8, 16, 1, a + 1024, 16, 0, a + 2048, None) == bnz.BNZ_ENODEV
    assert (buf == 0).all()


@pytest.mark.parametrize("h,w,W", [(4096, 4096, 15), (4096, 4096, 101), (1030, 1100, 101), (1031, 1024, 15),
                                   (2050, 700, 61), (1300, 1000, 4), (1100, 1000, 255), (16384, 16384, 101),
                                   (7016, 4960, 61), (512, 512, 15), (1023, 1024, 15), (300, 5000, 15),
                                   (1, 1 << 21, 1), (1 << 21, 1, 1)])
def test_host_bands_plan(h, w, W):
    # the row bands of the host-pointer calls: host logic, checked without a device
    b = bnz.host_bands(h, w, W)
    nb = len(b) - 1
    assert b[0] == 0 and b[-1] == h and all(b[i] < b[i + 1] for i in range(nb))
    sizes = [b[i + 1] - b[i] for i in range(nb)]
    if h * w < (1 << 20):
        assert nb == 1
        return
    assert 1 <= nb <= 4
    assert all(sizes[i] >= sizes[i + 1] for i in range(nb - 1))     # halving towards the page end
    assert b[:nb] == [h - (h >> i) for i in range(nb)]
    if nb > 1:
        assert min(sizes) >= max(128, 2 * W)
    if nb < 4:                                                       # as many bands as the rule allows
        assert (h >> nb) < max(128, 2 * W)


def test_host_bands_rejects_bad_arguments():
    with pytest.raises(bnz.BnzError):
        bnz.host_bands(0, 10, 3)
    with pytest.raises(bnz.BnzError):
        bnz.host_bands(10, 10, 256)


def test_reduced_set_and_confusion_argument_checks(lib):
    buf = np.zeros(8192, np.uint8)
    a = _aligned(buf)
    rc = lib.bnz_gs_binarize_dev(a, 16, 8, 16, 1, 2, bnz.BNZ_GS_CROSS, bnz.BNZ_SAUVOLA, 0.5, 128.0, a + 1024, 16,
                                 None, None)
    assert rc == bnz.BNZ_EINVAL and "W >= 3" in bnz.bnz_last_error()
    for gs in (0, 7):
        rc = lib.bnz_gs_binarize_dev(a, 16, 8, 16, 1, 5, gs, bnz.BNZ_SAUVOLA, 0.5, 128.0, a + 1024, 16, None, None)
        assert rc == bnz.BNZ_EINVAL and "unknown structure" in bnz.bnz_last_error()
    rc = lib.bnz_gs_binarize_dev(a, 16, 8, 16, 1, 5, 1, bnz.BNZ_SAUVOLA, 0.5, 0.0, a + 1024, 16, None, None)
    assert rc == bnz.BNZ_EINVAL and "R must be" in bnz.bnz_last_error()
    rc = lib.bnz_gs_binarize_dev(a, 16, 8, 16, 1, 256, 1, bnz.BNZ_SAUVOLA, 0.5, 128.0, a + 1024, 16, None, None)
    assert rc == bnz.BNZ_EINVAL and "window size" in bnz.bnz_last_error()
    rc = lib.bnz_confusion_dev(a, 8, 0, a + 1024, 16, 1, 4, 16, a + 4096, None)
    assert rc == bnz.BNZ_EINVAL and "pitch" in bnz.bnz_last_error()
    rc = lib.bnz_confusion_dev(a, 16, 256, a + 1024, 16, 1, 4, 16, a + 4096, None)
    assert rc == bnz.BNZ_EINVAL and "ink" in bnz.bnz_last_error()
    assert lib.bnz_confusion_dev(a, 16, 0, a + 1024, 16, 1, 0, 16, a + 4096, None) == bnz.BNZ_OK  # empty: no work
    assert (buf == 0).all()


def test_reduced_set_needs_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = bnz.load()
    buf = np.zeros(8192, np.uint8)
    a = _aligned(buf)
    assert lib.bnz_gs_binarize_dev(a, 16, 8, 16, 1, 5, 1, bnz.BNZ_SAUVOLA, 0.5, 128.0, a + 1024, 16, None,
                                   None) == bnz.BNZ_ENODEV
    assert lib.bnz_confusion_dev(a, 16, 0, a + 1024, 16, 1, 4, 16, a + 4096, None) == bnz.BNZ_ENODEV
    assert (buf == 0).all()


def test_window_call_checks(lib):
    src = np.zeros((64, 64), np.uint8)
    dst = np.zeros((64, 64), np.uint8)
    rc = lib.bnz_binarize_window(src.ctypes.data, 64, 64, 1, 15, bnz.BNZ_SAUVOLA, 0.5, 128.0, dst.ctypes.data, 1000)
    assert rc == bnz.BNZ_EINVAL and "too small" in bnz.bnz_last_error()
    rc = lib.bnz_binarize_window(src.ctypes.data, 64, 64, 1, 0, bnz.BNZ_SAUVOLA, 0.5, 128.0, dst.ctypes.data, 1 << 20)
    assert rc == bnz.BNZ_EINVAL and "window size" in bnz.bnz_last_error()
    import torch
    if not torch.cuda.is_available():
        rc = lib.bnz_binarize_window(src.ctypes.data, 64, 64, 1, 15, bnz.BNZ_SAUVOLA, 0.5, 128.0, dst.ctypes.data,
                                     1 << 20)
        assert rc == bnz.BNZ_ENODEV


def test_binding_constants_match_the_header():
    """Every numeric #define of include/bnz.h that the Python binding also defines has the same value there
    (buffer sizes such as BNZ_OTSU_SCRATCH_BYTES are allocated from the binding's copy)."""
    text = open(os.path.join(ROOT, "include", "bnz.h")).read()
    defs = dict(re.findall(r"^#define\s+(BNZ_[A-Z0-9_]+)\s+([-+0-9.eE]+)\b", text, flags=re.M))
    assert "BNZ_OTSU_SCRATCH_BYTES" in defs and "BNZ_MAX_W" in defs
    checked = 0
    for name, value in defs.items():
        if hasattr(bnz, name):
            assert float(getattr(bnz, name)) == float(value), (name, getattr(bnz, name), value)
            checked += 1
    assert checked >= 2
