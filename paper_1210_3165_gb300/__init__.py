"""Python binding of the GB300 locally adaptive binarization library (``libbnz.so``).

Thin ctypes layer with the same names as the C ABI in ``include/bnz.h``.  It
only marshals arguments: every pixel is computed by the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU path:
if the compiled library is missing, importing the binding raises, and on a
machine without a GPU the calls return ``BNZ_ENODEV``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

BNZ_OK, BNZ_EINVAL, BNZ_ENOMEM, BNZ_ECUDA, BNZ_ETIMEOUT, BNZ_ENODEV = range(6)
BNZ_SAUVOLA, BNZ_NIBLACK = 0, 1
BNZ_MAX_W = 255
STATUS_NAMES = {0: "BNZ_OK", 1: "BNZ_EINVAL", 2: "BNZ_ENOMEM", 3: "BNZ_ECUDA", 4: "BNZ_ETIMEOUT",
                5: "BNZ_ENODEV"}

LIB_PATH = _build.LIB


class BnzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class bnz_page(ctypes.Structure):
    _fields_ = [("d_src", ctypes.c_void_p), ("src_pitch", ctypes.c_size_t), ("height", ctypes.c_int),
                ("width", ctypes.c_int), ("channels", ctypes.c_int), ("W", ctypes.c_int),
                ("rule", ctypes.c_int), ("packed", ctypes.c_int), ("k", ctypes.c_double),
                ("R", ctypes.c_double), ("d_dst", ctypes.c_void_p), ("dst_pitch", ctypes.c_size_t),
                ("tile_w", ctypes.c_int), ("reserved", ctypes.c_int)]


class bnz_server_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int), ("compute_streams", ctypes.c_int),
                ("batched", ctypes.c_int), ("reserved", ctypes.c_int)]


class bnz_request(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("src_pitch", ctypes.c_size_t), ("src_on_device", ctypes.c_int),
                ("height", ctypes.c_int), ("width", ctypes.c_int), ("channels", ctypes.c_int), ("W", ctypes.c_int),
                ("rule", ctypes.c_int), ("k", ctypes.c_double), ("R", ctypes.c_double), ("packed", ctypes.c_int),
                ("dst", ctypes.c_void_p), ("dst_pitch", ctypes.c_size_t), ("tag", ctypes.c_ulonglong)]


class bnz_run(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("rule", ctypes.c_int), ("k", ctypes.c_double), ("R", ctypes.c_double),
                ("dst", ctypes.c_void_p)]


class bnz_tile(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("chunk", ctypes.c_int),
                ("edge_weight", ctypes.c_int)]


_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load ``libbnz.so`` (building it first if it is absent); raise if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1210_3165_gb300._build.build()")
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    P, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.bnz_sauvola.argtypes = [P, i, i, i, i, d, d, P]
    lib.bnz_niblack.argtypes = [P, i, i, i, i, d, P]
    lib.bnz_sauvola_dev.argtypes = [P, sz, i, i, i, i, d, d, P, sz, i, P, P]
    lib.bnz_niblack_dev.argtypes = [P, sz, i, i, i, i, d, P, sz, i, P, P]
    lib.bnz_binarize_dev.argtypes = [P, sz, i, i, i, i, i, d, d, P, sz, i, P, P, P]
    lib.bnz_dual_dev.argtypes = [P, sz, i, i, i, i, d, d, d, P, P, sz, i, P, P]
    lib.bnz_otsu_dev.argtypes = [P, sz, i, i, i, P, sz, i, P, P]
    lib.bnz_host_bands.argtypes = [i, i, i, P, i]
    lib.bnz_last_error.restype = ctypes.c_char_p
    lib.bnz_last_error.argtypes = []
    lib.bnz_version.argtypes = []
    lib.bnz_decision_margins.argtypes = [i, d, d, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_float)]
    lib.bnz_fused_plan.argtypes = [i, i, i, i, P, ctypes.POINTER(sz), ctypes.POINTER(i), ctypes.POINTER(i),
                                   ctypes.POINTER(i)]
    for name in ("bnz_sauvola", "bnz_niblack", "bnz_sauvola_dev", "bnz_niblack_dev", "bnz_binarize_dev",
                 "bnz_dual_dev", "bnz_otsu_dev", "bnz_host_bands", "bnz_version", "bnz_fused_plan",
                 "bnz_decision_margins"):
        getattr(lib, name).restype = ctypes.c_int
    _optional_symbols(lib)
    _lib = lib
    return lib


def _optional_symbols(lib):
    """Entry points added by later parts of the library (integral images, batches)."""
    P, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    table = {
        "bnz_batch_create": ([P, i, i, P, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "bnz_batch_run": ([P, P], ctypes.c_int),
        "bnz_batch_desc_bytes": ([i], ctypes.c_size_t),
        "bnz_batch_create_async": ([P, i, P, sz, P, P, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "bnz_batch_info": ([P, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(sz),
                            ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
        "bnz_batch_destroy": ([P], ctypes.c_int),
        "bnz_copy2d_async": ([P, sz, P, sz, sz, sz, P], ctypes.c_int),
        "bnz_server_create": ([P, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "bnz_server_submit": ([P, P], ctypes.c_int),
        "bnz_server_poll": ([P, P, P, P, i, i], ctypes.c_int),
        "bnz_server_stats": ([P, P, P, P, P, P], ctypes.c_int),
        "bnz_server_error": ([P, ctypes.c_char_p, sz], ctypes.c_int),
        "bnz_server_destroy": ([P], ctypes.c_int),
        "bnz_pool_create": ([P, sz, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "bnz_pool_alloc": ([P, sz, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "bnz_pool_free": ([P, P], ctypes.c_int),
        "bnz_pool_stats": ([P, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(i)],
                           ctypes.c_int),
        "bnz_pool_fail_next": ([P, i], ctypes.c_int),
        "bnz_pool_destroy": ([P], ctypes.c_int),
        "bnz_selftest_sqrt_approx": ([ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_double)],
                                     ctypes.c_int),
        "bnz_binarize_runs": ([P, i, i, i, P, i], ctypes.c_int),
        "bnz_selftest_gray": ([ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p], i),
        "bnz_selftest_fused_timeout": ([P, sz, i, i, i, i, i, d, d, P, sz, P, P], ctypes.c_int),
        "bnz_selftest_rcp_approx": ([ctypes.c_uint, ctypes.c_uint, ctypes.POINTER(ctypes.c_double)],
                                    ctypes.c_int),
        "bnz_selftest_wait_timeout": ([ctypes.c_longlong, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)],
                                      ctypes.c_int),
        "bnz_integral_scratch_bytes": ([i, i], ctypes.c_size_t),
        "bnz_binarize_integral_dev": ([P, sz, i, i, i, i, i, d, d, P, sz, i, P, sz, P, P], ctypes.c_int),
        "bnz_binarize_integral_static_dev": ([P, sz, i, i, i, i, i, d, d, P, sz, i, P, P], ctypes.c_int),
        "bnz_integral_images_dev": ([P, sz, i, i, i, P, sz, ctypes.POINTER(ctypes.c_longlong), P], ctypes.c_int),
        "bnz_binarize_window": ([P, i, i, i, i, i, d, d, P, sz], ctypes.c_int),
        "bnz_gs_binarize_dev": ([P, sz, i, i, i, i, i, i, d, d, P, sz, P, P], ctypes.c_int),
        "bnz_confusion_dev": ([P, sz, i, P, sz, i, i, i, P, P], ctypes.c_int),
    }
    for name, (args, res) in table.items():
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res


def bnz_last_error() -> str:
    return load().bnz_last_error().decode(errors="replace")


def bnz_version() -> int:
    return load().bnz_version()


def bnz_decision_margins(rule, k: float, R: float = 128.0) -> tuple:
    """(E, E_int, Tdf): the fused kernel's decision margins for these parameters (host computation)."""
    if isinstance(rule, str):
        rule = {"sauvola": BNZ_SAUVOLA, "niblack": BNZ_NIBLACK}[rule.lower()]
    E, Ei, T = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(load().bnz_decision_margins(int(rule), float(k), float(R), ctypes.byref(E), ctypes.byref(Ei),
                                       ctypes.byref(T)))
    return E.value, Ei.value, T.value


def _check(rc: int):
    if rc != BNZ_OK:
        raise BnzError(rc, bnz_last_error())


# ---------------------------------------------------------------------------
# host-pointer calls (numpy in, numpy out)
# ---------------------------------------------------------------------------

def _host_img(src):
    src = np.ascontiguousarray(src, dtype=np.uint8)
    if src.ndim == 2:
        return src, src.shape[0], src.shape[1], 1
    if src.ndim == 3 and src.shape[2] == 3:
        return src, src.shape[0], src.shape[1], 3
    raise ValueError("image must be HxW or HxWx3 uint8")


def bnz_sauvola(src, W: int, k: float = 0.5, R: float = 128.0) -> np.ndarray:
    """Synchronous Sauvola binarization of a host image; returns the {0,255} mask."""
    src, h, w, ch = _host_img(src)
    dst = np.empty((h, w), np.uint8)
    _check(load().bnz_sauvola(src.ctypes.data, h, w, ch, int(W), float(k), float(R), dst.ctypes.data))
    return dst


def bnz_niblack(src, W: int, k: float = -0.2) -> np.ndarray:
    src, h, w, ch = _host_img(src)
    dst = np.empty((h, w), np.uint8)
    _check(load().bnz_niblack(src.ctypes.data, h, w, ch, int(W), float(k), dst.ctypes.data))
    return dst


# ---------------------------------------------------------------------------
# device-pointer calls (torch CUDA tensors)
# ---------------------------------------------------------------------------

def binarize_window(src, W: int, rule: str | int = "sauvola", k: float | None = None, R: float = 128.0,
                    window_bytes: int = 256 << 20, out: np.ndarray | None = None) -> np.ndarray:
    """Host page -> host mask through a device window of at most window_bytes (bnz_binarize_window)."""
    if isinstance(rule, str):
        rule = {"sauvola": BNZ_SAUVOLA, "niblack": BNZ_NIBLACK}[rule.lower()]
    if k is None:
        k = 0.5 if rule == BNZ_SAUVOLA else -0.2
    a, h, w, ch = _host_img(src)
    if out is None:
        out = np.empty((h, w), np.uint8)
    if out.shape != (h, w) or out.dtype != np.uint8 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous HxW uint8 array")
    _check(load().bnz_binarize_window(a.ctypes.data, h, w, ch, int(W), int(rule), float(k), float(R),
                                      out.ctypes.data, int(window_bytes)))
    return out


def binarize_runs(src, runs, out=None) -> list:
    """One host page, several settings (bnz_binarize_runs): runs = [(W, rule, k, R), ...] with rule
    "sauvola"/"niblack" or BNZ_*; returns one {0,255} mask per setting (or fills the arrays in `out`)."""
    img, h, w, ch = _host_img(src)
    masks = out if out is not None else [np.empty((h, w), np.uint8) for _ in runs]
    arr = (bnz_run * len(runs))()
    for j, (W, rule, k, R) in enumerate(runs):
        rid = rule if isinstance(rule, int) else (BNZ_SAUVOLA if rule == "sauvola" else BNZ_NIBLACK)
        assert masks[j].shape == (h, w) and masks[j].dtype == np.uint8 and masks[j].flags.c_contiguous
        arr[j] = bnz_run(int(W), rid, float(k), float(R), masks[j].ctypes.data)
    _check(load().bnz_binarize_runs(img.ctypes.data, h, w, ch, arr, len(runs)))
    return masks


def alloc_pitched(height: int, row_bytes: int, device="cuda", align: int = 16):
    """uint8 CUDA tensor view of shape (height, row_bytes) whose row stride is a multiple of ``align``."""
    import torch
    pitch = (row_bytes + align - 1) // align * align
    base = torch.empty((max(height, 1), pitch), dtype=torch.uint8, device=device)
    return base[:height, :row_bytes]


def _dev_img(t):
    """(ptr, pitch, h, w, ch) of a uint8 CUDA tensor laid out HxW or HxWx3 with unit inner strides."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.uint8 or not t.is_cuda:
        raise TypeError("expected a uint8 CUDA tensor")
    # strides of size-1 dimensions carry no information: a single row gets the
    # smallest 16-byte multiple as its pitch (no other row is ever addressed)
    if t.dim() == 2:
        h, w = t.shape
        if w > 1 and t.stride(1) != 1:
            raise ValueError("inner stride must be 1")
        pitch = t.stride(0) if h > 1 else (w + 15) // 16 * 16
        return t.data_ptr(), pitch, h, w, 1
    if t.dim() == 3 and t.shape[2] == 3:
        h, w = t.shape[:2]
        if t.stride(2) != 1 or (w > 1 and t.stride(1) != 3):
            raise ValueError("RGB tensor must be interleaved (strides (pitch, 3, 1))")
        pitch = t.stride(0) if h > 1 else (3 * w + 15) // 16 * 16
        return t.data_ptr(), pitch, h, w, 3
    raise ValueError("image must be HxW or HxWx3")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _out_pitch(dst, w, packed):
    if dst.dim() != 2 or (dst.shape[1] > 1 and dst.stride(1) != 1) or dst.dtype.itemsize != 1:
        raise ValueError("dst must be a 2-D uint8 tensor with unit inner stride")
    need = (w + 7) // 8 if packed else w
    if dst.shape[1] < need:
        raise ValueError(f"dst rows must hold {need} bytes")
    return dst.stride(0) if dst.shape[0] > 1 else max(dst.shape[1], 1)


def bnz_binarize_dev(d_src, W: int, rule: int, k: float, R: float, d_dst, packed: bool = False,
                     tile: bnz_tile | None = None, stream=None, d_stats=None) -> None:
    """Enqueue one binarization on ``stream`` (default: torch's current stream)."""
    ptr, pitch, h, w, ch = _dev_img(d_src)
    dp = _out_pitch(d_dst, w, packed)
    _check(load().bnz_binarize_dev(ptr, pitch, h, w, ch, int(W), int(rule), float(k), float(R),
                                   d_dst.data_ptr(), dp, 1 if packed else 0,
                                   ctypes.byref(tile) if tile is not None else None,
                                   _stream_ptr(stream), d_stats.data_ptr() if d_stats is not None else None))


def bnz_sauvola_dev(d_src, W: int, k: float, R: float, d_dst, packed: bool = False, stream=None,
                    d_stats=None) -> None:
    ptr, pitch, h, w, ch = _dev_img(d_src)
    dp = _out_pitch(d_dst, w, packed)
    _check(load().bnz_sauvola_dev(ptr, pitch, h, w, ch, int(W), float(k), float(R), d_dst.data_ptr(), dp,
                                  1 if packed else 0, _stream_ptr(stream),
                                  d_stats.data_ptr() if d_stats is not None else None))


def bnz_niblack_dev(d_src, W: int, k: float, d_dst, packed: bool = False, stream=None, d_stats=None) -> None:
    ptr, pitch, h, w, ch = _dev_img(d_src)
    dp = _out_pitch(d_dst, w, packed)
    _check(load().bnz_niblack_dev(ptr, pitch, h, w, ch, int(W), float(k), d_dst.data_ptr(), dp,
                                  1 if packed else 0, _stream_ptr(stream),
                                  d_stats.data_ptr() if d_stats is not None else None))


def bnz_dual_dev(d_src, W: int, k_sauvola: float, R: float, k_niblack: float, d_dst_sauvola, d_dst_niblack,
                 packed: bool = False, stream=None, d_stats=None) -> None:
    """Both rules from one pass over the window sums: the Sauvola and the Niblack mask of one page."""
    ptr, pitch, h, w, ch = _dev_img(d_src)
    dp = _out_pitch(d_dst_sauvola, w, packed)
    if _out_pitch(d_dst_niblack, w, packed) != dp:
        raise ValueError("both masks must have the same row pitch")
    _check(load().bnz_dual_dev(ptr, pitch, h, w, ch, int(W), float(k_sauvola), float(R), float(k_niblack),
                               d_dst_sauvola.data_ptr(), d_dst_niblack.data_ptr(), dp, 1 if packed else 0,
                               _stream_ptr(stream), d_stats.data_ptr() if d_stats is not None else None))


def binarize_dual(d_src, W: int, k_sauvola: float = 0.5, R: float = 128.0, k_niblack: float = -0.2,
                  packed: bool = False, stream=None, d_stats=None):
    """Sauvola and Niblack masks of a pitched uint8 CUDA image from one kernel; returns (sauvola, niblack)."""
    _, _, h, w, _ = _dev_img(d_src)
    row = (w + 7) // 8 if packed else w
    out_s = alloc_pitched(h, row, d_src.device)
    out_n = alloc_pitched(h, row, d_src.device)
    bnz_dual_dev(d_src, W, k_sauvola, R, k_niblack, out_s, out_n, packed, stream, d_stats)
    return out_s, out_n


BNZ_OTSU_SCRATCH_BYTES = 20480


def bnz_otsu_dev(d_src, d_dst, d_scratch, packed: bool = False, stream=None) -> None:
    """Enqueue Eq. 2 with Otsu's threshold; d_scratch: uint8 CUDA tensor of BNZ_OTSU_SCRATCH_BYTES."""
    ptr, pitch, h, w, ch = _dev_img(d_src)
    dp = _out_pitch(d_dst, w, packed)
    if d_scratch.numel() * d_scratch.element_size() < BNZ_OTSU_SCRATCH_BYTES:
        raise ValueError(f"d_scratch must hold {BNZ_OTSU_SCRATCH_BYTES} bytes")
    _check(load().bnz_otsu_dev(ptr, pitch, h, w, ch, d_dst.data_ptr(), dp, 1 if packed else 0,
                               d_scratch.data_ptr(), _stream_ptr(stream)))


def otsu(d_src, packed: bool = False, stream=None):
    """Global binarization with Otsu's threshold: returns (mask, T, histogram) on the device; T and the
    histogram are views into the scratch the call writes (read them after the stream's work)."""
    import torch
    _, _, h, w, _ = _dev_img(d_src)
    out = alloc_pitched(h, (w + 7) // 8 if packed else w, d_src.device)
    scratch = torch.empty(BNZ_OTSU_SCRATCH_BYTES, dtype=torch.uint8, device=d_src.device)
    bnz_otsu_dev(d_src, out, scratch, packed, stream)
    hist = scratch[:2048].view(torch.int64)
    T = scratch[2048:2052].view(torch.int32)
    return out, T, hist


def host_bands(height: int, width: int, W: int) -> list:
    """Row-band boundaries [0, ..., height] the host-pointer calls use for a page (host logic, no device)."""
    import numpy as np
    starts = np.zeros(64, np.int32)
    nb = load().bnz_host_bands(int(height), int(width), int(W), starts.ctypes.data, len(starts))
    if nb < 0:
        raise BnzError(-nb, bnz_last_error())
    return [int(v) for v in starts[:nb + 1]]


def bnz_copy2d_async(dst: int, dst_pitch: int, src: int, src_pitch: int, width_bytes: int, height: int,
                     stream=None) -> None:
    """Stream-ordered 2-D copy between host and device pointers (a copy-engine transfer)."""
    _check(load().bnz_copy2d_async(dst, dst_pitch, src, src_pitch, width_bytes, height, _stream_ptr(stream)))


def bnz_integral_scratch_bytes(h: int, w: int) -> int:
    return load().bnz_integral_scratch_bytes(int(h), int(w))


def alloc_scratch(nbytes: int, device="cuda"):
    """Device scratch buffer (torch tensor of int64, 256-byte aligned base)."""
    import torch
    return torch.empty(((nbytes + 7) // 8,), dtype=torch.int64, device=device)


def bnz_binarize_integral_dev(d_src, W: int, rule: int, k: float, R: float, d_dst, d_scratch, packed=False,
                              stream=None, d_stats=None) -> None:
    """Integral-image variant; d_scratch: a CUDA tensor of at least bnz_integral_scratch_bytes bytes."""
    ptr, pitch, h, w, ch = _dev_img(d_src)
    dp = _out_pitch(d_dst, w, packed)
    nbytes = d_scratch.numel() * d_scratch.element_size()
    _check(load().bnz_binarize_integral_dev(ptr, pitch, h, w, ch, int(W), int(rule), float(k), float(R),
                                            d_dst.data_ptr(), dp, 1 if packed else 0, d_scratch.data_ptr(),
                                            nbytes, _stream_ptr(stream),
                                            d_stats.data_ptr() if d_stats is not None else None))


def bnz_binarize_integral_static_dev(d_src, W: int, rule: int, k: float, R: float, d_dst, packed=False,
                                     stream=None, d_stats=None) -> None:
    """Integral-image variant that allocates nothing (library-owned scratch; see include/bnz.h)."""
    ptr, pitch, h, w, ch = _dev_img(d_src)
    dp = _out_pitch(d_dst, w, packed)
    _check(load().bnz_binarize_integral_static_dev(ptr, pitch, h, w, ch, int(W), int(rule), float(k), float(R),
                                                   d_dst.data_ptr(), dp, 1 if packed else 0, _stream_ptr(stream),
                                                   d_stats.data_ptr() if d_stats is not None else None))


def bnz_integral_images_dev(d_src, d_scratch, stream=None):
    """Build the two int64 summed-area tables; returns views (I1, I2) of shape (h+1, w+1)."""
    ptr, pitch, h, w, ch = _dev_img(d_src)
    nbytes = d_scratch.numel() * d_scratch.element_size()
    ld = ctypes.c_longlong(0)
    _check(load().bnz_integral_images_dev(ptr, pitch, h, w, ch, d_scratch.data_ptr(), nbytes,
                                          ctypes.byref(ld), _stream_ptr(stream)))
    n = (h + 1) * ld.value
    I1 = d_scratch[:n].view(h + 1, ld.value)[:, :w + 1]
    I2 = d_scratch[n:2 * n].view(h + 1, ld.value)[:, :w + 1]
    return I1, I2


class Batch:
    """Many pages binarized by one persistent launch per channel count (optionally a CUDA graph).

    pages: dicts with src (pitched uint8 CUDA image), dst (pitched uint8 CUDA output), W, and optional
    rule ("sauvola"/"niblack"), k, R, packed, tile_w.  The tensors are bound at creation: run() reads
    the same inputs and writes the same outputs every time.
    """

    def __init__(self, pages, use_graph: bool = True, d_stats=None, desc_buffer=None, stream=None):
        arr = (bnz_page * len(pages))()
        self._keep = []
        for i, pg in enumerate(pages):
            ptr, pitch, h, w, ch = _dev_img(pg["src"])
            rule = pg.get("rule", "sauvola")
            if isinstance(rule, str):
                rule = {"sauvola": BNZ_SAUVOLA, "niblack": BNZ_NIBLACK}[rule.lower()]
            k = pg.get("k", 0.5 if rule == BNZ_SAUVOLA else -0.2)
            packed = bool(pg.get("packed", False))
            dst = pg["dst"]
            arr[i] = bnz_page(ptr, pitch, h, w, ch, int(pg["W"]), int(rule), 1 if packed else 0, float(k),
                              float(pg.get("R", 128.0)), dst.data_ptr(), _out_pitch(dst, w, packed),
                              int(pg.get("tile_w", 0)), 0)
            self._keep += [pg["src"], dst]
        self._stats = d_stats
        h = ctypes.c_void_p(None)
        stats_ptr = d_stats.data_ptr() if d_stats is not None else None
        if desc_buffer is not None:  # no allocation: descriptors into the caller's buffer, ordered on `stream`
            self._keep.append(desc_buffer)
            _check(load().bnz_batch_create_async(ctypes.cast(arr, ctypes.c_void_p), len(pages),
                                                 desc_buffer.data_ptr(),
                                                 desc_buffer.numel() * desc_buffer.element_size(),
                                                 _stream_ptr(stream), stats_ptr, ctypes.byref(h)))
        else:
            _check(load().bnz_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(pages), 1 if use_graph else 0,
                                           stats_ptr, ctypes.byref(h)))
        self._h = h

    @staticmethod
    def desc_bytes(n: int) -> int:
        return load().bnz_batch_desc_bytes(int(n))

    def run(self, stream=None) -> None:
        _check(load().bnz_batch_run(self._h, _stream_ptr(stream)))

    def info(self) -> dict:
        n, l, g = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        sm, rows = ctypes.c_size_t(0), ctypes.c_longlong(0)
        _check(load().bnz_batch_info(self._h, ctypes.byref(n), ctypes.byref(l), ctypes.byref(g),
                                     ctypes.byref(sm), ctypes.byref(rows)))
        return dict(pages=n.value, launches=l.value, grid=g.value, smem=sm.value, strip_rows=rows.value)

    def close(self) -> None:
        if self._h:
            load().bnz_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pool:
    """First-fit bookkeeping over one caller-owned device range (``bnz_pool_*``).

    ``base`` is an address (int) or a CUDA tensor whose memory the pool carves up; the tensor is kept
    alive.  ``alloc`` returns an address, or None when no free range fits (BNZ_ENOMEM)."""

    def __init__(self, base, nbytes: int | None = None):
        self._owner = None
        if not isinstance(base, int):
            self._owner = base
            nbytes = base.numel() * base.element_size() if nbytes is None else nbytes
            base = base.data_ptr()
        h = ctypes.c_void_p(None)
        _check(load().bnz_pool_create(ctypes.c_void_p(base), int(nbytes), ctypes.byref(h)))
        self._h, self.base, self.nbytes = h, base, int(nbytes)

    def alloc(self, nbytes: int):
        out = ctypes.c_void_p(None)
        rc = load().bnz_pool_alloc(self._h, int(nbytes), ctypes.byref(out))
        if rc == BNZ_ENOMEM:
            return None
        _check(rc)
        return out.value

    def free(self, ptr: int) -> None:
        _check(load().bnz_pool_free(self._h, ctypes.c_void_p(ptr)))

    def stats(self) -> dict:
        u, hw, lf, n = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_int(0)
        _check(load().bnz_pool_stats(self._h, ctypes.byref(u), ctypes.byref(hw), ctypes.byref(lf), ctypes.byref(n)))
        return dict(used=u.value, high_water=hw.value, largest_free=lf.value, live=n.value)

    def fail_next(self, n: int) -> None:
        _check(load().bnz_pool_fail_next(self._h, int(n)))

    def close(self) -> None:
        if self._h:
            load().bnz_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# reduced sets S' of Sec. 2 (Eq. 5): structures proposed by this library (see bnz.h)
BNZ_GS_CROSS, BNZ_GS_DIAGONALS, BNZ_GS_STAR, BNZ_GS_FRAME, BNZ_GS_FRAME_CROSS, BNZ_GS_FRAME_DIAGONALS = range(1, 7)
GS_NAMES = {BNZ_GS_CROSS: "cross", BNZ_GS_DIAGONALS: "diagonals", BNZ_GS_STAR: "star", BNZ_GS_FRAME: "frame",
            BNZ_GS_FRAME_CROSS: "frame+cross", BNZ_GS_FRAME_DIAGONALS: "frame+diagonals"}


def bnz_gs_binarize_dev(d_src, W: int, gs: int, rule: int, k: float, R: float, d_dst, stream=None,
                        d_stats=None) -> None:
    """Enqueue the reduced-set binarization (Eq. 5 on structure ``gs``) of a uint8 CUDA image."""
    ptr, pitch, h, w, ch = _dev_img(d_src)
    _check(load().bnz_gs_binarize_dev(ptr, pitch, h, w, ch, int(W), int(gs), int(rule), float(k), float(R),
                                      d_dst.data_ptr(), _out_pitch(d_dst, w, False),
                                      d_stats.data_ptr() if d_stats is not None else None,
                                      _stream_ptr(stream)))


def gs_binarize(d_src, W: int, gs: int, rule: str | int = "sauvola", k: float | None = None, R: float = 128.0,
                out=None, stream=None, d_stats=None):
    """Reduced-set mask of a uint8 CUDA image; returns the (pitched) output tensor view."""
    if isinstance(rule, str):
        rule = {"sauvola": BNZ_SAUVOLA, "niblack": BNZ_NIBLACK}[rule.lower()]
    if k is None:
        k = 0.5 if rule == BNZ_SAUVOLA else -0.2
    _, _, h, w, _ = _dev_img(d_src)
    if out is None:
        out = alloc_pitched(h, w, d_src.device)
    bnz_gs_binarize_dev(d_src, W, gs, rule, k, R, out, stream, d_stats)
    return out


def bnz_confusion_dev(d_mask, d_ref, d_counts, mask_ink: int = 0, ref_ink: int = 1, stream=None) -> None:
    """Add TP, FP, FN of d_mask against d_ref (text = the ink byte of each) to d_counts[0:3] (uint64/int64)."""
    mp, mpitch, h, w, mch = _dev_img(d_mask)
    rp, rpitch, rh, rw, rch = _dev_img(d_ref)
    if (h, w) != (rh, rw) or mch != 1 or rch != 1:
        raise BnzError(BNZ_EINVAL, "mask and reference must be equal-sized byte images")
    _check(load().bnz_confusion_dev(mp, mpitch, int(mask_ink), rp, rpitch, int(ref_ink), h, w, d_counts.data_ptr(),
                                    _stream_ptr(stream)))


def fmeasure(d_mask, d_ref, mask_ink: int = 0, ref_ink: int = 1, stream=None):
    """Eq. 6 from the device counts: returns (FM, recall, precision, (TP, FP, FN, TN))."""
    import torch
    counts = torch.zeros(4, dtype=torch.int64, device=d_mask.device)
    bnz_confusion_dev(d_mask, d_ref, counts, mask_ink, ref_ink, stream)
    if stream is not None:
        stream.synchronize()
    tp, fp, fn, _ = (int(v) for v in counts.cpu())
    tn = d_mask.shape[0] * d_mask.shape[1] - tp - fp - fn
    rec = tp / (tp + fn) if tp + fn else 0.0
    prec = tp / (tp + fp) if tp + fp else 0.0
    fm = 2.0 * rec * prec / (rec + prec) if rec + prec else 0.0
    return fm, rec, prec, (tp, fp, fn, tn)


def bnz_fused_plan(h: int, w: int, ch: int, W: int, tile: bnz_tile | None = None) -> dict:
    smem = ctypes.c_size_t(0)
    grid, tw, th = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().bnz_fused_plan(h, w, ch, W, ctypes.byref(tile) if tile is not None else None,
                                 ctypes.byref(smem), ctypes.byref(grid), ctypes.byref(tw), ctypes.byref(th)))
    return dict(smem=smem.value, grid=grid.value, tile_w=tw.value, rows_per_cta=th.value)


# ---------------------------------------------------------------------------
# convenience wrapper used by tests, bench and the server
# ---------------------------------------------------------------------------

def to_device_pitched(img: np.ndarray, device="cuda"):
    """Copy a host HxW / HxWx3 uint8 image into a 16-byte-pitched CUDA tensor view."""
    import torch
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape[:2]
    ch = 1 if img.ndim == 2 else 3
    t = alloc_pitched(h, w * ch, device)
    t.copy_(torch.from_numpy(img.reshape(h, w * ch)))
    if ch == 1:
        return t
    return torch.as_strided(t, (h, w, 3), (t.stride(0), 3, 1))


def binarize(d_src, W: int, rule: str | int = "sauvola", k: float | None = None, R: float = 128.0,
             packed: bool = False, out=None, tile: bnz_tile | None = None, stream=None, d_stats=None):
    """Binarize a pitched uint8 CUDA image; returns the (pitched) output tensor view."""
    if isinstance(rule, str):
        rule = {"sauvola": BNZ_SAUVOLA, "niblack": BNZ_NIBLACK}[rule.lower()]
    if k is None:
        k = 0.5 if rule == BNZ_SAUVOLA else -0.2
    _, _, h, w, _ = _dev_img(d_src)
    if out is None:
        out = alloc_pitched(h, (w + 7) // 8 if packed else w, d_src.device)
    bnz_binarize_dev(d_src, W, rule, k, R, out, packed, tile, stream, d_stats)
    return out
