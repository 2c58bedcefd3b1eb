"""CPU oracle for exact Sauvola / Niblack binarization -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  The product path (the CUDA
library and its binding) never does.  The oracle is plain C (``bnzref.c``),
compiled with gcc at ``-O2 -ffp-contract=off`` so that every fp64 operation
is a single IEEE-rounded step in the order the C source states:

* gray conversion, Eq. 1 (Sec. 1), integer round-half-up reading
  ``(299 r + 587 g + 114 b + 500) // 1000``;
* clipped W x W window sums (Sec. 2), exact int64, by two independent paths:
  naive O(W^2) per pixel and the O(W)-per-pixel sliding scheme (Sec. 3);
* m, s and the Sauvola threshold of Eq. 4 or the Niblack threshold in fp64;
* the decision of Eq. 3, with ties ``|f - t| < 1e-9`` counted;
* the global rule of Eq. 2 with Otsu's threshold (cited in Sec. 1; Otsu's
  published definition: the T maximising the between-class variance of the
  gray histogram, exact 128-bit class difference, fp64 criterion, smallest T
  among equal values);
* the reduced-set rule of Eq. 5 (Sec. 2): m', s' over a structure S' of O(W)
  window pixels.  Fig. 1, which draws the paper's six structures, is not
  available; the structures GS1..GS6 here are proposed by this project (cross,
  diagonals, star, frame, frame + cross, frame + diagonals; GS0 = the whole
  window).  Their agreement with the paper's accuracy figures is therefore
  unpinned; the oracle itself is pinned to brute-force set enumeration,
  closed forms and to Eq. 4 (GS0);
* the confusion counts behind the F-measure of Eq. 6.

Pins (tests/test_oracle_*.py) tie it to things other than itself: brute force
on tiny images, a library box filter, exact rational arithmetic, closed forms
(constant image, step edge, impulse; one- and two-level pages for Otsu) and
symmetry and offset invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bnzref.c")
_HDR = os.path.join(_HERE, "bnzref.h")
_LIB = os.path.join(_HERE, "libbnzref.so")

SAUVOLA = 0
NIBLACK = 1
NAIVE = 0
SLIDING = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libbnzref.so`` next to the source (gcc, no fast-math, no FMA contraction)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
               "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
               "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i, ll, d = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.bnzref_gray.argtypes = [P, i, i, i, ll, P]
        lib.bnzref_window_sums_naive.argtypes = [P, i, i, i, P, P, P]
        lib.bnzref_window_sums_sliding.argtypes = [P, i, i, i, P, P, P]
        lib.bnzref_threshold_value.argtypes = [ctypes.c_int64] * 3 + [i, d, d]
        lib.bnzref_threshold_value.restype = d
        lib.bnzref_decide.argtypes = [i, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, i, d, d,
                                      ctypes.POINTER(i), ctypes.POINTER(d)]
        lib.bnzref_threshold.argtypes = [P, P, P, P, i, i, i, d, d, P, i64p]
        lib.bnzref_binarize.argtypes = [P, i, i, i, ll, i, i, d, d, i, P, ll, i64p, i]
        lib.bnzref_pixel.argtypes = [P, i, i, i, ll, i, i, d, d, i, i, ctypes.POINTER(i),
                                     ctypes.POINTER(d)]
        lib.bnzref_integral.argtypes = [P, i, i, P, P]
        lib.bnzref_pack.argtypes = [P, i, i, ll, P, ll]
        lib.bnzref_histogram.argtypes = [P, i, i, i, ll, P]
        lib.bnzref_otsu_threshold.argtypes = [P, P]
        lib.bnzref_otsu.argtypes = [P, i, i, i, ll, P, ll, ctypes.POINTER(i)]
        lib.bnzref_gs_member.argtypes = [i, i, i, i]
        lib.bnzref_gs_offsets.argtypes = [i, i, P, P, i]
        lib.bnzref_gs_sums.argtypes = [P, i, i, i, i, P, P, P]
        lib.bnzref_gs_binarize.argtypes = [P, i, i, i, ll, i, i, i, d, d, P, ll, i64p]
        lib.bnzref_confusion.argtypes = [P, ll, i, P, ll, i, i, i, P]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _img(src: np.ndarray):
    src = np.ascontiguousarray(src, dtype=np.uint8)
    if src.ndim == 2:
        h, w = src.shape
        ch = 1
    elif src.ndim == 3 and src.shape[2] == 3:
        h, w, ch = src.shape
    else:
        raise ValueError("image must be HxW gray or HxWx3 RGB uint8")
    return src, h, w, ch


def _check(rc: int):
    if rc != 0:
        raise ValueError(f"oracle call failed with status {rc}")


def gray(src: np.ndarray) -> np.ndarray:
    """Eq. 1 gray conversion (integer round-half-up reading)."""
    src, h, w, ch = _img(src)
    out = np.empty((h, w), np.uint8)
    _check(_load().bnzref_gray(_ptr(src), h, w, ch, w * ch, _ptr(out)))
    return out


def window_sums(f: np.ndarray, W: int, method: int = SLIDING):
    """Exact clipped-window (n, S1, S2) for every pixel of a gray image."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    h, w = f.shape
    n = np.empty((h, w), np.int64)
    a = np.empty((h, w), np.int64)
    b = np.empty((h, w), np.int64)
    fn = _load().bnzref_window_sums_naive if method == NAIVE else _load().bnzref_window_sums_sliding
    _check(fn(_ptr(f), h, w, int(W), _ptr(n), _ptr(a), _ptr(b)))
    return n, a, b


def threshold_value(n: int, s1: int, s2: int, rule: int, k: float, R: float = 128.0) -> float:
    """fp64 threshold t of Eq. 4 (Sauvola) or Niblack, fixed operation order."""
    return _load().bnzref_threshold_value(int(n), int(s1), int(s2), int(rule), float(k), float(R))


def decide(f: int, n: int, s1: int, s2: int, rule: int, k: float, R: float = 128.0):
    """Eq. 3 decision for one pixel: returns (g, tie, t)."""
    tie = ctypes.c_int(0)
    t = ctypes.c_double(0.0)
    g = _load().bnzref_decide(int(f), int(n), int(s1), int(s2), int(rule), float(k), float(R),
                              ctypes.byref(tie), ctypes.byref(t))
    return g, bool(tie.value), t.value


def threshold(f: np.ndarray, n, s1, s2, rule: int, k: float, R: float = 128.0):
    f = np.ascontiguousarray(f, dtype=np.uint8)
    h, w = f.shape
    n, s1, s2 = (np.ascontiguousarray(v, dtype=np.int64) for v in (n, s1, s2))
    out = np.empty((h, w), np.uint8)
    ties = ctypes.c_int64(0)
    _check(_load().bnzref_threshold(_ptr(f), _ptr(n), _ptr(s1), _ptr(s2), h, w, int(rule),
                                    float(k), float(R), _ptr(out), ctypes.byref(ties)))
    return out, int(ties.value)


def binarize(src: np.ndarray, W: int, rule: int, k: float, R: float = 128.0,
             method: int = SLIDING, threads: int = 1, packed: bool = False):
    """Full oracle pipeline; returns (mask, ties).  mask is {0,255} bytes or packed bits."""
    src, h, w, ch = _img(src)
    out = np.empty((h, w), np.uint8)
    ties = ctypes.c_int64(0)
    _check(_load().bnzref_binarize(_ptr(src), h, w, ch, w * ch, int(W), int(rule), float(k),
                                   float(R), int(method), _ptr(out), w, ctypes.byref(ties),
                                   int(threads)))
    if packed:
        out = pack(out)
    return out, int(ties.value)


def sauvola(src, W, k=0.5, R=128.0, **kw):
    return binarize(src, W, SAUVOLA, k, R, **kw)


def niblack(src, W, k=-0.2, **kw):
    return binarize(src, W, NIBLACK, k, 128.0, **kw)


def pixel(src: np.ndarray, W: int, rule: int, k: float, R: float, y: int, x: int):
    """One output pixel by the naive definition: returns (g, tie, t)."""
    src, h, w, ch = _img(src)
    tie = ctypes.c_int(0)
    t = ctypes.c_double(0.0)
    g = _load().bnzref_pixel(_ptr(src), h, w, ch, w * ch, int(W), int(rule), float(k), float(R),
                             int(y), int(x), ctypes.byref(tie), ctypes.byref(t))
    if g < 0:
        raise ValueError("bad pixel query")
    return g, bool(tie.value), t.value


def integral(f: np.ndarray):
    """(h+1)x(w+1) int64 summed-area tables of f and f^2."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    h, w = f.shape
    I1 = np.empty((h + 1, w + 1), np.int64)
    I2 = np.empty((h + 1, w + 1), np.int64)
    _check(_load().bnzref_integral(_ptr(f), h, w, _ptr(I1), _ptr(I2)))
    return I1, I2


def pack(mask: np.ndarray) -> np.ndarray:
    """1 bit per pixel, LSB = leftmost pixel, bit set <=> 255."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    h, w = mask.shape
    pb = (w + 7) // 8
    out = np.empty((h, pb), np.uint8)
    _check(_load().bnzref_pack(_ptr(mask), h, w, w, _ptr(out), pb))
    return out


def histogram(src: np.ndarray) -> np.ndarray:
    """256-bin histogram of the Eq. 1 gray page (uint64)."""
    src, h, w, ch = _img(src)
    hist = np.zeros(256, np.uint64)
    _check(_load().bnzref_histogram(_ptr(src), h, w, ch, w * ch, _ptr(hist)))
    return hist


def otsu_threshold(hist: np.ndarray):
    """Otsu's T from a 256-bin histogram: returns (T, q) with q[t] the fp64 criterion (-1: no split)."""
    hist = np.ascontiguousarray(hist, dtype=np.uint64)
    if hist.shape != (256,):
        raise ValueError("histogram must have 256 bins")
    q = np.empty(256, np.float64)
    T = _load().bnzref_otsu_threshold(_ptr(hist), _ptr(q))
    return int(T), q


def otsu(src: np.ndarray, packed: bool = False):
    """Eq. 2 with Otsu's T: returns (mask, T); mask {0,255} bytes or packed bits."""
    src, h, w, ch = _img(src)
    out = np.empty((h, w), np.uint8)
    T = ctypes.c_int(0)
    _check(_load().bnzref_otsu(_ptr(src), h, w, ch, w * ch, _ptr(out), w, ctypes.byref(T)))
    if packed:
        out = pack(out)
    return out, int(T.value)


# ---- reduced sets S' (Sec. 2, Eq. 5) and the F-measure (Eq. 6) ----------------

GS_FULL, GS_CROSS, GS_DIAGONALS, GS_STAR, GS_FRAME, GS_FRAME_CROSS, GS_FRAME_DIAGONALS = range(7)
GS_NAMES = {GS_FULL: "full", GS_CROSS: "cross", GS_DIAGONALS: "diagonals", GS_STAR: "star",
            GS_FRAME: "frame", GS_FRAME_CROSS: "frame+cross", GS_FRAME_DIAGONALS: "frame+diagonals"}


def gs_offsets(gs: int, W: int):
    """(dy, dx) offsets of the structure S' in the W x W window, row-major."""
    lib = _load()
    n = lib.bnzref_gs_offsets(int(gs), int(W), None, None, 0)
    if n < 0:
        raise ValueError("bad structure or window")
    dy = np.empty(n, np.int32)
    dx = np.empty(n, np.int32)
    lib.bnzref_gs_offsets(int(gs), int(W), _ptr(dy), _ptr(dx), n)
    return list(zip(dy.tolist(), dx.tolist()))


def gs_sums(f: np.ndarray, W: int, gs: int):
    """Exact (n', S1', S2') of every pixel over the in-image samples of S'."""
    f = np.ascontiguousarray(f, dtype=np.uint8)
    h, w = f.shape
    n = np.empty((h, w), np.int64)
    a = np.empty((h, w), np.int64)
    b = np.empty((h, w), np.int64)
    _check(_load().bnzref_gs_sums(_ptr(f), h, w, int(W), int(gs), _ptr(n), _ptr(a), _ptr(b)))
    return n, a, b


def gs_binarize(src: np.ndarray, W: int, gs: int, rule: int, k: float, R: float = 128.0):
    """Eq. 5 (Sauvola on m', s' with R' = R) or Niblack on m', s'; returns (mask, ties)."""
    src, h, w, ch = _img(src)
    out = np.empty((h, w), np.uint8)
    ties = ctypes.c_int64(0)
    _check(_load().bnzref_gs_binarize(_ptr(src), h, w, ch, w * ch, int(W), int(gs), int(rule), float(k),
                                      float(R), _ptr(out), w, ctypes.byref(ties)))
    return out, int(ties.value)


def gs_binarize_rows(src: np.ndarray, W: int, gs: int, rule: int, k: float, R: float, y0: int, y1: int):
    """Rows [y0, y1) of gs_binarize, computed on the band that holds their windows (same values:
    a pixel's samples lie within its window, and the band keeps every in-image row of it)."""
    h = src.shape[0]
    lo, hi = max(0, y0 - W // 2), min(h, y1 + (W - 1 - W // 2))
    out, _ = gs_binarize(np.ascontiguousarray(src[lo:hi]), W, gs, rule, k, R)
    return out[y0 - lo:y1 - lo]


def confusion(mask: np.ndarray, ref: np.ndarray, mask_ink: int = 0, ref_ink: int = 1):
    """(TP, FP, FN, TN) of mask against ref; a pixel is text where it equals the array's ink value."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    if mask.shape != ref.shape or mask.ndim != 2:
        raise ValueError("mask and reference must be equal-shaped 2-D arrays")
    h, w = mask.shape
    c = np.zeros(4, np.int64)
    _check(_load().bnzref_confusion(_ptr(mask), w, int(mask_ink), _ptr(ref), w, int(ref_ink), h, w, _ptr(c)))
    return tuple(int(v) for v in c)


def fmeasure(counts):
    """Eq. 6: FM = 2 R P / (R + P), R = TP/(TP+FN), P = TP/(TP+FP); returns (FM, R, P), 0 where undefined."""
    tp, fp, fn = counts[0], counts[1], counts[2]
    rec = tp / (tp + fn) if tp + fn else 0.0
    prec = tp / (tp + fp) if tp + fp else 0.0
    fm = 2.0 * rec * prec / (rec + prec) if rec + prec else 0.0
    return fm, rec, prec
