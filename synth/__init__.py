"""Seeded synthetic document pages and workload recipes.

Shared input generator for the oracle tests, the GPU tests and the bench.  It
holds none of the binarization arithmetic (no gray conversion, no window
sums, no thresholds).  Pages come from ``synth.c`` (counter-based random
draws, so the result does not depend on the thread count); workload recipes
(uneven batches, serving traces) use numpy's PCG64 seeded generator.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

DOC = 0        # gradient 90->220, strokes ~40, sigma 8
STAINS = 1     # DOC plus coloured stains and low-frequency blotches
VIGNETTE = 2   # strong vignetting, sigma 15


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_SRC) > os.path.getmtime(_LIB):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.synth_page.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_longlong, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            _lib = lib
    return _lib


def page(h: int, w: int, seed: int, profile: int = DOC, channels: int = 1,
         random_dir: bool = False, ground_truth: bool = False, threads: int | None = None,
         out: np.ndarray | None = None):
    """Return an HxW (gray) or HxWx3 (RGB) uint8 page; optionally the stroke mask too.

    ``out`` may be a preallocated C-contiguous array of the right shape (for
    example pinned host memory viewed through numpy).
    """
    shape = (h, w) if channels == 1 else (h, w, 3)
    if out is None:
        out = np.empty(shape, np.uint8)
    assert out.shape == shape and out.dtype == np.uint8 and out.flags.c_contiguous
    gt = np.empty((h, w), np.uint8) if ground_truth else None
    threads = threads or os.cpu_count() or 1
    rc = _load().synth_page(out.ctypes.data, h, w, channels, w * channels, seed & (2**64 - 1),
                            profile, 1 if random_dir else 0,
                            gt.ctypes.data if gt is not None else None, threads)
    if rc != 0:
        raise ValueError(f"synth_page failed ({rc})")
    return (out, gt) if ground_truth else out


def batch_specs(n: int, seed: int, w_range=(600, 2480), h_range=(800, 3508),
                windows=(15, 25, 45, 75)):
    """Uneven page batch: widths/heights uniform in the ranges, W drawn from ``windows``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ws = rng.integers(w_range[0], w_range[1] + 1, n)
    hs = rng.integers(h_range[0], h_range[1] + 1, n)
    Ws = rng.choice(np.asarray(windows), n)
    return [dict(h=int(h), w=int(w), W=int(W), seed=int(seed) * 1000003 + i)
            for i, (h, w, W) in enumerate(zip(hs, ws, Ws))]


def serve_trace(n: int, seed: int, rate_per_s: float, w_range=(600, 4960), h_range=(800, 7016),
                W_range=(15, 101)):
    """Poisson arrivals of RGB pages with mixed sizes, odd W and mixed rules."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, n)
    t = np.cumsum(gaps) - gaps[0]
    ws = rng.integers(w_range[0], w_range[1] + 1, n)
    hs = rng.integers(h_range[0], h_range[1] + 1, n)
    lo, hi = W_range
    Ws = 2 * rng.integers(lo // 2, hi // 2 + 1, n) + 1
    rules = rng.integers(0, 2, n)
    out = []
    for i in range(n):
        rule = "sauvola" if rules[i] == 0 else "niblack"
        out.append(dict(t=float(t[i]), h=int(hs[i]), w=int(ws[i]), W=int(Ws[i]), rule=rule,
                        k=0.5 if rule == "sauvola" else -0.2, R=128.0,
                        seed=int(seed) * 7919 + i))
    return out
