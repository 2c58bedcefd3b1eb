"""Serving loop: continuous batching of binarization requests on one GPU.

Requests (uint8 gray or RGB pages with their own W, rule, k, R) arrive at any
time through ``Server.submit``.  A scheduler thread

* admits waiting requests in arrival order while their device memory (input +
  output) fits the budget; a request that does not fit waits (it is never
  dropped) until finished requests release memory;
* copies each admitted page to the device on a copy stream;
* every step, launches one batched kernel (``bnz_batch_create_async``: one
  persistent launch over the step's pages, no allocation) over admitted pages
  whose input has arrived and that run on the same kernel instance (channels,
  rule, W mod 8; the oldest ready page picks it), so the copies of other
  pages overlap the kernel on their own streams.  One compute stream is the
  default: two batches of different instances running side by side thrash the
  SMs' instruction caches;
* copies finished masks back and completes the requests' futures, recording
  the latency from arrival to result.

With ``batched=False`` the same loop launches the plain single-page kernel
once per page on one compute stream: the per-image baseline.

The GPU operations live behind a small executor interface (``TorchExecutor``)
so the scheduling logic can be tested without a GPU.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    image: object            # uint8 HxW or HxWx3: host array/tensor (pinned for overlap), or a CUDA
                             # tensor with a 16-byte row pitch already resident in device memory
    W: int
    rule: str = "sauvola"
    k: float | None = None
    R: float = 128.0
    packed: bool = False
    timeout_s: float | None = None   # give up (TimeoutError) if not admitted within this time
    arrival: float = 0.0     # time.perf_counter() of arrival (submit stamps it when left 0)
    future: Future = field(default_factory=Future)
    # scheduler bookkeeping
    nbytes: int = 0
    slot: object = None
    stage: str = "waiting"
    done_at: float = 0.0

    @property
    def shape(self):
        return tuple(self.image.shape)


class Rejected(RuntimeError):
    """The request can never fit the device-memory budget."""


def request_bytes(h: int, w: int, ch: int, packed: bool = False, with_input: bool = True) -> int:
    """Device bytes a request holds: pitched input (unless already on the device) plus output."""
    pitch = (w * ch + 15) // 16 * 16 if with_input else 0
    out_pitch = (((w + 7) // 8 if packed else w) + 15) // 16 * 16
    return h * (pitch + out_pitch)


def on_device(img) -> bool:
    return bool(getattr(img, "is_cuda", False))


MAX_W = 255


def instance_key(req: Request) -> tuple:
    """The kernel instance a page runs on: channels, rule and W mod 8."""
    return (1 if len(req.shape) == 2 else 3, req.rule, req.W % 8)


def validate(req: Request) -> str | None:
    """Why a request cannot be served, or None."""
    shape = tuple(getattr(req.image, "shape", ()))
    if len(shape) not in (2, 3) or (len(shape) == 3 and shape[2] != 3):
        return f"image must be HxW (gray) or HxWx3 (RGB), got shape {shape}"
    if shape[0] < 1 or shape[1] < 1:
        return f"empty image {shape}"
    dt = getattr(req.image, "dtype", None)
    if str(dt) not in ("uint8", "torch.uint8"):
        return f"image must be uint8, got {dt}"
    if not (isinstance(req.W, int) and 1 <= req.W <= MAX_W):
        return f"W must be an integer in [1, {MAX_W}], got {req.W!r}"
    if req.rule not in ("sauvola", "niblack"):
        return f"rule must be 'sauvola' or 'niblack', got {req.rule!r}"
    if req.rule == "sauvola" and not (req.R > 0):
        return f"R must be > 0 for Sauvola, got {req.R!r}"
    return None


class Server:
    def __init__(self, executor, budget_bytes: int | None = None, max_batch: int = 64, poll_s: float = 50e-6):
        self.ex = executor
        if budget_bytes is None:
            budget_bytes = getattr(executor, "budget_bytes", 16 << 30)
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.poll_s = poll_s
        self.reserved = 0
        self.high_water = 0
        self.latencies: list[float] = []
        self.completed = 0
        self._waiting: collections.deque[Request] = collections.deque()
        self._lock = threading.Lock()
        self._admitted: list[Request] = []   # input copy in flight
        self._ready: list[Request] = []      # on the device, not launched
        self._steps: list[tuple[object, list[Request], object]] = []  # (event, requests, keep-alive)
        self._to_host: list[Request] = []                                # computed, mask copy not yet issued
        self._back: list[tuple[object, Request, object]] = []          # (event, request, host result)
        self._stop = threading.Event()
        self._thread: threading.Thread | None = None
        self.steps_launched = 0
        self._outstanding = 0                # submitted and not yet completed
        self.alloc_waits = 0                 # admissions deferred because the pool had no fitting range
        self.timed_out = 0
        self.cancelled = 0

    # ---- client side --------------------------------------------------------
    def submit(self, req: Request) -> Future:
        """Queue a request; malformed or over-budget requests fail their future at once (never the loop)."""
        problem = validate(req)
        if problem:
            req.future.set_exception(ValueError(problem))
            return req.future
        h, w = req.shape[:2]
        ch = 1 if len(req.shape) == 2 else 3
        req.nbytes = request_bytes(h, w, ch, req.packed, with_input=not on_device(req.image))
        if not req.arrival:        # a caller replaying a trace may stamp the scheduled arrival itself
            req.arrival = time.perf_counter()
        if req.nbytes > self.budget:
            req.future.set_exception(Rejected(f"a {h}x{w}x{ch} page needs {req.nbytes} bytes, "
                                              f"more than the {self.budget}-byte budget"))
            return req.future
        with self._lock:
            self._waiting.append(req)
            self._outstanding += 1
        return req.future

    def start(self):
        self._thread = threading.Thread(target=self._loop, name="bnz-serve", daemon=True)
        self._thread.start()
        return self

    def stop(self, drain: bool = True, timeout: float | None = None):
        if drain:
            t0 = time.perf_counter()
            while self.pending() and (timeout is None or time.perf_counter() - t0 < timeout):
                time.sleep(1e-3)
        self._stop.set()
        if self._thread:
            self._thread.join()

    def pending(self) -> int:
        """Requests submitted and not yet completed (safe to call from any thread)."""
        with self._lock:
            return self._outstanding

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return dict(completed=self.completed, steps=self.steps_launched, alloc_waits=self.alloc_waits,
                    timed_out=self.timed_out, cancelled=self.cancelled,
                    p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                    max_ms=float(lat.max() * 1e3), high_water_bytes=self.high_water)

    # ---- scheduler ----------------------------------------------------------
    def step(self) -> bool:
        """One scheduler iteration; returns True if anything moved."""
        moved = False
        # 1. admission, in arrival order, while the budget and the pool allow
        now = time.perf_counter()
        while True:
            with self._lock:
                if not self._waiting:
                    break
                req = self._waiting[0]
                if req.timeout_s is not None and now - req.arrival > req.timeout_s:
                    self._waiting.popleft()
                    self._outstanding -= 1
                    self.timed_out += 1
                    req.future.set_exception(TimeoutError(f"not admitted within {req.timeout_s} s"))
                    continue
                if req.future.cancelled():
                    self._waiting.popleft()
                    self._outstanding -= 1
                    self.cancelled += 1
                    continue
                if self.reserved + req.nbytes > self.budget:
                    break
            slot = self.ex.alloc(req)
            if slot is None:             # no free range fits (fragmentation, injected failure): wait
                self.alloc_waits += 1
                break
            with self._lock:
                self._waiting.popleft()
            if not req.future.set_running_or_notify_cancel():   # cancelled just now
                self.ex.release(slot)
                with self._lock:
                    self._outstanding -= 1
                self.cancelled += 1
                continue
            self.reserved += req.nbytes
            self.high_water = max(self.high_water, self.reserved)
            req.slot = slot
            req.h2d_event = self.ex.h2d(req.slot, req)
            req.stage = "h2d"
            self._admitted.append(req)
            moved = True
        # 2. inputs that have landed become launchable (copies complete in
        #    issue order: stop at the first one still in flight)
        n = 0
        for req in self._admitted:
            if not self.ex.done(req.h2d_event):
                break
            req.stage = "ready"
            self._ready.append(req)
            n += 1
        if n:
            del self._admitted[:n]
            moved = True
        # 3. launch one step over the ready pages
        if self._ready and self.ex.can_launch():
            # one kernel instance per step (channels, rule, W mod 8), picked by the oldest ready page:
            # launches that mix instances thrash the SMs' instruction caches
            want = instance_key(self._ready[0])
            batch, rest = [], []
            for r in self._ready:
                (batch if len(batch) < self.max_batch and instance_key(r) == want else rest).append(r)
            self._ready = rest
            event, keep = self.ex.launch([r.slot for r in batch])
            for r in batch:
                r.stage = "running"
            self._steps.append((event, batch, keep))
            self.steps_launched += 1
            moved = True
        # 4. finished steps: results back to the host (in order; a request that finds no host
        #    memory for its mask waits in _to_host and is retried after deliveries free some)
        still_steps = []
        for event, batch, keep in self._steps:
            if self.ex.done(event):
                self._to_host.extend(batch)
                moved = True
            else:
                still_steps.append((event, batch, keep))
        self._steps = still_steps
        n = 0
        for r in self._to_host:
            got = self.ex.d2h(r.slot)
            if got is None:
                break
            ev, host = got
            r.stage = "d2h"
            self._back.append((ev, r, host))
            n += 1
        if n:
            del self._to_host[:n]
            moved = True
        # 5. delivered results (in issue order): complete, release memory
        n = 0
        for ev, r, host in self._back:
            if not self.ex.done(ev):
                break
            r.done_at = time.perf_counter()
            self.latencies.append(r.done_at - r.arrival)
            self.ex.release(r.slot)
            r.slot = None
            self.reserved -= r.nbytes
            self.completed += 1
            with self._lock:
                self._outstanding -= 1
            r.stage = "done"
            r.future.set_result(host)
            n += 1
        if n:
            del self._back[:n]
            moved = True
        return moved

    def _loop(self):
        while not self._stop.is_set():
            if not self.step():
                time.sleep(self.poll_s)


class _Block:
    """Owner of one arena block; numpy arrays over it keep it alive, the last one frees it."""

    def __init__(self, pool, ptr: int, h: int, w: int):
        self._pool, self.ptr = pool, ptr
        self.__array_interface__ = {"shape": (h, w), "typestr": "|u1", "data": (ptr, False), "version": 3}

    def __del__(self):
        try:
            self._pool.free(self.ptr)
        except Exception:
            pass


class HostArena:
    """Pinned host memory reserved once and carved by the native pool bookkeeping: mask buffers for the
    serving loops without a cudaHostAlloc per request.  Blocks are numpy arrays whose base object returns
    the memory when the last array viewing it goes away."""

    def __init__(self, nbytes: int):
        import torch
        from . import Pool
        self.buf = torch.empty((int(nbytes),), dtype=torch.uint8, pin_memory=True)
        self.pool = Pool(self.buf)

    def take(self, h: int, w: int, wait_s: float = 60.0) -> np.ndarray | None:
        """An (h, w) uint8 array in pinned memory.  While the arena is full it waits up to wait_s
        (wait_s = 0: returns None at once), then raises MemoryError."""
        t0 = time.perf_counter()
        while True:
            ptr = self.pool.alloc(h * w)
            if ptr is not None:
                break
            if wait_s == 0:
                return None
            if time.perf_counter() - t0 > wait_s:
                raise MemoryError(f"host arena full for {wait_s} s")
            time.sleep(1e-4)
        return np.asarray(_Block(self.pool, ptr, h, w))


class NativeServer:
    """The same service on the library's native engine (`bnz_server_*`): admission, batching, copies and
    completion detection run in a C++ scheduler thread; Python only submits requests and completes futures.

    Inputs: host arrays/tensors (pinned ones overlap with the GPU) or CUDA tensors already on the device
    (16-byte row pitch).  Masks land in a pinned host arena; the futures return numpy arrays over it."""

    def __init__(self, budget_bytes: int = 16 << 30, max_batch: int = 16, batched: bool = True,
                 compute_streams: int = 1, host_bytes: int = 4 << 30, inject_timeout_every: int = 0,
                 host_arena: HostArena | None = None):
        import ctypes
        from . import _check, bnz_server_config, load
        # host_arena: a caller-owned arena shared by several servers (one pinned reservation; submit waits
        # while it is full, so it should hold the masks of every request in flight)
        self.host = host_arena if host_arena is not None else HostArena(host_bytes)
        self._ct = ctypes
        self._lib = load()
        self.budget = int(budget_bytes)
        # inject_timeout_every (testing): every n-th launch step is reported as timed out by the engine
        cfg = bnz_server_config(self.budget, int(max_batch), int(compute_streams), 1 if batched else 0,
                                int(inject_timeout_every))
        h = ctypes.c_void_p(None)
        _check(self._lib.bnz_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._lock = threading.Lock()
        self._live: dict[int, tuple] = {}   # tag -> (future, output, input kept alive)
        self._tag = 0
        self.latencies: list[float] = []
        self.failed = 0
        self._stop = threading.Event()
        self._poller = threading.Thread(target=self._poll_loop, name="bnz-native-poll", daemon=True)
        self._poller.start()

    def submit(self, req: Request) -> Future:
        import torch
        from . import BNZ_NIBLACK, BNZ_SAUVOLA, BnzError, bnz_request
        problem = validate(req)
        if problem:
            req.future.set_exception(ValueError(problem))
            return req.future
        img = req.image if isinstance(req.image, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(req.image))
        h, w = img.shape[:2]
        ch = 1 if img.dim() == 2 else 3
        if (w > 1 and img.stride(1) != ch) or (ch == 3 and img.stride(2) != 1):
            img = img.contiguous()
        pitch = img.stride(0) if h > 1 else w * ch
        ow = (w + 7) // 8 if req.packed else w
        out = self.host.take(h, ow)
        k = req.k if req.k is not None else (0.5 if req.rule == "sauvola" else -0.2)
        with self._lock:
            self._tag += 1
            tag = self._tag
            self._live[tag] = (req.future, out, img)
        r = bnz_request(img.data_ptr(), pitch, 1 if img.is_cuda else 0, h, w, ch, req.W,
                        BNZ_SAUVOLA if req.rule == "sauvola" else BNZ_NIBLACK, float(k), float(req.R),
                        1 if req.packed else 0, out.ctypes.data, ow, tag)
        rc = self._lib.bnz_server_submit(self._h, self._ct.byref(r))
        if rc != 0:
            with self._lock:
                self._live.pop(tag, None)
            from . import bnz_last_error
            req.future.set_exception(BnzError(rc, bnz_last_error()))
        return req.future

    def _poll_loop(self):
        ct = self._ct
        n = 256
        tags = (ct.c_ulonglong * n)()
        st = (ct.c_int * n)()
        lat = (ct.c_double * n)()
        while not self._stop.is_set():
            got = self._lib.bnz_server_poll(self._h, tags, st, lat, n, 20)  # releases the GIL while waiting
            for i in range(max(got, 0)):
                with self._lock:
                    fut, out, _ = self._live.pop(tags[i])
                if st[i] == 0:
                    self.latencies.append(lat[i])
                    fut.set_result(out)
                else:
                    self.failed += 1
                    fut.set_exception(RuntimeError(f"request failed with status {st[i]}: {self.error()}"))

    def error(self) -> str:
        buf = self._ct.create_string_buffer(512)
        self._lib.bnz_server_error(self._h, buf, 512)
        return buf.value.decode(errors="replace")

    def pending(self) -> int:
        with self._lock:
            return len(self._live)

    def stats(self) -> dict:
        if not self._h:
            return dict(self._final)
        ct = self._ct
        o, c, s_, a = ct.c_longlong(0), ct.c_longlong(0), ct.c_longlong(0), ct.c_longlong(0)
        hw = ct.c_size_t(0)
        self._lib.bnz_server_stats(self._h, ct.byref(o), ct.byref(c), ct.byref(s_), ct.byref(a), ct.byref(hw))
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return dict(completed=c.value, steps=s_.value, alloc_waits=a.value, high_water_bytes=hw.value,
                    failed=self.failed, p50_ms=float(np.percentile(lat, 50) * 1e3),
                    p99_ms=float(np.percentile(lat, 99) * 1e3), max_ms=float(lat.max() * 1e3))

    def stop(self, drain: bool = True, timeout: float | None = None):
        if drain:
            t0 = time.perf_counter()
            while self.pending() and (timeout is None or time.perf_counter() - t0 < timeout):
                time.sleep(1e-3)
        self._stop.set()
        self._poller.join()
        if self._h:
            self._final = self.stats()
            self._lib.bnz_server_destroy(self._h)
            self._h = None


class TorchExecutor:
    """GPU side of the server: torch memory and streams, the bnz kernels."""

    def __init__(self, batched: bool = True, compute_streams: int = 1, tile_table=None, device="cuda",
                 budget_bytes: int = 16 << 30, host_bytes: int = 4 << 30):
        import torch
        from . import BNZ_NIBLACK, BNZ_SAUVOLA, Batch, Pool, bnz_binarize_dev, bnz_copy2d_async, load
        from .tune import tile_for
        load()
        self.torch = torch
        self.dev = torch.device(device)
        # the whole budget is reserved once; requests get their buffers from the pool over it
        self.budget_bytes = int(budget_bytes)
        self.arena = torch.empty((self.budget_bytes,), dtype=torch.uint8, device=self.dev)
        self.pool = Pool(self.arena)
        self.host = HostArena(host_bytes)
        self.batched = batched
        self.copy_in = torch.cuda.Stream(self.dev)
        self.copy_out = torch.cuda.Stream(self.dev)
        self.compute = [torch.cuda.Stream(self.dev) for _ in range(max(1, compute_streams if batched else 1))]
        self._rr = 0
        self._inflight = [None] * len(self.compute)
        self._Batch = Batch
        self._single = bnz_binarize_dev
        self._copy2d = bnz_copy2d_async
        self._rules = {"sauvola": BNZ_SAUVOLA, "niblack": BNZ_NIBLACK}
        self._table = tile_table
        self._tile_for = tile_for

    def alloc(self, req):
        """Input (unless resident) and output buffers, 16-byte row pitch, in one pool block; None if none fits."""
        h, w = req.shape[:2]
        ch = 1 if len(req.shape) == 2 else 3
        resident = on_device(req.image)
        pin = 0 if resident else (w * ch + 15) // 16 * 16
        ow = (w + 7) // 8 if req.packed else w
        pout = (ow + 15) // 16 * 16
        off_out = (h * pin + 255) // 256 * 256
        ptr = self.pool.alloc(off_out + h * pout)
        if ptr is None:
            return None
        off = ptr - self.pool.base
        st = self.torch.as_strided
        if resident:
            src = req.image
        elif ch == 1:
            src = st(self.arena, (h, w), (pin, 1), off)
        else:
            src = st(self.arena, (h, w, 3), (pin, 3, 1), off)
        dst = st(self.arena, (h, ow), (pout, 1), off + off_out)
        return dict(req=req, src=src, dst=dst, ch=ch, ptr=ptr)

    def h2d(self, slot, req):
        torch = self.torch
        if on_device(req.image):
            # already in device memory: order after the work queued so far on the producer's stream
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream(self.dev))
            return ev
        img = req.image if isinstance(req.image, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(req.image))
        h, w = img.shape[:2]
        ch = slot["ch"]
        # any row pitch on the host (a crop of a larger pinned canvas, say); rows themselves dense
        if (w > 1 and img.stride(1) != ch) or (ch == 3 and img.stride(2) != 1):
            img = img.contiguous()
        row = w * ch
        src = slot["src"]
        self._copy2d(src.data_ptr(), src.stride(0), img.data_ptr(), img.stride(0) if h > 1 else row, row, h,
                     self.copy_in)
        ev = torch.cuda.Event()
        ev.record(self.copy_in)
        slot["host_in"] = img      # kept alive until the copy has completed
        return ev

    def done(self, ev) -> bool:
        return ev.query()

    def can_launch(self) -> bool:
        # at most one step in flight per compute stream
        s = self._inflight[self._rr]
        return s is None or s.query()

    def launch(self, slots):
        torch = self.torch
        stream = self.compute[self._rr]
        self._rr = (self._rr + 1) % len(self.compute)
        keep = []
        with torch.cuda.stream(stream):
            if self.batched:
                pages = []
                for sl in slots:
                    r = sl["req"]
                    k = r.k if r.k is not None else (0.5 if r.rule == "sauvola" else -0.2)
                    tw = self._tile_for(self._table, sl["ch"], r.W) if self._table else 0
                    pages.append(dict(src=sl["src"], dst=sl["dst"], W=r.W, rule=r.rule, k=k, R=r.R,
                                      packed=r.packed, tile_w=tw))
                # descriptors in stream-ordered torch memory: no cudaMalloc once the cache is warm
                desc = torch.empty(((self._Batch.desc_bytes(len(pages)) + 7) // 8,), dtype=torch.int64,
                                   device=self.dev)
                b = self._Batch(pages, desc_buffer=desc, stream=stream)
                b.run(stream)
                keep += [b, desc]
            else:
                for sl in slots:
                    r = sl["req"]
                    k = r.k if r.k is not None else (0.5 if r.rule == "sauvola" else -0.2)
                    self._single(sl["src"], r.W, self._rules[r.rule], k, r.R, sl["dst"], packed=r.packed,
                                 stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self._inflight[(self._rr - 1) % len(self.compute)] = ev
        return ev, keep

    def d2h(self, slot):
        torch = self.torch
        dst = slot["dst"]
        h, wb = dst.shape
        host = self.host.take(h, wb, wait_s=0)
        if host is None:  # host arena full: the scheduler retries once delivered results free some
            return None
        self._copy2d(host.ctypes.data, wb, dst.data_ptr(), dst.stride(0) if h > 1 else wb, wb, h, self.copy_out)
        ev = torch.cuda.Event()
        ev.record(self.copy_out)
        slot["host_out"] = host
        return ev, host

    def release(self, slot):
        self.pool.free(slot["ptr"])
        slot.clear()
