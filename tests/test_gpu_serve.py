"""Serving loop on the GPU: every request's mask, served in a mix of uneven
pages with other windows and rules, equals the same page binarized alone and
the oracle's mask."""
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


def mix(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        h, w = int(rng.integers(1, 700)), int(rng.integers(1, 900))
        ch = 3 if i % 3 == 0 else 1
        W = int(rng.choice([3, 15, 31, 61, 101]))
        rule = "sauvola" if i % 2 == 0 else "niblack"
        packed = i % 5 == 4
        img = synth.page(h, w, 900 + i, synth.STAINS if ch == 3 else synth.DOC, ch, random_dir=True)
        out.append((img, W, rule, packed))
    return out


@pytest.mark.parametrize("batched", [True, False])
def test_served_masks_equal_alone_and_oracle(bnz, batched):
    from paper_1210_3165_gb300.serve import Request, Server, TorchExecutor
    items = mix(30, 7)
    # a budget that holds only a few pages at a time, so admission has to wait
    ex = TorchExecutor(batched=batched, compute_streams=2, budget_bytes=4 << 20)
    srv = Server(ex, max_batch=8).start()
    futs = []
    for i, (img, W, rule, packed) in enumerate(items):
        # most pages come from pinned host memory, every fourth is already resident on the device
        src = bnz.to_device_pitched(img) if i % 4 == 3 else torch.from_numpy(img).pin_memory()
        futs.append(srv.submit(Request(image=src, W=W, rule=rule, packed=packed)))
    srv.stop(drain=True, timeout=120)
    assert srv.reserved == 0 and srv.high_water <= 4 << 20
    st = ex.pool.stats()
    assert st["used"] == 0 and st["high_water"] <= 4 << 20
    for (img, W, rule, packed), f in zip(items, futs):
        got = np.asarray(f.result(timeout=0))
        k = 0.5 if rule == "sauvola" else -0.2
        alone = bnz.binarize(bnz.to_device_pitched(img), W, rule, k, packed=packed).cpu().numpy()
        np.testing.assert_array_equal(got, alone)
        rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
        ref, _ = oracle.binarize(img, W, rid, k, 128.0, threads=NTHREADS, packed=packed)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("batched", [True, False])
def test_native_server_masks_equal_alone_and_oracle(bnz, batched):
    """The C++ serving engine: same mix, same budget pressure, same bits."""
    from paper_1210_3165_gb300.serve import NativeServer, Request
    items = mix(30, 11)
    srv = NativeServer(budget_bytes=4 << 20, max_batch=8, batched=batched, compute_streams=2)
    futs = []
    for i, (img, W, rule, packed) in enumerate(items):
        src = bnz.to_device_pitched(img) if i % 4 == 3 else torch.from_numpy(img).pin_memory()
        futs.append(srv.submit(Request(image=src, W=W, rule=rule, packed=packed)))
    too_big = srv.submit(Request(image=np.zeros((4000, 4000), np.uint8), W=15))
    bad = srv.submit(Request(image=np.zeros((10, 10), np.uint8), W=300))
    srv.stop(drain=True, timeout=120)
    with pytest.raises(bnz.BnzError):
        too_big.result(timeout=0)
    with pytest.raises(ValueError):
        bad.result(timeout=0)
    st = srv.stats()
    assert st["completed"] == len(items) and st["failed"] == 0 and st["high_water_bytes"] <= 4 << 20
    for (img, W, rule, packed), f in zip(items, futs):
        got = np.asarray(f.result(timeout=0))
        k = 0.5 if rule == "sauvola" else -0.2
        alone = bnz.binarize(bnz.to_device_pitched(img), W, rule, k, packed=packed).cpu().numpy()
        np.testing.assert_array_equal(got, alone)
        rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
        ref, _ = oracle.binarize(img, W, rid, k, 128.0, threads=NTHREADS, packed=packed)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("rule,W", [("sauvola", 101), ("niblack", 15)])
def test_native_server_full_size_page(bnz, rule, W):
    """The largest page of the serving workload (7016 x 4960 RGB, 104 MB) through the native engine, once from
    pinned host memory and once resident on the device, equals the oracle bit for bit."""
    from paper_1210_3165_gb300.serve import NativeServer, Request
    img = synth.page(7016, 4960, 31, synth.STAINS, 3, random_dir=True)
    k = 0.5 if rule == "sauvola" else -0.2
    rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
    ref, _ = oracle.binarize(img, W, rid, k, 128.0, threads=NTHREADS)
    srv = NativeServer(budget_bytes=1 << 30, max_batch=4)
    f_host = srv.submit(Request(image=torch.from_numpy(img).pin_memory(), W=W, rule=rule, k=k))
    f_dev = srv.submit(Request(image=bnz.to_device_pitched(img), W=W, rule=rule, k=k))
    got_host, got_dev = np.asarray(f_host.result(timeout=120)), np.asarray(f_dev.result(timeout=120))
    srv.stop()
    np.testing.assert_array_equal(got_host, ref)
    np.testing.assert_array_equal(got_dev, ref)


@pytest.mark.parametrize("batched", [True, False])
def test_native_server_step_timeout_fails_its_requests(bnz, batched):
    """A launch step whose kernels report a timed-out wait (injected on the host: the engine's test hook
    marks every second step) fails exactly its own requests with BNZ_ETIMEOUT; the other requests still
    return the oracle's masks."""
    from paper_1210_3165_gb300.serve import NativeServer, Request
    items = mix(12, 23)
    srv = NativeServer(budget_bytes=64 << 20, max_batch=1, batched=batched, inject_timeout_every=2)
    futs = [srv.submit(Request(image=torch.from_numpy(img).pin_memory(), W=W, rule=rule, packed=packed))
            for img, W, rule, packed in items]
    srv.stop(drain=True, timeout=120)
    failed = ok = 0
    for (img, W, rule, packed), f in zip(items, futs):
        err = f.exception(timeout=0)
        if err is not None:
            assert "status 4" in str(err) and "timed out" in str(err)
            failed += 1
            continue
        k = 0.5 if rule == "sauvola" else -0.2
        rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
        ref, _ = oracle.binarize(img, W, rid, k, 128.0, threads=NTHREADS, packed=packed)
        np.testing.assert_array_equal(np.asarray(f.result(timeout=0)), ref)
        ok += 1
    # one request per step (max_batch 1): every second step, so half the requests, fail
    assert failed == len(items) // 2 and ok == len(items) - failed
