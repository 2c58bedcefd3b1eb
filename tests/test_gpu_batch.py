"""Batched persistent launch over uneven pages (with and without a CUDA graph):
every page's mask equals the single-page launch's and the oracle's."""
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


def make_pages(bnz, specs):
    pages, hosts = [], []
    for i, (h, w, ch, W, rule, packed, tile_w) in enumerate(specs):
        img = synth.page(h, w, 500 + i, synth.STAINS if ch == 3 else synth.DOC, ch, random_dir=True)
        hosts.append(img)
        pages.append(dict(src=bnz.to_device_pitched(img), dst=bnz.alloc_pitched(h, (w + 7) // 8 if packed else w),
                          W=W, rule=rule, k=0.5 if rule == "sauvola" else -0.2, packed=packed, tile_w=tile_w))
    return pages, hosts


SPECS = [(800, 600, 1, 15, "sauvola", False, 0), (1203, 977, 1, 25, "sauvola", False, 256),
         (35, 2100, 3, 45, "niblack", False, 0), (640, 480, 3, 75, "sauvola", True, 0),
         (1, 1, 1, 3, "sauvola", False, 0), (2000, 31, 1, 101, "niblack", True, 128),
         (517, 1333, 3, 31, "sauvola", False, 512), (999, 1001, 1, 254, "sauvola", False, 512)]


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_single_page_and_oracle(bnz, use_graph):
    pages, hosts = make_pages(bnz, SPECS)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    b = bnz.Batch(pages, use_graph=use_graph, d_stats=stats)
    info = b.info()
    assert info["pages"] == len(SPECS) and info["launches"] == 2
    for rep in range(2):  # a second run (graph replay) gives the same bytes
        for pg in pages:
            pg["dst"].fill_(7)
        b.run()
        torch.cuda.synchronize()
        assert int(stats[2]) == 0
        for pg, img, (h, w, ch, W, rule, packed, _) in zip(pages, hosts, SPECS):
            got = pg["dst"].cpu().numpy()
            single = bnz.binarize(pg["src"], W, rule, pg["k"], packed=packed).cpu().numpy()
            np.testing.assert_array_equal(got, single)
            rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
            ref, _ = oracle.binarize(img, W, rid, pg["k"], 128.0, threads=NTHREADS, packed=packed)
            np.testing.assert_array_equal(got, ref)
    b.close()


def test_async_batch_in_caller_memory_on_a_stream(bnz):
    """bnz_batch_create_async: descriptors uploaded into caller memory on the stream the batch then runs on."""
    pages, hosts = make_pages(bnz, SPECS)
    stream = torch.cuda.Stream()
    desc = bnz.alloc_scratch(bnz.Batch.desc_bytes(len(pages)))
    assert desc.data_ptr() % 128 == 0
    with pytest.raises(bnz.BnzError) as e:  # too small a descriptor buffer
        bnz.Batch(pages, desc_buffer=desc[:1], stream=stream)
    assert e.value.status == bnz.BNZ_EINVAL
    torch.cuda.synchronize()
    b = bnz.Batch(pages, desc_buffer=desc, stream=stream)
    assert b.info()["launches"] == 2
    b.run(stream)
    stream.synchronize()
    for pg, img, (h, w, ch, W, rule, packed, _) in zip(pages, hosts, SPECS):
        rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
        ref, _ = oracle.binarize(img, W, rid, pg["k"], 128.0, threads=NTHREADS, packed=packed)
        np.testing.assert_array_equal(pg["dst"].cpu().numpy(), ref)
    b.close()


def test_copy2d_round_trip(bnz):
    host = torch.from_numpy(np.arange(37 * 53, dtype=np.int64).astype(np.uint8).reshape(37, 53)).pin_memory()
    dev = bnz.alloc_pitched(37, 53)
    s = torch.cuda.Stream()
    bnz.bnz_copy2d_async(dev.data_ptr(), dev.stride(0), host.data_ptr(), 53, 53, 37, s)
    back = torch.empty((37, 53), dtype=torch.uint8, pin_memory=True)
    bnz.bnz_copy2d_async(back.data_ptr(), 53, dev.data_ptr(), dev.stride(0), 53, 37, s)
    s.synchronize()
    assert torch.equal(back, host) and torch.equal(dev.cpu(), host)
    with pytest.raises(bnz.BnzError):
        bnz.bnz_copy2d_async(dev.data_ptr(), 16, host.data_ptr(), 53, 53, 37, s)


def test_batch_rejects_a_bad_page(bnz):
    pages, _ = make_pages(bnz, SPECS[:3])
    pages[1]["W"] = 0
    with pytest.raises(bnz.BnzError) as e:
        bnz.Batch(pages)
    assert e.value.status == bnz.BNZ_EINVAL and "page 1" in str(e.value)


def test_autotuner_table_and_lookup(bnz, tmp_path, monkeypatch):
    from paper_1210_3165_gb300 import tune
    monkeypatch.setenv("BNZ_TUNE_CACHE", str(tmp_path / "t.json"))
    table = tune.tune(windows=(15, 101), channels=(1,), shape=(512, 1024), reps=3)
    assert set(table["1"]) == {"15", "101"}
    assert all(v["tile_w"] in (128, 256, 512) and v["tile_h"] in tune.TILE_HEIGHTS and
               v["edge_weight"] in tune.EDGE_WEIGHTS for v in table["1"].values())
    assert table["build"] == tune.build_key()
    assert tune.load_table() == table
    assert tune.tile_for(table, 1, 17) == table["1"]["15"]["tile_w"]
    t = tune.tile_shape_for(table, 1, 17)
    e = table["1"]["15"]
    assert (t.tile_w, t.tile_h, t.edge_weight) == (e["tile_w"], e["tile_h"], e["edge_weight"])
    assert tune.tile_for(None, 1, 17) == 0 and tune.tile_shape_for(None, 1, 17) is None
    # the tuned shape gives the oracle's mask
    img = synth.page(700, 1100, 5, synth.DOC, 1)
    got = bnz.binarize(bnz.to_device_pitched(img), 15, "sauvola", 0.5, 128.0, tile=t).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.sauvola(img, 15, 0.5, 128.0)[0])


def test_async_batch_many_descriptors(bnz):
    """More descriptors than one upload kernel carries in its parameters: every page still gets its own."""
    specs = [(40 + 7 * i, 50 + 11 * i, 1 + 2 * (i % 2), 3 + 2 * (i % 9), "sauvola" if i % 3 else "niblack", False, 0)
             for i in range(29)]
    pages, hosts = make_pages(bnz, specs)
    stream = torch.cuda.Stream()
    desc = bnz.alloc_scratch(bnz.Batch.desc_bytes(len(pages)))
    b = bnz.Batch(pages, desc_buffer=desc, stream=stream)
    b.run(stream)
    stream.synchronize()
    for pg, img, (h, w, ch, W, rule, packed, _) in zip(pages, hosts, specs):
        rid = oracle.SAUVOLA if rule == "sauvola" else oracle.NIBLACK
        ref, _ = oracle.binarize(img, W, rid, pg["k"], 128.0, threads=NTHREADS, packed=packed)
        np.testing.assert_array_equal(pg["dst"].cpu().numpy(), ref)
    b.close()
