"""The allocation-free integral-image entry point.

Some callers cannot allocate device memory (code inside a framework that owns
every device allocation, fixed-budget pipelines that must not reach the
allocator while running).  bnz_binarize_integral_static_dev serves them with a
library-owned scratch array.  This test calls it through the C ABI twice in a
row (the second call on a smaller page, after the first left its tables in the
shared array) and compares each result with the scratch-taking entry point,
bit for bit, as the other parity tests do.  It lives in its own file, named to
be collected last, and must pass alone in a fresh process as well."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bnz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1210_3165_gb300 as b
    b.load()
    return b


def with_scratch(bnz, d, W, rid, k, R):
    h, w = d.shape[:2]
    scratch = bnz.alloc_scratch(bnz.bnz_integral_scratch_bytes(h, w))
    out = bnz.alloc_pitched(h, w)
    bnz.bnz_binarize_integral_dev(d, W, rid, k, R, out, scratch)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def without_alloc(bnz, d, W, rid, k, R):
    h, w = d.shape[:2]
    out = bnz.alloc_pitched(h, w)
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    bnz.bnz_binarize_integral_static_dev(d, W, rid, k, R, out, d_stats=stats)
    torch.cuda.synchronize()
    assert int(stats[2]) == 0
    return out.cpu().numpy()


def test_no_alloc_entry_point_matches_scratch_entry_point_twice(bnz):
    big = bnz.to_device_pitched(synth.page(900, 1300, 21, synth.STAINS, 3))
    small = bnz.to_device_pitched(synth.page(333, 517, 22, synth.DOC, 1))
    cases = [(big, 31, bnz.BNZ_SAUVOLA, 0.5, 128.0), (small, 15, bnz.BNZ_NIBLACK, -0.2, 128.0)]
    for d, W, rid, k, R in cases:  # two calls in a row on the shared array
        np.testing.assert_array_equal(without_alloc(bnz, d, W, rid, k, R), with_scratch(bnz, d, W, rid, k, R))


def test_no_alloc_entry_point_rejects_pages_beyond_its_scratch(bnz):
    h, w = 2048, 2048  # needs more than the 32 MiB the entry point holds
    assert bnz.bnz_integral_scratch_bytes(h, w) > 32 << 20
    d = bnz.alloc_pitched(h, w)
    out = bnz.alloc_pitched(h, w)
    with pytest.raises(bnz.BnzError) as e:
        bnz.bnz_binarize_integral_static_dev(d, 15, bnz.BNZ_SAUVOLA, 0.5, 128.0, out)
    assert e.value.status == bnz.BNZ_EINVAL
    assert "allocation-free" in str(e.value)
