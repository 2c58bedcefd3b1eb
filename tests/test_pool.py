"""Device-memory pool bookkeeping through the C-ABI, on the CPU: the pool
never touches its range, so a fake base address serves."""
import random

import pytest

import paper_1210_3165_gb300 as bnz

BASE = 1 << 40   # never dereferenced


@pytest.fixture
def pool():
    p = bnz.Pool(BASE, 1 << 20)
    yield p
    p.close()


def test_alloc_aligned_disjoint_and_coalescing(pool):
    rng = random.Random(3)
    live = {}
    for it in range(3000):
        if live and (rng.random() < 0.45 or len(live) > 60):
            a = rng.choice(list(live))
            pool.free(a)
            del live[a]
        else:
            n = rng.choice([1, 255, 256, 257, 4096, rng.randrange(1, 40000)])
            a = pool.alloc(n)
            if a is None:
                # ENOMEM only when no free range fits the rounded size
                assert pool.stats()["largest_free"] < (n + 255) // 256 * 256
                continue
            assert a % 256 == 0 and BASE <= a and a + n <= BASE + (1 << 20)
            live[a] = (n + 255) // 256 * 256
        spans = sorted(live.items())
        for (a0, n0), (a1, _) in zip(spans, spans[1:]):
            assert a0 + n0 <= a1, "live blocks overlap"
        st = pool.stats()
        assert st["used"] == sum(live.values()) and st["live"] == len(live)
    for a in list(live):
        pool.free(a)
    st = pool.stats()
    assert st["used"] == 0 and st["largest_free"] == 1 << 20  # fully coalesced again
    assert 0 < st["high_water"] <= 1 << 20


def test_enomem_then_free_makes_room(pool):
    a = pool.alloc(600 << 10)
    assert a == BASE
    assert pool.alloc(600 << 10) is None
    pool.free(a)
    assert pool.alloc(600 << 10) == BASE


def test_first_fit_reuses_the_lowest_hole(pool):
    a, b, c = pool.alloc(1000), pool.alloc(1000), pool.alloc(1000)
    pool.free(a)
    pool.free(c)
    assert pool.alloc(512) == a


def test_injected_failures_and_bad_frees(pool):
    pool.fail_next(2)
    assert pool.alloc(16) is None and pool.alloc(16) is None
    a = pool.alloc(16)
    assert a is not None
    with pytest.raises(bnz.BnzError) as e:
        pool.free(a + 256)
    assert e.value.status == bnz.BNZ_EINVAL
    pool.free(a)
    with pytest.raises(bnz.BnzError):
        pool.free(a)          # double free


def test_create_rejects_unaligned_base():
    with pytest.raises(bnz.BnzError) as e:
        bnz.Pool(BASE + 16, 4096)
    assert e.value.status == bnz.BNZ_EINVAL
