"""Host-side logic of the serving loop (no GPU): the staging ring's
admission by footprint, wrap-around and FIFO release."""
import pytest

torch = pytest.importorskip("torch")

from paper_2311_00626_gb300.serving import StagingRing  # noqa: E402


def test_ring_admits_by_footprint_and_releases_in_order():
    r = StagingRing(torch, 4096, "cpu")
    a = r.alloc(1000)   # 1024 bytes
    b = r.alloc(2000)   # 2048
    assert a == (0, 1024) and b == (1024, 2048)
    assert r.alloc(1500) is None          # only 1024 left
    c = r.alloc(1024)
    assert c == (3072, 1024) and r.used == 4096
    r.release(1)                          # frees a
    assert r.alloc(2000) is None          # 1024 free at the start, head at the end
    d = r.alloc(1000)                     # fits in [0, 1024)
    assert d == (0, 1024)


def test_ring_wraps_with_waste_and_refuses_oversize():
    r = StagingRing(torch, 4096, "cpu")
    r.alloc(3000)                         # 3072
    r.release(1)
    assert r.used == 0
    x = r.alloc(2048)                     # head at 3072: wraps, wasting 1024
    assert x == (0, 2048) and r.used == 3072
    n_live = len(r.live)
    assert n_live == 2                    # waste slice + allocation
    r.release(2)
    assert r.used == 0
    with pytest.raises(ValueError):
        r.alloc(5000)


def test_ring_never_overlaps_live_slices():
    import random
    rnd = random.Random(3)
    r = StagingRing(torch, 1 << 16, "cpu")
    live = []
    for _ in range(2000):
        if live and rnd.random() < 0.45:
            r.release(live.pop(0)[2])
            continue
        before = len(r.live)
        got = r.alloc(rnd.randint(1, 20000))
        if got is None:
            continue
        slices = len(r.live) - before
        off, size = got
        for o2, s2, _ in live:
            assert off + size <= o2 or o2 + s2 <= off
        live.append((off, size, slices))
