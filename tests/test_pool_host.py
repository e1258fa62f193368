"""The device memory pool's bookkeeping (host only: the pool never touches
the memory, so any address range serves): first fit in address order,
256-byte blocks, merging of freed neighbours, errors."""
import numpy as np
import pytest

import paper_1802_02619_gb300 as lco

BASE = 1 << 30


class FirstFit:
    """Plain model: a sorted list of free (offset, size) blocks."""

    def __init__(self, n):
        self.free = [(0, n)]
        self.used = {}

    def alloc(self, b):
        need = max(256, (b + 255) // 256 * 256)
        for i, (o, s) in enumerate(self.free):
            if s >= need:
                if s == need:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + need, s - need)
                self.used[o] = need
                return o
        return None

    def release(self, o):
        s = self.used.pop(o)
        self.free.append((o, s))
        self.free.sort()
        merged = []
        for blk in self.free:
            if merged and merged[-1][0] + merged[-1][1] == blk[0]:
                merged[-1] = (merged[-1][0], merged[-1][1] + blk[1])
            else:
                merged.append(blk)
        self.free = merged


def test_matches_first_fit_model():
    rng = np.random.default_rng(0)
    n = 1 << 20
    pool, model = lco.Pool(BASE, n), FirstFit(n)
    live = []
    for _ in range(3000):
        if live and rng.random() < 0.45:
            k = live.pop(int(rng.integers(len(live))))
            pool.free(BASE + k)
            model.release(k)
        else:
            b = int(rng.integers(1, 40000))
            p, m = pool.alloc(b), model.alloc(b)
            assert (p is None) == (m is None)
            if p is not None:
                assert p - BASE == m and p % 256 == 0
                live.append(m)
        st = pool.stats()
        assert st["used"] == sum(model.used.values())
        assert st["largest_free"] == max([s for _, s in model.free], default=0)
    for k in live:
        pool.free(BASE + k)
    st = pool.stats()
    assert st["used"] == 0 and st["largest_free"] == n


def test_blocks_never_overlap():
    pool = lco.Pool(BASE, 1 << 16)
    got = []
    while True:
        p = pool.alloc(1000)
        if p is None:
            break
        got.append(p)
    assert len(got) == (1 << 16) // 1024
    spans = sorted((p, p + 1024) for p in got)
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))


def test_errors():
    pool = lco.Pool(BASE, 1 << 12)
    assert pool.alloc(1 << 13) is None                 # larger than the pool: no change
    p = pool.alloc(100)
    pool.free(p)
    with pytest.raises(lco.LcoError):
        pool.free(p)                                   # second free
    with pytest.raises(lco.LcoError):
        pool.free(BASE + 512)                          # never allocated
    with pytest.raises(lco.LcoError):
        pool.free(BASE + (1 << 20))                    # outside the pool
    with pytest.raises(lco.LcoError):
        lco.Pool(BASE, 100)                            # smaller than one block
