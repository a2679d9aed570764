"""Host-side logic of the serving loop (no GPU): the device-arena allocator."""
import numpy as np
import pytest

from paper_2106_01326_gb300 import server


def test_arena_first_fit_and_coalescing():
    a = server.Arena(4096, device="cpu")
    offs = [a.alloc(1000) for _ in range(4)]
    assert offs == [0, 1024, 2048, 3072]
    assert a.alloc(1) is None
    a.free(1024, 1000)
    a.free(2048, 1000)
    assert a.alloc(2048) == 1024  # the two neighbours merged
    a.free(0, 1000)
    a.free(1024, 2048)
    a.free(3072, 1000)
    assert a.used == 0
    assert a.alloc(4096) == 0
    assert a.peak == 4096


def test_arena_random_sequence_keeps_invariants():
    rng = np.random.default_rng(0)
    a = server.Arena(1 << 20, device="cpu")
    live = {}
    for _ in range(2000):
        if live and rng.random() < 0.5:
            off = list(live)[rng.integers(len(live))]
            a.free(off, live.pop(off))
        else:
            n = int(rng.integers(1, 50000))
            off = a.alloc(n)
            if off is not None:
                assert off % 256 == 0
                for o, m in live.items():  # no overlap with live blocks
                    assert off + n <= o or o + m <= off
                live[off] = n
        total_free = sum(sz for _, sz in a._free)
        assert total_free + a.used == a.nbytes
    for off, n in list(live.items()):
        a.free(off, n)
    assert a._free == [[0, a.nbytes]]


def test_grid_bytes():
    assert server.grid_bytes(64) == 64 * 64 * 2 * 4
    assert server.grid_bytes(8) == 8 * 8 * 1 * 4
