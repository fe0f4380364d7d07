"""Host-side bookkeeping of the serving loop's device arena (no GPU needed): first-fit
offsets, alignment, coalescing, exhaustion, and a random workload checked against a plain
model of the same policy."""
import random

import pytest


@pytest.fixture(scope="module")
def P():
    from paper_2111_08692_gb300.build import build
    build()
    import paper_2111_08692_gb300 as P
    return P


def _round(x, a):
    return (max(x, 1) + a - 1) // a * a


def test_first_fit_alignment_and_coalescing(P):
    a = P.Arena(1 << 20, 256)
    x = a.alloc(1000)
    y = a.alloc(5000)
    z = a.alloc(1)
    assert (x, y, z) == (0, 1024, 1024 + 5120)
    assert a.used() == 1024 + 5120 + 256
    assert a.free(y)
    assert not a.free(y)  # double free is refused
    assert a.alloc(4000) == 1024  # first fit reuses the hole
    assert a.free(x) and a.free(1024) and a.free(z)
    assert a.used() == 0 and a.free_blocks() == 1 and a.largest_free() == 1 << 20
    a.close()


def test_exhaustion_and_fragmentation(P):
    a = P.Arena(4096, 256)
    offs = [a.alloc(256) for _ in range(16)]
    assert offs == [256 * i for i in range(16)]
    assert a.alloc(1) is None
    for o in offs[::2]:
        assert a.free(o)
    assert a.largest_free() == 256 and a.alloc(512) is None  # holes too small
    assert a.free(offs[1])  # joins holes 0, 1, 2
    assert a.largest_free() == 768 and a.alloc(700) == 0
    a.close()


def test_random_workload_matches_a_model(P):
    cap, align = 1 << 24, 256
    a = P.Arena(cap, align)
    rng = random.Random(7)
    free = [(0, cap)]  # sorted (offset, size)
    live = {}
    for _ in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 300):
            off = rng.choice(list(live))
            size = live.pop(off)
            assert a.free(off)
            free.append((off, size))
            free.sort()
            merged = []
            for o, s in free:
                if merged and merged[-1][0] + merged[-1][1] == o:
                    merged[-1] = (merged[-1][0], merged[-1][1] + s)
                else:
                    merged.append((o, s))
            free = merged
        else:
            want = rng.choice([1, 100, 256, 3000, 65536, 1 << 20, rng.randrange(1, 1 << 21)])
            size = _round(want, align)
            model = next(((i, o, s) for i, (o, s) in enumerate(free) if s >= size), None)
            got = a.alloc(want)
            if model is None:
                assert got is None
                continue
            i, o, s = model
            assert got == o
            live[o] = size
            free[i:i + 1] = [(o + size, s - size)] if s > size else []
        assert a.used() == sum(live.values())
        assert a.free_blocks() == len(free)
        assert a.largest_free() == max((s for _, s in free), default=0)
    a.close()
