"""The sharded form on the CPU: one buffer split at character boundaries (the library's host
cut function), every shard handled on its own (here by the reference codec), and the shards'
results combined by the library's gbu_combine_shards.  The combination must equal the
reference codec's result on the whole buffer: the first error (kind, offset), the lengths and
the output of the valid prefix.  Also run as two gloo ranks, one shard each, the way a
multi-GPU job would split one input (the exchange is an all-gather of the shards' results and
output lengths)."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_2111_08692_gb300 as g
    from paper_2111_08692_gb300.build import build
    build()
    return g


def sharded_utf8(g, data, P):
    """(validate result, convert result, length, output) of `data` computed shard by shard."""
    cuts = g.shard_cuts_host(data, P)
    assert cuts[0] == 0 and cuts[-1] == data.size and np.all(np.diff(cuts.astype(np.int64)) >= 0)
    shards = [data[int(cuts[k]):int(cuts[k + 1])] for k in range(P)]
    lens = [oracle.utf16_length_from_utf8(s) for s in shards]
    v = g.combine_shards(cuts, [oracle.validate_utf8(s) for s in shards])
    conv = [oracle.convert_utf8_to_utf16le(s) for s in shards]
    c = g.combine_shards(cuts, [r for r, _ in conv])
    out = np.concatenate([o[:n] for (_, o), n in zip(conv, lens)]) if P else np.zeros(0, np.uint16)
    return v, c, sum(lens), out


def sharded_utf16(g, data, P):
    cuts = g.shard_cuts_host(data, P)
    assert cuts[0] == 0 and cuts[-1] == data.size and np.all(np.diff(cuts.astype(np.int64)) >= 0)
    shards = [data[int(cuts[k]):int(cuts[k + 1])] for k in range(P)]
    lens = [oracle.utf8_length_from_utf16le(s) for s in shards]
    v = g.combine_shards(cuts, [oracle.validate_utf16le(s) for s in shards])
    conv = [oracle.convert_utf16le_to_utf8(s) for s in shards]
    c = g.combine_shards(cuts, [r for r, _ in conv])
    out = np.concatenate([o[:n] for (_, o), n in zip(conv, lens)])
    return v, c, sum(lens), out


def check_utf8(g, data, P):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    v, c, n16, out = sharded_utf8(g, data, P)
    assert v == oracle.validate_utf8(data), (P, v, oracle.validate_utf8(data), bytes(data[:64]))
    want, wout = oracle.convert_utf8_to_utf16le(data)
    assert c == want, (P, c, want)
    assert n16 == oracle.utf16_length_from_utf8(data)
    m = want[1] if want[0] == "OK" else oracle.utf16_length_from_utf8(data[:want[1]])
    assert np.array_equal(out[:m], wout[:m])


def check_utf16(g, data, P):
    data = np.ascontiguousarray(data, dtype=np.uint16)
    v, c, n8, out = sharded_utf16(g, data, P)
    assert v == oracle.validate_utf16le(data), (P, v, oracle.validate_utf16le(data))
    want, wout = oracle.convert_utf16le_to_utf8(data)
    assert c == want, (P, c, want)
    assert n8 == oracle.utf8_length_from_utf16le(data)
    m = want[1] if want[0] == "OK" else oracle.utf8_length_from_utf16le(data[:want[1]])
    assert np.array_equal(out[:m], wout[:m])


@pytest.mark.parametrize("P", [1, 2, 3, 7, 16, 61])
def test_profiles_and_sweeps(P):
    g = _lib()
    for prof in ("mixed", "latin", "cjk", "emoji"):
        u8, u16 = W.profile_buffers(prof, 50_000, 25_000, 71, cache=False)
        check_utf8(g, u8, P)
        check_utf16(g, u16, P)
    for prof in ("cyrillic", "cjk"):
        for rate in (1e-4, 1e-2):
            d = W.sweep_buffers(prof, rate, n_bytes=1 << 16, seed=W.SWEEP_SEEDS[(prof, rate)], cache=False)
            for key in ("u8", "u8_cut_end"):
                check_utf8(g, d[key], P)
            for key in ("u16", "u16_cut_end"):
                check_utf16(g, d[key], P)


def test_short_strings_every_split():
    """Every UTF-8 string of up to two bytes, and random strings over the bytes that matter at a
    cut (ASCII, continuation bytes, each kind of leading byte, bad leads), split into 2 to 6
    shards; every pair of special UTF-16 words likewise."""
    g = _lib()
    for a in range(256):
        for b in range(256):
            check_utf8(g, np.array([a, b], np.uint8), 2)
    rng = np.random.default_rng(72)
    alphabet = np.array([0x41, 0x80, 0x8F, 0x90, 0x9F, 0xA0, 0xBF, 0xC0, 0xC2, 0xDF, 0xE0, 0xED, 0xEF, 0xF0,
                         0xF4, 0xF5, 0xF8, 0xFF], np.uint8)
    for _ in range(4000):
        s = rng.choice(alphabet, size=int(rng.integers(1, 14)))
        check_utf8(g, s, int(rng.integers(2, 7)))
    words = np.array([0x41, 0x7FF, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xE000], np.uint16)
    for _ in range(3000):
        s = rng.choice(words, size=int(rng.integers(1, 10)))
        check_utf16(g, s, int(rng.integers(2, 7)))


def test_cuts_move_to_character_starts():
    g = _lib()
    data = np.frombuffer("aé中😀".encode() * 4, np.uint8)  # 1 + 2 + 3 + 4 bytes per round
    cuts = g.shard_cuts_host(data, 10)
    assert all((data[int(c)] & 0xC0) != 0x80 for c in cuts[1:-1] if c < data.size)
    runs = np.array([0x41] + [0x80] * 9, np.uint8)  # a run of continuation bytes: cut at c + 3
    assert list(g.shard_cuts_host(runs, 5)) == [0, 5, 7, 9, 10, 10]
    w = np.array([0x41, 0xD83D, 0xDE00, 0x42], np.uint16)
    assert list(g.shard_cuts_host(w, 2)) == [0, 3, 4]  # never between a pair's two words
    assert list(g.shard_cuts_host(np.zeros(0, np.uint8), 3)) == [0, 0, 0, 0]


def test_combine_rules():
    g = _lib()
    cuts = np.array([0, 10, 20, 30], np.uint64)
    assert g.combine_shards(cuts, [("OK", 10), ("OK", 10), ("OK", 10)]) == ("OK", 30)
    assert g.combine_shards(cuts, [("OK", 10), ("OVERLONG", 4), ("TOO_LONG", 0)]) == ("OVERLONG", 14)
    assert g.combine_shards(cuts, [("OK", 9), ("OUTPUT_TOO_SMALL", 12), ("SURROGATE", 3)]) == ("SURROGATE", 23)
    assert g.combine_shards(cuts, [("OK", 9), ("OUTPUT_TOO_SMALL", 12), ("OUTPUT_TOO_SMALL", 5)]) == \
        ("OUTPUT_TOO_SMALL", 26)
    assert g.combine_shards(cuts, [("OK", 9), ("TIMEOUT", 0), ("SURROGATE", 3)]) == ("TIMEOUT", 0)
    with pytest.raises(Exception):
        g.combine_shards(np.array([0, 10, 5, 30], np.uint64), [("OK", 1)] * 3)


# ---- two gloo ranks, one shard each -----------------------------------------------------------

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import oracle as O
    import workloads as WL
    import paper_2111_08692_gb300 as g
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = []
        for rate in (1e-4, 1e-2):
            d = WL.sweep_buffers("cjk", rate, n_bytes=1 << 16, seed=WL.SWEEP_SEEDS[("cjk", rate)], cache=False)
            valid, _ = WL.profile_buffers("emoji", 1 << 16, 1 << 15, 73, cache=False)
            for data in (d["u8"], valid):
                cuts = g.shard_cuts_host(data, world)  # every rank computes the same cuts
                mine = data[int(cuts[rank]):int(cuts[rank + 1])]
                res, conv = O.convert_utf8_to_utf16le(mine)
                n16 = O.utf16_length_from_utf8(mine)
                # the exchange: every rank's result and output length (and, here, its output)
                gathered = [None] * world
                dist.all_gather_object(gathered, (res, n16, conv[:n16].tobytes()))
                combined = g.combine_shards(cuts, [r for r, _, _ in gathered])
                offs = np.concatenate([[0], np.cumsum([n for _, n, _ in gathered])])
                whole = b"".join(o for _, _, o in gathered)
                out.append((combined, int(offs[-1]), whole))
        queue.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    i = 0
    for rate in (1e-4, 1e-2):
        d = W.sweep_buffers("cjk", rate, n_bytes=1 << 16, seed=W.SWEEP_SEEDS[("cjk", rate)], cache=False)
        valid, _ = W.profile_buffers("emoji", 1 << 16, 1 << 15, 73, cache=False)
        for data in (d["u8"], valid):
            want, wout = oracle.convert_utf8_to_utf16le(data)
            m = want[1] if want[0] == "OK" else oracle.utf16_length_from_utf8(data[:want[1]])
            for rank in (0, 1):
                combined, total, whole = got[rank][i]
                assert combined == want
                assert total == oracle.utf16_length_from_utf8(data)
                assert np.frombuffer(whole, np.uint16)[:m].tobytes() == wout[:m].tobytes()
            i += 1
