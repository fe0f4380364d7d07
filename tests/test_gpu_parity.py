"""Bit-exact parity of the CUDA library with the reference codec (oracle/), through the C ABI.

Every comparison is exact: result kind and count, output lengths, every output unit that
the contract defines, and canaries around the destination.  Inputs come from the seeded
generators in workloads/ (or are built here from them), never from the CUDA path.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import char_starts_utf8, check_utf16_input, check_utf8_input

pytestmark = pytest.mark.gpu

# The kernels' geometry, read from the library by the `geometry` fixture: bytes per streaming
# warp tile (TILE), per transcoder round (one 512-byte region per warp, TTILE) and per
# transcoder partition (the unit of the look-back, PART).
TILE = TTILE = PART = None


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def codec(torch):
    from paper_2111_08692_gb300 import Codec
    from paper_2111_08692_gb300.build import build
    build()
    c = Codec(0, max_units=(1 << 30) + 4096)
    g = c.launch_config()
    global TILE, TTILE, PART
    TILE = g["stream_tile_bytes"]
    TTILE = g["transcoder_threads_per_cta"] * 16
    PART = g["partition_bytes"]
    yield c
    c.close()


def _mixed(n, seed):
    u8, _ = W.profile_buffers("mixed", n, 0, seed, cache=False)
    return u8


def test_empty_and_tiny(codec, torch):
    check_utf8_input(codec, torch, np.zeros(0, np.uint8))
    check_utf16_input(codec, torch, np.zeros(0, np.uint16))
    for b in range(256):
        check_utf8_input(codec, torch, np.array([b], np.uint8), src_off=b % 16, dst_off=b % 8)
    for w in (0, 0x41, 0x7F, 0x80, 0x7FF, 0x800, 0xD7FF, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xE000, 0xFFFF):
        check_utf16_input(codec, torch, np.array([w], np.uint16), src_off=w % 8, dst_off=w % 16)


def test_all_two_byte_strings(codec, torch):
    """Every two-byte UTF-8 string: validation (the asynchronous call) and conversion (the
    host-synchronising call), one call each, against the oracle."""
    from paper_2111_08692_gb300 import result_tuple
    data = np.zeros(2, np.uint8)
    dst = torch.full((4,), 0x5A5A, dtype=torch.int16, device="cuda")
    for b0 in range(0x80, 0x100):  # ASCII first bytes reduce to one-byte strings
        for b1 in range(256):
            data[0], data[1] = b0, b1
            want = oracle.validate_utf8(data)
            src = torch.from_numpy(data.copy()).to("cuda")
            got = result_tuple(codec.validate_utf8(src))
            assert got == want, (b0, b1, got, want)
            cwant, cdst = oracle.convert_utf8_to_utf16le(data, 2)
            cgot = codec.convert_utf8_to_utf16le_sync(src, dst[:2])
            assert cgot == cwant, (b0, b1, cgot, cwant)
            if cwant[0] == "OK":
                out = dst.cpu().numpy().view(np.uint16)
                assert np.array_equal(out[:cwant[1]], cdst[:cwant[1]]), (b0, b1)
                assert np.all(out[2:] == 0x5A5A), (b0, b1)


def test_lengths_and_alignments(codec, torch):
    rng = np.random.default_rng(5)
    for n in list(range(0, 80)) + [127, 128, 129, 255, 256, 300, 511, 512, 513]:
        data = _mixed(max(n, 1), 100 + n)[:n]
        check_utf8_input(codec, torch, data, src_off=int(rng.integers(0, 16)), dst_off=int(rng.integers(0, 8)))
        u16 = np.frombuffer(data.tobytes().decode("utf-8", errors="replace").encode("utf-16-le"), np.uint16)[:n]
        check_utf16_input(codec, torch, u16, src_off=int(rng.integers(0, 8)), dst_off=int(rng.integers(0, 16)))
    data = _mixed(20000, 7)
    u16 = np.frombuffer(data.tobytes().decode("utf-8").encode("utf-16-le"), np.uint16)
    for off in range(16):
        check_utf8_input(codec, torch, data, src_off=off, dst_off=(off * 3) % 8)
        check_utf16_input(codec, torch, u16, src_off=off % 8, dst_off=off)


def test_mixed_1mib_and_flipped_byte(codec, torch):
    """The 1 MiB mixed buffer (seed 0), its UTF-16 form, and the copy with one flipped byte."""
    u8, u16, flipped, o = W.mixed_1mib()
    v, c = check_utf8_input(codec, torch, u8)
    assert v[0] == "OK" and c[0] == "OK"
    v, c = check_utf16_input(codec, torch, u16)
    assert v[0] == "OK"
    v, c = check_utf8_input(codec, torch, flipped)
    assert v[0] != "OK" and o - 3 <= v[1] <= o + 1


@pytest.mark.parametrize("profile", W.PROFILE_ORDER + ("mixed",))
def test_profiles_multi_tile(codec, torch, profile):
    """4 MiB of each profile (1024 tiles), both directions, full output comparison."""
    u8, u16 = W.profile_buffers(profile, 1 << 22, 1 << 21, 31, cache=False)
    check_utf8_input(codec, torch, u8, src_off=3, dst_off=5)
    check_utf16_input(codec, torch, u16, src_off=1, dst_off=7)
    check_utf8_input(codec, torch, u8)
    check_utf16_input(codec, torch, u16)


INVALID_UTF8 = [bytes.fromhex(h) for h in (
    "80", "bf", "c0", "c1bf", "c3", "e282", "e0 80 80".replace(" ", ""), "e09fbf", "eda080",
    "edbfbf", "f08fbfbf", "f4908080", "f5808080", "f7bfbfbf", "f8", "ff", "f09f98", "e0", "f0")]


def test_errors_near_tile_and_warp_boundaries(codec, torch):
    base = _mixed(max(3 * PART, 5 * TILE) + 2 * TILE, 3)
    starts = char_starts_utf8(base)
    targets = []
    # streaming tiles, 512-byte and 1 KiB warp regions, 16- and 32-byte lane chunks, 4 KiB warp
    # slices and partitions
    for b in (TILE, 2 * TILE, 3 * TILE, 512, 1024 + 512, 5 * TILE, TTILE + 16, 2 * TTILE - 16,
              32, 992, 1024, 1056, 2048, 3072, 4096, 4096 + 1024, 8192 - 32, 12288,
              PART, PART + 512, 2 * PART, 3 * PART - 512):
        targets += [b - 5, b - 4, b - 3, b - 2, b - 1, b, b + 1, b + 2, b + 3]
    targets += [0, 1, 2, 15, 16, 17]
    for t in targets:
        i = int(starts[np.searchsorted(starts, t)]) if t < base.size else base.size
        for bad in INVALID_UTF8:
            data = np.concatenate([base[:i], np.frombuffer(bad, np.uint8), base[i:]])
            v, _ = check_utf8_input(codec, torch, data)
            assert v[0] != "OK" and v[1] == i, (t, bad.hex(), v)


STRADDLERS = ("\u00e9".encode(), "\u4e2d".encode(), "\U0001F600".encode())  # 2-, 3-, 4-byte


@pytest.mark.parametrize("profile", ("latin", "cyrillic", "cjk", "emoji"))
def test_single_class_regions(codec, torch, profile):
    """Text whose regions hold one class of leading byte (two-, three- or four-byte), with a
    character of another class cut by a region, round or partition boundary (so the region
    after it starts with that character's continuation bytes), and with each invalid
    sequence inside a region."""
    base = W.profile_buffers(profile, 3 * PART, 0, 41, cache=False)[0]
    starts = char_starts_utf8(base)
    for b in (512, 1024, 4096, TTILE, PART, PART + 512, 2 * PART - 512):
        s = int(starts[np.searchsorted(starts, b - 8)])
        s = s if s <= b - 4 else int(starts[np.searchsorted(starts, b - 8) - 1])
        for ch in STRADDLERS:
            for d in range(1, len(ch)):
                pad = np.full(b - d - s, 0x41, np.uint8)
                data = np.concatenate([base[:s], pad, np.frombuffer(ch, np.uint8), base[s:]])
                v, _ = check_utf8_input(codec, torch, data)
                assert v[0] == "OK", (profile, b, ch, d, v)
    for t in (700, 5000, PART - 300, PART + 4000):
        i = int(starts[np.searchsorted(starts, t)])
        for bad in INVALID_UTF8:
            data = np.concatenate([base[:i], np.frombuffer(bad, np.uint8), base[i:]])
            v, _ = check_utf8_input(codec, torch, data)
            assert v[0] != "OK" and v[1] == i, (profile, t, bad.hex(), v)


def test_error_at_the_last_byte_and_cut_at_the_end(codec, torch):
    base = _mixed(3 * TILE, 9)
    starts = char_starts_utf8(base)
    for end in (TILE - 1, TILE, TILE + 1, 2 * TILE - 2, 3 * TILE - 3):
        cut = int(starts[np.searchsorted(starts, end) - 1])
        for tail in (b"\xe4\xb8", b"\xf0\x9f\x98", b"\xc3", b"\x80", b"\xff"):
            data = np.concatenate([base[:cut], np.frombuffer(tail, np.uint8)])
            check_utf8_input(codec, torch, data)


def test_several_errors_the_first_wins(codec, torch):
    base = _mixed(8 * TILE, 11)
    starts = char_starts_utf8(base)
    rng = np.random.default_rng(1)
    for _ in range(30):
        pos = sorted(int(starts[j]) for j in rng.integers(0, starts.size, size=4))
        pieces, last = [], 0
        for p in pos:
            pieces += [base[last:p], np.frombuffer(INVALID_UTF8[int(rng.integers(0, len(INVALID_UTF8)))], np.uint8)]
            last = p
        pieces.append(base[last:])
        check_utf8_input(codec, torch, np.concatenate(pieces))


def test_utf16_errors_near_tile_boundaries(codec, torch):
    _, base = W.profile_buffers("emoji", 0, 5 * 2048, 13, cache=False)
    units = 2048
    for b in (units, 2 * units, 4 * units, 256, 1024):
        for d in range(-3, 4):
            i = b + d
            for bad in ([0xD800], [0xDC00], [0xDBFF, 0x41], [0xD800, 0xD800], [0xDFFF, 0xDFFF]):
                data = np.concatenate([base[:i], np.array(bad, np.uint16), base[i:]])
                check_utf16_input(codec, torch, data)
    # a high surrogate as the very last word, at and around a tile end
    for n in (units - 1, units, units + 1, 3 * units):
        data = base[:n].copy()
        data[-1] = 0xD9AB
        check_utf16_input(codec, torch, data)


def test_utf16_errors_at_the_start_of_an_aligned_buffer(codec, torch):
    """Unpaired surrogates in the first chunks of a buffer whose first word starts a 16-byte
    chunk (no word before it), and pairs cut by the chunk boundaries there."""
    _, base = W.profile_buffers("emoji", 0, 1 << 15, 17, cache=False)
    for i in range(0, 18):
        for bad in ([0xDC00], [0xD800], [0xD800, 0x41], [0xDFFF, 0xDFFF], [0xD83D, 0xDE00]):
            data = base.copy()
            data[i:i + len(bad)] = bad
            for src_off in (0, 8):
                check_utf16_input(codec, torch, data, src_off=src_off)


def test_surrogate_pairs_straddling_tiles(codec, torch):
    # pairs everywhere: each tile boundary splits some pair for one of the shifts
    pairs = np.tile(np.array([0xD83D, 0xDE00], np.uint16), 3 * 2048)
    for shift in range(3):
        data = np.concatenate([np.full(shift, 0x41, np.uint16), pairs])
        check_utf16_input(codec, torch, data, dst_off=shift)


def test_capacity_too_small(codec, torch):
    data = _mixed(3 * TILE, 21)
    total16 = oracle.utf16_length_from_utf8(data)
    for cap in (0, 1, 7, 8, 9, 100, 4095, 4096, 4097, total16 - 1):
        check_utf8_input(codec, torch, data, cap=cap, dst_off=cap % 8)
    u16 = np.frombuffer(data.tobytes().decode("utf-8").encode("utf-16-le"), np.uint16)
    total8 = oracle.utf8_length_from_utf16le(u16)
    for cap in (0, 1, 15, 16, 17, 4095, 4096, total8 - 1):
        check_utf16_input(codec, torch, u16, cap=cap, dst_off=cap % 16)
    # an input error takes precedence over the capacity
    bad = np.concatenate([data, np.array([0xFF], np.uint8)])
    check_utf8_input(codec, torch, bad, cap=10)


def test_sweep_small(codec, torch):
    """The invalid-input sweep at 8 MiB: exact first error (kind, offset) and output prefix."""
    for profile in ("cyrillic", "cjk"):
        for rate in (1e-6, 1e-4, 1e-2):
            d = W.sweep_buffers(profile, rate, n_bytes=1 << 23, seed=W.SWEEP_SEEDS[(profile, rate)], cache=False)
            check_utf8_input(codec, torch, d["u8"])
            check_utf8_input(codec, torch, d["u8_cut_end"])
            check_utf16_input(codec, torch, d["u16"])
            check_utf16_input(codec, torch, d["u16_cut_end"])


def test_early_exit_gives_the_same_results(codec, torch):
    """Early exit on invalid input changes no result: errors placed before, inside and after
    the tiles and partitions other warps work on, several at once, with early exit on and off."""
    from paper_2111_08692_gb300 import result_tuple
    from gpu_helpers import as_torch_u16
    u8, u16 = W.profile_buffers("cjk", 3 * PART + 777, (3 * PART + 777) // 2, 52, cache=False)
    starts = char_starts_utf8(u8)
    rng = np.random.default_rng(53)
    cases8, cases16 = [], []
    for k in range(24):
        b = u8.copy()
        for pos in rng.choice(starts[starts > 4], size=1 + k % 3, replace=False):
            b[pos] = (0x80, 0xC0, 0xFF)[k % 3]
        cases8.append(b)
        w = u16.copy()
        for pos in rng.integers(0, w.size, size=1 + k % 3):
            w[pos] = 0xDC00 + k
        cases16.append(w)
    for b, w in zip(cases8, cases16):
        s8 = torch.from_numpy(b).to("cuda")
        s16 = as_torch_u16(torch, w).to("cuda")
        d16 = torch.empty(b.size + 8, dtype=torch.int16, device="cuda")
        d8 = torch.empty(3 * w.size + 8, dtype=torch.uint8, device="cuda")
        want = (oracle.validate_utf8(b), oracle.convert_utf8_to_utf16le(b, b.size + 8)[0],
                oracle.validate_utf16le(w), oracle.convert_utf16le_to_utf8(w, 3 * w.size + 8)[0])
        for early in (True, False):
            codec.set_early_exit(early)
            got = (result_tuple(codec.validate_utf8(s8)), result_tuple(codec.convert_utf8_to_utf16le(s8, d16)),
                   result_tuple(codec.validate_utf16le(s16)), result_tuple(codec.convert_utf16le_to_utf8(s16, d8)))
            assert got == want, (early, got, want)
    codec.set_early_exit(True)


def test_repeated_runs_are_identical(codec, torch):
    from paper_2111_08692_gb300 import result_tuple
    u8, u16 = W.profile_buffers("emoji", 1 << 21, 1 << 20, 41, cache=False)
    src = torch.from_numpy(u8).to("cuda")
    cap = oracle.utf16_length_from_utf8(u8)
    first = None
    for _ in range(50):
        dst = torch.empty(cap, dtype=torch.int16, device="cuda")
        r = result_tuple(codec.convert_utf8_to_utf16le(src, dst))
        h = (r, dst.cpu().numpy().tobytes())
        if first is None:
            first = h
        assert h == first


def test_bad_arguments_are_rejected_without_launch(codec, torch):
    import paper_2111_08692_gb300 as g
    n0 = codec.launches()
    res = codec.new_result()
    assert g.gbu_validate_utf8(codec.ctx, 0, 10, res.data_ptr(), 0) == g.STATUS_CODE["BAD_ARGUMENT"]
    src16 = torch.zeros(8, dtype=torch.int16, device="cuda")
    assert g.gbu_validate_utf16le(codec.ctx, src16.data_ptr() + 1, 3, res.data_ptr(), 0) == g.STATUS_CODE["BAD_ARGUMENT"]
    assert g.gbu_convert_utf8_to_utf16le(codec.ctx, src16.data_ptr(), 4, 0, 4, res.data_ptr(), 0) == g.STATUS_CODE["BAD_ARGUMENT"]
    assert g.gbu_validate_utf8(codec.ctx, src16.data_ptr(), 4, 0, 0) == g.STATUS_CODE["BAD_ARGUMENT"]
    assert g.gbu_validate_utf8(codec.ctx, src16.data_ptr(), 1 << 40, res.data_ptr(), 0) == g.STATUS_CODE["BAD_ARGUMENT"]
    assert codec.launches() == n0


def test_wait_timeout_is_reported_and_recovered(codec, torch):
    """A tile that never publishes its scan state: the waits give up, the call reports
    GBU_TIMEOUT, and the next call on the same context is correct again."""
    from paper_2111_08692_gb300 import result_tuple
    data = _mixed(6 * PART, 17)
    src = torch.from_numpy(data).to("cuda")
    cap = oracle.utf16_length_from_utf8(data)
    dst = torch.empty(cap, dtype=torch.int16, device="cuda")
    codec.set_wait_limit(2000)
    codec.debug_skip_publish(2)  # partition 3 must look back past it
    try:
        r = result_tuple(codec.convert_utf8_to_utf16le(src, dst))
    finally:
        codec.debug_skip_publish(-1)
        codec.set_wait_limit(1 << 22)
    assert r[0] == "TIMEOUT"
    check_utf8_input(codec, torch, data)
