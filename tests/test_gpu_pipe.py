"""The host-buffer form (gbu_pipe_*) through the C ABI against the oracle: host arrays in,
pieces of 4096 units on three streams, the whole input's result out, and for the transcoders
every defined output unit and the guard zone past cap.  The inputs put errors, surrogate pairs,
four-byte characters and over-long continuation runs at and around the piece cuts."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

PIECE = 4096
CANARY16, CANARY8 = 0x5A5A, 0x5A


@pytest.fixture(scope="module")
def pipe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_08692_gb300 import Pipe
    from paper_2111_08692_gb300.build import build
    build()
    p = Pipe(0, piece_units=PIECE, streams=3)
    yield p
    p.close()


def _pinned(a):
    """A copy of a in page-locked host memory (the copies then overlap the kernels)."""
    import torch
    t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True)
    h = t.numpy().view(a.dtype)
    h[:] = a
    return h, t


def _utf8_cases():
    mixed, _ = W.profile_buffers("mixed", 40 * PIECE + 7, 0, 601, cache=False)
    emoji, _ = W.profile_buffers("emoji", 12 * PIECE + 3, 0, 602, cache=False)
    cases = [("mixed", mixed), ("emoji", emoji), ("empty", np.zeros(0, np.uint8)),
             ("short", np.frombuffer("aé中\U0001f600".encode(), np.uint8))]
    for k in (1, 2, 7):  # invalid bytes at and around the cuts of the nominal pieces
        for d in (-4, -3, -2, -1, 0, 1, 2, 3):
            bad = mixed.copy()
            bad[k * PIECE + d] = 0xFF
            cases.append((f"ff@{k}*P{d:+d}", bad))
    # a four-byte character at every position across the first cut
    base = np.full(3 * PIECE, 0x41, np.uint8)
    for d in (-3, -2, -1, 0):
        a = base.copy()
        a[PIECE + d:PIECE + d + 4] = [0xF0, 0x9F, 0x98, 0x80]
        cases.append((f"4byte@P{d:+d}", a))
    # runs of four and five continuation bytes across the cut (TOO_LONG), and a lead byte cut
    # off by the end of the input
    for run in (4, 5):
        a = base.copy()
        a[PIECE - 3:PIECE - 3 + run] = 0x80
        cases.append((f"run{run}", a))
    a = base.copy()
    a[PIECE - 4:PIECE] = [0xF0, 0x9F, 0x98, 0x80]
    a[PIECE:PIECE + 2] = 0x80
    cases.append(("4byte+2cont@P", a))
    cases.append(("cut_end", np.concatenate([base[:2 * PIECE], np.array([0xE4, 0xB8], np.uint8)])))
    return cases


def _utf16_cases():
    _, mixed = W.profile_buffers("mixed", 16, 30 * PIECE + 5, 603, cache=False)
    _, emoji = W.profile_buffers("emoji", 16, 10 * PIECE + 1, 604, cache=False)
    cases = [("mixed", mixed), ("emoji", emoji), ("empty", np.zeros(0, np.uint16))]
    base = np.full(3 * PIECE, 0x41, np.uint16)
    for d in (-2, -1, 0, 1):
        a = base.copy()
        a[PIECE + d:PIECE + d + 2] = [0xD83D, 0xDE00]  # a pair across (or beside) the cut
        cases.append((f"pair@P{d:+d}", a))
        for w in (0xD800, 0xDC00):  # a lone surrogate at and around the cut
            a = base.copy()
            a[PIECE + d] = w
            cases.append((f"lone{w:X}@P{d:+d}", a))
    a = base.copy()
    a[PIECE - 1:PIECE + 1] = [0xD800, 0xD800]
    cases.append(("high,high@P", a))
    a = base.copy()
    a[PIECE - 2:PIECE + 1] = [0xD800, 0xD800, 0xDC00]
    cases.append(("high,pair@P", a))
    cases.append(("cut_high", np.concatenate([base[:PIECE + 9], [0xD83D]]).astype(np.uint16)))
    return cases


def test_pipe_validation_and_lengths_match_the_oracle(pipe):
    for name, data in _utf8_cases():
        assert pipe.validate_utf8(data) == oracle.validate_utf8(data), name
        assert pipe.utf16_length_from_utf8(data) == ("OK", oracle.utf16_length_from_utf8(data)), name
    for name, data in _utf16_cases():
        assert pipe.validate_utf16le(data) == oracle.validate_utf16le(data), name
        assert pipe.utf8_length_from_utf16le(data) == ("OK", oracle.utf8_length_from_utf16le(data)), name


def _defined_prefix(want, cap, prefix_len):
    kind, count = want
    if kind == "OK":
        return count
    if kind == "OUTPUT_TOO_SMALL":
        return cap
    return min(prefix_len(count), cap)


@pytest.mark.parametrize("short", [0, 1, 5000])
def test_pipe_transcoders_match_the_oracle(pipe, short):
    """Each transcoder with a capacity of the exact length, one unit short, or 5000 units short
    (a cap that ends inside an earlier piece's output)."""
    for name, data in _utf8_cases():
        cap = max(oracle.utf16_length_from_utf8(data) - short, 0)
        want, odst = oracle.convert_utf8_to_utf16le(data, cap)
        buf = np.full(cap + 24, CANARY16, np.uint16)
        got = pipe.convert_utf8_to_utf16le(data, buf, cap=cap)
        assert got == want, (name, got, want)
        m = _defined_prefix(want, cap, lambda c: oracle.utf16_length_from_utf8(data[:c]))
        assert np.array_equal(buf[:m], odst[:m]), name
        assert np.all(buf[cap:] == CANARY16), name
    for name, data in _utf16_cases():
        cap = max(oracle.utf8_length_from_utf16le(data) - short, 0)
        want, odst = oracle.convert_utf16le_to_utf8(data, cap)
        buf = np.full(cap + 24, CANARY8, np.uint8)
        got = pipe.convert_utf16le_to_utf8(data, buf, cap=cap)
        assert got == want, (name, got, want)
        m = _defined_prefix(want, cap, lambda c: oracle.utf8_length_from_utf16le(data[:c]))
        assert np.array_equal(buf[:m], odst[:m]), name
        assert np.all(buf[cap:] == CANARY8), name


def test_pipe_on_pinned_buffers_with_the_default_pieces():
    """Pinned host memory, the default piece (64 Mi units) and three streams, on 300 MiB of
    mixed text: five pieces, so the copies of one overlap the kernels of the others; the
    output is checked whole against the oracle's."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_08692_gb300 import Pipe
    u8, _ = W.profile_buffers("mixed", 300 << 20, 0, 605)
    src, keep_src = _pinned(u8)
    n16 = oracle.utf16_length_from_utf8(u8)
    want, odst = oracle.convert_utf8_to_utf16le(u8, n16)
    dst, keep_dst = _pinned(np.zeros(n16, np.uint16))
    p = Pipe(0)
    try:
        assert p.validate_utf8(src) == ("OK", u8.size)
        assert p.convert_utf8_to_utf16le(src, dst) == want
        assert np.array_equal(dst, odst)
    finally:
        p.close()


def test_pipe_refuses_misaligned_and_missing_buffers(pipe):
    """A UTF-16 source or UTF-16 destination at an odd address, a NULL result, and a NULL
    destination with cap > 0 are GBU_BAD_ARGUMENT, with nothing written; empty inputs give
    {OK, 0}."""
    import ctypes
    from paper_2111_08692_gb300 import GbuResult, lib
    L = lib()
    raw = np.zeros(64, np.uint8)
    base = raw.ctypes.data
    odd = base + 1 if base % 2 == 0 else base
    res = GbuResult()
    assert L.gbu_pipe_validate_utf16le(pipe.handle, odd, 8, ctypes.byref(res)) == 17
    assert L.gbu_pipe_utf8_length_from_utf16le(pipe.handle, odd, 8, ctypes.byref(res)) == 17
    out = np.full(64, CANARY8, np.uint8)
    assert L.gbu_pipe_convert_utf8_to_utf16le(pipe.handle, base, 8, out.ctypes.data + 1, 8, ctypes.byref(res)) == 17
    assert np.all(out == CANARY8)
    assert L.gbu_pipe_convert_utf16le_to_utf8(pipe.handle, base, 8, None, 8, ctypes.byref(res)) == 17
    assert L.gbu_pipe_validate_utf8(pipe.handle, base, 8, None) == 17
    assert L.gbu_pipe_validate_utf8(pipe.handle, None, 8, ctypes.byref(res)) == 17
    for name in ("validate_utf8", "validate_utf16le", "utf16_length_from_utf8", "utf8_length_from_utf16le"):
        empty = np.zeros(0, np.uint16 if "16le" in name else np.uint8)
        assert getattr(pipe, name)(empty) == ("OK", 0), name
    assert pipe.convert_utf8_to_utf16le(np.zeros(0, np.uint8), np.zeros(0, np.uint16)) == ("OK", 0)
    assert pipe.convert_utf16le_to_utf8(np.zeros(0, np.uint16), np.zeros(0, np.uint8)) == ("OK", 0)
