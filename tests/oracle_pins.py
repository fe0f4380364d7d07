"""The checks that pin the reference codec to things other than itself.

Each function raises AssertionError when the codec under test disagrees with:
  * the hand-derived fixtures in tests/golden/ (paper Section 3 boundaries and rules),
  * CPython's strict ``utf-8`` / ``utf-16-le`` / ``utf-16-be`` / ``utf-32-le`` codecs (an
    independent library decoder),
  * the brute-force second formulation in tests/helpers/bruteforce.c, or
  * closed forms of the length formulas.
They take the codec and the brute-force library as arguments so that the mutation test can
run the same battery against deliberately broken copies of the codec.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            yield [c.strip() for c in line.split("|")]


def golden_scalars():
    out = []
    for cp, b8, w16, _why in _rows("utf8_utf16_scalars.txt"):
        cp = int(cp[2:], 16)
        u8 = bytes(int(x, 16) for x in b8.split())
        u16 = np.array([int(x, 16) for x in w16.split()], dtype=np.uint16)
        out.append((cp, u8, u16))
    return out


def golden_invalid(name, width):
    out = []
    for data, kind, off, _why in _rows(name):
        vals = [int(x, 16) for x in data.split()]
        arr = np.array(vals, dtype=np.uint8 if width == 8 else np.uint16)
        out.append((arr, kind, int(off)))
    return out


def check_golden(codec):
    scal = golden_scalars()
    assert len(scal) >= 18
    for cp, u8, u16 in scal:
        # the fixture itself agrees with CPython
        assert chr(cp).encode("utf-8") == u8, hex(cp)
        assert chr(cp).encode("utf-16-le") == u16.tobytes(), hex(cp)
        assert codec.validate_utf8(u8) == ("OK", len(u8)), hex(cp)
        assert codec.validate_utf16le(u16) == ("OK", len(u16)), hex(cp)
        assert codec.utf16_length_from_utf8(u8) == len(u16), hex(cp)
        assert codec.utf8_length_from_utf16le(u16) == len(u8), hex(cp)
        r, d = codec.convert_utf8_to_utf16le(u8)
        assert r == ("OK", len(u16)) and np.array_equal(d, u16), hex(cp)
        r, d = codec.convert_utf16le_to_utf8(u16)
        assert r == ("OK", len(u8)) and d.tobytes() == u8, hex(cp)
        # the same character as UTF-16BE (each word's bytes exchanged) and as one UTF-32 unit
        be = u16.byteswap()
        assert codec.validate_utf16be(be) == ("OK", len(u16)), hex(cp)
        r, d = codec.convert_utf16be_to_utf8(be)
        assert r == ("OK", len(u8)) and d.tobytes() == u8, hex(cp)
        r, d = codec.convert_utf8_to_utf16be(u8)
        assert r == ("OK", len(u16)) and np.array_equal(d, be), hex(cp)
        u32 = np.array([cp], dtype=np.uint32)
        assert codec.validate_utf32(u32) == ("OK", 1), hex(cp)
        r, d = codec.convert_utf8_to_utf32(u8)
        assert r == ("OK", 1) and np.array_equal(d, u32), hex(cp)
        r, d = codec.convert_utf32_to_utf8(u32)
        assert r == ("OK", len(u8)) and d.tobytes() == u8, hex(cp)
        r, d = codec.convert_utf32_to_utf16le(u32)
        assert r == ("OK", len(u16)) and np.array_equal(d, u16), hex(cp)
        r, d = codec.convert_utf16le_to_utf32(u16)
        assert r == ("OK", 1) and np.array_equal(d, u32), hex(cp)
    # all the fixture's characters in one string, then cut at every capacity
    all8 = b"".join(s[1] for s in scal)
    all16 = np.concatenate([s[2] for s in scal])
    r, d = codec.convert_utf8_to_utf16le(all8)
    assert r == ("OK", all16.size) and np.array_equal(d, all16)
    for cap in range(all16.size):
        r, d = codec.convert_utf8_to_utf16le(all8, cap)
        assert r == ("OUTPUT_TOO_SMALL", all16.size) and np.array_equal(d, all16[:cap])
    for cap in range(len(all8)):
        r, d = codec.convert_utf16le_to_utf8(all16, cap)
        assert r == ("OUTPUT_TOO_SMALL", len(all8)) and d.tobytes() == all8[:cap]

    for arr, kind, off in golden_invalid("utf8_invalid.txt", 8):
        assert codec.validate_utf8(arr) == (kind, off), arr.tobytes().hex()
        r, _ = codec.convert_utf8_to_utf16le(arr, 16)
        assert r == (kind, off), arr.tobytes().hex()
        r, _ = codec.convert_utf8_to_utf32(arr, 16)
        assert r == (kind, off), arr.tobytes().hex()
        # CPython's strict decoder reports the same first offset
        try:
            arr.tobytes().decode("utf-8")
            raise AssertionError("CPython accepted " + arr.tobytes().hex())
        except UnicodeDecodeError as e:
            assert e.start == off, arr.tobytes().hex()
    for arr, kind, off in golden_invalid("utf16_invalid.txt", 16):
        assert codec.validate_utf16le(arr) == (kind, off), arr
        r, _ = codec.convert_utf16le_to_utf8(arr, 16)
        assert r == (kind, off), arr
        r, _ = codec.convert_utf16le_to_utf32(arr, 16)
        assert r == (kind, off), arr
        assert codec.validate_utf16be(arr.byteswap()) == (kind, off), arr
        try:
            arr.tobytes().decode("utf-16-le")
            raise AssertionError("CPython accepted %r" % arr)
        except UnicodeDecodeError as e:
            assert e.start == 2 * off, arr


def all_scalars():
    cps = np.concatenate([np.arange(0, 0xD800), np.arange(0xE000, 0x110000)]).astype(np.uint32)
    assert cps.size == 1_112_064
    return cps


def check_all_scalars(codec):
    """Round trip of every Unicode scalar value against CPython's encoders."""
    cps = all_scalars()
    s = cps.astype("<u4").tobytes().decode("utf-32-le")
    u8 = np.frombuffer(s.encode("utf-8"), dtype=np.uint8)
    u16 = np.frombuffer(s.encode("utf-16-le"), dtype=np.uint16)
    assert codec.validate_utf8(u8) == ("OK", u8.size)
    assert codec.validate_utf16le(u16) == ("OK", u16.size)
    assert codec.utf16_length_from_utf8(u8) == u16.size
    assert codec.utf8_length_from_utf16le(u16) == u8.size
    r, d = codec.convert_utf8_to_utf16le(u8)
    assert r == ("OK", u16.size)
    assert np.array_equal(d, u16)
    r, d = codec.convert_utf16le_to_utf8(u16)
    assert r == ("OK", u8.size)
    assert np.array_equal(d, u8)
    # per-character sizes (Section 3): 1 byte below U+80, 2 below U+800, 3 below U+10000, else 4
    sizes = np.where(cps < 0x80, 1, np.where(cps < 0x800, 2, np.where(cps < 0x10000, 3, 4)))
    assert int(sizes.sum()) == u8.size


def check_all_scalars_utf16be(codec):
    """UTF-16BE (RFC 2781 byte order) against CPython's utf-16-be codec: every scalar value
    round trips, and the first unpaired surrogate of random word strings is where CPython's
    strict decoder reports it."""
    cps = all_scalars()
    s = cps.astype("<u4").tobytes().decode("utf-32-le")
    u8 = np.frombuffer(s.encode("utf-8"), dtype=np.uint8)
    be = np.frombuffer(s.encode("utf-16-be"), dtype=np.uint16)  # the words as they lie in memory
    assert codec.validate_utf16be(be) == ("OK", be.size)
    assert codec.utf8_length_from_utf16be(be) == u8.size
    r, d = codec.convert_utf16be_to_utf8(be)
    assert r == ("OK", u8.size) and np.array_equal(d, u8)
    r, d = codec.convert_utf8_to_utf16be(u8)
    assert r == ("OK", be.size) and d.tobytes() == s.encode("utf-16-be")
    rng = np.random.default_rng(7)
    words = np.array([0x41, 0x3B1, 0x4E2D, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xE000, 0xFFFD], dtype=">u2")
    for _ in range(20000):
        w = rng.choice(words, size=int(rng.integers(1, 9)))
        raw = w.tobytes()  # big-endian bytes
        mem = np.frombuffer(raw, dtype=np.uint16)
        try:
            raw.decode("utf-16-be")
            want = ("OK", mem.size)
        except UnicodeDecodeError as e:
            want = ("SURROGATE", e.start // 2)
        assert codec.validate_utf16be(mem) == want, (raw.hex(), want)
        r, _ = codec.convert_utf16be_to_utf8(mem)
        assert r == (want if want[0] != "OK" else ("OK", len(raw.decode("utf-16-be").encode("utf-8"))))


def check_all_scalars_utf32(codec):
    """UTF-32 against CPython's utf-32-le codec: every scalar value round trips through UTF-8
    and UTF-16LE, the lengths are exact, and the first invalid unit of random unit strings (above 10FFFF, or
    a surrogate value) is where CPython's strict decoder reports it, with the kind its value
    gives."""
    cps = all_scalars()
    s = cps.astype("<u4").tobytes().decode("utf-32-le")
    u8 = np.frombuffer(s.encode("utf-8"), dtype=np.uint8)
    u32 = np.frombuffer(s.encode("utf-32-le"), dtype=np.uint32)
    assert codec.validate_utf32(u32) == ("OK", u32.size)
    assert codec.utf8_length_from_utf32(u32) == u8.size
    assert codec.utf32_length_from_utf8(u8) == u32.size
    r, d = codec.convert_utf32_to_utf8(u32)
    assert r == ("OK", u8.size) and np.array_equal(d, u8)
    r, d = codec.convert_utf8_to_utf32(u8)
    assert r == ("OK", u32.size) and np.array_equal(d, u32)
    u16 = np.frombuffer(s.encode("utf-16-le"), dtype=np.uint16)
    assert codec.utf16_length_from_utf32(u32) == u16.size
    assert codec.utf32_length_from_utf16le(u16) == u32.size
    r, d = codec.convert_utf32_to_utf16le(u32)
    assert r == ("OK", u16.size) and np.array_equal(d, u16)
    r, d = codec.convert_utf16le_to_utf32(u16)
    assert r == ("OK", u32.size) and np.array_equal(d, u32)
    # UTF-16LE -> UTF-32 reports the first unpaired surrogate where CPython's utf-16-le decoder does
    rng16 = np.random.default_rng(9)
    words = np.array([0x41, 0x3B1, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xE000], dtype="<u2")
    for _ in range(20000):
        w = rng16.choice(words, size=int(rng16.integers(1, 9)))
        try:
            text = w.tobytes().decode("utf-16-le")
            want = ("OK", len(text))
        except UnicodeDecodeError as e:
            want = ("SURROGATE", e.start // 2)
        r, d = codec.convert_utf16le_to_utf32(w)
        assert r == want, (w, r, want)
        if want[0] == "OK":
            assert d.tobytes() == text.encode("utf-32-le")
    rng = np.random.default_rng(8)
    units = np.array([0x41, 0x7FF, 0xFFFF, 0x10000, 0x10FFFF, 0xD7FF, 0xD800, 0xDFFF, 0xE000, 0x110000,
                      0xFFFFFFFF], dtype="<u4")
    for _ in range(20000):
        u = rng.choice(units, size=int(rng.integers(1, 9)))
        try:
            text = u.tobytes().decode("utf-32-le")
            want = ("OK", u.size)
        except UnicodeDecodeError as e:
            bad = int(u[e.start // 4])
            want = ("TOO_LARGE" if bad > 0x10FFFF else "SURROGATE", e.start // 4)
        assert codec.validate_utf32(u) == want, (u, want)
        r, d = codec.convert_utf32_to_utf8(u)
        if want[0] == "OK":
            assert r == ("OK", len(text.encode("utf-8"))) and d.tobytes() == text.encode("utf-8")
        else:
            assert r == want
        r, d = codec.convert_utf32_to_utf16le(u)
        if want[0] == "OK":
            assert r == ("OK", len(text.encode("utf-16-le")) // 2) and d.tobytes() == text.encode("utf-16-le")
        else:
            assert r == want


def check_bruteforce(bf, max_len=3):
    """Every UTF-8 string of 1..max_len bytes against the second formulation."""
    assert bf.mixed_dead_prefixes() == 0
    for n in range(1, max_len + 1):
        mism, stats = bf.utf8(n, nthreads=os.cpu_count() or 4, roundtrip=True)
        assert mism == 0, (n, mism, bytes(int(x) for x in stats[9:9 + int(stats[13])]).hex())
    # known totals: valid one-byte strings are the 128 ASCII bytes; two-byte strings are
    # ASCII pairs (128^2) plus two-byte characters (30 leads C2-DF x 64 continuations)
    _, s1 = bf.utf8(1, 1, False)
    _, s2 = bf.utf8(2, 1, False)
    assert s1[0] == 128
    assert s2[0] == 128 * 128 + 30 * 64


def check_cpython_offsets(bf, three_byte_leads=range(0xC0, 0x100)):
    """CPython's first-error offsets on every 1- and 2-byte string and on every 3-byte string
    whose first byte is in three_byte_leads."""
    for n in (1, 2):
        kind, off = bf.table(n)
        for x in range(1 << (8 * n)):
            s = bytes((x >> (8 * k)) & 0xFF for k in range(n))
            try:
                s.decode("utf-8")
                ok, start = True, 255
            except UnicodeDecodeError as e:
                ok, start = False, e.start
            assert (kind[x] == 0) == ok, s.hex()
            assert off[x] == start, s.hex()
    kind, off = bf.table(3)
    for b0 in three_byte_leads:
        for t in range(65536):
            x = b0 | (t << 8)
            s = bytes((b0, t & 0xFF, t >> 8))
            try:
                s.decode("utf-8")
                ok, start = True, 255
            except UnicodeDecodeError as e:
                ok, start = False, e.start
            if (kind[x] == 0) != ok or off[x] != start:
                raise AssertionError(s.hex())


def check_utf16_pairs(bf, codec, full=True):
    if full:
        mism, stats = bf.utf16_pairs(nthreads=os.cpu_count() or 4)
        assert mism == 0, hex(int(stats[1]))
        # valid pairs: two non-surrogates, or a high followed by a low
        assert stats[0] == (65536 - 2048) ** 2 + 1024 * 1024
    # CPython on pairs drawn from the boundaries and all surrogate words
    words = np.array(
        sorted(set([0, 0x41, 0x7F, 0x80, 0x7FF, 0x800, 0xD7FF, 0xE000, 0xFFFD, 0xFFFF]
                   + list(range(0xD800, 0xD810)) + list(range(0xDBF0, 0xDC10))
                   + list(range(0xDFF0, 0xE000)))), dtype=np.uint16)
    kind, off = bf.utf16_pair_table(words)
    for i, a in enumerate(words):
        for j, b in enumerate(words):
            s = np.array([a, b], dtype=np.uint16).tobytes()
            try:
                s.decode("utf-16-le")
                ok, start = True, 255
            except UnicodeDecodeError as e:
                ok, start = False, e.start // 2
            assert (kind[i, j] == 0) == ok and off[i, j] == start, (hex(a), hex(b))
    # every valid surrogate pair converts to the scalar CPython decodes it to
    hi = np.repeat(np.arange(0xD800, 0xDC00, dtype=np.uint16), 1024)
    lo = np.tile(np.arange(0xDC00, 0xE000, dtype=np.uint16), 1024)
    pairs = np.stack([hi, lo], axis=1).reshape(-1)
    r, d = codec.convert_utf16le_to_utf8(pairs)
    expect = pairs.tobytes().decode("utf-16-le").encode("utf-8")
    assert r == ("OK", len(expect)) and d.tobytes() == expect


def check_length_closed_forms(codec):
    """Length formulas on strings whose answer is known without decoding."""
    rng = np.random.default_rng(7)
    for cp_lo, cp_hi, u8_per, u16_per in [
        (0x00, 0x80, 1, 1), (0x80, 0x800, 2, 1), (0x800, 0xD800, 3, 1),
        (0xE000, 0x10000, 3, 1), (0x10000, 0x110000, 4, 2)]:
        cps = rng.integers(cp_lo, cp_hi, size=1000).astype("<u4")
        s = cps.tobytes().decode("utf-32-le")
        u8 = np.frombuffer(s.encode("utf-8"), dtype=np.uint8)
        u16 = np.frombuffer(s.encode("utf-16-le"), dtype=np.uint16)
        assert u8.size == 1000 * u8_per and u16.size == 1000 * u16_per
        assert codec.utf16_length_from_utf8(u8) == 1000 * u16_per
        assert codec.utf8_length_from_utf16le(u16) == 1000 * u8_per
        # UTF-32: one unit per character whatever its size
        assert codec.utf8_length_from_utf32(cps) == 1000 * u8_per
        assert codec.utf16_length_from_utf32(cps) == 1000 * u16_per
        assert codec.utf32_length_from_utf8(u8) == 1000
        assert codec.utf32_length_from_utf16le(u16) == 1000
    # formulas on arbitrary (invalid) input: one word per non-continuation byte plus one per
    # byte F0-FF; two bytes per surrogate word
    junk = np.arange(256, dtype=np.uint8)
    assert codec.utf16_length_from_utf8(junk) == 256 - 64 + 16
    sur = np.arange(0xD800, 0xE000, dtype=np.uint16)
    assert codec.utf8_length_from_utf16le(sur) == 2 * 2048
    assert codec.utf16_length_from_utf8(b"") == 0 and codec.utf8_length_from_utf16le(b"") == 0
    # the UTF-32 lengths on arbitrary input: one unit per non-continuation byte; one per word
    # that is not a second surrogate (a first surrogate stands for its pair); UTF-8 bytes and
    # UTF-16 words of a unit by its value alone (a surrogate value as a three-byte form, a unit
    # above 10FFFF as a four-byte form or a pair)
    assert codec.utf32_length_from_utf8(junk) == 256 - 64
    assert codec.utf32_length_from_utf16le(np.arange(0xD800, 0xDC00, dtype=np.uint16)) == 1024
    assert codec.utf32_length_from_utf16le(np.arange(0xDC00, 0xE000, dtype=np.uint16)) == 0
    bad = np.array([0xD800, 0xDFFF, 0x110000, 0xFFFFFFFF], dtype=np.uint32)
    assert codec.utf8_length_from_utf32(bad) == 3 + 3 + 4 + 4
    assert codec.utf16_length_from_utf32(bad) == 1 + 1 + 2 + 2
    empty32 = np.zeros(0, dtype=np.uint32)
    assert codec.utf8_length_from_utf32(empty32) == 0 and codec.utf16_length_from_utf32(empty32) == 0
    assert codec.utf32_length_from_utf8(b"") == 0 and codec.utf32_length_from_utf16le(b"") == 0


def check_edge_cases(codec):
    """Empty inputs, and an input error that takes precedence over a too-small capacity (the
    error's offset lies past the capacity), for every transcoder; the units before the cut are
    still the conversion of the valid prefix."""
    e8, e16, e32 = np.zeros(0, np.uint8), np.zeros(0, np.uint16), np.zeros(0, np.uint32)
    assert codec.validate_utf8(e8) == ("OK", 0) and codec.validate_utf16le(e16) == ("OK", 0)
    assert codec.validate_utf16be(e16) == ("OK", 0) and codec.validate_utf32(e32) == ("OK", 0)
    for f, e in ((codec.convert_utf8_to_utf16le, e8), (codec.convert_utf16le_to_utf8, e16),
                 (codec.convert_utf8_to_utf16be, e8), (codec.convert_utf16be_to_utf8, e16),
                 (codec.convert_utf8_to_utf32, e8), (codec.convert_utf32_to_utf8, e32),
                 (codec.convert_utf16le_to_utf32, e16), (codec.convert_utf32_to_utf16le, e32)):
        assert f(e)[0] == ("OK", 0)
        assert f(e, 0)[0] == ("OK", 0)
    # "ab€" (U+20AC: E2 82 AC) then an invalid unit at index 5 (UTF-8) or 3 (words and units)
    u8 = np.frombuffer("ab€".encode() + b"\xff", np.uint8)
    u16 = np.array([0x61, 0x62, 0x20AC, 0xDC00], np.uint16)
    u32 = np.array([0x61, 0x62, 0x20AC, 0x110000], np.uint32)
    # (transcoder, input, expected result, first output unit as it lies in memory)
    cases = [(codec.convert_utf8_to_utf16le, u8, ("HEADER_BITS", 5), 0x61),
             (codec.convert_utf8_to_utf16be, u8, ("HEADER_BITS", 5), 0x6100),
             (codec.convert_utf8_to_utf32, u8, ("HEADER_BITS", 5), 0x61),
             (codec.convert_utf16le_to_utf8, u16, ("SURROGATE", 3), 0x61),
             (codec.convert_utf16be_to_utf8, u16.byteswap(), ("SURROGATE", 3), 0x61),
             (codec.convert_utf16le_to_utf32, u16, ("SURROGATE", 3), 0x61),
             (codec.convert_utf32_to_utf8, u32, ("TOO_LARGE", 3), 0x61),
             (codec.convert_utf32_to_utf16le, u32, ("TOO_LARGE", 3), 0x61)]
    for f, src, want, first in cases:
        for cap in (0, 1, 2):
            r, d = f(src, cap)
            assert r == want, (f.__name__, cap, r)
            assert cap == 0 or int(d[0]) == first, (f.__name__, cap, d)
