"""Pins the reference codec (oracle/) to the paper's Section 3 and to independent decoders.

CPU only.  See tests/oracle_pins.py for what each check compares against.
"""
import os

import pytest

import oracle
import oracle_pins as P
from bfhelper import BF, build


@pytest.fixture(scope="module")
def bf():
    return BF(build())


def test_golden_fixtures():
    P.check_golden(oracle.default())


def test_all_scalar_values_round_trip_against_cpython():
    P.check_all_scalars(oracle.default())


def test_utf16be_against_cpython():
    P.check_all_scalars_utf16be(oracle.default())


def test_utf32_against_cpython():
    P.check_all_scalars_utf32(oracle.default())


def test_bruteforce_up_to_three_bytes(bf):
    P.check_bruteforce(bf, max_len=3)


@pytest.mark.slow
def test_bruteforce_every_four_byte_string(bf):
    mism, stats = bf.utf8(4, nthreads=os.cpu_count() or 4, roundtrip=True)
    assert mism == 0, bytes(int(x) for x in stats[9:13]).hex()
    # every kind occurs among four-byte strings
    assert all(stats[1 + k] > 0 for k in range(7)), stats


def test_cpython_first_error_offsets(bf):
    P.check_cpython_offsets(bf)


@pytest.mark.slow
def test_every_utf16_word_pair(bf):
    P.check_utf16_pairs(bf, oracle.default(), full=True)


def test_length_formulas_closed_forms():
    P.check_length_closed_forms(oracle.default())


def test_empty_inputs():
    o = oracle.default()
    assert o.validate_utf8(b"") == ("OK", 0)
    assert o.validate_utf16le(b"") == ("OK", 0)
    assert o.convert_utf8_to_utf16le(b"")[0] == ("OK", 0)
    assert o.convert_utf16le_to_utf8(b"")[0] == ("OK", 0)


def test_edge_cases_every_transcoder():
    P.check_edge_cases(oracle.default())


def test_error_takes_precedence_over_capacity():
    o = oracle.default()
    src = "ab€".encode() + b"\xff"
    r, d = o.convert_utf8_to_utf16le(src, cap=1)
    assert r == ("HEADER_BITS", 5)
    assert d[0] == ord("a")


def test_batched_loops_match_single_calls():
    o = oracle.default()
    strs = [b"", "héllo".encode(), b"\xc3", "中\U0001F600".encode(), b"ok\x80"]
    buf = b"".join(strs)
    off = [0]
    for s in strs:
        off.append(off[-1] + len(s))
    res = o.validate_utf8_batched(buf, off)
    assert res == [o.validate_utf8(s) for s in strs]
    dst_off = [0]
    for s in strs:
        dst_off.append(dst_off[-1] + len(s))
    res, dst = o.convert_utf8_to_utf16le_batched(buf, off, dst_off)
    for i, s in enumerate(strs):
        r, d = o.convert_utf8_to_utf16le(s, cap=len(s))
        assert res[i] == r
        assert (dst[dst_off[i]:dst_off[i + 1]][: r[1] if r[0] == "OK" else 0] ==
                d[: r[1] if r[0] == "OK" else 0]).all()
