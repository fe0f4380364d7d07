"""The resumable (chunked) form against the reference codec: one input pushed in pieces of
random sizes (0 to a few thousand units, so that pieces cut characters, pairs and errors in
every way) must give exactly the whole-input result -- the first error's kind and offset, or
the total -- and outputs that concatenate to the whole-input output (of the valid prefix)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

MAX_CHUNK = 1 << 16


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_08692_gb300 as g
    from paper_2111_08692_gb300.build import build
    build()
    return g


def _pieces(n, rng, small):
    cuts, i = [], 0
    while i < n:
        k = int(rng.integers(0, 8)) if small else int(rng.integers(0, MAX_CHUNK // 4))
        cuts.append((i, min(n, i + k)))
        i = min(n, i + k)
    return cuts


def _run(ch, data, rng, small):
    outs, res = [], None
    pieces = _pieces(data.size, rng, small)
    for j, (a, b) in enumerate(pieces):
        out, res = ch.push(data[a:b], last=False)
        outs.append(out)
    out, res = ch.push(data[:0], last=True)
    outs.append(out)
    return res, (np.concatenate(outs) if outs else np.zeros(0))


def _check(lib, op, data, rng, small=False):
    ch = lib.Chunked(op, MAX_CHUNK)
    try:
        res, out = _run(ch, data, rng, small)
    finally:
        ch.close()
    if op == "validate_utf8":
        assert res == oracle.validate_utf8(data), (res, oracle.validate_utf8(data))
    elif op == "validate_utf16le":
        assert res == oracle.validate_utf16le(data), (res, oracle.validate_utf16le(data))
    else:
        if op == "convert_utf8_to_utf16le":
            want, wout = oracle.convert_utf8_to_utf16le(data)
            m = want[1] if want[0] == "OK" else oracle.utf16_length_from_utf8(data[:want[1]])
        else:
            want, wout = oracle.convert_utf16le_to_utf8(data)
            m = want[1] if want[0] == "OK" else oracle.utf8_length_from_utf16le(data[:want[1]])
        assert res == want, (res, want)
        assert out.size == m and np.array_equal(out, wout[:m])


OPS8 = ("validate_utf8", "convert_utf8_to_utf16le")
OPS16 = ("validate_utf16le", "convert_utf16le_to_utf8")


def test_profiles_and_sweeps_in_random_pieces(lib):
    rng = np.random.default_rng(91)
    for prof in ("mixed", "latin", "cjk", "emoji"):
        u8, u16 = W.profile_buffers(prof, 300_000, 150_000, 92, cache=False)
        for op in OPS8:
            _check(lib, op, u8, rng)
        for op in OPS16:
            _check(lib, op, u16, rng)
    for prof in ("cyrillic", "cjk"):
        for rate in (1e-4, 1e-2):
            d = W.sweep_buffers(prof, rate, n_bytes=1 << 18, seed=W.SWEEP_SEEDS[(prof, rate)], cache=False)
            for op in OPS8:
                _check(lib, op, d["u8"], rng)
                _check(lib, op, d["u8_cut_end"], rng)
            for op in OPS16:
                _check(lib, op, d["u16"], rng)
                _check(lib, op, d["u16_cut_end"], rng)


def test_tiny_pieces_cut_every_character(lib):
    """Pieces of 0 to 7 units, so that every multi-byte character and pair is cut somewhere, with
    errors of every kind near the cuts."""
    rng = np.random.default_rng(93)
    u8, u16 = W.profile_buffers("mixed", 6000, 3000, 94, cache=False)
    for op in OPS8:
        _check(lib, op, u8, rng, small=True)
    for op in OPS16:
        _check(lib, op, u16, rng, small=True)
    alphabet = np.array([0x41, 0x80, 0x9F, 0xA0, 0xBF, 0xC0, 0xC2, 0xDF, 0xE0, 0xED, 0xEF, 0xF0, 0xF4, 0xF5,
                         0xFF], np.uint8)
    words = np.array([0x41, 0x7FF, 0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0xE000], np.uint16)
    for _ in range(150):
        s8 = rng.choice(alphabet, size=int(rng.integers(1, 24)))
        s16 = rng.choice(words, size=int(rng.integers(1, 16)))
        for op in OPS8:
            _check(lib, op, s8, rng, small=True)
        for op in OPS16:
            _check(lib, op, s16, rng, small=True)


def test_small_output_buffer_is_retried_and_reset(lib):
    u8, _ = W.profile_buffers("cjk", 5000, 0, 95, cache=False)
    ch = lib.Chunked("convert_utf8_to_utf16le", MAX_CHUNK)
    try:
        out, res = ch.push(u8[:4000], out_cap=10)
        assert res[0] == "OUTPUT_TOO_SMALL" and out.size == 0
        need = res[1]
        out1, res = ch.push(u8[:4000], out_cap=need)
        assert res == ("OK", need) and out1.size == need
        out2, res = ch.push(u8[4000:], last=True)
        want, wout = oracle.convert_utf8_to_utf16le(u8)
        assert res == want and np.array_equal(np.concatenate([out1, out2]), wout)
        with pytest.raises(lib.GbuError):
            ch.push(u8[:10])  # a push after the last one
        ch.reset()
        out, res = ch.push(u8, last=True)
        assert res == want and np.array_equal(out, wout)
        with pytest.raises(lib.GbuError):
            ch.reset()
            ch.push(np.zeros(MAX_CHUNK + 1, np.uint8))  # above max_chunk_units
    finally:
        ch.close()
