"""Shared helpers for the GPU parity tests: run one operation through the C ABI and compare
it, bit for bit, with the reference codec on the same input."""
from __future__ import annotations

import numpy as np

import oracle

CANARY16 = 0xA5C3
CANARY8 = 0xA7


def _dev_copy(torch, data: np.ndarray, offset: int, pad: int = 64):
    """A device buffer holding `data` at element offset `offset` (so the view is unaligned),
    followed by `pad` spare elements; returns (buffer, view)."""
    t = torch.from_numpy(np.ascontiguousarray(data)) if data.size else torch.zeros(0, dtype=_tdtype(torch, data))
    buf = torch.zeros(data.size + offset + pad, dtype=t.dtype, device="cuda")
    view = buf[offset:offset + data.size]
    if data.size:
        view.copy_(t.to("cuda"))
    return buf, view


def _tdtype(torch, a):
    return torch.uint8 if a.dtype == np.uint8 else torch.int16


def as_torch_u16(torch, a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int16))


def check_utf8_input(codec, torch, data: np.ndarray, src_off: int = 0, dst_off: int = 0, cap=None):
    """Validation, UTF-16 length and UTF-8 -> UTF-16LE of `data` against the oracle."""
    from paper_2111_08692_gb300 import result_tuple
    data = np.ascontiguousarray(data, dtype=np.uint8)
    _, src = _dev_copy(torch, data, src_off)
    want_v = oracle.validate_utf8(data)
    got_v = result_tuple(codec.validate_utf8(src))
    assert got_v == want_v, ("validate_utf8", got_v, want_v, data.size, src_off)
    want_len = oracle.utf16_length_from_utf8(data)
    got_len = int(codec.utf16_length_from_utf8(src).item())
    assert got_len == want_len, ("utf16_length_from_utf8", got_len, want_len)
    if cap is None:
        cap = want_len
    want, odst = oracle.convert_utf8_to_utf16le(data, cap)
    guard = 40
    dbuf = torch.full((dst_off + cap + guard,), CANARY16, dtype=torch.int32, device="cuda").to(torch.int16)
    dst = dbuf[dst_off:dst_off + cap]
    got = result_tuple(codec.convert_utf8_to_utf16le(src, dst, cap=cap))
    assert got == want, ("convert_utf8_to_utf16le", got, want, data.size, src_off, dst_off, cap)
    host = dbuf.cpu().numpy().view(np.uint16)
    out = host[dst_off:dst_off + cap]
    kind, count = want
    if kind == "OK":
        m = count
    elif kind == "OUTPUT_TOO_SMALL":
        m = cap
    else:
        m = min(oracle.utf16_length_from_utf8(data[:count]), cap)
    if not np.array_equal(out[:m], odst[:m]):
        bad = int(np.flatnonzero(out[:m] != odst[:m])[0])
        raise AssertionError(("utf16 output differs", bad, int(out[bad]), int(odst[bad]), data.size))
    assert np.all(host[:dst_off] == CANARY16), "write before dst"
    assert np.all(host[dst_off + cap:] == CANARY16), "write at or past cap"
    return want_v, want


def check_utf16_input(codec, torch, data: np.ndarray, src_off: int = 0, dst_off: int = 0, cap=None):
    """Validation, UTF-8 length and UTF-16LE -> UTF-8 of `data` (uint16) against the oracle."""
    from paper_2111_08692_gb300 import result_tuple
    data = np.ascontiguousarray(data, dtype=np.uint16)
    buf = torch.zeros(data.size + src_off + 64, dtype=torch.int16, device="cuda")
    src = buf[src_off:src_off + data.size]
    if data.size:
        src.copy_(as_torch_u16(torch, data).to("cuda"))
    want_v = oracle.validate_utf16le(data)
    got_v = result_tuple(codec.validate_utf16le(src))
    assert got_v == want_v, ("validate_utf16le", got_v, want_v, data.size, src_off)
    want_len = oracle.utf8_length_from_utf16le(data)
    got_len = int(codec.utf8_length_from_utf16le(src).item())
    assert got_len == want_len, ("utf8_length_from_utf16le", got_len, want_len)
    if cap is None:
        cap = want_len
    want, odst = oracle.convert_utf16le_to_utf8(data, cap)
    guard = 48
    dbuf = torch.full((dst_off + cap + guard,), CANARY8, dtype=torch.uint8, device="cuda")
    dst = dbuf[dst_off:dst_off + cap]
    got = result_tuple(codec.convert_utf16le_to_utf8(src, dst, cap=cap))
    assert got == want, ("convert_utf16le_to_utf8", got, want, data.size, src_off, dst_off, cap)
    host = dbuf.cpu().numpy()
    out = host[dst_off:dst_off + cap]
    kind, count = want
    if kind == "OK":
        m = count
    elif kind == "OUTPUT_TOO_SMALL":
        m = cap
    else:
        m = min(oracle.utf8_length_from_utf16le(data[:count]), cap)
    if not np.array_equal(out[:m], odst[:m]):
        bad = int(np.flatnonzero(out[:m] != odst[:m])[0])
        raise AssertionError(("utf8 output differs", bad, int(out[bad]), int(odst[bad]), data.size))
    assert np.all(host[:dst_off] == CANARY8), "write before dst"
    assert np.all(host[dst_off + cap:] == CANARY8), "write at or past cap"
    return want_v, want


def char_starts_utf8(data: np.ndarray) -> np.ndarray:
    """Indices of bytes that are not continuation bytes (test-side helper for placing
    injected errors at character boundaries of VALID data)."""
    return np.flatnonzero((data & 0xC0) != 0x80)
