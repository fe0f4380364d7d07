"""The six host-synchronising calls (gbu_*_sync) through the C ABI against the oracle: the
result by value, and for the transcoders every defined output unit and the guard zones."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

CANARY16, CANARY8 = 0x5A5A, 0x5A


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
    c = Codec(0, max_units=1 << 26)
    yield c
    c.close()


def _utf8_cases():
    """(name, bytes): valid mixed text over several partitions, the same with an invalid byte,
    a cut sequence at the end, and the empty input."""
    u8, _ = W.profile_buffers("mixed", (3 << 20) + 11, 0, 501, cache=False)
    bad = u8.copy()
    k = 2_000_001
    while (bad[k] & 0xC0) == 0x80:
        k -= 1
    bad[k] = 0xC1
    i = 100000
    while (u8[i] & 0xC0) == 0x80:  # back to a character start
        i -= 1
    cut = np.concatenate([u8[:i], np.array([0xF0, 0x9F], np.uint8)])
    return [("valid", u8), ("invalid", bad), ("cut", cut), ("empty", np.zeros(0, np.uint8))]


def _utf16_cases():
    u8, u16 = W.profile_buffers("mixed", 16, (2 << 20) + 5, 502, cache=False)
    lone = u16.copy()
    lone[1_500_003] = 0xDC00
    if lone[1_500_002] >= 0xD800 and lone[1_500_002] <= 0xDBFF:
        lone[1_500_002] = 0x41
    return [("valid", u16), ("lone_low", lone), ("cut_high", np.concatenate([u16[:4099], [0xD83D]]).astype(np.uint16)),
            ("empty", np.zeros(0, np.uint16))]


def _dev(torch, a):
    if a.dtype == np.uint16:
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int16))
    else:
        t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if a.size else torch.zeros(0, dtype=t.dtype, device="cuda")


def _defined_prefix(want, cap, prefix_len):
    kind, count = want
    if kind == "OK":
        return count
    if kind == "OUTPUT_TOO_SMALL":
        return cap
    return min(prefix_len(count), cap)


def test_sync_validation_and_lengths_match_the_oracle(codec, torch):
    for name, data in _utf8_cases():
        src = _dev(torch, data)
        assert codec.validate_utf8_sync(src) == oracle.validate_utf8(data), name
        assert codec.utf16_length_from_utf8_sync(src) == ("OK", oracle.utf16_length_from_utf8(data)), name
    for name, data in _utf16_cases():
        src = _dev(torch, data)
        assert codec.validate_utf16le_sync(src) == oracle.validate_utf16le(data), name
        assert codec.utf8_length_from_utf16le_sync(src) == ("OK", oracle.utf8_length_from_utf16le(data)), name


@pytest.mark.parametrize("short", [False, True])
def test_sync_transcoders_match_the_oracle(codec, torch, short):
    """Each transcoder with a capacity of the exact length, or one unit short of it."""
    for name, data in _utf8_cases():
        src = _dev(torch, data)
        cap = max(oracle.utf16_length_from_utf8(data) - (1 if short else 0), 0)
        want, odst = oracle.convert_utf8_to_utf16le(data, cap)
        buf = torch.full((cap + 24,), CANARY16, dtype=torch.int16, device="cuda")
        got = codec.convert_utf8_to_utf16le_sync(src, buf[:cap], cap=cap)
        assert got == want, (name, got, want)
        m = _defined_prefix(want, cap, lambda c: oracle.utf16_length_from_utf8(data[:c]))
        host = buf.cpu().numpy().view(np.uint16)
        assert np.array_equal(host[:m], odst[:m]), name
        assert np.all(host[cap:] == CANARY16), name
    for name, data in _utf16_cases():
        src = _dev(torch, data)
        cap = max(oracle.utf8_length_from_utf16le(data) - (1 if short else 0), 0)
        want, odst = oracle.convert_utf16le_to_utf8(data, cap)
        buf = torch.full((cap + 24,), CANARY8, dtype=torch.uint8, device="cuda")
        got = codec.convert_utf16le_to_utf8_sync(src, buf[:cap], cap=cap)
        assert got == want, (name, got, want)
        m = _defined_prefix(want, cap, lambda c: oracle.utf8_length_from_utf16le(data[:c]))
        host = buf.cpu().numpy()
        assert np.array_equal(host[:m], odst[:m]), name
        assert np.all(host[cap:] == CANARY8), name


def test_sync_launch_errors_come_back_by_value(codec, torch):
    """An argument the launch refuses (a NULL source with n > 0, an odd UTF-16 destination)
    comes back as {BAD_ARGUMENT, 0}, with nothing enqueued."""
    from paper_2111_08692_gb300 import lib
    L = lib()
    r = L.gbu_validate_utf8_sync(codec.ctx, None, 16, None)
    assert (r.status, r.count) == (17, 0)
    src = torch.zeros(8, dtype=torch.uint8, device="cuda")
    dst = torch.zeros(16, dtype=torch.uint8, device="cuda")
    r = L.gbu_convert_utf8_to_utf16le_sync(codec.ctx, src.data_ptr(), 8, dst.data_ptr() + 1, 4, None)
    assert (r.status, r.count) == (17, 0)
