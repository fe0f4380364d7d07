"""UTF-32 through the C ABI against the reference codec's UTF-32 functions, bit for bit:
validation, the lengths, and both transcoding directions between UTF-32 and UTF-8 / UTF-16LE,
on the profiles, invalid units near tile and partition boundaries, the UTF-8 and UTF-16
invalid-input sweeps, surrogate pairs cut by partitions, unaligned views and too-small
outputs."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import CANARY16, CANARY8, as_torch_u16

pytestmark = pytest.mark.gpu
CANARY32 = 0x5A5A5A5A


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


def to_utf32(u8):
    return np.frombuffer(u8.tobytes().decode("utf-8").encode("utf-32-le"), dtype=np.uint32)


def check_utf32_input(codec, torch, u32, src_off=0, dst_off=0, cap=None):
    from paper_2111_08692_gb300 import result_tuple
    u32 = np.ascontiguousarray(u32, dtype=np.uint32)
    buf = torch.zeros(u32.size + src_off + 16, dtype=torch.int32, device="cuda")
    src = buf[src_off:src_off + u32.size]
    if u32.size:
        src.copy_(torch.from_numpy(u32.view(np.int32)).to("cuda"))
    assert result_tuple(codec.validate_utf32(src)) == oracle.validate_utf32(u32)
    want_len = oracle.utf8_length_from_utf32(u32)
    assert int(codec.utf8_length_from_utf32(src).item()) == want_len
    cap = want_len if cap is None else cap
    want, odst = oracle.convert_utf32_to_utf8(u32, cap)
    dbuf = torch.full((dst_off + cap + 48,), CANARY8, dtype=torch.uint8, device="cuda")
    got = result_tuple(codec.convert_utf32_to_utf8(src, dbuf[dst_off:dst_off + cap], cap=cap))
    assert got == want, (got, want, u32.size, src_off, dst_off, cap)
    host = dbuf.cpu().numpy()
    m = want[1] if want[0] == "OK" else (cap if want[0] == "OUTPUT_TOO_SMALL" else
                                          min(oracle.utf8_length_from_utf32(u32[:want[1]]), cap))
    assert np.array_equal(host[dst_off:dst_off + m], odst[:m])
    assert np.all(host[:dst_off] == CANARY8) and np.all(host[dst_off + cap:] == CANARY8)


def check_utf8_to_32(codec, torch, u8, src_off=0, dst_off=0, cap=None):
    from paper_2111_08692_gb300 import result_tuple
    u8 = np.ascontiguousarray(u8, dtype=np.uint8)
    buf = torch.zeros(u8.size + src_off + 64, dtype=torch.uint8, device="cuda")
    src = buf[src_off:src_off + u8.size]
    if u8.size:
        src.copy_(torch.from_numpy(u8.copy()).to("cuda"))
    want_len = oracle.utf32_length_from_utf8(u8)
    assert int(codec.utf32_length_from_utf8(src).item()) == want_len
    cap = want_len if cap is None else cap
    want, odst = oracle.convert_utf8_to_utf32(u8, cap)
    dbuf = torch.full((dst_off + cap + 24,), CANARY32, dtype=torch.int32, device="cuda")
    got = result_tuple(codec.convert_utf8_to_utf32(src, dbuf[dst_off:dst_off + cap], cap=cap))
    assert got == want, (got, want, u8.size, src_off, dst_off, cap)
    host = dbuf.cpu().numpy().view(np.uint32)
    m = want[1] if want[0] == "OK" else (cap if want[0] == "OUTPUT_TOO_SMALL" else
                                          min(oracle.utf32_length_from_utf8(u8[:want[1]]), cap))
    assert np.array_equal(host[dst_off:dst_off + m], odst[:m])
    assert np.all(host[:dst_off] == CANARY32) and np.all(host[dst_off + cap:] == CANARY32)


@pytest.mark.parametrize("profile", W.PROFILE_ORDER + ("mixed",))
def test_profiles(codec, torch, profile):
    u8, _ = W.profile_buffers(profile, 1 << 21, 0, 71, cache=False)
    u32 = to_utf32(u8)
    check_utf32_input(codec, torch, u32)
    check_utf32_input(codec, torch, u32, src_off=3, dst_off=5)
    check_utf8_to_32(codec, torch, u8)
    check_utf8_to_32(codec, torch, u8, src_off=3, dst_off=1)


def test_invalid_units_near_boundaries(codec, torch):
    u8, _ = W.profile_buffers("mixed", 5 * 16384, 0, 72, cache=False)
    base = to_utf32(u8)
    for b in (128, 1024, 4096, 8192, base.size - 1):
        for d in (-2, -1, 0, 1):
            for bad in (0x110000, 0xD800, 0xDFFF, 0xFFFFFFFF):
                i = min(max(b + d, 0), base.size - 1)
                x = base.copy()
                x[i] = bad
                x[min(i + 37, x.size - 1)] = 0xDC00  # a later error never wins
                check_utf32_input(codec, torch, x)
    for n in (0, 1, 3, 4, 5, 127, 128, 129):
        check_utf32_input(codec, torch, base[:n])
    total = oracle.utf8_length_from_utf32(base)
    for cap in (0, 1, 15, 16, 17, 4095, total - 1):
        check_utf32_input(codec, torch, base, cap=cap, dst_off=cap % 16)


def test_utf8_sweep_and_capacity(codec, torch):
    for profile in ("cyrillic", "cjk"):
        for rate in (1e-6, 1e-4, 1e-2):
            d = W.sweep_buffers(profile, rate, n_bytes=1 << 22, seed=W.SWEEP_SEEDS[(profile, rate)], cache=False)
            check_utf8_to_32(codec, torch, d["u8"])
            check_utf8_to_32(codec, torch, d["u8_cut_end"])
    u8, _ = W.profile_buffers("emoji", 3 * 16384 + 7, 0, 73, cache=False)
    total = oracle.utf32_length_from_utf8(u8)
    for cap in (0, 1, 3, 4, 5, 4095, total - 1):
        check_utf8_to_32(codec, torch, u8, cap=cap, dst_off=cap % 4)
    for n in (0, 1, 2, 3, 15, 16, 17, 511, 512, 513):
        check_utf8_to_32(codec, torch, u8[:n])


def check_utf32_to_16(codec, torch, u32, dst_off=0, cap=None):
    from paper_2111_08692_gb300 import result_tuple
    u32 = np.ascontiguousarray(u32, dtype=np.uint32)
    src = torch.from_numpy(u32.view(np.int32).copy()).to("cuda") if u32.size else torch.zeros(0, dtype=torch.int32,
                                                                                                 device="cuda")
    want_len = oracle.utf16_length_from_utf32(u32)
    assert int(codec.utf16_length_from_utf32(src).item()) == want_len
    cap = want_len if cap is None else cap
    want, odst = oracle.convert_utf32_to_utf16le(u32, cap)
    dbuf = torch.full((dst_off + cap + 40,), CANARY16, dtype=torch.int32, device="cuda").to(torch.int16)
    got = result_tuple(codec.convert_utf32_to_utf16le(src, dbuf[dst_off:dst_off + cap], cap=cap))
    assert got == want, (got, want, u32.size, dst_off, cap)
    host = dbuf.cpu().numpy().view(np.uint16)
    m = want[1] if want[0] == "OK" else (cap if want[0] == "OUTPUT_TOO_SMALL" else
                                          min(oracle.utf16_length_from_utf32(u32[:want[1]]), cap))
    assert np.array_equal(host[dst_off:dst_off + m], odst[:m])
    assert np.all(host[:dst_off] == CANARY16) and np.all(host[dst_off + cap:] == CANARY16)


def check_utf16_to_32(codec, torch, u16, src_off=0, dst_off=0, cap=None):
    from paper_2111_08692_gb300 import result_tuple
    u16 = np.ascontiguousarray(u16, dtype=np.uint16)
    buf = torch.zeros(u16.size + src_off + 16, dtype=torch.int16, device="cuda")
    src = buf[src_off:src_off + u16.size]
    if u16.size:
        src.copy_(as_torch_u16(torch, u16).to("cuda"))
    want_len = oracle.utf32_length_from_utf16le(u16)
    assert int(codec.utf32_length_from_utf16le(src).item()) == want_len
    cap = want_len if cap is None else cap
    want, odst = oracle.convert_utf16le_to_utf32(u16, cap)
    dbuf = torch.full((dst_off + cap + 24,), CANARY32, dtype=torch.int32, device="cuda")
    got = result_tuple(codec.convert_utf16le_to_utf32(src, dbuf[dst_off:dst_off + cap], cap=cap))
    assert got == want, (got, want, u16.size, src_off, dst_off, cap)
    host = dbuf.cpu().numpy().view(np.uint32)
    m = want[1] if want[0] == "OK" else (cap if want[0] == "OUTPUT_TOO_SMALL" else
                                          min(oracle.utf32_length_from_utf16le(u16[:want[1]]), cap))
    assert np.array_equal(host[dst_off:dst_off + m], odst[:m])
    assert np.all(host[:dst_off] == CANARY32) and np.all(host[dst_off + cap:] == CANARY32)


@pytest.mark.parametrize("profile", W.PROFILE_ORDER + ("mixed",))
def test_utf16_utf32_profiles(codec, torch, profile):
    u8, u16 = W.profile_buffers(profile, 1 << 20, 1 << 20, 74, cache=False)
    check_utf32_to_16(codec, torch, to_utf32(u8))
    check_utf32_to_16(codec, torch, to_utf32(u8), dst_off=3)
    check_utf16_to_32(codec, torch, u16)
    check_utf16_to_32(codec, torch, u16, src_off=1, dst_off=3)


def test_utf16_utf32_errors_pairs_and_capacity(codec, torch):
    for profile in ("cyrillic", "cjk"):
        for rate in (1e-4, 1e-2):
            d = W.sweep_buffers(profile, rate, n_bytes=1 << 21, seed=W.SWEEP_SEEDS[(profile, rate)], cache=False)
            check_utf16_to_32(codec, torch, d["u16"])
            check_utf16_to_32(codec, torch, d["u16_cut_end"])
    pairs = np.tile(np.array([0xD83D, 0xDE00], np.uint16), 3 * 8192)
    for shift in range(3):  # every partition and region boundary cuts some pair for one shift
        check_utf16_to_32(codec, torch, np.concatenate([np.full(shift, 0x41, np.uint16), pairs]), dst_off=shift)
    _, base = W.profile_buffers("emoji", 0, 3 * 8192 + 5, 75, cache=False)
    for b in (256, 8192, 16384):
        for bad in ([0xD800], [0xDC00], [0xDBFF, 0x41]):
            check_utf16_to_32(codec, torch, np.concatenate([base[:b], np.array(bad, np.uint16), base[b:]]))
    total = oracle.utf32_length_from_utf16le(base)
    for cap in (0, 1, 3, 4, 5, 4095, total - 1):
        check_utf16_to_32(codec, torch, base, cap=cap, dst_off=cap % 4)
    u8, _ = W.profile_buffers("emoji", 1 << 16, 0, 76, cache=False)
    u32 = to_utf32(u8)
    for i in (0, 127, 128, 4095, u32.size - 1):
        for bad in (0x110000, 0xDABC):
            x = u32.copy()
            x[i] = bad
            check_utf32_to_16(codec, torch, x)
    total = oracle.utf16_length_from_utf32(u32)
    for cap in (0, 1, 7, 8, 9, 4095, total - 1):
        check_utf32_to_16(codec, torch, u32, cap=cap, dst_off=cap % 8)
