"""UTF-16BE through the C ABI against the reference codec's UTF-16BE functions (RFC 2781 byte
order), bit for bit: validation, the UTF-8 length, and both transcoding directions, on the
profiles, the invalid-input sweep, errors at tile and partition boundaries, surrogate pairs cut
by partitions, unaligned views and too-small outputs."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import CANARY16, CANARY8, as_torch_u16

pytestmark = pytest.mark.gpu


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


def check_be_input(codec, torch, be, src_off=0, dst_off=0, cap=None):
    """be: uint16 words as they lie in memory (big-endian bytes)."""
    from paper_2111_08692_gb300 import result_tuple
    be = np.ascontiguousarray(be, dtype=np.uint16)
    buf = torch.zeros(be.size + src_off + 64, dtype=torch.int16, device="cuda")
    src = buf[src_off:src_off + be.size]
    if be.size:
        src.copy_(as_torch_u16(torch, be).to("cuda"))
    assert result_tuple(codec.validate_utf16be(src)) == oracle.validate_utf16be(be)
    want_len = oracle.utf8_length_from_utf16be(be)
    assert int(codec.utf8_length_from_utf16be(src).item()) == want_len
    cap = want_len if cap is None else cap
    want, odst = oracle.convert_utf16be_to_utf8(be, cap)
    dbuf = torch.full((dst_off + cap + 48,), CANARY8, dtype=torch.uint8, device="cuda")
    got = result_tuple(codec.convert_utf16be_to_utf8(src, dbuf[dst_off:dst_off + cap], cap=cap))
    assert got == want, (got, want, be.size, src_off, dst_off, cap)
    host = dbuf.cpu().numpy()
    m = want[1] if want[0] == "OK" else (cap if want[0] == "OUTPUT_TOO_SMALL" else
                                          min(oracle.utf8_length_from_utf16be(be[:want[1]]), cap))
    assert np.array_equal(host[dst_off:dst_off + m], odst[:m])
    assert np.all(host[:dst_off] == CANARY8) and np.all(host[dst_off + cap:] == CANARY8)


def check_utf8_to_be(codec, torch, data, src_off=0, dst_off=0, cap=None):
    from paper_2111_08692_gb300 import result_tuple
    data = np.ascontiguousarray(data, dtype=np.uint8)
    buf = torch.zeros(data.size + src_off + 64, dtype=torch.uint8, device="cuda")
    src = buf[src_off:src_off + data.size]
    if data.size:
        src.copy_(torch.from_numpy(data).to("cuda"))
    cap = oracle.utf16_length_from_utf8(data) if cap is None else cap
    want, odst = oracle.convert_utf8_to_utf16be(data, cap)
    dbuf = torch.full((dst_off + cap + 40,), CANARY16, dtype=torch.int32, device="cuda").to(torch.int16)
    got = result_tuple(codec.convert_utf8_to_utf16be(src, dbuf[dst_off:dst_off + cap], cap=cap))
    assert got == want, (got, want, data.size, src_off, dst_off, cap)
    host = dbuf.cpu().numpy().view(np.uint16)
    m = want[1] if want[0] == "OK" else (cap if want[0] == "OUTPUT_TOO_SMALL" else
                                          min(oracle.utf16_length_from_utf8(data[:want[1]]), cap))
    assert np.array_equal(host[dst_off:dst_off + m], odst[:m])
    assert np.all(host[:dst_off] == CANARY16) and np.all(host[dst_off + cap:] == CANARY16)


@pytest.mark.parametrize("profile", W.PROFILE_ORDER + ("mixed",))
def test_profiles(codec, torch, profile):
    u8, u16 = W.profile_buffers(profile, 1 << 21, 1 << 20, 61, cache=False)
    be = u16.byteswap()
    check_be_input(codec, torch, be)
    check_be_input(codec, torch, be, src_off=1, dst_off=7)
    check_utf8_to_be(codec, torch, u8)
    check_utf8_to_be(codec, torch, u8, src_off=3, dst_off=5)


def test_sweep(codec, torch):
    for profile in ("cyrillic", "cjk"):
        for rate in (1e-6, 1e-4, 1e-2):
            d = W.sweep_buffers(profile, rate, n_bytes=1 << 22, seed=W.SWEEP_SEEDS[(profile, rate)], cache=False)
            check_be_input(codec, torch, d["u16"].byteswap())
            check_be_input(codec, torch, d["u16_cut_end"].byteswap())
            check_utf8_to_be(codec, torch, d["u8"])
            check_utf8_to_be(codec, torch, d["u8_cut_end"])


def test_boundaries_pairs_and_capacity(codec, torch):
    _, base = W.profile_buffers("emoji", 0, 5 * 8192, 62, cache=False)
    for b in (256, 2048, 8192, 16384):
        for d in range(-2, 3):
            for bad in ([0xD800], [0xDC00], [0xDBFF, 0x41]):
                data = np.concatenate([base[:b + d], np.array(bad, np.uint16), base[b + d:]])
                check_be_input(codec, torch, data.byteswap())
    pairs = np.tile(np.array([0xD83D, 0xDE00], np.uint16), 3 * 8192)
    for shift in range(3):
        check_be_input(codec, torch, np.concatenate([np.full(shift, 0x41, np.uint16), pairs]).byteswap(),
                       dst_off=shift)
    for n in (0, 1, 7, 8, 9, 255, 256, 257):
        check_be_input(codec, torch, base[:n].byteswap())
    u8, u16 = W.profile_buffers("mixed", 3 * 16384 + 5, 3 * 8192 + 3, 63, cache=False)
    total16 = oracle.utf16_length_from_utf8(u8)
    for cap in (0, 1, 15, 16, 17, 4095, total16 - 1):
        check_utf8_to_be(codec, torch, u8, cap=cap, dst_off=cap % 8)
    total8 = oracle.utf8_length_from_utf16le(u16)
    for cap in (0, 1, 15, 16, 17, 4095, total8 - 1):
        check_be_input(codec, torch, u16.byteswap(), cap=cap, dst_off=cap % 16)
