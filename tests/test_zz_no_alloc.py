"""The allocation-free transcoder (gbu_convert_utf8_to_utf16le_noalloc) gives what the context
path (gbu_convert_utf8_to_utf16le) gives, call after call.

Its workspace is one static device array per device, left ready for the next launch by
each launch's last CTA; two calls in a row on each input check that hand-over.  The file
is named to be collected last, and passes alone too (the first call does the setup)."""
import numpy as np
import pytest

import workloads as W

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
    torch.cuda.set_device(0)
    c = Codec(0, max_units=1 << 28)
    yield c
    c.close()


def _inputs():
    """(name, UTF-8 bytes): valid text of every profile, an invalid byte late in a buffer of
    several partitions, an input cut inside a sequence, and the empty input."""
    out = []
    for i, p in enumerate(("ascii", "cyrillic", "cjk", "emoji", "mixed")):
        u8, _ = W.profile_buffers(p, (1 << 20) + 37 * i, 0, 300 + i, cache=False)
        out.append((p, u8))
    u8, _ = W.profile_buffers("mixed", 3 << 20, 0, 310, cache=False)
    bad = u8.copy()
    k = 3 * (1 << 20) - 70001
    while (bad[k] & 0xC0) == 0x80:
        k -= 1
    bad[k] = 0xFF
    out.append(("invalid", bad))
    cut = u8[: (2 << 20) + 1].copy()
    while cut.size and (cut[-1] & 0xC0) == 0x80:
        cut = cut[:-1]
    cut = cut[:-1] if cut.size and cut[-1] >= 0xC0 else cut
    out.append(("cut", np.concatenate([cut, np.array([0xE2, 0x82], np.uint8)])))
    out.append(("empty", np.zeros(0, np.uint8)))
    return out


@pytest.mark.parametrize("src_off,dst_off", [(0, 0), (5, 3)])
def test_noalloc_matches_context_path_twice(torch, codec, src_off, dst_off):
    from paper_2111_08692_gb300 import convert_utf8_to_utf16le_noalloc, result_tuple
    for name, data in _inputs():
        n = data.size
        sbuf = torch.zeros(n + src_off + 16, dtype=torch.uint8, device="cuda")
        if n:
            sbuf[src_off:src_off + n].copy_(torch.from_numpy(data).cuda())
        src = sbuf[src_off:src_off + n]
        cap = n + 8
        ref_buf = torch.full((cap + dst_off + 16,), 0x5A5A, dtype=torch.int16, device="cuda")
        ref = result_tuple(codec.convert_utf8_to_utf16le(src, ref_buf[dst_off:dst_off + cap]))
        ref_out = ref_buf.cpu()
        # buffers of the allocation-free calls are made before them (the calls allocate nothing)
        results = [torch.zeros(2, dtype=torch.int64, device="cuda") for _ in range(2)]
        bufs = [torch.full((cap + dst_off + 16,), 0x5A5A, dtype=torch.int16, device="cuda") for _ in range(2)]
        for call in range(2):
            convert_utf8_to_utf16le_noalloc(src, bufs[call][dst_off:dst_off + cap], results[call])
        torch.cuda.synchronize()
        for call in range(2):
            got = result_tuple(results[call])
            assert got == ref, (name, call, got, ref)
            assert torch.equal(bufs[call].cpu(), ref_out), (name, call)


def test_noalloc_rejects_inputs_above_its_limit(torch):
    from paper_2111_08692_gb300 import (NOALLOC_MAX_UNITS, STATUS_CODE, GbuError,
                                        convert_utf8_to_utf16le_noalloc, gbu_convert_utf8_to_utf16le_noalloc)
    # the size check comes first: nothing is read or enqueued
    rc = gbu_convert_utf8_to_utf16le_noalloc(0, NOALLOC_MAX_UNITS + 1, 0, 0, 0, 0)
    assert rc == STATUS_CODE["NOALLOC_TOO_LARGE"]

    class _Big:  # a stand-in with the size of an oversized input; never dereferenced
        def numel(self):
            return NOALLOC_MAX_UNITS + 1

    with pytest.raises(GbuError, match="limit"):
        convert_utf8_to_utf16le_noalloc(_Big(), None, None)
