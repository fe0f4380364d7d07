"""The allocation-free transcoder (gbu_convert_utf8_to_utf16le_noalloc) gives what the context
path (gbu_convert_utf8_to_utf16le) and the oracle give, call after call, and allocates nothing.

Some callers cannot create a context, because creating one calls cudaMalloc: a latency-bound
serving loop where that call would synchronise the device, or a process whose device memory
is owned by another allocator.  This form keeps its workspace in a static device array instead.
That array is left ready for the next launch by each launch's last CTA; two calls in a row on
each input check that hand-over.  The file is named to be collected last, and passes alone too
(the first call does the setup)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CANARY = 0x5A5A


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
    several partitions, an input cut inside a sequence, an invalid byte near the start of a
    48 MiB buffer (where early exit skips most partitions), and the empty input."""
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
    big, _ = W.profile_buffers("cjk", 48 << 20, 0, 311, cache=False)
    big = big.copy()
    k = 200003
    while (big[k] & 0xC0) == 0x80:
        k -= 1
    big[k] = 0xC0  # an overlong two-byte lead
    out.append(("invalid_early_48mib", big))
    out.append(("empty", np.zeros(0, np.uint8)))
    return out


def _compared_prefix(data: np.ndarray, want, cap: int) -> int:
    """How many leading output words are defined for this input and capacity: all of them on
    success, cap when the output does not fit, else the conversion of the valid prefix."""
    kind, count = want
    if kind == "OK":
        return count
    if kind == "OUTPUT_TOO_SMALL":
        return cap
    return min(oracle.utf16_length_from_utf8(data[:count]), cap)


@pytest.mark.parametrize("src_off,dst_off", [(0, 0), (5, 3)])
def test_noalloc_matches_oracle_and_context_path_twice(torch, codec, src_off, dst_off):
    from paper_2111_08692_gb300 import convert_utf8_to_utf16le_noalloc, result_tuple
    for name, data in _inputs():
        n = data.size
        sbuf = torch.zeros(n + src_off + 16, dtype=torch.uint8, device="cuda")
        if n:
            sbuf[src_off:src_off + n].copy_(torch.from_numpy(data).cuda())
        src = sbuf[src_off:src_off + n]
        cap = n + 8
        want, odst = oracle.convert_utf8_to_utf16le(data, cap)
        m = _compared_prefix(data, want, cap)
        ref_buf = torch.full((cap + dst_off + 16,), CANARY, dtype=torch.int16, device="cuda")
        ref = result_tuple(codec.convert_utf8_to_utf16le(src, ref_buf[dst_off:dst_off + cap]))
        assert ref == want, (name, "context path", ref, want)
        ref_out = ref_buf.cpu().numpy().view(np.uint16)
        # buffers of the allocation-free calls are made before them (the calls allocate nothing)
        results = [torch.zeros(2, dtype=torch.int64, device="cuda") for _ in range(2)]
        bufs = [torch.full((cap + dst_off + 16,), CANARY, dtype=torch.int16, device="cuda") for _ in range(2)]
        for call in range(2):
            convert_utf8_to_utf16le_noalloc(src, bufs[call][dst_off:dst_off + cap], results[call])
        torch.cuda.synchronize()
        for call in range(2):
            got = result_tuple(results[call])
            assert got == want, (name, call, got, want)
            host = bufs[call].cpu().numpy().view(np.uint16)
            out = host[dst_off:dst_off + cap]
            assert np.array_equal(out[:m], odst[:m]), (name, call, "differs from the oracle")
            assert np.array_equal(out[:m], ref_out[dst_off:dst_off + m]), (name, call, "differs from the context path")
            assert np.all(host[:dst_off] == CANARY), (name, call, "write before dst")
            assert np.all(host[dst_off + cap:] == CANARY), (name, call, "write at or past cap")


def test_noalloc_calls_allocate_no_device_memory(torch, codec):
    """After the first call on the device (which does the setup), further calls change neither
    the device's free memory nor torch's allocated bytes."""
    from paper_2111_08692_gb300 import convert_utf8_to_utf16le_noalloc, result_tuple
    data, _ = W.profile_buffers("mixed", 5 << 20, 0, 312, cache=False)
    src = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    dst = torch.empty(data.size, dtype=torch.int16, device="cuda")
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    convert_utf8_to_utf16le_noalloc(src, dst, res)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        convert_utf8_to_utf16le_noalloc(src, dst, res)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert result_tuple(res) == oracle.validate_utf8(data)[:1] + (oracle.utf16_length_from_utf8(data),)


_CAPTURE_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2111_08692_gb300 import STATUS_CODE, gbu_convert_utf8_to_utf16le_noalloc, result_tuple
torch.cuda.set_device(0)
data = np.frombuffer("café 中文 \U0001F600 ok".encode() * 1000, dtype=np.uint8)
src = torch.from_numpy(data.copy()).cuda()
dst = torch.zeros(data.size, dtype=torch.int16, device="cuda")
res = torch.zeros(2, dtype=torch.int64, device="cuda")
s = torch.cuda.Stream()
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s):
    rc = gbu_convert_utf8_to_utf16le_noalloc(src.data_ptr(), data.size, dst.data_ptr(), data.size,
                                             res.data_ptr(), s.cuda_stream)
assert rc == STATUS_CODE["CUDA_ERROR"], rc
rc = gbu_convert_utf8_to_utf16le_noalloc(src.data_ptr(), data.size, dst.data_ptr(), data.size,
                                         res.data_ptr(), torch.cuda.current_stream().cuda_stream)
assert rc == 0, rc
torch.cuda.synchronize()
want, odst = oracle.convert_utf8_to_utf16le(data, data.size)
assert result_tuple(res) == want, (result_tuple(res), want)
assert np.array_equal(dst.cpu().numpy().view(np.uint16)[:want[1]], odst[:want[1]])
print("capture refusal ok")
"""


def test_noalloc_setup_is_refused_during_capture_then_runs(torch):
    """In a fresh process, a first call made while its stream is being captured returns
    GBU_CUDA_ERROR without doing the setup; the next call, outside the capture, does the setup
    and transcodes correctly."""
    r = subprocess.run([sys.executable, "-c", _CAPTURE_SCRIPT, ROOT], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "capture refusal ok" in r.stdout


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
