"""Bit-exact parity of the batched calls with the reference codec, string by string.

Each string of a batch must get exactly what the reference codec gives for it alone: result
kind and offset, output length, and every output unit the contract defines.  Inputs come
from the seeded CSR generator in workloads/ (log-normal lengths, the five profiles, injected
errors); expected values come from oracle/ only.  Launch geometries cover the warp-per-string
path, the whole-CTA path for long strings, and claims of one string to the maximum.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

GEOMETRIES = [  # (warps per CTA, strings per claim, long-string threshold in bytes)
    (8, 64, 4096),
    (4, 8, 512),
    (16, 1, 512),
    (16, 1024, 1 << 30),
    (8, 32, 2048),
]


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
    c = Codec(0, max_units=1 << 28)
    yield c
    c.close()


def _dev(torch, a, dtype=None):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    t = torch.from_numpy(a.copy()) if a.size else torch.zeros(0, dtype=dtype or torch.uint8)
    return t.to("cuda")


def _gpu_results(t):
    """[(status name, count)] of a (B, 2) int64 results tensor."""
    from paper_2111_08692_gb300 import STATUS
    a = t.cpu().numpy().view(np.uint64)
    st = (a[:, 0] & 0xFFFFFFFF).astype(np.int64)
    return [(STATUS.get(int(s), int(s)), int(c)) for s, c in zip(st, a[:, 1])]


def _oracle_lengths(fn, src, off):
    return np.array([fn(src[int(off[i]):int(off[i + 1])]) for i in range(off.size - 1)], dtype=np.uint64)


def _defined_mask(dst_off, want, src, off, prefix_len):
    """Output units the contract defines, per string: all `count` units when OK, `cap` when
    the output is too small, else the conversion of the valid prefix (clipped to cap)."""
    mask = np.zeros(int(dst_off[-1]), dtype=bool)
    for i, (kind, count) in enumerate(want):
        d0, d1 = int(dst_off[i]), int(dst_off[i + 1])
        cap = d1 - d0
        if kind == "OK":
            m = count
        elif kind == "OUTPUT_TOO_SMALL":
            m = cap
        else:
            m = min(prefix_len(src[int(off[i]):int(off[i]) + count]), cap)
        mask[d0:d0 + m] = True
    return mask


def _batch(B, seed, median=64, max_len=65536, err=0.05):
    return W.batched_strings(B, seed, median=median, max_len=max_len, error_fraction=err, cache=False)


def _check_all(torch, codec, b, geometry=None, tight_seed=None):
    """Every batched operation on batch b against the oracle."""
    u8, off8, u16, off16 = b["u8"], b["off8"], b["u16"], b["off16"]
    if geometry is not None:
        for op in ("validate_utf8", "utf16_length_from_utf8", "convert_utf8_to_utf16le", "validate_utf16le",
                   "utf8_length_from_utf16le", "convert_utf16le_to_utf8"):
            codec.set_batch_config(op, *geometry)
    s8, o8, s16, o16 = _dev(torch, u8), _dev(torch, off8), _dev(torch, u16, torch.int16), _dev(torch, off16)

    # validation
    got = _gpu_results(codec.validate_utf8_batched(s8, o8))
    want = oracle.validate_utf8_batched(u8, off8)
    assert got == want, _first_diff(got, want)
    got = _gpu_results(codec.validate_utf16le_batched(s16, o16))
    want = oracle.validate_utf16le_batched(u16, off16)
    assert got == want, _first_diff(got, want)

    # lengths
    len16 = _oracle_lengths(oracle.utf16_length_from_utf8, u8, off8)
    got = codec.utf16_length_from_utf8_batched(s8, o8).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, len16), _first_diff(list(got), list(len16))
    len8 = _oracle_lengths(oracle.utf8_length_from_utf16le, u16, off16)
    got = codec.utf8_length_from_utf16le_batched(s16, o16).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, len8), _first_diff(list(got), list(len8))

    # transcoding, into exact (or, with tight_seed, partly too small) output slots
    for direction, lens, src, off, s_dev, o_dev, unit in (
            ("8to16", len16, u8, off8, s8, o8, np.uint16), ("16to8", len8, u16, off16, s16, o16, np.uint8)):
        caps = lens.astype(np.int64)
        if tight_seed is not None:
            rng = np.random.default_rng(tight_seed)
            cut = rng.random(caps.size) < 0.2
            caps = np.where(cut, np.maximum(caps - rng.integers(1, 40, caps.size), 0), caps)
        dst_off = np.zeros(caps.size + 1, dtype=np.uint64)
        np.cumsum(caps, out=dst_off[1:].view(np.int64))
        canary = 0x5A5A if unit == np.uint16 else 0x5A
        dst = torch.full((int(dst_off[-1]) + 64,), canary, dtype=torch.int16 if unit == np.uint16 else torch.uint8,
                         device="cuda")
        d_off = _dev(torch, dst_off)
        if direction == "8to16":
            res = codec.convert_utf8_to_utf16le_batched(s_dev, o_dev, dst, d_off)
            want, odst = oracle.convert_utf8_to_utf16le_batched(src, off, dst_off)
            plen = oracle.utf16_length_from_utf8
        else:
            res = codec.convert_utf16le_to_utf8_batched(s_dev, o_dev, dst, d_off)
            want, odst = oracle.convert_utf16le_to_utf8_batched(src, off, dst_off)
            plen = oracle.utf8_length_from_utf16le
        got = _gpu_results(res)
        assert got == want, (direction, _first_diff(got, want))
        host = dst.cpu().numpy()
        host = host.view(np.uint16) if unit == np.uint16 else host
        mask = _defined_mask(dst_off, want, src, off, plen)
        bad = np.flatnonzero(mask & (host[:mask.size] != odst))
        assert bad.size == 0, (direction, "output differs at", bad[:10])
        assert np.all(host[mask.size:] == canary), (direction, "write past the last slot")


def _first_diff(got, want):
    for i, (g, w) in enumerate(zip(got, want)):
        if g != w:
            return f"string {i}: got {g}, want {w}"
    return f"lengths {len(got)} vs {len(want)}"


@pytest.mark.parametrize("geometry", GEOMETRIES)
def test_batched_matches_oracle(torch, codec, geometry):
    _check_all(torch, codec, _batch(3000, 11), geometry)


def test_batched_long_strings_and_tight_outputs(torch, codec):
    # median 2 KiB: most strings take several regions and many the whole-CTA path
    b = _batch(400, 12, median=2048, max_len=65536, err=0.1)
    for geometry in ((8, 16, 4096), (4, 4, 512), (16, 64, 8192)):
        _check_all(torch, codec, b, geometry, tight_seed=5)


def test_batched_edge_cases(torch, codec):
    from paper_2111_08692_gb300 import STATUS_CODE, gbu_validate_utf8_batched
    codec.set_batch_config("validate_utf8", 8, 64, 4096)
    # B == 0: nothing enqueued, nothing written
    res = torch.full((1, 2), -1, dtype=torch.int64, device="cuda")
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    src = torch.zeros(16, dtype=torch.uint8, device="cuda")
    codec.validate_utf8_batched(src, off, res)
    assert res.cpu().tolist() == [[-1, -1]]
    # NULL arrays with B > 0 are refused
    assert gbu_validate_utf8_batched(codec.ctx, 0, 0, 5, 0, 0) == STATUS_CODE["BAD_ARGUMENT"]
    # empty strings among others, strings ending in cut sequences, region-sized strings
    rng = np.random.default_rng(3)
    parts = []
    for k in range(300):
        r = k % 6
        if r == 0:
            parts.append(np.zeros(0, np.uint8))
        elif r == 1:
            parts.append(np.frombuffer("é漢🎉".encode()[: int(rng.integers(1, 9))], np.uint8))
        elif r == 2:
            parts.append(W.encode_utf8(W.draw_codepoints("mixed", 600, rng))[:512])
        elif r == 3:
            parts.append(W.encode_utf8(W.draw_codepoints("cjk", 3000, rng))[:4096 + int(rng.integers(-3, 4))])
        elif r == 4:
            parts.append(np.array([0xF4, 0x90, 0x80, 0x80, 0x41], np.uint8))
        else:
            parts.append(np.array([0xED, 0xA0, 0x80], np.uint8))
    off8 = np.zeros(len(parts) + 1, dtype=np.uint64)
    np.cumsum([p.size for p in parts], out=off8[1:].view(np.int64))
    u8 = np.concatenate(parts)
    text = [bytes(p).decode("utf-8", "replace") for p in parts]
    u16 = np.frombuffer("".join(text).encode("utf-16-le"), np.uint16)
    off16 = np.zeros(len(parts) + 1, dtype=np.uint64)
    np.cumsum([len(t.encode("utf-16-le")) // 2 for t in text], out=off16[1:].view(np.int64))
    b = {"u8": u8, "off8": off8, "u16": u16, "off16": off16}
    for geometry in ((8, 64, 4096), (4, 3, 512), (16, 1024, 1 << 20)):
        _check_all(torch, codec, b, geometry, tight_seed=9)


@pytest.mark.parametrize("count", [0, 1, 4095, 4096, 4097, 123457])
def test_exclusive_scan_matches_prefix_sums(torch, codec, count):
    from paper_2111_08692_gb300 import result_tuple
    rng = np.random.default_rng(count)
    vals = rng.integers(0, 1 << 20, size=count, dtype=np.int64)
    out, res = codec.exclusive_scan_u64(_dev(torch, vals, torch.int64))
    want = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(vals, out=want[1:])
    assert np.array_equal(out.cpu().numpy(), want)
    assert result_tuple(res) == ("OK", int(want[-1]))


def test_exclusive_scan_refuses_totals_beyond_44_bits(torch, codec):
    from paper_2111_08692_gb300 import result_tuple
    vals = np.full(8, 1 << 42, dtype=np.int64)
    _, res = codec.exclusive_scan_u64(_dev(torch, vals, torch.int64))
    assert result_tuple(res) == ("BAD_ARGUMENT", 8 << 42)
    # the workspace is fine afterwards
    out, res = codec.exclusive_scan_u64(_dev(torch, np.arange(10, dtype=np.int64), torch.int64))
    assert result_tuple(res) == ("OK", 45)


def test_batched_scan_then_convert_in_a_cuda_graph(torch, codec):
    """lengths -> scan -> convert, captured once and replayed: the replays give the oracle's
    results, and the graph holds exactly three library kernels."""
    b = _batch(5000, 13)
    u8, off8 = b["u8"], b["off8"]
    codec.set_batch_config("utf16_length_from_utf8", 8, 64, 4096)
    codec.set_batch_config("convert_utf8_to_utf16le", 8, 64, 4096)
    s8, o8 = _dev(torch, u8), _dev(torch, off8)
    B = off8.size - 1
    lens = torch.empty(B, dtype=torch.int64, device="cuda")
    d_off = torch.empty(B + 1, dtype=torch.int64, device="cuda")
    scan_res = codec.new_result()
    dst = torch.zeros(u8.size + 64, dtype=torch.int16, device="cuda")
    res = codec.new_results(B)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()

    def body():
        codec.utf16_length_from_utf8_batched(s8, o8, lens, stream=stream)
        codec.exclusive_scan_u64(lens, d_off, scan_res, stream=stream)
        codec.convert_utf8_to_utf16le_batched(s8, o8, dst, d_off, res, stream=stream)

    graph = codec.capture(body, stream)
    assert graph.kernels() == 3
    want, odst = None, None
    len16 = _oracle_lengths(oracle.utf16_length_from_utf8, u8, off8)
    want_off = np.zeros(B + 1, dtype=np.uint64)
    np.cumsum(len16, out=want_off[1:])
    want, odst = oracle.convert_utf8_to_utf16le_batched(u8, off8, want_off)
    mask = _defined_mask(want_off, want, u8, off8, oracle.utf16_length_from_utf8)
    for _ in range(2):
        dst.zero_()
        res.fill_(-1)
        graph.launch(stream)
        stream.synchronize()
        assert np.array_equal(d_off.cpu().numpy().view(np.uint64), want_off)
        assert _gpu_results(res) == want
        host = dst.cpu().numpy().view(np.uint16)[:mask.size]
        assert np.array_equal(host[mask], odst[mask])
    graph.close()


def test_autotuner_picks_a_valid_geometry_and_leaves_valid_outputs(torch, codec):
    b = _batch(20000, 14)
    u8, off8 = b["u8"], b["off8"]
    s8, o8 = _dev(torch, u8), _dev(torch, off8)
    res = codec.new_results(off8.size - 1)
    cfg = codec.tune_batched("validate_utf8", s8, o8, res, reps=1)
    assert cfg["warps_per_cta"] in (4, 8, 16)
    assert 1 <= cfg["strings_per_claim"] <= 1024 and cfg["long_bytes"] >= 512
    assert cfg["tuned_ms"] > 0
    assert codec.batch_config("validate_utf8") == cfg
    assert _gpu_results(res) == oracle.validate_utf8_batched(u8, off8)


def test_batched_full_size_one_million_strings(torch, codec):
    """The full batched workload (1,000,000 strings, median 64 B, sigma 1.5, 1% with an
    error): every string's validation result and UTF-16 length, both directions of
    transcoding into exact slots, against the oracle."""
    b = W.batched_strings(1_000_000, 1000)
    _check_all(torch, codec, b, (8, 64, 4096))


def test_per_string_loop_matches_the_oracle_string_by_string(torch, codec):
    """gbu_per_string_loop (one single-buffer call per string, issued from the library's C loop,
    host offsets): every operation, each string's result and defined output units against the
    oracle, and the destination's canary after the last slot."""
    from paper_2111_08692_gb300 import lib
    L = lib()
    b = _batch(400, 77, err=0.1)
    u8, off8, u16, off16 = b["u8"], b["off8"], b["u16"], b["off16"]
    off8, off16 = np.ascontiguousarray(off8, np.uint64), np.ascontiguousarray(off16, np.uint64)
    B = off8.size - 1
    s8, s16 = _dev(torch, u8), _dev(torch, u16, torch.int16)
    stream = torch.cuda.current_stream().cuda_stream
    res = torch.zeros((B, 2), dtype=torch.int64, device="cuda")
    for op, fn, src, s_dev, off in ((0, oracle.validate_utf8, u8, s8, off8), (3, oracle.validate_utf16le, u16, s16, off16)):
        assert L.gbu_per_string_loop(codec.ctx, op, s_dev.data_ptr(), off.ctypes.data, B, None, None,
                                     res.data_ptr(), stream) == 0
        want = [fn(src[int(off[i]):int(off[i + 1])]) for i in range(B)]
        assert _gpu_results(res) == want
    for op, fn, src, s_dev, off in ((1, oracle.utf16_length_from_utf8, u8, s8, off8),
                                    (4, oracle.utf8_length_from_utf16le, u16, s16, off16)):
        assert L.gbu_per_string_loop(codec.ctx, op, s_dev.data_ptr(), off.ctypes.data, B, None, None,
                                     res.data_ptr(), stream) == 0
        got = res.cpu().numpy().view(np.uint64).reshape(-1)[:B]  # lengths: a packed uint64 array
        assert np.array_equal(got, _oracle_lengths(fn, src, off))
    for op, conv, plen, lenf, src, s_dev, off, unit in (
            (2, oracle.convert_utf8_to_utf16le_batched, oracle.utf16_length_from_utf8, oracle.utf16_length_from_utf8,
             u8, s8, off8, np.uint16),
            (5, oracle.convert_utf16le_to_utf8_batched, oracle.utf8_length_from_utf16le, oracle.utf8_length_from_utf16le,
             u16, s16, off16, np.uint8)):
        caps = _oracle_lengths(lenf, src, off).astype(np.int64)
        dst_off = np.zeros(B + 1, dtype=np.uint64)
        np.cumsum(caps, out=dst_off[1:].view(np.int64))
        canary = 0x5A5A if unit == np.uint16 else 0x5A
        dst = torch.full((int(dst_off[-1]) + 64,), canary, dtype=torch.int16 if unit == np.uint16 else torch.uint8,
                         device="cuda")
        assert L.gbu_per_string_loop(codec.ctx, op, s_dev.data_ptr(), off.ctypes.data, B, dst.data_ptr(),
                                     dst_off.ctypes.data, res.data_ptr(), stream) == 0
        want, odst = conv(src, off, dst_off)
        assert _gpu_results(res) == want
        host = dst.cpu().numpy()
        if unit == np.uint16:
            host = host.view(np.uint16)
        mask = _defined_mask(dst_off, want, src, off, plen)
        assert np.array_equal(host[:int(dst_off[-1])][mask], odst[mask])
        assert np.all(host[int(dst_off[-1]):] == canary)
