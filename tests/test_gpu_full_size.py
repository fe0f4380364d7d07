"""Parity at the full sizes: the five 1 GiB single buffers the benchmark times (UTF-8 and
UTF-16LE, one per profile) and the 256 MiB invalid-input sweep, in the launch configuration
the benchmark uses (one context, default geometry).  Every result, every output length and
every output unit the contract defines is compared with the reference codec, which handles a
1 GiB buffer in about a second.  The sweep runs with early exit on (the default) and off:
both must give the reference codec's result."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import as_torch_u16, check_utf16_input, check_utf8_input

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
    c = Codec(0, max_units=(1 << 30) + 4096)
    yield c
    c.close()


@pytest.mark.parametrize("profile", W.PROFILE_ORDER)
def test_single_buffer_full_size(codec, torch, profile):
    """One 1 GiB UTF-8 buffer and one 2^29-word UTF-16LE buffer of the profile: all six
    operations, whole outputs compared."""
    u8, u16 = W.single_buffer_1gib(profile)
    assert u8.size == 1 << 30 and u16.size == 1 << 29
    check_utf8_input(codec, torch, np.asarray(u8))
    torch.cuda.empty_cache()
    check_utf16_input(codec, torch, np.asarray(u16))
    torch.cuda.empty_cache()


def _results_without_early_exit(codec, torch, u8, u16):
    from paper_2111_08692_gb300 import result_tuple
    s8 = torch.from_numpy(u8).to("cuda")
    s16 = as_torch_u16(torch, u16).to("cuda")
    d16 = torch.empty(u8.size + 8, dtype=torch.int16, device="cuda")
    d8 = torch.empty(3 * u16.size + 8, dtype=torch.uint8, device="cuda")
    codec.set_early_exit(False)
    try:
        got = (result_tuple(codec.validate_utf8(s8)), result_tuple(codec.convert_utf8_to_utf16le(s8, d16)),
               result_tuple(codec.validate_utf16le(s16)), result_tuple(codec.convert_utf16le_to_utf8(s16, d8)))
    finally:
        codec.set_early_exit(True)
    return got


@pytest.mark.parametrize("profile", ("cyrillic", "cjk"))
def test_sweep_full_size(codec, torch, profile):
    """256 MiB buffers with errors injected at per-character rates 1e-6, 1e-4 and 1e-2, plus
    the siblings cut at the buffer end: the exact first error (kind, offset) and the output of
    the valid prefix, with early exit on; the results again with it off."""
    for rate in (1e-6, 1e-4, 1e-2):
        d = W.sweep_buffers(profile, rate)
        v8, c8 = check_utf8_input(codec, torch, d["u8"])
        v16, c16 = check_utf16_input(codec, torch, d["u16"])
        assert v8[0] != "OK" and v16[0] == "SURROGATE"
        assert _results_without_early_exit(codec, torch, d["u8"], d["u16"]) == (v8, c8, v16, c16)
        assert check_utf8_input(codec, torch, d["u8_cut_end"])[0][0] == "TOO_SHORT"
        assert check_utf16_input(codec, torch, d["u16_cut_end"])[0][0] == "SURROGATE"
        torch.cuda.empty_cache()
