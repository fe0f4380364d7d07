"""The sharded form on one GPU: one buffer split by the device cut kernel, each shard handled by
the single-buffer calls on its own stream and context (P streams standing in for P GPUs), the
output lengths exchanged (an exclusive scan gives each shard its output offset), and the
results combined by gbu_combine_shards.  Everything must equal the single call on the whole
buffer and the reference codec: results, lengths and every output unit of the valid prefix."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import as_torch_u16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def codecs(torch):
    from paper_2111_08692_gb300 import Codec
    from paper_2111_08692_gb300.build import build
    build()
    cs = [Codec(0, max_units=1 << 24) for _ in range(16)]
    yield cs
    for c in cs:
        c.close()


def run_sharded(torch, codecs, src, P, utf16):
    """Validation, length and transcoding of device buffer src in P shards on P streams."""
    import paper_2111_08692_gb300 as g
    from paper_2111_08692_gb300 import result_tuple
    cuts_d = codecs[0].shard_cuts(src, P)
    cuts = cuts_d.cpu().numpy().astype(np.uint64)
    streams = [torch.cuda.Stream() for _ in range(P)]
    torch.cuda.synchronize()
    shards = [src[int(cuts[k]):int(cuts[k + 1])] for k in range(P)]
    vres, lens = [], []
    for k in range(P):
        with torch.cuda.stream(streams[k]):
            c = codecs[k]
            vres.append(c.validate_utf16le(shards[k], stream=streams[k]) if utf16
                        else c.validate_utf8(shards[k], stream=streams[k]))
            lens.append(c.utf8_length_from_utf16le(shards[k], stream=streams[k]) if utf16
                        else c.utf16_length_from_utf8(shards[k], stream=streams[k]))
    torch.cuda.synchronize()
    n_out = [int(x.item()) for x in lens]
    off = np.concatenate([[0], np.cumsum(n_out)]).astype(np.int64)  # the exchange: output offsets
    dst = torch.empty(int(off[-1]) + 8, dtype=torch.uint8 if utf16 else torch.int16, device="cuda")
    cres = []
    for k in range(P):
        with torch.cuda.stream(streams[k]):
            d = dst[int(off[k]):int(off[k + 1])]
            c = codecs[k]
            cres.append(c.convert_utf16le_to_utf8(shards[k], d, stream=streams[k]) if utf16
                        else c.convert_utf8_to_utf16le(shards[k], d, stream=streams[k]))
    torch.cuda.synchronize()
    v = g.combine_shards(cuts, [result_tuple(r) for r in vres])
    cv = g.combine_shards(cuts, [result_tuple(r) for r in cres])
    return cuts, v, cv, int(off[-1]), dst[:int(off[-1])]


@pytest.mark.parametrize("P", [1, 2, 5, 16])
def test_sharded_matches_single_call_and_oracle(torch, codecs, P):
    from paper_2111_08692_gb300 import shard_cuts_host
    inputs = []
    for prof in ("mixed", "cjk", "emoji"):
        u8, u16 = W.profile_buffers(prof, 3 << 20, 3 << 19, 81, cache=False)
        inputs.append((u8, u16))
    for rate in (1e-6, 1e-4, 1e-2):
        d = W.sweep_buffers("cyrillic", rate, n_bytes=1 << 22, seed=W.SWEEP_SEEDS[("cyrillic", rate)], cache=False)
        inputs.append((d["u8"], d["u16"]))
    for u8, u16 in inputs:
        for data, utf16 in ((u8, False), (u16, True)):
            src = as_torch_u16(torch, data).to("cuda") if utf16 else torch.from_numpy(data).to("cuda")
            cuts, v, cv, total, out = run_sharded(torch, codecs, src, P, utf16)
            assert np.array_equal(cuts, shard_cuts_host(data, P))  # device and host cuts agree
            if utf16:
                wv, (wc, wout), wlen = (oracle.validate_utf16le(data), oracle.convert_utf16le_to_utf8(data),
                                        oracle.utf8_length_from_utf16le(data))
            else:
                wv, (wc, wout), wlen = (oracle.validate_utf8(data), oracle.convert_utf8_to_utf16le(data),
                                        oracle.utf16_length_from_utf8(data))
            assert v == wv and cv == wc and total == wlen, (P, utf16, v, wv, cv, wc)
            if wc[0] == "OK":
                m = wc[1]
            elif utf16:
                m = oracle.utf8_length_from_utf16le(data[:wc[1]])
            else:
                m = oracle.utf16_length_from_utf8(data[:wc[1]])
            host = out.cpu().numpy()
            host = host.view(np.uint16) if not utf16 else host
            assert np.array_equal(host[:m], wout[:m])
