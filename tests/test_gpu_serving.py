"""The serving loop: every request's result is the same alone and in the mix, and equals the
reference codec's; admission follows the memory budget; cancellation and over-budget
requests are refused on the host.  Requests are slices of seeded per-profile pools
(workloads.serving_pools / serving_trace), some from copies with injected errors."""
import time

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

OPS = W.SERVING_OPS


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def lib(torch):
    from paper_2111_08692_gb300.build import build
    build()
    import paper_2111_08692_gb300 as P
    return P


@pytest.fixture(scope="module")
def pools(torch):
    host = W.serving_pools(1 << 20, seed=2100)
    dev = {}
    for prof, p in host.items():
        dev[prof] = {k: torch.from_numpy(p[k].view(np.int16) if p[k].dtype == np.uint16 else p[k]).cuda()
                     for k in ("u8", "u16", "bad8", "bad16")}
    return host, dev


def _request_tensor(dev, trace, i):
    prof = W.PROFILE_ORDER[trace["profile"][i]]
    op = OPS[trace["op"][i]]
    utf16 = op in ("validate_utf16le", "convert_utf16le_to_utf8")
    key = ("bad" if trace["bad"][i] else "u") + ("16" if utf16 else "8")
    s, n = int(trace["start"][i]), int(trace["n"][i])
    return dev[prof][key][s:s + n]


def _request_host(host, trace, i):
    prof = W.PROFILE_ORDER[trace["profile"][i]]
    op = OPS[trace["op"][i]]
    utf16 = op in ("validate_utf16le", "convert_utf16le_to_utf8")
    key = ("bad" if trace["bad"][i] else "u") + ("16" if utf16 else "8")
    s, n = int(trace["start"][i]), int(trace["n"][i])
    return host[prof][key][s:s + n]


def _collect(srv, ids, timeout=60.0):
    """Waits for the completions of `ids`; returns id -> (status, count, output or None)."""
    want = set(ids)
    got = {}
    t_end = time.time() + timeout
    while want - set(got) and time.time() < t_end:
        for c in srv.poll():
            got[c["id"]] = c
        if want - set(got):
            time.sleep(0.0005)
    assert not (want - set(got)), f"{len(want - set(got))} requests did not complete"
    return got


def _output(srv, c, op):
    """The defined part of a completion's output (copied to the host), then release."""
    if c["dst"] is None:
        return None
    dtype = np.uint16 if op == "convert_utf8_to_utf16le" else np.uint8
    units = c["count"] if c["status"] == "OK" else 0
    out = srv.copy_output(c["id"], units, dtype)
    srv.release(c["id"])
    return out


def _expected(data, op):
    if op == "validate_utf8":
        return oracle.validate_utf8(data), None
    if op == "validate_utf16le":
        return oracle.validate_utf16le(data), None
    if op == "convert_utf8_to_utf16le":
        r, d = oracle.convert_utf8_to_utf16le(data, data.size)
    else:
        r, d = oracle.convert_utf16le_to_utf8(data, 3 * data.size)
    return r, (d[:r[1]] if r[0] == "OK" else np.zeros(0, d.dtype))


@pytest.mark.parametrize("device_rings", [0, 1])
def test_results_are_the_same_alone_and_in_the_mix(torch, lib, pools, device_rings):
    """Descriptors and results in mapped host memory (0) or in device memory with copies (1)."""
    host, dev = pools
    trace = W.serving_trace(600, 2e5, host, seed=3100, max_bytes=512 << 10, p_bad=0.15)
    srv = lib.Server(0, budget_bytes=256 << 20, device_rings=device_rings)
    try:
        t0 = srv.now_ns() + 2_000_000
        reqs = [(OPS[trace["op"][i]], _request_tensor(dev, trace, i), t0 + int(trace["arrival_ns"][i]), i)
                for i in range(len(trace["op"]))]
        first = srv.submit(reqs)
        ids = list(range(first, first + len(reqs)))
        mix = _collect(srv, ids)
        mixed = {}
        for k, rid in enumerate(ids):
            c = mix[rid]
            assert c["tag"] == k
            mixed[k] = (c["status"], c["count"], _output(srv, c, reqs[k][0]))
        # the same requests one at a time
        for k, (op, src, _, _) in enumerate(reqs):
            rid = srv.submit([(op, src, 0, k)])
            c = _collect(srv, [rid])[rid]
            alone = (c["status"], c["count"], _output(srv, c, op))
            m = mixed[k]
            assert alone[:2] == m[:2], (k, op, alone[:2], m[:2])
            assert (alone[2] is None) == (m[2] is None) and (alone[2] is None or np.array_equal(alone[2], m[2])), k
            want, wdst = _expected(_request_host(host, trace, k), op)
            assert alone[:2] == want, (k, op, alone[:2], want)
            if wdst is not None:
                assert np.array_equal(alone[2], wdst), k
        st = srv.stats()
        assert st["completed"] == 2 * len(reqs) and st["inflight"] == 0 and st["budget_used_bytes"] == 0
        assert st["groups"] < st["completed"]  # requests shared launches
    finally:
        srv.close()


def test_admission_waits_for_budget_and_releases(torch, lib, pools):
    _, dev = pools
    src = dev["ascii"]["u8"][:200_000]
    # each request holds 200,000 input bytes while it runs and 400,128 output bytes until it
    # is released: with a 1 MiB budget two complete, then a third needs a release
    srv = lib.Server(0, budget_bytes=1 << 20)
    try:
        first = srv.submit([("convert_utf8_to_utf16le", src, 0, k) for k in range(4)])
        got = {}
        t_end = time.time() + 5
        while len(got) < 2 and time.time() < t_end:
            for c in srv.poll():
                got[c["id"]] = c
        time.sleep(0.2)
        for c in srv.poll():
            got[c["id"]] = c
        assert sorted(got) == [first, first + 1]
        st = srv.stats()
        assert st["pending"] == 2 and st["budget_used_bytes"] == 2 * 400_128
        srv.release(first)
        c3 = _collect(srv, [first + 2])[first + 2]
        assert c3["status"] == "OK" and c3["count"] == 200_000
        assert c3["admit_ns"] >= max(c["complete_ns"] for c in got.values())
        srv.release(first + 1)
        srv.release(first + 2)
        c4 = _collect(srv, [first + 3])[first + 3]
        assert c4["status"] == "OK"
        srv.release(first + 3)
        assert srv.stats()["budget_used_bytes"] == 0
    finally:
        srv.close()


def test_cancel_and_refusals(torch, lib, pools):
    _, dev = pools
    src = dev["ascii"]["u8"][:1000]  # whole characters
    srv = lib.Server(0, budget_bytes=1 << 20)
    try:
        rid = srv.submit([("validate_utf8", src, srv.now_ns() + 10_000_000_000, 7)])
        assert srv.cancel(rid)
        assert not srv.cancel(rid)
        c = _collect(srv, [rid])[rid]
        assert c["status"] == "CANCELLED" and c["tag"] == 7
        # a request that can never fit the budget, an unknown op code, a NULL source
        big = dev["ascii"]["u8"][:400_000]  # 400,000 in + 800,000 out > 1 MiB
        with pytest.raises(lib.GbuError, match="OVER_BUDGET"):
            srv.submit([("convert_utf8_to_utf16le", big, 0, 0)])
        from paper_2111_08692_gb300 import GbuRequest
        bad = (GbuRequest * 1)(GbuRequest(9, 0, src.data_ptr(), 10, 0, 0))
        with pytest.raises(lib.GbuError, match="BAD_ARGUMENT"):
            srv.submit_raw(bad, 1)
        bad = (GbuRequest * 1)(GbuRequest(0, 0, 0, 10, 0, 0))
        with pytest.raises(lib.GbuError, match="BAD_ARGUMENT"):
            srv.submit_raw(bad, 1)
        # still serving afterwards
        rid = srv.submit([("validate_utf8", src, 0, 1)])
        assert _collect(srv, [rid])[rid]["status"] == "OK"
    finally:
        srv.close()


@pytest.mark.parametrize("device_rings", [0, 1])
def test_large_transcodings_share_partitioned_launches(torch, lib, pools, device_rings):
    """Requests of 70 KiB to 1 MiB in both directions (clean and with injected errors) are
    grouped into one partitioned launch per direction; each result equals the oracle's."""
    host, dev = pools
    trace = W.serving_trace(40, 1e6, host, seed=3200, min_bytes=70 << 10, max_bytes=1 << 20, p_validate=0.0,
                            p_bad=0.3)
    srv = lib.Server(0, budget_bytes=1 << 30, device_rings=device_rings)
    try:
        reqs = [(OPS[trace["op"][i]], _request_tensor(dev, trace, i), 0, i) for i in range(len(trace["op"]))]
        first = srv.submit(reqs)
        got = _collect(srv, list(range(first, first + len(reqs))))
        for k in range(len(reqs)):
            c = got[first + k]
            op = reqs[k][0]
            want, wdst = _expected(_request_host(host, trace, k), op)
            assert (c["status"], c["count"]) == want, (k, op, c["status"], c["count"], want)
            out = _output(srv, c, op)
            if wdst is not None:
                assert np.array_equal(out, wdst), k
        st = srv.stats()
        assert st["launches"] < len(reqs)  # requests of one direction shared launches
    finally:
        srv.close()
