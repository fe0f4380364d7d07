"""The host logic of the multi-GPU bench path (replicas: one process per GPU, no data-path
collective), run as two gloo ranks on the CPU: rank bookkeeping from the launcher's
environment, the max over ranks of the timed region, and the whole-job sum of units."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    r, lr, ws = bench.dist_env()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cpu")
        # each rank timed a different duration and processed a different number of units
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, dev)
        units = bench.sum_over_ranks(1000 * (rank + 1), dist, dev)
        dist.barrier()
        queue.put((r, lr, ws, ms, units))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for r, (rank, local_rank, world, ms, units) in enumerate(got):
        assert (rank, local_rank, world) == (r, r, 2)
        assert ms == 15.0  # the slowest rank's time
        assert units == 3000  # all ranks' units


def test_single_process_has_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.sum_over_ranks(7, None, None) == 7.0


@pytest.mark.parametrize("flag", ["--no-batched", "--no-serving", "--no-e2e"])
def test_bench_arguments_parse(flag, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", flag, "--steps", "4", "--warmup", "3"])
    a = bench.parse()
    assert a.steps == 4 and a.warmup == 3 and a.gpus == 1


def _run_bench(args, tmp_path, extra_env=None):
    import subprocess
    env = dict(os.environ, GBU_WORKLOAD_CACHE=str(tmp_path / "cache"))
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_line(tmp_path):
    """`bench.py --impl reference` (the oracle on the host cores, on bounded samples of the same
    workload) prints one JSON line with the contract's keys."""
    import json
    p = _run_bench(["--impl", "reference", "--size", str(1 << 20), "--cpu-sample", str(1 << 18),
                    "--steps", "2", "--warmup", "1"], tmp_path)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] and "model" not in d["config"]


def test_reference_arm_other_ranks_exit_quietly(tmp_path):
    p = _run_bench(["--impl", "reference", "--size", str(1 << 20), "--steps", "1", "--warmup", "1"], tmp_path,
                   {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_cpu_baseline_shards_combine_to_the_whole_buffer_result():
    """The all-cores CPU baseline's own cut and combination: shards cut at character
    boundaries and run through the oracle give, combined, the oracle's result on the whole
    buffer (valid input, and input with errors in several shards)."""
    import numpy as np

    import bench
    import oracle
    import workloads as W
    u8, u16 = W.profile_buffers("mixed", 200_003, 100_001, 77, cache=False)
    bad8 = u8.copy()
    for k in (150_000, 60_000, 180_000):  # several errors; the first one decides
        while (bad8[k] & 0xC0) == 0x80:
            k -= 1
        bad8[k] = 0xFF
    bad16 = u16.copy()
    bad16[70_000] = 0xDC00
    bad16[30_000] = 0xD800
    bad16[30_001] = 0x41
    for P in (1, 2, 7, 16):
        for a in (u8, bad8):
            cuts = bench._cpu_cuts(a, P)
            assert cuts[0] == 0 and cuts[-1] == a.size and cuts == sorted(cuts)
            assert all(c == a.size or (int(a[c]) & 0xC0) != 0x80 for c in cuts[1:-1])
            got = bench._cpu_combine(cuts, [oracle.validate_utf8(a[cuts[k]:cuts[k + 1]]) for k in range(P)])
            assert got == oracle.validate_utf8(a), (P, got)
            conv = [oracle.convert_utf8_to_utf16le(a[cuts[k]:cuts[k + 1]])[0] for k in range(P)]
            assert bench._cpu_combine(cuts, conv) == oracle.convert_utf8_to_utf16le(a)[0]
        for a in (u16, bad16):
            cuts = bench._cpu_cuts(a, P)
            assert all(not (0xDC00 <= int(a[c]) <= 0xDFFF and 0xD800 <= int(a[c - 1]) <= 0xDBFF)
                       for c in cuts[1:-1] if 0 < c < a.size)
            got = bench._cpu_combine(cuts, [oracle.validate_utf16le(a[cuts[k]:cuts[k + 1]]) for k in range(P)])
            assert got == oracle.validate_utf16le(a), (P, got)
            conv = [oracle.convert_utf16le_to_utf8(a[cuts[k]:cuts[k + 1]])[0] for k in range(P)]
            assert bench._cpu_combine(cuts, conv) == oracle.convert_utf16le_to_utf8(a)[0]
