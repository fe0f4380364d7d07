#!/usr/bin/env python3
"""Benchmark: UTF-8 <-> UTF-16LE validation and transcoding of 1 GiB buffers on GB300.

One step = for each of the five profiles (ascii, latin, cyrillic, cjk, emoji), on a resident
1 GiB UTF-8 buffer and a resident 1 GiB UTF-16LE buffer:
    validate_utf8, utf16_length_from_utf8, convert_utf8_to_utf16le,
    validate_utf16le, utf8_length_from_utf16le, convert_utf16le_to_utf8
(30 library calls, 32.2 GB of input).  `value` is input GB/s over the whole job (all ranks).
Inputs are larger than L2 (1 GiB vs 129 MB), so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the reference codec (oracle/, a
scalar CPU program) on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "UTF-8↔UTF-16 GB/s input & % HBM roofline; batched strings/s; p99 latency"
OPS = ("validate_utf8", "utf16_length_from_utf8", "convert_utf8_to_utf16le",
       "validate_utf16le", "utf8_length_from_utf16le", "convert_utf16le_to_utf8")
UTF8_INPUT_OPS = ("validate_utf8", "utf16_length_from_utf8", "convert_utf8_to_utf16le")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth (context beside the measured copy peak)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--size", type=int, default=1 << 30, help="bytes per UTF-8 (and UTF-16) buffer")
    ap.add_argument("--profiles", default="ascii,latin,cyrillic,cjk,emoji")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=32 << 20, help="bytes per buffer for the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-strings", type=int, default=1_000_000)
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--loop-sample", type=int, default=3000,
                    help="strings timed through the per-string launch loop")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the L2-resident 1 MiB latency table")
    ap.add_argument("--no-be", action="store_true", help="skip the UTF-16BE leg")
    ap.add_argument("--no-utf32", action="store_true", help="skip the UTF-32 leg")
    ap.add_argument("--small-reps", type=int, default=200)
    ap.add_argument("--sweep-size", type=int, default=256 << 20, help="UTF-8 bytes per invalid-input sweep buffer")
    ap.add_argument("--sweep-reps", type=int, default=5)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-loads", default="1e4,3e4,1e5,3e5,1e6", help="offered loads, requests/s")
    ap.add_argument("--serving-requests", type=int, default=20000, help="requests per offered load (at most)")
    ap.add_argument("--serving-seconds", type=float, default=1.0, help="arrival window per load (at most)")
    ap.add_argument("--serving-streams", type=int, default=None)
    ap.add_argument("--serving-groups", type=int, default=None, help="launch groups in flight per stream")
    ap.add_argument("--serving-large-group", type=int, default=None)
    ap.add_argument("--serving-rings", default="host,device",
                    help="descriptor/result ring placements to measure (host: mapped pinned memory, device: device "
                         "memory with copies); the first is the headline")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    """The sum of x over all ranks (x itself without a process group)."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload_config(args, profiles):
    return {
        "workload": f"single {args.size >> 20} MiB buffers per profile ({', '.join(profiles)}): "
                    "validate + length + transcode, UTF-8->UTF-16LE and UTF-16LE->UTF-8",
        "buffer_bytes": args.size,
        "profiles": list(profiles),
        "ops_per_profile": list(OPS),
        "input_bytes_per_step": 6 * args.size * len(profiles),
        "l2": "inputs larger than L2 (no flush needed)",
        "parallelism": "replicas" if args.gpus > 1 else "single GPU",
    }


# ---- clocks --------------------------------------------------------------------------------

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons every 20 ms while running.  Entering
    waits (up to 3 s) for the first sample, so that nvidia-smi's start-up does not eat into
    the timed region; only the samples after that are summarised."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.gpu = ids[local_rank].strip() if local_rank < len(ids) and ids[local_rank].strip().isdigit() \
            else str(local_rank)
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t_end = time.time() + 3.0
            while not self.lines and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        self.start = len(self.lines)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "start", 0):]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


# ---- roofline bookkeeping -------------------------------------------------------------------

def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def ncu_traffic(op: str):
    """DRAM bytes per launch (read + write) from the committed ncu summary, if it was taken
    on the current sources of that kernel (the summary records their hash), else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None, None
    from paper_2111_08692_gb300.build import kernel_hash
    want = kernel_hash(op)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 5 and parts[0] == op and parts[1] == want:
            # op  hash  profile  bytes_per_launch_at_scale  scale_note...
            return float(parts[3]), parts[2]
    return None, None


# ---- our arm ------------------------------------------------------------------------------

def run_ours(args):
    rank, local_rank, world = dist_env()
    profiles = [p for p in args.profiles.split(",") if p]
    import workloads as W
    if local_rank == 0:
        W.prepare_single_buffers(profiles, args.size)  # spawn pool, before any CUDA work
        if not args.no_sweep:
            W.prepare_sweeps(args.sweep_size)
    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        dist.barrier()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    from paper_2111_08692_gb300 import Codec, result_tuple
    from paper_2111_08692_gb300.build import build
    build()
    codec = Codec(local_rank, max_units=args.size + 4096)
    stream = torch.cuda.current_stream(dev)

    bufs = []
    for prof in profiles:
        u8, u16 = W.single_buffer_1gib(prof, args.size, mmap=True)
        s8 = torch.from_numpy(np.asarray(u8)).to(dev)
        s16 = torch.from_numpy(np.asarray(u16).view(np.int16)).to(dev)
        n16 = int(codec.utf16_length_from_utf8(s8).item())
        n8 = int(codec.utf8_length_from_utf16le(s16).item())
        d16 = torch.empty(n16, dtype=torch.int16, device=dev)
        d8 = torch.empty(n8, dtype=torch.uint8, device=dev)
        res = torch.empty((6, 2), dtype=torch.int64, device=dev)
        ln = torch.empty((2, 1), dtype=torch.int64, device=dev)
        bufs.append(dict(profile=prof, s8=s8, s16=s16, d16=d16, d8=d8, res=res, len=ln, n16=n16, n8=n8,
                         u8=u8, u16=u16))
    torch.cuda.synchronize()

    def call(b, op):
        if op == "validate_utf8":
            codec.validate_utf8(b["s8"], result=b["res"][0])
        elif op == "utf16_length_from_utf8":
            codec.utf16_length_from_utf8(b["s8"], out=b["len"][0])
        elif op == "convert_utf8_to_utf16le":
            codec.convert_utf8_to_utf16le(b["s8"], b["d16"], result=b["res"][2])
        elif op == "validate_utf16le":
            codec.validate_utf16le(b["s16"], result=b["res"][3])
        elif op == "utf8_length_from_utf16le":
            codec.utf8_length_from_utf16le(b["s16"], out=b["len"][1])
        else:
            codec.convert_utf16le_to_utf8(b["s16"], b["d8"], result=b["res"][5])

    def algo_bytes(b, op):
        if op in ("validate_utf8", "utf16_length_from_utf8"):
            return b["s8"].numel()
        if op in ("validate_utf16le", "utf8_length_from_utf16le"):
            return 2 * b["s16"].numel()
        if op == "convert_utf8_to_utf16le":
            return b["s8"].numel() + 2 * b["n16"]
        return 2 * b["s16"].numel() + b["n8"]

    def step(events=None):
        for b in bufs:
            for op in OPS:
                if events is not None:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    call(b, op)
                    e1.record(stream)
                    events.append((b["profile"], op, e0, e1))
                else:
                    call(b, op)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of what is timed: every call succeeded and the lengths agree
    for b in bufs:
        r = [result_tuple(b["res"][i]) for i in (0, 2, 3, 5)]
        assert r[0] == ("OK", b["s8"].numel()) and r[1] == ("OK", b["n16"]), (b["profile"], r)
        assert r[2] == ("OK", b["s16"].numel()) and r[3] == ("OK", b["n8"]), (b["profile"], r)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    launches0 = codec.launches()
    events = []
    with ClockSampler(local_rank) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(events)
        t1.record(stream)
        torch.cuda.synchronize()
    launches = codec.launches() - launches0
    total_ms = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    if dist:
        dist.barrier()

    in_bytes_step = sum(b["s8"].numel() * 3 + 2 * b["s16"].numel() * 3 for b in bufs)
    ms_per_step = total_ms / args.steps
    # whole job: the input bytes every rank processed in one step over the slowest rank's time
    value = sum_over_ranks(in_bytes_step, dist, dev) / (ms_per_step * 1e-3) / 1e9

    # per-kernel durations (same stream, inside the timed region)
    per = {}
    for prof, op, e0, e1 in events:
        per.setdefault(op, {}).setdefault(prof, []).append(e0.elapsed_time(e1))
    peak, peak_kind = measured_peak()
    breakdown = {}
    op_tot = {}
    for op in OPS:
        breakdown[op] = {}
        tot_ms, tot_bytes = 0.0, 0
        for b in bufs:
            ms = statistics.mean(per[op][b["profile"]])
            ab = algo_bytes(b, op)
            inb = b["s8"].numel() if op in UTF8_INPUT_OPS else 2 * b["s16"].numel()
            breakdown[op][b["profile"]] = {"ms": round(ms, 4), "min_ms": round(min(per[op][b["profile"]]), 4),
                                           "median_ms": round(statistics.median(per[op][b["profile"]]), 4),
                                           "input_gbs": round(inb / ms / 1e6, 1),
                                           "traffic_gbs": round(ab / ms / 1e6, 1),
                                           "frac": round(ab / ms / 1e6 / peak, 3)}
            tot_ms += ms
            tot_bytes += ab
        op_tot[op] = (tot_ms, tot_bytes)
    dom = max(op_tot, key=lambda o: op_tot[o][0])
    dom_ms, dom_bytes = op_tot[dom]
    achieved = dom_bytes / dom_ms / 1e6  # GB/s: bytes per launch averaged over the profiles
    traffic, traffic_note = ncu_traffic(dom)
    if args.size != 1 << 30 or tuple(profiles) != tuple(W.PROFILE_ORDER):
        traffic, traffic_note = None, None  # the summary holds the five 1 GiB launches' traffic
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "algorithmic_bytes_per_launch": dom_bytes / len(bufs),
                "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4), "nominal_peak": NOMINAL_HBM_GBS}
    if traffic_note:
        roofline["traffic_profile"] = traffic_note

    cfg = workload_config(args, profiles)
    cfg["launch"] = codec.launch_config()
    line = {"metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded profiles standing in for the paper's lipsum texts)",
            "config": cfg, "roofline": roofline,
            "gpu_launches": int(launches), "clocks": clk.summary(), "breakdown": breakdown}

    if not args.no_e2e and args.e2e_steps > 0:
        pinned = pinned_host(bufs)
        line["e2e"] = run_e2e(args, bufs, dist, pinned)
        line["e2e_async"] = run_e2e_async(args, codec, bufs, stream, dist, world, call, pinned)
        del pinned
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(bufs, args.cpu_sample)
    if not args.no_sweep:
        line["sweep"] = run_sweep(args, codec, dev)
    if not args.no_small:
        line["l2_resident_1mib"] = run_small(args, codec, dev)
    if not args.no_be:
        line["utf16be"] = run_be(args, codec, bufs, stream, peak)
    if not args.no_utf32:
        line["utf32"] = run_utf32(args, codec, bufs, stream, peak)
    if not args.no_batched and args.batched_strings > 0:
        line["batched"] = run_batched(args, codec, dev, dist, world)
    if not args.no_serving:
        line["serving"] = run_serving(args, dev, dist, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    codec.close()
    if dist:
        dist.destroy_process_group()


def run_be(args, codec, bufs, stream, peak, reps=3):
    """The UTF-16BE calls on the same buffers: each profile's UTF-16 buffer with its words'
    bytes exchanged (the same text in big-endian order), and its UTF-8 buffer transcoded to
    UTF-16BE.  Mean of `reps` launches after one untimed, CUDA events on the launching stream;
    the fraction counts input + output bytes against the measured copy bandwidth."""
    import torch
    from paper_2111_08692_gb300 import result_tuple
    out = {"reps": reps, "ops": {}}
    for b in bufs:
        be = b["s16"].view(torch.uint8).view(-1, 2).flip(1).contiguous().view(torch.int16).view(-1)
        res = torch.empty(2, dtype=torch.int64, device=be.device)
        ln = torch.empty(1, dtype=torch.int64, device=be.device)
        n16, n8 = b["n16"], b["n8"]
        calls = {"validate_utf16be": (lambda: codec.validate_utf16be(be, result=res), 2 * be.numel(), 0),
                 "utf8_length_from_utf16be": (lambda: codec.utf8_length_from_utf16be(be, out=ln), 2 * be.numel(), 0),
                 "convert_utf16be_to_utf8": (lambda: codec.convert_utf16be_to_utf8(be, b["d8"], result=res),
                                             2 * be.numel(), n8),
                 "convert_utf8_to_utf16be": (lambda: codec.convert_utf8_to_utf16be(b["s8"], b["d16"], result=res),
                                             b["s8"].numel(), 2 * n16)}
        for op, (fn, inb, outb) in calls.items():
            fn()
            torch.cuda.synchronize()
            if op.startswith("convert") or op.startswith("validate"):
                r = result_tuple(res)
                assert r[0] == "OK", (b["profile"], op, r)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out["ops"].setdefault(op, {})[b["profile"]] = {
                "ms": round(ms, 4), "input_gbs": round(inb / ms / 1e6, 1),
                "frac": round((inb + outb) / ms / 1e6 / peak, 3)}
        assert int(ln.item()) == n8
        del be
        torch.cuda.empty_cache()
    return out


def run_utf32(args, codec, bufs, stream, peak, reps=3):
    """The UTF-32 calls on the same text: each profile's UTF-8 buffer transcoded to UTF-32 (by
    the library, untimed), then validation and the UTF-8 length of that UTF-32 buffer and its
    transcoding to UTF-8 and to UTF-16LE, the UTF-32 length and transcoding of the UTF-8 buffer,
    and the transcoding of the UTF-16LE buffer to UTF-32.  Mean of
    `reps` launches after one untimed; the fraction counts input + output bytes against the
    measured copy bandwidth."""
    import torch
    from paper_2111_08692_gb300 import result_tuple
    out = {"reps": reps, "ops": {}}
    for b in bufs:
        s8 = b["s8"]
        ln = torch.empty(1, dtype=torch.int64, device=s8.device)
        res = torch.empty(2, dtype=torch.int64, device=s8.device)
        n32 = int(codec.utf32_length_from_utf8(s8, out=ln).item())
        u32 = torch.empty(n32, dtype=torch.int32, device=s8.device)
        r = result_tuple(codec.convert_utf8_to_utf32(s8, u32, result=res))
        assert r == ("OK", n32), (b["profile"], r)
        n8 = s8.numel()
        d8 = torch.empty(n8, dtype=torch.uint8, device=s8.device)
        n16 = int(codec.utf16_length_from_utf32(u32, out=ln).item())
        d16 = torch.empty(n16, dtype=torch.int16, device=s8.device)
        s16 = b["s16"]
        n32b = int(codec.utf32_length_from_utf16le(s16, out=ln).item())
        u32b = torch.empty(n32b, dtype=torch.int32, device=s8.device)
        calls = {"validate_utf32": (lambda: codec.validate_utf32(u32, result=res), 4 * n32, 0),
                 "utf8_length_from_utf32": (lambda: codec.utf8_length_from_utf32(u32, out=ln), 4 * n32, 0),
                 "convert_utf32_to_utf8": (lambda: codec.convert_utf32_to_utf8(u32, d8, result=res), 4 * n32, n8),
                 "utf32_length_from_utf8": (lambda: codec.utf32_length_from_utf8(s8, out=ln), n8, 0),
                 "convert_utf8_to_utf32": (lambda: codec.convert_utf8_to_utf32(s8, u32, result=res), n8, 4 * n32),
                 "convert_utf32_to_utf16le": (lambda: codec.convert_utf32_to_utf16le(u32, d16, result=res),
                                              4 * n32, 2 * n16),
                 "convert_utf16le_to_utf32": (lambda: codec.convert_utf16le_to_utf32(s16, u32b, result=res),
                                              2 * s16.numel(), 4 * n32b)}
        for op, (fn, inb, outb) in calls.items():
            fn()
            torch.cuda.synchronize()
            if "length" in op:
                want = n8 if op == "utf8_length_from_utf32" else n32
                assert int(ln.item()) == want, (b["profile"], op)
            else:
                assert result_tuple(res)[0] == "OK", (b["profile"], op, result_tuple(res))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out["ops"].setdefault(op, {})[b["profile"]] = {
                "ms": round(ms, 4), "input_gbs": round(inb / ms / 1e6, 1),
                "frac": round((inb + outb) / ms / 1e6 / peak, 3)}
        del u32, d8, d16, u32b
        torch.cuda.empty_cache()
    return out


def run_small(args, codec, dev):
    """The 1 MiB mixed-profile buffer (50% U+0000-007F, 20% U+0080-07FF, 20% U+0800-FFFF, 10%
    U+10000-10FFFF) and its UTF-16LE form: each of the six operations launched small_reps times
    back to back, each launch timed by CUDA events.  The buffers stay in L2, so these are
    L2-resident latencies (min and median per launch), not HBM-roofline numbers."""
    import numpy as np
    import torch
    import workloads as W
    stream = torch.cuda.current_stream(dev)
    u8, u16, _, _ = W.mixed_1mib()
    s8 = torch.from_numpy(np.ascontiguousarray(u8)).to(dev)
    s16 = torch.from_numpy(np.ascontiguousarray(u16).view(np.int16)).to(dev)
    d16 = torch.empty(s8.numel() + 8, dtype=torch.int16, device=dev)
    d8 = torch.empty(3 * s16.numel() + 8, dtype=torch.uint8, device=dev)
    res = torch.empty(2, dtype=torch.int64, device=dev)
    ln = torch.empty(1, dtype=torch.int64, device=dev)
    calls = {"validate_utf8": lambda: codec.validate_utf8(s8, result=res),
             "utf16_length_from_utf8": lambda: codec.utf16_length_from_utf8(s8, out=ln),
             "convert_utf8_to_utf16le": lambda: codec.convert_utf8_to_utf16le(s8, d16, result=res),
             "validate_utf16le": lambda: codec.validate_utf16le(s16, result=res),
             "utf8_length_from_utf16le": lambda: codec.utf8_length_from_utf16le(s16, out=ln),
             "convert_utf16le_to_utf8": lambda: codec.convert_utf16le_to_utf8(s16, d8, result=res)}
    out = {"utf8_bytes": int(s8.numel()), "utf16_words": int(s16.numel()), "reps": args.small_reps,
           "unit": "us per launch", "ops": {}}
    for op, fn in calls.items():
        for _ in range(5):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.small_reps)]
        for e0, e1 in ev:
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        t = [e0.elapsed_time(e1) * 1e3 for e0, e1 in ev]
        out["ops"][op] = {"min_us": round(min(t), 2), "median_us": round(statistics.median(t), 2)}
    return out


def run_sweep(args, codec, dev):
    """The invalid-input sweep: Cyrillic and CJK buffers (sweep_size UTF-8 bytes, half as many
    UTF-16 words) with errors at per-character rates 1e-6, 1e-4 and 1e-2.  Each validating
    operation is timed (CUDA events, mean of sweep_reps launches after one untimed) with early
    exit on -- the default, which stops work past the first flagged chunk -- and off (a full
    scan); both give the same first error, which is reported."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2111_08692_gb300 import result_tuple
    stream = torch.cuda.current_stream(dev)
    out = {"buffer_bytes": args.sweep_size, "reps": args.sweep_reps, "unit": "ms per launch",
           "ops": {}}
    for prof in W.SWEEP_PROFILES:
        for rate in W.SWEEP_RATES:
            d = W.sweep_buffers(prof, rate, args.sweep_size)
            s8 = torch.from_numpy(np.asarray(d["u8"])).to(dev)
            s16 = torch.from_numpy(np.asarray(d["u16"]).view(np.int16)).to(dev)
            d16 = torch.empty(s8.numel() + 8, dtype=torch.int16, device=dev)
            d8 = torch.empty(3 * s16.numel() + 8, dtype=torch.uint8, device=dev)
            res = torch.empty(2, dtype=torch.int64, device=dev)
            calls = {"validate_utf8": lambda: codec.validate_utf8(s8, result=res),
                     "convert_utf8_to_utf16le": lambda: codec.convert_utf8_to_utf16le(s8, d16, result=res),
                     "validate_utf16le": lambda: codec.validate_utf16le(s16, result=res),
                     "convert_utf16le_to_utf8": lambda: codec.convert_utf16le_to_utf8(s16, d8, result=res)}
            for op, fn in calls.items():
                rec = {}
                for mode in ("early_exit", "full_scan"):
                    codec.set_early_exit(mode == "early_exit")
                    fn()
                    torch.cuda.synchronize()
                    first = result_tuple(res)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(args.sweep_reps):
                        fn()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    assert result_tuple(res) == first
                    rec[mode + "_ms"] = round(e0.elapsed_time(e1) / args.sweep_reps, 4)
                    rec[mode + "_result"] = list(first)
                assert rec["early_exit_result"] == rec["full_scan_result"], (prof, rate, op, rec)
                rec["first_error"] = rec.pop("early_exit_result")
                del rec["full_scan_result"]
                out["ops"].setdefault(op, {}).setdefault(prof, {})[f"{rate:g}"] = rec
            codec.set_early_exit(True)
            del s8, s16, d16, d8
            torch.cuda.empty_cache()
    return out


def run_batched(args, codec, dev, dist, world):
    """Batched strings/s: B strings (log-normal lengths, median 64 B, sigma 1.5, the five
    profiles, 1% with an error), each validated, measured and transcoded in both directions
    into packed outputs.  One step = six library kernels replayed from one CUDA graph:
    UTF-16 lengths of the UTF-8 strings, their exclusive scan (output offsets), UTF-8 ->
    UTF-16LE; UTF-8 lengths of the UTF-16LE strings, scan, UTF-16LE -> UTF-8.  Compared with
    a per-string launch loop (two single-buffer transcoder calls per string, worst-case
    output capacities) timed on the first --loop-sample strings."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2111_08692_gb300 import result_tuple
    b = W.batched_strings(args.batched_strings, 1000)
    B = b["off8"].size - 1
    s8 = torch.from_numpy(b["u8"]).to(dev)
    s16 = torch.from_numpy(b["u16"].view(np.int16)).to(dev)
    o8 = torch.from_numpy(b["off8"].view(np.int64)).to(dev)
    o16 = torch.from_numpy(b["off16"].view(np.int64)).to(dev)
    side = torch.cuda.Stream(dev)
    len16 = torch.empty(B, dtype=torch.int64, device=dev)
    len8 = torch.empty(B, dtype=torch.int64, device=dev)
    doff16 = torch.empty(B + 1, dtype=torch.int64, device=dev)
    doff8 = torch.empty(B + 1, dtype=torch.int64, device=dev)
    sres = torch.empty((2, 2), dtype=torch.int64, device=dev)
    res8 = codec.new_results(B)
    res16 = codec.new_results(B)
    with torch.cuda.stream(side):
        codec.utf16_length_from_utf8_batched(s8, o8, len16, stream=side)
        codec.exclusive_scan_u64(len16, doff16, sres[0], stream=side)
        codec.utf8_length_from_utf16le_batched(s16, o16, len8, stream=side)
        codec.exclusive_scan_u64(len8, doff8, sres[1], stream=side)
    side.synchronize()
    n16, n8 = int(doff16[-1].item()), int(doff8[-1].item())
    d16 = torch.empty(n16 + 8, dtype=torch.int16, device=dev)
    d8 = torch.empty(n8 + 16, dtype=torch.uint8, device=dev)
    # autotune each kernel's geometry on this batch (untimed)
    tuned = {
        "utf16_length_from_utf8": codec.tune_batched("utf16_length_from_utf8", s8, o8, len16, stream=side),
        "convert_utf8_to_utf16le": codec.tune_batched("convert_utf8_to_utf16le", s8, o8, res8, d16, doff16,
                                                      stream=side),
        "utf8_length_from_utf16le": codec.tune_batched("utf8_length_from_utf16le", s16, o16, len8, stream=side),
        "convert_utf16le_to_utf8": codec.tune_batched("convert_utf16le_to_utf8", s16, o16, res16, d8, doff8,
                                                      stream=side),
    }

    def body():
        codec.utf16_length_from_utf8_batched(s8, o8, len16, stream=side)
        codec.exclusive_scan_u64(len16, doff16, sres[0], stream=side)
        codec.convert_utf8_to_utf16le_batched(s8, o8, d16, doff16, res8, stream=side)
        codec.utf8_length_from_utf16le_batched(s16, o16, len8, stream=side)
        codec.exclusive_scan_u64(len8, doff8, sres[1], stream=side)
        codec.convert_utf16le_to_utf8_batched(s16, o16, d8, doff8, res16, stream=side)

    graph = codec.capture(body, side)
    for _ in range(max(args.warmup, 3)):
        graph.launch(side)
    side.synchronize()
    # what is timed is correct: the strings with an injected error, and only they, fail
    r8 = res8.cpu().numpy()[:, 0] & 0xFFFFFFFF
    r16 = res16.cpu().numpy()[:, 0] & 0xFFFFFFFF
    assert np.array_equal(r8 != 0, b["err8"]) and np.array_equal(r16 != 0, b["err16"])
    assert result_tuple(sres[0])[0] == "OK" and result_tuple(sres[1])[0] == "OK"
    if dist:
        dist.barrier()
    launches0 = codec.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(side)
    for _ in range(args.batched_steps):
        graph.launch(side)
    e1.record(side)
    side.synchronize()
    launches = codec.launches() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.batched_steps, dist, dev)
    strings_all = sum_over_ranks(B, dist, dev)
    graph.close()
    # per-kernel times (each call bracketed by events, outside the graph)
    per = {}
    for name, fn in (("utf16_length_from_utf8", lambda: codec.utf16_length_from_utf8_batched(s8, o8, len16, stream=side)),
                     ("exclusive_scan_u64", lambda: codec.exclusive_scan_u64(len16, doff16, sres[0], stream=side)),
                     ("convert_utf8_to_utf16le", lambda: codec.convert_utf8_to_utf16le_batched(s8, o8, d16, doff16, res8, stream=side)),
                     ("utf8_length_from_utf16le", lambda: codec.utf8_length_from_utf16le_batched(s16, o16, len8, stream=side)),
                     ("convert_utf16le_to_utf8", lambda: codec.convert_utf16le_to_utf8_batched(s16, o16, d8, doff8, res16, stream=side))):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        a.record(side)
        for _ in range(3):
            fn()
        z.record(side)
        side.synchronize()
        per[name] = round(a.elapsed_time(z) / 3, 4)

    # the per-string launch loop: each string through the single-buffer transcoders, issued
    # by the library's C loop (gbu_per_string_loop), so that the ratio counts launches, not the
    # interpreter
    S = min(args.loop_sample, B)
    from paper_2111_08692_gb300 import lib as _lib
    L = _lib()
    off8 = np.ascontiguousarray(b["off8"][:S + 1], dtype=np.uint64)
    off16 = np.ascontiguousarray(b["off16"][:S + 1], dtype=np.uint64)
    n8s, n16s = np.diff(off8.astype(np.int64)), np.diff(off16.astype(np.int64))
    # worst-case packed outputs: n words for 8 -> 16, 3n bytes for 16 -> 8
    doff16 = np.concatenate([[0], np.cumsum(n8s)]).astype(np.uint64)
    doff8 = np.concatenate([[0], np.cumsum(3 * n16s)]).astype(np.uint64)
    ld16 = torch.empty(max(int(doff16[-1]), 1), dtype=torch.int16, device=dev)
    ld8 = torch.empty(max(int(doff8[-1]), 1), dtype=torch.uint8, device=dev)
    lres = torch.empty((2, S, 2), dtype=torch.int64, device=dev)
    ctx, sh = codec.ctx, side.cuda_stream
    p8, p16 = s8.data_ptr(), s16.data_ptr()

    def loop():
        for rc in (L.gbu_per_string_loop(ctx, 2, p8, off8.ctypes.data, S, ld16.data_ptr(), doff16.ctypes.data,
                                         lres[0].data_ptr(), sh),
                   L.gbu_per_string_loop(ctx, 5, p16, off16.ctypes.data, S, ld8.data_ptr(), doff8.ctypes.data,
                                         lres[1].data_ptr(), sh)):
            if rc != 0:
                raise RuntimeError(f"gbu_per_string_loop: {rc}")

    loop()
    side.synchronize()
    l0 = codec.launches()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(side)
    loop()
    z.record(side)
    side.synchronize()
    loop_launches = codec.launches() - l0
    loop_ms = a.elapsed_time(z)
    loop_sps = S / (loop_ms * 1e-3)
    value = strings_all / (ms * 1e-3)
    return {"metric": "batched strings/s", "value": round(value, 1), "unit": "strings/s",
            "ms_per_step": round(ms, 4), "steps": args.batched_steps, "strings_per_step": B,
            "input_bytes_per_step": int(b["u8"].size + 2 * b["u16"].size),
            "input_gbs": round((b["u8"].size + 2 * b["u16"].size) / (ms * 1e-3) / 1e9, 1),
            "gpu_launches": int(launches), "kernel_ms": per, "tuned": tuned,
            "per_string_loop": {"strings": S, "ms": round(loop_ms, 3), "strings_per_s": round(loop_sps, 1),
                                "gpu_launches": int(loop_launches),
                                "calls": "convert_utf8_to_utf16le then convert_utf16le_to_utf8, one "
                                         "launch per string from the library's C loop (gbu_per_string_loop)"},
            "speedup_vs_loop": round(value / world / loop_sps, 1),
            "config": {"workload": f"{B} strings, log-normal UTF-8 lengths (median 64 B, sigma 1.5, 1 B..64 KiB), "
                                   "five profiles, 1% with one injected error; both directions into packed outputs",
                       "graph": "6 kernels per replay", "l2": "inputs (198 MB + 285 MB) larger than L2"}}


def run_serving(args, dev, dist, world):
    """Serving: requests arrive as a Poisson process at each offered load, with input sizes
    log-uniform on 16 B - 16 MiB, 10% validate-only, the rest split 50/50 between the two
    transcoding directions, the five profiles mixed; inputs are slices of device-resident
    per-profile pools (64 MiB of UTF-8 and 32 Mi words of UTF-16LE each).  The library's
    serving loop admits them against an 8 GiB budget and batches them continuously; the
    client discards outputs at completion.  Latency = completion - scheduled arrival."""
    import numpy as np
    import torch
    import workloads as W
    host = W.serving_pools(64 << 20, seed=2000)
    pools = {}
    for prof, p in host.items():
        pools[prof] = (torch.from_numpy(p["u8"]).to(dev), torch.from_numpy(p["u16"].view(np.int16)).to(dev))
    req_dt = np.dtype([("op", "<i4"), ("flags", "<i4"), ("src", "<u8"), ("n", "<u8"), ("arrival", "<u8"),
                       ("tag", "<u8")])
    comp_dt = np.dtype([("id", "<u8"), ("tag", "<u8"), ("status", "<i4"), ("res", "<i4"), ("count", "<u8"),
                        ("dst", "<u8"), ("arrival", "<u8"), ("admit", "<u8"), ("complete", "<u8")])
    rings = [r for r in args.serving_rings.split(",") if r]
    by_rings = {}
    for ring in rings:
        by_rings[ring], st, srv_cfg = _serving_loads(args, dev, host, pools, req_dt, comp_dt, ring)
    out = by_rings[rings[0]]
    return {"metric": "serving p50/p99 latency at each offered load", "loads": out,
            "rings": rings[0], "loads_by_rings": by_rings,
            "launches": int(st["launches"]), "groups": int(st["groups"]), "completed": int(st["completed"]),
            "peak_budget_bytes": int(st["peak_budget_bytes"]),
            "config": {"workload": "Poisson arrivals; input sizes log-uniform 16 B - 16 MiB; 10% validate-only, "
                                   "45%/45% UTF-8->UTF-16LE / UTF-16LE->UTF-8; five profiles mixed; inputs "
                                   "resident on the device, outputs discarded at completion",
                       "budget_bytes": 8 << 30, "streams": srv_cfg.streams,
                       "groups_per_stream": srv_cfg.groups_per_stream, "max_large_group": srv_cfg.max_large_group,
                       "large_bytes": srv_cfg.large_bytes}}


def _serving_loads(args, dev, host, pools, req_dt, comp_dt, ring):
    """One serving run over every offered load with the given ring placement ("host": request
    descriptors and results in mapped pinned host memory; "device": in device memory, copied
    once each way per launch group).  Returns (per-load rows, final stats, the config)."""
    import numpy as np
    import workloads as W
    from paper_2111_08692_gb300 import OP_CODE, REQ_DISCARD_OUTPUT, Server, gbu_server_poll
    scfg = {"budget_bytes": 8 << 30, "device_rings": 1 if ring == "device" else 0}
    for key, val in (("streams", args.serving_streams), ("groups_per_stream", args.serving_groups),
                     ("max_large_group", args.serving_large_group)):
        if val is not None:
            scfg[key] = val
    srv = Server(dev.index if dev.index is not None else 0, **scfg)
    out = []
    try:
        for rate in [float(x) for x in args.serving_loads.split(",") if x]:
            count = int(min(args.serving_requests, max(100, rate * args.serving_seconds)))
            tr = W.serving_trace(count, rate, host, seed=3000 + int(rate) % 1000)
            reqs = np.zeros(count, dtype=req_dt)
            base = np.zeros(count, dtype=np.uint64)
            in_bytes = 0
            for k, prof in enumerate(W.PROFILE_ORDER):
                sel = tr["profile"] == k
                u8p, u16p = pools[prof][0].data_ptr(), pools[prof][1].data_ptr()
                utf16 = (tr["op"] == 1) | (tr["op"] == 3)
                base[sel & ~utf16] = u8p
                base[sel & utf16] = u16p
            utf16 = (tr["op"] == 1) | (tr["op"] == 3)
            unit = np.where(utf16, 2, 1).astype(np.uint64)
            reqs["op"] = [OP_CODE[W.SERVING_OPS[o]] for o in tr["op"]]
            reqs["flags"] = REQ_DISCARD_OUTPUT
            reqs["src"] = base + tr["start"].astype(np.uint64) * unit
            reqs["n"] = tr["n"]
            reqs["tag"] = np.arange(count)
            in_bytes = int(np.sum(tr["n"].astype(np.uint64) * unit))
            t0 = srv.now_ns() + 20_000_000
            reqs["arrival"] = t0 + tr["arrival_ns"]
            srv.submit_raw(reqs.ctypes.data, count)
            got = np.zeros(count, dtype=comp_dt)
            buf = np.zeros(8192, dtype=comp_dt)
            k = 0
            t_end = time.time() + 120
            while k < count and time.time() < t_end:
                m = gbu_server_poll(srv.handle, buf.ctypes.data, buf.size)
                if m > 0:
                    got[k:k + m] = buf[:m]
                    k += m
                else:
                    time.sleep(0.0002)
            assert k == count, f"serving: {count - k} requests did not complete"
            assert np.all(got["status"] == 0), "serving: a request failed"
            lat_us = (got["complete"].astype(np.int64) - got["arrival"].astype(np.int64)) / 1e3
            span_s = (int(got["complete"].max()) - t0) / 1e9
            st = srv.stats()
            out.append({"offered_rps": rate, "requests": count,
                        "achieved_rps": round(count / span_s, 1),
                        "input_gbs": round(in_bytes / span_s / 1e9, 2),
                        "p50_us": round(float(np.percentile(lat_us, 50)), 1),
                        "p99_us": round(float(np.percentile(lat_us, 99)), 1),
                        "max_us": round(float(lat_us.max()), 1)})
        st = srv.stats()
        cfg = srv.cfg
    finally:
        srv.close()
    return out, st, cfg


def run_e2e(args, bufs, dist, pinned):
    """Same workload through the host-buffer form (gbu_pipe_*): each step makes the 30 calls,
    one synchronous C-ABI call per operation and profile on pinned host buffers; each call
    copies its own input to the device in pieces, runs the single-buffer kernels on them and
    copies the result (and a transcoder's output) back, the copies of one piece overlapping the
    kernels of the others.  Timed on the host clock around the synchronous calls."""
    import time

    import numpy as np
    import torch
    from paper_2111_08692_gb300 import Pipe
    dev = bufs[0]["s8"].device
    pipe = Pipe(dev.index)
    host = [(h8.numpy(), h16.numpy().view(np.uint16), o16.numpy().view(np.uint16), o8.numpy())
            for h8, h16, o16, o8 in pinned]

    def step():
        out = []
        for h8, h16, o16, o8 in host:
            out.append((pipe.validate_utf8(h8), pipe.utf16_length_from_utf8(h8), pipe.convert_utf8_to_utf16le(h8, o16),
                        pipe.validate_utf16le(h16), pipe.utf8_length_from_utf16le(h16),
                        pipe.convert_utf16le_to_utf8(h16, o8)))
        return out

    res = step()
    # the host-buffer calls give the device-resident run's results and outputs
    for b, (h8, h16, o16, o8), r in zip(bufs, host, res):
        n8, n16 = h8.size, h16.size
        assert r == (("OK", n8), ("OK", b["n16"]), ("OK", b["n16"]), ("OK", n16), ("OK", b["n8"]),
                     ("OK", b["n8"])), (b["profile"], r)
        assert torch.equal(torch.from_numpy(o16.view(np.int16)).to(dev), b["d16"][:b["n16"]]), b["profile"]
        assert torch.equal(torch.from_numpy(o8).to(dev), b["d8"][:b["n8"]]), b["profile"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step()
    ms = (time.perf_counter() - t0) * 1e3
    ms = max_over_ranks(ms, dist, dev)
    pipe.close()
    in_bytes = sum(b["s8"].numel() * 3 + 2 * b["s16"].numel() * 3 for b in bufs)
    in_all = sum_over_ranks(in_bytes, dist, dev)
    piece = 64 << 20
    pieces = sum(3 * -(-b["s8"].numel() // piece) + 3 * -(-b["s16"].numel() // piece) for b in bufs)
    return {"value": round(in_all * args.e2e_steps / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": sum(2 * b["n16"] + b["n8"] for b in bufs) + 16 * pieces,
            "steps": args.e2e_steps, "ms_per_step": round(ms / args.e2e_steps, 3),
            "api": "gbu_pipe_* (host buffers, pinned), one synchronous call per operation; pieces of 64 Mi units "
                   "on three streams; every call copies its own input"}


def pinned_host(bufs):
    """Page-locked host copies of every profile's inputs and room for both outputs:
    (UTF-8 input, UTF-16LE input as int16, UTF-16LE output as int16, UTF-8 output)."""
    import numpy as np
    import torch
    host = []
    for b in bufs:
        h8 = torch.empty(b["s8"].numel(), dtype=torch.uint8, pin_memory=True)
        h8.copy_(torch.from_numpy(np.asarray(b["u8"])))
        h16 = torch.empty(b["s16"].numel(), dtype=torch.int16, pin_memory=True)
        h16.copy_(torch.from_numpy(np.asarray(b["u16"]).view(np.int16)))
        o16 = torch.empty(b["n16"], dtype=torch.int16, pin_memory=True)
        o8 = torch.empty(b["n8"], dtype=torch.uint8, pin_memory=True)
        host.append((h8, h16, o16, o8))
    return host


def run_e2e_async(args, codec, bufs, stream, dist, world, call, pinned):
    """Same workload through host memory with the asynchronous device-buffer calls: each step
    copies every profile's inputs from pinned host buffers once, runs the 30 calls, and copies
    results and both transcoded outputs back.
    Three streams pipeline the profiles: the host-to-device copy of profile i+1 and the
    device-to-host copy of profile i-1 overlap the kernels of profile i (the kernels stay on
    the context's one stream), and events order each buffer's reuse across steps."""
    import torch
    host = []
    for h8, h16, o16, o8 in pinned:
        hres = torch.empty((6, 2), dtype=torch.int64, pin_memory=True)
        hlen = torch.empty((2, 1), dtype=torch.int64, pin_memory=True)
        host.append((h8, h16, o16, o8, hres, hlen))
    s_in = torch.cuda.Stream(device=stream.device)
    s_out = torch.cuda.Stream(device=stream.device)
    done_compute = [None] * len(bufs)  # previous step's kernels on buffer i (its inputs are free after)
    done_out = [None] * len(bufs)      # previous step's read-back of buffer i (its outputs are free after)

    def step():
        for i, (b, (h8, h16, o16, o8, hres, hlen)) in enumerate(zip(bufs, host)):
            if done_compute[i] is not None:
                s_in.wait_event(done_compute[i])
            with torch.cuda.stream(s_in):
                b["s8"].copy_(h8, non_blocking=True)
                b["s16"].copy_(h16, non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(s_in)
            stream.wait_event(ev_in)
            if done_out[i] is not None:
                stream.wait_event(done_out[i])
            for op in OPS:
                call(b, op)
            ev_c = torch.cuda.Event()
            ev_c.record(stream)
            done_compute[i] = ev_c
            s_out.wait_event(ev_c)
            with torch.cuda.stream(s_out):
                hres.copy_(b["res"], non_blocking=True)
                hlen.copy_(b["len"], non_blocking=True)
                o16.copy_(b["d16"], non_blocking=True)
                o8.copy_(b["d8"], non_blocking=True)
            ev_o = torch.cuda.Event()
            ev_o.record(s_out)
            done_out[i] = ev_o
        stream.wait_stream(s_out)  # the step ends when its last read-back has landed
        stream.wait_stream(s_in)

    step()
    torch.cuda.synchronize()
    # the pipelined step gives the same results as the device-resident run
    for b, (_, _, o16, o8, hres, hlen) in zip(bufs, host):
        r = hres.tolist()
        assert r[2][1] == b["n16"] and r[5][1] == b["n8"] and r[2][0] == 0 and r[5][0] == 0, (b["profile"], r)
    if dist:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_stream(stream)  # no copy of the timed steps starts before e0
    s_out.wait_stream(stream)
    for _ in range(args.e2e_steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, bufs[0]["s8"].device)
    in_bytes = sum(b["s8"].numel() * 3 + 2 * b["s16"].numel() * 3 for b in bufs)
    in_all = sum_over_ranks(in_bytes, dist, bufs[0]["s8"].device)
    h2d = sum(b["s8"].numel() + 2 * b["s16"].numel() for b in bufs)
    d2h = sum(2 * b["n16"] + b["n8"] + 6 * 16 + 2 * 8 for b in bufs)
    return {"value": round(in_all * args.e2e_steps / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
            "ms_per_step": round(ms / args.e2e_steps, 3),
            "pipeline": "host-to-device copies, kernels and device-to-host copies of consecutive profiles "
                        "overlap on three streams"}


def cpu_baseline(bufs, sample):
    """The reference codec, as it stands, on one host core: the six operations on the first
    `sample` bytes of every profile's UTF-8 buffer and the first sample/2 words of its UTF-16
    buffer (cut back to a character boundary by CPython's codec)."""
    import numpy as np
    import oracle
    o = oracle.default()
    work = []
    for b in bufs:
        a8 = np.asarray(b["u8"][:sample])
        a8 = np.frombuffer(a8.tobytes().decode("utf-8", errors="ignore").encode("utf-8"), np.uint8)
        a16 = np.asarray(b["u16"][:sample // 2])
        a16 = np.frombuffer(a16.tobytes().decode("utf-16-le", errors="ignore").encode("utf-16-le"), np.uint16)
        work.append((a8, a16))
    t = time.perf_counter()
    nbytes = 0
    for a8, a16 in work:
        o.validate_utf8(a8)
        o.utf16_length_from_utf8(a8)
        o.convert_utf8_to_utf16le(a8)
        o.validate_utf16le(a16)
        o.utf8_length_from_utf16le(a16)
        o.convert_utf16le_to_utf8(a16)
        nbytes += 3 * a8.size + 3 * 2 * a16.size
    dt = time.perf_counter() - t
    out = {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"first {sample >> 20} MiB of each profile's UTF-8 and UTF-16 buffer, the same six "
                     f"operations, single thread ({dt:.1f} s)"}
    out["all_cores"] = cpu_baseline_all_cores(o, work)
    return out


def _cpu_cuts(a, P: int):
    """Shard boundaries of the CPU baseline: P + 1 positions, the nominal start floor(k n / P)
    of each shard moved forward to a character start (UTF-8: past continuation bytes, at most
    three; UTF-16: off a second surrogate that follows a first one)."""
    import numpy as np
    n = a.size
    cuts = [0]
    for k in range(1, P):
        c = max(k * n // P, cuts[-1])
        if a.dtype == np.uint8:
            for _ in range(3):
                if c < n and (int(a[c]) & 0xC0) == 0x80:
                    c += 1
        elif 0 < c < n and 0xDC00 <= int(a[c]) <= 0xDFFF and 0xD800 <= int(a[c - 1]) <= 0xDBFF:
            c += 1
        cuts.append(min(c, n))
    cuts.append(n)
    return cuts


def _cpu_combine(cuts, parts):
    """The whole buffer's (status, count) from its shards' results: the first shard (in order)
    with an input error gives the error, its offset moved by the shard's start; otherwise the
    counts add up (an output that is too small is reported as for the whole buffer)."""
    total = 0
    for k, (kind, count) in enumerate(parts):
        if kind not in ("OK", "OUTPUT_TOO_SMALL"):
            return kind, cuts[k] + count
        total += count
    return "OK", total


def cpu_baseline_all_cores(o, work):
    """The same work on every host core: each buffer is split into as many shards as cores at
    character boundaries (_cpu_cuts), the reference codec runs on the shards in parallel threads
    (its calls release the interpreter lock), and the shards' results are combined
    (_cpu_combine)."""
    import concurrent.futures as cf
    cores = os.cpu_count() or 1
    jobs = []
    for a8, a16 in work:
        c8, c16 = _cpu_cuts(a8, cores), _cpu_cuts(a16, cores)
        jobs.append((a8, c8, [a8[c8[k]:c8[k + 1]] for k in range(cores)],
                     a16, c16, [a16[c16[k]:c16[k + 1]] for k in range(cores)]))

    def shard8(s):
        return (o.validate_utf8(s), o.utf16_length_from_utf8(s), o.convert_utf8_to_utf16le(s)[0])

    def shard16(s):
        return (o.validate_utf16le(s), o.utf8_length_from_utf16le(s), o.convert_utf16le_to_utf8(s)[0])

    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        t = time.perf_counter()
        nbytes = 0
        for a8, c8, s8, a16, c16, s16 in jobs:
            r8 = list(ex.map(shard8, s8))
            r16 = list(ex.map(shard16, s16))
            for r, c in ((r8, c8), (r16, c16)):
                _cpu_combine(c, [x[0] for x in r])
                _cpu_combine(c, [x[2] for x in r])
            nbytes += 3 * a8.size + 6 * a16.size
        dt = time.perf_counter() - t
    return {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": cores,
            "sample": f"the same sample split into {cores} shards per buffer at character boundaries, "
                      f"one thread per shard ({dt:.2f} s)"}


# ---- the reference arm ----------------------------------------------------------------------

def run_reference(args):
    rank, local_rank, world = dist_env()
    if rank != 0:
        return
    profiles = [p for p in args.profiles.split(",") if p]
    import numpy as np
    import oracle
    import workloads as W
    W.prepare_single_buffers(profiles, args.size)
    o = oracle.default()
    sample = min(args.cpu_sample, args.size) // 4
    work = []
    for prof in profiles:
        u8, u16 = W.single_buffer_1gib(prof, args.size, mmap=True)
        a8 = np.frombuffer(np.asarray(u8[:sample]).tobytes().decode("utf-8", errors="ignore").encode(), np.uint8)
        a16 = np.frombuffer(np.asarray(u16[:sample // 2]).tobytes().decode("utf-16-le", errors="ignore")
                            .encode("utf-16-le"), np.uint16)
        work.append((a8, a16))

    def step():
        n = 0
        for a8, a16 in work:
            o.validate_utf8(a8)
            o.utf16_length_from_utf8(a8)
            o.convert_utf8_to_utf16le(a8)
            o.validate_utf16le(a16)
            o.utf8_length_from_utf16le(a16)
            o.convert_utf16le_to_utf8(a16)
            n += 3 * a8.size + 6 * a16.size
        return n

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    nbytes = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t
    value = nbytes / dt / 1e9
    sample_desc = (f"first {sample >> 20} MiB of each profile's UTF-8 and UTF-16 buffer per step, the same "
                   "six operations, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded profiles standing in for the paper's lipsum texts)",
            "config": workload_config(args, profiles),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
