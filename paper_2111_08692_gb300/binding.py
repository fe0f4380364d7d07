"""Thin ctypes binding of the C ABI in include/gbutf.h.

The ``gbu_*`` functions mirror the C entry points one to one (pointers and sizes as Python
ints); ``Codec`` adds argument marshalling for torch tensors.  Every step of the work runs in
the CUDA library: this module only passes pointers, sizes and stream handles.  If the
library has not been built, loading fails with an error instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

STATUS = {
    0: "OK", 1: "HEADER_BITS", 2: "TOO_SHORT", 3: "TOO_LONG", 4: "OVERLONG", 5: "TOO_LARGE",
    6: "SURROGATE", 16: "OUTPUT_TOO_SMALL", 17: "BAD_ARGUMENT", 18: "CUDA_ERROR", 19: "TIMEOUT",
    20: "NOALLOC_TOO_LARGE", 21: "CANCELLED", 22: "OVER_BUDGET",
}
# Largest input (bytes) of gbu_convert_utf8_to_utf16le_noalloc (GBU_NOALLOC_MAX_UNITS).
NOALLOC_MAX_UNITS = 1 << 28
STATUS_CODE = {v: k for k, v in STATUS.items()}


class GbuResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("count", ctypes.c_uint64)]


class GbuBatchConfig(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("strings_per_claim", ctypes.c_uint32),
                ("long_bytes", ctypes.c_uint32), ("tuned_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class GbuServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("streams", ctypes.c_int32),
                ("groups_per_stream", ctypes.c_int32), ("max_group", ctypes.c_uint32),
                ("max_large_group", ctypes.c_uint32), ("large_bytes", ctypes.c_uint64),
                ("max_request_units", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("device_rings", ctypes.c_uint32)]


class GbuRequest(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("flags", ctypes.c_int32), ("src", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("arrival_ns", ctypes.c_uint64), ("tag", ctypes.c_uint64)]


class GbuCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("result", GbuResult),
                ("dst", ctypes.c_void_p), ("arrival_ns", ctypes.c_uint64), ("admit_ns", ctypes.c_uint64),
                ("complete_ns", ctypes.c_uint64)]


class GbuServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "admitted", "completed", "launches", "groups",
                                                "budget_used_bytes", "peak_budget_bytes", "inflight", "pending")]


REQ_DISCARD_OUTPUT = 1  # gbu_request.flags: free the output at completion

# Operation codes of the batched calls (gbu_op).
OPS = ("validate_utf8", "utf16_length_from_utf8", "convert_utf8_to_utf16le", "validate_utf16le",
       "utf8_length_from_utf16le", "convert_utf16le_to_utf8")
OP_CODE = {name: i for i, name in enumerate(OPS)}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it was not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(
                    f"CUDA library {path} is missing: build it with "
                    "paper_2111_08692_gb300.build.build() (there is no CPU fallback)")
            L = ctypes.CDLL(path)
            vp, u64, i32, u32, i64 = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                      ctypes.c_int64)
            L.gbu_create.restype = vp
            L.gbu_create.argtypes = [i32, u64]
            L.gbu_destroy.restype = None
            L.gbu_destroy.argtypes = [vp]
            L.gbu_reset.restype = i32
            L.gbu_reset.argtypes = [vp]
            L.gbu_set_wait_limit.restype = None
            L.gbu_set_wait_limit.argtypes = [vp, u32]
            L.gbu_debug_skip_publish.restype = None
            L.gbu_debug_skip_publish.argtypes = [vp, i64]
            L.gbu_set_early_exit.restype = None
            L.gbu_set_early_exit.argtypes = [vp, i32]
            for name in ("gbu_shard_cuts_utf8", "gbu_shard_cuts_utf16le"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, u32, vp, vp]
            for name in ("gbu_shard_cuts_utf8_host", "gbu_shard_cuts_utf16le_host"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, u64, u32, vp]
            L.gbu_combine_shards.restype = i32
            L.gbu_combine_shards.argtypes = [vp, vp, u32, vp]
            for name in ("gbu_validate_utf16be", "gbu_utf8_length_from_utf16be"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, vp, vp]
            for name in ("gbu_convert_utf16be_to_utf8", "gbu_convert_utf8_to_utf16be"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, vp, u64, vp, vp]
            for name in ("gbu_validate_utf32", "gbu_utf8_length_from_utf32", "gbu_utf32_length_from_utf8"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, vp, vp]
            for name in ("gbu_utf16_length_from_utf32", "gbu_utf32_length_from_utf16le"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, vp, vp]
            for name in ("gbu_convert_utf32_to_utf8", "gbu_convert_utf8_to_utf32", "gbu_convert_utf32_to_utf16le",
                         "gbu_convert_utf16le_to_utf32"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, vp, u64, vp, vp]
            for name in ("gbu_validate_utf8_sync", "gbu_validate_utf16le_sync", "gbu_utf16_length_from_utf8_sync",
                         "gbu_utf8_length_from_utf16le_sync"):
                getattr(L, name).restype = GbuResult
                getattr(L, name).argtypes = [vp, vp, u64, vp]
            for name in ("gbu_convert_utf8_to_utf16le_sync", "gbu_convert_utf16le_to_utf8_sync"):
                getattr(L, name).restype = GbuResult
                getattr(L, name).argtypes = [vp, vp, u64, vp, u64, vp]
            L.gbu_per_string_loop.restype = i32
            L.gbu_per_string_loop.argtypes = [vp, i32, vp, vp, u64, vp, vp, vp, vp]
            L.gbu_chunked_create.restype = vp
            L.gbu_chunked_create.argtypes = [i32, i32, u64]
            L.gbu_chunked_push.restype = i32
            L.gbu_chunked_push.argtypes = [vp, vp, u64, i32, vp, u64, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(GbuResult)]
            L.gbu_chunked_reset.restype = i32
            L.gbu_chunked_reset.argtypes = [vp]
            L.gbu_chunked_destroy.restype = None
            L.gbu_chunked_destroy.argtypes = [vp]
            L.gbu_launch_count.restype = u64
            L.gbu_launch_count.argtypes = [vp]
            L.gbu_launch_config.restype = i32
            L.gbu_launch_config.argtypes = [vp, vp, i32]
            for name in ("gbu_validate_utf8", "gbu_validate_utf16le", "gbu_utf16_length_from_utf8",
                         "gbu_utf8_length_from_utf16le"):
                f = getattr(L, name)
                f.restype = i32
                f.argtypes = [vp, vp, u64, vp, vp]
            for name in ("gbu_convert_utf8_to_utf16le", "gbu_convert_utf16le_to_utf8"):
                f = getattr(L, name)
                f.restype = i32
                f.argtypes = [vp, vp, u64, vp, u64, vp, vp]
            for name in ("gbu_validate_utf8_batched", "gbu_validate_utf16le_batched",
                         "gbu_utf16_length_from_utf8_batched", "gbu_utf8_length_from_utf16le_batched"):
                f = getattr(L, name)
                f.restype = i32
                f.argtypes = [vp, vp, vp, u64, vp, vp]
            for name in ("gbu_convert_utf8_to_utf16le_batched", "gbu_convert_utf16le_to_utf8_batched"):
                f = getattr(L, name)
                f.restype = i32
                f.argtypes = [vp, vp, vp, u64, vp, vp, vp, vp]
            L.gbu_exclusive_scan_u64.restype = i32
            L.gbu_exclusive_scan_u64.argtypes = [vp, vp, u64, vp, vp, vp]
            L.gbu_get_batch_config.restype = i32
            L.gbu_get_batch_config.argtypes = [vp, i32, ctypes.POINTER(GbuBatchConfig)]
            L.gbu_set_batch_config.restype = i32
            L.gbu_set_batch_config.argtypes = [vp, i32, ctypes.POINTER(GbuBatchConfig)]
            L.gbu_tune_batched.restype = i32
            L.gbu_tune_batched.argtypes = [vp, i32, vp, vp, u64, vp, vp, vp, i32, vp,
                                           ctypes.POINTER(GbuBatchConfig)]
            L.gbu_graph_begin.restype = i32
            L.gbu_graph_begin.argtypes = [vp, vp]
            L.gbu_graph_end.restype = vp
            L.gbu_graph_end.argtypes = [vp, vp]
            L.gbu_graph_launch.restype = i32
            L.gbu_graph_launch.argtypes = [vp, vp]
            L.gbu_graph_kernels.restype = u64
            L.gbu_graph_kernels.argtypes = [vp]
            L.gbu_graph_destroy.restype = None
            L.gbu_graph_destroy.argtypes = [vp]
            L.gbu_server_default_config.restype = None
            L.gbu_server_default_config.argtypes = [ctypes.POINTER(GbuServerConfig)]
            L.gbu_server_create.restype = vp
            L.gbu_server_create.argtypes = [i32, ctypes.POINTER(GbuServerConfig)]
            L.gbu_server_destroy.restype = None
            L.gbu_server_destroy.argtypes = [vp]
            L.gbu_server_now_ns.restype = u64
            L.gbu_server_now_ns.argtypes = [vp]
            L.gbu_server_submit.restype = i32
            L.gbu_server_submit.argtypes = [vp, vp, u64, ctypes.POINTER(ctypes.c_uint64)]
            L.gbu_server_cancel.restype = i32
            L.gbu_server_cancel.argtypes = [vp, u64]
            L.gbu_server_poll.restype = i32
            L.gbu_server_poll.argtypes = [vp, vp, i32]
            L.gbu_server_release.restype = i32
            L.gbu_server_release.argtypes = [vp, u64]
            L.gbu_server_get_stats.restype = i32
            L.gbu_server_get_stats.argtypes = [vp, ctypes.POINTER(GbuServerStats)]
            L.gbu_server_copy_output.restype = i32
            L.gbu_server_copy_output.argtypes = [vp, u64, vp, u64]
            L.gbu_arena_create.restype = vp
            L.gbu_arena_create.argtypes = [u64, u64]
            L.gbu_arena_alloc.restype = i32
            L.gbu_arena_alloc.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_uint64)]
            L.gbu_arena_free.restype = i32
            L.gbu_arena_free.argtypes = [vp, u64]
            for name in ("gbu_arena_used", "gbu_arena_largest_free", "gbu_arena_free_blocks"):
                getattr(L, name).restype = u64
                getattr(L, name).argtypes = [vp]
            L.gbu_arena_destroy.restype = None
            L.gbu_arena_destroy.argtypes = [vp]
            L.gbu_pipe_create.restype = vp
            L.gbu_pipe_create.argtypes = [i32, u64, i32]
            L.gbu_pipe_destroy.restype = None
            L.gbu_pipe_destroy.argtypes = [vp]
            for name in ("gbu_pipe_validate_utf8", "gbu_pipe_validate_utf16le", "gbu_pipe_utf16_length_from_utf8",
                         "gbu_pipe_utf8_length_from_utf16le"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, ctypes.POINTER(GbuResult)]
            for name in ("gbu_pipe_convert_utf8_to_utf16le", "gbu_pipe_convert_utf16le_to_utf8"):
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(GbuResult)]
            L.gbu_convert_utf8_to_utf16le_noalloc.restype = i32
            L.gbu_convert_utf8_to_utf16le_noalloc.argtypes = [vp, u64, vp, u64, vp, vp]
            _lib = L
    return _lib


# ---- the C entry points, same names -------------------------------------------------------

def gbu_create(device: int, max_units: int) -> int:
    return lib().gbu_create(device, max_units)


def gbu_destroy(ctx: int) -> None:
    lib().gbu_destroy(ctx)


def gbu_reset(ctx: int) -> int:
    return lib().gbu_reset(ctx)


def gbu_set_wait_limit(ctx: int, rounds: int) -> None:
    lib().gbu_set_wait_limit(ctx, rounds)


def gbu_debug_skip_publish(ctx: int, tile: int) -> None:
    lib().gbu_debug_skip_publish(ctx, tile)


def gbu_set_early_exit(ctx: int, enable: bool) -> None:
    lib().gbu_set_early_exit(ctx, 1 if enable else 0)


def gbu_launch_count(ctx: int) -> int:
    return int(lib().gbu_launch_count(ctx))


def gbu_launch_config(ctx: int) -> list[int]:
    buf = (ctypes.c_int32 * 16)()
    m = lib().gbu_launch_config(ctx, buf, 16)
    return [int(buf[i]) for i in range(m)]


def gbu_validate_utf8(ctx, src, n, result, stream) -> int:
    return lib().gbu_validate_utf8(ctx, src, n, result, stream)


def gbu_validate_utf16le(ctx, src, n, result, stream) -> int:
    return lib().gbu_validate_utf16le(ctx, src, n, result, stream)


def gbu_utf16_length_from_utf8(ctx, src, n, length, stream) -> int:
    return lib().gbu_utf16_length_from_utf8(ctx, src, n, length, stream)


def gbu_utf8_length_from_utf16le(ctx, src, n, length, stream) -> int:
    return lib().gbu_utf8_length_from_utf16le(ctx, src, n, length, stream)


def gbu_convert_utf8_to_utf16le(ctx, src, n, dst, cap, result, stream) -> int:
    return lib().gbu_convert_utf8_to_utf16le(ctx, src, n, dst, cap, result, stream)


def gbu_convert_utf16le_to_utf8(ctx, src, n, dst, cap, result, stream) -> int:
    return lib().gbu_convert_utf16le_to_utf8(ctx, src, n, dst, cap, result, stream)


def gbu_validate_utf8_batched(ctx, src, off, B, results, stream) -> int:
    return lib().gbu_validate_utf8_batched(ctx, src, off, B, results, stream)


def gbu_validate_utf16le_batched(ctx, src, off, B, results, stream) -> int:
    return lib().gbu_validate_utf16le_batched(ctx, src, off, B, results, stream)


def gbu_utf16_length_from_utf8_batched(ctx, src, off, B, lens, stream) -> int:
    return lib().gbu_utf16_length_from_utf8_batched(ctx, src, off, B, lens, stream)


def gbu_utf8_length_from_utf16le_batched(ctx, src, off, B, lens, stream) -> int:
    return lib().gbu_utf8_length_from_utf16le_batched(ctx, src, off, B, lens, stream)


def gbu_convert_utf8_to_utf16le_batched(ctx, src, off, B, dst, dst_off, results, stream) -> int:
    return lib().gbu_convert_utf8_to_utf16le_batched(ctx, src, off, B, dst, dst_off, results, stream)


def gbu_convert_utf16le_to_utf8_batched(ctx, src, off, B, dst, dst_off, results, stream) -> int:
    return lib().gbu_convert_utf16le_to_utf8_batched(ctx, src, off, B, dst, dst_off, results, stream)


def gbu_exclusive_scan_u64(ctx, src, count, out, result, stream) -> int:
    return lib().gbu_exclusive_scan_u64(ctx, src, count, out, result, stream)


def gbu_get_batch_config(ctx, op: int) -> GbuBatchConfig:
    cfg = GbuBatchConfig()
    _check(lib().gbu_get_batch_config(ctx, op, ctypes.byref(cfg)), "gbu_get_batch_config")
    return cfg


def gbu_set_batch_config(ctx, op: int, cfg: GbuBatchConfig) -> int:
    return lib().gbu_set_batch_config(ctx, op, ctypes.byref(cfg))


def gbu_tune_batched(ctx, op, src, off, B, dst, dst_off, out, reps, stream, chosen) -> int:
    return lib().gbu_tune_batched(ctx, op, src, off, B, dst, dst_off, out, reps, stream, chosen)


def gbu_graph_begin(ctx, stream) -> int:
    return lib().gbu_graph_begin(ctx, stream)


def gbu_graph_end(ctx, stream) -> int:
    return lib().gbu_graph_end(ctx, stream)


def gbu_graph_launch(graph, stream) -> int:
    return lib().gbu_graph_launch(graph, stream)


def gbu_graph_kernels(graph) -> int:
    return lib().gbu_graph_kernels(graph)


def gbu_graph_destroy(graph) -> None:
    lib().gbu_graph_destroy(graph)


def gbu_convert_utf8_to_utf16le_noalloc(src, n, dst, cap, result, stream) -> int:
    return lib().gbu_convert_utf8_to_utf16le_noalloc(src, n, dst, cap, result, stream)


# ---- torch marshalling --------------------------------------------------------------------

class GbuError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise GbuError(f"{what}: {STATUS.get(rc, rc)}")


def result_tuple(t) -> tuple[str, int]:
    """(status name, count) of a result tensor (2 x int64: status word, count)."""
    v = t.detach().to("cpu").view(-1).tolist()
    return STATUS.get(int(v[0]) & 0xFFFFFFFF, int(v[0])), int(v[1]) & 0xFFFFFFFFFFFFFFFF


class Codec:
    """One library context on one CUDA device, driven with torch tensors.

    Methods enqueue work on ``stream`` (default: torch's current stream) and return the
    device tensor that will hold the result; ``result_tuple`` reads it.  One Codec serves one
    stream at a time (its workspace is shared by its calls)."""

    def __init__(self, device: int | None = None, max_units: int = 1 << 31):
        import torch
        self.torch = torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        self.ctx = gbu_create(device, max_units)
        if not self.ctx:
            raise GbuError("gbu_create failed")

    def close(self):
        if self.ctx:
            gbu_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # helpers
    def _stream(self, stream):
        if stream is None:
            stream = self.torch.cuda.current_stream(self.device)
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    def new_result(self):
        return self.torch.empty(2, dtype=self.torch.int64, device=f"cuda:{self.device}")

    @staticmethod
    def _ptr(t):
        return t.data_ptr() if t is not None and t.numel() else 0

    def launches(self) -> int:
        return gbu_launch_count(self.ctx)

    def launch_config(self) -> dict:
        v = gbu_launch_config(self.ctx)
        names = ("validate_utf8", "utf16_length_from_utf8", "convert_utf8_to_utf16le",
                 "validate_utf16le", "utf8_length_from_utf16le", "convert_utf16le_to_utf8")
        return {"sms": v[0], "ctas_per_sm": dict(zip(names, v[1:7])), "threads_per_cta": v[7],
                "transcoder_threads_per_cta": v[8], "stream_tile_bytes": v[9], "partition_bytes": v[10]}

    def set_wait_limit(self, rounds: int):
        gbu_set_wait_limit(self.ctx, rounds)

    def debug_skip_publish(self, tile: int):
        gbu_debug_skip_publish(self.ctx, tile)

    def set_early_exit(self, enable: bool):
        gbu_set_early_exit(self.ctx, enable)

    def shard_cuts(self, src, P: int, out=None, stream=None):
        """Cuts (P + 1 int64 values, on this device) of a device buffer: uint8 (UTF-8) or
        int16 (UTF-16LE), split into P shards at character boundaries."""
        out = self.torch.empty(P + 1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        fn = lib().gbu_shard_cuts_utf16le if src.dtype == self.torch.int16 else lib().gbu_shard_cuts_utf8
        _check(fn(self.ctx, self._ptr(src), src.numel(), P, out.data_ptr(), self._stream(stream)),
               "gbu_shard_cuts")
        return out

    def reset(self):
        _check(gbu_reset(self.ctx), "gbu_reset")

    # operations (tensors are 1-D, contiguous, on this device)
    def validate_utf8(self, src, result=None, stream=None):
        result = self.new_result() if result is None else result
        _check(gbu_validate_utf8(self.ctx, self._ptr(src), src.numel(), result.data_ptr(),
                                 self._stream(stream)), "gbu_validate_utf8")
        return result

    def validate_utf16le(self, src, result=None, stream=None):
        result = self.new_result() if result is None else result
        _check(gbu_validate_utf16le(self.ctx, self._ptr(src), src.numel(), result.data_ptr(),
                                    self._stream(stream)), "gbu_validate_utf16le")
        return result

    def utf16_length_from_utf8(self, src, out=None, stream=None):
        out = self.torch.empty(1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        _check(gbu_utf16_length_from_utf8(self.ctx, self._ptr(src), src.numel(), out.data_ptr(),
                                          self._stream(stream)), "gbu_utf16_length_from_utf8")
        return out

    def utf8_length_from_utf16le(self, src, out=None, stream=None):
        out = self.torch.empty(1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        _check(gbu_utf8_length_from_utf16le(self.ctx, self._ptr(src), src.numel(), out.data_ptr(),
                                            self._stream(stream)), "gbu_utf8_length_from_utf16le")
        return out

    def convert_utf8_to_utf16le(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(gbu_convert_utf8_to_utf16le(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                           result.data_ptr(), self._stream(stream)),
               "gbu_convert_utf8_to_utf16le")
        return result

    # host-synchronising forms: (status name, count) by value, the stream waited for
    def _sync(self, fn, name, *args):
        r = fn(self.ctx, *args)
        return STATUS.get(r.status, r.status), int(r.count)

    def validate_utf8_sync(self, src, stream=None):
        return self._sync(lib().gbu_validate_utf8_sync, "gbu_validate_utf8_sync", self._ptr(src), src.numel(),
                          self._stream(stream))

    def validate_utf16le_sync(self, src, stream=None):
        return self._sync(lib().gbu_validate_utf16le_sync, "gbu_validate_utf16le_sync", self._ptr(src), src.numel(),
                          self._stream(stream))

    def utf16_length_from_utf8_sync(self, src, stream=None):
        return self._sync(lib().gbu_utf16_length_from_utf8_sync, "gbu_utf16_length_from_utf8_sync", self._ptr(src),
                          src.numel(), self._stream(stream))

    def utf8_length_from_utf16le_sync(self, src, stream=None):
        return self._sync(lib().gbu_utf8_length_from_utf16le_sync, "gbu_utf8_length_from_utf16le_sync",
                          self._ptr(src), src.numel(), self._stream(stream))

    def convert_utf8_to_utf16le_sync(self, src, dst, stream=None, cap=None):
        cap = dst.numel() if cap is None else cap
        return self._sync(lib().gbu_convert_utf8_to_utf16le_sync, "gbu_convert_utf8_to_utf16le_sync", self._ptr(src),
                          src.numel(), self._ptr(dst), cap, self._stream(stream))

    def convert_utf16le_to_utf8_sync(self, src, dst, stream=None, cap=None):
        cap = dst.numel() if cap is None else cap
        return self._sync(lib().gbu_convert_utf16le_to_utf8_sync, "gbu_convert_utf16le_to_utf8_sync", self._ptr(src),
                          src.numel(), self._ptr(dst), cap, self._stream(stream))

    # UTF-16BE forms: int16 tensors holding the words as they lie in memory (big-endian bytes)
    def validate_utf16be(self, src, result=None, stream=None):
        result = self.new_result() if result is None else result
        _check(lib().gbu_validate_utf16be(self.ctx, self._ptr(src), src.numel(), result.data_ptr(),
                                          self._stream(stream)), "gbu_validate_utf16be")
        return result

    def utf8_length_from_utf16be(self, src, out=None, stream=None):
        out = self.torch.empty(1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        _check(lib().gbu_utf8_length_from_utf16be(self.ctx, self._ptr(src), src.numel(), out.data_ptr(),
                                                  self._stream(stream)), "gbu_utf8_length_from_utf16be")
        return out

    def convert_utf16be_to_utf8(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(lib().gbu_convert_utf16be_to_utf8(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                                 result.data_ptr(), self._stream(stream)),
               "gbu_convert_utf16be_to_utf8")
        return result

    def convert_utf8_to_utf16be(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(lib().gbu_convert_utf8_to_utf16be(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                                 result.data_ptr(), self._stream(stream)),
               "gbu_convert_utf8_to_utf16be")
        return result

    # UTF-32 forms: int32 tensors of units (host byte order)
    def validate_utf32(self, src, result=None, stream=None):
        result = self.new_result() if result is None else result
        _check(lib().gbu_validate_utf32(self.ctx, self._ptr(src), src.numel(), result.data_ptr(),
                                        self._stream(stream)), "gbu_validate_utf32")
        return result

    def utf8_length_from_utf32(self, src, out=None, stream=None):
        out = self.torch.empty(1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        _check(lib().gbu_utf8_length_from_utf32(self.ctx, self._ptr(src), src.numel(), out.data_ptr(),
                                                self._stream(stream)), "gbu_utf8_length_from_utf32")
        return out

    def utf32_length_from_utf8(self, src, out=None, stream=None):
        out = self.torch.empty(1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        _check(lib().gbu_utf32_length_from_utf8(self.ctx, self._ptr(src), src.numel(), out.data_ptr(),
                                                self._stream(stream)), "gbu_utf32_length_from_utf8")
        return out

    def convert_utf32_to_utf8(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(lib().gbu_convert_utf32_to_utf8(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                               result.data_ptr(), self._stream(stream)), "gbu_convert_utf32_to_utf8")
        return result

    def convert_utf8_to_utf32(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(lib().gbu_convert_utf8_to_utf32(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                               result.data_ptr(), self._stream(stream)), "gbu_convert_utf8_to_utf32")
        return result

    def utf16_length_from_utf32(self, src, out=None, stream=None):
        out = self.torch.empty(1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        _check(lib().gbu_utf16_length_from_utf32(self.ctx, self._ptr(src), src.numel(), out.data_ptr(),
                                                 self._stream(stream)), "gbu_utf16_length_from_utf32")
        return out

    def utf32_length_from_utf16le(self, src, out=None, stream=None):
        out = self.torch.empty(1, dtype=self.torch.int64, device=f"cuda:{self.device}") if out is None else out
        _check(lib().gbu_utf32_length_from_utf16le(self.ctx, self._ptr(src), src.numel(), out.data_ptr(),
                                                   self._stream(stream)), "gbu_utf32_length_from_utf16le")
        return out

    def convert_utf32_to_utf16le(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(lib().gbu_convert_utf32_to_utf16le(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                                  result.data_ptr(), self._stream(stream)),
               "gbu_convert_utf32_to_utf16le")
        return result

    def convert_utf16le_to_utf32(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(lib().gbu_convert_utf16le_to_utf32(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                                  result.data_ptr(), self._stream(stream)),
               "gbu_convert_utf16le_to_utf32")
        return result

    # batched forms: src is the concatenation, off the B+1 offsets (int64 tensor, code units)
    def new_results(self, B: int):
        return self.torch.empty((B, 2), dtype=self.torch.int64, device=f"cuda:{self.device}")

    def _batched(self, fn, name, src, off, out, dst=None, dst_off=None, stream=None):
        B = off.numel() - 1
        args = [self.ctx, self._ptr(src), self._ptr(off), max(B, 0)]
        if dst is not None:
            args += [self._ptr(dst), self._ptr(dst_off)]
        _check(fn(*args, self._ptr(out), self._stream(stream)), name)
        return out

    def validate_utf8_batched(self, src, off, results=None, stream=None):
        results = self.new_results(off.numel() - 1) if results is None else results
        return self._batched(gbu_validate_utf8_batched, "gbu_validate_utf8_batched", src, off, results,
                             stream=stream)

    def validate_utf16le_batched(self, src, off, results=None, stream=None):
        results = self.new_results(off.numel() - 1) if results is None else results
        return self._batched(gbu_validate_utf16le_batched, "gbu_validate_utf16le_batched", src, off, results,
                             stream=stream)

    def utf16_length_from_utf8_batched(self, src, off, lens=None, stream=None):
        lens = self.torch.empty(off.numel() - 1, dtype=self.torch.int64, device=off.device) if lens is None else lens
        return self._batched(gbu_utf16_length_from_utf8_batched, "gbu_utf16_length_from_utf8_batched", src, off,
                             lens, stream=stream)

    def utf8_length_from_utf16le_batched(self, src, off, lens=None, stream=None):
        lens = self.torch.empty(off.numel() - 1, dtype=self.torch.int64, device=off.device) if lens is None else lens
        return self._batched(gbu_utf8_length_from_utf16le_batched, "gbu_utf8_length_from_utf16le_batched", src,
                             off, lens, stream=stream)

    def convert_utf8_to_utf16le_batched(self, src, off, dst, dst_off, results=None, stream=None):
        results = self.new_results(off.numel() - 1) if results is None else results
        return self._batched(gbu_convert_utf8_to_utf16le_batched, "gbu_convert_utf8_to_utf16le_batched", src, off,
                             results, dst, dst_off, stream=stream)

    def convert_utf16le_to_utf8_batched(self, src, off, dst, dst_off, results=None, stream=None):
        results = self.new_results(off.numel() - 1) if results is None else results
        return self._batched(gbu_convert_utf16le_to_utf8_batched, "gbu_convert_utf16le_to_utf8_batched", src, off,
                             results, dst, dst_off, stream=stream)

    def exclusive_scan_u64(self, values, out=None, result=None, stream=None):
        """out[k] = sum(values[:k]) for k = 0 .. len(values) (int64 tensors on this device)."""
        out = self.torch.empty(values.numel() + 1, dtype=self.torch.int64, device=values.device) if out is None else out
        result = self.new_result() if result is None else result
        _check(gbu_exclusive_scan_u64(self.ctx, self._ptr(values), values.numel(), out.data_ptr(),
                                      result.data_ptr(), self._stream(stream)), "gbu_exclusive_scan_u64")
        return out, result

    def batch_config(self, op: str) -> dict:
        return gbu_get_batch_config(self.ctx, OP_CODE[op]).as_dict()

    def set_batch_config(self, op: str, warps_per_cta: int, strings_per_claim: int, long_bytes: int):
        cfg = GbuBatchConfig(warps_per_cta, strings_per_claim, long_bytes, 0.0)
        _check(gbu_set_batch_config(self.ctx, OP_CODE[op], cfg), "gbu_set_batch_config")

    def tune_batched(self, op: str, src, off, out, dst=None, dst_off=None, reps: int = 3, stream=None) -> dict:
        """Autotunes the geometry of batched `op` on this batch; returns the chosen one."""
        chosen = GbuBatchConfig()
        _check(gbu_tune_batched(self.ctx, OP_CODE[op], self._ptr(src), self._ptr(off), max(off.numel() - 1, 0),
                                self._ptr(dst), self._ptr(dst_off), self._ptr(out), reps, self._stream(stream),
                                ctypes.byref(chosen)), "gbu_tune_batched")
        return chosen.as_dict()

    def capture(self, fn, stream):
        """Runs fn() with `stream` captured into a CUDA graph of library calls; returns a Graph."""
        s = self._stream(stream)
        _check(gbu_graph_begin(self.ctx, s), "gbu_graph_begin")
        try:
            fn()
        finally:
            g = gbu_graph_end(self.ctx, s)
        if not g:
            raise GbuError("gbu_graph_end failed")
        return Graph(g, self)

    def convert_utf16le_to_utf8(self, src, dst, result=None, stream=None, cap=None):
        result = self.new_result() if result is None else result
        cap = dst.numel() if cap is None else cap
        _check(gbu_convert_utf16le_to_utf8(self.ctx, self._ptr(src), src.numel(), self._ptr(dst), cap,
                                           result.data_ptr(), self._stream(stream)),
               "gbu_convert_utf16le_to_utf8")
        return result


def shard_cuts_host(data, P: int):
    """Cuts (P + 1 uint64 values) of a host buffer: a uint8 numpy array (UTF-8) or a uint16
    one (UTF-16LE), split into P shards at character boundaries (gbu_shard_cuts_*_host)."""
    import numpy as np
    data = np.ascontiguousarray(data)
    cuts = np.empty(P + 1, dtype=np.uint64)
    fn = lib().gbu_shard_cuts_utf16le_host if data.dtype == np.uint16 else lib().gbu_shard_cuts_utf8_host
    _check(fn(data.ctypes.data if data.size else None, data.size, P, cuts.ctypes.data), "gbu_shard_cuts_host")
    return cuts


def combine_shards(cuts, parts) -> tuple[str, int]:
    """The whole buffer's (status name, count) from its shards' results (gbu_combine_shards);
    parts: P (status name, count) pairs."""
    import numpy as np
    cuts = np.ascontiguousarray(cuts, dtype=np.uint64)
    P = len(parts)
    arr = (GbuResult * P)()
    for k, (name, count) in enumerate(parts):
        arr[k] = GbuResult(STATUS_CODE[name], 0, int(count))
    out = GbuResult()
    _check(lib().gbu_combine_shards(cuts.ctypes.data, arr, P, ctypes.byref(out)), "gbu_combine_shards")
    return STATUS.get(out.status, out.status), int(out.count)


def convert_utf8_to_utf16le_noalloc(src, dst, result, stream=None, cap=None):
    """The context-free transcoder on the current device (no allocation: the caller passes
    ``dst`` and ``result``).  ``src`` holds at most NOALLOC_MAX_UNITS bytes; calls must not
    overlap one another (they share one workspace per device).

    The tensors are checked before the call, since the C function has no context device to
    check them against and takes ``cap`` in 16-bit units: ``src`` must be uint8, ``dst`` have
    2-byte elements, ``result`` hold at least 16 bytes, and all three lie on the current CUDA
    device.  A tensor that fails a check raises GbuError and nothing is enqueued."""
    import torch
    name = "gbu_convert_utf8_to_utf16le_noalloc"
    if src.numel() > NOALLOC_MAX_UNITS:
        raise GbuError(f"{name}: input of {src.numel()} bytes is above "
                       f"the limit of {NOALLOC_MAX_UNITS} bytes of the allocation-free form")
    if src.dtype != torch.uint8:
        raise GbuError(f"{name}: src must be a uint8 tensor, not {src.dtype}")
    if dst.element_size() != 2:
        raise GbuError(f"{name}: dst must have 2-byte elements (UTF-16 units), not {dst.dtype}")
    if result.numel() * result.element_size() < 16:
        raise GbuError(f"{name}: result must hold at least 16 bytes (one gbu_result)")
    for what, t in (("src", src), ("dst", dst), ("result", result)):
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise GbuError(f"{name}: {what} is not on the current CUDA device")
    if stream is None:
        stream = torch.cuda.current_stream()
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    cap = dst.numel() if cap is None else cap
    _check(gbu_convert_utf8_to_utf16le_noalloc(Codec._ptr(src), src.numel(), Codec._ptr(dst), cap,
                                               result.data_ptr(), s),
           "gbu_convert_utf8_to_utf16le_noalloc")
    return result


class Chunked:
    """The resumable form (gbu_chunked_*): push host chunks of one input (numpy uint8 for
    UTF-8, uint16 for UTF-16LE); each push returns (output units as a numpy array, (status
    name, count)) with the same meaning as the C call."""

    def __init__(self, op: str, max_chunk_units: int, device: int = 0):
        self.op = op
        self.handle = lib().gbu_chunked_create(device, OP_CODE[op], max_chunk_units)
        if not self.handle:
            raise GbuError("gbu_chunked_create failed")
        self.out_dtype = {"convert_utf8_to_utf16le": "uint16", "convert_utf16le_to_utf8": "uint8"}.get(op)
        self.max_chunk = max_chunk_units

    def push(self, chunk, last: bool = False, out_cap: int | None = None):
        import numpy as np
        chunk = np.ascontiguousarray(chunk)
        n = chunk.size
        if out_cap is None:
            out_cap = (n + 4) * (3 if self.op == "convert_utf16le_to_utf8" else 1)
        out = np.empty(out_cap if self.out_dtype else 0, dtype=self.out_dtype or "uint8")
        out_n = ctypes.c_uint64(0)
        res = GbuResult()
        _check(lib().gbu_chunked_push(self.handle, chunk.ctypes.data if n else None, n, 1 if last else 0,
                                      out.ctypes.data if out.size else None, out.size, ctypes.byref(out_n),
                                      ctypes.byref(res)), "gbu_chunked_push")
        return out[:out_n.value], (STATUS.get(res.status, res.status), int(res.count))

    def reset(self):
        _check(lib().gbu_chunked_reset(self.handle), "gbu_chunked_reset")

    def close(self):
        if self.handle:
            lib().gbu_chunked_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipe:
    """The host-buffer form (gbu_pipe_*): the six operations on host arrays (numpy uint8 for
    UTF-8, uint16 for UTF-16LE; pinned memory for the copies to overlap the kernels), one
    synchronous call each.  Each method returns (status name, count) with the meaning of the
    single-buffer call on the whole input; the transcoders write into the given host array."""

    def __init__(self, device: int = 0, piece_units: int = 0, streams: int = 0):
        self.handle = lib().gbu_pipe_create(device, piece_units, streams)
        if not self.handle:
            raise GbuError("gbu_pipe_create failed")

    @staticmethod
    def _ptr(a):
        return a.ctypes.data if a is not None and a.size else None

    def _call(self, name, src, *rest):
        res = GbuResult()
        _check(getattr(lib(), "gbu_pipe_" + name)(self.handle, self._ptr(src), src.size, *rest, ctypes.byref(res)),
               "gbu_pipe_" + name)
        return STATUS.get(res.status, res.status), int(res.count)

    def validate_utf8(self, src):
        return self._call("validate_utf8", src)

    def validate_utf16le(self, src):
        return self._call("validate_utf16le", src)

    def utf16_length_from_utf8(self, src):
        return self._call("utf16_length_from_utf8", src)

    def utf8_length_from_utf16le(self, src):
        return self._call("utf8_length_from_utf16le", src)

    def convert_utf8_to_utf16le(self, src, dst, cap=None):
        return self._call("convert_utf8_to_utf16le", src, self._ptr(dst), dst.size if cap is None else cap)

    def convert_utf16le_to_utf8(self, src, dst, cap=None):
        return self._call("convert_utf16le_to_utf8", src, self._ptr(dst), dst.size if cap is None else cap)

    def close(self):
        if self.handle:
            lib().gbu_pipe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """An instantiated CUDA graph of library calls (Codec.capture)."""

    def __init__(self, handle: int, codec: Codec):
        self.handle = handle
        self.codec = codec  # keeps the context alive

    def launch(self, stream=None):
        _check(gbu_graph_launch(self.handle, self.codec._stream(stream)), "gbu_graph_launch")

    def kernels(self) -> int:
        return gbu_graph_kernels(self.handle)

    def close(self):
        if self.handle:
            gbu_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving loop -------------------------------------------------------------------------

def gbu_server_default_config() -> GbuServerConfig:
    cfg = GbuServerConfig()
    lib().gbu_server_default_config(ctypes.byref(cfg))
    return cfg


def gbu_server_create(device: int, cfg: GbuServerConfig | None) -> int:
    return lib().gbu_server_create(device, ctypes.byref(cfg) if cfg is not None else None)


def gbu_server_destroy(server) -> None:
    lib().gbu_server_destroy(server)


def gbu_server_now_ns(server) -> int:
    return lib().gbu_server_now_ns(server)


def gbu_server_submit(server, reqs, count, first_id) -> int:
    return lib().gbu_server_submit(server, reqs, count, first_id)


def gbu_server_cancel(server, rid) -> int:
    return lib().gbu_server_cancel(server, rid)


def gbu_server_poll(server, out, max_out) -> int:
    return lib().gbu_server_poll(server, out, max_out)


def gbu_server_release(server, rid) -> int:
    return lib().gbu_server_release(server, rid)


def gbu_server_copy_output(server, rid, host, nbytes) -> int:
    return lib().gbu_server_copy_output(server, rid, host, nbytes)


def gbu_server_get_stats(server, out) -> int:
    return lib().gbu_server_get_stats(server, out)


class Server:
    """The serving loop (gbu_server_*) on one device.  Requests are (op, src tensor, arrival
    time in server-clock ns, tag); completions come back as dicts."""

    def __init__(self, device: int = 0, **cfg):
        c = gbu_server_default_config()
        for k, v in cfg.items():
            setattr(c, k, v)
        self.cfg = c
        self.handle = gbu_server_create(device, c)
        if not self.handle:
            raise GbuError("gbu_server_create failed")
        self._buf = (GbuCompletion * 4096)()

    def now_ns(self) -> int:
        return gbu_server_now_ns(self.handle)

    def submit(self, requests) -> int:
        """requests: iterable of (op name, src tensor or (pointer, n), arrival_ns, tag)."""
        reqs = list(requests)
        arr = (GbuRequest * max(len(reqs), 1))()
        for i, (op, src, arrival, tag) in enumerate(reqs):
            ptr, n = (src.data_ptr() if src.numel() else 0, src.numel()) if hasattr(src, "data_ptr") else src
            arr[i] = GbuRequest(OP_CODE[op], 0, ptr, n, int(arrival), int(tag))
        first = ctypes.c_uint64(0)
        _check(gbu_server_submit(self.handle, arr, len(reqs), ctypes.byref(first)), "gbu_server_submit")
        return first.value

    def submit_raw(self, arr, count: int) -> int:
        """Submits a prepared (GbuRequest * k) array."""
        first = ctypes.c_uint64(0)
        _check(gbu_server_submit(self.handle, arr, count, ctypes.byref(first)), "gbu_server_submit")
        return first.value

    def cancel(self, rid: int) -> bool:
        return gbu_server_cancel(self.handle, rid) == 0

    def poll(self, max_out: int = 4096) -> list[dict]:
        k = gbu_server_poll(self.handle, self._buf, min(max_out, len(self._buf)))
        out = []
        for i in range(k):
            c = self._buf[i]
            out.append({"id": c.id, "tag": c.tag, "status": STATUS.get(c.result.status, c.result.status),
                        "count": c.result.count, "dst": c.dst, "arrival_ns": c.arrival_ns,
                        "admit_ns": c.admit_ns, "complete_ns": c.complete_ns})
        return out

    def release(self, rid: int) -> None:
        _check(gbu_server_release(self.handle, rid), "gbu_server_release")

    def copy_output(self, rid: int, units: int, dtype):
        """The first `units` output units of completed request rid, as a numpy array."""
        import numpy as np
        out = np.empty(units, dtype=dtype)
        _check(gbu_server_copy_output(self.handle, rid, out.ctypes.data if units else None, out.nbytes),
               "gbu_server_copy_output")
        return out

    def stats(self) -> dict:
        st = GbuServerStats()
        _check(gbu_server_get_stats(self.handle, ctypes.byref(st)), "gbu_server_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self.handle:
            gbu_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Arena:
    """The server's arena bookkeeping (offsets only), for host-side tests."""

    def __init__(self, capacity: int, align: int = 256):
        self.handle = lib().gbu_arena_create(capacity, align)
        if not self.handle:
            raise GbuError("gbu_arena_create failed")

    def alloc(self, size: int):
        off = ctypes.c_uint64(0)
        rc = lib().gbu_arena_alloc(self.handle, size, ctypes.byref(off))
        return off.value if rc == 0 else None

    def free(self, off: int) -> bool:
        return lib().gbu_arena_free(self.handle, off) == 0

    def used(self) -> int:
        return lib().gbu_arena_used(self.handle)

    def largest_free(self) -> int:
        return lib().gbu_arena_largest_free(self.handle)

    def free_blocks(self) -> int:
        return lib().gbu_arena_free_blocks(self.handle)

    def close(self):
        if self.handle:
            lib().gbu_arena_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
