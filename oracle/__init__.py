"""Loader for the scalar reference codec in ``oracle/gbu_oracle.c``.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  The CUDA library and its Python binding never import this package.
This module only compiles the C file with gcc and marshals numpy arrays through ctypes; all
of the codec's arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbu_oracle.c")
_HDR = os.path.join(_HERE, "gbu_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libgbu_oracle.so")

# Result kinds, by name (values are the oracle's own; tests map them to the library's by name).
KINDS = {
    "OK": 0,
    "HEADER_BITS": 1,
    "TOO_SHORT": 2,
    "TOO_LONG": 3,
    "OVERLONG": 4,
    "TOO_LARGE": 5,
    "SURROGATE": 6,
    "OUTPUT_TOO_SMALL": 16,
}
KIND_NAMES = {v: k for k, v in KINDS.items()}


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("count", ctypes.c_uint64)]

    def as_tuple(self):
        return (KIND_NAMES[self.status], int(self.count))


_lock = threading.Lock()
_default = None


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/_build/libgbu_oracle.so`` (skipped when up to date)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-fPIC", "-shared", _SRC, "-o", tmp]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a)
    assert a.dtype == np.uint8, a.dtype
    return a


def _u16(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(a), dtype="<u2")
    a = np.ascontiguousarray(a)
    assert a.dtype == np.uint16, a.dtype
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


class Codec:
    """The codec's functions over numpy arrays, bound to one loaded build of the C file
    (the default build, or any library exporting the same ``or_*`` symbols)."""

    def __init__(self, L: ctypes.CDLL):
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        for name in ("or_validate_utf8", "or_validate_utf16le"):
            getattr(L, name).restype = Result
            getattr(L, name).argtypes = [vp, sz]
        for name in ("or_utf16_length_from_utf8", "or_utf8_length_from_utf16le"):
            getattr(L, name).restype = ctypes.c_uint64
            getattr(L, name).argtypes = [vp, sz]
        for name in ("or_convert_utf8_to_utf16le", "or_convert_utf16le_to_utf8"):
            getattr(L, name).restype = Result
            getattr(L, name).argtypes = [vp, sz, vp, sz]
        L.or_validate_utf16be.restype = Result
        L.or_validate_utf16be.argtypes = [vp, sz]
        L.or_utf8_length_from_utf16be.restype = ctypes.c_uint64
        L.or_utf8_length_from_utf16be.argtypes = [vp, sz]
        for name in ("or_convert_utf16be_to_utf8", "or_convert_utf8_to_utf16be"):
            getattr(L, name).restype = Result
            getattr(L, name).argtypes = [vp, sz, vp, sz]
        L.or_validate_utf32.restype = Result
        L.or_validate_utf32.argtypes = [vp, sz]
        for name in ("or_utf8_length_from_utf32", "or_utf32_length_from_utf8"):
            getattr(L, name).restype = ctypes.c_uint64
            getattr(L, name).argtypes = [vp, sz]
        for name in ("or_utf16_length_from_utf32", "or_utf32_length_from_utf16le"):
            getattr(L, name).restype = ctypes.c_uint64
            getattr(L, name).argtypes = [vp, sz]
        for name in ("or_convert_utf32_to_utf8", "or_convert_utf8_to_utf32", "or_convert_utf32_to_utf16le",
                     "or_convert_utf16le_to_utf32"):
            getattr(L, name).restype = Result
            getattr(L, name).argtypes = [vp, sz, vp, sz]
        for name in ("or_validate_utf8_batched", "or_validate_utf16le_batched"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [vp, vp, sz, vp]
        for name in ("or_convert_utf8_to_utf16le_batched", "or_convert_utf16le_to_utf8_batched"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [vp, vp, sz, vp, vp, vp]
        self.lib = L

    def validate_utf8(self, src):
        a = _u8(src)
        return self.lib.or_validate_utf8(_ptr(a), a.size).as_tuple()

    def validate_utf16le(self, src):
        a = _u16(src)
        return self.lib.or_validate_utf16le(_ptr(a), a.size).as_tuple()

    def utf16_length_from_utf8(self, src) -> int:
        a = _u8(src)
        return int(self.lib.or_utf16_length_from_utf8(_ptr(a), a.size))

    def utf8_length_from_utf16le(self, src) -> int:
        a = _u16(src)
        return int(self.lib.or_utf8_length_from_utf16le(_ptr(a), a.size))

    def convert_utf8_to_utf16le(self, src, cap=None):
        """Returns ((kind, count), dst); dst has ``cap`` words (default: the length formula)."""
        a = _u8(src)
        if cap is None:
            cap = self.utf16_length_from_utf8(a)
        dst = np.zeros(cap, dtype=np.uint16)
        r = self.lib.or_convert_utf8_to_utf16le(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    def convert_utf16le_to_utf8(self, src, cap=None):
        """Returns ((kind, count), dst); dst has ``cap`` bytes (default: the length formula)."""
        a = _u16(src)
        if cap is None:
            cap = self.utf8_length_from_utf16le(a)
        dst = np.zeros(cap, dtype=np.uint8)
        r = self.lib.or_convert_utf16le_to_utf8(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    # UTF-16BE: uint16 arrays holding the words as they lie in memory (big-endian bytes), e.g.
    # a little-endian word array after .byteswap()
    def validate_utf16be(self, src):
        a = _u16(src)
        return self.lib.or_validate_utf16be(_ptr(a), a.size).as_tuple()

    def utf8_length_from_utf16be(self, src) -> int:
        a = _u16(src)
        return int(self.lib.or_utf8_length_from_utf16be(_ptr(a), a.size))

    def convert_utf16be_to_utf8(self, src, cap=None):
        a = _u16(src)
        if cap is None:
            cap = self.utf8_length_from_utf16be(a)
        dst = np.zeros(cap, dtype=np.uint8)
        r = self.lib.or_convert_utf16be_to_utf8(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    def convert_utf8_to_utf16be(self, src, cap=None):
        a = _u8(src)
        if cap is None:
            cap = self.utf16_length_from_utf8(a)
        dst = np.zeros(cap, dtype=np.uint16)
        r = self.lib.or_convert_utf8_to_utf16be(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    # UTF-32: uint32 arrays of units (host byte order)
    def validate_utf32(self, src):
        a = np.ascontiguousarray(src, dtype=np.uint32)
        return self.lib.or_validate_utf32(_ptr(a), a.size).as_tuple()

    def utf8_length_from_utf32(self, src) -> int:
        a = np.ascontiguousarray(src, dtype=np.uint32)
        return int(self.lib.or_utf8_length_from_utf32(_ptr(a), a.size))

    def utf32_length_from_utf8(self, src) -> int:
        a = _u8(src)
        return int(self.lib.or_utf32_length_from_utf8(_ptr(a), a.size))

    def convert_utf32_to_utf8(self, src, cap=None):
        a = np.ascontiguousarray(src, dtype=np.uint32)
        if cap is None:
            cap = self.utf8_length_from_utf32(a)
        dst = np.zeros(cap, dtype=np.uint8)
        r = self.lib.or_convert_utf32_to_utf8(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    def convert_utf8_to_utf32(self, src, cap=None):
        a = _u8(src)
        if cap is None:
            cap = self.utf32_length_from_utf8(a)
        dst = np.zeros(cap, dtype=np.uint32)
        r = self.lib.or_convert_utf8_to_utf32(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    def utf16_length_from_utf32(self, src) -> int:
        a = np.ascontiguousarray(src, dtype=np.uint32)
        return int(self.lib.or_utf16_length_from_utf32(_ptr(a), a.size))

    def utf32_length_from_utf16le(self, src) -> int:
        a = _u16(src)
        return int(self.lib.or_utf32_length_from_utf16le(_ptr(a), a.size))

    def convert_utf32_to_utf16le(self, src, cap=None):
        a = np.ascontiguousarray(src, dtype=np.uint32)
        if cap is None:
            cap = self.utf16_length_from_utf32(a)
        dst = np.zeros(cap, dtype=np.uint16)
        r = self.lib.or_convert_utf32_to_utf16le(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    def convert_utf16le_to_utf32(self, src, cap=None):
        a = _u16(src)
        if cap is None:
            cap = self.utf32_length_from_utf16le(a)
        dst = np.zeros(cap, dtype=np.uint32)
        r = self.lib.or_convert_utf16le_to_utf32(_ptr(a), a.size, _ptr(dst), cap)
        return r.as_tuple(), dst

    def validate_utf8_batched(self, src, off):
        a, o = _u8(src), np.ascontiguousarray(off, dtype=np.uint64)
        B = o.size - 1
        res = (Result * max(B, 1))()
        self.lib.or_validate_utf8_batched(_ptr(a), _ptr(o), B, res)
        return [res[i].as_tuple() for i in range(B)]

    def validate_utf16le_batched(self, src, off):
        a, o = _u16(src), np.ascontiguousarray(off, dtype=np.uint64)
        B = o.size - 1
        res = (Result * max(B, 1))()
        self.lib.or_validate_utf16le_batched(_ptr(a), _ptr(o), B, res)
        return [res[i].as_tuple() for i in range(B)]

    def convert_utf8_to_utf16le_batched(self, src, off, dst_off):
        a, o = _u8(src), np.ascontiguousarray(off, dtype=np.uint64)
        d = np.ascontiguousarray(dst_off, dtype=np.uint64)
        B = o.size - 1
        dst = np.zeros(int(d[-1]) if d.size else 0, dtype=np.uint16)
        res = (Result * max(B, 1))()
        self.lib.or_convert_utf8_to_utf16le_batched(_ptr(a), _ptr(o), B, _ptr(dst), _ptr(d), res)
        return [res[i].as_tuple() for i in range(B)], dst

    def convert_utf16le_to_utf8_batched(self, src, off, dst_off):
        a, o = _u16(src), np.ascontiguousarray(off, dtype=np.uint64)
        d = np.ascontiguousarray(dst_off, dtype=np.uint64)
        B = o.size - 1
        dst = np.zeros(int(d[-1]) if d.size else 0, dtype=np.uint8)
        res = (Result * max(B, 1))()
        self.lib.or_convert_utf16le_to_utf8_batched(_ptr(a), _ptr(o), B, _ptr(dst), _ptr(d), res)
        return [res[i].as_tuple() for i in range(B)], dst


def default() -> Codec:
    """The codec built from ``oracle/gbu_oracle.c``."""
    global _default
    with _lock:
        if _default is None:
            _default = Codec(ctypes.CDLL(build()))
    return _default


def validate_utf8(src):
    return default().validate_utf8(src)


def validate_utf16le(src):
    return default().validate_utf16le(src)


def utf16_length_from_utf8(src) -> int:
    return default().utf16_length_from_utf8(src)


def utf8_length_from_utf16le(src) -> int:
    return default().utf8_length_from_utf16le(src)


def convert_utf8_to_utf16le(src, cap=None):
    return default().convert_utf8_to_utf16le(src, cap)


def convert_utf16le_to_utf8(src, cap=None):
    return default().convert_utf16le_to_utf8(src, cap)


def validate_utf8_batched(src, off):
    return default().validate_utf8_batched(src, off)


def validate_utf16le_batched(src, off):
    return default().validate_utf16le_batched(src, off)


def convert_utf8_to_utf16le_batched(src, off, dst_off):
    return default().convert_utf8_to_utf16le_batched(src, off, dst_off)


def convert_utf16le_to_utf8_batched(src, off, dst_off):
    return default().convert_utf16le_to_utf8_batched(src, off, dst_off)


def validate_utf16be(src):
    return default().validate_utf16be(src)


def utf8_length_from_utf16be(src) -> int:
    return default().utf8_length_from_utf16be(src)


def convert_utf16be_to_utf8(src, cap=None):
    return default().convert_utf16be_to_utf8(src, cap)


def convert_utf8_to_utf16be(src, cap=None):
    return default().convert_utf8_to_utf16be(src, cap)


def validate_utf32(src):
    return default().validate_utf32(src)


def utf8_length_from_utf32(src) -> int:
    return default().utf8_length_from_utf32(src)


def utf32_length_from_utf8(src) -> int:
    return default().utf32_length_from_utf8(src)


def convert_utf32_to_utf8(src, cap=None):
    return default().convert_utf32_to_utf8(src, cap)


def convert_utf8_to_utf32(src, cap=None):
    return default().convert_utf8_to_utf32(src, cap)


def utf16_length_from_utf32(src) -> int:
    return default().utf16_length_from_utf32(src)


def utf32_length_from_utf16le(src) -> int:
    return default().utf32_length_from_utf16le(src)


def convert_utf32_to_utf16le(src, cap=None):
    return default().convert_utf32_to_utf16le(src, cap)


def convert_utf16le_to_utf32(src, cap=None):
    return default().convert_utf16le_to_utf32(src, cap)
