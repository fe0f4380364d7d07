"""Builds and loads tests/helpers/bruteforce.c linked with a copy of the reference codec.

Test infrastructure: used by the oracle pin tests and the mutation test only.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HELPER = os.path.join(ROOT, "tests", "helpers", "bruteforce.c")
ORACLE_SRC = os.path.join(ROOT, "oracle", "gbu_oracle.c")
ORACLE_DIR = os.path.join(ROOT, "oracle")
BUILD = os.path.join(ROOT, "tests", "_build")


def build(oracle_source: str | None = None) -> str:
    """Compiles helper + oracle (or the given oracle source text) into a shared library."""
    os.makedirs(BUILD, exist_ok=True)
    src_text = oracle_source if oracle_source is not None else open(ORACLE_SRC).read()
    helper_text = open(HELPER).read()
    hdr_text = open(os.path.join(ORACLE_DIR, "gbu_oracle.h")).read()
    key = hashlib.sha1((src_text + helper_text + hdr_text).encode()).hexdigest()[:16]
    so = os.path.join(BUILD, f"libbf_{key}.so")
    if not os.path.exists(so):
        osrc = os.path.join(BUILD, f"oracle_{key}.c")
        with open(osrc, "w") as f:
            f.write(src_text)
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-pthread", "-I", ORACLE_DIR,
             HELPER, osrc, "-o", tmp]
        )
        os.replace(tmp, so)
    return so


class BF:
    """ctypes view of one build of the helper (the oracle's own symbols are exported too)."""

    def __init__(self, so_path: str):
        self.lib = L = ctypes.CDLL(so_path)
        L.bf_utf8.restype = ctypes.c_long
        L.bf_utf8.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.bf_table.restype = None
        L.bf_table.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.bf_utf16_pairs.restype = ctypes.c_long
        L.bf_utf16_pairs.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.bf_mixed_dead_prefixes.restype = ctypes.c_long
        L.bf_utf16_pair_table.restype = None
        L.bf_utf16_pair_table.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                          ctypes.c_void_p]

    def utf8(self, length: int, nthreads: int = 8, roundtrip: bool = True):
        stats = np.zeros(14, dtype=np.int64)
        m = self.lib.bf_utf8(length, nthreads, int(roundtrip), stats.ctypes.data)
        return int(m), stats

    def table(self, length: int):
        kind = np.zeros(1 << (8 * length), dtype=np.uint8)
        off = np.zeros(1 << (8 * length), dtype=np.uint8)
        self.lib.bf_table(length, kind.ctypes.data, off.ctypes.data)
        return kind, off

    def utf16_pairs(self, nthreads: int = 8):
        stats = np.zeros(2, dtype=np.int64)
        m = self.lib.bf_utf16_pairs(nthreads, stats.ctypes.data)
        return int(m), stats

    def mixed_dead_prefixes(self) -> int:
        return int(self.lib.bf_mixed_dead_prefixes())

    def utf16_pair_table(self, words: np.ndarray):
        w = np.ascontiguousarray(words, dtype=np.uint16)
        m = w.size
        kind = np.zeros(m * m, dtype=np.uint8)
        off = np.zeros(m * m, dtype=np.uint8)
        self.lib.bf_utf16_pair_table(w.ctypes.data, m, kind.ctypes.data, off.ctypes.data)
        return kind.reshape(m, m), off.reshape(m, m)
