"""Builds the CUDA library ``_lib/libgbutf.so`` in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked with ``nvcc -shared``.  Nothing is
rebuilt when the library is newer than every source and header.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_DIR = os.path.join(PKG, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libgbutf.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def sources_hash() -> str:
    """Short hash of the kernel sources and headers (ties profile summaries to a build)."""
    import hashlib
    h = hashlib.sha1()
    files = sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h")))
    for f in files:
        if os.path.isfile(f):
            h.update(os.path.basename(f).encode())
            h.update(open(f, "rb").read())
    return h.hexdigest()[:12]


# The sources each single-buffer kernel is compiled from (its device code), by operation.
_STREAM = ["gbu_stream.cu", "gbu_chunk.cuh", "gbu_device.cuh"]
KERNEL_SOURCES = {
    "validate_utf8": _STREAM, "utf16_length_from_utf8": _STREAM,
    "validate_utf16le": _STREAM, "utf8_length_from_utf16le": _STREAM,
    "convert_utf8_to_utf16le": ["gbu_utf8.cu", "gbu_wide_utf8.cuh", "gbu_wide.cuh", "gbu_codec_utf8.cuh",
                                "gbu_xcode.cuh", "gbu_chunk.cuh", "gbu_device.cuh"],
    "convert_utf16le_to_utf8": ["gbu_utf16.cu", "gbu_wide_utf16.cuh", "gbu_wide.cuh", "gbu_codec_utf16.cuh",
                                "gbu_xcode.cuh", "gbu_chunk.cuh", "gbu_device.cuh"],
}


def strip_comments(text: str) -> str:
    """C/C++ source without its comments and whitespace (comment markers inside string and
    character literals are kept), so that editing a comment or the layout does not change a
    kernel's hash."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = ["".join(ln.split()) for ln in "".join(out).splitlines()]
    return "\n".join(ln for ln in lines if ln)


def kernel_hash(op: str) -> str:
    """Short hash of the sources of the kernel behind single-buffer operation `op`, comments left
    out (ties an ncu capture of that kernel to the code it measured)."""
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SOURCES[op]:
        h.update(name.encode())
        h.update(strip_comments(open(os.path.join(CSRC, name)).read()).encode())
    return h.hexdigest()[:12]


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
