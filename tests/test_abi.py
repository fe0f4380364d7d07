"""CPU checks of the C ABI library: it builds, loads, and exports every entry point that
include/*.h declares; the product code never reaches the reference codec."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gbu_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2111_08692_gb300.build import build
    path = build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gbu_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, sorted(declared - exported)


def test_library_loads_with_ctypes():
    import paper_2111_08692_gb300 as g
    L = g.lib()
    for name in _declared():
        assert hasattr(L, name)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2111_08692_gb300.binding as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b._build, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        b.lib()


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2111_08692_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
            assert "gbu_oracle" not in text, f


_HANDLES = r"(?:const\s+)?(?:gbu_ctx|gbu_chunked|gbu_server|gbu_arena|gbu_graph)\s*\*"


def _int_entry_points_taking_a_handle():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\bint\s+(gbu_[a-z0-9_]+)\s*\(\s*" + _HANDLES, text):
            names.add(m.group(1))
    names.discard("gbu_launch_config")  # returns the number of values written (0 for NULL)
    return sorted(names)


def _placeholder(t):
    # pointers NULL; counts, sizes and ops 1 (so that "n > 0 with a NULL pointer" applies too)
    import ctypes
    if t is ctypes.c_void_p or isinstance(t, type(ctypes.POINTER(ctypes.c_int))):
        return None
    return 1


def test_null_handles_are_bad_arguments_without_a_launch():
    """Every int entry point that takes a context, resumable stream, server, arena or graph
    rejects a NULL one with GBU_BAD_ARGUMENT before touching a device (the header's argument
    rule), and the binding declares the argument types of each."""
    import paper_2111_08692_gb300 as g
    L = g.lib()
    names = _int_entry_points_taking_a_handle()
    assert len(names) >= 40, names
    for name in names:
        f = getattr(L, name)
        assert f.argtypes, name + " has no argtypes in the binding"
        rc = f(*[_placeholder(t) for t in f.argtypes])
        want = -17 if name == "gbu_server_poll" else 17  # poll returns a count, or minus a status
        assert rc == want, (name, rc)


def test_null_safe_queries_and_argument_checks_before_the_device():
    import paper_2111_08692_gb300 as g
    L = g.lib()
    assert L.gbu_launch_count(None) == 0
    assert L.gbu_launch_config(None, None, 0) == 0
    assert L.gbu_graph_kernels(None) == 0
    assert L.gbu_server_now_ns(None) == 0
    assert L.gbu_arena_used(None) == 0 and L.gbu_arena_largest_free(None) == 0
    for destroy in ("gbu_destroy", "gbu_chunked_destroy", "gbu_server_destroy", "gbu_graph_destroy",
                    "gbu_arena_destroy"):
        getattr(L, destroy)(None)  # a NULL handle is ignored
    # the allocation-free transcoder checks its size and pointers before its device setup
    assert L.gbu_convert_utf8_to_utf16le_noalloc(None, 16, None, 0, None, None) == 17
    assert L.gbu_convert_utf8_to_utf16le_noalloc(None, (1 << 28) + 1, None, 0, None, None) == 20
    # a resumable stream with an unknown operation or no chunk size is refused before any device call
    assert not L.gbu_chunked_create(0, 99, 1024)
    assert not L.gbu_chunked_create(0, 0, 0)
    # the host-side cut and combination functions check their arguments
    assert L.gbu_shard_cuts_utf8_host(None, 0, 0, None) == 17
    assert L.gbu_combine_shards(None, None, 0, None) == 17


def test_create_without_a_device_returns_null():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2111_08692_gb300 as g
    L = g.lib()
    assert not L.gbu_create(0, 1 << 20)
    assert not L.gbu_chunked_create(0, 0, 1024)


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++11")])
def test_header_is_plain_c(lang, std):
    """include/gbutf.h needs no CUDA or torch header: it compiles on its own as strict C99 and
    as C++11 (streams are opaque pointers, results plain structs)."""
    import shutil
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = ('#include "gbutf.h"\n'
           'typedef char gbu_result_is_16_bytes[sizeof(gbu_result) == 16 ? 1 : -1];\n'
           'int main(void) { return 0; }\n')
    subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only", "-x", lang,
                    "-I", os.path.join(ROOT, "include"), "-"], input=src, text=True, check=True,
                   capture_output=True)


def test_kernel_hash_ignores_comments_only():
    """The hash that ties an ncu capture to a kernel's sources ignores comments and whitespace, and
    nothing else: comment markers inside string and character literals are kept."""
    from paper_2111_08692_gb300 import build as b
    src = 'int f(int a) { // one\n  /* two\n three */ return a + 1; }\nconst char *s = "a // b /* c */";\nchar q = \'"\';\n'
    edited = src.replace("// one", "// a longer comment").replace("two", "four") + "\n\n// trailing\n"
    assert b.strip_comments(src) == b.strip_comments(edited)
    assert '"a//b/*c*/"' in b.strip_comments(src) and "'\"'" in b.strip_comments(src)
    assert b.strip_comments(src) != b.strip_comments(src.replace("a + 1", "a + 2"))
    for op in b.KERNEL_SOURCES:
        h = b.kernel_hash(op)
        assert len(h) == 12 and int(h, 16) >= 0 and h == b.kernel_hash(op)


def test_sync_forms_return_bad_argument_by_value_for_a_null_context():
    """The six host-synchronising calls return their gbu_result by value; a NULL context gives
    {GBU_BAD_ARGUMENT, 0} before any device call."""
    import paper_2111_08692_gb300 as g
    L = g.lib()
    for name in ("gbu_validate_utf8_sync", "gbu_validate_utf16le_sync", "gbu_utf16_length_from_utf8_sync",
                 "gbu_utf8_length_from_utf16le_sync"):
        r = getattr(L, name)(None, None, 0, None)
        assert (r.status, r.reserved, r.count) == (17, 0, 0), name
    for name in ("gbu_convert_utf8_to_utf16le_sync", "gbu_convert_utf16le_to_utf8_sync"):
        r = getattr(L, name)(None, None, 0, None, 0, None)
        assert (r.status, r.reserved, r.count) == (17, 0, 0), name


def test_pipe_refuses_bad_arguments_before_the_device():
    """The host-buffer form: a NULL pipe or result is GBU_BAD_ARGUMENT, a NULL pipe handle is
    ignored by destroy, and creation refuses a piece below 4096 units or a stream count outside
    1..8 before any device call (and returns NULL without a device)."""
    import torch
    import paper_2111_08692_gb300 as g
    L = g.lib()
    res = g.GbuResult()
    for name in ("gbu_pipe_validate_utf8", "gbu_pipe_validate_utf16le", "gbu_pipe_utf16_length_from_utf8",
                 "gbu_pipe_utf8_length_from_utf16le"):
        assert getattr(L, name)(None, None, 0, ctypes.byref(res)) == 17, name
    for name in ("gbu_pipe_convert_utf8_to_utf16le", "gbu_pipe_convert_utf16le_to_utf8"):
        assert getattr(L, name)(None, None, 0, None, 0, ctypes.byref(res)) == 17, name
    L.gbu_pipe_destroy(None)
    assert not L.gbu_pipe_create(0, 4095, 1)
    assert not L.gbu_pipe_create(0, 4096, 9)
    assert not L.gbu_pipe_create(0, 4096, -1)
    if not torch.cuda.is_available():
        assert not L.gbu_pipe_create(0, 0, 0)
