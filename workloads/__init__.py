"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the codec's arithmetic: code points are drawn with numpy's PCG64
generator, and every encoding (UTF-32 -> str -> UTF-8 / UTF-16LE) is done by CPython's own
codecs.  Error injection overwrites whole placeholder characters with byte templates; the
expected result of an injected input is never computed here (the tests ask the reference
codec).  The same seed gives the same bytes on every machine.

Profiles (per-character mixtures, drawn i.i.d.):
  mixed     50% U+0000-007F, 20% U+0080-07FF, 20% U+0800-FFFF minus D800-DFFF,
            10% U+10000-10FFFF
  ascii     printable ASCII U+0020-007E
  latin     95% printable ASCII, 5% U+00C0-017F
  cyrillic  70% U+0400-04FF, 30% ASCII space/punctuation (half U+0020, half one of the 32
            ASCII punctuation characters)
  cjk       85% U+4E00-9FFF, 15% printable ASCII
  emoji     70% printable ASCII, 30% U+1F300-1FAFF
Buffers are filled to an exact size: characters are appended while they fit, then the rest
is padded with U+0020.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

VERSION = "2"  # bump when any generator's output changes (invalidates the on-disk cache)

PROFILE_ORDER = ("ascii", "latin", "cyrillic", "cjk", "emoji")
PROFILE_SEEDS = {"ascii": 1, "latin": 2, "cyrillic": 3, "cjk": 4, "emoji": 5}
SWEEP_SEEDS = {("cyrillic", 1e-6): 11, ("cyrillic", 1e-4): 12, ("cyrillic", 1e-2): 13,
               ("cjk", 1e-6): 14, ("cjk", 1e-4): 15, ("cjk", 1e-2): 16}

_PUNCT = np.array([c for c in range(0x21, 0x7F) if not chr(c).isalnum()], dtype=np.uint32)
assert _PUNCT.size == 32

# (weight, kind, lo, hi), hi exclusive.  "range": uniform on [lo, hi); "bmp_nosurr": uniform
# on U+0800-FFFF minus D800-DFFF; "space_punct": half U+0020, half one of the punctuation.
_MIX = {
    "mixed": [(0.50, "range", 0x0000, 0x0080), (0.20, "range", 0x0080, 0x0800),
              (0.20, "bmp_nosurr", 0, 0), (0.10, "range", 0x10000, 0x110000)],
    "ascii": [(1.00, "range", 0x20, 0x7F)],
    "latin": [(0.95, "range", 0x20, 0x7F), (0.05, "range", 0xC0, 0x180)],
    "cyrillic": [(0.70, "range", 0x0400, 0x0500), (0.30, "space_punct", 0, 0)],
    "cjk": [(0.85, "range", 0x4E00, 0xA000), (0.15, "range", 0x20, 0x7F)],
    "emoji": [(0.70, "range", 0x20, 0x7F), (0.30, "range", 0x1F300, 0x1FB00)],
}
PROFILES = tuple(_MIX)
# a non-ASCII range of each profile, used to build truncated sequences
_WIDE_RANGE = {"latin": (0xC0, 0x180), "cyrillic": (0x400, 0x500), "cjk": (0x4E00, 0xA000),
               "emoji": (0x1F300, 0x1FB00), "mixed": (0x800, 0xD800), "ascii": (0x80, 0x800)}

PLACEHOLDER_8 = 0xF0000   # plane-15 private use: its UTF-8 form starts with byte F3
PLACEHOLDER_16 = 0xE000   # BMP private use: one UTF-16 word E000


def _draw_component(comp, m, rng):
    _w, kind, lo, hi = comp
    if kind == "range":
        return rng.integers(lo, hi, size=m, dtype=np.uint32)
    if kind == "bmp_nosurr":
        v = rng.integers(0x800, 0x10000 - 0x800, size=m, dtype=np.uint32)
        return np.where(v >= 0xD800, v + 0x800, v).astype(np.uint32)
    half = rng.random(m) < 0.5  # space_punct
    return np.where(half, np.uint32(0x20), _PUNCT[rng.integers(0, 32, size=m)]).astype(np.uint32)


def draw_codepoints(profile: str, count: int, rng: np.random.Generator) -> np.ndarray:
    """`count` code points of `profile`, as uint32.  A uniform draw u per position picks the
    component whose cumulative-weight interval holds u; every component is drawn for every
    position and the picks are merged (vectorised, and independent of the order of the
    components' values)."""
    mix = _MIX[profile]
    if len(mix) == 1:
        return _draw_component(mix[0], count, rng)
    u = rng.random(count)
    cum = np.cumsum([w for w, *_ in mix])
    cum = cum / cum[-1]
    out = _draw_component(mix[-1], count, rng)
    for k in range(len(mix) - 2, -1, -1):
        np.copyto(out, _draw_component(mix[k], count, rng), where=u < cum[k])
    return out


def to_str(cps: np.ndarray) -> str:
    return np.ascontiguousarray(cps, dtype="<u4").tobytes().decode("utf-32-le")


def encode_utf8(cps: np.ndarray) -> np.ndarray:
    return np.frombuffer(to_str(cps).encode("utf-8"), dtype=np.uint8)


def encode_utf16le(cps: np.ndarray) -> np.ndarray:
    return np.frombuffer(to_str(cps).encode("utf-16-le"), dtype=np.uint16)


class _Filler:
    """Appends encoded chunks until a byte budget is met: the first character that does not
    fit ends the fill and the remaining budget is padded with U+0020."""

    def __init__(self, enc: str, budget_bytes: int):
        self.enc, self.left, self.parts = enc, budget_bytes, []

    @property
    def done(self):
        return self.left == 0

    def feed(self, s: str):
        if self.left == 0:
            return
        b = s.encode(self.enc)
        if len(b) > self.left:
            # CPython drops the character cut at the budget (its 'ignore' error handler)
            b = b[: self.left].decode(self.enc, errors="ignore").encode(self.enc)
            self.parts.append(b)
            self.left -= len(b)
            self.parts.append(" ".encode(self.enc) * (self.left // len(" ".encode(self.enc))))
            self.left = 0
        else:
            self.parts.append(b)
            self.left -= len(b)

    def result(self, dtype) -> np.ndarray:
        return np.frombuffer(b"".join(self.parts), dtype=dtype)


def _fill_buffers(profile, n8, n16, rng, chunk_chars=1 << 22, transform=None):
    f8 = _Filler("utf-8", n8) if n8 is not None else None
    f16 = _Filler("utf-16-le", 2 * n16) if n16 is not None else None
    while (f8 and not f8.done) or (f16 and not f16.done):
        cps = draw_codepoints(profile, chunk_chars, rng)
        if transform is not None:
            cps = transform(cps)
        s = to_str(cps)
        if f8:
            f8.feed(s)
        if f16:
            f16.feed(s)
    u8 = f8.result(np.uint8) if f8 else None
    u16 = f16.result(np.uint16) if f16 else None
    return u8, u16


# ---- on-disk cache (large buffers are slow to draw in Python) ------------------------------

def cache_dir() -> str:
    d = os.environ.get("GBU_WORKLOAD_CACHE", os.path.join("/tmp", "gbu_workloads"))
    os.makedirs(d, exist_ok=True)
    return d


def _cache_path(key: str) -> str:
    h = hashlib.sha1((VERSION + key).encode()).hexdigest()[:20]
    return os.path.join(cache_dir(), h)


def _cached(key: str, make, mmap: bool = False):
    """make() -> dict of numpy arrays, cached as one directory of .npy files per key (loaded
    memory-mapped when mmap is true)."""
    path = _cache_path(key)
    done = os.path.join(path, "DONE")
    if os.path.exists(done):
        try:
            names = [f[:-4] for f in os.listdir(path) if f.endswith(".npy")]
            return {k: np.load(os.path.join(path, k + ".npy"), mmap_mode="r" if mmap else None)
                    for k in names}
        except Exception:
            pass
    out = make()
    tmp = path + f".tmp{os.getpid()}"
    os.makedirs(tmp, exist_ok=True)
    for k, v in out.items():
        np.save(os.path.join(tmp, k + ".npy"), v)
    open(os.path.join(tmp, "DONE"), "w").close()
    try:
        os.rename(tmp, path)
    except OSError:  # another process made it first
        pass
    return out


# ---- single-buffer workloads -----------------------------------------------------------------

def profile_buffers(profile: str, n_utf8_bytes: int, n_utf16_units: int, seed: int,
                    cache: bool = True, mmap: bool = False):
    """One UTF-8 buffer of exactly n_utf8_bytes and one UTF-16LE buffer of exactly
    n_utf16_units, both prefixes of the same seeded character stream."""
    def make():
        u8, u16 = _fill_buffers(profile, n_utf8_bytes, n_utf16_units, np.random.default_rng(seed))
        return {"u8": u8, "u16": u16}
    if cache and n_utf8_bytes + 2 * n_utf16_units >= (1 << 24):
        d = _cached(f"profile:{profile}:{n_utf8_bytes}:{n_utf16_units}:{seed}", make, mmap=mmap)
    else:
        d = make()
    assert d["u8"].size == n_utf8_bytes and d["u16"].size == n_utf16_units
    return d["u8"], d["u16"]


def single_buffer_1gib(profile: str, scale: int = 1 << 30, mmap: bool = False):
    """The 1 GiB workload of one profile: 2^30 UTF-8 bytes and 2^29 UTF-16 words (scale sets
    the UTF-8 byte count; the UTF-16 buffer has scale/2 words, the same number of bytes)."""
    return profile_buffers(profile, scale, scale // 2, PROFILE_SEEDS[profile], mmap=mmap)


def _make_one(args):
    profile, scale = args
    single_buffer_1gib(profile, scale, mmap=True)
    return profile


def prepare_single_buffers(profiles=PROFILE_ORDER, scale: int = 1 << 30, workers: int | None = None):
    """Generates (into the on-disk cache) the single-buffer workloads of several profiles in
    parallel worker processes.  The pool uses the 'spawn' start method, so it is safe to call
    from a process that already uses CUDA."""
    import concurrent.futures as cf
    import multiprocessing as mp
    todo = [p for p in profiles
            if not os.path.exists(os.path.join(_cache_path(
                f"profile:{p}:{scale}:{scale // 2}:{PROFILE_SEEDS[p]}"), "DONE"))]
    if len(todo) <= 1 or (workers or os.cpu_count() or 1) <= 1:
        for p in todo:
            _make_one((p, scale))
        return
    with cf.ProcessPoolExecutor(max_workers=min(len(todo), workers or os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_make_one, [(p, scale) for p in todo]))


def mixed_1mib(seed: int = 0, n: int = 1 << 20):
    """The 1 MiB mixed-profile UTF-8 buffer, its UTF-16LE form (CPython's encoding of the same
    characters), and a copy with one byte XOR 0xFF at a seeded offset.  Returns
    (u8, u16, flipped, flip_offset)."""
    rng = np.random.default_rng(seed)
    u8, _ = _fill_buffers("mixed", n, None, rng, chunk_chars=1 << 16)
    u16 = np.frombuffer(u8.tobytes().decode("utf-8").encode("utf-16-le"), dtype=np.uint16)
    o = int(rng.integers(0, n))
    flipped = u8.copy()
    flipped[o] ^= 0xFF
    return u8, u16, flipped, o


# ---- error injection -------------------------------------------------------------------------

UTF8_ERROR_KINDS = ("overlong", "surrogate", "too_large", "stray_continuation", "truncated")
UTF16_ERROR_KINDS = ("lone_high", "lone_low")


def _wide_chars_utf8(profile, m, rng):
    """m random non-ASCII characters of the profile, CPython-encoded, as an (m, L) array."""
    lo, hi = _WIDE_RANGE[profile]
    cps = rng.integers(lo, hi, size=m, dtype=np.uint32)
    b = encode_utf8(cps)
    L = b.size // max(m, 1)
    assert m == 0 or L * m == b.size, "profile's wide range must have one encoded length"
    return b.reshape(m, L) if m else np.zeros((0, 1), np.uint8)


def utf8_error_templates(kinds: np.ndarray, profile: str, rng: np.random.Generator) -> np.ndarray:
    """A 4-byte template per entry of `kinds` (indices into UTF8_ERROR_KINDS), padded with
    U+0020:
      overlong            C0/C1 + continuation (an ASCII character in two bytes), or
                          E0 80-9F + continuation, or F0 80-8F + two continuations
      surrogate           ED A0-BF + continuation
      too_large           F4 90-BF + two continuations, or F5-F7 + three continuations
      stray_continuation  one byte 80-BF
      truncated           a multi-byte character of the profile without its last byte
    """
    m = kinds.size
    t = np.full((m, 4), 0x20, dtype=np.uint8)
    c = lambda lo, hi, k: rng.integers(lo, hi, size=k).astype(np.uint8)  # noqa: E731
    for ki, name in enumerate(UTF8_ERROR_KINDS):
        idx = np.flatnonzero(kinds == ki)
        k = idx.size
        if k == 0:
            continue
        if name == "overlong":
            form = rng.integers(0, 3, size=k)
            ch = rng.integers(0x00, 0x80, size=k)
            row = np.full((k, 4), 0x20, dtype=np.uint8)
            f0, f1, f2 = form == 0, form == 1, form == 2
            row[f0, 0] = (0xC0 | (ch[f0] >> 6)).astype(np.uint8)
            row[f0, 1] = (0x80 | (ch[f0] & 0x3F)).astype(np.uint8)
            row[f1, 0] = 0xE0
            row[f1, 1] = c(0x80, 0xA0, int(f1.sum()))
            row[f1, 2] = c(0x80, 0xC0, int(f1.sum()))
            row[f2, 0] = 0xF0
            row[f2, 1] = c(0x80, 0x90, int(f2.sum()))
            row[f2, 2] = c(0x80, 0xC0, int(f2.sum()))
            row[f2, 3] = c(0x80, 0xC0, int(f2.sum()))
            t[idx] = row
        elif name == "surrogate":
            t[idx, 0] = 0xED
            t[idx, 1] = c(0xA0, 0xC0, k)
            t[idx, 2] = c(0x80, 0xC0, k)
        elif name == "too_large":
            form = rng.integers(0, 2, size=k)
            row = np.empty((k, 4), dtype=np.uint8)
            row[:, 0] = np.where(form == 0, 0xF4, c(0xF5, 0xF8, k))
            row[:, 1] = np.where(form == 0, c(0x90, 0xC0, k), c(0x80, 0xC0, k))
            row[:, 2] = c(0x80, 0xC0, k)
            row[:, 3] = c(0x80, 0xC0, k)
            t[idx] = row
        elif name == "stray_continuation":
            t[idx, 0] = c(0x80, 0xC0, k)
        else:  # truncated
            w = _wide_chars_utf8(profile, k, rng)
            t[idx, : w.shape[1] - 1] = w[:, :-1]
    return t


def sweep_buffers(profile: str, rate: float, n_bytes: int = 256 << 20, seed: int | None = None,
                  cache: bool = True):
    """The invalid-input sweep: a UTF-8 buffer of n_bytes and a UTF-16LE buffer of n_bytes/2
    words of `profile` (cyrillic or cjk), where each character is independently replaced,
    with probability `rate`, by an error: a UTF-8 template (kinds drawn uniformly from
    UTF8_ERROR_KINDS) or, in UTF-16, a lone high or low surrogate word.  Also returns the
    siblings whose final character is cut at the buffer end: UTF-8 ends with a multi-byte
    character missing its last byte, UTF-16 ends with a high surrogate.
    Returns dict(u8, u16, u8_cut_end, u16_cut_end)."""
    if seed is None:
        seed = SWEEP_SEEDS[(profile, rate)]

    def make():
        rng = np.random.default_rng(seed)

        def mark(cps, placeholder):
            hit = rng.random(cps.size) < rate
            cps = cps.copy()
            cps[hit] = placeholder
            return cps

        u8, _ = _fill_buffers(profile, n_bytes, None, rng, transform=lambda x: mark(x, PLACEHOLDER_8))
        u8 = u8.copy()
        pos = np.flatnonzero(u8 == 0xF3)  # the placeholder's first byte; absent otherwise
        kinds = rng.integers(0, len(UTF8_ERROR_KINDS), size=pos.size)
        tmpl = utf8_error_templates(kinds, profile, rng)
        for j in range(4):
            u8[pos + j] = tmpl[:, j]
        _, u16 = _fill_buffers(profile, None, n_bytes // 2, rng,
                               transform=lambda x: mark(x, PLACEHOLDER_16))
        u16 = u16.copy()
        pos16 = np.flatnonzero(u16 == PLACEHOLDER_16)
        hi = rng.random(pos16.size) < 0.5
        u16[pos16] = np.where(hi, rng.integers(0xD800, 0xDC00, size=pos16.size),
                              rng.integers(0xDC00, 0xE000, size=pos16.size)).astype(np.uint16)
        # siblings cut at the end
        w = _wide_chars_utf8(profile, 1, rng)[0]
        cut = w[:-1]
        u8c, _ = _fill_buffers(profile, n_bytes - cut.size, None, np.random.default_rng(seed))
        u8c = np.concatenate([u8c, cut])
        _, u16c = _fill_buffers(profile, None, n_bytes // 2 - 1, np.random.default_rng(seed))
        u16c = np.concatenate([u16c, np.array([rng.integers(0xD800, 0xDC00)], dtype=np.uint16)])
        return {"u8": u8, "u16": u16, "u8_cut_end": u8c, "u16_cut_end": u16c}

    if cache and n_bytes >= (1 << 24):
        return _cached(f"sweep:{profile}:{rate}:{n_bytes}:{seed}", make)
    return make()


SWEEP_PROFILES = ("cyrillic", "cjk")
SWEEP_RATES = (1e-6, 1e-4, 1e-2)


def _make_sweep(args):
    profile, rate, n_bytes = args
    sweep_buffers(profile, rate, n_bytes)
    return profile, rate


def prepare_sweeps(n_bytes: int = 256 << 20, workers: int | None = None):
    """Generates (into the on-disk cache) the six sweep workloads (two profiles x three error
    rates) in parallel 'spawn' worker processes, like prepare_single_buffers."""
    import concurrent.futures as cf
    import multiprocessing as mp
    todo = [(p, r, n_bytes) for p in SWEEP_PROFILES for r in SWEEP_RATES
            if not os.path.exists(os.path.join(_cache_path(f"sweep:{p}:{r}:{n_bytes}:{SWEEP_SEEDS[(p, r)]}"),
                                               "DONE"))]
    if len(todo) <= 1 or (workers or os.cpu_count() or 1) <= 1 or n_bytes < (1 << 24):
        for t in todo:
            _make_sweep(t)
        return
    with cf.ProcessPoolExecutor(max_workers=min(len(todo), workers or os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_make_sweep, todo))


# ---- batched strings --------------------------------------------------------------------------

def _char_sizes(cps: np.ndarray):
    """UTF-8 bytes and UTF-16 words of each code point, looked up from CPython's encodings of
    every code point in the ranges that occur."""
    u = np.unique(cps)
    s = to_str(u)
    b8 = np.array([len(ch.encode("utf-8")) for ch in s], dtype=np.int64)
    b16 = np.array([len(ch.encode("utf-16-le")) // 2 for ch in s], dtype=np.int64)
    idx = np.searchsorted(u, cps)
    return b8[idx], b16[idx]


def batched_strings(B: int = 1_000_000, seed: int = 1000, median: int = 64, sigma: float = 1.5,
                    max_len: int = 65536, error_fraction: float = 0.01, cache: bool = True):
    """B strings with log-normal UTF-8 byte lengths (median `median`, sigma `sigma`, clipped
    to 1..max_len), each of a profile drawn uniformly from the five profiles, each filled to
    its exact length with U+0020 padding.  The UTF-16LE strings hold the same characters.
    A fraction `error_fraction` of the strings get one injected error at a random character:
    in UTF-8 the character's bytes are replaced by an ill-formed sequence of the same length;
    in UTF-16 one word of a character is replaced by a lone surrogate.
    Returns dict(u8, off8, u16, off16, profile, err8, err16)."""

    def make():
        rng = np.random.default_rng(seed)
        lens = np.clip(np.rint(np.exp(np.log(median) + sigma * rng.standard_normal(B))), 1,
                       max_len).astype(np.int64)
        prof = rng.integers(0, len(PROFILE_ORDER), size=B)
        off8 = np.zeros(B + 1, dtype=np.int64)
        np.cumsum(lens, out=off8[1:])
        u8 = np.full(int(off8[-1]), 0x20, dtype=np.uint8)
        n16 = np.zeros(B, dtype=np.int64)
        chunks16 = [None] * B
        # per-string start (in characters) within its profile's stream, and the stream itself
        for p, name in enumerate(PROFILE_ORDER):
            sel = np.flatnonzero(prof == p)
            if sel.size == 0:
                continue
            L = lens[sel]
            start = np.zeros(sel.size + 1, dtype=np.int64)
            np.cumsum(L, out=start[1:])  # a string never needs more characters than bytes
            cps = draw_codepoints(name, int(start[-1]), rng)
            s8, s16 = _char_sizes(cps)
            c8 = np.zeros(cps.size + 1, dtype=np.int64)
            np.cumsum(s8, out=c8[1:])
            c16 = np.zeros(cps.size + 1, dtype=np.int64)
            np.cumsum(s16, out=c16[1:])
            # characters that fit: largest m with c8[start+m] - c8[start] <= L
            end = np.searchsorted(c8, c8[start[:-1]] + L, side="right") - 1
            end = np.minimum(end, start[1:])
            enc8 = encode_utf8(cps)
            enc16 = encode_utf16le(cps)
            for j, i in enumerate(sel):
                a, e = start[j], end[j]
                nb = c8[e] - c8[a]
                u8[off8[i]:off8[i] + nb] = enc8[c8[a]:c8[e]]
                pad = int(L[j] - nb)
                w = enc16[c16[a]:c16[e]]
                if pad:
                    w = np.concatenate([w, np.full(pad, 0x20, dtype=np.uint16)])
                chunks16[i] = w
                n16[i] = w.size
        off16 = np.zeros(B + 1, dtype=np.int64)
        np.cumsum(n16, out=off16[1:])
        u16 = np.concatenate(chunks16) if B else np.zeros(0, np.uint16)
        # error injection
        err8 = rng.random(B) < error_fraction
        err16 = rng.random(B) < error_fraction
        for i in np.flatnonzero(err8):
            seg = u8[off8[i]:off8[i + 1]]
            # character starts: CPython tells us where each character begins
            text = seg.tobytes().decode("utf-8")
            sizes = np.array([len(ch.encode("utf-8")) for ch in text], dtype=np.int64)
            starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
            k = int(rng.integers(0, sizes.size))
            seg[starts[k]:starts[k] + sizes[k]] = _same_length_error(int(sizes[k]), rng)
        for i in np.flatnonzero(err16):
            seg = u16[off16[i]:off16[i + 1]]
            text = seg.tobytes().decode("utf-16-le")
            sizes = np.array([len(ch.encode("utf-16-le")) // 2 for ch in text], dtype=np.int64)
            starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
            k = int(rng.integers(0, sizes.size))
            if sizes[k] == 1:  # a one-word character becomes a lone high or low surrogate
                seg[starts[k]] = (rng.integers(0xD800, 0xDC00) if rng.random() < 0.5
                                  else rng.integers(0xDC00, 0xE000))
            else:  # a pair's first word becomes a second word: two low surrogates in a row
                seg[starts[k]] = rng.integers(0xDC00, 0xE000)
        return {"u8": u8, "off8": off8.astype(np.uint64), "u16": u16,
                "off16": off16.astype(np.uint64), "profile": prof.astype(np.int8),
                "err8": err8, "err16": err16}

    if cache and B >= 10000:
        return _cached(f"batched:{B}:{seed}:{median}:{sigma}:{max_len}:{error_fraction}", make)
    return make()


def _same_length_error(size: int, rng) -> np.ndarray:
    """An ill-formed byte sequence of `size` bytes (1..4) to put in place of one character."""
    r = lambda lo, hi: int(rng.integers(lo, hi))  # noqa: E731
    form = int(rng.integers(0, 2))
    if size == 1:
        return np.array([r(0x80, 0xC0) if form == 0 else r(0xF8, 0x100)], dtype=np.uint8)
    if size == 2:
        return np.array([r(0xC0, 0xC2), r(0x80, 0xC0)] if form == 0 else [r(0xE1, 0xED), r(0x80, 0xC0)],
                        dtype=np.uint8)
    if size == 3:
        return np.array([0xED, r(0xA0, 0xC0), r(0x80, 0xC0)] if form == 0 else [0xE0, r(0x80, 0xA0), r(0x80, 0xC0)],
                        dtype=np.uint8)
    return np.array([0xF4, r(0x90, 0xC0), r(0x80, 0xC0), r(0x80, 0xC0)] if form == 0
                    else [0xF0, r(0x80, 0x90), r(0x80, 0xC0), r(0x80, 0xC0)], dtype=np.uint8)


# ---- serving: request pools and arrival traces ---------------------------------------------

SERVING_OPS = ("validate_utf8", "validate_utf16le", "convert_utf8_to_utf16le", "convert_utf16le_to_utf8")


def serving_pools(pool_bytes: int = 64 << 20, seed: int = 2000, error_every: int = 1 << 16):
    """Per profile: a UTF-8 text of pool_bytes bytes and the UTF-16LE text of pool_bytes / 2
    words (seeded like the profile buffers), the indices where characters start in each, and
    a copy of each with one corrupted character about every `error_every` units (a byte F8-FF
    over a UTF-8 lead byte, a lone low surrogate over a UTF-16 word).  Requests are slices of
    these pools between character starts, so a request taken from a clean pool is valid."""
    pools = {}
    for k, prof in enumerate(PROFILE_ORDER):
        u8, u16 = profile_buffers(prof, pool_bytes, pool_bytes // 2, seed + k, cache=pool_bytes >= (16 << 20))
        starts8 = np.flatnonzero((u8 & 0xC0) != 0x80)
        starts16 = np.flatnonzero((u16 < 0xDC00) | (u16 >= 0xE000))
        rng = np.random.default_rng(seed + 100 + k)
        bad8, bad16 = u8.copy(), u16.copy()
        pos8 = starts8[rng.integers(0, starts8.size, size=max(1, u8.size // error_every))]
        bad8[pos8] = rng.integers(0xF8, 0x100, size=pos8.size)
        pos16 = starts16[rng.integers(0, starts16.size, size=max(1, u16.size // error_every))]
        bad16[pos16] = rng.integers(0xDC00, 0xE000, size=pos16.size)
        pools[prof] = {"u8": u8, "u16": u16, "starts8": np.append(starts8, u8.size),
                       "starts16": np.append(starts16, u16.size), "bad8": bad8, "bad16": bad16}
    return pools


def serving_trace(count: int, rate: float, pools, seed: int = 3000, min_bytes: int = 16,
                  max_bytes: int = 16 << 20, p_validate: float = 0.10, p_bad: float = 0.0):
    """`count` requests with Poisson arrivals at `rate` per second (arrival_ns from 0), sizes
    log-uniform on [min_bytes, max_bytes] bytes of input, 10% validate-only (half UTF-8, half
    UTF-16LE) and the rest split 50/50 between the two transcoding directions, each of a
    profile drawn uniformly, starting at a random character start of that profile's pool (the
    corrupted copy with probability p_bad) and ending at the last character start that keeps
    the request within its size.  Returns a dict of numpy arrays: op (index into
    SERVING_OPS), profile (index into PROFILE_ORDER), bad, start, n (code units), arrival_ns."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrival = np.rint(np.cumsum(gaps) * 1e9).astype(np.int64)
    arrival -= arrival[0] if count else 0
    size = np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes), size=count))
    u = rng.random(count)
    op = np.where(u < p_validate / 2, 0, np.where(u < p_validate, 1,
                  np.where(u < p_validate + (1 - p_validate) / 2, 2, 3))).astype(np.int8)
    prof = rng.integers(0, len(PROFILE_ORDER), size=count).astype(np.int8)
    bad = rng.random(count) < p_bad
    start = np.zeros(count, np.int64)
    n = np.zeros(count, np.int64)
    pos = rng.random(count)
    for i in range(count):
        p = pools[PROFILE_ORDER[prof[i]]]
        utf16 = op[i] in (1, 3)
        st = p["starts16"] if utf16 else p["starts8"]
        units = max(1, int(size[i] / (2 if utf16 else 1)))
        total = st[-1]
        units = min(units, total)
        # a character start at or before total - units, then the last start within the size
        j = int(pos[i] * np.searchsorted(st, total - units, side="right"))
        s0 = int(st[j])
        e = int(st[np.searchsorted(st, s0 + units, side="right") - 1])
        start[i], n[i] = s0, max(e - s0, 0)
    return {"op": op, "profile": prof, "bad": bad, "start": start, "n": n, "arrival_ns": arrival}
