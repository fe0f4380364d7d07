"""The synthetic inputs against their stated recipe: each profile's character mix, the bytes per
character behind the roofline's algorithmic bytes, exact buffer sizes and padding, the injected
errors of the invalid-input sweep and of the batched strings, and reproducibility from the seed.
CPython's strict codecs judge validity here; nothing of the library or the reference codec runs."""
import codecs

import numpy as np
import pytest

import workloads as W

N = 400_000

# profile: (lo, hi, weight) ranges, hi exclusive; every drawn character lies in one of them
RANGES = {
    "ascii": [(0x20, 0x7F, 1.0)],
    "latin": [(0x20, 0x7F, 0.95), (0xC0, 0x180, 0.05)],
    "cyrillic": [(0x400, 0x500, 0.70), (0x20, 0x7F, 0.30)],
    "cjk": [(0x4E00, 0xA000, 0.85), (0x20, 0x7F, 0.15)],
    "emoji": [(0x20, 0x7F, 0.70), (0x1F300, 0x1FB00, 0.30)],
    "mixed": [(0x0, 0x80, 0.50), (0x80, 0x800, 0.20), (0x800, 0x10000, 0.20), (0x10000, 0x110000, 0.10)],
}


def _utf8_size(cp):
    return 1 if cp < 0x80 else 2 if cp < 0x800 else 3 if cp < 0x10000 else 4


@pytest.mark.parametrize("profile", sorted(RANGES))
def test_profile_mixes(profile):
    cps = W.draw_codepoints(profile, N, np.random.default_rng(7))
    assert cps.size == N and cps.dtype == np.uint32
    assert not np.any((cps >= 0xD800) & (cps <= 0xDFFF)), "a surrogate value is not a character"
    covered = np.zeros(N, dtype=bool)
    for lo, hi, w in RANGES[profile]:
        inside = (cps >= lo) & (cps < hi)
        covered |= inside
        sigma = (w * (1 - w) / N) ** 0.5
        assert abs(inside.mean() - w) <= 5 * sigma + 1e-12, (profile, hex(lo), inside.mean(), w)
    assert covered.all()
    if profile == "cyrillic":
        # the ASCII part: half U+0020, half the 32 punctuation characters, no letters or digits
        ascii_part = cps[cps < 0x80]
        assert not any(chr(c).isalnum() for c in np.unique(ascii_part))
        assert len(np.unique(ascii_part)) == 33
        sigma = (0.25 / ascii_part.size) ** 0.5
        assert abs((ascii_part == 0x20).mean() - 0.5) <= 5 * sigma


@pytest.mark.parametrize("profile", W.PROFILE_ORDER)
def test_bytes_per_character_match_the_mix(profile):
    """The algorithmic bytes per input byte of both transcoders, from the mix's expected UTF-8
    bytes and UTF-16 words per character, against the generator's encoded output."""
    assert all(_utf8_size(lo) == _utf8_size(hi - 1) for lo, hi, _ in RANGES[profile])  # one size per range
    b8 = sum(w * _utf8_size(lo) for lo, hi, w in RANGES[profile])
    w16 = sum(w * (2 if lo >= 0x10000 else 1) for lo, hi, w in RANGES[profile])
    cps = W.draw_codepoints(profile, N, np.random.default_rng(11))
    n8, n16 = W.encode_utf8(cps).size, W.encode_utf16le(cps).size
    want_816, want_168 = (b8 + 2 * w16) / b8, (2 * w16 + b8) / (2 * w16)
    assert abs((n8 + 2 * n16) / n8 - want_816) <= 0.01 * want_816, profile
    assert abs((2 * n16 + n8) / (2 * n16) - want_168) <= 0.01 * want_168, profile


@pytest.mark.parametrize("profile", W.PROFILE_ORDER)
def test_profile_buffers_exact_valid_and_reproducible(profile):
    n8, n16 = (1 << 20) + 3, (1 << 19) + 1
    u8, u16 = W.profile_buffers(profile, n8, n16, W.PROFILE_SEEDS[profile], cache=False)
    assert u8.size == n8 and u16.size == n16 and u8.dtype == np.uint8 and u16.dtype == np.uint16
    t8, t16 = u8.tobytes().decode("utf-8"), u16.tobytes().decode("utf-16-le")  # strict: valid text
    # both are prefixes of one character stream, padded with U+0020
    a, b = t8.rstrip(" "), t16.rstrip(" ")
    assert a.startswith(b) or b.startswith(a)
    again8, again16 = W.profile_buffers(profile, n8, n16, W.PROFILE_SEEDS[profile], cache=False)
    assert np.array_equal(u8, again8) and np.array_equal(u16, again16)


def test_mixed_1mib_and_its_flipped_copy():
    u8, u16, flipped, o = W.mixed_1mib()
    assert u8.size == 1 << 20
    text = u8.tobytes().decode("utf-8")
    assert u16.tobytes() == text.encode("utf-16-le")
    assert np.flatnonzero(u8 != flipped).tolist() == [o] and flipped[o] == u8[o] ^ 0xFF
    with pytest.raises(UnicodeDecodeError):
        flipped.tobytes().decode("utf-8")


@pytest.mark.parametrize("profile", ["latin", "cyrillic", "cjk", "emoji", "mixed"])
def test_every_error_template_is_ill_formed_at_its_first_byte(profile):
    """An injected UTF-8 error starts where its template starts, for every kind, so the first
    error of a sweep buffer lies at a template position."""
    rng = np.random.default_rng(5)
    kinds = np.repeat(np.arange(len(W.UTF8_ERROR_KINDS)), 400)
    t = W.utf8_error_templates(kinds, profile, rng)
    assert t.shape == (kinds.size, 4)
    for row in t:
        with pytest.raises(UnicodeDecodeError) as e:
            (row.tobytes() + b"  ").decode("utf-8")
        assert e.value.start == 0, row.tobytes().hex()


@pytest.mark.parametrize("profile", W.SWEEP_PROFILES)
def test_sweep_buffers(profile):
    n = 1 << 20
    d = W.sweep_buffers(profile, 1e-2, n_bytes=n, seed=99, cache=False)
    assert d["u8"].size == n and d["u8_cut_end"].size == n
    assert d["u16"].size == n // 2 and d["u16_cut_end"].size == n // 2
    # about one error per hundred characters (CPython's replacement count is at least one per site)
    hits = []
    codecs.register_error("gbu_count", lambda e: (hits.append(e.start) or "", e.end))
    chars = len(d["u8"].tobytes().decode("utf-8", errors="gbu_count"))
    assert 0.3 * 0.01 * chars <= len(hits) <= 4 * 0.01 * chars, (len(hits), chars)
    hits.clear()
    words = d["u16"].size
    d["u16"].tobytes().decode("utf-16-le", errors="gbu_count")
    assert 0.5 * 0.01 * words <= len(hits) <= 2 * 0.01 * words, (len(hits), words)  # one word per character
    # the cut siblings: valid up to a final character missing its last unit
    with pytest.raises(UnicodeDecodeError) as e:
        d["u8_cut_end"].tobytes().decode("utf-8")
    assert "unexpected end of data" in e.value.reason and e.value.start >= n - 3
    d["u8_cut_end"][: e.value.start].tobytes().decode("utf-8")
    with pytest.raises(UnicodeDecodeError) as e:
        d["u16_cut_end"].tobytes().decode("utf-16-le")
    assert e.value.start == n - 2 and 0xD800 <= int(d["u16_cut_end"][-1]) <= 0xDBFF


def test_batched_strings():
    B = 5000
    d = W.batched_strings(B=B, cache=False)
    off8, off16 = d["off8"], d["off16"]
    assert off8.size == B + 1 and off16.size == B + 1 and off8[0] == 0 and off16[0] == 0
    assert off8[-1] == d["u8"].size and off16[-1] == d["u16"].size
    lens = np.diff(off8)
    assert lens.min() >= 1 and lens.max() <= 65536
    assert 48 <= np.median(lens) <= 80  # log-normal with median 64
    assert 20 <= d["err8"].sum() <= 100 and 20 <= d["err16"].sum() <= 100  # about 1% of 5000
    for i in range(B):
        s8 = d["u8"][off8[i]:off8[i + 1]].tobytes()
        s16 = d["u16"][off16[i]:off16[i + 1]].tobytes()
        if d["err8"][i]:
            with pytest.raises(UnicodeDecodeError):
                s8.decode("utf-8")
        if d["err16"][i]:
            with pytest.raises(UnicodeDecodeError):
                s16.decode("utf-16-le")
        if not d["err8"][i] and not d["err16"][i]:
            assert s8.decode("utf-8") == s16.decode("utf-16-le"), i


def test_serving_pools_and_trace():
    pools = W.serving_pools(pool_bytes=1 << 20, error_every=1 << 14)
    assert set(pools) == set(W.PROFILE_ORDER)
    for prof, p in pools.items():
        u8, u16 = p["u8"], p["u16"]
        u8.tobytes().decode("utf-8")
        u16.tobytes().decode("utf-16-le")
        # character starts (plus the end), and the corrupted copies differ only at some of them
        assert np.array_equal(p["starts8"][:-1], np.flatnonzero((u8 & 0xC0) != 0x80)) and p["starts8"][-1] == u8.size
        d8 = np.flatnonzero(p["bad8"] != u8)
        d16 = np.flatnonzero(p["bad16"] != u16)
        assert 1 <= d8.size <= u8.size // (1 << 14) and 1 <= d16.size <= u16.size // (1 << 14)
        assert np.isin(d8, p["starts8"]).all() and np.isin(d16, p["starts16"]).all()
        assert (p["bad8"][d8] >= 0xF8).all() and ((p["bad16"][d16] >= 0xDC00) & (p["bad16"][d16] < 0xE000)).all()

    count, rate = 20000, 1e5
    t = W.serving_trace(count, rate, pools, p_bad=0.1)
    arr = t["arrival_ns"]
    assert arr[0] == 0 and (np.diff(arr) >= 0).all()
    mean_gap = arr[-1] / (count - 1) / 1e9
    assert abs(mean_gap * rate - 1) < 0.05  # Poisson arrivals at the offered rate
    frac = np.bincount(t["op"], minlength=4) / count
    for f, want in zip(frac, (0.05, 0.05, 0.45, 0.45)):
        assert abs(f - want) <= 5 * (want * (1 - want) / count) ** 0.5, frac
    assert abs(t["bad"].mean() - 0.1) <= 5 * (0.09 / count) ** 0.5
    for i in range(count):
        p = pools[W.PROFILE_ORDER[t["profile"][i]]]
        utf16 = t["op"][i] in (1, 3)
        st = p["starts16"] if utf16 else p["starts8"]
        s0, n = int(t["start"][i]), int(t["n"][i])
        assert n * (2 if utf16 else 1) <= 16 << 20
        # every request is a slice between character starts, so a clean one is valid text
        k = np.searchsorted(st, [s0, s0 + n])
        assert (k < st.size).all() and st[k[0]] == s0 and st[k[1]] == s0 + n, i
        if not t["bad"][i] and i % 50 == 0:
            src = p["u16"] if utf16 else p["u8"]
            src[s0:s0 + n].tobytes().decode("utf-16-le" if utf16 else "utf-8")
