"""Mutation test for the pins: each plausible mistake, planted in a copy of the reference
codec on the CPU, must make at least one pin fail.  The real codec is never modified."""
import os

import pytest

import oracle
import oracle_pins as P
from bfhelper import BF, ORACLE_SRC, build

MUTANTS = [
    ("rule 6 dropped",
     "  if (lo >= 0xD800 && hi <= 0xDFFF) return OR_SURROGATE;   /* rule 6 */\n", ""),
    ("rule 5 bound off by one", "if (lo >= 1114112u) return OR_TOO_LARGE;",
     "if (lo > 1114112u) return OR_TOO_LARGE;"),
    ("rule 4 three-byte limit off by one", "{0, 0x0, 0x80, 0x800, 0x10000}",
     "{0, 0x0, 0x80, 0x7FF, 0x10000}"),
    ("surrogate pair words transposed", "cp = (((w & 0x3FF) << 10) | (w2 & 0x3FF)) + 0x10000;",
     "cp = (((w2 & 0x3FF) << 10) | (w & 0x3FF)) + 0x10000;"),
    ("high surrogate shift wrong", "(uint16_t)(0xD800 + (v >> 10))", "(uint16_t)(0xD800 + (v >> 9))"),
    ("low surrogate mask wrong", "(uint16_t)(0xDC00 + (v & 0x3FF))", "(uint16_t)(0xDC00 + (v & 0x1FF))"),
    ("TOO_SHORT reported at the missing byte", "return make_result(OR_TOO_SHORT, i); /* rule 2 */",
     "return make_result(OR_TOO_SHORT, i + k); /* rule 2 */"),
    ("lone low surrogate accepted",
     "    } else {\n      return make_result(OR_SURROGATE, i);\n    }",
     "    } else {\n      cp = w;\n      i += 1;\n    }"),
    ("four-byte lead length off by one", "if (src[i] >= 0xF0) total += 1;", "if (src[i] > 0xF0) total += 1;"),
    ("three-byte encoding boundary off by one", "  if (cp < 0x800) {", "  if (cp <= 0x800) {"),
    ("continuation test too loose", "static int is_continuation(uint8_t b) { return (b & 0xC0) == 0x80; }",
     "static int is_continuation(uint8_t b) { return (b & 0x80) == 0x80; }"),
    ("surrogate words counted as three bytes",
     "    else if (w >= 0xD800 && w <= 0xDFFF)\n      total += 2;",
     "    else if (w >= 0xD800 && w <= 0xDFFF)\n      total += 3;"),
    ("validation returns the output length", "  if (r.status == OR_OK) r.count = n;\n  return r;\n}\n\nor_result or_validate_utf16le",
     "  return r;\n}\n\nor_result or_validate_utf16le"),
    ("rule 1 reported as rule 3", "if ((lead & 0xF8) == 0xF8) return make_result(OR_HEADER_BITS, i);",
     "if ((lead & 0xF8) == 0xF8) return make_result(OR_TOO_LONG, i);"),
    # UTF-16BE and UTF-32
    ("UTF-16BE output left in little-endian order",
     "  for (uint64_t i = 0; i < written && i < cap; ++i) dst[i] = swap16(dst[i]);\n", ""),
    ("UTF-16BE byte exchange loses the high byte", "return (uint16_t)((w >> 8) | (w << 8));",
     "return (uint16_t)(w >> 8);"),
    ("UTF-32 rule 5 bound off by one", "if (u >= 1114112u) return OR_TOO_LARGE;",
     "if (u > 1114112u) return OR_TOO_LARGE;"),
    ("UTF-32 surrogate range only the first surrogates", "if (u >= 0xD800 && u <= 0xDFFF) return OR_SURROGATE;",
     "if (u >= 0xD800 && u <= 0xDBFF) return OR_SURROGATE;"),
    ("UTF-32 to UTF-8 skips validation",
     "    if (k != OR_OK) return make_result(k, i);\n    uint8_t b[4];", "    uint8_t b[4];"),
    ("UTF-8 length of a UTF-32 unit: four-byte bound off by one", "(src[i] < 0x10000 ? 3 : 4)",
     "(src[i] <= 0x10000 ? 3 : 4)"),
    ("UTF-32 length of UTF-8 counts four-byte leads twice",
     "    if (!is_continuation(src[i])) total += 1;\n  return total;",
     "    if (!is_continuation(src[i])) total += 1 + (src[i] >= 0xF0);\n  return total;"),
    ("UTF-16 length of a UTF-32 unit: pair bound off by one", "total += src[i] < 0x10000 ? 1 : 2;",
     "total += src[i] < 0xFFFF ? 1 : 2;"),
    ("UTF-32 length of UTF-16 counts second surrogates instead of first",
     "if (src[i] < 0xDC00 || src[i] > 0xDFFF) total += 1;", "if (src[i] < 0xD800 || src[i] > 0xDBFF) total += 1;"),
    ("UTF-8 to UTF-16 capacity checked before the input error",
     "or_result r = scan_utf8(src, n, dst, cap);\n  if (r.status == OR_OK && r.count > cap)",
     "or_result r = scan_utf8(src, n, dst, cap);\n  if (r.count > cap)"),
    ("UTF-16 to UTF-8 capacity checked before the input error",
     "or_result r = scan_utf16(src, n, dst, cap);\n  if (r.status == OR_OK && r.count > cap)",
     "or_result r = scan_utf16(src, n, dst, cap);\n  if (r.count > cap)"),
    ("UTF-8 to UTF-32 stores the low 16 bits", "if (dst32 && out < cap) dst32[out] = value;",
     "if (dst32 && out < cap) dst32[out] = value & 0xFFFF;"),
]


def _battery(codec, bf):
    P.check_golden(codec)
    P.check_all_scalars(codec)
    P.check_all_scalars_utf16be(codec)
    P.check_all_scalars_utf32(codec)
    P.check_bruteforce(bf, max_len=3)
    P.check_utf16_pairs(bf, codec, full=False)
    P.check_length_closed_forms(codec)
    P.check_edge_cases(codec)
    P.check_cpython_offsets(bf, three_byte_leads=range(0xE0, 0xF8))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new):
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, "mutation site not unique or missing: " + name
    so = build(src.replace(old, new))
    bf = BF(so)
    codec = oracle.Codec(bf.lib)
    with pytest.raises(AssertionError):
        _battery(codec, bf)


def test_battery_passes_on_the_real_codec():
    bf = BF(build())
    _battery(oracle.Codec(bf.lib), bf)
