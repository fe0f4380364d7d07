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
]


def _battery(codec, bf):
    P.check_golden(codec)
    P.check_all_scalars(codec)
    P.check_bruteforce(bf, max_len=3)
    P.check_utf16_pairs(bf, codec, full=False)
    P.check_length_closed_forms(codec)
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
