/*
 * gbu_oracle.c -- scalar CPU reference codec for UTF-8, UTF-16 (LE and BE) and UTF-32.
 *
 * TEST INFRASTRUCTURE ONLY: see gbu_oracle.h.  Plain C, one character at a time, no tables,
 * no blocking, no SIMD.  Nothing here is shared with the CUDA library.
 *
 * Source of each part (paper sections):
 *   - UTF-8 layout: Section 3, the list of leading-byte prefixes (0, 110, 1110, 11110), the
 *     10xxxxxx continuation bytes and the most-significant-bits-first payload order.
 *   - UTF-8 validity: Section 3, rules 1-6.
 *   - UTF-16: Section 3, the two single-word ranges and the surrogate-pair formula (ten low
 *     bits of each word, second word least significant, plus 0x10000).
 *   - Every transcoding validates: Section 5.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - the offset of an error is the index of the first unit of the ill-formed sequence: the
 *     leading byte, or the stray continuation byte itself, or the unpaired surrogate word;
 *   - the kind of an error is the rule that the bytes read so far already break, checked in
 *     reading order: after each byte the set of values the sequence could still take is an
 *     interval, and the sequence fails as soon as that whole interval breaks rule 4, 5 or 6;
 *     a missing continuation byte is rule 2 (TOO_SHORT), also at the end of the buffer;
 *   - rule 5's bound is "less than 1,114,112" (Section 1 prints "between 0 and 1,114,112");
 *   - the byte-order mark and noncharacters are ordinary characters; UTF-16 is little endian
 *     (the UTF-16BE functions at the end take the same words with their bytes in big-endian
 *     order, as RFC 2781 serialises them, and there is no byte-order-mark sniffing).
 *
 * Parity pins (tests/test_oracle_pins.py): boundary scalars and invalid sequences derived by
 * hand from Section 3 (tests/golden/), a round trip of all 1,112,064 scalar values against
 * CPython's codecs, brute force over every UTF-8 string of up to four bytes against a second
 * formulation and against CPython's decoder offsets, and every pair of 16-bit words against a
 * closed form; the UTF-16BE and UTF-32 functions are pinned by CPython's utf-16-be and
 * utf-32-le codecs on every scalar value and by random unpaired surrogates and out-of-range
 * units, and the UTF-32 lengths also by closed forms on arbitrary input.  Every function below
 * is pinned; the error kinds are pinned by the brute force's completion enumeration (a kind
 * other than TOO_SHORT must be broken by every completion of the bytes read).
 */
#include "gbu_oracle.h"

#include <stdlib.h>

/* Section 3: payload bits carried by a leading byte, by sequence length 1..4. */
static const uint8_t LEAD_PAYLOAD_MASK[5] = {0x00, 0x7F, 0x1F, 0x0F, 0x07};
/* Section 3, rule 4: the smallest value that a sequence of length 1..4 may encode. */
static const uint32_t SMALLEST_VALUE[5] = {0, 0x0, 0x80, 0x800, 0x10000};

static or_result make_result(int32_t status, uint64_t count) {
  or_result r;
  r.status = status;
  r.reserved = 0;
  r.count = count;
  return r;
}

/* Section 3: the most significant bits of a leading byte give the sequence length.
 * Returns 0 for a byte that is not a leading byte (10xxxxxx or 11111xxx). */
static int sequence_length(uint8_t b) {
  if ((b & 0x80) == 0x00) return 1; /* 0xxxxxxx */
  if ((b & 0xE0) == 0xC0) return 2; /* 110xxxxx */
  if ((b & 0xF0) == 0xE0) return 3; /* 1110xxxx */
  if ((b & 0xF8) == 0xF0) return 4; /* 11110xxx */
  return 0;
}

static int is_continuation(uint8_t b) { return (b & 0xC0) == 0x80; } /* 10xxxxxx */

/* The values a sequence of length N may still take once `value` holds the payload of the
 * bytes read so far and `remaining` continuation bytes are still to come form the interval
 * [value << 6*remaining, ((value + 1) << 6*remaining) - 1].  Returns the rule (as a result
 * kind) that every value of that interval breaks, or OR_OK if some value is still allowed. */
static int32_t interval_violation(uint32_t value, int remaining, int N) {
  uint32_t lo = value << (6 * remaining);
  uint32_t hi = ((value + 1) << (6 * remaining)) - 1;
  if (hi < SMALLEST_VALUE[N]) return OR_OVERLONG;          /* rule 4 */
  if (lo >= 1114112u) return OR_TOO_LARGE;                 /* rule 5 */
  if (lo >= 0xD800 && hi <= 0xDFFF) return OR_SURROGATE;   /* rule 6 */
  return OR_OK;
}

/* Section 3, UTF-16: the words of a value -- itself below U+10000, else the surrogate pair
 * (the value minus 0x10000, ten high bits on D800 and ten low bits on DC00).  Returns 1 or 2. */
static int utf16_encode(uint32_t value, uint16_t w[2]) {
  if (value < 0x10000) {
    w[0] = (uint16_t)value;
    return 1;
  }
  uint32_t v = value - 0x10000;
  w[0] = (uint16_t)(0xD800 + (v >> 10));
  w[1] = (uint16_t)(0xDC00 + (v & 0x3FF));
  return 2;
}

/* Scans UTF-8 in reading order.  Each character is counted, and written at indices below cap
 * when the destination is not NULL, as one or two UTF-16 words (Section 3) or, when utf32 is
 * set, as one UTF-32 unit (the value itself).  Returns the first error, or {OK, output units
 * the whole input needs}. */
static or_result scan_utf8_to(const uint8_t *src, size_t n, uint16_t *dst16, uint32_t *dst32, size_t cap,
                              int utf32);

static or_result scan_utf8(const uint8_t *src, size_t n, uint16_t *dst16, size_t cap) {
  return scan_utf8_to(src, n, dst16, 0, cap, 0);
}

static or_result scan_utf8_to(const uint8_t *src, size_t n, uint16_t *dst16, uint32_t *dst32, size_t cap,
                              int utf32) {
  uint64_t out = 0;
  size_t i = 0;
  while (i < n) {
    uint8_t lead = src[i];
    int N = sequence_length(lead);
    if (N == 0) {
      if ((lead & 0xF8) == 0xF8) return make_result(OR_HEADER_BITS, i); /* rule 1 */
      return make_result(OR_TOO_LONG, i);                               /* rule 3 */
    }
    uint32_t value = lead & LEAD_PAYLOAD_MASK[N];
    int32_t kind = interval_violation(value, N - 1, N);
    if (kind != OR_OK) return make_result(kind, i);
    for (int k = 1; k < N; ++k) {
      if (i + k >= n || !is_continuation(src[i + k])) return make_result(OR_TOO_SHORT, i); /* rule 2 */
      value = (value << 6) | (src[i + k] & 0x3F);
      kind = interval_violation(value, N - 1 - k, N);
      if (kind != OR_OK) return make_result(kind, i);
    }
    if (utf32) {
      if (dst32 && out < cap) dst32[out] = value;
      out += 1;
    } else {
      uint16_t w[2];
      int len = utf16_encode(value, w);
      for (int k = 0; k < len; ++k) {
        if (dst16 && out < cap) dst16[out] = w[k];
        out += 1;
      }
    }
    i += (size_t)N;
  }
  return make_result(OR_OK, out);
}

/* Section 3, UTF-8 layout: the byte count of a value and its bytes, payload most significant
 * bits first. */
static int utf8_encode(uint32_t cp, uint8_t b[4]) {
  if (cp < 0x80) {
    b[0] = (uint8_t)cp;
    return 1;
  }
  if (cp < 0x800) {
    b[0] = (uint8_t)(0xC0 | (cp >> 6));
    b[1] = (uint8_t)(0x80 | (cp & 0x3F));
    return 2;
  }
  if (cp < 0x10000) {
    b[0] = (uint8_t)(0xE0 | (cp >> 12));
    b[1] = (uint8_t)(0x80 | ((cp >> 6) & 0x3F));
    b[2] = (uint8_t)(0x80 | (cp & 0x3F));
    return 3;
  }
  b[0] = (uint8_t)(0xF0 | (cp >> 18));
  b[1] = (uint8_t)(0x80 | ((cp >> 12) & 0x3F));
  b[2] = (uint8_t)(0x80 | ((cp >> 6) & 0x3F));
  b[3] = (uint8_t)(0x80 | (cp & 0x3F));
  return 4;
}

/* Scans UTF-16LE in reading order (Section 3: a word in D800-DBFF must be followed by one in
 * DC00-DFFF; a word in DC00-DFFF must follow one in D800-DBFF).  When dst8 is not NULL, each
 * character's UTF-8 bytes are written at indices below cap.  Returns the first error, or
 * {OK, UTF-8 bytes the whole input needs}. */
static or_result scan_utf16_to(const uint16_t *src, size_t n, uint8_t *dst8, uint32_t *dst32, size_t cap,
                               int utf32);

static or_result scan_utf16(const uint16_t *src, size_t n, uint8_t *dst8, size_t cap) {
  return scan_utf16_to(src, n, dst8, 0, cap, 0);
}

/* As scan_utf16, but when utf32 is set each character is counted (and written) as one UTF-32
 * unit instead of its UTF-8 bytes. */
static or_result scan_utf16_to(const uint16_t *src, size_t n, uint8_t *dst8, uint32_t *dst32, size_t cap,
                               int utf32) {
  uint64_t out = 0;
  size_t i = 0;
  while (i < n) {
    uint32_t w = src[i];
    uint32_t cp;
    if (w < 0xD800 || w > 0xDFFF) {
      cp = w;
      i += 1;
    } else if (w <= 0xDBFF) {
      if (i + 1 >= n) return make_result(OR_SURROGATE, i);
      uint32_t w2 = src[i + 1];
      if (w2 < 0xDC00 || w2 > 0xDFFF) return make_result(OR_SURROGATE, i);
      cp = (((w & 0x3FF) << 10) | (w2 & 0x3FF)) + 0x10000;
      i += 2;
    } else {
      return make_result(OR_SURROGATE, i);
    }
    if (utf32) {
      if (dst32 && out < cap) dst32[out] = cp;
      out += 1;
      continue;
    }
    uint8_t b[4];
    int len = utf8_encode(cp, b);
    for (int k = 0; k < len; ++k) {
      if (dst8 && out < cap) dst8[out] = b[k];
      out += 1;
    }
  }
  return make_result(OR_OK, out);
}

or_result or_validate_utf8(const uint8_t *src, size_t n) {
  or_result r = scan_utf8(src, n, 0, 0);
  if (r.status == OR_OK) r.count = n;
  return r;
}

or_result or_validate_utf16le(const uint16_t *src, size_t n) {
  or_result r = scan_utf16(src, n, 0, 0);
  if (r.status == OR_OK) r.count = n;
  return r;
}

/* Length of the UTF-16 form, counted on the raw bytes: one word per byte that is not a
 * continuation byte, plus one more for each leading byte of a four-byte sequence (Section 3:
 * such characters need a surrogate pair).  Bytes F8-FF count like four-byte leads. */
uint64_t or_utf16_length_from_utf8(const uint8_t *src, size_t n) {
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) {
    if (!is_continuation(src[i])) total += 1;
    if (src[i] >= 0xF0) total += 1;
  }
  return total;
}

/* Length of the UTF-8 form, counted on the raw words: 1, 2 or 3 bytes by value, and 2 for
 * each surrogate word (a pair needs 4 bytes). */
uint64_t or_utf8_length_from_utf16le(const uint16_t *src, size_t n) {
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) {
    uint16_t w = src[i];
    if (w < 0x80)
      total += 1;
    else if (w < 0x800)
      total += 2;
    else if (w >= 0xD800 && w <= 0xDFFF)
      total += 2;
    else
      total += 3;
  }
  return total;
}

or_result or_convert_utf8_to_utf16le(const uint8_t *src, size_t n, uint16_t *dst, size_t cap) {
  or_result r = scan_utf8(src, n, dst, cap);
  if (r.status == OR_OK && r.count > cap) r.status = OR_OUTPUT_TOO_SMALL;
  return r;
}

or_result or_convert_utf16le_to_utf8(const uint16_t *src, size_t n, uint8_t *dst, size_t cap) {
  or_result r = scan_utf16(src, n, dst, cap);
  if (r.status == OR_OK && r.count > cap) r.status = OR_OUTPUT_TOO_SMALL;
  return r;
}

void or_validate_utf8_batched(const uint8_t *src, const uint64_t *off, size_t B, or_result *res) {
  for (size_t s = 0; s < B; ++s) res[s] = or_validate_utf8(src + off[s], off[s + 1] - off[s]);
}

void or_validate_utf16le_batched(const uint16_t *src, const uint64_t *off, size_t B,
                                 or_result *res) {
  for (size_t s = 0; s < B; ++s) res[s] = or_validate_utf16le(src + off[s], off[s + 1] - off[s]);
}

void or_convert_utf8_to_utf16le_batched(const uint8_t *src, const uint64_t *off, size_t B,
                                        uint16_t *dst, const uint64_t *dst_off, or_result *res) {
  for (size_t s = 0; s < B; ++s)
    res[s] = or_convert_utf8_to_utf16le(src + off[s], off[s + 1] - off[s], dst + dst_off[s],
                                        dst_off[s + 1] - dst_off[s]);
}

void or_convert_utf16le_to_utf8_batched(const uint16_t *src, const uint64_t *off, size_t B,
                                        uint8_t *dst, const uint64_t *dst_off, or_result *res) {
  for (size_t s = 0; s < B; ++s)
    res[s] = or_convert_utf16le_to_utf8(src + off[s], off[s + 1] - off[s], dst + dst_off[s],
                                        dst_off[s + 1] - dst_off[s]);
}

/* UTF-16BE: the UTF-16 words of Section 3 with each word's most significant byte first (RFC
 * 2781).  src and dst hold the words as they lie in memory, so each is read (written) with its
 * two bytes exchanged; the scan is the UTF-16LE one on the exchanged words. */
static uint16_t swap16(uint16_t w) { return (uint16_t)((w >> 8) | (w << 8)); }

static uint16_t *swapped_copy(const uint16_t *src, size_t n) {
  uint16_t *t = (uint16_t *)malloc((n ? n : 1) * sizeof(uint16_t));
  if (!t) abort();
  for (size_t i = 0; i < n; ++i) t[i] = swap16(src[i]);
  return t;
}

or_result or_validate_utf16be(const uint16_t *src, size_t n) {
  uint16_t *t = swapped_copy(src, n);
  or_result r = or_validate_utf16le(t, n);
  free(t);
  return r;
}

uint64_t or_utf8_length_from_utf16be(const uint16_t *src, size_t n) {
  uint16_t *t = swapped_copy(src, n);
  uint64_t len = or_utf8_length_from_utf16le(t, n);
  free(t);
  return len;
}

or_result or_convert_utf16be_to_utf8(const uint16_t *src, size_t n, uint8_t *dst, size_t cap) {
  uint16_t *t = swapped_copy(src, n);
  or_result r = or_convert_utf16le_to_utf8(t, n, dst, cap);
  free(t);
  return r;
}

or_result or_convert_utf8_to_utf16be(const uint8_t *src, size_t n, uint16_t *dst, size_t cap) {
  or_result r = or_convert_utf8_to_utf16le(src, n, dst, cap);
  const uint64_t written = r.status == OR_OK ? r.count : cap;  /* every unit written (at most cap) */
  for (uint64_t i = 0; i < written && i < cap; ++i) dst[i] = swap16(dst[i]);
  return r;
}

/* UTF-32 (not in the paper, whose problem is UTF-8 and UTF-16): one 32-bit unit per character
 * holding its value.  A unit is valid when it is a value Section 3 allows: below 1,114,112
 * (rule 5) and outside D800-DFFF (rule 6); the kinds are those rules' (TOO_LARGE, SURROGATE),
 * at the unit's index.  Units are little-endian in memory (host order). */
static int32_t utf32_unit_violation(uint32_t u) {
  if (u >= 1114112u) return OR_TOO_LARGE;
  if (u >= 0xD800 && u <= 0xDFFF) return OR_SURROGATE;
  return OR_OK;
}

or_result or_validate_utf32(const uint32_t *src, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    int32_t k = utf32_unit_violation(src[i]);
    if (k != OR_OK) return make_result(k, i);
  }
  return make_result(OR_OK, n);
}

/* UTF-8 bytes by value, for any unit: 1 below 0x80, 2 below 0x800, 3 below 0x10000, else 4. */
uint64_t or_utf8_length_from_utf32(const uint32_t *src, size_t n) {
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) total += src[i] < 0x80 ? 1 : (src[i] < 0x800 ? 2 : (src[i] < 0x10000 ? 3 : 4));
  return total;
}

/* UTF-32 units of a UTF-8 input: one per byte that is not a continuation byte. */
uint64_t or_utf32_length_from_utf8(const uint8_t *src, size_t n) {
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i)
    if (!is_continuation(src[i])) total += 1;
  return total;
}

or_result or_convert_utf32_to_utf8(const uint32_t *src, size_t n, uint8_t *dst, size_t cap) {
  uint64_t out = 0;
  for (size_t i = 0; i < n; ++i) {
    int32_t k = utf32_unit_violation(src[i]);
    if (k != OR_OK) return make_result(k, i);
    uint8_t b[4];
    int len = utf8_encode(src[i], b);
    for (int j = 0; j < len; ++j) {
      if (out < cap) dst[out] = b[j];
      out += 1;
    }
  }
  return make_result(out > cap ? OR_OUTPUT_TOO_SMALL : OR_OK, out);
}

or_result or_convert_utf8_to_utf32(const uint8_t *src, size_t n, uint32_t *dst, size_t cap) {
  or_result r = scan_utf8_to(src, n, 0, dst, cap, 1);
  if (r.status == OR_OK && r.count > cap) r.status = OR_OUTPUT_TOO_SMALL;
  return r;
}

/* UTF-16 words of a UTF-32 input, for any unit: 1 below 0x10000, else 2 (a surrogate pair). */
uint64_t or_utf16_length_from_utf32(const uint32_t *src, size_t n) {
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) total += src[i] < 0x10000 ? 1 : 2;
  return total;
}

/* UTF-32 units of a UTF-16LE input: one per word that is not a second surrogate (DC00-DFFF). */
uint64_t or_utf32_length_from_utf16le(const uint16_t *src, size_t n) {
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i)
    if (src[i] < 0xDC00 || src[i] > 0xDFFF) total += 1;
  return total;
}

/* Section 3, UTF-16: one word below U+10000, else the surrogate pair. */
or_result or_convert_utf32_to_utf16le(const uint32_t *src, size_t n, uint16_t *dst, size_t cap) {
  uint64_t out = 0;
  for (size_t i = 0; i < n; ++i) {
    int32_t k = utf32_unit_violation(src[i]);
    if (k != OR_OK) return make_result(k, i);
    uint16_t w[2];
    int len = utf16_encode(src[i], w);
    for (int k = 0; k < len; ++k) {
      if (out < cap) dst[out] = w[k];
      out += 1;
    }
  }
  return make_result(out > cap ? OR_OUTPUT_TOO_SMALL : OR_OK, out);
}

or_result or_convert_utf16le_to_utf32(const uint16_t *src, size_t n, uint32_t *dst, size_t cap) {
  or_result r = scan_utf16_to(src, n, 0, dst, cap, 1);
  if (r.status == OR_OK && r.count > cap) r.status = OR_OUTPUT_TOO_SMALL;
  return r;
}
