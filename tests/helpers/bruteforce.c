/*
 * bruteforce.c -- exhaustive checks of the reference codec (test helper, CPU only).
 *
 * Compiled together with oracle/gbu_oracle.c (or a deliberately broken copy of it, for the
 * mutation test) into a shared library that the tests call through ctypes.  Nothing here is
 * used by the CUDA library.
 *
 * The UTF-8 checks compare the codec with a second formulation written from the paper's
 * Section 3 in a different way: a sequence is judged after its bytes are read, and a prefix
 * of a sequence is "dead" when ENUMERATING every possible completion of it yields no value
 * that the rules accept for that length.  The codec instead reasons on interval bounds.  The
 * offset, the kind and the validity must agree on every string of up to four bytes.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "gbu_oracle.h"

/* ---- second formulation ------------------------------------------------------------ */

/* Section 3: bits of the leading byte -> sequence length (0: not a leading byte). */
static int bf_length(uint8_t b) {
  if (b <= 0x7F) return 1;
  if (b >= 0xC0 && b <= 0xDF) return 2;
  if (b >= 0xE0 && b <= 0xEF) return 3;
  if (b >= 0xF0 && b <= 0xF7) return 4;
  return 0;
}

/* Rule check on one decoded value for a sequence of `len` bytes: 0 if acceptable, else the
 * kind (4 overlong, 5 too large, 6 surrogate), rules tested in the order they are listed. */
static int bf_rule(uint32_t v, int len) {
  static const uint32_t largest_shorter[5] = {0, 0, 0x7F, 0x7FF, 0xFFFF}; /* rule 4 */
  if (len >= 2 && v <= largest_shorter[len]) return OR_OVERLONG;
  if (v >= 1114112u) return OR_TOO_LARGE;                       /* rule 5 */
  if (v >= 0xD800 && v <= 0xDFFF) return OR_SURROGATE;         /* rule 6 */
  return 0;
}

#define DEAD_MIXED 100
/* dead[lead - 0xC0][m - 1][payload]: for the incomplete prefix made of the lead and m-1
 * continuation bytes (m < sequence length) whose continuation payload bits are `payload`,
 * the kind that EVERY completion breaks, 0 if some completion is accepted, DEAD_MIXED if
 * every completion is rejected but not all by one rule.  A complete sequence has a single
 * completion (itself) and is judged by bf_rule directly. */
static uint8_t *dead; /* 0x38 leads x 4 prefix lengths x 4096 payloads */
static const uint32_t LEAD_BITS_MASK[5] = {0, 0x7F, 0x1F, 0x0F, 0x07};

static size_t dead_index(int lead, int m, uint32_t payload) {
  return ((size_t)(lead - 0xC0) * 4 + (size_t)(m - 1)) * 4096 + payload;
}

static void build_dead_table(void) {
  dead = (uint8_t *)calloc((size_t)0x38 * 4 * 4096, 1);
  for (int lead = 0xC0; lead <= 0xF7; ++lead) {
    int len = bf_length((uint8_t)lead);
    uint32_t lead_bits = (uint32_t)lead & LEAD_BITS_MASK[len];
    for (int m = 1; m < len; ++m) {
      uint32_t npay = 1u << (6 * (m - 1));
      uint32_t ncomp = 1u << (6 * (len - m));
      for (uint32_t p = 0; p < npay; ++p) {
        uint32_t prefix = (lead_bits << (6 * (m - 1))) | p;
        int any_ok = 0, all4 = 1, all5 = 1, all6 = 1;
        for (uint32_t t = 0; t < ncomp; ++t) {
          uint32_t v = (prefix << (6 * (len - m))) | t;
          int k = bf_rule(v, len);
          if (k == 0) { any_ok = 1; break; }
          uint32_t small[5] = {0, 0, 0x7F, 0x7FF, 0xFFFF};
          if (!(v <= small[len])) all4 = 0;
          if (!(v >= 1114112u)) all5 = 0;
          if (!(v >= 0xD800 && v <= 0xDFFF)) all6 = 0;
        }
        uint8_t kind = 0;
        if (!any_ok) kind = all4 ? OR_OVERLONG : all5 ? OR_TOO_LARGE : all6 ? OR_SURROGATE : DEAD_MIXED;
        dead[dead_index(lead, m, p)] = kind;
      }
    }
  }
}

/* Second formulation of UTF-8 validation; returns the kind and sets *offset. */
static int bf_validate(const uint8_t *s, size_t n, uint64_t *offset) {
  size_t i = 0;
  while (i < n) {
    uint8_t b = s[i];
    if (b >= 0xF8) { *offset = i; return OR_HEADER_BITS; }          /* rule 1 */
    if (b >= 0x80 && b <= 0xBF) { *offset = i; return OR_TOO_LONG; } /* rule 3 */
    int len = bf_length(b);
    if (len == 1) { i += 1; continue; }
    /* walk the prefixes in reading order */
    uint32_t payload = 0;
    for (int m = 1; m <= len; ++m) {
      if (m >= 2) {
        size_t j = i + (size_t)m - 1;
        if (j >= n || (s[j] & 0xC0) != 0x80) { *offset = i; return OR_TOO_SHORT; } /* rule 2 */
        payload = (payload << 6) | (s[j] & 0x3Fu);
      }
      int k;
      if (m < len) {
        k = dead[dead_index(b, m, payload)];
      } else {
        uint32_t v = (((uint32_t)b & LEAD_BITS_MASK[len]) << (6 * (len - 1))) | payload;
        k = bf_rule(v, len);
      }
      if (k) { *offset = i; return k; }
    }
    i += (size_t)len;
  }
  *offset = n;
  return OR_OK;
}

/* ---- exhaustive UTF-8 sweep ---------------------------------------------------------- */

typedef struct {
  int len;
  uint32_t first_lo, first_hi; /* range of the first byte handled by this thread */
  int roundtrip;
  long mismatches;
  long valid;
  long kinds[8];
  uint8_t example[4];
  int example_len;
} bf_job;

static int roundtrip_ok(const uint8_t *s, size_t n, uint64_t units) {
  uint16_t w[8];
  uint8_t back[16];
  if (or_utf16_length_from_utf8(s, n) != units) return 0;
  or_result r = or_convert_utf8_to_utf16le(s, n, w, 8);
  if (r.status != OR_OK || r.count != units) return 0;
  if (or_utf8_length_from_utf16le(w, units) != n) return 0;
  or_result v16 = or_validate_utf16le(w, units);
  if (v16.status != OR_OK || v16.count != units) return 0;
  or_result r2 = or_convert_utf16le_to_utf8(w, units, back, 16);
  if (r2.status != OR_OK || r2.count != n) return 0;
  return memcmp(back, s, n) == 0;
}

static void *bf_worker(void *arg) {
  bf_job *job = (bf_job *)arg;
  int len = job->len;
  uint8_t s[4];
  uint64_t tail = 1ull << (8 * (len - 1));
  for (uint32_t first = job->first_lo; first < job->first_hi; ++first) {
    for (uint64_t t = 0; t < tail; ++t) {
      s[0] = (uint8_t)first;
      for (int k = 1; k < len; ++k) s[k] = (uint8_t)(t >> (8 * (k - 1)));
      uint64_t off2;
      int k2 = bf_validate(s, (size_t)len, &off2);
      or_result r = or_validate_utf8(s, (size_t)len);
      uint16_t w[8];
      or_result c = or_convert_utf8_to_utf16le(s, (size_t)len, w, 8);
      int bad = 0;
      if (r.status != k2) bad = 1;
      if (k2 == OR_OK && r.count != (uint64_t)len) bad = 1;
      if (k2 != OR_OK && r.count != off2) bad = 1;
      if (c.status != r.status) bad = 1;
      if (k2 != OR_OK && c.count != off2) bad = 1;
      if (k2 == OR_OK) {
        job->valid++;
        if (job->roundtrip && !roundtrip_ok(s, (size_t)len, c.count)) bad = 1;
      }
      if (k2 >= 0 && k2 < 8) job->kinds[k2]++;
      if (bad) {
        if (job->mismatches == 0) {
          memcpy(job->example, s, 4);
          job->example_len = len;
        }
        job->mismatches++;
      }
    }
  }
  return 0;
}

/* Checks every UTF-8 string of exactly `len` bytes (1..4).  Returns the number of strings on
 * which the codec and the second formulation disagree (or, with roundtrip != 0, on which a
 * valid string fails to survive UTF-8 -> UTF-16 -> UTF-8 with consistent lengths).  stats
 * receives [valid, count per kind 0..7, first mismatching string as 4 bytes + its length]. */
long bf_utf8(int len, int nthreads, int roundtrip, long *stats) {
  if (!dead) build_dead_table();
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  bf_job jobs[64];
  pthread_t th[64];
  uint32_t per = (256 + (uint32_t)nthreads - 1) / (uint32_t)nthreads;
  for (int t = 0; t < nthreads; ++t) {
    memset(&jobs[t], 0, sizeof(bf_job));
    jobs[t].len = len;
    jobs[t].roundtrip = roundtrip;
    jobs[t].first_lo = (uint32_t)t * per;
    jobs[t].first_hi = ((uint32_t)t + 1) * per > 256 ? 256 : ((uint32_t)t + 1) * per;
    if (jobs[t].first_lo > 256) jobs[t].first_lo = 256;
    pthread_create(&th[t], 0, bf_worker, &jobs[t]);
  }
  long mism = 0;
  memset(stats, 0, sizeof(long) * 14);
  int have_example = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], 0);
    mism += jobs[t].mismatches;
    stats[0] += jobs[t].valid;
    for (int k = 0; k < 8; ++k) stats[1 + k] += jobs[t].kinds[k];
    if (jobs[t].mismatches && !have_example) {
      have_example = 1;
      for (int k = 0; k < 4; ++k) stats[9 + k] = jobs[t].example[k];
      stats[13] = jobs[t].example_len;
    }
  }
  return mism;
}

/* Writes the codec's (kind, offset) for every string of exactly `len` bytes (len <= 3),
 * indexed by the string read as a little-endian integer (first byte least significant). */
void bf_table(int len, uint8_t *kind, uint8_t *offset) {
  uint64_t total = 1ull << (8 * len);
  uint8_t s[4];
  for (uint64_t x = 0; x < total; ++x) {
    for (int k = 0; k < len; ++k) s[k] = (uint8_t)(x >> (8 * k));
    or_result r = or_validate_utf8(s, (size_t)len);
    kind[x] = (uint8_t)r.status;
    offset[x] = (uint8_t)(r.status == OR_OK ? 255 : r.count);
  }
}

/* Number of dead prefixes for which every completion is rejected but not by a single rule
 * (the kind is then undefined; the reading used by the codec assumes there are none). */
long bf_mixed_dead_prefixes(void) {
  if (!dead) build_dead_table();
  long c = 0;
  for (size_t i = 0; i < (size_t)0x38 * 4 * 4096; ++i) c += dead[i] == DEAD_MIXED;
  return c;
}

/* ---- UTF-16: every pair of 16-bit words -------------------------------------------- */

typedef struct {
  uint32_t a_lo, a_hi;
  long mismatches;
  long valid;
  uint32_t example;
} pair_job;

static int is_high(uint32_t w) { return w >= 0xD800 && w <= 0xDBFF; }
static int is_low(uint32_t w) { return w >= 0xDC00 && w <= 0xDFFF; }

/* Closed form for two words a, b (Section 3: only surrogates need attention; a high word
 * must be followed by a low word and a low word must follow a high word). */
static int pair_closed_form(uint32_t a, uint32_t b, uint64_t *offset) {
  if (is_high(a)) {
    if (is_low(b)) return OR_OK;
    *offset = 0;
    return OR_SURROGATE;
  }
  if (is_low(a)) { *offset = 0; return OR_SURROGATE; }
  if (is_high(b) || is_low(b)) { *offset = 1; return OR_SURROGATE; }
  return OR_OK;
}

static void *pair_worker(void *arg) {
  pair_job *job = (pair_job *)arg;
  uint16_t s[2];
  for (uint32_t a = job->a_lo; a < job->a_hi; ++a) {
    for (uint32_t b = 0; b < 65536; ++b) {
      s[0] = (uint16_t)a;
      s[1] = (uint16_t)b;
      uint64_t off = 0;
      int k = pair_closed_form(a, b, &off);
      or_result r = or_validate_utf16le(s, 2);
      int bad = r.status != k || (k == OR_OK ? r.count != 2 : r.count != off);
      if (k == OR_OK) job->valid++;
      if (bad) {
        if (!job->mismatches) job->example = (a << 16) | b;
        job->mismatches++;
      }
    }
  }
  return 0;
}

/* Validates every two-word UTF-16LE string; returns disagreements with the closed form.
 * stats = [valid count, first mismatch as (a << 16 | b)]. */
long bf_utf16_pairs(int nthreads, long *stats) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  pair_job jobs[64];
  pthread_t th[64];
  uint32_t per = (65536 + (uint32_t)nthreads - 1) / (uint32_t)nthreads;
  for (int t = 0; t < nthreads; ++t) {
    memset(&jobs[t], 0, sizeof(pair_job));
    jobs[t].a_lo = (uint32_t)t * per > 65536 ? 65536 : (uint32_t)t * per;
    jobs[t].a_hi = ((uint32_t)t + 1) * per > 65536 ? 65536 : ((uint32_t)t + 1) * per;
    pthread_create(&th[t], 0, pair_worker, &jobs[t]);
  }
  long mism = 0;
  stats[0] = stats[1] = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], 0);
    if (jobs[t].mismatches && !mism) stats[1] = jobs[t].example;
    mism += jobs[t].mismatches;
    stats[0] += jobs[t].valid;
  }
  return mism;
}

/* Writes the codec's (kind, offset) for the two-word strings [a, b] with a, b taken from
 * `words` (m entries each), row-major, for a cross-check against another decoder. */
void bf_utf16_pair_table(const uint16_t *words, size_t m, uint8_t *kind, uint8_t *offset) {
  uint16_t s[2];
  for (size_t i = 0; i < m; ++i)
    for (size_t j = 0; j < m; ++j) {
      s[0] = words[i];
      s[1] = words[j];
      or_result r = or_validate_utf16le(s, 2);
      kind[i * m + j] = (uint8_t)r.status;
      offset[i * m + j] = (uint8_t)(r.status == OR_OK ? 255 : r.count);
    }
}
