// gbu_chunk.cuh -- per-thread analysis of one 16-byte chunk (4 x 32-bit words), shared by
// the streaming kernels (validation, lengths) and the transcoders.
//
// UTF-8 (paper Section 3): a leading byte's top bits give the sequence length (0xxxxxxx,
// 110xxxxx, 1110xxxx, 11110xxx); continuation bytes are 10xxxxxx; rules 1-6 make a byte
// sequence valid.  All tests run on 32-bit words (SWAR):
//   * classification: per byte, flags "continuation", ">= C0", ">= E0", ">= F0" as the
//     most significant bit of each byte;
//   * structure (rules 1-3): a byte must be a continuation exactly when one of the three
//     bytes before it is a leading byte that needs it (>= C0 one back, >= E0 two back, >= F0
//     three back): the three flag words are funnel-shifted by 1, 2 and 3 bytes and compared
//     with the continuation flags (bytes past the end of the input read as zero, so a cut
//     sequence fails there);
//   * values (rules 4-6, and rule 1 for F8-FF): given a correct structure, only six leading
//     bytes with particular second bytes can encode an out-of-range value; they are found by
//     byte tests on whole words (utf8_special_errors).  The transcoder, which decodes
//     every position anyway, range-checks the decoded 16-bit values instead.
// UTF-16 (Section 3): a word in D800-DBFF must be followed by one in DC00-DFFF and a word
// in DC00-DFFF must follow one in D800-DBFF.
#pragma once

#include <stdint.h>

#include "gbu_device.cuh"

namespace gbu {

struct Flags8 {
  uint32_t isC, geC0, geE0, geF0;
};

// Per byte (as bit 7 of each byte): continuation 10xxxxxx, >= C0, >= E0, >= F0.
__device__ __forceinline__ Flags8 classify8(uint32_t w) {
  Flags8 f;
  const uint32_t s1 = w << 1;
  f.geC0 = w & s1 & 0x80808080u;
  f.isC = w & ~s1 & 0x80808080u;
  f.geE0 = f.geC0 & (w << 2);
  f.geF0 = f.geE0 & (w << 3);
  return f;
}

// Bytes of word [c, c+4) whose virtual position lies in [lo, hi), as bit 7 of each byte.
__device__ __forceinline__ uint32_t byte_range_mask(long long c, long long lo, long long hi) {
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (c + j >= lo && c + j < hi) m |= 0x80u << (8 * j);
  return m;
}

// Byte selectors for a pair of positions (q, q+1), q = 0 or 2, inside W[k]:W[k+1].
__device__ __forceinline__ uint32_t selE(int h) { return h ? 0x3322u : 0x1100u; }
__device__ __forceinline__ uint32_t selO(int h) { return h ? 0x4433u : 0x2211u; }
__device__ __forceinline__ uint32_t selM(int h) { return h ? 0xBBAAu : 0x9988u; }

// Rules 1-3 for the 16 bytes W[1..4], given the word before (W[0]).  Nonzero = error.
__device__ __forceinline__ uint32_t utf8_structure_errors(const Flags8 f[5]) {
  uint32_t err = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t req = __funnelshift_l(f[k].geC0, f[k + 1].geC0, 8) |
                         __funnelshift_l(f[k].geE0, f[k + 1].geE0, 16) |
                         __funnelshift_l(f[k].geF0, f[k + 1].geF0, 24);
    err |= req ^ f[k + 1].isC;
  }
  return err;
}

// Rules 4-6 (and rule 1 for F8-FF) for the 16 bytes W[1..4], with W[5] the word after and
// f[1..4] their classification, as byte tests on whole words.  With the structure (rules 1-3)
// already checked, the value of a sequence can only be out of range for these leading bytes
// and second bytes: C0 or C1 (overlong), E0 then 80-9F (overlong), ED then A0-BF (D800-DFFF),
// F0 then 80-8F (overlong), F4 then 90-BF or F5-FF (above U+10FFFF; F8-FF also break rule
// 1).  Each test looks at a byte's low bits and, for E0/ED and F0/F4, at the byte after it
// (N = the stream shifted by one byte); the per-byte sums below never carry into the next
// byte.  Nonzero = some position of the chunk starts such a sequence (the caller only needs
// to know that the chunk holds an error; the kind and offset are resolved separately).
// has2/has3/has4: whether the warp has two-, three-, four-byte leading bytes at all (absent
// classes cost nothing).
__device__ __forceinline__ uint32_t utf8_special_errors(const uint32_t W[6], const Flags8 f[5], bool has2, bool has3,
                                                        bool has4) {
  uint32_t bad = 0;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const uint32_t w = W[k];
    const uint32_t n = __funnelshift_r(W[k], W[k + 1], 8);  // byte j: the byte after byte j
    // C0/C1: a leading byte >= C0 whose bits 5-1 are zero
    if (has2) bad |= f[k].geC0 & ~((w & 0x3E3E3E3Eu) + 0x7F7F7F7Fu);
    if (has3) {
      // E0-EF with low nibble 0 and next byte 80-9F, or low nibble D and next byte A0-BF:
      // with y = 1 where the next byte has bit 5 set, exactly where (nibble ^ 0D*y) is zero
      const uint32_t y = (n >> 5) & 0x01010101u;
      const uint32_t q = (w & 0x0F0F0F0Fu) ^ (y * 0x0Du);
      bad |= f[k].geE0 & ~f[k].geF0 & ~(q + 0x7F7F7F7Fu);
    }
    if (has4) {
      // F0-FF with low nibble 0 and next byte 80-8F, or nibble 4 and next byte 90-BF
      // (y4 = 4 where the next byte has bit 4 or 5 set: (nibble ^ y4) is zero), or nibble >= 5
      const uint32_t y4 = ((n >> 2) | (n >> 3)) & 0x04040404u;
      const uint32_t L = w & 0x0F0F0F0Fu;
      bad |= f[k].geF0 & (~((L ^ y4) + 0x7F7F7F7Fu) | (L + 0x7B7B7B7Bu));
    }
  }
  return bad;
}

// UTF-16 words of the chunk's positions inside [lo, hi) (length formula: one per byte that is
// not a continuation byte, one more per byte F0-FF).
__device__ __forceinline__ uint32_t utf8_count_units(const Flags8 f[5], long long c, bool edge,
                                                     long long lo, long long hi) {
  // flags sit in bit 7 of each byte: a byte dot product with 0x01 weights adds 0x80 per flag
  // (FMA pipe, where a population count would take the slower XU pipe)
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t vm = edge ? byte_range_mask(c + 4 * k, lo, hi) : 0x80808080u;
    acc = __dp4a(~f[k + 1].isC & vm, 0x01010101u, acc);
    acc = __dp4a(f[k + 1].geF0 & vm, 0x01010101u, acc);
  }
  return acc >> 7;
}

__device__ __forceinline__ bool is_high16(uint32_t w) { return (w & 0xFC00u) == 0xD800u; }
__device__ __forceinline__ bool is_low16(uint32_t w) { return (w & 0xFC00u) == 0xDC00u; }

// UTF-8 bytes of one word for the length function (2 per surrogate word).
__device__ __forceinline__ uint32_t len8_of_word(uint32_t w) {
  return w < 0x80u ? 1u : (w < 0x800u ? 2u : ((w & 0xF800u) == 0xD800u ? 2u : 3u));
}

// ---- two UTF-16 words per 32-bit register ------------------------------------------------
// Bit 15 of each 16-bit lane of the result is set where that word is >= 0x80, >= 0x800 or a
// surrogate (D800-DFFF).  No addition carries out of a lane (bit 15 is masked off first and
// the sums stay below 0x10000).
__device__ __forceinline__ uint32_t lanes16_nonzero(uint32_t t) {
  return (((t & 0x7FFF7FFFu) + 0x7FFF7FFFu) | t) & 0x80008000u;
}
__device__ __forceinline__ uint32_t lanes16_ge80(uint32_t X) {
  return (((X & 0x7FFF7FFFu) + 0x7F807F80u) | X) & 0x80008000u;
}
__device__ __forceinline__ uint32_t lanes16_ge800(uint32_t X) {
  return (((X & 0x7FFF7FFFu) + 0x78007800u) | X) & 0x80008000u;
}
__device__ __forceinline__ uint32_t lanes16_sur(uint32_t X) {
  return ~lanes16_nonzero((X & 0xF800F800u) ^ 0xD800D800u) & 0x80008000u;
}

// UTF-8 bytes of the 8 words of a chunk inside the buffer: one per word, one more per word
// >= 0x80 and one more per word >= 0x800, one less per surrogate (Section 3 sizes; a pair
// counts 2 + 2).  The flags are summed by byte dot products (0x80 per flag, FMA pipe).
__device__ __forceinline__ uint32_t utf16_len8_inside(const uint32_t W[4]) {
  uint32_t acc = 0, sub = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    acc = __dp4a(lanes16_ge80(W[k]), 0x01000100u, acc);
    acc = __dp4a(lanes16_ge800(W[k]), 0x01000100u, acc);
    sub = __dp4a(lanes16_sur(W[k]), 0x01000100u, sub);
  }
  return 8u + ((acc - sub) >> 7);
}

// Unpaired surrogates among the 8 words of a chunk inside the buffer, given the word before
// (prevw's high half) and after (nextw's low half): a first surrogate whose next word is not
// a second one, or a second surrogate whose previous word is not a first one.  The surrogate
// flags are computed once per word and split by bit 10 (clear: first surrogate D800-DBFF,
// set: second DC00-DFFF).
__device__ __forceinline__ bool utf16_pair_errors_inside(const uint32_t W[4], uint32_t prevw, uint32_t nextw) {
  uint32_t H[5], L[5];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t S = lanes16_sur(W[k]);
    const uint32_t b10 = W[k] << 5;  // bit 10 of each word at bit 15
    H[k + 1] = S & ~b10;
    L[k] = S & b10;
  }
  H[0] = lanes16_sur(prevw) & ~(prevw << 5);
  L[4] = lanes16_sur(nextw) & (nextw << 5);
  uint32_t err = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t low_after = __funnelshift_r(L[k], L[k + 1], 16);   // word i+1's flag at word i
    const uint32_t high_before = __funnelshift_l(H[k], H[k + 1], 16);  // word i-1's flag at word i
    err |= (H[k + 1] & ~low_after) | (L[k] & ~high_before);
  }
  return err != 0;
}

// Surrogate flags of the four bytes of P (bit 7 of each byte): the byte is D8-DF, i.e. it is
// the high byte of a surrogate word.  Exact per byte (a zero-byte test on (b & F8) ^ D8).
__device__ __forceinline__ uint32_t bytes_sur(uint32_t P) {
  const uint32_t t = (P & 0xF8F8F8F8u) ^ 0xD8D8D8D8u;
  return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
}

// The high bytes of the 8 words of a chunk, four to a register in word order (the high byte
// of a UTF-16LE word is its second byte).
__device__ __forceinline__ void utf16_high_bytes(const uint32_t W[4], uint32_t &P0, uint32_t &P1) {
  P0 = __byte_perm(W[0], W[1], 0x7531);
  P1 = __byte_perm(W[2], W[3], 0x7531);
}

// Unpaired surrogates among the 8 words of a chunk inside the buffer, judged on the words'
// high bytes alone (a word is a surrogate exactly when its high byte is D8-DF, a first one
// when that byte's bit 2 is clear).  S0, S1: bytes_sur of the high bytes P0, P1; prevw's
// high half and nextw's low half are the words before and after the chunk.  The pair rule
// for two adjacent words a, b is: a is a first surrogate exactly when b is a second one, so
// one XOR per pair judges the nine pairs from (word before, first word) to (last word, word
// after).  A pair across a chunk boundary is judged by both chunks; the smaller chunk start
// is the one the first-error search keeps, and it scans on from there.
__device__ __forceinline__ bool utf16_pair_errors_bytes(uint32_t P0, uint32_t P1, uint32_t S0, uint32_t S1,
                                                        uint32_t prevw, uint32_t nextw) {
  const uint32_t Pe = __byte_perm(prevw, nextw, 0x3445);  // byte 0: the word after; byte 3: the word before
  const uint32_t Se = bytes_sur(Pe) & 0x80000080u;
  const uint32_t b0 = P0 << 5, b1 = P1 << 5, be = Pe << 5;  // bit 2 of each byte at bit 7
  const uint32_t H0 = S0 & ~b0, L0 = S0 & b0, H1 = S1 & ~b1, L1 = S1 & b1;
  const uint32_t He = Se & ~be, Le = Se & be;
  // word i's second-surrogate flag against word i-1's first-surrogate flag, i = 0..7, then
  // the word after against the last word
  uint32_t err = L0 ^ __funnelshift_l(He, H0, 8);
  err |= L1 ^ __funnelshift_l(H0, H1, 8);
  err |= (Le & 0x80u) ^ (H1 >> 24);
  return err != 0;
}

// Unpaired surrogates among the 8 words of a chunk, given the word before (prevw's high
// half) and after (nextw's low half); words outside [lo, hi) are not judged.
__device__ __forceinline__ bool utf16_chunk_errors(const uint32_t W[4], uint32_t prevw,
                                                   uint32_t nextw, long long c, bool edge,
                                                   long long lo, long long hi) {
  if (!edge) {
    uint32_t P0, P1;
    utf16_high_bytes(W, P0, P1);
    const uint32_t S0 = bytes_sur(P0), S1 = bytes_sur(P1);
    return (S0 | S1) != 0 && utf16_pair_errors_bytes(P0, P1, S0, S1, prevw, nextw);
  }
  // fast exit: no surrogate word in the chunk, and the word before is not a first surrogate
  // followed by our first word (that one is judged by the chunk that owns it)
  const uint32_t any = (W[0] | W[1] | W[2] | W[3]);
  uint32_t u[10];
  u[0] = prevw >> 16;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    u[1 + 2 * k] = W[k] & 0xFFFFu;
    u[2 + 2 * k] = W[k] >> 16;
  }
  u[9] = nextw & 0xFFFFu;
  if ((any & 0x80008000u) == 0) return false;  // all words below 0x8000: no surrogates
  bool err = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t w = u[j + 1];
    const bool valid = !edge || (c + 2 * j >= lo && c + 2 * j < hi);
    err |= valid && ((is_high16(w) && !is_low16(u[j + 2])) || (is_low16(w) && !is_high16(u[j])));
  }
  return err;
}

// ---- exact first error (single thread, only when an error was flagged) --------------------

// `chunk` is the smallest start (in code units of src) of a 16-byte chunk that failed a
// check.  Every check flags a position at most 3 bytes after the start of the ill-formed
// sequence it belongs to, and nothing before the first error is flagged, so the first error
// starts in [chunk - 3, chunk + 15].  Decoding in reading order from a character start at or
// before chunk - 3 finds it; the kind is the first rule the bytes read so far break.
static __device__ __noinline__ void resolve_utf8_error(const uint8_t *s, uint64_t n, long long chunk,
                                                       int32_t *kind, uint64_t *off) {
  long long q = chunk - 3;
  if (q < 0) q = 0;
  if (q > (long long)n) q = (long long)n;
  for (int k = 0; k < 4 && q > 0 && (q >= (long long)n || (s[q] & 0xC0) == 0x80); ++k) --q;
  uint64_t i = (uint64_t)q;
  const uint64_t stop = (uint64_t)(chunk + 64) < n ? (uint64_t)(chunk + 64) : n;
  while (i < stop) {
    const uint32_t b = s[i];
    if (b < 0x80) { ++i; continue; }
    int32_t k = GBU_OK;
    if (b < 0xC0) k = GBU_TOO_LONG;
    else if (b >= 0xF8) k = GBU_HEADER_BITS;
    else if (b < 0xC2) k = GBU_OVERLONG;
    else if (b >= 0xF5) k = GBU_TOO_LARGE;
    if (k != GBU_OK) { *kind = k; *off = i; return; }
    const int len = b >= 0xF0 ? 4 : (b >= 0xE0 ? 3 : 2);
    if (i + 1 >= n || (s[i + 1] & 0xC0) != 0x80) { *kind = GBU_TOO_SHORT; *off = i; return; }
    const uint32_t c1 = s[i + 1];
    if ((b == 0xE0 && c1 < 0xA0) || (b == 0xF0 && c1 < 0x90)) k = GBU_OVERLONG;
    else if (b == 0xED && c1 >= 0xA0) k = GBU_SURROGATE;
    else if (b == 0xF4 && c1 >= 0x90) k = GBU_TOO_LARGE;
    if (k != GBU_OK) { *kind = k; *off = i; return; }
    for (int j = 2; j < len; ++j)
      if (i + j >= n || (s[i + j] & 0xC0) != 0x80) { *kind = GBU_TOO_SHORT; *off = i; return; }
    i += len;
  }
  // Not reached for a real error (the flagged chunk always holds or follows the first error).
  *kind = GBU_TOO_SHORT;
  *off = chunk < 0 ? 0 : (uint64_t)chunk;
}

// UTF-16: a word is flagged exactly when it is the first word of an ill-formed sequence, so
// the first error lies in the flagged chunk [chunk, chunk + 8).  BE: the words lie in memory
// with their bytes in big-endian order.
template <bool BE = false>
static __device__ __noinline__ void resolve_utf16_error(const uint16_t *s, uint64_t n, long long chunk,
                                                        uint64_t *off) {
  auto word = [&](long long i) -> uint32_t {
    const uint32_t w = s[i];
    return BE ? ((w >> 8) | ((w & 0xFFu) << 8)) : w;
  };
  long long i = chunk < 0 ? 0 : chunk;
  if (i > 0 && i < (long long)n && is_low16(word(i)) && is_high16(word(i - 1))) --i;
  const long long stop = (chunk + 64) < (long long)n ? chunk + 64 : (long long)n;
  while (i < stop) {
    const uint32_t w = word(i);
    if ((w & 0xF800u) != 0xD800u) { ++i; continue; }
    if (is_high16(w) && i + 1 < (long long)n && is_low16(word(i + 1))) { i += 2; continue; }
    *off = (uint64_t)i;
    return;
  }
  *off = chunk < 0 ? 0 : (uint64_t)chunk;  // not reached for a real error
}

}  // namespace gbu
