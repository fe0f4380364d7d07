// gbu_wide_utf8.cuh -- the UTF-8 -> UTF-16LE codec (validating) of the wide partition loop
// (gbu_wide.cuh): a lane validates and converts 32 consecutive bytes.
//
// Paper Section 3 defines both formats; Section 5 states that transcoding validates.  A lane
// treats its 32 bytes as eight 32-bit words and works on four byte positions at a time:
//   * classification and rules 1-6 as in gbu_chunk.cuh (lead and continuation flags in bit 7
//     of each byte; structure by funnel-shifted lead flags; values by word-level byte tests of
//     the special leading bytes);
//   * decoding keeps the output word of every position as two byte planes, its high byte H and
//     low byte L, each computed for four positions per operation from the position's byte and
//     the one or two bytes after it (S1, S2 = the byte stream moved by one and two positions):
//       two bytes   110abcde 10fghijk      -> H = 00000abc,  L = de fghijk
//       three bytes 1110abcd 10efghij 10k.. -> H = abcd efgh, L = ij k.....
//     and for a four-byte sequence the two surrogates (the first as D7C0 + the code point's
//     bits 20-10, the second as DC00 + its bits 9-0);
//   * PRMT interleaves H and L into 16-bit words, and each non-continuation byte stores its word
//     (a four-byte leading byte two) at the lane's running staging index, through 32-bit
//     shared-memory addresses.
// A lane that breaks a rule reports its start; the last CTA turns the smallest one into the
// exact offset and kind (resolve_utf8_error).
#pragma once

#include <stdint.h>

#include "gbu_codec_utf8.cuh"
#include "gbu_wide.cuh"

namespace gbu {

// Byte mask (0xFF where bit 7 of the byte of x is set).
__device__ __forceinline__ uint32_t byte_mask(uint32_t x) { return prmt(x, 0u, 0xBA98u); }

// The 16-bit word of position j (0..3) from the byte planes L and H.
__device__ __forceinline__ uint32_t plane_word(uint32_t L, uint32_t H, int j) {
  return __byte_perm(L, H, (uint32_t)(j | ((4 + j) << 4)));
}

struct Utf8ToUtf16Wide {
  using Out = uint16_t;
  using Narrow = Utf8ToUtf16;
  // A valid 1 KiB region yields at most 1024 words, +1 for a four-byte leading byte in its last
  // byte.  A lane that breaks a rule can count up to 64 words while every lane before it is
  // valid, so a lane's own staging always fits: 32 x 31 + 1 + 64, plus 7 words of alignment
  // offset, <= WSTAGE.  Words past the buffer can only come after the first error.
  static constexpr uint32_t WSTAGE = 1024 + 48;
  static_assert(32 * 31 + 1 + 64 + 7 <= WSTAGE, "staging buffer too small");

  static constexpr uint32_t F_NONASCII = Narrow::F_NONASCII;
  static constexpr uint32_t F_C2 = Narrow::F_C2;
  static constexpr uint32_t F_C3 = Narrow::F_C3;
  static constexpr uint32_t F_C4 = Narrow::F_C4;

  static constexpr uint32_t ASCII_MASK = 0x80808080u;  // nonzero in a word: a byte >= 0x80
  static constexpr uint32_t LANE_UNITS = 32;            // words out of 32 ASCII bytes
  static constexpr uint32_t WREGION_UNITS = 1024;       // words out of an all-ASCII region
  static constexpr uint32_t WDIRECT_ALIGN = 8;          // its lanes store 32 words (64 bytes) each

  __device__ __forceinline__ static bool wascii_region(uint32_t, uint32_t rflags) { return rflags == 0; }

  // Rule 2 across the region's start: a leading byte in the word before it that wants
  // continuation bytes inside it (the region's bytes are all ASCII).  Lane 0 only.
  __device__ __forceinline__ static void check_prev_lead(uint32_t prev, long long c, unsigned long long &err_pos) {
    const Flags8 fp = classify8(prev);
    const uint32_t req = __funnelshift_l(fp.geC0, 0u, 8) | __funnelshift_l(fp.geE0, 0u, 16) |
                         __funnelshift_l(fp.geF0, 0u, 24);
    if (req && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
  }

  // An all-ASCII region inside the buffer whose output starts at dst, 16-byte aligned: each
  // lane widens its 32 bytes and stores them with two 32-byte stores (or four 16-byte ones)
  // (Section 4's ASCII path).  The 32-byte stores carry an evict-first L2 policy: the output,
  // twice the input, would otherwise push out of L2 the input lines the count pass has read
  // for the conversion to read again.
  __device__ __forceinline__ static void wascii_direct(uint16_t *dst, const uint32_t W[8], uint32_t prev, long long c,
                                                       unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) check_prev_lead(prev, c, err_pos);
    uint4 q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      q[i] = make_uint4(__byte_perm(W[2 * i], 0, 0x4140), __byte_perm(W[2 * i], 0, 0x4342),
                        __byte_perm(W[2 * i + 1], 0, 0x4140), __byte_perm(W[2 * i + 1], 0, 0x4342));
    uint4 *d = reinterpret_cast<uint4 *>(dst) + 4 * lane;
    if (((uintptr_t)dst & 31) == 0) {
      const uint64_t pol = l2_policy_last_use();
      st_global_32B_hint(d, q[0], q[1], pol);
      st_global_32B_hint(d + 2, q[2], q[3], pol);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) d[i] = q[i];
    }
  }

  // UTF-16 words of the lane's 32 bytes (one per byte that is not a continuation byte, one
  // more per byte F0-FF: the length formula) and the leading-byte classes present.
  __device__ __forceinline__ static uint32_t wcount(const Params &p, const uint32_t W[8], long long c, bool edge,
                                                    uint32_t &flags) {
    uint32_t any = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) any |= W[k];
    if (!edge && (any & 0x80808080u) == 0) {  // all ASCII
      flags = 0;
      return 32;
    }
    // per byte, as bit 7: not a continuation byte (10xxxxxx), >= C0, >= E0 and >= F0.  Byte dot
    // products with 0x01 weights (FMA pipe) add 0x80 per flag; the leading-byte classes follow
    // from the sums (C0-DF present when there are more bytes >= C0 than >= E0, and so on), so
    // the integer ALU does four logic operations per word
    uint32_t an = 0, aG = 0, aE = 0, aF = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t w = W[k], s1 = w * 2u, s2 = w * 4u, s3 = w * 8u;
      const uint32_t vm = edge ? byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes) : 0x80808080u;
      const uint32_t ge = w & s1 & vm;  // >= C0
      const uint32_t gE = ge & s2;      // >= E0
      const uint32_t f0 = gE & s3;      // >= F0
      an = __dp4a((~w | s1) & vm, 0x01010101u, an);
      aG = __dp4a(ge, 0x01010101u, aG);
      aE = __dp4a(gE, 0x01010101u, aE);
      aF = __dp4a(f0, 0x01010101u, aF);
    }
    flags = F_NONASCII | (aG > aE ? F_C2 : 0u) | (aE > aF ? F_C3 : 0u) | (aF ? F_C4 : 0u);
    return (an + aF) >> 7;
  }

  // Validates the lane's 32 bytes W[1..8] (W[0] the word before, W[9] the word after) of a
  // region that lies inside the buffer and whose output fits the staging buffer, and stages
  // their words from shared address sa on; returns nonzero when a rule is broken.  H2 / H3 /
  // H4: leading bytes C0-DF / E0-EF / F0-FF occur in the region or in bytes 1-3 of the word
  // before it (the code for an absent class is left out).  Each non-continuation byte stores
  // one word (a four-byte leading byte two), the count the count pass gave the lane.
  template <bool H2, bool H3, bool H4>
  __device__ __forceinline__ static uint32_t wconvert_fast(const uint32_t W[10], uint32_t sa) {
    // with a single class present, every byte >= C0 is a leading byte of that class; without
    // H4 there is no byte >= F0
    constexpr bool ONE = (int)H2 + (int)H3 + (int)H4 == 1;
    uint32_t bad = 0;
    // lead flags of the word before (bytes 1-3 reach into the lane's bytes)
    uint32_t pg, pE = 0, pF = 0;
    {
      const uint32_t w = W[0];
      pg = w & (w << 1) & 0x80808080u;
      if (H3 || H4) pE = ONE ? pg : pg & (w << 2);
      if (H4) pF = ONE ? pg : pE & (w << 3);
    }
#pragma unroll
    for (int k = 1; k <= 8; ++k) {
      const uint32_t w = W[k], wn = W[k + 1];
      const uint32_t s1 = w << 1;
      const uint32_t g = w & s1 & 0x80808080u;     // >= C0
      const uint32_t isC = w & ~s1 & 0x80808080u;  // continuation byte
      uint32_t gE = 0, gF = 0;
      if (H3 || H4) gE = ONE ? g : g & (w << 2);   // >= E0
      if (H4) gF = ONE ? g : gE & (w << 3);        // >= F0
      // rules 1-3: a byte is a continuation exactly when a leading byte 1, 2 or 3 back wants it
      uint32_t req = __funnelshift_l(pg, g, 8);
      if (H3 || H4) req |= __funnelshift_l(pE, gE, 16);
      if (H4) req |= __funnelshift_l(pF, gF, 24);
      bad |= req ^ isC;
      pg = g;
      pE = gE;
      pF = gF;

      const uint32_t S1 = __funnelshift_r(w, wn, 8);  // byte j: the byte after byte j
      const uint32_t wF = w & 0x0F0F0F0Fu;
      // rules 4-6 for the special leading bytes (see utf8_special_errors)
      if (H2) bad |= g & ~((w & 0x3E3E3E3Eu) + 0x7F7F7F7Fu);  // C0, C1
      if (H3) {
        const uint32_t y = (S1 >> 5) & 0x01010101u;
        const uint32_t q = wF ^ (y * 0x0Du);
        bad |= (ONE ? g : gE & ~gF) & ~(q + 0x7F7F7F7Fu);  // E0 + 80..9F, ED + A0..BF
      }
      if (H4) {
        const uint32_t y4 = ((S1 >> 2) | (S1 >> 3)) & 0x04040404u;
        bad |= gF & (~((wF ^ y4) + 0x7F7F7F7Fu) | (wF + 0x7B7B7B7Bu));  // F0 + 80..8F, F4 + 90..BF, F5..FF
      }

      // byte planes of the output words
      uint32_t L = w, H = 0, Lls = 0, Hls = 0;
      uint32_t S2 = 0;
      if (H3 || H4) S2 = __funnelshift_r(w, wn, 16);
      if (H2) {
        const uint32_t L2 = (w & 0x03030303u) * 64u + (S1 & 0x3F3F3F3Fu);
        const uint32_t H2v = (w >> 2) & 0x07070707u;
        const uint32_t M2 = byte_mask(ONE ? g : g & ~gE);
        L = (L2 & M2) | (L & ~M2);
        H = H2v & M2;
      }
      if (H3) {
        const uint32_t L3 = (S1 & 0x03030303u) * 64u + (S2 & 0x3F3F3F3Fu);
        const uint32_t H3v = wF * 16u + ((S1 >> 2) & 0x0F0F0F0Fu);
        const uint32_t M3 = byte_mask(ONE ? g : (H4 ? gE & ~gF : gE));
        L = (L3 & M3) | (L & ~M3);
        H = (H3v & M3) | (H & ~M3);
      }
      if (H4) {
        const uint32_t S3 = __funnelshift_r(w, wn, 24);
        const uint32_t M4 = byte_mask(gF);
        // second surrogate: DC00 | (third byte & 0F) << 6 | (fourth byte & 3F)
        Lls = (S2 & 0x03030303u) * 64u + (S3 & 0x3F3F3F3Fu);
        Hls = ((S2 >> 2) & 0x03030303u) | 0xDCDCDCDCu;
        // first surrogate: D7C0 + ((lead & 7) << 8 | Y), Y = (second & 3F) << 2 | (third >> 4) & 3;
        // Y is cleared outside F0-FF positions, so the per-byte sums below carry at most into
        // the byte after a leading byte (a continuation position, which stores nothing)
        const uint32_t Y = ((S1 & 0x3F3F3F3Fu) * 4u + ((S2 >> 4) & 0x03030303u)) & M4;
        const uint32_t cy = ((Y | (Y << 1)) >> 7) & 0x01010101u;  // Y >= 0x40: the low byte wraps
        const uint32_t Lhs = Y + 0xC0C0C0C0u;
        const uint32_t Hhs = (w & 0x07070707u) + cy + 0xD7D7D7D7u;
        L = (Lhs & M4) | (L & ~M4);
        H = (Hhs & M4) | (H & ~M4);
      }
      // stage the words of the non-continuation bytes (and the second surrogates)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t bit = 0x80u << (8 * j);
        sts_u16_if_clear<2>(sa, plane_word(L, H, j), isC, bit);
        if (H4) sts_u16_if_set<2>(sa, plane_word(Lls, Hls, j), gF, bit);
      }
    }
    return bad;
  }

  // Validates the lane's 32 bytes and stages their UTF-16 words.  x0 (the lane's offset in
  // the region), rtot and rflags come from the count pass.
  __device__ __forceinline__ static Region wconvert(const Params &p, const uint32_t W[8], uint32_t prev,
                                                    uint32_t next, long long c, bool edge, bool inside, uint16_t *st,
                                                    uint32_t base, uint32_t x0, uint32_t rtot, uint32_t rflags,
                                                    unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    const uint32_t sbase = smem_addr(st);
    if (rflags == 0) {
      // an all-ASCII region: one word per byte; the only possible error is a leading byte
      // just before the region that wants continuation bytes inside it (lane 0's bytes)
      if (lane == 0) check_prev_lead(prev, c, err_pos);
      const uint32_t x = base + 32 * lane;
      const uint32_t a = sbase + 2 * x;
      if ((x & 7) == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          sts_v4(a + 16 * i, __byte_perm(W[2 * i], 0, 0x4140), __byte_perm(W[2 * i], 0, 0x4342),
                 __byte_perm(W[2 * i + 1], 0, 0x4140), __byte_perm(W[2 * i + 1], 0, 0x4342));
      } else if ((x & 1) == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          sts_u32(a + 8 * k, __byte_perm(W[k], 0, 0x4140));
          sts_u32(a + 8 * k + 4, __byte_perm(W[k], 0, 0x4342));
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int j = 0; j < 4; ++j) sts_u16(a + 8 * k + 2 * j, (W[k] >> (8 * j)) & 0xFFu);
      }
      return Region{1024u, 0u, 0u, 1024u};
    }
    if (inside && base + rtot <= WSTAGE) {
      const uint32_t Wx[10] = {prev, W[0], W[1], W[2], W[3], W[4], W[5], W[6], W[7], next};
      // the leading-byte classes: the region's own (from the count pass) and those of bytes
      // 1-3 of the word before it (a sequence starting there reaches into the region, and the
      // structure test reads those bytes)
      const uint32_t pc = lane == 0 ? Narrow::lead_classes(prev, 0x80808000u) : 0u;
      const uint32_t cls = rflags | __shfl_sync(0xffffffffu, pc, 0);
      const bool h2 = cls & F_C2, h3 = cls & F_C3, h4 = cls & F_C4;
      const uint32_t sa = sbase + 2 * (base + x0);
      uint32_t bad;
      if (h4) {
        bad = (h2 || h3) ? wconvert_fast<true, true, true>(Wx, sa) : wconvert_fast<false, false, true>(Wx, sa);
      } else if (h3) {
        bad = h2 ? wconvert_fast<true, true, false>(Wx, sa) : wconvert_fast<false, true, false>(Wx, sa);
      } else {
        bad = h2 ? wconvert_fast<true, false, false>(Wx, sa) : wconvert_fast<true, true, true>(Wx, sa);
      }
      if (bad && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
      return Region{rtot, 0u, 0u, rtot};
    }
    const Narrow::General r = wconvert_general(p, make_uint4(W[0], W[1], W[2], W[3]),
                                               make_uint4(W[4], W[5], W[6], W[7]), prev, next, c, edge, st, base,
                                               x0, rtot, err_pos);
    err_pos = r.err_pos;
    return r.g;
  }

  // A region at a buffer end (or one whose output overflows the staging buffer, which only
  // happens after an error): the 16-byte general path of the narrow codec on each half of the
  // lane's bytes (A, B).
  __device__ __forceinline__ static Narrow::General wconvert_general(const Params &p, uint4 A, uint4 B, uint32_t prev,
                                                                  uint32_t next, long long c, bool edge, uint16_t *st,
                                                                  uint32_t base, uint32_t x0, uint32_t rtot,
                                                                  unsigned long long err_pos) {
    const long long lo = p.off0, hi = (long long)p.vbytes;
    uint32_t fa;
    const uint32_t na = Narrow::count(p, A, c, edge, fa);
    const Narrow::General ra = Narrow::convert_general_body(lo, hi, A, prev, B.x, c, edge, st, base, x0, rtot, err_pos, WSTAGE);
    return Narrow::convert_general_body(lo, hi, B, A.w, next, c + 16, edge, st, base, x0 + na, rtot, ra.err_pos, WSTAGE);
  }
};

}  // namespace gbu
