// gbu_wide_utf16.cuh -- the UTF-16LE -> UTF-8 codec (validating) of the wide partition loop
// (gbu_wide.cuh): a lane validates and converts 16 consecutive words (32 bytes).
//
// Paper Section 3: words 0000-D7FF and E000-FFFF are characters by themselves; a word in
// D800-DBFF must be followed by one in DC00-DFFF and the pair encodes
// ((first & 0x3FF) << 10 | (second & 0x3FF)) + 0x10000.  The UTF-8 sizes are 1 byte below
// 0x80, 2 below 0x800, 3 otherwise, and 2 per surrogate word (a pair's first word writes all 4
// bytes, over its own 2 slots and its partner's).  Section 4 routes whole registers by range;
// here the routes are taken per warp region from the count pass's flags: all ASCII (words
// narrowed to bytes), one and two bytes, no surrogates, ASCII and pairs only (emoji-heavy
// text), and the general pair route.  Words are encoded one at a time into the warp's staging
// buffer through 32-bit shared-memory addresses.
#pragma once

#include <stdint.h>

#include "gbu_codec_utf16.cuh"
#include "gbu_wide.cuh"

namespace gbu {

struct Utf16ToUtf8Wide {
  using Out = uint8_t;
  using Narrow = Utf16ToUtf8;
  // a region of 512 words yields at most 1536 bytes, +2 for a pair cut at its end, plus 15
  // bytes of alignment offset
  static constexpr uint32_t WSTAGE = 3 * 512 + 32;
  static_assert(3 * 512 + 2 + 15 + 1 <= WSTAGE, "staging buffer too small");

  static constexpr uint32_t F_SUR = Narrow::F_SUR;
  static constexpr uint32_t F_THREE = Narrow::F_THREE;
  static constexpr uint32_t F_WIDE = Narrow::F_WIDE;

  static constexpr uint32_t ASCII_MASK = 0xFF80FF80u;  // nonzero in a word: a word >= 0x80
  static constexpr uint32_t LANE_UNITS = 16;            // bytes out of 16 ASCII words
  static constexpr uint32_t WREGION_UNITS = 512;        // bytes out of an all-ASCII region
  static constexpr uint32_t WDIRECT_ALIGN = 16;         // its lanes store 16 bytes each

  // 512 words and 512 bytes: every word of an inside region is ASCII.
  __device__ __forceinline__ static bool wascii_region(uint32_t rtot, uint32_t) { return rtot == 512u; }

  // The low bytes of the lane's 16 words (all ASCII).
  __device__ __forceinline__ static uint4 narrow16(const uint32_t W[8]) {
    return make_uint4(__byte_perm(W[0], W[1], 0x6420), __byte_perm(W[2], W[3], 0x6420),
                      __byte_perm(W[4], W[5], 0x6420), __byte_perm(W[6], W[7], 0x6420));
  }

  // An all-ASCII region inside the buffer whose output starts at dst, 16-byte aligned: each
  // lane narrows its 16 words into one 16-byte store (Section 4's ASCII route).
  __device__ __forceinline__ static void wascii_direct(uint8_t *dst, const uint32_t W[8], uint32_t, long long,
                                                       unsigned long long &) {
    const int lane = threadIdx.x & 31;
    reinterpret_cast<uint4 *>(dst)[lane] = narrow16(W);
  }

  // UTF-8 bytes of the lane's 16 words and the route flags.  Inside the buffer the high bytes
  // of four words are gathered into one register (and their low bytes into another) and
  // tested four at a time: >= 0x80 (a nonzero high byte, or bit 7 of the low byte), >= 0x800
  // (high byte >= 08) and surrogate (high byte D8-DF); the flags, in bit 7 of each byte, are
  // summed by byte dot products.
  __device__ __forceinline__ static uint32_t wcount(const Params &p, const uint32_t W[8], long long c, bool edge,
                                                    uint32_t &flags) {
    if (!edge) {
      uint32_t any = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) any |= W[k];
      flags = 0;
      if ((any & ASCII_MASK) == 0) return 16;  // all ASCII
      uint32_t a80 = 0, a800 = 0, sub = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t hb = __byte_perm(W[2 * i], W[2 * i + 1], 0x7531);
        const uint32_t lb = __byte_perm(W[2 * i], W[2 * i + 1], 0x6420);
        const uint32_t g80 = (((hb & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | hb | lb) & 0x80808080u;
        const uint32_t g800 = (((hb & 0x78787878u) + 0x78787878u) | hb) & 0x80808080u;
        const uint32_t t = (hb & 0xF8F8F8F8u) ^ 0xD8D8D8D8u;
        const uint32_t sr = ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
        a80 = __dp4a(g80, 0x01010101u, a80);
        a800 = __dp4a(g800, 0x01010101u, a800);
        sub = __dp4a(sr, 0x01010101u, sub);
      }
      // every surrogate is >= 0x800: a80 - sub counts the words >= 0x80 that are not surrogates
      flags = (sub ? F_SUR : 0u) | (a800 ? F_THREE : 0u) | (a80 != sub ? F_WIDE : 0u);
      return 16u + ((a80 + a800 - sub) >> 7);
    }
    flags = F_SUR | F_THREE | F_WIDE;
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t w = (W[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
      const bool valid = c + 2 * j >= (long long)p.off0 && c + 2 * j < (long long)p.vbytes;
      cnt += valid ? len8_of_word(w) : 0u;
    }
    return cnt;
  }

  // Word j (0..15) of the lane.
  __device__ __forceinline__ static uint32_t word(const uint32_t W[8], int j) {
    return (j & 1) ? W[j >> 1] >> 16 : W[j >> 1] & 0xFFFFu;
  }

  // Staging stores, each a single PTX block whose predicates come from mask tests of the word
  // (one logic op each), so that ptxas emits predicated stores and adds and no branch.

  // One word of a register: its first byte b0 at o, and b1 at o+1 where (S & BIT) != 0; o
  // advances by the bytes written.
  template <uint32_t BIT>
  __device__ __forceinline__ static void sts_1or2(uint32_t &o, uint32_t S, uint32_t b0, uint32_t b1) {
    asm volatile(
        "{\n\t.reg .pred q;\n\t.reg .b32 t;\n\tand.b32 t, %1, %4;\n\tsetp.ne.b32 q, t, 0;\n\t"
        "st.shared.u8 [%0], %2;\n\t@q st.shared.u8 [%0+1], %3;\n\tadd.u32 %0, %0, 1;\n\t@q add.u32 %0, %0, 1;\n\t}"
        : "+r"(o)
        : "r"(S), "r"(b0), "r"(b1), "n"(BIT)
        : "memory");
  }

  // One word of a register: b0 at o, b1 at o+1 where (S1 & BIT) != 0, b2 at o+2 where
  // (S2 & BIT) != 0 (S1, S2: its >= 0x80 and >= 0x800 flags); o advances by the bytes written.
  template <uint32_t BIT>
  __device__ __forceinline__ static void sts_123m(uint32_t &o, uint32_t S1, uint32_t S2, uint32_t b0, uint32_t b1,
                                                  uint32_t b2) {
    asm volatile(
        "{\n\t.reg .pred q1, q2;\n\t.reg .b32 t1, t2;\n\tand.b32 t1, %1, %6;\n\tsetp.ne.b32 q1, t1, 0;\n\t"
        "and.b32 t2, %2, %6;\n\tsetp.ne.b32 q2, t2, 0;\n\t"
        "st.shared.u8 [%0], %3;\n\t@q1 st.shared.u8 [%0+1], %4;\n\t@q2 st.shared.u8 [%0+2], %5;\n\t"
        "add.u32 %0, %0, 1;\n\t@q1 add.u32 %0, %0, 1;\n\t@q2 add.u32 %0, %0, 1;\n\t}"
        : "+r"(o)
        : "r"(S1), "r"(S2), "r"(b0), "r"(b1), "r"(b2), "n"(BIT)
        : "memory");
  }

  __device__ __forceinline__ static Region wconvert(const Params &p, const uint32_t W[8], uint32_t prev,
                                                    uint32_t next, long long c, bool edge, bool inside, uint8_t *st,
                                                    uint32_t base, uint32_t x0, uint32_t rtot, uint32_t rflags,
                                                    unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    const uint32_t sbase = smem_addr(st);
    if (!inside) {
      // a region at a buffer end: the 16-byte generic path of the narrow codec on each half
      // (a pair cut by the region's start is judged by lane 0's first half, one cut by its end
      // by lane 31's second half)
      const uint4 A = make_uint4(W[0], W[1], W[2], W[3]), B = make_uint4(W[4], W[5], W[6], W[7]);
      uint32_t fa;
      const uint32_t na = Narrow::count(p, A, c, edge, fa);
      const Region ga = Narrow::convert_generic(p, A, prev, W[4], c, edge, st, base, x0, rtot, err_pos);
      const Region gb = Narrow::convert_generic(p, B, W[3], next, c + 16, edge, st, base, x0 + na, rtot, err_pos);
      return Region{rtot, ga.skip, gb.extra, rtot};
    }
    if (rtot == 512u) {
      // 512 words and 512 bytes: every word is ASCII (Section 4's ASCII route)
      const uint4 b = narrow16(W);
      const uint32_t x = base + 16 * lane;
      const uint32_t a = sbase + x;
      if ((x & 15) == 0) {
        sts_v4(a, b.x, b.y, b.z, b.w);
      } else if ((x & 3) == 0) {
        sts_u32(a, b.x);
        sts_u32(a + 4, b.y);
        sts_u32(a + 8, b.z);
        sts_u32(a + 12, b.w);
      } else {
        const uint32_t q[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 16; ++i) sts_u8(a + i, q[i >> 2] >> (8 * (i & 3)));
      }
      return Region{512u, 0u, 0u, 512u};
    }
    Region g{rtot, 0u, 0u, rtot};
    uint32_t o = sbase + base + x0;
    if (!(rflags & (F_SUR | F_THREE))) {
      // Only words below 0x800 (Section 4's one-and-two-byte route), two words per register:
      // per 16-bit lane, the first byte is the word itself or C0 | w >> 6, the second 80 | w & 3F.
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t X = W[k];
        const uint32_t g1 = lanes16_ge80(X);       // bit 15 of a lane: the word is >= 0x80
        const uint32_t G1 = prmt(g1, 0u, 0xBB99u);  // the same as a lane mask
        const uint32_t B0 = (((X >> 6) & 0x001F001Fu) | 0x00C000C0u) & G1 | (X & ~G1);
        const uint32_t B1 = (X & 0x003F003Fu) | 0x00800080u;
        sts_1or2<0x8000u>(o, g1, B0, B1);
        sts_1or2<0x80000000u>(o, g1, B0 >> 16, B1 >> 16);
      }
      return g;
    }
    if (!(rflags & F_SUR)) {
      // No surrogate in the region: every word is a character of one to three bytes, two words
      // per register.  Per 16-bit lane: the first byte is w, C0 | w >> 6 or E0 | w >> 12; the
      // second 80 | w & 3F (two bytes) or 80 | (w >> 6) & 3F (three); the third 80 | w & 3F.
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t X = W[k];
        const uint32_t g1 = lanes16_ge80(X), g2 = lanes16_ge800(X);
        const uint32_t G1 = prmt(g1, 0u, 0xBB99u), G2 = prmt(g2, 0u, 0xBB99u);
        const uint32_t A6 = X >> 6;
        const uint32_t T2 = (A6 & 0x001F001Fu) | 0x00C000C0u;
        const uint32_t T3 = ((X >> 12) & 0x000F000Fu) | 0x00E000E0u;
        const uint32_t B0 = (T3 & G2) | (((T2 & G1) | (X & ~G1)) & ~G2);
        const uint32_t B2 = (X & 0x003F003Fu) | 0x00800080u;
        const uint32_t B1 = (((A6 & 0x003F003Fu) | 0x00800080u) & G2) | (B2 & ~G2);
        sts_123m<0x8000u>(o, g1, g2, B0, B1, B2);
        sts_123m<0x80000000u>(o, g1, g2, B0 >> 16, B1 >> 16, B2 >> 16);
      }
      return g;
    }
    // Surrogates present.  A first surrogate followed by a second one writes all four bytes
    // of the pair (its two slots and its partner's); the second writes nothing.  A pair cut
    // by the region's end is written by this region (2 bytes past its end), a pair cut by
    // its start by the previous region.
    const uint32_t u0 = prev >> 16, u17 = next & 0xFFFFu;
    const bool cut_start = is_low16(word(W, 0)) && is_high16(u0);
    const bool cut_end = is_high16(word(W, 15)) && is_low16(u17);
    g.skip = __shfl_sync(0xffffffffu, cut_start ? 2u : 0u, 0);
    g.extra = __shfl_sync(0xffffffffu, cut_end ? 2u : 0u, 31);
    if (!(rflags & F_WIDE)) {
      // Only ASCII words and surrogates (emoji-heavy text), two words per register at a time.
      // An ASCII word writes its byte.  Each surrogate writes the two bytes of its own two
      // slots: a first surrogate (code point bits 20-12) F0 | t >> 8 and 80 | (t >> 2) & 3F with
      // t = (w & 3FF) + 40, a second one (bits 11-0) 80 | (w' & 3) << 4 | (w >> 6) & F and
      // 80 | w & 3F, w' the word before it.  For a valid pair that is its four bytes; an
      // unpaired surrogate is an error, and what it writes lies past the first error.
      uint32_t hprev = lanes16_sur(prev) & ~(prev << 5);  // the word before: a first surrogate (bit 31)
      uint32_t wprev = prev;
      uint32_t err = 0;
      uint32_t Lc = 0, Hc = 0;  // the current register's second- and first-surrogate flags
      {
        const uint32_t S = lanes16_sur(W[0]);
        Hc = S & ~(W[0] << 5);
        Lc = S & (W[0] << 5);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t X = W[k];
        // flags of the next register (for lane 31, the word after the region)
        uint32_t Hn, Ln;
        {
          const uint32_t Y = k < 7 ? W[k + 1] : (next & 0xFFFFu);
          const uint32_t S = lanes16_sur(Y);
          Hn = S & ~(Y << 5);
          Ln = S & (Y << 5);
        }
        // pair rules: a first surrogate must be followed by a second one, a second one preceded
        // by a first one (flags in bit 15 of each 16-bit lane)
        const uint32_t low_after = __funnelshift_r(Lc, Ln, 16);
        const uint32_t high_before = __funnelshift_l(hprev, Hc, 16);
        err |= (Hc & ~low_after) | (Lc & ~high_before);
        // both slot pairs of both words, as 16-bit lanes (low byte first)
        const uint32_t T = (X & 0x03FF03FFu) + 0x00400040u;
        const uint32_t hb0 = ((T >> 8) & 0x00070007u) | 0x00F000F0u;
        const uint32_t hb1 = ((T >> 2) & 0x003F003Fu) | 0x00800080u;
        const uint32_t HI = hb1 * 256u + hb0;
        const uint32_t Xp = __funnelshift_l(wprev, X, 16);  // each lane's word before
        const uint32_t lb2 = (Xp & 0x00030003u) * 16u + (((X >> 6) & 0x000F000Fu) | 0x00800080u);
        const uint32_t lb3 = (X & 0x003F003Fu) | 0x00800080u;
        const uint32_t LO = lb3 * 256u + lb2;
        const uint32_t Hm = prmt(Hc, 0u, 0xBB99u), Lm = prmt(Lc, 0u, 0xBB99u);
        const uint32_t R = (HI & Hm) | (LO & Lm) | (X & ~(Hm | Lm));
        const uint32_t Sc = Hc | Lc;
        sts_1or2<0x8000u>(o, Sc, R, R >> 8);
        sts_1or2<0x80000000u>(o, Sc, R >> 16, R >> 24);
        hprev = Hc;
        wprev = X;
        Hc = Hn;
        Lc = Ln;
      }
      // a pair cut by the region's end: lane 31 also writes its second half (2 bytes past the
      // region's end, as in the other routes)
      if (lane == 31 && is_high16(word(W, 15)) && is_low16(u17)) {
        sts_u8(o, 0x80u | ((word(W, 15) & 3u) << 4) | ((u17 >> 6) & 0xFu));
        sts_u8(o + 1, 0x80u | (u17 & 0x3Fu));
      }
      if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
      return g;
    }
    bool err = false;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t w = word(W, j);
      const uint32_t wp = j > 0 ? word(W, j - 1) : u0, wn = j < 15 ? word(W, j + 1) : u17;
      const bool g1 = w >= 0x80u, g2 = w >= 0x800u;
      const bool hs = is_high16(w), ls = is_low16(w);
      const bool pair = hs && is_low16(wn);
      const bool follows = ls && is_high16(wp);
      err |= (hs && !pair) || (ls && !follows);
      // the word's bytes: a pair's four, nothing for a pair's second word, else its one to
      // three (a lone surrogate takes the three-byte form)
      const uint32_t c6 = w & 0x3Fu, t6 = w >> 6;
      const uint32_t t = (w & 0x3FFu) + 0x40u;  // a pair's code point >> 10
      const uint32_t b0 = pair ? 0xF0u | (t >> 8) : (g2 ? 0xE0u + (w >> 12) : (g1 ? 0xC0u + t6 : w));
      const uint32_t b1 = pair ? 0x80u | ((t >> 2) & 0x3Fu) : (g2 ? 0x80u | (t6 & 0x3Fu) : 0x80u + c6);
      const uint32_t b2 = pair ? 0x80u | ((t & 3u) << 4) | ((wn >> 6) & 0xFu) : 0x80u + c6;
      const uint32_t nb = pair ? 4u : (follows ? 0u : 1u + (g1 ? 1u : 0u) + (g2 ? 1u : 0u));
      // nb = 0..4 bytes: byte i is stored where nb > i, i.e. where bit i of m = 0xF >> (4 - nb)
      // is set (tested by the fused stores)
      const uint32_t m = 0xFu >> (4u - nb);
      sts_u8_if_set<0>(o, b0, m, 1u);
      sts_u8_if_set<1>(o, b1, m, 2u);
      sts_u8_if_set<2>(o, b2, m, 4u);
      sts_u8_if_set<3>(o, 0x80u | (wn & 0x3Fu), m, 8u);
      o += (hs || ls) ? 2u : 1u + (g1 ? 1u : 0u) + (g2 ? 1u : 0u);
    }
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    return g;
  }
};

}  // namespace gbu
