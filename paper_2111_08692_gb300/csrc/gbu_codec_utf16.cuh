// gbu_codec_utf16.cuh -- the UTF-16LE -> UTF-8 codec (validating), used by the single-buffer
// transcoder (gbu_utf16.cu) and the batched kernels (gbu_batch.cu).
//
// Paper Section 3: words 0000-D7FF and E000-FFFF are characters by themselves; a word in
// D800-DBFF must be followed by one in DC00-DFFF and the pair encodes
// ((first & 0x3FF) << 10 | (second & 0x3FF)) + 0x10000.  Section 4 routes whole registers
// by range (all ASCII, all below 0x800, no surrogates, else a scalar fallback); here a warp
// handles a 512-byte region, 8 words (16 bytes) per lane:
//   * a word is in error when it is a first surrogate not followed by a second one, or a
//     second surrogate not preceded by a first one (neighbours come from adjacent lanes);
//   * UTF-8 sizes: 1 byte below 0x80, 2 below 0x800, 3 otherwise, and 2 per surrogate word:
//     the first word of a pair writes all 4 bytes of the character, over its own 2 slots and
//     its partner's, and the second word writes nothing.  A pair cut by a region boundary is
//     written by the region holding its first word (2 bytes past its end), and the next
//     region leaves its first 2 slots alone;
//   * an all-ASCII warp narrows words to bytes directly (Section 4's ASCII route);
//   * other words are encoded one at a time into the warp's staging buffer.
#pragma once

#include <stdint.h>

#include "gbu_chunk.cuh"
#include "gbu_device.cuh"
#include "gbu_xcode.cuh"

namespace gbu {

struct Utf16ToUtf8 {
  using Out = uint8_t;
  // a region of 256 words yields at most 768 bytes, +2 for a pair cut at its end, plus 15
  // bytes of alignment slack
  static constexpr uint32_t STAGE = 3 * 256 + 32;
  // the most a region stages: 256 words of 3 bytes (a pair: 2 + 2), 2 bytes of a pair cut at
  // its end, 15 bytes of alignment offset
  static_assert(3 * 256 + 2 + 15 + 1 <= STAGE, "staging buffer too small");

  // UTF-8 bytes of the 8 words of a chunk that lies wholly inside the buffer: one per word,
  // one more per word >= 0x80 and one more per word >= 0x800, one less per surrogate word
  // (Section 3 sizes; a pair counts 2 + 2).  The flags are summed with byte dot products
  // (0x80 per flag), which run on the FMA pipe.
  __device__ __forceinline__ static uint32_t count_inside(const uint32_t W[4], uint32_t *sur_any,
                                                         uint32_t *ge800_any, uint32_t *wide_any) {
    uint32_t a80 = 0, a800 = 0, sub = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a80 = __dp4a(lanes16_ge80(W[k]), 0x01000100u, a80);
      a800 = __dp4a(lanes16_ge800(W[k]), 0x01000100u, a800);
      sub = __dp4a(lanes16_sur(W[k]), 0x01000100u, sub);
    }
    *sur_any = sub;  // the sums double as the "any" flags
    *ge800_any = a800;
    *wide_any = a80 - sub;  // words >= 0x80 that are not surrogates (every surrogate is >= 0x80)
    return 8u + ((a80 + a800 - sub) >> 7);
  }

  // Flag bits of a chunk (and, ORed over the lanes, of a region).
  static constexpr uint32_t F_SUR = 1;     // a surrogate word (or a chunk at a buffer end)
  static constexpr uint32_t F_THREE = 2;   // a word >= 0x800 (three UTF-8 bytes, or a surrogate)
  static constexpr uint32_t F_WIDE = 4;    // a word >= 0x80 that is not a surrogate

  static constexpr uint32_t ASCII_MASK = 0xFF80FF80u;  // nonzero in a word: a word >= 0x80
  static constexpr uint32_t CHUNK_UNITS = 8;            // bytes out of an all-ASCII chunk
  static constexpr uint32_t REGION_UNITS = 256;  // bytes out of an all-ASCII region
  static constexpr uint32_t DIRECT_ALIGN = 8;    // its lanes store 8 bytes each

  __device__ __forceinline__ static bool ascii_region(uint32_t rtot, uint32_t) { return rtot == 256u; }

  // An all-ASCII region inside the buffer whose output starts at dst, 8-byte aligned: each
  // lane narrows its 8 words and stores them with one 8-byte store (Section 4's ASCII route).
  __device__ __forceinline__ static void ascii_direct(uint8_t *dst, uint4 v, uint32_t, long long,
                                                      unsigned long long &) {
    const int lane = threadIdx.x & 31;
    uint2 *d = reinterpret_cast<uint2 *>(dst) + lane;
    *d = make_uint2(__byte_perm(v.x, v.y, 0x6420), __byte_perm(v.z, v.w, 0x6420));
  }

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge,
                                                   uint32_t &flags) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    flags = F_SUR | F_THREE | F_WIDE;
    if (!edge) {
      flags = 0;
      if (((W[0] | W[1] | W[2] | W[3]) & 0xFF80FF80u) == 0) return 8;  // all ASCII
      uint32_t sa, g3, wd;
      const uint32_t n = count_inside(W, &sa, &g3, &wd);
      flags = (sa != 0 ? F_SUR : 0u) | (g3 != 0 ? F_THREE : 0u) | (wd != 0 ? F_WIDE : 0u);
      return n;
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t w = (W[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
      const bool valid = !edge || (c + 2 * j >= (long long)p.off0 && c + 2 * j < (long long)p.vbytes);
      cnt += valid ? len8_of_word(w) : 0u;
    }
    return cnt;
  }

  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t prev,
                                                   uint32_t next, long long c, bool edge, bool inside,
                                                   uint8_t *st, uint32_t base, uint32_t x0, uint32_t rtot,
                                                   uint32_t rflags, unsigned long long &err_pos) {
    if (!inside) return convert_generic(p, v, prev, next, c, edge, st, base, x0, rtot, err_pos);
    return convert_inside(v, prev, next, c, st, base, x0, rtot, rflags, err_pos);
  }

  // Stores the UTF-8 form of one word that is not part of a surrogate pair at st[o..]: one,
  // two or three bytes (a lone surrogate takes the three-byte form; its third byte lands in
  // the next word's slot, and is overwritten there, or lies after the first error).
  __device__ __forceinline__ static void store_bmp(uint8_t *st, uint32_t o, uint32_t w, bool g1, bool g2) {
    const uint32_t c6 = w & 0x3Fu, t6 = w >> 6;
    const uint32_t b0 = g2 ? 0xE0u + (w >> 12) : (g1 ? 0xC0u + t6 : w);
    const uint32_t b1 = g2 ? (0x80u | (t6 & 0x3Fu)) : 0x80u + c6;
    st[o] = (uint8_t)b0;
    if (g1) st[o + 1] = (uint8_t)b1;
    if (g2) st[o + 2] = (uint8_t)(0x80u + c6);
  }

  // A region none of whose chunks touches a buffer end; x0 / rtot / rflags come from the
  // count pass.
  __device__ __forceinline__ static Region convert_inside(uint4 v, uint32_t prev, uint32_t next, long long c,
                                                          uint8_t *st, uint32_t base, uint32_t x0,
                                                          uint32_t rtot, uint32_t rflags,
                                                          unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    if (rtot == 256u) {
      // 256 words and 256 bytes: every word is ASCII (Section 4's ASCII route)
      const uint32_t xa = base + 8 * lane;
      const uint32_t lo8 = __byte_perm(W[0], W[1], 0x6420);
      const uint32_t hi8 = __byte_perm(W[2], W[3], 0x6420);
      if ((xa & 7) == 0) {
        *reinterpret_cast<uint2 *>(st + xa) = make_uint2(lo8, hi8);
      } else if ((xa & 3) == 0) {
        reinterpret_cast<uint32_t *>(st + xa)[0] = lo8;
        reinterpret_cast<uint32_t *>(st + xa)[1] = hi8;
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          st[xa + b] = (uint8_t)(lo8 >> (8 * b));
          st[xa + 4 + b] = (uint8_t)(hi8 >> (8 * b));
        }
      }
      return Region{256u, 0u, 0u, 256u};
    }
    Region g{rtot, 0u, 0u, rtot};
    uint32_t o = base + x0;
    if (!(rflags & (F_SUR | F_THREE))) {
      // only words below 0x800 (Section 4's one-and-two-byte route)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t w = (j & 1) ? W[j >> 1] >> 16 : W[j >> 1] & 0xFFFFu;
        const bool g1 = w >= 0x80u;
        st[o] = (uint8_t)(g1 ? 0xC0u + (w >> 6) : w);
        if (g1) st[o + 1] = (uint8_t)(0x80u | (w & 0x3Fu));
        o += g1 ? 2u : 1u;
      }
      return g;
    }
    if (!(rflags & F_SUR)) {
      // no surrogate in the region: every word is a character of one to three bytes
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t w = (j & 1) ? W[j >> 1] >> 16 : W[j >> 1] & 0xFFFFu;
        const bool g1 = w >= 0x80u, g2 = w >= 0x800u;
        store_bmp(st, o, w, g1, g2);
        o += 1u + (g1 ? 1u : 0u) + (g2 ? 1u : 0u);
      }
      return g;
    }
    // Surrogates present.  A first surrogate followed by a second one writes all four bytes
    // of the pair (its two slots and its partner's); the second writes nothing.  A pair cut
    // by the region's end is written by this region (2 bytes past its end), a pair cut by
    // its start by the previous region.
    uint32_t u[10];  // u[0] = word before the chunk, u[1..8] own words, u[9] = word after
    u[0] = prev >> 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      u[1 + 2 * k] = W[k] & 0xFFFFu;
      u[2 + 2 * k] = W[k] >> 16;
    }
    u[9] = next & 0xFFFFu;
    const bool cut_start = is_low16(u[1]) && is_high16(u[0]);
    const bool cut_end = is_high16(u[8]) && is_low16(u[9]);
    g.skip = __shfl_sync(0xffffffffu, cut_start ? 2u : 0u, 0);
    g.extra = __shfl_sync(0xffffffffu, cut_end ? 2u : 0u, 31);
    if (!(rflags & F_WIDE)) {
      // only ASCII words and surrogates (emoji-heavy text): an ASCII word writes its byte and
      // every other word two slots' worth, all four bytes of a pair coming from its first
      // word; the pair rules are checked on whole words (an unpaired surrogate is an error,
      // and what it would write lies past the first error)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t w = u[j + 1], wn = u[j + 2];
        const bool sur = (w & 0xF800u) == 0xD800u;
        if (!sur) st[o] = (uint8_t)w;
        if (is_high16(w) && is_low16(wn)) {
          const uint32_t t = (w & 0x3FFu) + 0x40u;  // the code point >> 10
          st[o] = (uint8_t)(0xF0u | (t >> 8));
          st[o + 1] = (uint8_t)(0x80u | ((t >> 2) & 0x3Fu));
          st[o + 2] = (uint8_t)(0x80u | ((t & 3u) << 4) | ((wn >> 6) & 0xFu));
          st[o + 3] = (uint8_t)(0x80u | (wn & 0x3Fu));
        }
        o += sur ? 2u : 1u;
      }
      if (utf16_pair_errors_inside(W, prev, next) && (unsigned long long)c < err_pos)
        err_pos = (unsigned long long)c;
      return g;
    }
    bool err = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t w = u[j + 1];
      const bool g1 = w >= 0x80u, g2 = w >= 0x800u;
      const bool hs = is_high16(w), ls = is_low16(w);
      const bool pair = hs && is_low16(u[j + 2]);
      const bool follows = ls && is_high16(u[j]);
      err |= (hs && !pair) || (ls && !follows);
      if (pair) {
        const uint32_t wn = u[j + 2];
        const uint32_t t = (w & 0x3FFu) + 0x40u;  // the code point >> 10
        st[o] = (uint8_t)(0xF0u | (t >> 8));
        st[o + 1] = (uint8_t)(0x80u | ((t >> 2) & 0x3Fu));
        st[o + 2] = (uint8_t)(0x80u | ((t & 3u) << 4) | ((wn >> 6) & 0xFu));
        st[o + 3] = (uint8_t)(0x80u | (wn & 0x3Fu));
      } else if (!follows) {
        store_bmp(st, o, w, g1, g2);
      }
      o += (hs || ls) ? 2u : 1u + (g1 ? 1u : 0u) + (g2 ? 1u : 0u);
    }
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    return g;
  }

  // A region that touches a buffer end (positions outside [off0, vbytes) are not data; the
  // count pass gave them no units).  Word by word, with the pair rules of convert_inside.
  __device__ __forceinline__ static Region convert_generic(const Params &p, uint4 v, uint32_t prev,
                                                           uint32_t next, long long c, bool edge,
                                                           uint8_t *st, uint32_t base, uint32_t x0,
                                                           uint32_t rtot, unsigned long long &err_pos) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    uint32_t u[10];  // u[0] = word before the chunk, u[1..8] own words, u[9] = word after
    u[0] = prev >> 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      u[1 + 2 * k] = W[k] & 0xFFFFu;
      u[2 + 2 * k] = W[k] >> 16;
    }
    u[9] = next & 0xFFFFu;
    bool valid[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      valid[j] = !edge || (c + 2 * j >= (long long)p.off0 && c + 2 * j < (long long)p.vbytes);
    bool err = false;
    uint32_t o = base + x0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!valid[j]) continue;
      const uint32_t w = u[j + 1];
      const bool g1 = w >= 0x80u, g2 = w >= 0x800u;
      const bool hs = is_high16(w), ls = is_low16(w);
      // a word outside the buffer reads as 0: never a surrogate
      const bool pair = hs && is_low16(u[j + 2]);
      const bool follows = ls && is_high16(u[j]);
      err |= (hs && !pair) || (ls && !follows);
      if (pair) {
        const uint32_t wn = u[j + 2];
        const uint32_t t = (w & 0x3FFu) + 0x40u;
        st[o] = (uint8_t)(0xF0u | (t >> 8));
        st[o + 1] = (uint8_t)(0x80u | ((t >> 2) & 0x3Fu));
        st[o + 2] = (uint8_t)(0x80u | ((t & 3u) << 4) | ((wn >> 6) & 0xFu));
        st[o + 3] = (uint8_t)(0x80u | (wn & 0x3Fu));
      } else if (!follows) {
        store_bmp(st, o, w, g1, g2);
      }
      o += (hs || ls) ? 2u : 1u + (g1 ? 1u : 0u) + (g2 ? 1u : 0u);
    }
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    Region g{rtot, 0u, 0u, rtot};
    // a pair cut by the region's start or end (lane 0's first word, lane 31's last word)
    const bool cut_start = valid[0] && is_low16(u[1]) && is_high16(u[0]);
    const bool cut_end = valid[7] && is_high16(u[8]) && is_low16(u[9]);
    g.skip = __shfl_sync(0xffffffffu, cut_start ? 2u : 0u, 0);
    g.extra = __shfl_sync(0xffffffffu, cut_end ? 2u : 0u, 31);
    return g;
  }
};

}  // namespace gbu
