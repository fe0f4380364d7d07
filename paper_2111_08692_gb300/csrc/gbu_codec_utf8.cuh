// gbu_codec_utf8.cuh -- the UTF-8 -> UTF-16LE codec (validating), used by the single-buffer
// transcoder (gbu_utf8.cu) and the batched kernels (gbu_batch.cu).
//
// Paper Section 3 defines both formats; Section 5 states that transcoding validates.
// Section 4's design (64-byte blocks, a 12-byte shuffle-table routine) is a 128-bit-register
// idiom; here a warp handles a 512-byte region, one 16-byte chunk per lane:
//   * the chunk is classified and validated as in gbu_chunk.cuh;
//   * output: one UTF-16 word per leading byte, two for a four-byte sequence, counted on the
//     leading byte; word offsets are prefix sums of per-byte counts (a lane's chunk by byte
//     dot products in the count pass and a running index while staging, lanes via a warp
//     scan, regions via the partition count, and partitions via the look-back);
//   * an all-ASCII warp widens its bytes directly (Section 4's ASCII path).
// A lane whose chunk breaks any check reports the chunk start; the last CTA turns the
// smallest one into the exact offset and kind (resolve_utf8_error).
#pragma once

#include <stdint.h>

#include "gbu_chunk.cuh"
#include "gbu_device.cuh"
#include "gbu_xcode.cuh"

namespace gbu {

// Stores 16 UTF-16 words (8 packed words) at staging index x.
__device__ __forceinline__ void stage16(uint16_t *st, uint32_t x, const uint32_t u[8]) {
  if ((x & 7) == 0) {
    uint4 *d = reinterpret_cast<uint4 *>(st + x);
    d[0] = make_uint4(u[0], u[1], u[2], u[3]);
    d[1] = make_uint4(u[4], u[5], u[6], u[7]);
  } else if ((x & 1) == 0) {
    uint32_t *d = reinterpret_cast<uint32_t *>(st + x);
#pragma unroll
    for (int j = 0; j < 8; ++j) d[j] = u[j];
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      st[x + 2 * j] = (uint16_t)(u[j] & 0xFFFF);
      st[x + 2 * j + 1] = (uint16_t)(u[j] >> 16);
    }
  }
}

struct Utf8ToUtf16 {
  using Out = uint16_t;
  // a valid 512-byte region yields at most 512 words (+1 for a four-byte lead in its last
  // byte), plus 7 words of alignment slack; words past this can only come from bytes after
  // the first error and are dropped
  static constexpr uint32_t STAGE = 512 + 16 + 16;

  static constexpr uint32_t F_NONASCII = 1;  // flag: a byte >= 0x80 (or a chunk at a buffer end)
  static constexpr uint32_t F_C2 = 2;        // flag: a leading byte C0-DF
  static constexpr uint32_t F_C3 = 4;        // flag: a leading byte E0-EF
  static constexpr uint32_t F_C4 = 8;        // flag: a byte F0-FF

  // F_C2 / F_C3 / F_C4 for the bytes of w selected by m (bit 7 of each byte).
  __device__ __forceinline__ static uint32_t lead_classes(uint32_t w, uint32_t m) {
    const uint32_t s2 = w << 2, s3 = w << 3;
    const uint32_t ge = w & (w << 1) & m;  // >= C0
    return ((ge & ~s2) ? F_C2 : 0u) | ((ge & s2 & ~s3) ? F_C3 : 0u) | ((ge & s2 & s3) ? F_C4 : 0u);
  }

  static constexpr uint32_t ASCII_MASK = 0x80808080u;  // nonzero in a word: a byte >= 0x80
  static constexpr uint32_t CHUNK_UNITS = 16;           // words out of an all-ASCII chunk
  static constexpr uint32_t REGION_UNITS = 512;  // words out of an all-ASCII region
  static constexpr uint32_t DIRECT_ALIGN = 8;    // its lanes store 16 words (32 bytes) each

  __device__ __forceinline__ static bool ascii_region(uint32_t, uint32_t rflags) { return rflags == 0; }

  // An all-ASCII region inside the buffer whose output starts at dst, 16-byte aligned: each
  // lane widens its 16 bytes and stores them with two 16-byte stores (Section 4's ASCII path).  The only
  // possible error is a leading byte just before the region that wants continuation bytes
  // inside it (lane 0's chunk).
  __device__ __forceinline__ static void ascii_direct(uint16_t *dst, uint4 v, uint32_t prev, long long c,
                                                      unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
      const Flags8 fp = classify8(prev);
      const uint32_t req = __funnelshift_l(fp.geC0, 0u, 8) | __funnelshift_l(fp.geE0, 0u, 16) |
                           __funnelshift_l(fp.geF0, 0u, 24);
      if (req && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    }
    const uint4 a = make_uint4(__byte_perm(v.x, 0, 0x4140), __byte_perm(v.x, 0, 0x4342),
                               __byte_perm(v.y, 0, 0x4140), __byte_perm(v.y, 0, 0x4342));
    const uint4 b = make_uint4(__byte_perm(v.z, 0, 0x4140), __byte_perm(v.z, 0, 0x4342),
                               __byte_perm(v.w, 0, 0x4140), __byte_perm(v.w, 0, 0x4342));
    uint4 *d = reinterpret_cast<uint4 *>(dst) + 2 * lane;
    if (((uintptr_t)dst & 31) == 0) {
      st_global_32B(d, a, b);  // the warp writes its 1 KB in whole sectors
    } else {
      d[0] = a;
      d[1] = b;
    }
  }

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge,
                                                   uint32_t &flags) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    flags = F_NONASCII;
    if (!edge && ((W[0] | W[1] | W[2] | W[3]) & 0x80808080u) == 0) {  // all ASCII
      flags = 0;
      return 16;
    }
    // per byte, as bit 7: not a continuation byte (10xxxxxx), and >= F0; a byte dot product
    // with 0x01 weights adds 0x80 per flag (FMA pipe rather than the XU pipe of popc).  The
    // classes of the leading bytes go to the flags.
    uint32_t acc = 0, c2 = 0, c3 = 0, c4 = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t w = W[k], s1 = w << 1, s2 = w << 2, s3 = w << 3;
      const uint32_t vm = edge ? byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes) : 0x80808080u;
      const uint32_t ge = w & s1 & vm;  // >= C0
      const uint32_t f0 = ge & s2 & s3;  // >= F0
      acc = __dp4a((~w | s1) & vm, 0x01010101u, acc);
      acc = __dp4a(f0, 0x01010101u, acc);
      c2 |= ge & ~s2;
      c3 |= ge & s2 & ~s3;
      c4 |= f0;
    }
    flags = F_NONASCII | (c2 ? F_C2 : 0u) | (c3 ? F_C3 : 0u) | (c4 ? F_C4 : 0u);
    return acc >> 7;
  }

  // Validates one chunk of a region that lies inside the buffer and whose output fits the
  // staging buffer, and stages its words from index addr on; returns nonzero when the chunk
  // breaks a rule.  H2 / H3 / H4: leading bytes C0-DF / E0-EF / F0-FF occur in the warp
  // (the code for an absent class is left out).  Rules 1-3 by the funnel-shifted lead flags
  // of the classes present; rules 4-5 for the two- and three-byte forms by the word-level
  // tests of utf8_special_errors; the four-byte form by the range of the decoded first
  // surrogate (D800-DBFF exactly when the code point is in 10000-10FFFF).  Each
  // non-continuation byte stages one word (a four-byte sequence two), which is the count the
  // count pass gave the chunk, so no store needs a bounds test.
  template <bool H2, bool H3, bool H4>
  __device__ __forceinline__ static uint32_t convert_fast(const uint32_t W[6], uint16_t *st, uint32_t addr) {
    // with a single class present, every byte >= C0 is a leading byte of that class; without
    // H4 there is no byte >= F0
    constexpr bool ONE = (int)H2 + (int)H3 + (int)H4 == 1;
    Flags8 f[5];  // isC for W[1..4]; geC0, and geE0 / geF0 where the variant needs them
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const uint32_t w = W[k], s1 = w << 1;
      f[k].geC0 = w & s1 & 0x80808080u;
      f[k].isC = w & ~s1 & 0x80808080u;
      f[k].geE0 = ONE ? f[k].geC0 : f[k].geC0 & (w << 2);
      f[k].geF0 = H4 ? (ONE ? f[k].geC0 : f[k].geE0 & (w << 3)) : 0u;  // zero without H4 (the E0-EF test reads it)
    }
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t req = __funnelshift_l(f[k].geC0, f[k + 1].geC0, 8);
      if (H3 || H4) req |= __funnelshift_l(f[k].geE0, f[k + 1].geE0, 16);
      if (H4) req |= __funnelshift_l(f[k].geF0, f[k + 1].geF0, 24);
      bad |= req ^ f[k + 1].isC;
    }
    if (H2 || H3) bad |= utf8_special_errors(W, f, H2, H3, false);
    // pair i covers positions 2i, 2i+1 (two 16-bit lanes): E = bytes (2i, 2i+1),
    // O = bytes (2i+1, 2i+2); the next pair's E and O hold the third and fourth bytes
    uint32_t E = __byte_perm(W[1], W[2], selE(0));
    uint32_t O = __byte_perm(W[1], W[2], selO(0));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = i >> 1, h = i & 1;
      const int kn = (i + 1) >> 1, hn = (i + 1) & 1;
      const uint32_t En = __byte_perm(W[kn + 1], W[kn + 2 <= 5 ? kn + 2 : 5], selE(hn));
      const uint32_t On = __byte_perm(W[kn + 1], W[kn + 2 <= 5 ? kn + 2 : 5], selO(hn));
      const Flags8 &g = f[k + 1];
      uint32_t r = E & 0x00FF00FFu;
      uint32_t lo4 = 0;
      if (H2) {
        const uint32_t M2 = prmt(ONE ? g.geC0 : g.geC0 & ~g.geE0, 0, selM(h));  // C0-DF
        const uint32_t U2 = (E & 0x001F001Fu) * 64u + (O & 0x003F003Fu);
        r = (U2 & M2) | (r & ~M2);
      }
      if (H3) {
        const uint32_t M3 = prmt(H4 && !ONE ? g.geE0 & ~g.geF0 : g.geE0, 0, selM(h));  // E0-EF
        const uint32_t U3 = ((E & 0x000F000Fu) * 64u + (O & 0x003F003Fu)) * 64u + (En & 0x003F003Fu);
        r = (U3 & M3) | (r & ~M3);
      }
      if (H4) {
        const uint32_t M4 = prmt(g.geF0, 0, selM(h));  // F0-FF
        // first surrogate: (code point >> 10) + D7C0, from bits of the first three bytes
        const uint32_t hi = (E & 0x001F001Fu) * 256u + (O & 0x003F003Fu) * 4u + ((En >> 4) & 0x00030003u) +
                            0xC7C0C7C0u;
        const uint32_t t = ((hi ^ 0xD800D800u) >> 10) & 0x003F003Fu;  // 0 iff 10000-10FFFF
        bad |= (t + 0x7FFF7FFFu) & M4 & 0x80008000u;
        r = (hi & M4) | (r & ~M4);
        lo4 = (En & 0x000F000Fu) * 64u + (On & 0x003F003Fu) + 0xDC00DC00u;
      }
      const uint32_t nc = ~g.isC;  // bit 7 of each byte: not a continuation byte
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int bit = 16 * h + 8 * q + 7;
        if ((nc >> bit) & 1u) {
          st[addr] = (uint16_t)(r >> (16 * q));
          if (H4 && ((g.geF0 >> bit) & 1u)) st[++addr] = (uint16_t)(lo4 >> (16 * q));
          ++addr;
        }
      }
      E = En;
      O = On;
    }
    return bad;
  }

  // Validates the chunk and stages its UTF-16 words.  The lane's offset x0 (inside the
  // region), the region total rtot and the region flags rflags (F_NONASCII: a byte >= 0x80
  // in the region, or a chunk at a buffer end) come from the count pass, so each pair of positions is
  // decoded and stored in one pass without keeping decoded words in registers.
  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t prev,
                                                   uint32_t next, long long c, bool edge, bool inside,
                                                   uint16_t *st, uint32_t base, uint32_t x0, uint32_t rtot,
                                                   uint32_t rflags, unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    if (rflags == 0) {
      // an all-ASCII region: one word per byte; the only possible error is a leading byte
      // just before the region that wants continuation bytes inside it (lane 0's chunk)
      if (lane == 0) {
        const Flags8 fp = classify8(prev);
        const uint32_t req = __funnelshift_l(fp.geC0, 0u, 8) | __funnelshift_l(fp.geE0, 0u, 16) |
                             __funnelshift_l(fp.geF0, 0u, 24);
        if (req && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
      }
      uint32_t u[8];
      u[0] = __byte_perm(v.x, 0, 0x4140); u[1] = __byte_perm(v.x, 0, 0x4342);
      u[2] = __byte_perm(v.y, 0, 0x4140); u[3] = __byte_perm(v.y, 0, 0x4342);
      u[4] = __byte_perm(v.z, 0, 0x4140); u[5] = __byte_perm(v.z, 0, 0x4342);
      u[6] = __byte_perm(v.w, 0, 0x4140); u[7] = __byte_perm(v.w, 0, 0x4342);
      stage16(st, base + 16 * lane, u);
      return Region{512u, 0u, 0u, 512u};
    }
    if (inside && base + rtot <= STAGE) {
      const uint32_t W[6] = {prev, v.x, v.y, v.z, v.w, next};
      // the leading-byte classes: the region's own (from the count pass) and those of bytes
      // 1-3 of the word before it (a sequence starting there reaches into the region, and the
      // structure test reads those bytes)
      const uint32_t pc = lane == 0 ? lead_classes(prev, 0x80808000u) : 0u;
      const uint32_t cls = rflags | __shfl_sync(0xffffffffu, pc, 0);
      const bool h2 = cls & F_C2, h3 = cls & F_C3, h4 = cls & F_C4;
      const uint32_t addr = base + x0;
      uint32_t bad;
      if (h4) {
        bad = (h2 || h3) ? convert_fast<true, true, true>(W, st, addr) : convert_fast<false, false, true>(W, st, addr);
      } else if (h3) {
        bad = h2 ? convert_fast<true, true, false>(W, st, addr) : convert_fast<false, true, false>(W, st, addr);
      } else {
        bad = h2 ? convert_fast<true, false, false>(W, st, addr) : convert_fast<true, true, true>(W, st, addr);
      }
      if (bad && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
      return Region{rtot, 0u, 0u, rtot};
    }
    const General r =
        convert_general(p.off0, (long long)p.vbytes, v, prev, next, c, edge, st, base, x0, rtot, err_pos, STAGE);
    err_pos = r.err_pos;
    return r.g;
  }

  struct General {
    Region g;
    unsigned long long err_pos;
  };

  // Any region (one at a buffer end, or one whose output would overflow the staging buffer,
  // which only happens after an error): per-byte word counts with the buffer's bounds, and
  // a bounds test before every store.  `stage` is the staging buffer's size in words.  Kept
  // out of line so that the hot loop does not carry its registers.
  __device__ __noinline__ static General convert_general(long long lo, long long hi, uint4 v, uint32_t prev, uint32_t next,
                                                          long long c, bool edge, uint16_t *st, uint32_t base,
                                                          uint32_t x0, uint32_t rtot, unsigned long long err_pos,
                                                          uint32_t stage) {
    return convert_general_body(lo, hi, v, prev, next, c, edge, st, base, x0, rtot, err_pos, stage);
  }

  // The body of convert_general, for callers that inline it.
  __device__ __forceinline__ static General convert_general_body(long long lo, long long hi, uint4 v, uint32_t prev,
                                                                 uint32_t next, long long c, bool edge, uint16_t *st,
                                                                 uint32_t base, uint32_t x0, uint32_t rtot,
                                                                 unsigned long long err_pos, uint32_t stage) {
    uint32_t W[6];
    W[0] = prev;
    W[1] = v.x; W[2] = v.y; W[3] = v.z; W[4] = v.w;
    W[5] = next;
    Flags8 f[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k] = classify8(W[k]);
    uint32_t uw[4];  // per byte: UTF-16 words produced at that position (0, 1 or 2)
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t vm = 0x80808080u;
      if (edge) vm = byte_range_mask(c + 4 * k, lo, hi);
      uw[k] = ((~f[k + 1].isC & vm) >> 7) + ((f[k + 1].geF0 & vm) >> 7);
      cnt = __dp4a(uw[k], 0x01010101u, cnt);
    }
    uint32_t err = utf8_structure_errors(f);

    Region g{rtot, 0u, 0u, rtot};
    x0 += base;
    // a chunk that would overflow the staging buffer lies after the first error: it stores
    // nothing (its validation still runs)
    const bool store = x0 + cnt <= stage;
    {
      uint32_t c2 = 0, c3 = 0, c4 = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        c2 |= f[k + 1].geC0 & ~f[k + 1].geE0;
        c3 |= f[k + 1].geE0 & ~f[k + 1].geF0;
        c4 |= f[k + 1].geF0;
      }
      const bool has2 = __any_sync(0xffffffffu, c2 != 0);
      const bool has3 = __any_sync(0xffffffffu, c3 != 0);
      const bool has4 = __any_sync(0xffffffffu, c4 != 0);
      uint32_t bad = 0;
      uint32_t addr = x0;
      // pair i covers positions 2i, 2i+1: E = bytes (2i, 2i+1), O = bytes (2i+1, 2i+2); the
      // next pair's E and O supply the third and fourth bytes of a sequence
      uint32_t E = __byte_perm(W[1], W[2], selE(0));
      uint32_t O = __byte_perm(W[1], W[2], selO(0));
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = i >> 1, h = i & 1;
        const int kn = (i + 1) >> 1, hn = (i + 1) & 1;
        const uint32_t En = __byte_perm(W[kn + 1], W[kn + 2 <= 5 ? kn + 2 : 5], selE(hn));
        const uint32_t On = __byte_perm(W[kn + 1], W[kn + 2 <= 5 ? kn + 2 : 5], selO(hn));
        uint32_t r = E & 0x00FF00FFu;
        uint32_t lo4 = 0;
        const uint32_t U2 = ((E << 6) & 0x07C007C0u) | (O & 0x003F003Fu);
        if (has2) {
          const uint32_t M2 = prmt(f[k + 1].geC0 & ~f[k + 1].geE0, 0, selM(h));
          const uint32_t t = E & 0x001E001Eu;  // U2 < 0x80 exactly when the lead is C0/C1
          bad |= ~(t + 0x7FFF7FFFu) & M2 & 0x80008000u;
          r = (U2 & M2) | (r & ~M2);
        }
        if (has3) {
          const uint32_t M3 = prmt(f[k + 1].geE0 & ~f[k + 1].geF0, 0, selM(h));
          const uint32_t U3 = ((U2 << 6) & 0xFFC0FFC0u) | (En & 0x003F003Fu);
          const uint32_t t = (U3 >> 11) & 0x001F001Fu;  // 0: below U+800; 0x1B: D800-DFFF
          bad |= ~((t + 0x7FFF7FFFu) & ((t ^ 0x001B001Bu) + 0x7FFF7FFFu)) & M3 & 0x80008000u;
          r = (U3 & M3) | (r & ~M3);
        }
        if (has4) {
          const uint32_t M4 = prmt(f[k + 1].geF0, 0, selM(h));
          const uint32_t hi = (U2 << 2) + ((En >> 4) & 0x00030003u) + 0xC7C0C7C0u;
          const uint32_t t = ((hi ^ 0xD800D800u) >> 10) & 0x003F003Fu;  // 0 iff U+10000-10FFFF
          bad |= (t + 0x7FFF7FFFu) & M4 & 0x80008000u;
          r = (hi & M4) | (r & ~M4);
          lo4 = ((En << 6) & 0x03C003C0u) | (On & 0x003F003Fu) | 0xDC00DC00u;
        }
        const uint32_t ua = (uw[k] >> (16 * h)) & 3u, ub = (uw[k] >> (16 * h + 8)) & 3u;
        if (store && ua) st[addr] = (uint16_t)r;
        if (has4 && store && ua == 2) st[addr + 1] = (uint16_t)lo4;
        addr += ua;
        if (store && ub) st[addr] = (uint16_t)(r >> 16);
        if (has4 && store && ub == 2) st[addr + 1] = (uint16_t)(lo4 >> 16);
        addr += ub;
        E = En;
        O = On;
      }
      err |= bad;
    }
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    if (g.total > stage - base) g.total = stage - base;  // only after the first error
    return General{g, err_pos};
  }
};

}  // namespace gbu
