// gbu_utf32.cu -- UTF-32: validation, lengths, and transcoding to and from UTF-8 and UTF-16LE.
//
// UTF-32 is not in the paper, whose problem is UTF-8 and UTF-16: each 32-bit unit (host byte
// order) holds one value, valid when Section 3 allows it -- below 1,114,112 (rule 5) and outside
// D800-DFFF (rule 6); the first invalid unit is reported with that rule's kind at its index.
//   * utf32_stream_kernel: the read-only operations (validation, the UTF-8 and UTF-16 lengths of
//     a UTF-32 input, the UTF-32 length of a UTF-8 or UTF-16LE input), streaming 4 KB warp tiles
//     like the UTF-8 and UTF-16 read-only kernels; a unit needs no neighbour.
//   * utf32_to_utf8_kernel / utf8_to_utf32_kernel: the partition loop of gbu_xcode.cuh with the
//     two codecs below.  UTF-32 -> UTF-8 encodes each unit in 1-4 bytes; UTF-8 -> UTF-32 checks
//     rules 1-6 with the word-level tests of gbu_chunk.cuh and stores one unit per leading byte,
//     decoded from the four bytes that start there.
//   * utf32_to_utf16_kernel / utf16_to_utf32_kernel: the same loop between UTF-16LE and UTF-32:
//     a unit becomes one word (below 0x10000) or a surrogate pair; a UTF-16 word that is not a
//     second surrogate becomes one unit (a first surrogate with its partner, which may be the
//     first word of the next region), with Section 3's pair rules checked word by word.
#include <stdint.h>

#include "gbu_chunk.cuh"
#include "gbu_device.cuh"
#include "gbu_kernels.h"
#include "gbu_xcode.cuh"

namespace gbu {

__device__ __forceinline__ bool utf32_bad(uint32_t u) { return u > 0x10FFFFu || (u & 0xFFFFF800u) == 0xD800u; }
__device__ __forceinline__ uint32_t utf8_len_of_unit(uint32_t u) {
  return 1u + (u >= 0x80u ? 1u : 0u) + (u >= 0x800u ? 1u : 0u) + (u >= 0x10000u ? 1u : 0u);
}

// The first invalid unit at or after unit `chunk` (the start of the smallest flagged chunk).
static __device__ __noinline__ void resolve_utf32_error(const uint32_t *s, uint64_t n, long long chunk,
                                                        int32_t *kind, uint64_t *off) {
  long long i = chunk < 0 ? 0 : chunk;
  const long long stop = chunk + 8 < (long long)n ? chunk + 8 : (long long)n;
  for (; i < stop; ++i) {
    if (s[i] > 0x10FFFFu) { *kind = GBU_TOO_LARGE; *off = (uint64_t)i; return; }
    if ((s[i] & 0xFFFFF800u) == 0xD800u) { *kind = GBU_SURROGATE; *off = (uint64_t)i; return; }
  }
  *kind = GBU_TOO_LARGE;  // not reached for a real error
  *off = chunk < 0 ? 0 : (uint64_t)chunk;
}

// ---- read-only kernel ---------------------------------------------------------------------

enum Utf32Mode { U_V32 = 0, U_L8 = 1, U_L32 = 2, U_L16 = 3, U_L32F16 = 4 };

template <int MODE>
__global__ void __launch_bounds__(STREAM_THREADS) utf32_stream_kernel(const Params p) {
  constexpr int WARPS = STREAM_THREADS / 32;
  constexpr int ROUNDS = 8;
  constexpr uint32_t TILE = 32u * 16u * ROUNDS;
  __shared__ unsigned long long red[WARPS];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * WARPS + warp;
  const long long nw = (long long)gridDim.x * WARPS;
  const long long lo = p.off0, hi = (long long)p.vbytes;
  unsigned long long err_pos = NO_ERROR, total = 0;
  for (long long wt = gw; wt < (long long)p.ntiles; wt += nw) {
    const long long t0 = wt * TILE;
    const bool fast = t0 >= lo && t0 + (long long)TILE <= hi;
    uint4 v[ROUNDS];
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) v[r] = load_chunk(p, t0 + 512 * r + 16 * lane, fast);
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
      const long long c = t0 + 512 * r + 16 * lane;
      const bool edge = !fast && (c < lo || c + 16 > hi);
      const uint32_t U[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
      if (MODE == U_V32) {
        // units outside the buffer read as zero, which is valid
        const bool bad = utf32_bad(U[0]) || utf32_bad(U[1]) || utf32_bad(U[2]) || utf32_bad(U[3]);
        if (bad && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
      } else if (MODE == U_L8) {
        uint32_t n = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool valid = !edge || (c + 4 * j >= lo && c + 4 * j < hi);
          n += valid ? utf8_len_of_unit(U[j]) : 0u;
        }
        total += n;
      } else if (MODE == U_L16) {
        uint32_t n = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool valid = !edge || (c + 4 * j >= lo && c + 4 * j < hi);
          n += valid ? (U[j] >= 0x10000u ? 2u : 1u) : 0u;
        }
        total += n;
      } else if (MODE == U_L32F16) {
        // UTF-16LE input: one unit per word that is not a second surrogate
        uint32_t n = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t w = (U[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
          const bool valid = !edge || (c + 2 * j >= lo && c + 2 * j < hi);
          n += (valid && (w & 0xFC00u) != 0xDC00u) ? 1u : 0u;
        }
        total += n;
      } else {
        // UTF-8 input: one unit per byte that is not a continuation byte (flags in bit 7,
        // summed by byte dot products)
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t vm = edge ? byte_range_mask(c + 4 * k, lo, hi) : 0x80808080u;
          acc = __dp4a((~U[k] | (U[k] << 1)) & vm, 0x01010101u, acc);
        }
        total += acc >> 7;
      }
    }
  }
  const bool want_err = MODE == U_V32;
  if (!fold_and_finish<STREAM_THREADS>(p, want_err ? err_pos : total, want_err, red, &is_last)) return;
  if (threadIdx.x == 0) {
    const unsigned long long key = *(volatile unsigned long long *)&p.ws->errkey;
    const unsigned long long tot = *(volatile unsigned long long *)&p.ws->total;
    if (MODE != U_V32) {
      *p.len_out = tot;
    } else if (key == NO_ERROR) {
      write_result(p.result, GBU_OK, p.n);
    } else {
      int32_t kind;
      uint64_t off;
      resolve_utf32_error(reinterpret_cast<const uint32_t *>(p.base + p.off0), p.n,
                          ((long long)key - (long long)p.off0) / 4, &kind, &off);
      write_result(p.result, kind, off);
    }
  }
  reset_workspace(p);
}

// ---- UTF-32 -> UTF-8 codec ------------------------------------------------------------------

struct Utf32ToUtf8 {
  using Out = uint8_t;
  static constexpr uint32_t STAGE = 4 * 128 + 32;  // 128 units of at most 4 bytes + alignment slack
  static constexpr uint32_t F_WIDE = 1;            // a unit >= 0x80 (or a chunk at a buffer end)
  static constexpr uint32_t ASCII_MASK = 0xFFFFFF80u;
  static constexpr uint32_t CHUNK_UNITS = 4;    // bytes out of an all-ASCII chunk
  static constexpr uint32_t REGION_UNITS = 128;
  static constexpr uint32_t DIRECT_ALIGN = 4;   // its lanes store 4 bytes each

  __device__ __forceinline__ static bool ascii_region(uint32_t, uint32_t rflags) { return rflags == 0; }

  __device__ __forceinline__ static void ascii_direct(uint8_t *dst, uint4 v, uint32_t, long long,
                                                      unsigned long long &) {
    const int lane = threadIdx.x & 31;
    const uint32_t t1 = __byte_perm(v.x, v.y, 0x0040), t2 = __byte_perm(v.z, v.w, 0x0040);
    reinterpret_cast<uint32_t *>(dst)[lane] = __byte_perm(t1, t2, 0x5410);
  }

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge,
                                                   uint32_t &flags) {
    const uint32_t U[4] = {v.x, v.y, v.z, v.w};
    if (!edge && ((U[0] | U[1] | U[2] | U[3]) & ASCII_MASK) == 0) {
      flags = 0;
      return 4;
    }
    flags = F_WIDE;
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool valid = !edge || (c + 4 * j >= (long long)p.off0 && c + 4 * j < (long long)p.vbytes);
      n += valid ? utf8_len_of_unit(U[j]) : 0u;
    }
    return n;
  }

  // Encodes the chunk's units (Section 3's UTF-8 layout) into the staging buffer from index
  // base + x0; an invalid unit flags the chunk (its bytes lie past the first error).
  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t, uint32_t, long long c,
                                                   bool edge, bool, uint8_t *st, uint32_t base, uint32_t x0,
                                                   uint32_t rtot, uint32_t, unsigned long long &err_pos) {
    const uint32_t U[4] = {v.x, v.y, v.z, v.w};
    uint32_t o = base + x0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool valid = !edge || (c + 4 * j >= (long long)p.off0 && c + 4 * j < (long long)p.vbytes);
      if (!valid) continue;
      const uint32_t u = U[j];
      bad = bad || utf32_bad(u);
      const uint32_t len = utf8_len_of_unit(u);
      if (len == 1) {
        st[o] = (uint8_t)u;
      } else if (len == 2) {
        st[o] = (uint8_t)(0xC0u | (u >> 6));
        st[o + 1] = (uint8_t)(0x80u | (u & 0x3Fu));
      } else if (len == 3) {
        st[o] = (uint8_t)(0xE0u | (u >> 12));
        st[o + 1] = (uint8_t)(0x80u | ((u >> 6) & 0x3Fu));
        st[o + 2] = (uint8_t)(0x80u | (u & 0x3Fu));
      } else {
        st[o] = (uint8_t)(0xF0u | ((u >> 18) & 0x07u));
        st[o + 1] = (uint8_t)(0x80u | ((u >> 12) & 0x3Fu));
        st[o + 2] = (uint8_t)(0x80u | ((u >> 6) & 0x3Fu));
        st[o + 3] = (uint8_t)(0x80u | (u & 0x3Fu));
      }
      o += len;
    }
    if (bad && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    return Region{rtot, 0u, 0u, rtot};
  }
};

// ---- UTF-8 -> UTF-32 codec ------------------------------------------------------------------

struct Utf8ToUtf32 {
  using Out = uint32_t;
  static constexpr uint32_t STAGE = 512 + 16 + 16;  // at most one unit per byte + alignment slack
  static constexpr uint32_t F_NONASCII = 1;          // a byte >= 0x80 (or a chunk at a buffer end)
  static constexpr uint32_t ASCII_MASK = 0x80808080u;
  static constexpr uint32_t CHUNK_UNITS = 16;
  static constexpr uint32_t REGION_UNITS = 512;
  static constexpr uint32_t DIRECT_ALIGN = 4;  // its lanes store 16 units (64 bytes) each

  __device__ __forceinline__ static bool ascii_region(uint32_t, uint32_t rflags) { return rflags == 0; }

  // An all-ASCII region: each byte zero-extended to a unit; the only possible error is a leading
  // byte just before the region that wants continuation bytes inside it (lane 0's chunk).
  __device__ __forceinline__ static void ascii_direct(uint32_t *dst, uint4 v, uint32_t prev, long long c,
                                                      unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
      const Flags8 fp = classify8(prev);
      const uint32_t req = __funnelshift_l(fp.geC0, 0u, 8) | __funnelshift_l(fp.geE0, 0u, 16) |
                           __funnelshift_l(fp.geF0, 0u, 24);
      if (req && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    }
    uint4 *d = reinterpret_cast<uint4 *>(dst) + 4 * lane;
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      d[k] = make_uint4(__byte_perm(W[k], 0, 0x4440), __byte_perm(W[k], 0, 0x4441), __byte_perm(W[k], 0, 0x4442),
                        __byte_perm(W[k], 0, 0x4443));
  }

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge,
                                                   uint32_t &flags) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    if (!edge && ((W[0] | W[1] | W[2] | W[3]) & 0x80808080u) == 0) {
      flags = 0;
      return 16;
    }
    flags = F_NONASCII;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t vm = edge ? byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes) : 0x80808080u;
      acc = __dp4a((~W[k] | (W[k] << 1)) & vm, 0x01010101u, acc);
    }
    return acc >> 7;
  }

  // Validates the chunk (rules 1-3 by the lead/continuation flags, rules 4-6 by the word-level
  // byte tests) and stores one unit per leading byte, decoded from the four bytes that start
  // there (Section 3's payload bits, most significant first).
  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t prev, uint32_t next,
                                                   long long c, bool edge, bool, uint32_t *st, uint32_t base,
                                                   uint32_t x0, uint32_t rtot, uint32_t,
                                                   unsigned long long &err_pos) {
    const uint32_t W[6] = {prev, v.x, v.y, v.z, v.w, next};
    Flags8 f[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k] = classify8(W[k]);
    uint32_t err = utf8_structure_errors(f);
    uint32_t c2 = 0, c3 = 0, c4 = 0;
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
      c2 |= f[k].geC0 & ~f[k].geE0;
      c3 |= f[k].geE0 & ~f[k].geF0;
      c4 |= f[k].geF0;
    }
    err |= utf8_special_errors(W, f, __any_sync(0xffffffffu, c2 != 0), __any_sync(0xffffffffu, c3 != 0),
                               __any_sync(0xffffffffu, c4 != 0));
    uint32_t addr = base + x0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t vm = edge ? byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes) : 0x80808080u;
      const uint32_t keep = ~f[k + 1].isC & vm;  // bit 7 of each byte: a unit starts here
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if ((keep >> (8 * q + 7)) & 1u) {
          // the four bytes from this position on
          const uint32_t x = __byte_perm(W[k + 1], W[k + 2], 0x3210 + 0x1111 * q);
          const uint32_t b0 = x & 0xFFu, b1 = (x >> 8) & 0x3Fu, b2 = (x >> 16) & 0x3Fu, b3 = (x >> 24) & 0x3Fu;
          const uint32_t cp = b0 < 0x80u   ? b0
                              : b0 < 0xE0u ? ((b0 & 0x1Fu) << 6) | b1
                              : b0 < 0xF0u ? ((b0 & 0x0Fu) << 12) | (b1 << 6) | b2
                                           : ((b0 & 0x07u) << 18) | (b1 << 12) | (b2 << 6) | b3;
          st[addr++] = cp;
        }
      }
    }
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    return Region{rtot, 0u, 0u, rtot};
  }
};

// ---- UTF-32 -> UTF-16LE codec ----------------------------------------------------------------

struct Utf32ToUtf16 {
  using Out = uint16_t;
  static constexpr uint32_t STAGE = 2 * 128 + 32;  // 128 units of at most 2 words + alignment slack
  static constexpr uint32_t F_NONASCII = 1;        // a unit >= 0x80 (or a chunk at a buffer end)
  static constexpr uint32_t ASCII_MASK = 0xFFFFFF80u;
  static constexpr uint32_t CHUNK_UNITS = 4;
  static constexpr uint32_t REGION_UNITS = 128;
  static constexpr uint32_t DIRECT_ALIGN = 4;  // its lanes store 4 words (8 bytes) each

  __device__ __forceinline__ static bool ascii_region(uint32_t, uint32_t rflags) { return rflags == 0; }

  __device__ __forceinline__ static void ascii_direct(uint16_t *dst, uint4 v, uint32_t, long long,
                                                      unsigned long long &) {
    const int lane = threadIdx.x & 31;
    reinterpret_cast<uint2 *>(dst)[lane] = make_uint2(__byte_perm(v.x, v.y, 0x5410), __byte_perm(v.z, v.w, 0x5410));
  }

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge,
                                                   uint32_t &flags) {
    const uint32_t U[4] = {v.x, v.y, v.z, v.w};
    if (!edge && ((U[0] | U[1] | U[2] | U[3]) & ASCII_MASK) == 0) {
      flags = 0;
      return 4;
    }
    flags = F_NONASCII;
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool valid = !edge || (c + 4 * j >= (long long)p.off0 && c + 4 * j < (long long)p.vbytes);
      n += valid ? (U[j] >= 0x10000u ? 2u : 1u) : 0u;
    }
    return n;
  }

  // One word per unit below 0x10000, else the surrogate pair (Section 3); an invalid unit flags
  // the chunk.
  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t, uint32_t, long long c,
                                                   bool edge, bool, uint16_t *st, uint32_t base, uint32_t x0,
                                                   uint32_t rtot, uint32_t, unsigned long long &err_pos) {
    const uint32_t U[4] = {v.x, v.y, v.z, v.w};
    uint32_t o = base + x0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool valid = !edge || (c + 4 * j >= (long long)p.off0 && c + 4 * j < (long long)p.vbytes);
      if (!valid) continue;
      const uint32_t u = U[j];
      bad = bad || utf32_bad(u);
      if (u < 0x10000u) {
        st[o++] = (uint16_t)u;
      } else {
        const uint32_t t = u - 0x10000u;
        st[o] = (uint16_t)(0xD800u + ((t >> 10) & 0x3FFu));
        st[o + 1] = (uint16_t)(0xDC00u + (t & 0x3FFu));
        o += 2;
      }
    }
    if (bad && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    return Region{rtot, 0u, 0u, rtot};
  }
};

// ---- UTF-16LE -> UTF-32 codec ----------------------------------------------------------------

struct Utf16ToUtf32 {
  using Out = uint32_t;
  static constexpr uint32_t STAGE = 256 + 32;  // at most one unit per word + alignment slack
  static constexpr uint32_t F_NONASCII = 1;    // a word >= 0x80 (or a chunk at a buffer end)
  static constexpr uint32_t ASCII_MASK = 0xFF80FF80u;
  static constexpr uint32_t CHUNK_UNITS = 8;
  static constexpr uint32_t REGION_UNITS = 256;
  static constexpr uint32_t DIRECT_ALIGN = 4;  // its lanes store 8 units (32 bytes) each

  __device__ __forceinline__ static bool ascii_region(uint32_t, uint32_t rflags) { return rflags == 0; }

  __device__ __forceinline__ static void ascii_direct(uint32_t *dst, uint4 v, uint32_t, long long,
                                                      unsigned long long &) {
    const int lane = threadIdx.x & 31;
    uint4 *d = reinterpret_cast<uint4 *>(dst) + 2 * lane;
    d[0] = make_uint4(v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16);
    d[1] = make_uint4(v.z & 0xFFFFu, v.z >> 16, v.w & 0xFFFFu, v.w >> 16);
  }

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge,
                                                   uint32_t &flags) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    if (!edge && ((W[0] | W[1] | W[2] | W[3]) & ASCII_MASK) == 0) {
      flags = 0;
      return 8;
    }
    flags = F_NONASCII;
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t w = (W[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
      const bool valid = !edge || (c + 2 * j >= (long long)p.off0 && c + 2 * j < (long long)p.vbytes);
      n += (valid && !is_low16(w)) ? 1u : 0u;
    }
    return n;
  }

  // A word that is not a second surrogate stores one unit: its value, or with its partner the
  // pair's value (the partner may be the next region's first word, `next`).  A word breaking
  // the pair rules flags the chunk.
  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t prev, uint32_t next,
                                                   long long c, bool edge, bool, uint32_t *st, uint32_t base,
                                                   uint32_t x0, uint32_t rtot, uint32_t,
                                                   unsigned long long &err_pos) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    uint32_t u[10];  // u[0] = word before the chunk, u[1..8] own words, u[9] = word after
    u[0] = prev >> 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      u[1 + 2 * k] = W[k] & 0xFFFFu;
      u[2 + 2 * k] = W[k] >> 16;
    }
    u[9] = next & 0xFFFFu;
    uint32_t o = base + x0;
    bool err = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool valid = !edge || (c + 2 * j >= (long long)p.off0 && c + 2 * j < (long long)p.vbytes);
      if (!valid) continue;
      const uint32_t w = u[j + 1];
      const bool hs = is_high16(w), ls = is_low16(w);
      const bool pair = hs && is_low16(u[j + 2]);
      err = err || (hs && !pair) || (ls && !is_high16(u[j]));
      if (!ls) st[o++] = pair ? (((w & 0x3FFu) << 10) | (u[j + 2] & 0x3FFu)) + 0x10000u : w;
    }
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    return Region{rtot, 0u, 0u, rtot};
  }
};

__global__ void __launch_bounds__(XT, XBLOCKS) utf32_to_utf16_kernel(const Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(XSmem), set at launch
  XSmem<Utf32ToUtf16> &sm = *reinterpret_cast<XSmem<Utf32ToUtf16> *>(smem_raw);
  transcode<Utf32ToUtf16>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
    if (status) {
      write_result(p.result, GBU_TIMEOUT, 0);
    } else if (key != NO_ERROR) {
      int32_t kind;
      uint64_t off;
      resolve_utf32_error(reinterpret_cast<const uint32_t *>(p.base + p.off0), p.n,
                          ((long long)key - (long long)p.off0) / 4, &kind, &off);
      write_result(p.result, kind, off);
    } else {
      write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
    }
  });
}

__global__ void __launch_bounds__(XT, XBLOCKS) utf16_to_utf32_kernel(const Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(XSmem), set at launch
  XSmem<Utf16ToUtf32> &sm = *reinterpret_cast<XSmem<Utf16ToUtf32> *>(smem_raw);
  transcode<Utf16ToUtf32>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
    if (status) {
      write_result(p.result, GBU_TIMEOUT, 0);
    } else if (key != NO_ERROR) {
      uint64_t off;
      resolve_utf16_error(reinterpret_cast<const uint16_t *>(p.base + p.off0), p.n,
                          ((long long)key - (long long)p.off0) / 2, &off);
      write_result(p.result, GBU_SURROGATE, off);
    } else {
      write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
    }
  });
}

__global__ void __launch_bounds__(XT, XBLOCKS) utf32_to_utf8_kernel(const Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(XSmem), set at launch
  XSmem<Utf32ToUtf8> &sm = *reinterpret_cast<XSmem<Utf32ToUtf8> *>(smem_raw);
  transcode<Utf32ToUtf8>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
    if (status) {
      write_result(p.result, GBU_TIMEOUT, 0);
    } else if (key != NO_ERROR) {
      int32_t kind;
      uint64_t off;
      resolve_utf32_error(reinterpret_cast<const uint32_t *>(p.base + p.off0), p.n,
                          ((long long)key - (long long)p.off0) / 4, &kind, &off);
      write_result(p.result, kind, off);
    } else {
      write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
    }
  });
}

__global__ void __launch_bounds__(XT, XBLOCKS) utf8_to_utf32_kernel(const Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(XSmem), set at launch
  XSmem<Utf8ToUtf32> &sm = *reinterpret_cast<XSmem<Utf8ToUtf32> *>(smem_raw);
  transcode<Utf8ToUtf32>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
    if (status) {
      write_result(p.result, GBU_TIMEOUT, 0);
    } else if (key != NO_ERROR) {
      int32_t kind;
      uint64_t off;
      resolve_utf8_error(p.base + p.off0, p.n, (long long)key - (long long)p.off0, &kind, &off);
      write_result(p.result, kind, off);
    } else {
      write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
    }
  });
}

const void *utf32_stream_kernel_ptr(int mode) {
  switch (mode) {
    case U_V32: return (const void *)utf32_stream_kernel<U_V32>;
    case U_L8: return (const void *)utf32_stream_kernel<U_L8>;
    case U_L16: return (const void *)utf32_stream_kernel<U_L16>;
    case U_L32F16: return (const void *)utf32_stream_kernel<U_L32F16>;
    default: return (const void *)utf32_stream_kernel<U_L32>;
  }
}
const void *utf32_to_utf16_kernel_ptr() { return (const void *)utf32_to_utf16_kernel; }
size_t utf32_to_utf16_smem_bytes() { return sizeof(XSmem<Utf32ToUtf16>); }
const void *utf16_to_utf32_kernel_ptr() { return (const void *)utf16_to_utf32_kernel; }
size_t utf16_to_utf32_smem_bytes() { return sizeof(XSmem<Utf16ToUtf32>); }
const void *utf32_to_utf8_kernel_ptr() { return (const void *)utf32_to_utf8_kernel; }
size_t utf32_to_utf8_smem_bytes() { return sizeof(XSmem<Utf32ToUtf8>); }
const void *utf8_to_utf32_kernel_ptr() { return (const void *)utf8_to_utf32_kernel; }
size_t utf8_to_utf32_smem_bytes() { return sizeof(XSmem<Utf8ToUtf32>); }

}  // namespace gbu
