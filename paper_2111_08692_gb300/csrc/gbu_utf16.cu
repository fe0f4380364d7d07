// gbu_utf16.cu -- the UTF-16LE -> UTF-8 transcoder (validating).
//
// Paper Section 3: words 0000-D7FF and E000-FFFF are characters by themselves; a word in
// D800-DBFF must be followed by one in DC00-DFFF and the pair encodes
// ((first & 0x3FF) << 10 | (second & 0x3FF)) + 0x10000.  Section 4 routes whole registers
// by range (all ASCII, all below 0x800, no surrogates, else a scalar fallback); here the
// partition loop of gbu_xcode.cuh hands each lane 8 words (16 bytes) per round:
//   * a word is in error when it is a first surrogate not followed by a second one, or a
//     second surrogate not preceded by a first one (neighbours come from adjacent lanes);
//   * UTF-8 sizes: 1 byte below 0x80, 2 below 0x800, 3 otherwise, and 2 per surrogate word:
//     the first word of a pair writes all 4 bytes of the character, over its own 2 slots and
//     its partner's, and the second word writes nothing.  A pair cut by a region boundary is
//     written by the region holding its first word (2 bytes past its end), and the next
//     region leaves its first 2 slots alone;
//   * an all-ASCII warp narrows words to bytes directly (Section 4's ASCII route);
//   * other words are encoded one at a time into the warp's staging buffer.
#include <stdint.h>

#include "gbu_chunk.cuh"
#include "gbu_device.cuh"
#include "gbu_kernels.h"
#include "gbu_xcode.cuh"

namespace gbu {

struct Utf16ToUtf8 {
  using Out = uint8_t;
  // a region of 256 words yields at most 768 bytes, +2 for a pair cut at its end, plus 15
  // bytes of alignment slack
  static constexpr uint32_t STAGE = 3 * 256 + 32;

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
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
                                                   uint32_t next, long long c, bool edge,
                                                   uint8_t *st, uint32_t base,
                                                   unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
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

    const uint32_t nonascii = (W[0] | W[1] | W[2] | W[3]) & 0xFF80FF80u;
    const bool warp_ascii = __all_sync(0xffffffffu, nonascii == 0 && !edge);
    uint32_t cnt = 0;
    uint32_t sz[8];
    bool err = false;
    if (warp_ascii) {
      cnt = 8;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t w = u[j + 1];
        sz[j] = valid[j] ? len8_of_word(w) : 0u;
        cnt += sz[j];
        const bool hw = is_high16(w), lw = is_low16(w);
        err |= valid[j] && ((hw && !is_low16(u[j + 2])) || (lw && !is_high16(u[j])));
      }
    }
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;

    Region g;
    const uint32_t x0 = base + warp_exclusive_scan(cnt, &g.total);
    // a pair cut by the region's start or end (lane 0's first word, lane 31's last word)
    const bool cut_start = valid[0] && is_low16(u[1]) && is_high16(u[0]);
    const bool cut_end = valid[7] && is_high16(u[8]) && is_low16(u[9]);
    g.skip = __shfl_sync(0xffffffffu, cut_start ? 2u : 0u, 0);
    g.extra = __shfl_sync(0xffffffffu, cut_end ? 2u : 0u, 31);
    if (warp_ascii) {
      const uint32_t lo8 = __byte_perm(W[0], W[1], 0x6420);
      const uint32_t hi8 = __byte_perm(W[2], W[3], 0x6420);
      if ((x0 & 7) == 0) {
        *reinterpret_cast<uint2 *>(st + x0) = make_uint2(lo8, hi8);
      } else if ((x0 & 3) == 0) {
        reinterpret_cast<uint32_t *>(st + x0)[0] = lo8;
        reinterpret_cast<uint32_t *>(st + x0)[1] = hi8;
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          st[x0 + b] = (uint8_t)(lo8 >> (8 * b));
          st[x0 + 4 + b] = (uint8_t)(hi8 >> (8 * b));
        }
      }
    } else {
      uint32_t o = x0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t w = u[j + 1];
        uint32_t nb = sz[j];  // bytes written by this word
        uint32_t bytes;
        if (is_high16(w) && is_low16(u[j + 2])) {
          const uint32_t cp = (((w & 0x3FFu) << 10) | (u[j + 2] & 0x3FFu)) + 0x10000u;
          bytes = (0xF0u | (cp >> 18)) | ((0x80u | ((cp >> 12) & 0x3Fu)) << 8) |
                  ((0x80u | ((cp >> 6) & 0x3Fu)) << 16) | ((0x80u | (cp & 0x3Fu)) << 24);
          nb = valid[j] ? 4u : 0u;
        } else if (is_low16(w) && is_high16(u[j])) {
          nb = 0;  // written with its first word
        } else if (nb == 1) {
          bytes = w;
        } else if (nb == 2) {
          // a two-byte character, or a lone surrogate (output unspecified past an error)
          bytes = (0xC0u | (w >> 6)) | ((0x80u | (w & 0x3Fu)) << 8);
        } else {
          bytes = (0xE0u | (w >> 12)) | ((0x80u | ((w >> 6) & 0x3Fu)) << 8) |
                  ((0x80u | (w & 0x3Fu)) << 16);
        }
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q)
          if (q < nb && o + q < STAGE) st[o + q] = (uint8_t)(bytes >> (8 * q));
        o += sz[j];
      }
    }
    if (g.total + g.extra > STAGE - base) {  // only after the first error
      g.extra = 0;
      if (g.total > STAGE - base) g.total = STAGE - base;
    }
    return g;
  }
};

__global__ void __launch_bounds__(XT, 2) utf16_to_utf8_kernel(const Params p) {
  __shared__ XSmem<Utf16ToUtf8> sm;
  transcode<Utf16ToUtf8>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
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

const void *utf16_to_utf8_kernel_ptr() { return (const void *)utf16_to_utf8_kernel; }

}  // namespace gbu
