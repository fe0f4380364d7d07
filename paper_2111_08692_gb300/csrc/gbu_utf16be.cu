// gbu_utf16be.cu -- the single-buffer transcoders between UTF-8 and UTF-16BE (validating).
//
// UTF-16BE holds the same words as UTF-16LE (Section 3's ranges and pair formula) with each
// word's most significant byte first, the byte order RFC 2781 names.  Both kernels are the
// wide UTF-16LE partition loop (gbu_wide.cuh) with a codec that exchanges the two bytes of
// every word where words meet memory: on loading UTF-16BE input (the count pass, the
// conversion pass and the neighbouring words), and on the UTF-16 output staged for a region
// (after the region is staged, before its bulk store) or widened straight from ASCII.
#include <stdint.h>

#include "gbu_kernels.h"
#include "gbu_wide_utf16.cuh"
#include "gbu_wide_utf8.cuh"

namespace gbu {

__device__ __forceinline__ uint32_t swap_words(uint32_t w) { return __byte_perm(w, 0, 0x2301); }

// UTF-16BE input: the UTF-16LE codec on byte-exchanged words.
struct Utf16BEToUtf8Wide : Utf16ToUtf8Wide {
  static constexpr uint32_t ASCII_MASK = 0x80FF80FFu;  // nonzero in a raw word: a word >= 0x80

  __device__ __forceinline__ static void swap8(const uint32_t W[8], uint32_t S[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) S[k] = swap_words(W[k]);
  }
  __device__ __forceinline__ static void wascii_direct(uint8_t *dst, const uint32_t W[8], uint32_t prev, long long c,
                                                       unsigned long long &err_pos) {
    uint32_t S[8];
    swap8(W, S);
    Utf16ToUtf8Wide::wascii_direct(dst, S, prev, c, err_pos);
  }
  __device__ __forceinline__ static uint32_t wcount(const Params &p, const uint32_t W[8], long long c, bool edge,
                                                    uint32_t &flags) {
    uint32_t S[8];
    swap8(W, S);
    return Utf16ToUtf8Wide::wcount(p, S, c, edge, flags);
  }
  __device__ __forceinline__ static Region wconvert(const Params &p, const uint32_t W[8], uint32_t prev,
                                                    uint32_t next, long long c, bool edge, bool inside, uint8_t *st,
                                                    uint32_t base, uint32_t x0, uint32_t rtot, uint32_t rflags,
                                                    unsigned long long &err_pos) {
    uint32_t S[8];
    swap8(W, S);
    return Utf16ToUtf8Wide::wconvert(p, S, swap_words(prev), swap_words(next), c, edge, inside, st, base, x0, rtot,
                                     rflags, err_pos);
  }
};

// UTF-16BE output: the UTF-8 -> UTF-16LE codec, then the staged words byte-exchanged.
struct Utf8ToUtf16BEWide : Utf8ToUtf16Wide {
  // An all-ASCII region widened straight to global memory, each byte as the word 00 xx.
  __device__ __forceinline__ static void wascii_direct(uint16_t *dst, const uint32_t W[8], uint32_t prev, long long c,
                                                       unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) check_prev_lead(prev, c, err_pos);
    uint4 *d = reinterpret_cast<uint4 *>(dst) + 4 * lane;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      d[i] = make_uint4(__byte_perm(W[2 * i], 0, 0x1404), __byte_perm(W[2 * i], 0, 0x3424),
                        __byte_perm(W[2 * i + 1], 0, 0x1404), __byte_perm(W[2 * i + 1], 0, 0x3424));
  }
  __device__ __forceinline__ static Region wconvert(const Params &p, const uint32_t W[8], uint32_t prev,
                                                    uint32_t next, long long c, bool edge, bool inside, uint16_t *st,
                                                    uint32_t base, uint32_t x0, uint32_t rtot, uint32_t rflags,
                                                    unsigned long long &err_pos) {
    const Region g =
        Utf8ToUtf16Wide::wconvert(p, W, prev, next, c, edge, inside, st, base, x0, rtot, rflags, err_pos);
    // exchange the bytes of every staged word of the region (whole 32-bit words; a word of the
    // buffer outside the region's units is never stored)
    __syncwarp();
    uint32_t *st32 = reinterpret_cast<uint32_t *>(st);
    const uint32_t w0 = base >> 1, w1 = (base + g.total + g.extra + 1) >> 1;
    for (uint32_t i = w0 + (threadIdx.x & 31); i < w1; i += 32) st32[i] = swap_words(st32[i]);
    return g;
  }
};

__global__ void __launch_bounds__(XT, XBLOCKS) utf16be_to_utf8_kernel(const Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(WSmem), set at launch
  WSmem<Utf16BEToUtf8Wide> &sm = *reinterpret_cast<WSmem<Utf16BEToUtf8Wide> *>(smem_raw);
  wtranscode<Utf16BEToUtf8Wide>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
    if (status) {
      write_result(p.result, GBU_TIMEOUT, 0);
    } else if (key != NO_ERROR) {
      uint64_t off;
      resolve_utf16_error<true>(reinterpret_cast<const uint16_t *>(p.base + p.off0), p.n,
                                ((long long)key - (long long)p.off0) / 2, &off);
      write_result(p.result, GBU_SURROGATE, off);
    } else {
      write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
    }
  });
}

__global__ void __launch_bounds__(XT, XBLOCKS) utf8_to_utf16be_kernel(const Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(WSmem), set at launch
  WSmem<Utf8ToUtf16BEWide> &sm = *reinterpret_cast<WSmem<Utf8ToUtf16BEWide> *>(smem_raw);
  wtranscode<Utf8ToUtf16BEWide>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
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

const void *utf16be_to_utf8_kernel_ptr() { return (const void *)utf16be_to_utf8_kernel; }
size_t utf16be_to_utf8_smem_bytes() { return sizeof(WSmem<Utf16BEToUtf8Wide>); }
const void *utf8_to_utf16be_kernel_ptr() { return (const void *)utf8_to_utf16be_kernel; }
size_t utf8_to_utf16be_smem_bytes() { return sizeof(WSmem<Utf8ToUtf16BEWide>); }

}  // namespace gbu
