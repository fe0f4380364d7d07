// gbu_utf16be.cu -- the single-buffer transcoders between UTF-8 and UTF-16BE (validating).
//
// UTF-16BE holds the same words as UTF-16LE (Section 3's ranges and pair formula) with each
// word's most significant byte first, the byte order RFC 2781 names.  Both kernels are the
// UTF-16LE partition loops with a codec that exchanges the two bytes of every word where words
// meet memory: on loading UTF-16BE input (the count pass, the conversion pass and the
// neighbouring words), and on the UTF-16 output staged for a region (after the region is
// staged, before its bulk store) or widened straight from ASCII.
#include <stdint.h>

#include "gbu_codec_utf16.cuh"
#include "gbu_codec_utf8.cuh"
#include "gbu_kernels.h"

namespace gbu {

__device__ __forceinline__ uint32_t swap_words(uint32_t w) { return __byte_perm(w, 0, 0x2301); }
__device__ __forceinline__ uint4 swap_words(uint4 v) {
  return make_uint4(swap_words(v.x), swap_words(v.y), swap_words(v.z), swap_words(v.w));
}

// UTF-16BE input: the UTF-16LE codec on byte-exchanged words.
struct Utf16BEToUtf8 : Utf16ToUtf8 {
  static constexpr uint32_t ASCII_MASK = 0x80FF80FFu;  // nonzero in a raw word: a word >= 0x80

  __device__ __forceinline__ static void ascii_direct(uint8_t *dst, uint4 v, uint32_t prev, long long c,
                                                      unsigned long long &err_pos) {
    Utf16ToUtf8::ascii_direct(dst, swap_words(v), prev, c, err_pos);
  }
  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge,
                                                   uint32_t &flags) {
    return Utf16ToUtf8::count(p, swap_words(v), c, edge, flags);
  }
  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t prev, uint32_t next,
                                                   long long c, bool edge, bool inside, uint8_t *st, uint32_t base,
                                                   uint32_t x0, uint32_t rtot, uint32_t rflags,
                                                   unsigned long long &err_pos) {
    return Utf16ToUtf8::convert(p, swap_words(v), swap_words(prev), swap_words(next), c, edge, inside, st, base, x0,
                                rtot, rflags, err_pos);
  }
};

// UTF-16BE output: the UTF-8 -> UTF-16LE codec, then the staged words byte-exchanged.
struct Utf8ToUtf16BE : Utf8ToUtf16 {
  // An all-ASCII region widened straight to global memory, each byte as the word 00 xx.
  __device__ __forceinline__ static void ascii_direct(uint16_t *dst, uint4 v, uint32_t prev, long long c,
                                                      unsigned long long &err_pos) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
      const Flags8 fp = classify8(prev);
      const uint32_t req = __funnelshift_l(fp.geC0, 0u, 8) | __funnelshift_l(fp.geE0, 0u, 16) |
                           __funnelshift_l(fp.geF0, 0u, 24);
      if (req && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    }
    const uint4 a = make_uint4(__byte_perm(v.x, 0, 0x1404), __byte_perm(v.x, 0, 0x3424),
                               __byte_perm(v.y, 0, 0x1404), __byte_perm(v.y, 0, 0x3424));
    const uint4 b = make_uint4(__byte_perm(v.z, 0, 0x1404), __byte_perm(v.z, 0, 0x3424),
                               __byte_perm(v.w, 0, 0x1404), __byte_perm(v.w, 0, 0x3424));
    uint4 *d = reinterpret_cast<uint4 *>(dst) + 2 * lane;
    d[0] = a;
    d[1] = b;
  }
  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t prev, uint32_t next,
                                                   long long c, bool edge, bool inside, uint16_t *st, uint32_t base,
                                                   uint32_t x0, uint32_t rtot, uint32_t rflags,
                                                   unsigned long long &err_pos) {
    const Region g = Utf8ToUtf16::convert(p, v, prev, next, c, edge, inside, st, base, x0, rtot, rflags, err_pos);
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
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(XSmem), set at launch
  XSmem<Utf16BEToUtf8> &sm = *reinterpret_cast<XSmem<Utf16BEToUtf8> *>(smem_raw);
  transcode<Utf16BEToUtf8>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
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
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(XSmem), set at launch
  XSmem<Utf8ToUtf16BE> &sm = *reinterpret_cast<XSmem<Utf8ToUtf16BE> *>(smem_raw);
  transcode<Utf8ToUtf16BE>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
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
size_t utf16be_to_utf8_smem_bytes() { return sizeof(XSmem<Utf16BEToUtf8>); }
const void *utf8_to_utf16be_kernel_ptr() { return (const void *)utf8_to_utf16be_kernel; }
size_t utf8_to_utf16be_smem_bytes() { return sizeof(XSmem<Utf8ToUtf16BE>); }

}  // namespace gbu
