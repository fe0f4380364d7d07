// gbu_utf8.cu -- the UTF-8 -> UTF-16LE transcoder (validating).
//
// Paper Section 3 defines both formats; Section 5 states that transcoding validates.
// Section 4's design (64-byte blocks, a 12-byte shuffle-table routine) is a 128-bit-register
// idiom; here the partition loop of gbu_xcode.cuh hands each lane one 16-byte chunk per
// round:
//   * the chunk is classified and validated as in gbu_chunk.cuh;
//   * output: one UTF-16 word per leading byte, two for a four-byte sequence, counted on the
//     leading byte; word offsets are prefix sums of per-byte counts (bytes inside a word via
//     a multiply by 0x01010101, lanes via a warp scan, regions via the partition count, and
//     partitions via the look-back);
//   * an all-ASCII warp widens its bytes directly (Section 4's ASCII path).
// A lane whose chunk breaks any check reports the chunk start; the last CTA turns the
// smallest one into the exact offset and kind (resolve_utf8_error).
#include <stdint.h>

#include "gbu_chunk.cuh"
#include "gbu_device.cuh"
#include "gbu_kernels.h"
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

  __device__ __forceinline__ static uint32_t count(const Params &p, uint4 v, long long c, bool edge) {
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const Flags8 f = classify8(W[k]);
      const uint32_t vm = edge ? byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes) : 0x80808080u;
      cnt += __popc(~f.isC & vm) + __popc(f.geF0 & vm);
    }
    return cnt;
  }

  __device__ __forceinline__ static Region convert(const Params &p, uint4 v, uint32_t prev,
                                                   uint32_t next, long long c, bool edge,
                                                   uint16_t *st, uint32_t base,
                                                   unsigned long long &err_pos) {
    uint32_t W[6];
    W[0] = prev;
    W[1] = v.x; W[2] = v.y; W[3] = v.z; W[4] = v.w;
    W[5] = next;
    Flags8 f[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k] = classify8(W[k]);
    uint32_t lead[4], four[4], excl_b[4], base_w[4];
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t vm = 0x80808080u;
      if (edge) vm = byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes);
      lead[k] = ~f[k + 1].isC & 0x80808080u & vm;
      four[k] = f[k + 1].geF0 & vm;
      const uint32_t u = (lead[k] >> 7) + (four[k] >> 7);
      const uint32_t incl = u * 0x01010101u;
      excl_b[k] = incl - u;
      base_w[k] = cnt;
      cnt += incl >> 24;
    }
    uint32_t err = utf8_structure_errors(f);
    const uint32_t nonascii = (W[1] | W[2] | W[3] | W[4]) & 0x80808080u;
    const bool warp_ascii = __all_sync(0xffffffffu, nonascii == 0 && !edge);
    uint32_t R[8], L4[8];
    if (!warp_ascii) err |= utf8_value_errors<true>(W, f, R, L4);
    if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;

    Region g;
    const uint32_t x0 = base + warp_exclusive_scan(cnt, &g.total);
    g.skip = 0;
    g.extra = 0;
    if (warp_ascii) {
      uint32_t u[8];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        u[2 * k] = __byte_perm(W[k + 1], 0, 0x4140);
        u[2 * k + 1] = __byte_perm(W[k + 1], 0, 0x4342);
      }
      stage16(st, x0, u);  // an all-ASCII region fits: x0 + 16 <= 7 + 512
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int k = j >> 2, b = j & 3, i = j >> 1;
        if (lead[k] & (0x80u << (8 * b))) {
          const uint32_t o = x0 + base_w[k] + ((excl_b[k] >> (8 * b)) & 0xFF);
          if (o < STAGE) st[o] = (uint16_t)((j & 1) ? (R[i] >> 16) : (R[i] & 0xFFFF));
          if ((four[k] & (0x80u << (8 * b))) && o + 1 < STAGE)
            st[o + 1] = (uint16_t)((j & 1) ? (L4[i] >> 16) : (L4[i] & 0xFFFF));
        }
      }
    }
    if (g.total > STAGE - base) g.total = STAGE - base;  // only after the first error
    return g;
  }
};

__global__ void __launch_bounds__(XT, 2) utf8_to_utf16_kernel(const Params p) {
  __shared__ XSmem<Utf8ToUtf16> sm;
  transcode<Utf8ToUtf16>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
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

const void *utf8_to_utf16_kernel_ptr() { return (const void *)utf8_to_utf16_kernel; }

}  // namespace gbu
