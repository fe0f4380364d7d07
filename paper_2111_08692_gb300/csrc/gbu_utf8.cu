// gbu_utf8.cu -- kernels whose input is UTF-8: validation, UTF-16 length, UTF-8 -> UTF-16LE.
//
// What is computed (paper Section 3): a leading byte's top bits give the sequence length
// (0xxxxxxx, 110xxxxx, 1110xxxx, 11110xxx); continuation bytes are 10xxxxxx; the six rules
// make a byte sequence valid.  Section 4's design (64-byte blocks, a 12-byte shuffle-table
// routine) is a 128-bit-register idiom; here each consumer thread owns 16 input bytes of a
// tile and works on 32-bit words:
//   * classification (SWAR): per byte, flags "continuation", ">= C0", ">= E0", ">= F0" as the
//     most significant bit of each byte of a word;
//   * structure (rules 1-3): a byte must be a continuation exactly when one of the three
//     bytes before it is a leading byte that needs it (>= C0 one back, >= E0 two back, >= F0
//     three back); the three flag words are funnel-shifted by 1, 2 and 3 bytes and compared
//     with the continuation flags (positions past the end of the input hold zero bytes, so a
//     cut sequence fails there);
//   * values (rules 4-6, and rule 1 for F8-FF): each position is decoded as if it were a
//     leading byte, two positions per 32-bit register (16-bit lanes), and the decoded value
//     is range-checked for its class: two-byte >= U+80, three-byte >= U+800 and outside
//     D800-DFFF, four-byte in U+10000-10FFFF (tested on the high surrogate it produces);
//   * output: one UTF-16 word per leading byte, two for a four-byte sequence; the word
//     offsets are prefix sums of per-byte counts (bytes inside a word via a multiply by
//     0x01010101, threads via a warp/CTA scan, tiles via the producer's look-back scan);
//   * an all-ASCII warp takes a fast path that widens bytes directly (Section 4's ASCII path).
// A thread whose 16 bytes break any check reports its chunk start; the first error lies in
// [start - 3, start + 15], and the last CTA finds its exact offset and kind by decoding that
// short stretch in reading order (resolve_utf8_error).
#include <stdint.h>

#include "gbu_device.cuh"
#include "gbu_kernels.h"

namespace gbu {

enum Utf8Mode { U8_VALIDATE = 0, U8_LENGTH = 1, U8_CONVERT = 2 };

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

// Decodes in reading order from a position at or before the first error (backed up to a
// byte that starts a character) and returns the first ill-formed sequence (kind, offset).
// Single thread; used only on error.
__device__ void resolve_utf8_error(const uint8_t *s, uint64_t n, long long chunk, int32_t *kind,
                                   uint64_t *off) {
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

// UTF-16 words of one tile (length formula), counted by one warp.
__device__ __forceinline__ uint32_t count_utf16_units_warp(const Params &p, uint32_t tile,
                                                           const uint8_t *win) {
  const int lane = threadIdx.x & 31;
  uint32_t cnt = 0;
#pragma unroll
  for (int r = 0; r < NC / 32; ++r) {
    const int chunk = r * 32 + lane;
    const long long c = (long long)tile * TILE_BYTES + (long long)CHUNK * chunk;
    const bool edge = c < (long long)p.off0 || c + (long long)CHUNK > (long long)p.vbytes;
    const uint4 v = *reinterpret_cast<const uint4 *>(win + HALO + CHUNK * chunk);
    const uint32_t W[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const Flags8 f = classify8(W[k]);
      const uint32_t vm = edge ? byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes) : 0x80808080u;
      cnt += __popc(~f.isC & vm) + __popc(f.geF0 & vm);
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
  return cnt;
}

template <int MODE>
struct Utf8Cfg {
  static constexpr int NS = MODE == U8_CONVERT ? 4 : 8;  // input ring depth
};

template <int MODE>
struct Utf8Smem {
  PipeSmem<Utf8Cfg<MODE>::NS> pipe;
  uint8_t win[Utf8Cfg<MODE>::NS][WIN_BYTES];
};

// Output staging: at most 2 words per input byte (F0-FF count 2 each), plus alignment slack.
constexpr uint32_t STAGE8_UNITS = 2 * TILE_BYTES + 8;

template <int MODE>
__global__ void __launch_bounds__(NTHREADS) utf8_kernel(const Params p) {
  constexpr int NS = Utf8Cfg<MODE>::NS;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  Utf8Smem<MODE> &sm = *reinterpret_cast<Utf8Smem<MODE> *>(smem_raw);
  uint16_t *staging =
      reinterpret_cast<uint16_t *>(smem_raw + ((sizeof(Utf8Smem<MODE>) + 127) & ~size_t(127)));
  PipeSmem<NS> &ps = sm.pipe;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t epoch = p.ws->epoch;
  pipe_init(ps, MODE == U8_CONVERT ? 1u : (uint32_t)NCW);

  unsigned long long err_pos = NO_ERROR;  // smallest erroring chunk start seen by this thread
  unsigned long long total = 0;           // length / output units counted by this thread

  if (warp == PRODUCER_WARP) {
    if (MODE == U8_CONVERT) {
      run_producer<NS, true>(p, ps, sm.win, epoch, [&](uint32_t t, const uint8_t *w) {
        return count_utf16_units_warp(p, t, w);
      });
    } else {
      run_producer<NS, false>(p, ps, sm.win, epoch, [](uint32_t, const uint8_t *) { return 0u; });
    }
  } else {
    for (uint32_t it = 0;; ++it) {
      const int s = it % NS;
      mbar_wait(p, &ps.ready[s], (it / NS) & 1);
      const TileInfo inf = ps.info[s];
      if (inf.tile >= p.ntiles) break;
      const uint32_t tile = inf.tile;

      const uint8_t *my = sm.win[s] + HALO + CHUNK * tid;
      const uint4 v = *reinterpret_cast<const uint4 *>(my);
      uint32_t W[6];
      W[0] = *reinterpret_cast<const uint32_t *>(my - 4);  // previous word
      W[1] = v.x; W[2] = v.y; W[3] = v.z; W[4] = v.w;
      W[5] = *reinterpret_cast<const uint32_t *>(my + 16);  // next word
      const long long c = (long long)tile * TILE_BYTES + (long long)CHUNK * tid;  // virtual pos of W[1]
      const bool edge = c < (long long)p.off0 || c + (long long)CHUNK > (long long)p.vbytes;

      Flags8 f[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) f[k] = classify8(W[k]);

      // counted (and, when converting, written) positions: not continuations, inside the data
      uint32_t lead[4], four[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t vm = 0x80808080u;
        if (edge) vm = byte_range_mask(c + 4 * k, p.off0, (long long)p.vbytes);
        lead[k] = ~f[k + 1].isC & 0x80808080u & vm;
        four[k] = f[k + 1].geF0 & vm;
      }
      uint32_t cnt = 0;
      uint32_t excl_b[4];  // per byte: words before this byte inside its 32-bit word
      uint32_t base_w[4];  // words before each 32-bit word inside the chunk
      if (MODE != U8_VALIDATE) {
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t u = (lead[k] >> 7) + (four[k] >> 7);
          const uint32_t incl = u * 0x01010101u;
          excl_b[k] = incl - u;
          base_w[k] = acc;
          acc += incl >> 24;
        }
        cnt = acc;
      }

      if (MODE == U8_LENGTH) {
        total += cnt;
        __syncwarp();
        if (lane == 0) mbar_arrive(&ps.empty[s]);
        continue;
      }

      // ---- validation ----------------------------------------------------------------
      uint32_t err = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t req = __funnelshift_l(f[k].geC0, f[k + 1].geC0, 8) |
                             __funnelshift_l(f[k].geE0, f[k + 1].geE0, 16) |
                             __funnelshift_l(f[k].geF0, f[k + 1].geF0, 24);
        err |= req ^ f[k + 1].isC;
      }
      const uint32_t nonascii = (W[1] | W[2] | W[3] | W[4]) & 0x80808080u;
      const bool warp_ascii = __all_sync(0xffffffffu, nonascii == 0 && !edge);

      uint32_t R[8], L4[8];  // decoded words per pair of positions (lanes); second words of 4-byte
      if (!warp_ascii) {
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
        // pair i covers positions 2i, 2i+1; E[i] = bytes (2i, 2i+1), O[i] = bytes (2i+1, 2i+2)
        uint32_t E[9], O[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int k = i >> 1, h = i & 1;
          E[i] = __byte_perm(W[k + 1], W[k + 2 <= 5 ? k + 2 : 5], selE(h));
          O[i] = __byte_perm(W[k + 1], W[k + 2 <= 5 ? k + 2 : 5], selO(h));
        }
        uint32_t bad = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = i >> 1, h = i & 1;
          uint32_t r = E[i] & 0x00FF00FFu;
          L4[i] = 0;
          if (has2 || has3 || has4) {
            const uint32_t U2 = ((E[i] << 6) & 0x07C007C0u) | (O[i] & 0x003F003Fu);
            if (has2) {
              const uint32_t M2 = prmt(f[k + 1].geC0 & ~f[k + 1].geE0, 0, selM(h));
              const uint32_t t = E[i] & 0x001E001Eu;  // U2 < 0x80 exactly when the lead is C0/C1
              bad |= ~(t + 0x7FFF7FFFu) & M2 & 0x80008000u;
              r = (U2 & M2) | (r & ~M2);
            }
            if (has3) {
              const uint32_t M3 = prmt(f[k + 1].geE0 & ~f[k + 1].geF0, 0, selM(h));
              const uint32_t U3 = ((U2 << 6) & 0xFFC0FFC0u) | (E[i + 1] & 0x003F003Fu);
              const uint32_t t = (U3 >> 11) & 0x001F001Fu;  // 0: below U+800; 0x1B: D800-DFFF
              const uint32_t nz0 = t + 0x7FFF7FFFu;
              const uint32_t nzS = (t ^ 0x001B001Bu) + 0x7FFF7FFFu;
              bad |= ~(nz0 & nzS) & M3 & 0x80008000u;
              r = (U3 & M3) | (r & ~M3);
            }
            if (has4) {
              const uint32_t M4 = prmt(f[k + 1].geF0, 0, selM(h));
              const uint32_t hi = (U2 << 2) + ((E[i + 1] >> 4) & 0x00030003u) + 0xC7C0C7C0u;
              const uint32_t lo =
                  ((E[i + 1] << 6) & 0x03C003C0u) | (O[i + 1] & 0x003F003Fu) | 0xDC00DC00u;
              const uint32_t t = ((hi ^ 0xD800D800u) >> 10) & 0x003F003Fu;  // 0 iff U+10000-10FFFF
              bad |= (t + 0x7FFF7FFFu) & M4 & 0x80008000u;
              r = (hi & M4) | (r & ~M4);
              L4[i] = lo;
            }
          }
          R[i] = r;
        }
        err |= bad;
      }
      if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;

      if (MODE == U8_VALIDATE) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&ps.empty[s]);
        continue;
      }

      // ---- conversion: offsets, staging, write-back -------------------------------------
      if (tid == 0) bulk_wait_read<1>();  // the staging buffer written below is free again
      uint32_t tile_total;
      const uint32_t texcl = consumer_exclusive_scan(cnt, ps.warp_sums, &tile_total);
      const uint64_t S = inf.excl;
      uint16_t *st = staging + (it & 1) * STAGE8_UNITS;
      const uint32_t x0 = (uint32_t)((p.dshift + S) & 7) + texcl;  // this thread's first word

      if (warp_ascii) {
        uint32_t u[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          u[2 * k] = __byte_perm(W[k + 1], 0, 0x4140);
          u[2 * k + 1] = __byte_perm(W[k + 1], 0, 0x4342);
        }
        stage16(st, x0, u);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int k = j >> 2, b = j & 3, i = j >> 1;
          if (lead[k] & (0x80u << (8 * b))) {
            const uint32_t o = x0 + base_w[k] + ((excl_b[k] >> (8 * b)) & 0xFF);
            st[o] = (uint16_t)((j & 1) ? (R[i] >> 16) : (R[i] & 0xFFFF));
            if (four[k] & (0x80u << (8 * b)))
              st[o + 1] = (uint16_t)((j & 1) ? (L4[i] >> 16) : (L4[i] & 0xFFFF));
          }
        }
      }
      fence_proxy_async_smem();  // staging writes -> visible to the bulk-copy engine
      consumer_sync();           // staging complete; every consumer is done with stage s
      if (tid == 0) mbar_arrive(&ps.empty[s]);
      store_staged<uint16_t>(p, st, S, tile_total);
    }
    if (MODE == U8_CONVERT && tid == 0) bulk_wait_all<0>();
  }

  cta_fold(p, ps, err_pos, total, MODE != U8_LENGTH, MODE == U8_LENGTH);

  if (finish_cta(p, ps)) {
    if (tid == 0) {
      WsHeader *ws = p.ws;
      const uint32_t status = *(volatile uint32_t *)&ws->status;
      const unsigned long long key = *(volatile unsigned long long *)&ws->errkey;
      const unsigned long long tot = *(volatile unsigned long long *)&ws->total;
      if (MODE == U8_LENGTH) {
        *p.len_out = tot;
      } else if (status) {
        write_result(p.result, GBU_TIMEOUT, 0);
      } else if (key != NO_ERROR) {
        int32_t kind;
        uint64_t off;
        const uint8_t *src = p.base + p.off0;
        resolve_utf8_error(src, p.n, (long long)key - (long long)p.off0, &kind, &off);
        write_result(p.result, kind, off);
      } else if (MODE == U8_CONVERT) {
        write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
      } else {
        write_result(p.result, GBU_OK, p.n);
      }
    }
    reset_workspace(p);
  }
}

size_t utf8_smem_bytes(int mode) {
  size_t base;
  switch (mode) {
    case U8_VALIDATE: base = sizeof(Utf8Smem<U8_VALIDATE>); break;
    case U8_LENGTH: base = sizeof(Utf8Smem<U8_LENGTH>); break;
    default: base = sizeof(Utf8Smem<U8_CONVERT>); break;
  }
  base = (base + 127) & ~size_t(127);
  if (mode == U8_CONVERT) base += 2 * STAGE8_UNITS * sizeof(uint16_t);
  return base;
}

const void *utf8_kernel_ptr(int mode) {
  switch (mode) {
    case U8_VALIDATE: return (const void *)utf8_kernel<U8_VALIDATE>;
    case U8_LENGTH: return (const void *)utf8_kernel<U8_LENGTH>;
    default: return (const void *)utf8_kernel<U8_CONVERT>;
  }
}

}  // namespace gbu
