// gbu_utf16.cu -- kernels whose input is UTF-16LE: validation, UTF-8 length, UTF-16LE -> UTF-8.
//
// What is computed (paper Section 3): words 0000-D7FF and E000-FFFF are characters by
// themselves; a word in D800-DBFF must be followed by one in DC00-DFFF and the pair encodes
// ((first & 0x3FF) << 10 | (second & 0x3FF)) + 0x10000; only surrogates need attention.
// Section 4 routes whole registers by range (all ASCII, all below 0x800, no surrogates,
// else a scalar fallback); here each consumer thread owns 8 words (16 bytes) of a tile:
//   * a word is in error when it is a first surrogate not followed by a second one, or a
//     second surrogate not preceded by a first one (the neighbours come from the halo);
//     the first flagged word is exactly the first invalid offset;
//   * UTF-8 sizes: 1 byte below 0x80, 2 below 0x800, 3 otherwise; a pair is 4 bytes, all
//     counted on its first word (the length function counts 2 per surrogate word instead,
//     which gives the same totals per tile);
//   * an all-ASCII warp narrows words to bytes directly (Section 4's ASCII route);
//   * other words are encoded one at a time into shared-memory staging at prefix-sum offsets.
#include <stdint.h>

#include "gbu_device.cuh"
#include "gbu_kernels.h"

namespace gbu {

enum Utf16Mode { U16_VALIDATE = 0, U16_LENGTH = 1, U16_CONVERT = 2 };

__device__ __forceinline__ bool is_high(uint32_t w) { return (w & 0xFC00u) == 0xD800u; }
__device__ __forceinline__ bool is_low(uint32_t w) { return (w & 0xFC00u) == 0xDC00u; }

// UTF-8 bytes of one word for the length function (2 per surrogate word).
__device__ __forceinline__ uint32_t len8_of_word(uint32_t w) {
  return w < 0x80u ? 1u : (w < 0x800u ? 2u : ((w & 0xF800u) == 0xD800u ? 2u : 3u));
}

// First unpaired surrogate at or after a chunk start (single thread; used only on error).
__device__ void resolve_utf16_error(const uint16_t *s, uint64_t n, long long chunk, uint64_t *off) {
  long long i = chunk < 0 ? 0 : chunk;
  if (i > 0 && i < (long long)n && is_low(s[i]) && is_high(s[i - 1])) --i;
  const long long stop = (chunk + 64) < (long long)n ? chunk + 64 : (long long)n;
  while (i < stop) {
    const uint32_t w = s[i];
    if ((w & 0xF800u) != 0xD800u) { ++i; continue; }
    if (is_high(w) && i + 1 < (long long)n && is_low(s[i + 1])) { i += 2; continue; }
    *off = (uint64_t)i;
    return;
  }
  *off = chunk < 0 ? 0 : (uint64_t)chunk;  // not reached for a real error
}

// UTF-8 bytes of one tile (length formula), counted by one warp.
__device__ __forceinline__ uint32_t count_utf8_bytes_warp(const Params &p, uint32_t tile,
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
    for (int j = 0; j < 8; ++j) {
      const uint32_t w = (W[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
      const long long pos = c + 2 * j;
      const bool valid = !edge || (pos >= (long long)p.off0 && pos < (long long)p.vbytes);
      cnt += valid ? len8_of_word(w) : 0u;
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
  // The consumers count a surrogate pair as 4 bytes on its first word and 0 on its second;
  // inside the tile that only moves bytes between neighbours, so the tile total differs from
  // the formula only for a pair cut by the tile's first or last word.
  const long long t0 = (long long)tile * TILE_BYTES;
  const auto word_at = [&](long long pos) -> uint32_t {
    return *reinterpret_cast<const uint16_t *>(win + (pos - (t0 - HALO)));
  };
  const auto is_data = [&](long long pos) {
    return pos >= (long long)p.off0 && pos < (long long)p.vbytes;
  };
  const long long first = t0, last = t0 + TILE_BYTES - 2;
  if (is_data(first) && is_low(word_at(first)) && is_high(word_at(first - 2))) cnt -= 2;
  if (is_data(last) && is_high(word_at(last)) && is_low(word_at(last + 2))) cnt += 2;
  return cnt;
}

template <int MODE>
struct Utf16Cfg {
  static constexpr int NS = MODE == U16_CONVERT ? 4 : 8;
};

template <int MODE>
struct Utf16Smem {
  PipeSmem<Utf16Cfg<MODE>::NS> pipe;
  uint8_t win[Utf16Cfg<MODE>::NS][WIN_BYTES];
};

constexpr uint32_t UNITS_PER_TILE = TILE_BYTES / 2;  // 2048 words
// at most 3 bytes per word, plus one pair counted in full on the tile's last word (4 bytes
// where 3 were budgeted), plus 15 bytes of alignment slack: rounded up to 16
constexpr uint32_t STAGE16_BYTES = 3 * UNITS_PER_TILE + 32;

template <int MODE>
__global__ void __launch_bounds__(NTHREADS) utf16_kernel(const Params p) {
  constexpr int NS = Utf16Cfg<MODE>::NS;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  Utf16Smem<MODE> &sm = *reinterpret_cast<Utf16Smem<MODE> *>(smem_raw);
  uint8_t *staging = smem_raw + ((sizeof(Utf16Smem<MODE>) + 127) & ~size_t(127));
  PipeSmem<NS> &ps = sm.pipe;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t epoch = p.ws->epoch;
  pipe_init(ps, MODE == U16_CONVERT ? 1u : (uint32_t)NCW);

  unsigned long long err_pos = NO_ERROR;
  unsigned long long total = 0;

  if (warp == PRODUCER_WARP) {
    if (MODE == U16_CONVERT) {
      run_producer<NS, true>(p, ps, sm.win, epoch, [&](uint32_t t, const uint8_t *w) {
        return count_utf8_bytes_warp(p, t, w);
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
      const uint32_t prevw = *reinterpret_cast<const uint32_t *>(my - 4);
      const uint32_t nextw = *reinterpret_cast<const uint32_t *>(my + 16);
      const uint32_t W[4] = {v.x, v.y, v.z, v.w};
      const long long c = (long long)tile * TILE_BYTES + (long long)CHUNK * tid;  // virtual byte
      const bool edge = c < (long long)p.off0 || c + (long long)CHUNK > (long long)p.vbytes;

      uint32_t u[10];  // u[0] = word before the chunk, u[1..8] own words, u[9] = word after
      u[0] = prevw >> 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        u[1 + 2 * k] = W[k] & 0xFFFFu;
        u[2 + 2 * k] = W[k] >> 16;
      }
      u[9] = nextw & 0xFFFFu;
      bool valid[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long pos = c + 2 * j;
        valid[j] = !edge || (pos >= (long long)p.off0 && pos < (long long)p.vbytes);
      }

      if (MODE == U16_LENGTH) {
        uint32_t cnt = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) cnt += valid[j] ? len8_of_word(u[j + 1]) : 0u;
        total += cnt;
        __syncwarp();
        if (lane == 0) mbar_arrive(&ps.empty[s]);
        continue;
      }

      const uint32_t nonascii = (W[0] | W[1] | W[2] | W[3]) & 0xFF80FF80u;
      const bool warp_ascii = __all_sync(0xffffffffu, nonascii == 0 && !edge);
      bool err = false;
      uint32_t cnt = 0;
      uint32_t sz[8];
      if (warp_ascii) {
        cnt = 8;  // no surrogate here; a first surrogate just before the chunk is flagged by
                  // the thread that owns it
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t w = u[j + 1];
          const bool hi = is_high(w), lo = is_low(w);
          const bool nlo = is_low(u[j + 2]), phi = is_high(u[j]);
          uint32_t b = w < 0x80u ? 1u : (w < 0x800u ? 2u : 3u);
          if (hi) b = nlo ? 4u : 2u;
          if (lo) b = phi ? 0u : 2u;
          if (!valid[j]) b = 0;
          err |= valid[j] && ((hi && !nlo) || (lo && !phi));
          sz[j] = b;
          cnt += b;
        }
      }
      if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;

      if (MODE == U16_VALIDATE) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&ps.empty[s]);
        continue;
      }

      if (tid == 0) bulk_wait_read<1>();
      uint32_t tile_total;
      const uint32_t texcl = consumer_exclusive_scan(cnt, ps.warp_sums, &tile_total);
      const uint64_t S = inf.excl;
      uint8_t *st = staging + (it & 1) * STAGE16_BYTES;
      const uint32_t x0 = (uint32_t)((p.dshift + S) & 15) + texcl;

      if (warp_ascii) {
        const uint32_t lo = __byte_perm(W[0], W[1], 0x6420);
        const uint32_t hi = __byte_perm(W[2], W[3], 0x6420);
        if ((x0 & 7) == 0) {
          *reinterpret_cast<uint2 *>(st + x0) = make_uint2(lo, hi);
        } else if ((x0 & 3) == 0) {
          reinterpret_cast<uint32_t *>(st + x0)[0] = lo;
          reinterpret_cast<uint32_t *>(st + x0)[1] = hi;
        } else {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            st[x0 + b] = (uint8_t)(lo >> (8 * b));
            st[x0 + 4 + b] = (uint8_t)(hi >> (8 * b));
          }
        }
      } else {
        uint32_t o = x0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t w = u[j + 1];
          const uint32_t b = sz[j];
          uint32_t bytes;
          if (b == 1) {
            bytes = w;
          } else if (b == 2) {
            // a two-byte character, or a lone surrogate (output unspecified past an error)
            bytes = (0xC0u | (w >> 6)) | ((0x80u | (w & 0x3Fu)) << 8);
          } else if (b == 3) {
            bytes = (0xE0u | (w >> 12)) | ((0x80u | ((w >> 6) & 0x3Fu)) << 8) |
                    ((0x80u | (w & 0x3Fu)) << 16);
          } else {
            const uint32_t cp = (((w & 0x3FFu) << 10) | (u[j + 2] & 0x3FFu)) + 0x10000u;
            bytes = (0xF0u | (cp >> 18)) | ((0x80u | ((cp >> 12) & 0x3Fu)) << 8) |
                    ((0x80u | ((cp >> 6) & 0x3Fu)) << 16) | ((0x80u | (cp & 0x3Fu)) << 24);
          }
#pragma unroll
          for (uint32_t q = 0; q < 4; ++q)
            if (q < b) st[o + q] = (uint8_t)(bytes >> (8 * q));
          o += b;
        }
      }
      fence_proxy_async_smem();
      consumer_sync();
      if (tid == 0) mbar_arrive(&ps.empty[s]);
      store_staged<uint8_t>(p, st, S, tile_total);
    }
    if (MODE == U16_CONVERT && tid == 0) bulk_wait_all<0>();
  }

  cta_fold(p, ps, err_pos, total, MODE != U16_LENGTH, MODE == U16_LENGTH);

  if (finish_cta(p, ps)) {
    if (tid == 0) {
      WsHeader *ws = p.ws;
      const uint32_t status = *(volatile uint32_t *)&ws->status;
      const unsigned long long key = *(volatile unsigned long long *)&ws->errkey;
      const unsigned long long tot = *(volatile unsigned long long *)&ws->total;
      if (MODE == U16_LENGTH) {
        *p.len_out = tot;
      } else if (status) {
        write_result(p.result, GBU_TIMEOUT, 0);
      } else if (key != NO_ERROR) {
        uint64_t off;
        const uint16_t *src = reinterpret_cast<const uint16_t *>(p.base + p.off0);
        resolve_utf16_error(src, p.n, ((long long)key - (long long)p.off0) / 2, &off);
        write_result(p.result, GBU_SURROGATE, off);
      } else if (MODE == U16_CONVERT) {
        write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
      } else {
        write_result(p.result, GBU_OK, p.n);
      }
    }
    reset_workspace(p);
  }
}

size_t utf16_smem_bytes(int mode) {
  size_t base;
  switch (mode) {
    case U16_VALIDATE: base = sizeof(Utf16Smem<U16_VALIDATE>); break;
    case U16_LENGTH: base = sizeof(Utf16Smem<U16_LENGTH>); break;
    default: base = sizeof(Utf16Smem<U16_CONVERT>); break;
  }
  base = (base + 127) & ~size_t(127);
  if (mode == U16_CONVERT) base += 2 * STAGE16_BYTES;
  return base;
}

const void *utf16_kernel_ptr(int mode) {
  switch (mode) {
    case U16_VALIDATE: return (const void *)utf16_kernel<U16_VALIDATE>;
    case U16_LENGTH: return (const void *)utf16_kernel<U16_LENGTH>;
    default: return (const void *)utf16_kernel<U16_CONVERT>;
  }
}

}  // namespace gbu
