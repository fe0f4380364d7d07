// gbu_stream.cu -- read-only kernels: validate_utf8, utf16_length_from_utf8,
// validate_utf16le, utf8_length_from_utf16le.
//
// These never wait on another CTA, so they stream straight from global memory: each warp
// owns 4 KB warp tiles (round-robin over all warps of the grid), issues all eight 16-byte
// loads of a lane before using any (ld.global.nc, no L1 allocation), and takes each chunk's
// neighbouring words from the adjacent lanes with shuffles (the warp tile's outer
// neighbours with two extra 4-byte loads).  Only the warp tiles that straddle the ends of
// the buffer read byte by byte with bounds checks.  Per-thread results (smallest erroring
// chunk start, or unit count) are folded over the CTA and into the workspace; the last CTA
// writes the result.
#include <stdint.h>

#include "gbu_chunk.cuh"
#include "gbu_device.cuh"
#include "gbu_kernels.h"

namespace gbu {

enum StreamMode { S_V8 = 0, S_L16 = 1, S_V16 = 2, S_L8 = 3, S_V16BE = 4, S_L8BE = 5 };

// A UTF-16BE mode runs its UTF-16LE mode on words whose two bytes it exchanges after loading.
template <int MODE>
__host__ __device__ constexpr int base_mode() { return MODE == S_V16BE ? S_V16 : (MODE == S_L8BE ? S_L8 : MODE); }
template <int MODE>
__host__ __device__ constexpr bool big_endian() { return MODE == S_V16BE || MODE == S_L8BE; }
__device__ __forceinline__ uint32_t swap16x2(uint32_t w) { return __byte_perm(w, 0, 0x2301); }

constexpr int ST_WARPS = STREAM_THREADS / 32;
constexpr int ST_ROUNDS = 8;                              // 16-byte chunks per lane per tile
constexpr uint32_t WT_BYTES = 32u * 16u * ST_ROUNDS;      // 4096 bytes per warp tile

// Resident CTAs per SM the register budget is held to: three for the validations (at most 80
// registers), four for the lengths (64).
template <int MODE>
__host__ __device__ constexpr int stream_min_blocks() {
  return (base_mode<MODE>() == S_L16 || base_mode<MODE>() == S_L8) ? 4 : 3;
}

template <int KMODE>
__global__ void __launch_bounds__(STREAM_THREADS, stream_min_blocks<KMODE>()) stream_kernel(const Params p) {
  constexpr int MODE = base_mode<KMODE>();
  constexpr bool BE = big_endian<KMODE>();
  __shared__ unsigned long long red[ST_WARPS];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * ST_WARPS + warp;
  const long long nw = (long long)gridDim.x * ST_WARPS;
  const long long lo = p.off0, hi = (long long)p.vbytes;
  unsigned long long err_pos = NO_ERROR, total = 0;
  // Early exit (validation): a warp's tiles lie at increasing positions, so once a warp has
  // flagged a chunk it stops, and no warp starts a tile past the smallest tile flagged so far
  // (the workspace's stop tile, published at once; a snapshot is refreshed every 8th tile of
  // the warp -- all warps read that one word, so reading it every tile would queue them on one
  // L2 slice -- by a load that overlaps the tile's own loads).  The smallest flagged chunk is
  // never skipped.
  const bool early = (MODE == S_V8 || MODE == S_V16) && p.early_exit != 0;
  uint32_t known = 0xFFFFFFFFu;
  // after a tile: publish a flagged tile and stop, or take the refreshed snapshot
  uint32_t it = 0;  // tiles this warp has started
  auto stop_after_tile = [&](long long wt, uint32_t snap) -> bool {
    if (__any_sync(0xffffffffu, err_pos != NO_ERROR)) {
      if (lane == 0) atomicMin(&p.ws->stop_tile, (uint32_t)wt);
      return true;
    }
    if ((it & 7u) == 1u) known = __shfl_sync(0xffffffffu, snap, 0);
    return false;
  };

  for (long long wt = gw; wt < (long long)p.ntiles; wt += nw) {
    const long long t0 = wt * WT_BYTES;
    if (early && (uint32_t)wt > known) break;  // uniform over the warp
    uint32_t snap = 0xFFFFFFFFu;
    if (early && lane == 0 && (it & 7u) == 0) snap = ld_relaxed_u32(&p.ws->stop_tile);
    ++it;
    const bool fast = t0 - 4 >= lo && t0 + (long long)WT_BYTES + 4 <= hi;
    uint4 v[ST_ROUNDS];
    uint32_t pre, post;
#pragma unroll
    for (int r = 0; r < ST_ROUNDS; ++r) v[r] = load_chunk(p, t0 + 512 * r + 16 * lane, fast);
    if (fast) {
      pre = ldg_word(p.base + t0 - 4);
      post = ldg_word(p.base + t0 + WT_BYTES);
    } else {
      pre = load_word_checked(p, t0 - 4);
      post = load_word_checked(p, t0 + WT_BYTES);
    }
    if (BE) {
#pragma unroll
      for (int r = 0; r < ST_ROUNDS; ++r)
        v[r] = make_uint4(swap16x2(v[r].x), swap16x2(v[r].y), swap16x2(v[r].z), swap16x2(v[r].w));
      pre = swap16x2(pre);
      post = swap16x2(post);
    }
    if (MODE == S_V8 || MODE == S_L16) {
      uint32_t any = 0;
#pragma unroll
      for (int r = 0; r < ST_ROUNDS; ++r) any |= v[r].x | v[r].y | v[r].z | v[r].w;
      if (__all_sync(0xffffffffu, fast && (any & 0x80808080u) == 0)) {
        // an all-ASCII warp tile: 16 units per chunk, and the only possible error is a
        // leading byte just before the tile that wants continuation bytes in it (lane 0)
        if (MODE == S_L16) {
          total += 16 * ST_ROUNDS;
        } else if (lane == 0) {
          const Flags8 fp = classify8(pre);
          const uint32_t req = __funnelshift_l(fp.geC0, 0u, 8) | __funnelshift_l(fp.geE0, 0u, 16) |
                               __funnelshift_l(fp.geF0, 0u, 24);
          if (req && (unsigned long long)t0 < err_pos) err_pos = (unsigned long long)t0;
        }
        if (early && stop_after_tile(wt, snap)) break;
        continue;
      }
    }
    if (MODE == S_V16 && fast) {
      // A warp tile inside the buffer: surrogate flags of every word's high byte first; a tile
      // without a surrogate word has no error and needs no neighbouring words, and in any
      // other tile every chunk is judged, its neighbours taken from the adjacent lanes.
      uint32_t anys = 0;
#pragma unroll
      for (int r = 0; r < ST_ROUNDS; ++r) {
        const uint32_t Wd[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
        uint32_t P0, P1;
        utf16_high_bytes(Wd, P0, P1);
        anys |= bytes_sur(P0) | bytes_sur(P1);
      }
      if (__any_sync(0xffffffffu, anys != 0)) {
#pragma unroll
        for (int r = 0; r < ST_ROUNDS; ++r) {
          const uint32_t Wd[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
          const uint32_t up = __shfl_up_sync(0xffffffffu, v[r].w, 1);
          const uint32_t down = __shfl_down_sync(0xffffffffu, v[r].x, 1);
          const uint32_t before = r == 0 ? pre : __shfl_sync(0xffffffffu, v[r > 0 ? r - 1 : 0].w, 31);
          const uint32_t after =
              r == ST_ROUNDS - 1 ? post : __shfl_sync(0xffffffffu, v[r < ST_ROUNDS - 1 ? r + 1 : r].x, 0);
          uint32_t P0, P1;
          utf16_high_bytes(Wd, P0, P1);
          const uint32_t S0 = bytes_sur(P0), S1 = bytes_sur(P1);
          const bool bad = ((S0 | S1) != 0) & utf16_pair_errors_bytes(P0, P1, S0, S1, lane == 0 ? before : up,
                                                                    lane == 31 ? after : down);
          const long long c = t0 + 512 * r + 16 * lane;
          if (bad && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
        }
      }
      if (early && stop_after_tile(wt, snap)) break;
      continue;
    }
    // UTF-8 validation: the rounds whose chunk of this lane holds an error; the first one gives
    // the lane's error position after the tile (one test per tile instead of one per round)
    uint32_t em = 0;
#pragma unroll
    for (int r = 0; r < ST_ROUNDS; ++r) {
      const long long c = t0 + 512 * r + 16 * lane;
      const bool edge = !fast && (c < lo || c + 16 > hi);
      uint32_t W[6];
      W[1] = v[r].x; W[2] = v[r].y; W[3] = v[r].z; W[4] = v[r].w;
      const uint32_t up = __shfl_up_sync(0xffffffffu, v[r].w, 1);
      const uint32_t down = __shfl_down_sync(0xffffffffu, v[r].x, 1);
      const uint32_t before = r == 0 ? pre : __shfl_sync(0xffffffffu, v[r > 0 ? r - 1 : 0].w, 31);
      const uint32_t after =
          r == ST_ROUNDS - 1 ? post : __shfl_sync(0xffffffffu, v[r < ST_ROUNDS - 1 ? r + 1 : r].x, 0);
      W[0] = lane == 0 ? before : up;
      W[5] = lane == 31 ? after : down;

      if (MODE == S_V8) {
        // Three routes, chosen per warp region by the leading bytes it holds (and the word
        // before it): without bytes >= E0 (Latin, Cyrillic and other one- and two-byte text) a
        // byte must be a continuation byte exactly when the byte before it is >= C0, and only
        // C0/C1 can break rules 4-6; without bytes >= F0 (CJK) the >= F0 flags and tests drop
        // out; else all three lead flags.
        uint32_t s1[5], geC0[5], hi3 = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          s1[k] = W[k] << 1;
          geC0[k] = W[k] & s1[k] & 0x80808080u;
          hi3 |= geC0[k] & (W[k] << 2);
        }
        if (!__any_sync(0xffffffffu, hi3 != 0)) {
          uint32_t err = 0;
#pragma unroll
          for (int k = 1; k <= 4; ++k) {
            const uint32_t isC = W[k] & ~s1[k] & 0x80808080u;
            err |= __funnelshift_l(geC0[k - 1], geC0[k], 8) ^ isC;
            err |= geC0[k] & ~((W[k] & 0x3E3E3E3Eu) + 0x7F7F7F7Fu);  // C0, C1
          }
          em |= err ? 1u << r : 0u;
          continue;
        }
        // No leading byte >= F0 in the region (CJK and other text of one to three bytes):
        // structure by the >= C0 and >= E0 flags only (the region holds bytes E0-EF).
        Flags8 g[5];
        uint32_t hi4 = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          g[k].geC0 = geC0[k];
          g[k].geE0 = geC0[k] & (W[k] << 2);
          g[k].geF0 = g[k].geE0 & (W[k] << 3);
          g[k].isC = W[k] & ~s1[k] & 0x80808080u;
          hi4 |= g[k].geF0;
        }
        if (!__any_sync(0xffffffffu, hi4 != 0)) {
          uint32_t err = 0, c2 = 0;
#pragma unroll
          for (int k = 1; k <= 4; ++k) {
            const uint32_t req = __funnelshift_l(g[k - 1].geC0, g[k].geC0, 8) |
                                 __funnelshift_l(g[k - 1].geE0, g[k].geE0, 16);
            err |= req ^ g[k].isC;
            c2 |= g[k].geC0 & ~g[k].geE0;
          }
          err |= utf8_special_errors(W, g, __any_sync(0xffffffffu, c2 != 0), true, false);
          em |= err ? 1u << r : 0u;
          continue;
        }
        // leading bytes >= F0 occur in the region: all three flags
        uint32_t err = 0, c2 = 0, c3 = 0;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
          const uint32_t req = __funnelshift_l(g[k - 1].geC0, g[k].geC0, 8) |
                               __funnelshift_l(g[k - 1].geE0, g[k].geE0, 16) |
                               __funnelshift_l(g[k - 1].geF0, g[k].geF0, 24);
          err |= req ^ g[k].isC;
          c2 |= g[k].geC0 & ~g[k].geE0;
          c3 |= g[k].geE0 & ~g[k].geF0;
        }
        err |= utf8_special_errors(W, g, __any_sync(0xffffffffu, c2 != 0), __any_sync(0xffffffffu, c3 != 0), true);
        em |= err ? 1u << r : 0u;
        continue;
      }
      if (MODE == S_L16) {
        Flags8 f[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) f[k] = classify8(W[k]);
        total += utf8_count_units(f, c, edge, lo, hi);
      } else if (MODE == S_V16) {
        const uint32_t Wd[4] = {W[1], W[2], W[3], W[4]};
        if (utf16_chunk_errors(Wd, W[0], W[5], c, edge, lo, hi) && (unsigned long long)c < err_pos)
          err_pos = (unsigned long long)c;
      } else if (MODE == S_L8) {
        const uint32_t Wd[4] = {W[1], W[2], W[3], W[4]};
        uint32_t cnt = 0;
        if (!edge) {
          cnt = utf16_len8_inside(Wd);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t w = (Wd[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
            const bool valid = c + 2 * j >= lo && c + 2 * j < hi;
            cnt += valid ? len8_of_word(w) : 0u;
          }
        }
        total += cnt;
      }
    }
    if (MODE == S_V8 && em) {
      const unsigned long long c = (unsigned long long)(t0 + 512 * (__ffs(em) - 1) + 16 * lane);
      if (c < err_pos) err_pos = c;
    }
    if (early && stop_after_tile(wt, snap)) break;
  }

  const bool want_err = MODE == S_V8 || MODE == S_V16;
  if (!fold_and_finish<STREAM_THREADS>(p, want_err ? err_pos : total, want_err, red, &is_last)) return;
  if (threadIdx.x == 0) {
    const unsigned long long key = *(volatile unsigned long long *)&p.ws->errkey;
    const unsigned long long tot = *(volatile unsigned long long *)&p.ws->total;
    if (MODE == S_L16 || MODE == S_L8) {
      *p.len_out = tot;
    } else if (key == NO_ERROR) {
      write_result(p.result, GBU_OK, p.n);
    } else if (MODE == S_V8) {
      int32_t kind;
      uint64_t off;
      resolve_utf8_error(p.base + p.off0, p.n, (long long)key - (long long)p.off0, &kind, &off);
      write_result(p.result, kind, off);
    } else {
      uint64_t off;
      resolve_utf16_error<BE>(reinterpret_cast<const uint16_t *>(p.base + p.off0), p.n,
                              ((long long)key - (long long)p.off0) / 2, &off);
      write_result(p.result, GBU_SURROGATE, off);
    }
  }
  reset_workspace(p);
}

const void *stream_kernel_ptr(int mode) {
  switch (mode) {
    case S_V8: return (const void *)stream_kernel<S_V8>;
    case S_L16: return (const void *)stream_kernel<S_L16>;
    case S_V16: return (const void *)stream_kernel<S_V16>;
    case S_V16BE: return (const void *)stream_kernel<S_V16BE>;
    case S_L8BE: return (const void *)stream_kernel<S_L8BE>;
    default: return (const void *)stream_kernel<S_L8>;
  }
}

uint32_t stream_tile_bytes() { return WT_BYTES; }

}  // namespace gbu
