// gbu_batch.cu -- batched forms of the six operations: many strings in one launch, and the
// exclusive scan that turns batched output lengths into output offsets.
//
// The strings come in CSR form (one buffer holding them back to back and B+1 offsets in
// code units) or as an array of descriptors (pointer and length of each input and output).
// A persistent grid of CTAs (NWARPS warps each) claims GRAB consecutive
// strings at a time from a counter in the workspace; inside a claim,
//   * every warp takes strings one by one (a shared-memory counter) and handles each on its
//     own, walking it in 512-byte regions (one 16-byte chunk per lane) with the same per-chunk
//     analysis and the same codecs as the single-buffer kernels, so each string's result is
//     the one a single-buffer call on it gives;
//   * a string of at least long_bytes input bytes is set aside and handled afterwards by the
//     whole CTA, NWARPS regions per step: for a transcoding each warp counts its region first
//     and the CTA scans the counts, so every region knows where its output starts.
// Strings never wait on one another, so nothing spins.  Output offsets of a transcoding come
// from the caller's dst_off (for example the exclusive scan of the batched lengths).
// The launch geometry (warps per CTA, strings per claim, long-string threshold) is chosen by
// the library's autotuner from timed candidates.
#include <stdint.h>

#include "gbu_chunk.cuh"
#include "gbu_codec_utf16.cuh"
#include "gbu_codec_utf8.cuh"
#include "gbu_device.cuh"
#include "gbu_kernels.h"

namespace gbu {

constexpr uint32_t BATCH_GRAB_MAX = 1024;  // strings per claim, at most

template <int MODE>
struct BatchTraits {
  static constexpr bool UTF8_IN = MODE == B_V8 || MODE == B_L16 || MODE == B_C8;
  static constexpr uint32_t IN_UNIT = UTF8_IN ? 1u : 2u;
  static constexpr bool CONVERT = MODE == B_C8 || MODE == B_C16;
  static constexpr bool LENGTH = MODE == B_L16 || MODE == B_L8;
  // UTF-8 validation (also inside a transcoding) judges the three positions past the end
  static constexpr uint32_t TAIL = (MODE == B_V8 || MODE == B_C8) ? 3u : 0u;
};

template <int MODE>
struct BatchCodec {
  using C = Utf8ToUtf16;
};
template <>
struct BatchCodec<B_C16> {
  using C = Utf16ToUtf8;
};

template <int MODE, int NWARPS>
struct __align__(128) BatchSmem {
  using Out = typename BatchCodec<MODE>::C::Out;
  static constexpr int SW = BatchTraits<MODE>::CONVERT ? NWARPS : 1;
  static constexpr uint32_t SU = BatchTraits<MODE>::CONVERT ? BatchCodec<MODE>::C::STAGE : 8u;
  Out staging[SW][2][SU];
  uint32_t rcount[2][NWARPS];        // long strings: units of each warp's region in a step
  unsigned long long red[NWARPS];    // long strings: per-warp error position or count
  uint32_t longs[BATCH_GRAB_MAX];    // long strings of the current claim (index in the claim)
  unsigned long long g0;             // first string of the current claim
  uint32_t next;                     // next string of the claim to hand to a warp
  uint32_t nlong;
  int is_last;
};

// The single-buffer parameters of string i (base, off0, vbytes, n; destination and cap for a
// transcoding).
template <int MODE>
__device__ __forceinline__ Params string_params(const BatchParams &bp, uint64_t i) {
  using T = BatchTraits<MODE>;
  constexpr uint32_t OUT_UNIT = MODE == B_C8 ? 2u : 1u;
  Params sp;
  uintptr_t a, da = 0;
  uint64_t n, cap = 0;
  if (bp.desc) {
    const StringDesc d = bp.desc[i];
    a = (uintptr_t)d.src;
    n = d.n;
    if (T::CONVERT) {
      da = (uintptr_t)d.dst;
      cap = d.cap;
    }
  } else {
    const uint64_t start = bp.off[i], end = bp.off[i + 1];
    n = end > start ? end - start : 0;
    a = (uintptr_t)(bp.src + start * T::IN_UNIT);
    if (T::CONVERT) {
      const uint64_t d0 = bp.dst_off[i], d1 = bp.dst_off[i + 1];
      da = (uintptr_t)(bp.dst + d0 * OUT_UNIT);
      cap = d1 > d0 ? d1 - d0 : 0;
    }
  }
  sp.base = (const uint8_t *)(a & ~(uintptr_t)15);
  sp.off0 = (uint32_t)(a & 15);
  sp.n = n;
  sp.vbytes = sp.off0 + n * T::IN_UNIT;
  sp.dbase = (uint8_t *)(da & ~(uintptr_t)15);
  sp.dshift = (uint32_t)((da & 15) / OUT_UNIT);
  sp.cap = cap;
  return sp;
}

// Input code units of string i.
__device__ __forceinline__ uint64_t string_units(const BatchParams &bp, uint64_t i) {
  if (bp.desc) return bp.desc[i].n;
  const uint64_t s = bp.off[i], e = bp.off[i + 1];
  return e > s ? e - s : 0;
}

// Virtual end of the positions to judge (0 for an empty string).
template <int MODE>
__device__ __forceinline__ long long string_span(const Params &sp) {
  return sp.n == 0 ? 0 : (long long)sp.vbytes + BatchTraits<MODE>::TAIL;
}

// The chunk at virtual position c (lane's chunk of a region) and the words just before and
// after it (one warp, all lanes).
__device__ __forceinline__ void region_load(const Params &sp, long long c, uint4 &v, uint32_t &prev,
                                            uint32_t &next) {
  const int lane = threadIdx.x & 31;
  const long long lo = sp.off0, hi = (long long)sp.vbytes;
  const bool inside = c - 4 >= lo && c + 20 <= hi;
  v = load_chunk(sp, c, inside);
  prev = __shfl_up_sync(0xffffffffu, v.w, 1);
  next = __shfl_down_sync(0xffffffffu, v.x, 1);
  if (lane == 0) prev = inside ? ldg_word(sp.base + c - 4) : load_word_checked(sp, c - 4);
  if (lane == 31) next = inside ? ldg_word(sp.base + c + 16) : load_word_checked(sp, c + 16);
}

// Read-only analysis of one chunk: the smallest erroring chunk start goes to err_pos
// (validation), the units to total (lengths).
template <int MODE>
__device__ __forceinline__ void region_read(const Params &sp, long long c, uint4 v, uint32_t prev,
                                            uint32_t next, unsigned long long &err_pos,
                                            unsigned long long &total) {
  const long long lo = sp.off0, hi = (long long)sp.vbytes;
  const bool edge = c < lo || c + 16 > hi;
  if (MODE == B_V8 || MODE == B_L16) {
    const uint32_t W[6] = {prev, v.x, v.y, v.z, v.w, next};
    Flags8 f[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k] = classify8(W[k]);
    if (MODE == B_L16) {
      total += utf8_count_units(f, c, edge, lo, hi);
    } else {
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
      if (err && (unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    }
  } else {
    const uint32_t Wd[4] = {v.x, v.y, v.z, v.w};
    if (MODE == B_L8) {
      uint32_t cnt = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t w = (Wd[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
        const bool valid = !edge || (c + 2 * j >= lo && c + 2 * j < hi);
        cnt += valid ? len8_of_word(w) : 0u;
      }
      total += cnt;
    } else if (utf16_chunk_errors(Wd, prev, next, c, edge, lo, hi)) {
      if ((unsigned long long)c < err_pos) err_pos = (unsigned long long)c;
    }
  }
}

// Converts one region whose output starts at unit S of the string's destination (one warp).
template <int MODE, int NWARPS>
__device__ __forceinline__ uint32_t region_convert(const Params &sp, long long c, uint4 v, uint32_t prev,
                                                   uint32_t next, uint64_t S, BatchSmem<MODE, NWARPS> &sm,
                                                   uint32_t &use, unsigned long long &err_pos) {
  using C = typename BatchCodec<MODE>::C;
  constexpr uint32_t V = 16 / sizeof(typename C::Out);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long lo = sp.off0, hi = (long long)sp.vbytes;
  const bool edge = c < lo || c + 16 > hi;
  typename C::Out *st = sm.staging[warp][use & 1];
  ++use;
  const uint32_t h = (uint32_t)((sp.dshift + S) & (V - 1));
  if (lane == 0) bulk_wait_read<1>();  // the store of two regions ago has read this buffer
  __syncwarp();
  const long long r0 = c - (long long)CHUNK * lane;  // the region's start
  const bool inside = r0 >= (long long)sp.off0 && r0 + (long long)REGION_BYTES <= (long long)sp.vbytes;
  const Region g = convert_counted<C>(sp, v, prev, next, c, edge, inside, st, h, err_pos);
  fence_proxy_async_smem();
  __syncwarp();
  store_region(sp, st, S, g.skip, g.total, g.extra);
  return g.units;
}

// Writes string i's result (lane 0 / thread 0).
template <int MODE>
__device__ __forceinline__ void string_result(const BatchParams &bp, uint64_t i, const Params &sp,
                                              unsigned long long err_pos, unsigned long long total,
                                              uint64_t units) {
  using T = BatchTraits<MODE>;
  if (T::LENGTH) {
    bp.lens[i] = total;
  } else if (err_pos != NO_ERROR) {
    int32_t kind = GBU_SURROGATE;
    uint64_t off;
    if (T::UTF8_IN)
      resolve_utf8_error(sp.base + sp.off0, sp.n, (long long)err_pos - (long long)sp.off0, &kind, &off);
    else
      resolve_utf16_error(reinterpret_cast<const uint16_t *>(sp.base + sp.off0), sp.n,
                          ((long long)err_pos - (long long)sp.off0) / 2, &off);
    write_result(&bp.results[i], kind, off);
  } else if (T::CONVERT) {
    write_result(&bp.results[i], units > sp.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, units);
  } else {
    write_result(&bp.results[i], GBU_OK, sp.n);
  }
}

// A string handled by one warp, region after region.
template <int MODE, int NWARPS>
__device__ __forceinline__ void warp_string(const BatchParams &bp, uint64_t i, BatchSmem<MODE, NWARPS> &sm,
                                            uint32_t &use) {
  using T = BatchTraits<MODE>;
  const int lane = threadIdx.x & 31;
  const Params sp = string_params<MODE>(bp, i);
  const long long span = string_span<MODE>(sp);
  unsigned long long err_pos = NO_ERROR, total = 0;
  uint64_t running = 0;
  for (long long r0 = 0; r0 < span; r0 += REGION_BYTES) {
    const long long c = r0 + CHUNK * lane;
    uint4 v;
    uint32_t prev, next;
    region_load(sp, c, v, prev, next);
    if (T::CONVERT)
      running += region_convert<MODE, NWARPS>(sp, c, v, prev, next, running, sm, use, err_pos);
    else
      region_read<MODE>(sp, c, v, prev, next, err_pos, total);
  }
  if (T::LENGTH) total = warp_sum_u64(total);
  else err_pos = warp_min_u64(err_pos);
  if (lane == 0) string_result<MODE>(bp, i, sp, err_pos, total, running);
}

// A string handled by the whole CTA, NWARPS regions per step (all threads).
template <int MODE, int NWARPS>
__device__ __forceinline__ void cta_string(const BatchParams &bp, uint64_t i, BatchSmem<MODE, NWARPS> &sm,
                                           uint32_t &use) {
  using T = BatchTraits<MODE>;
  using C = typename BatchCodec<MODE>::C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Params sp = string_params<MODE>(bp, i);
  const long long span = string_span<MODE>(sp);
  const long long lo = sp.off0, hi = (long long)sp.vbytes;
  unsigned long long err_pos = NO_ERROR, total = 0;
  uint64_t running = 0;
  int buf = 0;
  for (long long s0 = 0; s0 < span; s0 += (long long)NWARPS * REGION_BYTES, buf ^= 1) {
    const long long c = s0 + (long long)warp * REGION_BYTES + CHUNK * lane;
    uint4 v;
    uint32_t prev, next;
    region_load(sp, c, v, prev, next);
    if (T::CONVERT) {
      // region offsets inside the step: count first, then scan the NWARPS region counts
      const bool edge = c < lo || c + 16 > hi;
      uint32_t cf;
      uint32_t cnt = C::count(sp, v, c, edge, cf);
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
      if (lane == 0) sm.rcount[buf][warp] = cnt;
      __syncthreads();  // also: rcount[buf ^ 1] of the step before is no longer read
      uint32_t before = 0, step_total = 0;
#pragma unroll
      for (int w = 0; w < NWARPS; ++w) {
        const uint32_t x = sm.rcount[buf][w];
        before += w < warp ? x : 0u;
        step_total += x;
      }
      region_convert<MODE, NWARPS>(sp, c, v, prev, next, running + before, sm, use, err_pos);
      running += step_total;
    } else {
      region_read<MODE>(sp, c, v, prev, next, err_pos, total);
    }
  }
  unsigned long long x = T::LENGTH ? warp_sum_u64(total) : warp_min_u64(err_pos);
  if (lane == 0) sm.red[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = T::LENGTH ? 0ull : NO_ERROR;
    for (int w = 0; w < NWARPS; ++w) a = T::LENGTH ? a + sm.red[w] : (sm.red[w] < a ? sm.red[w] : a);
    string_result<MODE>(bp, i, sp, T::LENGTH ? NO_ERROR : a, T::LENGTH ? a : 0ull, running);
  }
  __syncthreads();  // sm.red and sm.rcount are reused by the next long string
}

template <int MODE, int NWARPS>
__global__ void __launch_bounds__(NWARPS * 32) batch_kernel(const BatchParams bp) {
  using T = BatchTraits<MODE>;
  __shared__ BatchSmem<MODE, NWARPS> sm;
  const int lane = threadIdx.x & 31;
  uint32_t use = 0;  // regions staged by this warp (picks its staging buffer)
  const uint32_t grab = bp.grab < 1 ? 1u : (bp.grab > BATCH_GRAB_MAX ? BATCH_GRAB_MAX : bp.grab);
  while (true) {
    if (threadIdx.x == 0) {
      sm.g0 = (unsigned long long)atomicAdd(&bp.ws->ticket, 1u) * grab;
      sm.next = 0;
      sm.nlong = 0;
    }
    __syncthreads();
    const uint64_t g0 = sm.g0;
    if (g0 >= bp.B) break;
    const uint32_t gn = bp.B - g0 < grab ? (uint32_t)(bp.B - g0) : grab;
    while (true) {
      uint32_t j = 0;
      if (lane == 0) j = atomicAdd(&sm.next, 1u);
      j = __shfl_sync(0xffffffffu, j, 0);
      if (j >= gn) break;
      const uint64_t i = g0 + j;
      if (string_units(bp, i) * T::IN_UNIT >= bp.long_bytes) {
        if (lane == 0) sm.longs[atomicAdd(&sm.nlong, 1u)] = j;
        continue;
      }
      warp_string<MODE, NWARPS>(bp, i, sm, use);
    }
    __syncthreads();
    const uint32_t nl = sm.nlong;
    for (uint32_t k = 0; k < nl; ++k) cta_string<MODE, NWARPS>(bp, g0 + sm.longs[k], sm, use);
    __syncthreads();  // sm.g0, next, nlong, longs are rewritten by the next claim
  }
  if (T::CONVERT && lane == 0) bulk_wait_all<0>();
  // the last CTA to finish resets the claim counter for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&bp.ws->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      bp.ws->ticket = 0;
      bp.ws->done = 0;
      __threadfence();
    }
  }
}

// ---- exclusive scan of uint64 values (output offsets from batched lengths) -----------------

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr uint32_t SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// out[k] = in[0] + ... + in[k-1] for k = 0 .. count (out has count + 1 entries; out[count] is
// the total).  Tiles of SCAN_TILE values are claimed by ticket and chained by the decoupled
// look-back; the last CTA writes the result {status, total} and resets the workspace.
__global__ void __launch_bounds__(SCAN_THREADS) scan_u64_kernel(const ScanParams sp) {
  __shared__ unsigned long long warp_tot[SCAN_THREADS / 32 + 1];
  __shared__ LookbackSmem<SCAN_THREADS> lb;
  __shared__ uint32_t ticket;
  __shared__ int is_last;
  const Params &p = sp.lb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t epoch = p.ws->epoch;
  while (true) {
    if (threadIdx.x == 0) ticket = atomicAdd(&p.ws->ticket, 1u);
    __syncthreads();
    const uint32_t t = ticket;
    if (t >= p.ntiles) break;
    const uint64_t b0 = (uint64_t)t * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t x[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      x[k] = b0 + k < sp.count ? sp.in[b0 + k] : 0ull;
      s += x[k];
    }
    uint64_t incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint64_t w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0ull;
      uint64_t wi = w;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, wi, d);
        if (lane >= d) wi += y;
      }
      if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;
      if (lane == SCAN_THREADS / 32 - 1) warp_tot[SCAN_THREADS / 32] = wi;
    }
    __syncthreads();
    const uint64_t tile_total = warp_tot[SCAN_THREADS / 32];
    uint64_t run = warp_tot[warp] + incl - s;
    if (threadIdx.x == 0) {
      publish_aggregate(p, t, tile_total, epoch);
      atomicAdd(&p.ws->total, (unsigned long long)tile_total);
    }
    run += lookback_cta<SCAN_THREADS>(p, t, tile_total, epoch, lb);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      if (b0 + k <= sp.count) sp.out[b0 + k] = run;
      run += x[k];
    }
    __syncthreads();  // warp_tot and ticket are rewritten by the next tile
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&p.ws->done, 1u);
    is_last = prev == gridDim.x - 1;
    if (is_last) {
      __threadfence();
      const uint32_t status = *(volatile uint32_t *)&p.ws->status;
      const unsigned long long tot = *(volatile unsigned long long *)&p.ws->total;
      // look-back values carry 44 bits: a larger total cannot be chained
      write_result(sp.result, status ? GBU_TIMEOUT : (tot > ST_VALUE_MASK ? GBU_BAD_ARGUMENT : GBU_OK), tot);
    }
  }
  __syncthreads();
  if (is_last) reset_workspace(p);
}

// ---- host-side handles -------------------------------------------------------------------

template <int MODE>
static const void *batch_ptr_for(int nwarps) {
  switch (nwarps) {
    case 4: return (const void *)batch_kernel<MODE, 4>;
    case 16: return (const void *)batch_kernel<MODE, 16>;
    default: return (const void *)batch_kernel<MODE, 8>;
  }
}

const void *batch_kernel_ptr(int mode, int nwarps) {
  switch (mode) {
    case B_V8: return batch_ptr_for<B_V8>(nwarps);
    case B_L16: return batch_ptr_for<B_L16>(nwarps);
    case B_C8: return batch_ptr_for<B_C8>(nwarps);
    case B_V16: return batch_ptr_for<B_V16>(nwarps);
    case B_L8: return batch_ptr_for<B_L8>(nwarps);
    default: return batch_ptr_for<B_C16>(nwarps);
  }
}

const void *scan_kernel_ptr() { return (const void *)scan_u64_kernel; }
uint32_t scan_tile_items() { return SCAN_TILE; }
int scan_threads() { return SCAN_THREADS; }

}  // namespace gbu
