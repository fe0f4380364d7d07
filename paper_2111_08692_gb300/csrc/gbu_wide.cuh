// gbu_wide.cuh -- the partition loop of the single-buffer UTF-8 <-> UTF-16LE transcoders, with
// 32 input bytes per lane and 1 KiB warp regions.
//
// The loop has the shape of gbu_xcode.cuh's: a CTA of XT threads claims 16 KiB partitions from
// a ticket counter, counts the output of the NEXT partition (a read from HBM) and publishes
// that aggregate before it takes the CURRENT partition's output offset from the CTA-wide
// decoupled look-back, then converts the current partition (a re-read, normally from L2)
// through per-warp staging buffers and bulk stores.  What differs is the grain, chosen so that
// the fixed work of a region -- the lane scan, the neighbour shuffles, the staging bookkeeping,
// the proxy fence and the bulk store -- is paid once per KiB of input instead of once per 512
// bytes:
//   * a lane owns 32 consecutive bytes of its region, read by one 256-bit load; the words just
//     before and after them come from the adjacent lanes, or from the previous region's lane 31
//     and the next region's lane 0;
//   * warp w owns the w-th 4 KiB slice of the partition, four regions of 1 KiB;
//   * the count pass keeps, per region, every lane's exclusive output offset and the region's
//     total and codec flags, and per slice its total; a warp finds its regions' offsets from
//     the slice totals of the warps before it and a running sum over its own regions.
// The direction-specific parts are a wide codec:
//   struct Codec {
//     using Out = uint8_t or uint16_t;
//     static constexpr uint32_t WSTAGE;           // staged units per warp buffer
//     static constexpr uint32_t ASCII_MASK;       // nonzero in an input word: a unit >= 0x80
//     static constexpr uint32_t LANE_UNITS;       // units out of 32 bytes of ASCII input
//     static constexpr uint32_t WREGION_UNITS;    // units out of an all-ASCII region
//     static constexpr uint32_t WDIRECT_ALIGN;    // output alignment (units) of ascii_direct
//     __device__ static uint32_t wcount(const Params&, const uint32_t W[8], long long c, bool edge,
//                                       uint32_t& flags);
//     __device__ static Region wconvert(const Params&, const uint32_t W[8], uint32_t prev,
//                                       uint32_t next, long long c, bool edge, bool inside,
//                                       Out* st, uint32_t base, uint32_t x0, uint32_t rtot,
//                                       uint32_t rflags, unsigned long long& err_pos);
//     __device__ static bool wascii_region(uint32_t rtot, uint32_t rflags);
//     __device__ static void wascii_direct(Out* dst, const uint32_t W[8], uint32_t prev,
//                                          long long c, unsigned long long& err_pos);
//   };
// wconvert() stages the lane's units from staged index base + x0 on, in the warp buffer st (a
// shared-memory buffer); everything else is as in gbu_xcode.cuh.
#pragma once

#include <stdint.h>

#include "gbu_xcode.cuh"

namespace gbu {

constexpr uint32_t WLANE = 32;                        // input bytes per lane per region
constexpr uint32_t WREGION = 32 * WLANE;              // 1 KiB per warp region
constexpr int WROUNDS = (int)(SLICE_BYTES / WREGION); // regions per warp slice
constexpr int WREGIONS = WROUNDS * XWARPS;            // regions per partition
static_assert(SLICE_BYTES == WREGION * WROUNDS, "a slice is whole regions");
static_assert(WROUNDS % 2 == 0, "the count pass scans two regions at a time");

struct __align__(16) WideCounts {
  uint16_t lane_off[WREGIONS][32];  // each lane's exclusive offset inside its region
  uint32_t rinfo[WREGIONS];         // region total (bits 0-15) | codec flags << 16
  uint32_t slice[XWARPS];           // slice total (bits 0-30) | 1 << 31 for an all-ASCII slice inside the buffer
};

template <class Codec>
struct __align__(128) WSmem {
  typename Codec::Out staging[XWARPS][2][Codec::WSTAGE];
  WideCounts counts[2];
  LookbackSmem<XT> lb;
  unsigned long long red[XWARPS];
  uint32_t ticket;
  int is_last;
  unsigned long long known;  // snapshot of the error key (early exit)
};

// 32 bytes at p (32-byte aligned) with an L2 cache policy, read-only, no L1 allocation.
__device__ __forceinline__ void ldg32_hint(const uint8_t *p, uint64_t pol, uint32_t (&w)[8]) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
               : "l"(p), "l"(pol));
}

// The 32 bytes at virtual position c (a multiple of 32): one 256-bit load when the caller knows
// them to lie inside the data, else two bounds-checked 16-byte chunks (bytes outside
// [off0, vbytes) read as zero).
__device__ __forceinline__ void load32(const Params &p, long long c, bool inside, uint64_t pol, uint32_t (&w)[8]) {
  if (inside) {
    ldg32_hint(p.base + c, pol, w);
    return;
  }
  const uint4 a = load_chunk(p, c, false), b = load_chunk(p, c + 16, false);
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}

// Virtual position of lane `lane`'s 32 bytes in region r of warp w's slice of partition part.
__device__ __forceinline__ long long wchunk_pos(uint32_t part, int w, int r, int lane) {
  return (long long)part * PART_BYTES + (long long)w * SLICE_BYTES + (long long)r * WREGION +
         (long long)lane * WLANE;
}

// Counts partition `part` into pc (all threads; the caller puts a barrier after it).  INSIDE:
// the partition lies inside the buffer with a word to spare at each end.
template <class Codec, bool INSIDE>
__device__ __forceinline__ void wcount_partition(const Params &p, uint32_t part, WideCounts &pc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long s0 = wchunk_pos(part, warp, 0, 0);
  const long long lo = p.off0, hi = (long long)p.vbytes;
  const bool inside = INSIDE || (s0 >= lo && s0 + (long long)SLICE_BYTES <= hi);
  // the slice is read again by its conversion one partition later: keep it in L2
  const uint64_t keep = l2_policy_keep();
  uint32_t v[WROUNDS][8];
#pragma unroll
  for (int r = 0; r < WROUNDS; ++r) load32(p, s0 + (long long)r * WREGION + WLANE * lane, inside, keep, v[r]);
  bool slice_ascii = false;
  if (INSIDE) {
    uint32_t any = 0;
#pragma unroll
    for (int r = 0; r < WROUNDS; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) any |= v[r][k];
    slice_ascii = __all_sync(0xffffffffu, (any & Codec::ASCII_MASK) == 0);
  }
  uint32_t stot = 0;
  if (slice_ascii) {
    // every lane gives LANE_UNITS units: no scan needed
#pragma unroll
    for (int r = 0; r < WROUNDS; ++r) pc.lane_off[warp * WROUNDS + r][lane] = (uint16_t)(lane * Codec::LANE_UNITS);
    if (lane < WROUNDS) pc.rinfo[warp * WROUNDS + lane] = Codec::WREGION_UNITS;
    stot = WROUNDS * Codec::WREGION_UNITS;
  } else {
#pragma unroll
    for (int r = 0; r < WROUNDS; r += 2) {
      uint32_t a[2], f[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const long long c = s0 + (long long)(r + q) * WREGION + WLANE * lane;
        const bool edge = !inside && (c < lo || c + (long long)WLANE > hi);
        a[q] = Codec::wcount(p, v[r + q], c, edge, f[q]);
      }
      // two regions per scan: a region has at most 32 x 64 units
      const uint32_t x = a[0] | (a[1] << 16);
      uint32_t incl;
      const uint32_t x_first = __shfl_sync(0xffffffffu, x, 0);
      if (__all_sync(0xffffffffu, x == x_first)) {
        incl = x * (uint32_t)(lane + 1);  // equal counts (all-ASCII regions): no scan needed
      } else {
        incl = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
      }
      const uint32_t ex = incl - x;
      const int ri = warp * WROUNDS + r;
      pc.lane_off[ri][lane] = (uint16_t)(ex & 0xFFFFu);
      pc.lane_off[ri + 1][lane] = (uint16_t)(ex >> 16);
      const uint32_t fr0 = __reduce_or_sync(0xffffffffu, f[0]), fr1 = __reduce_or_sync(0xffffffffu, f[1]);
      if (lane == 31) {
        pc.rinfo[ri] = (incl & 0xFFFFu) | (fr0 << 16);
        pc.rinfo[ri + 1] = (incl >> 16) | (fr1 << 16);
      }
      stot += (incl & 0xFFFFu) + (incl >> 16);  // meaningful in lane 31
    }
  }
  if (lane == 31) pc.slice[warp] = stot | (slice_ascii ? 0x80000000u : 0u);
}

// Step 3 for partition `part` (all threads; each warp on its slice): transcodes the
// partition, whose output starts at unit S0, with the counts of its count pass in pc.
template <class Codec, bool INSIDE>
__device__ __forceinline__ void wconvert_partition(const Params &p, uint32_t part, const WideCounts &pc, uint64_t S0,
                                                   WSmem<Codec> &sm, uint32_t &use, unsigned long long &err_pos) {
  using Out = typename Codec::Out;
  constexpr uint32_t V = 16 / sizeof(Out);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long lo = p.off0, hi = (long long)p.vbytes;
  const long long s0 = wchunk_pos(part, warp, 0, 0);
  const bool slice_inside = INSIDE || (s0 - 4 >= lo && s0 + (long long)SLICE_BYTES + 4 <= hi);
  const uint32_t before = slice_inside ? ldg_word(p.base + s0 - 4) : load_word_checked(p, s0 - 4);
  const uint32_t after =
      slice_inside ? ldg_word(p.base + s0 + SLICE_BYTES) : load_word_checked(p, s0 + SLICE_BYTES);
  // the slice's first output unit inside the partition: the totals of the slices before it
  uint32_t sbase = 0;
#pragma unroll
  for (int w = 0; w < XWARPS - 1; ++w)
    if (w < warp) sbase += pc.slice[w] & 0x7FFFFFFFu;
  const uint32_t sinfo = pc.slice[warp];
  // the slice's output: its first unit counted from the 16-byte-rounded destination base, and
  // the units the destination holds from there on (clamped to 32 bits)
  const uint64_t S = S0 + sbase;
  const uint64_t D0 = p.dshift + S;
  const uint64_t room64 = p.cap > S ? p.cap - S : 0;
  const uint32_t room0 = room64 < 0xFFFFFFFFull ? (uint32_t)room64 : 0xFFFFFFFFu;
  Out *const dslice = reinterpret_cast<Out *>(p.dbase) + D0;
  const uint64_t last_use = l2_policy_last_use();
  const uint8_t *const src = p.base + s0 + WLANE * lane;  // the lane's 32 bytes of region 0
  if (INSIDE && (sinfo >> 31) && ((uint32_t)D0 & (Codec::WDIRECT_ALIGN - 1)) == 0 &&
      room0 >= (uint32_t)WROUNDS * Codec::WREGION_UNITS) {
    // an all-ASCII slice whose output is aligned and fits: every region goes straight to
    // global memory; only the word before the slice can hold a leading byte that wants
    // continuation bytes in it
    uint32_t w[WROUNDS][8];
#pragma unroll
    for (int r = 0; r < WROUNDS; ++r) ldg32_hint(src + r * WREGION, last_use, w[r]);
#pragma unroll
    for (int r = 0; r < WROUNDS; ++r)
      Codec::wascii_direct(dslice + r * Codec::WREGION_UNITS, w[r], r == 0 ? before : 0u,
                           s0 + (long long)r * WREGION + WLANE * lane, err_pos);
    return;
  }
  uint32_t prev_last = before;  // last word of the previous region (lane 31's), for lane 0
  uint32_t off = 0;             // the region's first unit inside the slice's output
#pragma unroll 1
  for (int r = 0; r < WROUNDS; ++r) {
    const long long c = s0 + (long long)r * WREGION + WLANE * lane;
    const bool edge = !INSIDE && (c < lo || c + (long long)WLANE > hi);
    // the lane's 32 bytes (other warps cover the L2 latency; a load kept a region ahead would
    // hold eight more registers through the conversion), and for lane 31 the word after the
    // region: the next region's first word, or the word after the slice
    uint32_t v[8];
    load32(p, c, slice_inside, last_use, v);
    uint32_t next_first = after;
    if (lane == 31 && r + 1 < WROUNDS)
      next_first = slice_inside ? ldg_word(p.base + c + WLANE) : load_word_checked(p, c + WLANE);
    uint32_t prev = __shfl_up_sync(0xffffffffu, v[7], 1);
    uint32_t next = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lane == 0) prev = prev_last;
    if (lane == 31) next = next_first;
    prev_last = __shfl_sync(0xffffffffu, v[7], 31);

    const int ri = warp * WROUNDS + r;
    const uint32_t info = pc.rinfo[ri];
    const uint32_t rtot = info & 0xFFFFu, rflags = info >> 16;
    const uint32_t dlo = (uint32_t)D0 + off;  // low bits of the region's destination unit
    const uint32_t room = room0 > off ? room0 - off : 0u;
    const long long rc = s0 + (long long)r * WREGION;
    const bool rin = INSIDE || (rc >= lo && rc + (long long)WREGION <= hi);  // uniform over the warp
    if (rin && Codec::wascii_region(rtot, rflags) && (dlo & (Codec::WDIRECT_ALIGN - 1)) == 0 &&
        Codec::WREGION_UNITS <= room) {
      Codec::wascii_direct(dslice + off, v, prev, c, err_pos);
      off += rtot;
      continue;
    }
    Out *st = sm.staging[warp][use & 1];
    ++use;
    const uint32_t x0 = pc.lane_off[ri][lane];
    const uint32_t h = dlo & (V - 1);
    bulk_wait_read_if<1>(lane == 0);  // the store of two regions ago has read this buffer
    __syncwarp();
    const Region g = Codec::wconvert(p, v, prev, next, c, edge, rin, st, h, x0, rtot, rflags, err_pos);
    fence_proxy_async_smem();
    __syncwarp();
    store_staged(dslice + off - h, st, h, room, g.skip, g.total, g.extra);
    off += rtot;
  }
}

template <class Codec>
__device__ __forceinline__ void wcount_part(const Params &p, uint32_t part, WideCounts &pc) {
  if (part_inside(p, part)) wcount_partition<Codec, true>(p, part, pc);
  else wcount_partition<Codec, false>(p, part, pc);
}

template <class Codec>
__device__ __forceinline__ void wconvert_part(const Params &p, uint32_t part, const WideCounts &pc, uint64_t S0,
                                              WSmem<Codec> &sm, uint32_t &use, unsigned long long &err_pos) {
  if (part_inside(p, part)) wconvert_partition<Codec, true>(p, part, pc, S0, sm, use, err_pos);
  else wconvert_partition<Codec, false>(p, part, pc, S0, sm, use, err_pos);
}

// The partition's total output (after the barrier that follows its count pass).
__device__ __forceinline__ uint32_t wpart_total(const WideCounts &pc) {
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < XWARPS; ++w) t += pc.slice[w] & 0x7FFFFFFFu;
  return t;
}

// The whole transcoder kernel body.  finalize(status, key, total) runs in thread 0 of the
// last CTA and writes the result.
template <class Codec, class Final>
__device__ __forceinline__ void wtranscode(const Params &p, WSmem<Codec> &sm, Final finalize) {
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t epoch = p.ws->epoch;
  unsigned long long err_pos = NO_ERROR;
  uint32_t use = 0;  // regions staged by this warp (picks the staging buffer)
  int cb = 0;        // which counts[] holds the current partition

  if (tid == 0) sm.ticket = atomicAdd(&p.ws->ticket, 1u);
  __syncthreads();
  uint32_t cur = sm.ticket;
  uint32_t cur_total = 0;
  if (cur < p.ntiles) {
    wcount_part<Codec>(p, cur, sm.counts[cb]);
    __syncthreads();
    cur_total = wpart_total(sm.counts[cb]);
    if (tid == 0) {
      publish_aggregate(p, cur, cur_total, epoch);
      atomicAdd(&p.ws->total, (unsigned long long)cur_total);
    }
  }
  // Early exit: output past the first error is unspecified, so a partition that starts past
  // a chunk some thread already flagged (the error key, published at once) is counted and
  // chained as usual -- later partitions still need its aggregate -- but not converted.  The
  // first error lies at most 31 bytes past the smallest flagged chunk, so it is always
  // converted up to its start.
  unsigned long long published = NO_ERROR;
  while (cur < p.ntiles) {
    // claim and count the next partition, so that its aggregate is out a partition early
    if (tid == 0) {
      sm.ticket = atomicAdd(&p.ws->ticket, 1u);
      sm.known = p.early_exit ? ld_relaxed_u64(reinterpret_cast<const uint64_t *>(&p.ws->errkey)) : NO_ERROR;
    }
    __syncthreads();
    const uint32_t nxt = sm.ticket;
    const unsigned long long known = sm.known;
    uint32_t nxt_total = 0;
    if (nxt < p.ntiles) {
      wcount_part<Codec>(p, nxt, sm.counts[cb ^ 1]);
      __syncthreads();
      nxt_total = wpart_total(sm.counts[cb ^ 1]);
      if (tid == 0) {
        publish_aggregate(p, nxt, nxt_total, epoch);
        atomicAdd(&p.ws->total, (unsigned long long)nxt_total);
      }
    }
    const uint64_t S0 = lookback_cta<XT>(p, cur, cur_total, epoch, sm.lb);

    if ((unsigned long long)cur * PART_BYTES <= known) {  // uniform over the CTA
      wconvert_part<Codec>(p, cur, sm.counts[cb], S0, sm, use, err_pos);
      if (p.early_exit && err_pos < published) {  // rare: this thread flagged a new error
        atomicMin(&p.ws->errkey, err_pos);
        published = err_pos;
      }
    }
    cur = nxt;
    cur_total = nxt_total;
    cb ^= 1;
    __syncthreads();  // counts[cb ^ 1] is rewritten by the next count pass
  }
  if (lane == 0) bulk_wait_all<0>();

  if (!fold_and_finish<XT>(p, err_pos, true, sm.red, &sm.is_last)) return;
  if (tid == 0) {
    WsHeader *ws = p.ws;
    const uint32_t status = *(volatile uint32_t *)&ws->status;
    const unsigned long long key = *(volatile unsigned long long *)&ws->errkey;
    const unsigned long long tot = *(volatile unsigned long long *)&ws->total;
    finalize(status, key, tot);
  }
  reset_workspace(p);
}

// ---- explicit shared-memory stores (32-bit shared addresses) ------------------------------

__device__ __forceinline__ void sts_u16(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}
__device__ __forceinline__ void sts_u8(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}
// Stores issued only where a flag bit is clear (or set), with the staging address advanced in
// the same predicate: one PTX block per position, so that ptxas emits a logic op that sets the
// predicate, the predicated store and the predicated add, and nothing else (an `if` around an
// asm statement would become a branch, and a condition passed in as a value would be tested
// again).  `sa` advances by `step` bytes where the store happens.
template <int STEP>
__device__ __forceinline__ void sts_u16_if_clear(uint32_t &sa, uint32_t v, uint32_t flags, uint32_t bit) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t.reg .b32 t;\n\tand.b32 t, %2, %3;\n\tsetp.eq.b32 q, t, 0;\n\t"
      "@q st.shared.u16 [%0], %1;\n\t@q add.u32 %0, %0, %4;\n\t}"
      : "+r"(sa)
      : "h"((unsigned short)v), "r"(flags), "r"(bit), "n"(STEP)
      : "memory");
}
template <int STEP>
__device__ __forceinline__ void sts_u16_if_set(uint32_t &sa, uint32_t v, uint32_t flags, uint32_t bit) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t.reg .b32 t;\n\tand.b32 t, %2, %3;\n\tsetp.ne.b32 q, t, 0;\n\t"
      "@q st.shared.u16 [%0], %1;\n\t@q add.u32 %0, %0, %4;\n\t}"
      : "+r"(sa)
      : "h"((unsigned short)v), "r"(flags), "r"(bit), "n"(STEP)
      : "memory");
}
// A byte at a + OFF where (flags & bit) != 0 (the address is not advanced).
template <int OFF>
__device__ __forceinline__ void sts_u8_if_set(uint32_t a, uint32_t v, uint32_t flags, uint32_t bit) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t.reg .b32 t;\n\tand.b32 t, %2, %3;\n\tsetp.ne.b32 q, t, 0;\n\t"
      "@q st.shared.u8 [%0+%4], %1;\n\t}" ::"r"(a),
      "h"((unsigned short)v), "r"(flags), "r"(bit), "n"(OFF)
      : "memory");
}
}  // namespace gbu
