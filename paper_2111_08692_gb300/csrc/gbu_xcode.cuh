// gbu_xcode.cuh -- the partition loop shared by both transcoders.
//
// A CTA of XT threads (XWARPS warps) claims 16 KB partitions from a ticket counter.  Warp w
// owns the partition's w-th 4 KB slice and walks it in eight 512-byte regions (one 16-byte
// chunk per lane per region), so a chunk's neighbouring words come from the adjacent lane,
// or from the previous / next region's registers.  For every partition the CTA
//   1. counts the output units of each region of the NEXT partition (a read from HBM), turns
//      the region counts (32 per partition) into region offsets inside it, and publishes the
//      partition total as its aggregate -- a whole partition before any look-back needs it;
//   2. gets the CURRENT partition's output offset from a CTA-wide decoupled look-back;
//   3. transcodes the current partition (a re-read, normally from L2): every warp handles its
//      regions on its own -- a warp-level scan orders the lanes' output, the region's output
//      is staged in the warp's shared-memory buffer and leaves with one bulk store (whole
//      16-byte chunks) plus plain stores for the ragged ends.  No CTA-wide barrier is needed
//      inside the region loop.
// The direction-specific parts are a Codec class:
//   struct Codec {
//     using Out = uint8_t or uint16_t;                 // output code unit
//     static constexpr uint32_t STAGE;                 // staged units per warp buffer
//     static constexpr uint32_t REGION_UNITS, DIRECT_ALIGN;  // all-ASCII region output
//     __device__ static uint32_t count(const Params&, uint4 v, long long c, bool edge,
//                                      uint32_t& flags);
//     __device__ static Region convert(const Params&, uint4 v, uint32_t prev, uint32_t next,
//                                      long long c, bool edge, bool inside, Out* st,
//                                      uint32_t base, uint32_t x0, uint32_t rtot, uint32_t rflags,
//                                      unsigned long long& err_pos);
//     __device__ static bool ascii_region(uint32_t rtot, uint32_t rflags);
//     __device__ static void ascii_direct(Out* dst, uint4 v, uint32_t prev, long long c,
//                                         unsigned long long& err_pos);
//   };
// count() returns the units one chunk contributes to its region (the total that converting
// the region stages) and sets codec-defined flag bits (the region's flags are the OR over its
// lanes).  An all-ASCII region inside the buffer whose output starts on a 16-byte boundary
// (DIRECT_ALIGN units) skips the staging: ascii_direct() stores each lane's units straight
// to global memory.  The count pass keeps, for every region, each lane's exclusive offset x0, the
// region total rtot and the flag, so convert() neither recounts nor rescans: it stages the
// lane's units at base + x0 and returns the region's unit count and the units it writes past
// its end or leaves to its predecessor at its start.  `inside` (uniform over the warp) says
// that no chunk of the region touches a buffer end.
#pragma once

#include <stdint.h>

#include "gbu_device.cuh"

namespace gbu {

constexpr uint32_t SLICE_BYTES = PART_BYTES / XWARPS;  // 4 KB per warp
constexpr uint32_t REGION_BYTES = 32 * CHUNK;          // 512 bytes per warp per round
static_assert(SLICE_BYTES == REGION_BYTES * PART_ROUNDS, "a slice is PART_ROUNDS regions");

struct Region {
  uint32_t total;  // units to store for the region (clamped to the staging buffer)
  uint32_t skip;   // leading units written by the previous region (not to be stored here)
  uint32_t extra;  // units this region writes past its end (a pair cut by the region end)
  uint32_t units;  // units counted for the region (unclamped: the region's output length)
};

constexpr int PART_REGIONS = PART_ROUNDS * XWARPS;  // 32 regions per partition

struct __align__(16) PartCounts {
  uint32_t off[PART_REGIONS];           // region offsets inside the partition, in byte order
  uint16_t lane_off[PART_REGIONS][32];  // each lane's exclusive offset inside its region
  uint16_t rtot[PART_REGIONS];          // region totals
  uint8_t flags[PART_REGIONS];          // OR of the codec flags of the region's lanes
  uint32_t total;
  uint32_t all_ascii;                   // the partition lies inside the buffer and is all ASCII
};

template <class Codec>
struct __align__(128) XSmem {
  typename Codec::Out staging[XWARPS][2][Codec::STAGE];
  PartCounts counts[2];
  LookbackSmem<XT> lb;
  unsigned long long red[XWARPS];
  uint32_t ticket;
  int is_last;
  unsigned long long known;  // snapshot of the error key (single-buffer early exit)
  Params prm[2];   // several-string launches: the string of counts[0] / counts[1]
  uint32_t sid[2];
};

// Virtual position of lane `lane`'s chunk in region r of warp w's slice of partition part.
__device__ __forceinline__ long long chunk_pos(uint32_t part, int w, int r, int lane) {
  return (long long)part * PART_BYTES + (long long)w * SLICE_BYTES + (long long)r * REGION_BYTES +
         (long long)lane * CHUNK;
}

// Counts partition `part` into pc (all threads).  Warp w scans the lane counts of each of its
// regions (two regions packed per register: a region has at most 32 x 48 units), keeping
// every lane's exclusive offset; then warp 0 turns the 128 region totals into offsets.
// INSIDE: the partition lies inside the buffer with a word to spare at each end
// (part_inside), so that no chunk needs a bounds test.
template <class Codec, bool INSIDE>
__device__ __forceinline__ void count_partition(const Params &p, uint32_t part, PartCounts &pc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long p0 = (long long)part * PART_BYTES;
  const long long lo = p.off0, hi = (long long)p.vbytes;
  const bool inside = INSIDE || (p0 >= lo && p0 + (long long)PART_BYTES <= hi);
  // the partition is read again by its conversion one partition later: keep it in L2
  const uint64_t keep = l2_policy_keep();
  uint4 v[PART_ROUNDS];
#pragma unroll
  for (int r = 0; r < PART_ROUNDS; ++r)
    v[r] = load_chunk_hint(p, chunk_pos(part, warp, r, lane), inside, keep);
  bool slice_ascii = false;
  if (INSIDE) {
    uint32_t any = 0;
#pragma unroll
    for (int r = 0; r < PART_ROUNDS; ++r) any |= v[r].x | v[r].y | v[r].z | v[r].w;
    slice_ascii = __all_sync(0xffffffffu, (any & Codec::ASCII_MASK) == 0);
  }
  if (slice_ascii) {
    // an all-ASCII slice: every chunk gives CHUNK_UNITS units, no scan needed
#pragma unroll
    for (int r = 0; r < PART_ROUNDS; ++r)
      pc.lane_off[warp * PART_ROUNDS + r][lane] = (uint16_t)(lane * Codec::CHUNK_UNITS);
    if (lane < PART_ROUNDS) {
      pc.off[warp * PART_ROUNDS + lane] = Codec::REGION_UNITS;
      pc.rtot[warp * PART_ROUNDS + lane] = (uint16_t)Codec::REGION_UNITS;
      pc.flags[warp * PART_ROUNDS + lane] = 0;
    }
  } else {
#pragma unroll
    for (int r = 0; r < PART_ROUNDS; r += 2) {
      uint32_t a[2], f[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const long long c = chunk_pos(part, warp, r + q, lane);
        const bool edge = !inside && (c < lo || c + 16 > hi);
        a[q] = Codec::count(p, v[r + q], c, edge, f[q]);
      }
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
      const int ri = warp * PART_ROUNDS + r;
      pc.lane_off[ri][lane] = (uint16_t)(ex & 0xFFFFu);
      pc.lane_off[ri + 1][lane] = (uint16_t)(ex >> 16);
      const uint32_t fr0 = __reduce_or_sync(0xffffffffu, f[0]), fr1 = __reduce_or_sync(0xffffffffu, f[1]);
      if (lane == 31) {
        pc.off[ri] = incl & 0xFFFFu;
        pc.off[ri + 1] = incl >> 16;
        pc.rtot[ri] = (uint16_t)(incl & 0xFFFFu);
        pc.rtot[ri + 1] = (uint16_t)(incl >> 16);
        pc.flags[ri] = (uint8_t)fr0;
        pc.flags[ri + 1] = (uint8_t)fr1;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    // consecutive values per lane (one per lane, and none past the last region, when the
    // partition has at most 32 regions)
    constexpr int PER = PART_REGIONS >= 32 ? PART_REGIONS / 32 : 1;
    static_assert(PART_REGIONS < 32 || PART_REGIONS % 32 == 0, "regions per partition");
    uint32_t vals[PER], s = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      vals[i] = lane * PER + i < PART_REGIONS ? pc.off[lane * PER + i] : 0u;
      s += vals[i];
    }
    uint32_t incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    uint32_t run = incl - s;
    bool ascii = INSIDE;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int ri = lane * PER + i;
      if (ri < PART_REGIONS) {
        pc.off[ri] = run;
        ascii = ascii && Codec::ascii_region(vals[i], pc.flags[ri]);
      }
      run += vals[i];
    }
    ascii = __all_sync(0xffffffffu, ascii);
    if (lane == 31) {
      pc.total = incl;
      pc.all_ascii = ascii ? 1u : 0u;
    }
  }
  __syncthreads();
}

// Writes a region's staged units [skip, cnt + extra) (one warp).  gdst is the 16-byte-aligned
// destination of staged index 0 and h the staged index of the region's first unit, so that
// staged chunk boundaries fall on 16-byte destination boundaries; units at or past `room`
// (counted from the region's first unit) are not written.  Lane 0 issues the bulk store of
// the whole 16-byte chunks and commits it as one bulk group; the lanes write the ragged
// ends.  Every lane that wrote the staging buffer must have run fence_proxy_async_smem()
// before the __syncwarp preceding this call.
template <typename U>
__device__ __forceinline__ void store_staged(U *gdst, const U *staging, uint32_t h, uint32_t room, uint32_t skip,
                                             uint32_t cnt, uint32_t extra) {
  constexpr uint32_t V = 16 / sizeof(U);
  const uint32_t lane = threadIdx.x & 31;
  uint32_t lim = cnt + extra;
  if (room < lim) lim = room;
  const uint32_t beg = h + (skip < lim ? skip : lim);
  const uint32_t end = h + lim;
  const uint32_t head_end = (beg + V - 1) & ~(V - 1);  // first 16-byte boundary at or after beg
  const uint32_t tail_beg = end & ~(V - 1);            // last 16-byte boundary at or before end
  if (head_end < tail_beg) {
    bulk_store_if(lane == 0, gdst + head_end, staging + head_end, (tail_beg - head_end) * 16u / V);
    // the ragged ends hold fewer than V <= 16 units each
    if (beg + lane < head_end) gdst[beg + lane] = staging[beg + lane];
    if (tail_beg + lane < end) gdst[tail_beg + lane] = staging[tail_beg + lane];
  } else if (beg + lane < end) {  // fewer than 2V <= 32 units
    gdst[beg + lane] = staging[beg + lane];
  }
  bulk_commit_if(lane == 0);
}

// store_staged for a region whose output starts at global unit S of the buffer p describes.
template <typename U>
__device__ __forceinline__ void store_region(const Params &p, const U *staging, uint64_t S, uint32_t skip,
                                             uint32_t cnt, uint32_t extra) {
  constexpr uint32_t V = 16 / sizeof(U);
  const uint32_t h = (uint32_t)(p.dshift + S) & (V - 1);
  const uint64_t room = p.cap > S ? p.cap - S : 0;
  U *gdst = reinterpret_cast<U *>(p.dbase) + ((p.dshift + S) - h);
  store_staged(gdst, staging, h, room < 0xFFFFFFFFull ? (uint32_t)room : 0xFFFFFFFFu, skip, cnt, extra);
}

// Warp-level exclusive scan of per-lane counts; *total receives the warp sum.
__device__ __forceinline__ uint32_t warp_exclusive_scan(uint32_t x, uint32_t *total) {
  const int lane = threadIdx.x & 31;
  uint32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  *total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - x;
}

// Converts one region without a count pass (one warp): counts and scans the lanes first.
template <class Codec>
__device__ __forceinline__ Region convert_counted(const Params &p, uint4 v, uint32_t prev, uint32_t next,
                                                  long long c, bool edge, bool inside, typename Codec::Out *st,
                                                  uint32_t base, unsigned long long &err_pos) {
  uint32_t f;
  const uint32_t cnt = Codec::count(p, v, c, edge, f);
  uint32_t tot;
  const uint32_t x0 = warp_exclusive_scan(cnt, &tot);
  const uint32_t rf = __reduce_or_sync(0xffffffffu, f);
  return Codec::convert(p, v, prev, next, c, edge, inside, st, base, x0, tot, rf, err_pos);
}

// The whole transcoder kernel body.  finalize(status, key, total) runs in thread 0 of the
// last CTA and writes the result.
// Step 3 for partition `part` of the buffer that p describes (all threads; each warp on its
// slice): transcodes the partition, whose output starts at unit S0, with the region offsets,
// lane offsets and flags of its count pass in pc.
template <class Codec, bool INSIDE>
__device__ __forceinline__ void convert_partition(const Params &p, uint32_t part, const PartCounts &pc, uint64_t S0,
                                                  XSmem<Codec> &sm, uint32_t &use, unsigned long long &err_pos) {
  using Out = typename Codec::Out;
  constexpr uint32_t V = 16 / sizeof(Out);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long lo = p.off0, hi = (long long)p.vbytes;
  // this warp's slice: the words just before and after it, and its first chunk
  const long long s0 = chunk_pos(part, warp, 0, 0);
  const bool slice_inside = INSIDE || (s0 - 4 >= lo && s0 + (long long)SLICE_BYTES + 4 <= hi);
  const uint32_t before = slice_inside ? ldg_word(p.base + s0 - 4) : load_word_checked(p, s0 - 4);
  const uint32_t after =
      slice_inside ? ldg_word(p.base + s0 + SLICE_BYTES) : load_word_checked(p, s0 + SLICE_BYTES);
  const uint64_t last_use = l2_policy_last_use();
  const uint8_t *const src = p.base + s0 + CHUNK * lane;  // the lane's chunk of the first region
  // the partition's output: its first unit counted from the 16-byte-rounded destination base,
  // and the units the destination holds from there on (clamped to 32 bits)
  const uint64_t D0 = p.dshift + S0;
  const uint64_t room64 = p.cap > S0 ? p.cap - S0 : 0;
  const uint32_t room0 = room64 < 0xFFFFFFFFull ? (uint32_t)room64 : 0xFFFFFFFFu;
  Out *const dpart = reinterpret_cast<Out *>(p.dbase) + D0;
  if (INSIDE && pc.all_ascii && ((uint32_t)D0 & (Codec::DIRECT_ALIGN - 1)) == 0 &&
      room0 >= (uint32_t)PART_REGIONS * Codec::REGION_UNITS) {
    // an all-ASCII partition whose output is aligned and fits: every region goes straight
    // to global memory (no offsets, shuffles or staging); only the word before the slice
    // can hold a leading byte that wants continuation bytes in it
    uint4 w[PART_ROUNDS];
#pragma unroll
    for (int r = 0; r < PART_ROUNDS; ++r) w[r] = ldg_stream_hint(src + r * REGION_BYTES, last_use);
#pragma unroll
    for (int r = 0; r < PART_ROUNDS; ++r)
      Codec::ascii_direct(dpart + (warp * PART_ROUNDS + r) * Codec::REGION_UNITS, w[r], r == 0 ? before : 0u,
                          s0 + (long long)r * REGION_BYTES + CHUNK * lane, err_pos);
    return;
  }
  // two regions in flight ahead of the one being converted (the convert pass reads from L2)
  uint4 v_next = load_chunk_hint(p, s0 + CHUNK * lane, slice_inside, last_use);
  uint4 v_next2 = load_chunk_hint(p, s0 + REGION_BYTES + CHUNK * lane, slice_inside, last_use);
  uint32_t prev_last = before;  // last word of the previous region (lane 31's), for lane 0
#pragma unroll 1
  for (int r = 0; r < PART_ROUNDS; ++r) {
    const long long c = s0 + (long long)r * REGION_BYTES + CHUNK * lane;
    const bool edge = !INSIDE && (c < lo || c + 16 > hi);
    const uint4 v = v_next;
    v_next = v_next2;
    if (r + 2 < PART_ROUNDS)
      v_next2 = INSIDE ? ldg_stream_hint(src + (r + 2) * REGION_BYTES, last_use)
                       : load_chunk_hint(p, c + 2 * REGION_BYTES, slice_inside, last_use);
    uint32_t prev = __shfl_up_sync(0xffffffffu, v.w, 1);
    uint32_t next = __shfl_down_sync(0xffffffffu, v.x, 1);
    const uint32_t next_first = __shfl_sync(0xffffffffu, v_next.x, 0);  // next region's first word
    if (lane == 0) prev = prev_last;
    if (lane == 31) next = r + 1 < PART_ROUNDS ? next_first : after;
    prev_last = __shfl_sync(0xffffffffu, v.w, 31);

    const int ri = warp * PART_ROUNDS + r;
    const uint32_t off = pc.off[ri];  // the region's first unit inside the partition's output
    const uint32_t rtot = pc.rtot[ri];
    const uint32_t rflags = pc.flags[ri];
    const uint32_t dlo = (uint32_t)D0 + off;  // low bits of its destination unit
    const uint32_t room = room0 > off ? room0 - off : 0u;
    const long long rc = s0 + (long long)r * REGION_BYTES;
    const bool rin = INSIDE || (rc >= lo && rc + (long long)REGION_BYTES <= hi);  // uniform over the warp
    if (rin && Codec::ascii_region(rtot, rflags) && (dlo & (Codec::DIRECT_ALIGN - 1)) == 0 &&
        Codec::REGION_UNITS <= room) {
      Codec::ascii_direct(dpart + off, v, prev, c, err_pos);
      continue;
    }
    Out *st = sm.staging[warp][use & 1];
    ++use;
    const uint32_t x0 = pc.lane_off[ri][lane];
    const uint32_t h = dlo & (V - 1);
    bulk_wait_read_if<1>(lane == 0);  // the store of two regions ago has read this buffer
    __syncwarp();
    const Region g = Codec::convert(p, v, prev, next, c, edge, rin, st, h, x0, rtot, rflags, err_pos);
    fence_proxy_async_smem();
    __syncwarp();
    store_staged(dpart + off - h, st, h, room, g.skip, g.total, g.extra);
  }
}

// Whether partition `part` lies inside the buffer with a word to spare at each end (then no
// chunk of it, nor a neighbouring word, needs a bounds test).
__device__ __forceinline__ bool part_inside(const Params &p, uint32_t part) {
  const long long p0 = (long long)part * PART_BYTES;
  return p0 - 4 >= (long long)p.off0 && p0 + (long long)PART_BYTES + 4 <= (long long)p.vbytes;
}

template <class Codec>
__device__ __forceinline__ void count_part(const Params &p, uint32_t part, PartCounts &pc) {
  if (part_inside(p, part)) count_partition<Codec, true>(p, part, pc);
  else count_partition<Codec, false>(p, part, pc);
}

template <class Codec>
__device__ __forceinline__ void convert_part(const Params &p, uint32_t part, const PartCounts &pc, uint64_t S0,
                                             XSmem<Codec> &sm, uint32_t &use, unsigned long long &err_pos) {
  if (part_inside(p, part)) convert_partition<Codec, true>(p, part, pc, S0, sm, use, err_pos);
  else convert_partition<Codec, false>(p, part, pc, S0, sm, use, err_pos);
}

template <class Codec, class Final>
__device__ __forceinline__ void transcode(const Params &p, XSmem<Codec> &sm, Final finalize) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t epoch = p.ws->epoch;
  const long long lo = p.off0, hi = (long long)p.vbytes;
  unsigned long long err_pos = NO_ERROR;
  uint32_t use = 0;  // regions staged by this warp (picks the staging buffer)
  int cb = 0;        // which counts[] holds the current partition

  if (tid == 0) sm.ticket = atomicAdd(&p.ws->ticket, 1u);
  __syncthreads();
  uint32_t cur = sm.ticket;
  if (cur < p.ntiles) {
    count_part<Codec>(p, cur, sm.counts[cb]);
    if (tid == 0) {
      publish_aggregate(p, cur, sm.counts[cb].total, epoch);
      atomicAdd(&p.ws->total, (unsigned long long)sm.counts[cb].total);
    }
  }
  // Early exit: output past the first error is unspecified, so a partition that starts past
  // a chunk some thread already flagged (the error key, published at once) is counted and
  // chained as usual -- later partitions still need its aggregate -- but not converted.  The
  // first error lies at most 15 bytes past the smallest flagged chunk, so it is always
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
    if (nxt < p.ntiles) {
      count_part<Codec>(p, nxt, sm.counts[cb ^ 1]);
      if (tid == 0) {
        publish_aggregate(p, nxt, sm.counts[cb ^ 1].total, epoch);
        atomicAdd(&p.ws->total, (unsigned long long)sm.counts[cb ^ 1].total);
      }
    }
    const uint64_t S0 = lookback_cta<XT>(p, cur, sm.counts[cb].total, epoch, sm.lb);

    if ((unsigned long long)cur * PART_BYTES <= known) {  // uniform over the CTA
      convert_part<Codec>(p, cur, sm.counts[cb], S0, sm, use, err_pos);
      if (p.early_exit && err_pos < published) {  // rare: this thread flagged a new error
        atomicMin(&p.ws->errkey, err_pos);
        published = err_pos;
      }
    }
    cur = nxt;
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

// ---- several strings in one launch -----------------------------------------------------------
//
// Long strings (the serving loop's large requests) are transcoded together: their partitions
// are numbered one after the other (string s owns partitions pstart[s] .. pstart[s+1]-1),
// CTAs claim them from one ticket counter, and each string has its own look-back chain (its
// Params point at its own run of states, so its first partition publishes an inclusive
// prefix at once).  A thread that flags an error adds it to its string's minimum; the CTA
// that finishes a string's last outstanding partition writes that string's result.

// The string that owns launch partition t: the last s with pstart[s] <= t.
__device__ __forceinline__ uint32_t seg_of(const SegParams &q, uint32_t t) {
  uint32_t lo = 0, hi = q.B;  // pstart[lo] <= t < pstart[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (q.pstart[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The single-buffer parameters of string s.
template <class Codec>
__device__ __forceinline__ void seg_params(const SegParams &q, uint32_t s, Params &p) {
  constexpr uint32_t OUT_UNIT = sizeof(typename Codec::Out);
  constexpr uint32_t IN_UNIT = OUT_UNIT == 2 ? 1u : 2u;
  const StringDesc d = q.desc[s];
  const uintptr_t a = (uintptr_t)d.src, da = (uintptr_t)d.dst;
  p.base = (const uint8_t *)(a & ~(uintptr_t)15);
  p.off0 = (uint32_t)(a & 15);
  p.n = d.n;
  p.vbytes = p.off0 + d.n * IN_UNIT;
  p.dbase = (uint8_t *)(da & ~(uintptr_t)15);
  p.dshift = (uint32_t)((da & 15) / OUT_UNIT);
  p.cap = d.cap;
  p.ntiles = q.pstart[s + 1] - q.pstart[s];
  p.result = q.results + s;
  p.len_out = nullptr;
  p.ws = q.ws;
  p.states = q.states + q.pstart[s];
  p.max_states = q.max_states;
  p.wait_limit = q.wait_limit;
  p.skip_tile = -1;
  p.early_exit = 0;
}

// The kernel body.  finalize(p, st, s) runs in one thread once string s is finished (p: its
// parameters, st: its error minimum and output length) and writes its result.
template <class Codec, class Final>
__device__ __forceinline__ void transcode_segments(const SegParams &q, XSmem<Codec> &sm, Final finalize) {
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t epoch = q.ws->epoch;
  unsigned long long err_pos = NO_ERROR;
  uint32_t use = 0;  // regions staged by this warp (picks the staging buffer)
  int cb = 0;        // which counts[] / prm[] hold the current partition

  if (tid == 0) {
    const uint32_t t = atomicAdd(&q.ws->ticket, 1u);
    sm.ticket = t;
    if (t < q.ntiles) {
      sm.sid[0] = seg_of(q, t);
      seg_params<Codec>(q, sm.sid[0], sm.prm[0]);
    }
  }
  __syncthreads();
  uint32_t cur = sm.ticket;
  if (cur < q.ntiles) {
    const uint32_t lc = cur - q.pstart[sm.sid[0]];
    count_part<Codec>(sm.prm[0], lc, sm.counts[0]);
    if (tid == 0) publish_aggregate(sm.prm[0], lc, sm.counts[0].total, epoch);
  }
  while (cur < q.ntiles) {
    // claim and count the next partition, so that its aggregate is out a partition early
    if (tid == 0) {
      const uint32_t t = atomicAdd(&q.ws->ticket, 1u);
      sm.ticket = t;
      if (t < q.ntiles) {
        sm.sid[cb ^ 1] = seg_of(q, t);
        seg_params<Codec>(q, sm.sid[cb ^ 1], sm.prm[cb ^ 1]);
      }
    }
    __syncthreads();
    const uint32_t nxt = sm.ticket;
    if (nxt < q.ntiles) {
      const uint32_t ln = nxt - q.pstart[sm.sid[cb ^ 1]];
      count_part<Codec>(sm.prm[cb ^ 1], ln, sm.counts[cb ^ 1]);
      if (tid == 0) publish_aggregate(sm.prm[cb ^ 1], ln, sm.counts[cb ^ 1].total, epoch);
    }
    const Params &p = sm.prm[cb];
    const uint32_t s = sm.sid[cb];
    const uint32_t lc = cur - q.pstart[s];
    const uint64_t S0 = lookback_cta<XT>(p, lc, sm.counts[cb].total, epoch, sm.lb);
    convert_part<Codec>(p, lc, sm.counts[cb], S0, sm, use, err_pos);
    if (err_pos != NO_ERROR) {  // rare: this thread saw an error in the partition
      atomicMin(&q.seg[s].errkey, err_pos);
      __threadfence();
      err_pos = NO_ERROR;
    }
    __syncthreads();  // every warp is done with the partition
    if (tid == 0) {
      if (lc + 1 == p.ntiles) *(volatile unsigned long long *)&q.seg[s].total = S0 + sm.counts[cb].total;
      __threadfence();
      const uint32_t prev = atomicAdd(&q.seg[s].done, 1u);
      if (prev + 1 == p.ntiles) {
        __threadfence();
        finalize(p, q.seg[s], s);
        q.seg[s].errkey = NO_ERROR;  // ready for the next launch
        q.seg[s].total = 0;
        q.seg[s].done = 0;
      }
    }
    cur = nxt;
    cb ^= 1;
    __syncthreads();  // counts[cb ^ 1] and prm[cb ^ 1] are rewritten by the next claim
  }
  if (lane == 0) bulk_wait_all<0>();

  // the last CTA to finish resets the launch's workspace
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&q.ws->done, 1u);
    sm.is_last = prev == gridDim.x - 1;
    if (sm.is_last) __threadfence();
  }
  __syncthreads();
  if (sm.is_last) {
    Params r;
    r.ws = q.ws;
    r.states = q.states;
    r.max_states = q.max_states;
    reset_workspace(r);
  }
}

}  // namespace gbu
