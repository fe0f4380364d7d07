// gbu_device.cuh -- device-side building blocks shared by the UTF-8 and UTF-16 kernels.
//
// Every kernel is a persistent grid of warp-specialised CTAs that walk fixed-size tiles:
//   * one producer warp per CTA claims tiles (a global ticket counter for transcoders,
//     round-robin for read-only kernels), copies each tile plus a 16-byte halo on both sides
//     into a shared-memory ring with the bulk-copy engine (cp.async.bulk + mbarrier), and
//     hands the stage to the consumers through a "ready" mbarrier;
//   * for transcoders the producer also counts the tile's output units as soon as it lands,
//     publishes that aggregate, and runs the single-pass decoupled look-back (Merrill &
//     Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016) that turns
//     it into the tile's output offset -- ahead of the consumers, so its latency is hidden;
//   * eight consumer warps decode their 16-byte chunks, stage the output in shared memory
//     and write it back with cp.async.bulk stores for the 16-byte-aligned middle and plain
//     stores for the ragged ends, then release the stage through an "empty" mbarrier;
//   * the first error is a 64-bit atomicMin over input positions; the last CTA to finish
//     (a completion counter) turns it into the exact offset and kind and writes the result.
// Every spin wait is bounded; when a bound is hit the kernel records GBU_TIMEOUT and keeps
// going, so a launch always terminates.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbutf.h"

namespace gbu {

constexpr int NCW = 8;                        // consumer warps per CTA
constexpr int NC = NCW * 32;                  // consumer threads
constexpr int NTHREADS = NC + 32;             // + one producer warp
constexpr int PRODUCER_WARP = NCW;
constexpr int HALO = 16;                      // halo bytes on each side of a tile
constexpr uint32_t CHUNK = 16;                // input bytes per consumer thread per tile
constexpr uint32_t TILE_BYTES = NC * CHUNK;   // 4096 input bytes per tile
constexpr uint32_t WIN_BYTES = TILE_BYTES + 2 * HALO;

// Scan state word: [63:62] flag, [61:44] epoch, [43:0] value.
constexpr uint64_t ST_FLAG_AGG = 1ull << 62;
constexpr uint64_t ST_FLAG_INC = 2ull << 62;
constexpr int ST_EPOCH_SHIFT = 44;
constexpr uint32_t ST_EPOCH_MASK = (1u << 18) - 1;
constexpr uint64_t ST_VALUE_MASK = (1ull << 44) - 1;

constexpr unsigned long long NO_ERROR = ~0ull;

// Polling rounds before a wait on the bulk-copy engine or on another warp of the CTA gives up
// (each try_wait round also suspends for a hardware-chosen time, so this is seconds).
constexpr uint32_t LOCAL_WAIT_ROUNDS = 1u << 24;

// Workspace header, one per context (device memory, initialised at creation).  The last CTA
// of a launch resets ticket/done/errkey/total/status and advances the epoch, so consecutive
// launches on one stream need no memset.
struct WsHeader {
  uint32_t epoch;                 // tags scan states of the current launch (1 .. 2^18-1)
  uint32_t ticket;                // next tile to claim (transcoders)
  uint32_t done;                  // CTAs that have finished
  uint32_t status;                // sticky: 1 = a wait gave up (GBU_TIMEOUT)
  unsigned long long errkey;      // smallest input position of a thread chunk with an error
  unsigned long long total;       // sum of tile aggregates (output length)
  uint32_t pad[24];
};
static_assert(sizeof(WsHeader) == 128, "header is one 128-byte line");

struct Params {
  const uint8_t *base;     // source rounded down to 16 bytes
  uint64_t vbytes;         // off0 + source bytes: virtual positions [off0, vbytes) are data
  uint32_t off0;           // source address - base (bytes)
  uint32_t ntiles;
  uint64_t n;              // source length in code units
  uint8_t *dbase;          // destination rounded down to 16 bytes (transcoders)
  uint32_t dshift;         // (destination - dbase) in output code units
  uint64_t cap;            // destination capacity in output code units
  gbu_result *result;      // where the last CTA writes the result (validate/convert)
  uint64_t *len_out;       // where the last CTA writes the length (length functions)
  WsHeader *ws;
  uint64_t *states;        // one scan state per tile
  uint32_t max_states;     // entries in states[]
  uint32_t wait_limit;     // polling rounds before a look-back wait gives up
  long long skip_tile;     // test hook: this tile never publishes (-1: off)
};

// ---- small PTX wrappers -----------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// global -> shared bulk copy; completes `bytes` of transaction count on `bar`
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// shared -> global bulk copy in the current bulk group
__device__ __forceinline__ void bulk_store(void *dst_gmem, const void *src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(smem_addr(src_smem)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// wait until at most N committed bulk groups still read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// order this thread's generic-proxy shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// barrier among the NC consumer threads only (the producer warp does not take part)
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// PRMT with the full 4-bit selector nibbles (bit 3 = replicate the sign bit of the selected
// byte); __byte_perm only honours the low three bits of each nibble.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o < v ? o : v;
  }
  return v;
}

// Records a failed wait: the launch reports GBU_TIMEOUT.
__device__ __forceinline__ void note_timeout(WsHeader *ws) { atomicOr(&ws->status, 1u); }

// Bounded wait on an mbarrier phase.  Returns false (and records a timeout) if it gave up.
__device__ __forceinline__ bool mbar_wait(const Params &p, uint64_t *bar, uint32_t parity) {
  uint32_t rounds = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++rounds >= LOCAL_WAIT_ROUNDS) {
      note_timeout(p.ws);
      return false;
    }
  }
  return true;
}

// ---- shared memory common to every kernel -------------------------------------------------

struct TileInfo {
  uint32_t tile;             // tile of this stage use (>= ntiles: no more tiles)
  uint32_t total;            // output units of the tile (transcoders)
  unsigned long long excl;   // output units before the tile (transcoders)
};

template <int NS>
struct __align__(16) PipeSmem {
  uint64_t full[NS];    // bulk copy landed
  uint64_t ready[NS];   // producer done with the stage: consumers may read it
  uint64_t empty[NS];   // consumers done with the stage: producer may refill it
  TileInfo info[NS];
  uint32_t warp_sums[NCW + 2];
  unsigned long long red[NTHREADS / 32];
  int is_last;
};

template <int NS>
__device__ __forceinline__ void pipe_init(PipeSmem<NS> &ps, uint32_t empty_count) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&ps.full[s], 1);
      mbar_init(&ps.ready[s], 1);
      mbar_init(&ps.empty[s], empty_count);
    }
    fence_mbar_init();
  }
  __syncthreads();
}

// Exclusive scan over the NC consumer threads.  Returns this thread's exclusive prefix and
// the consumer-wide total.  Two consumer barriers.
__device__ __forceinline__ uint32_t consumer_exclusive_scan(uint32_t x, uint32_t *warp_sums,
                                                            uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  consumer_sync();
  if (warp == 0) {
    const uint32_t s = lane < NCW ? warp_sums[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int d = 1; d < NCW; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, si, d);
      if (lane >= d) si += y;
    }
    if (lane < NCW) warp_sums[lane] = si - s;
    if (lane == NCW - 1) warp_sums[NCW] = si;
  }
  consumer_sync();
  *total = warp_sums[NCW];
  return warp_sums[warp] + incl - x;
}

// ---- the tile window ---------------------------------------------------------------------

struct WindowSpan {
  long long w0, w1;  // virtual byte range of the window
  long long b0, b1;  // part covered by the bulk copy (b0 == b1: none)
};

// The window of `tile` is virtual bytes [tile*T - HALO, tile*T + T + HALO); the bulk copy
// takes the whole 16-byte source segments that lie inside [off0, vbytes).
__device__ __forceinline__ WindowSpan window_span(const Params &p, uint32_t tile) {
  WindowSpan w;
  w.w0 = (long long)tile * TILE_BYTES - HALO;
  w.w1 = w.w0 + WIN_BYTES;
  const long long seg_lo = (long long)((p.off0 + 15u) & ~15u);
  const long long seg_hi = (long long)(p.vbytes & ~15ull);
  w.b0 = w.w0 > seg_lo ? w.w0 : seg_lo;
  w.b1 = w.w1 < seg_hi ? w.w1 : seg_hi;
  if (w.b1 <= w.b0) w.b0 = w.b1 = w.w0;
  return w;
}

// Issues the bulk copy of `tile`'s window into `buf` (one thread).
__device__ __forceinline__ void issue_window(const Params &p, uint32_t tile, uint8_t *buf,
                                             uint64_t *bar) {
  const WindowSpan w = window_span(p, tile);
  if (w.b1 > w.b0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(w.b1 - w.b0));
    bulk_load(buf + (w.b0 - w.w0), p.base + w.b0, (uint32_t)(w.b1 - w.b0), bar);
  } else {
    mbar_arrive(bar);
  }
}

// Fills the window bytes the bulk copy does not cover: source bytes where the virtual
// position is inside [off0, vbytes), zero elsewhere.  One warp; ends with __syncwarp.
__device__ __forceinline__ void fill_window_edges_warp(const Params &p, uint32_t tile, uint8_t *buf) {
  const WindowSpan w = window_span(p, tile);
  if (w.b0 == w.w0 && w.b1 == w.w1) return;
  for (long long v = w.w0 + (threadIdx.x & 31); v < w.w1; v += 32) {
    if (v >= w.b0 && v < w.b1) continue;
    uint8_t byte = 0;
    if (v >= (long long)p.off0 && v < (long long)p.vbytes) byte = p.base[v];
    buf[v - w.w0] = byte;
  }
  __syncwarp();
}

// ---- the producer warp -------------------------------------------------------------------

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// mbar_test as seen by lane 0, the same for the whole warp (a phase can complete between two
// lanes' tests; the producer's control flow must not diverge on that).
__device__ __forceinline__ bool mbar_test_warp(uint64_t *bar, uint32_t parity) {
  uint32_t ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_test(bar, parity);
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Resumable decoupled look-back (one warp).  poll() reads the 32 states before `pred` once;
// it returns true when the exclusive prefix is complete.  The caller interleaves polls with
// other work instead of spinning.
struct LookBack {
  long long pred;       // next predecessor to read (lane 0's)
  uint64_t excl;        // sum collected so far
  uint32_t polls;       // polls that found a predecessor not yet published
  __device__ __forceinline__ void start(uint32_t tile) {
    pred = (long long)tile - 1;
    excl = 0;
    polls = 0;
  }
  __device__ __forceinline__ bool poll(const Params &p, uint32_t epoch) {
    const int lane = threadIdx.x & 31;
    const long long idx = pred - lane;
    uint64_t s = ST_FLAG_INC;  // before tile 0: an inclusive prefix of 0
    bool ok = true;
    if (idx >= 0) {
      s = ld_relaxed_u64(&p.states[idx]);
      ok = (s >> 62) != 0 && (uint32_t)((s >> ST_EPOCH_SHIFT) & ST_EPOCH_MASK) == epoch;
    }
    if (!__all_sync(0xffffffffu, ok)) {
      if (++polls >= p.wait_limit || ((polls & 63) == 0 && ld_relaxed_u32(&p.ws->status))) {
        note_timeout(p.ws);
        return true;  // give up: the prefix collected so far is used
      }
      return false;
    }
    const uint32_t incmask = __ballot_sync(0xffffffffu, (s >> 62) == 2);
    const int first_inc = incmask ? __ffs(incmask) - 1 : 32;
    excl += warp_sum_u64(lane <= first_inc ? (s & ST_VALUE_MASK) : 0ull);
    if (incmask) return true;
    pred -= 32;
    return false;
  }
};

// Runs the producer warp as a non-blocking event loop over the NS-stage ring:
//   * issue: while a stage is free (its previous use released by the consumers), claim the
//     next tile (a global ticket when SCAN, else round-robin) and start its bulk copy;
//   * land: when the copy of the oldest unlanded use arrives, fill the window's edges and,
//     when SCAN, count the tile (count(tile, window) -> output units, whole warp) and publish
//     that aggregate at once, so that later tiles' look-backs never wait on this CTA's queue;
//   * finish: advance the look-back of the oldest landed use by one poll; when it completes,
//     publish the inclusive prefix, record the tile's offset and hand the stage over.
// Uses are handed over in the order they were issued; one use past the last tile carries
// the end marker.  If nothing progresses for LOCAL_WAIT_ROUNDS polls the launch records
// GBU_TIMEOUT and the remaining uses are handed over as end markers.
template <int NS, bool SCAN, class Count>
__device__ __forceinline__ void run_producer(const Params &p, PipeSmem<NS> &ps,
                                             uint8_t (*win)[WIN_BYTES], uint32_t epoch,
                                             Count count) {
  const int lane = threadIdx.x & 31;
  const uint64_t tag = (uint64_t)epoch << ST_EPOCH_SHIFT;
  uint32_t issued = 0, landed = 0, finished = 0, idle = 0;
  bool ended = false, lb_active = false;
  LookBack lb;
  while (true) {
    bool progress = false;
    // issue
    while (!ended && issued < finished + NS) {
      const int s = issued % NS;
      if (issued >= (uint32_t)NS && !mbar_test_warp(&ps.empty[s], ((issued / NS) - 1) & 1)) break;
      uint32_t tile = 0;
      if (lane == 0) {
        tile = SCAN ? atomicAdd(&p.ws->ticket, 1u) : blockIdx.x + issued * gridDim.x;
        ps.info[s].tile = tile;
        if (tile < p.ntiles) issue_window(p, tile, win[s], &ps.full[s]);
      }
      tile = __shfl_sync(0xffffffffu, tile, 0);
      ended = tile >= p.ntiles;
      ++issued;
      progress = true;
    }
    // land
    while (landed < issued) {
      const int s = landed % NS;
      // lane 0 wrote info[s]; broadcast its value (a shuffle does not order shared memory)
      const uint32_t t = __shfl_sync(0xffffffffu, lane == 0 ? ps.info[s].tile : 0u, 0);
      if (t < p.ntiles) {
        if (!mbar_test_warp(&ps.full[s], (landed / NS) & 1)) break;
        fill_window_edges_warp(p, t, win[s]);
        if (SCAN) {
          const uint32_t agg = count(t, win[s]);
          if (lane == 0) {
            ps.info[s].total = agg;
            atomicAdd(&p.ws->total, (unsigned long long)agg);
            if ((long long)t != p.skip_tile)
              st_relaxed_u64(&p.states[t], (t == 0 ? ST_FLAG_INC : ST_FLAG_AGG) | tag |
                                               ((uint64_t)agg & ST_VALUE_MASK));
          }
        }
      }
      ++landed;
      progress = true;
    }
    // finish
    if (finished < landed) {
      const int s = finished % NS;
      const uint32_t t = __shfl_sync(0xffffffffu, lane == 0 ? ps.info[s].tile : 0u, 0);
      bool done = true;
      if (SCAN && t < p.ntiles && t > 0) {
        if (!lb_active) {
          lb.start(t);
          lb_active = true;
        }
        done = lb.poll(p, epoch);
        progress = true;
      }
      if (done) {
        lb_active = false;
        if (lane == 0) {
          if (SCAN && t < p.ntiles) {
            const uint64_t ex = t > 0 ? lb.excl : 0;
            ps.info[s].excl = ex;
            if (t > 0 && (long long)t != p.skip_tile)
              st_relaxed_u64(&p.states[t], ST_FLAG_INC | tag |
                                               ((ex + ps.info[s].total) & ST_VALUE_MASK));
          }
          mbar_arrive(&ps.ready[s]);
        }
        __syncwarp();
        ++finished;
        progress = true;
      }
    }
    if (ended && finished == issued) break;
    if (progress) {
      idle = 0;
    } else if (++idle >= LOCAL_WAIT_ROUNDS) {
      note_timeout(p.ws);
      // hand every unfinished use over as an end marker so that the consumers stop
      for (; finished < issued; ++finished) {
        const int s = finished % NS;
        if (lane == 0) {
          ps.info[s].tile = 0xFFFFFFFFu;
          mbar_arrive(&ps.ready[s]);
        }
      }
      break;
    } else {
      __nanosleep(20);
    }
  }
}

// ---- output staging ----------------------------------------------------------------------

// Writes the staged output of one tile (called by all NC consumer threads).  The tile's `cnt`
// output units start at global unit S; staged index h + k holds global unit S + k, where
// h = (dshift + S) & (V - 1) puts staged chunk boundaries on 16-byte destination boundaries.
// Units at or past cap are not written.  Whole 16-byte chunks go out with one bulk store
// issued (and committed as one bulk group) by consumer thread 0; the ragged head and tail are
// written by the other threads.  Every thread that wrote the staging buffer must have run
// fence_proxy_async_smem() before the consumer barrier preceding this call.
template <typename U>
__device__ __forceinline__ void store_staged(const Params &p, const U *staging, uint64_t S,
                                             uint32_t cnt) {
  constexpr uint32_t V = 16 / sizeof(U);
  uint64_t lim = cnt;
  if (S >= p.cap) lim = 0;
  else if (p.cap - S < lim) lim = p.cap - S;
  const uint32_t h = (uint32_t)((p.dshift + S) & (V - 1));
  const uint64_t A0 = (p.dshift + S) - h;  // aligned unit index (relative to dbase) of staging[0]
  U *gdst = reinterpret_cast<U *>(p.dbase) + A0;
  const uint32_t end = h + (uint32_t)lim;
  const uint32_t first_full = (h + V - 1) / V;
  const uint32_t last_full = end / V;
  if (first_full < last_full) {
    if (threadIdx.x == 0)
      bulk_store(gdst + first_full * V, staging + first_full * V, (last_full - first_full) * 16u);
    const uint32_t head_end = first_full * V;
    for (uint32_t i = h + threadIdx.x; i < head_end; i += NC) gdst[i] = staging[i];
    for (uint32_t i = last_full * V + threadIdx.x; i < end; i += NC) gdst[i] = staging[i];
  } else {
    for (uint32_t i = h + threadIdx.x; i < end; i += NC) gdst[i] = staging[i];
  }
  if (threadIdx.x == 0) bulk_commit();
}

// ---- completion ---------------------------------------------------------------------------

// Reduces per-thread error positions and totals over the CTA and folds them into the
// workspace (all NTHREADS threads).
template <int NS>
__device__ __forceinline__ void cta_fold(const Params &p, PipeSmem<NS> &ps, unsigned long long err,
                                         unsigned long long total, bool want_err, bool want_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (want_err) {
    err = warp_min_u64(err);
    if (lane == 0) ps.red[warp] = err;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = NO_ERROR;
      for (int w = 0; w < NTHREADS / 32; ++w) m = ps.red[w] < m ? ps.red[w] : m;
      if (m != NO_ERROR) atomicMin(&p.ws->errkey, m);
    }
    __syncthreads();
  }
  if (want_total) {
    total = warp_sum_u64(total);
    if (lane == 0) ps.red[warp] = total;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < NTHREADS / 32; ++w) t += ps.red[w];
      if (t) atomicAdd(&p.ws->total, t);
    }
    __syncthreads();
  }
}

// Called by every CTA after its loops.  Returns true in exactly one CTA (the last to finish),
// after which that CTA may read the accumulated header fields.  All threads participate.
template <int NS>
__device__ __forceinline__ bool finish_cta(const Params &p, PipeSmem<NS> &ps) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&p.ws->done, 1u);
    ps.is_last = prev == gridDim.x - 1;
    if (ps.is_last) __threadfence();
  }
  __syncthreads();
  return ps.is_last != 0;
}

// Resets the per-launch header fields and advances the epoch (last CTA, all threads; the
// whole CTA clears the scan states when the epoch wraps).
__device__ __forceinline__ void reset_workspace(const Params &p) {
  __shared__ uint32_t wrap;
  if (threadIdx.x == 0) {
    WsHeader *ws = p.ws;
    ws->ticket = 0;
    ws->done = 0;
    ws->errkey = NO_ERROR;
    ws->total = 0;
    ws->status = 0;
    const uint32_t e = ws->epoch + 1;
    wrap = e > ST_EPOCH_MASK;
    ws->epoch = wrap ? 1u : e;
  }
  __syncthreads();
  if (wrap) {
    for (uint32_t i = threadIdx.x; i < p.max_states; i += NTHREADS) p.states[i] = 0;
  }
  __threadfence();
}

__device__ __forceinline__ void write_result(gbu_result *r, int32_t status, uint64_t count) {
  r->status = status;
  r->reserved = 0;
  r->count = count;
}

}  // namespace gbu
