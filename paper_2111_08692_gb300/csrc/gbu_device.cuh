// gbu_device.cuh -- device-side building blocks shared by the UTF-8 and UTF-16 kernels.
//
// Every kernel of the library is a persistent grid that walks fixed-size tiles of the input:
//   * tiles are claimed with a global ticket counter, so a CTA only ever waits on tiles that
//     running CTAs already hold (forward progress does not depend on CTA scheduling);
//   * each tile's bytes, plus a 16-byte halo on both sides, are copied into a shared-memory
//     ring by the bulk-copy engine (cp.async.bulk + mbarrier), NSTAGE tiles ahead;
//   * transcoders give every tile its output offset with a single-pass decoupled look-back
//     scan (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back",
//     2016): a tile publishes its aggregate, then its inclusive prefix, in one 64-bit word;
//   * output is staged in shared memory and written back with cp.async.bulk stores for the
//     16-byte-aligned middle and plain stores for the two ragged ends;
//   * the first error is a 64-bit atomicMin over input positions; the last CTA to finish
//     (a completion counter) turns it into the exact offset and kind and writes the result.
// Every spin wait is bounded; when a bound is hit the kernel records GBU_TIMEOUT and keeps
// going, so a launch always terminates.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbutf.h"

namespace gbu {

constexpr int NT = 256;                       // threads per CTA
constexpr int NSTAGE = 3;                     // depth of the input ring
constexpr int HALO = 16;                      // halo bytes on each side of a tile
constexpr uint32_t CHUNK = 16;                // input bytes per thread per tile
constexpr uint32_t TILE_BYTES = NT * CHUNK;   // 4096 input bytes per tile
constexpr uint32_t WIN_BYTES = TILE_BYTES + 2 * HALO;

// Scan state word: [63:62] flag, [61:44] epoch, [43:0] value.
constexpr uint64_t ST_FLAG_AGG = 1ull << 62;
constexpr uint64_t ST_FLAG_INC = 2ull << 62;
constexpr int ST_EPOCH_SHIFT = 44;
constexpr uint32_t ST_EPOCH_MASK = (1u << 18) - 1;
constexpr uint64_t ST_VALUE_MASK = (1ull << 44) - 1;

constexpr unsigned long long NO_ERROR = ~0ull;

// Workspace header, one per context (device memory, zeroed at creation).  The last CTA of a
// launch resets ticket/done/errkey/total and advances the epoch, so consecutive launches on
// one stream need no memset.
struct WsHeader {
  uint32_t epoch;                 // tags scan states of the current launch (1 .. 2^18-1)
  uint32_t ticket;                // next tile to claim
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
  uint32_t wait_limit;     // polling rounds before a wait gives up
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

// ---- shared memory common to every kernel -------------------------------------------------

struct __align__(16) LoopSmem {
  uint64_t bar[NSTAGE];
  uint32_t ticket[NSTAGE];
  uint32_t warp_sums[NT / 32 + 2];
  uint32_t tile_err[2];          // smallest erroring thread index per tile (NT: none), by
                                 // iteration parity so that a reset never races a new tile
  unsigned long long excl;       // exclusive output prefix of the current tile
  unsigned long long cta_total;  // CTA-local sum (length kernels)
  int is_last;
};

// Inclusive scan over the CTA (one value per thread).  Returns the exclusive prefix of this
// thread; *total receives the CTA sum.  Contains two __syncthreads.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_sums,
                                                         uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < NT / 32 ? warp_sums[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int d = 1; d < NT / 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, si, d);
      if (lane >= d) si += y;
    }
    if (lane < NT / 32) warp_sums[lane] = si - s;
    if (lane == NT / 32 - 1) warp_sums[NT / 32] = si;
  }
  __syncthreads();
  *total = warp_sums[NT / 32];
  return warp_sums[warp] + incl - x;
}

// Records a failed wait: the launch reports GBU_TIMEOUT.
__device__ __forceinline__ void note_timeout(WsHeader *ws) { atomicOr(&ws->status, 1u); }

// Decoupled look-back for tile `tile` with aggregate `agg`; executed by all 32 lanes of one
// warp.  Returns the tile's exclusive prefix.  Waits are bounded by p.wait_limit rounds.
__device__ __forceinline__ uint64_t lookback(const Params &p, uint32_t tile, uint64_t agg,
                                          uint32_t epoch) {
  const int lane = threadIdx.x & 31;
  const uint64_t tag = (uint64_t)epoch << ST_EPOCH_SHIFT;
  const bool skip = (long long)tile == p.skip_tile;
  if (tile == 0) {
    if (lane == 0 && !skip) st_relaxed_u64(&p.states[0], ST_FLAG_INC | tag | (agg & ST_VALUE_MASK));
    return 0;
  }
  if (lane == 0 && !skip) st_relaxed_u64(&p.states[tile], ST_FLAG_AGG | tag | (agg & ST_VALUE_MASK));
  uint64_t excl = 0;
  long long pred = (long long)tile - 1;
  while (true) {
    const long long idx = pred - lane;
    uint64_t s = ST_FLAG_INC;  // before tile 0: an inclusive prefix of 0
    if (idx >= 0) {
      uint32_t rounds = 0;
      uint32_t ns = 32;
      while (true) {
        s = ld_relaxed_u64(&p.states[idx]);
        if ((s >> 62) != 0 && (uint32_t)((s >> ST_EPOCH_SHIFT) & ST_EPOCH_MASK) == epoch) break;
        if (++rounds >= p.wait_limit || ((rounds & 63) == 0 && ld_relaxed_u32(&p.ws->status))) {
          note_timeout(p.ws);
          s = ST_FLAG_INC;  // give up: treat as an inclusive prefix of 0
          break;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
      }
    }
    const bool inc = (s >> 62) == 2;
    const uint32_t incmask = __ballot_sync(0xffffffffu, inc);
    const int first_inc = incmask ? __ffs(incmask) - 1 : 32;
    const uint64_t v = lane <= first_inc ? (s & ST_VALUE_MASK) : 0ull;
    excl += warp_sum_u64(v);
    if (incmask) break;
    pred -= 32;
  }
  if (lane == 0 && !skip)
    st_relaxed_u64(&p.states[tile], ST_FLAG_INC | tag | ((excl + agg) & ST_VALUE_MASK));
  return excl;
}

// ---- the tile window ---------------------------------------------------------------------

// Issues the bulk copy of tile `tile`'s window into `buf`: virtual bytes
// [tile*T - HALO, tile*T + T + HALO), restricted to whole 16-byte segments of the source
// that lie inside [off0, vbytes).  Called by one thread.  The rest of the window is filled
// by fill_window_edges after the copy has landed.
__device__ __forceinline__ void issue_window(const Params &p, uint32_t tile, uint8_t *buf,
                                             uint64_t *bar) {
  const long long w0 = (long long)tile * TILE_BYTES - HALO;
  const long long w1 = w0 + WIN_BYTES;
  const long long seg_lo = (long long)((p.off0 + 15u) & ~15u);
  const long long seg_hi = (long long)(p.vbytes & ~15ull);
  const long long b0 = w0 > seg_lo ? w0 : seg_lo;
  const long long b1 = w1 < seg_hi ? w1 : seg_hi;
  if (b1 > b0) {
    mbar_arrive_expect_tx(bar, (uint32_t)(b1 - b0));
    bulk_load(buf + (b0 - w0), p.base + b0, (uint32_t)(b1 - b0), bar);
  } else {
    mbar_arrive(bar);
  }
}

// True if the window of `tile` has bytes that the bulk copy does not cover.
__device__ __forceinline__ bool window_has_edges(const Params &p, uint32_t tile) {
  const long long w0 = (long long)tile * TILE_BYTES - HALO;
  const long long w1 = w0 + WIN_BYTES;
  const long long seg_lo = (long long)((p.off0 + 15u) & ~15u);
  const long long seg_hi = (long long)(p.vbytes & ~15ull);
  return w0 < seg_lo || w1 > seg_hi;
}

// Fills the window bytes outside the bulk-copied range: source bytes where the virtual
// position is inside [off0, vbytes), zero elsewhere.  All threads; ends with __syncthreads.
__device__ __forceinline__ void fill_window_edges(const Params &p, uint32_t tile, uint8_t *buf) {
  const long long w0 = (long long)tile * TILE_BYTES - HALO;
  const long long w1 = w0 + WIN_BYTES;
  const long long seg_lo = (long long)((p.off0 + 15u) & ~15u);
  const long long seg_hi = (long long)(p.vbytes & ~15ull);
  long long b0 = w0 > seg_lo ? w0 : seg_lo;
  long long b1 = w1 < seg_hi ? w1 : seg_hi;
  if (b1 < b0) b1 = b0 = w0;  // nothing copied
  for (long long v = w0 + threadIdx.x; v < w1; v += NT) {
    if (v >= b0 && v < b1) continue;
    uint8_t byte = 0;
    if (v >= (long long)p.off0 && v < (long long)p.vbytes) byte = p.base[v];
    buf[v - w0] = byte;
  }
  __syncthreads();
}

// Polling rounds before a wait on the bulk-copy engine gives up (each try_wait round also
// suspends for a hardware-chosen time, so this is seconds).
constexpr uint32_t COPY_WAIT_ROUNDS = 1u << 24;

// Bounded wait for the bulk copy of a stage (all threads).  Returns false on timeout.
__device__ __forceinline__ bool wait_stage(const Params &p, uint64_t *bar, uint32_t parity) {
  uint32_t rounds = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++rounds >= COPY_WAIT_ROUNDS) {
      note_timeout(p.ws);
      return false;
    }
  }
  return true;
}

// After the loop gave up at iteration `it`, waits (bounded) for the copies that were issued
// for iterations it .. it+NSTAGE-1 and never consumed.  Thread 0 only.
__device__ __forceinline__ void drain_stages(const Params &p, LoopSmem &ls, uint32_t it) {
  for (uint32_t j = 0; j < (uint32_t)NSTAGE; ++j) {
    const uint32_t k = it + j;
    const int s = k % NSTAGE;
    if (ls.ticket[s] >= p.ntiles) continue;
    uint32_t rounds = 0;
    while (!mbar_try_wait(&ls.bar[s], (k / NSTAGE) & 1) && ++rounds < COPY_WAIT_ROUNDS) {
    }
  }
}

// ---- output staging ----------------------------------------------------------------------

// Writes the staged output of one tile.  The tile's `cnt` output units start at global unit
// S; in the staging buffer unit i corresponds to global unit (S & ~(V-1) aligned with dshift)
// as set up by the caller: staged index h + k holds global unit S + k, with
// h = (dshift + S) & (V - 1).  Units at or past cap are not written.  Whole 16-byte chunks
// go out with one bulk store (issued by thread 0, committed as one bulk group); the ragged
// head and tail are written by other threads.  Every thread that wrote the staging buffer
// must have executed fence_proxy_async_smem() before the __syncthreads preceding this call.
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
    if (threadIdx.x == 0) {
      bulk_store(gdst + first_full * V, staging + first_full * V, (last_full - first_full) * 16u);
    }
    const uint32_t head_end = first_full * V;
    for (uint32_t i = h + threadIdx.x; i < head_end; i += NT) gdst[i] = staging[i];
    for (uint32_t i = last_full * V + threadIdx.x; i < end; i += NT) gdst[i] = staging[i];
  } else {
    for (uint32_t i = h + threadIdx.x; i < end; i += NT) gdst[i] = staging[i];
  }
  if (threadIdx.x == 0) bulk_commit();
}

// ---- completion ---------------------------------------------------------------------------

// Called by every CTA after its loop.  Returns true in exactly one CTA (the last to finish),
// after which that CTA may read the accumulated header fields.  All threads participate.
__device__ __forceinline__ bool finish_cta(const Params &p, LoopSmem &ls) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&p.ws->done, 1u);
    ls.is_last = prev == gridDim.x - 1;
    if (ls.is_last) __threadfence();
  }
  __syncthreads();
  return ls.is_last != 0;
}

// Resets the per-launch header fields and advances the epoch (last CTA, thread 0 after the
// result is written; the whole CTA when the epoch wraps and the states must be cleared).
__device__ __forceinline__ void reset_workspace(const Params &p) {
  __shared__ uint32_t wrap;
  if (threadIdx.x == 0) {
    WsHeader *ws = p.ws;
    ws->ticket = 0;
    ws->done = 0;
    ws->errkey = NO_ERROR;
    ws->total = 0;
    ws->status = 0;
    uint32_t e = ws->epoch + 1;
    wrap = e > ST_EPOCH_MASK;
    ws->epoch = wrap ? 1u : e;
  }
  __syncthreads();
  if (wrap) {
    for (uint32_t i = threadIdx.x; i < p.max_states; i += NT) p.states[i] = 0;
  }
  __threadfence();
}

// Writes a gbu_result (one 16-byte store where the pointer allows it).
__device__ __forceinline__ void write_result(gbu_result *r, int32_t status, uint64_t count) {
  r->status = status;
  r->reserved = 0;
  r->count = count;
}

}  // namespace gbu
