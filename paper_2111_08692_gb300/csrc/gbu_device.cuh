// gbu_device.cuh -- device-side building blocks shared by the kernels.
//
// Two kernel shapes:
//   * read-only kernels (validation, lengths; gbu_stream.cu) stream 4 KB warp tiles with
//     16-byte loads, never waiting on another CTA;
//   * transcoders (gbu_utf8.cu, gbu_utf16.cu) walk 16 KB partitions claimed from a ticket
//     counter.  A CTA counts the output units of partition k+1 (a read from HBM) and
//     publishes that aggregate before it transcodes partition k (a re-read, normally from
//     L2).  Partition k's output offset comes from the single-pass decoupled look-back of
//     Merrill & Garland ("Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016):
//     every partition publishes its aggregate, then its inclusive prefix, in one 64-bit
//     state word; a partition sums its predecessors' words back to the nearest inclusive
//     prefix.  Counting one partition ahead means the aggregates a look-back needs were
//     published a whole partition earlier.  Output goes through shared-memory staging and
//     cp.async.bulk stores (16-byte-aligned middle) plus plain stores for the ragged ends.
// The first error is a 64-bit atomicMin over input positions; the last CTA to finish (a
// completion counter) turns it into the exact offset and kind and writes the result.  Every
// spin wait is bounded: when a bound is hit the launch records GBU_TIMEOUT and finishes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbutf.h"

namespace gbu {

constexpr int STREAM_THREADS = 256;           // threads per CTA of the read-only kernels
// Transcoders: small CTAs (4 warps, 8 resident per SM at 64 registers a thread), so that
// the phases of many CTAs (count pass, look-back, conversion) overlap on each SM.
constexpr int XT = 128;                       // threads per CTA of the transcoders
constexpr int XWARPS = XT / 32;
constexpr int XBLOCKS = 1024 / XT;            // transcoder CTAs resident per SM
constexpr uint32_t CHUNK = 16;                // input bytes per thread per round
constexpr uint32_t ROUND_BYTES = XT * CHUNK;  // 2 KB
constexpr int PART_ROUNDS = 8;
constexpr uint32_t PART_BYTES = ROUND_BYTES * PART_ROUNDS;  // 16 KB per partition

// Scan state word: [63:62] flag, [61:44] epoch, [43:0] value.
constexpr uint64_t ST_FLAG_AGG = 1ull << 62;
constexpr uint64_t ST_FLAG_INC = 2ull << 62;
constexpr int ST_EPOCH_SHIFT = 44;
constexpr uint32_t ST_EPOCH_MASK = (1u << 18) - 1;
constexpr uint64_t ST_VALUE_MASK = (1ull << 44) - 1;

constexpr unsigned long long NO_ERROR = ~0ull;

// Workspace header, one per context (device memory, initialised at creation).  The last CTA
// of a launch resets ticket/done/errkey/total/status and advances the epoch, so consecutive
// launches on one stream need no memset.
struct WsHeader {
  uint32_t epoch;                 // tags scan states of the current launch (1 .. 2^18-1)
  uint32_t ticket;                // next partition to claim (transcoders)
  uint32_t done;                  // CTAs that have finished
  uint32_t status;                // sticky: 1 = a wait gave up (GBU_TIMEOUT)
  unsigned long long errkey;      // smallest input position of a thread chunk with an error
  unsigned long long total;       // sum of partition aggregates (output length)
  uint32_t stop_tile;             // validation early exit: smallest warp tile with a flagged chunk
  uint32_t pad[23];
};
static_assert(sizeof(WsHeader) == 128, "header is one 128-byte line");

struct Params {
  const uint8_t *base;     // source rounded down to 16 bytes
  uint64_t vbytes;         // off0 + source bytes: virtual positions [off0, vbytes) are data
  uint32_t off0;           // source address - base (bytes)
  uint32_t ntiles;         // warp tiles (read-only kernels) or partitions (transcoders)
  uint64_t n;              // source length in code units
  uint8_t *dbase;          // destination rounded down to 16 bytes (transcoders)
  uint32_t dshift;         // (destination - dbase) in output code units
  uint64_t cap;            // destination capacity in output code units
  gbu_result *result;      // where the last CTA writes the result (validate/convert)
  uint64_t *len_out;       // where the last CTA writes the length (length functions)
  WsHeader *ws;
  uint64_t *states;        // one scan state per partition
  uint32_t max_states;     // entries in states[]
  uint32_t wait_limit;     // look-back polls before a wait gives up
  long long skip_tile;     // test hook: this partition never publishes (-1: off)
  uint32_t early_exit;     // validation and single-buffer transcoders: skip work past a known error
  uint32_t pad_;
};

// Batched operations (gbu_batch.cu), in the order of the single-buffer kernels.
enum BatchMode { B_V8 = 0, B_L16 = 1, B_C8 = 2, B_V16 = 3, B_L8 = 4, B_C16 = 5 };

// One string given by pointers instead of CSR offsets (the serving loop's requests).
struct StringDesc {
  const void *src;           // n input code units
  uint64_t n;
  void *dst;                 // transcoders: cap output code units
  uint64_t cap;
};
static_assert(sizeof(StringDesc) == 32, "descriptor layout");

struct BatchParams {
  const StringDesc *desc;    // non-NULL: string i is desc[i] (src, off, dst, dst_off unused)
  const uint8_t *src;        // the strings, back to back
  const uint64_t *off;       // B+1 input offsets (input code units)
  uint64_t B;                // number of strings
  uint8_t *dst;              // transcoders: the outputs, back to back
  const uint64_t *dst_off;   // transcoders: B+1 output offsets (output code units)
  gbu_result *results;       // validation, transcoding: B results
  uint64_t *lens;            // length functions: B lengths
  WsHeader *ws;              // claim counter (ticket) and completion counter (done)
  uint32_t grab;             // strings per claim
  uint32_t long_bytes;       // strings of at least this many input bytes go to a whole CTA
};

// Several strings transcoded by one launch, each split into partitions with its own look-back
// chain (gbu_xcode.cuh, transcode_segments).
struct SegState {            // per string; starts {NO_ERROR, 0, 0}, left so by the launch
  unsigned long long errkey; // smallest erroring chunk start of the string
  unsigned long long total;  // output units (set by the CTA of the string's last partition)
  uint32_t done;             // partitions finished
  uint32_t pad;
};

struct SegParams {
  const StringDesc *desc;    // B strings, each n >= 1
  const uint32_t *pstart;    // B+1: first partition of each string in the launch's numbering
  uint32_t B;
  uint32_t ntiles;           // pstart[B]
  SegState *seg;             // B entries
  gbu_result *results;       // B results
  WsHeader *ws;              // claim counter, completion counter, epoch, timeout flag
  uint64_t *states;          // ntiles look-back states (pstart[s] onwards for string s)
  uint32_t max_states;
  uint32_t wait_limit;
};

struct ScanParams {
  const uint64_t *in;
  uint64_t *out;             // count + 1 entries
  uint64_t count;
  gbu_result *result;        // {status, total}
  Params lb;                 // ws, states, ntiles, max_states, wait_limit, skip_tile
};

// ---- small PTX wrappers -----------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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
// The same three operations issued only where `pred` holds, as predicated instructions (no
// branch around them).
__device__ __forceinline__ void bulk_store_if(bool pred, void *dst_gmem, const void *src_smem, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
      "@p cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t}" ::"l"(dst_gmem),
      "r"(smem_addr(src_smem)), "r"(bytes), "r"((uint32_t)pred)
      : "memory");
}
__device__ __forceinline__ void bulk_commit_if(bool pred) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t@p cp.async.bulk.commit_group;\n\t}" ::"r"(
                   (uint32_t)pred)
               : "memory");
}

// wait until at most N committed bulk groups still read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait_read_if(bool pred) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %1, 0;\n\t@p cp.async.bulk.wait_group.read %0;\n\t}" ::"n"(N),
               "r"((uint32_t)pred)
               : "memory");
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

// 16-byte streaming load (read-only, no L1 allocation)
__device__ __forceinline__ uint4 ldg_stream(const uint8_t *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t ldg_word(const uint8_t *p) {
  return __ldg(reinterpret_cast<const unsigned int *>(p));
}

// L2 cache policies: keep a line resident (it will be read again soon), or mark it as the
// line's last use.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_last_use() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// One 32-byte store (p 32-byte aligned): a warp storing 32 consecutive such blocks writes whole
// 32-byte sectors in a single instruction.
__device__ __forceinline__ void st_global_32B(void *p, uint4 a, uint4 b) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a.x), "r"(a.y), "r"(a.z),
               "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

// The same with an L2 cache policy (output that no later work reads: an evict-first policy
// keeps it from displacing input lines that are read again).
__device__ __forceinline__ void st_global_32B_hint(void *p, uint4 a, uint4 b, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8}, %9;" ::"l"(p), "r"(a.x),
               "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w), "l"(pol)
               : "memory");
}

// 16-byte streaming load with an L2 cache policy
__device__ __forceinline__ uint4 ldg_stream_hint(const uint8_t *p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
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

// Mask keeping the bytes of a 32-bit word at virtual position w whose positions lie in
// [lo, hi) (bytes outside read as zero).
__device__ __forceinline__ uint32_t word_keep_mask(long long w, long long lo, long long hi) {
  const long long a = lo - w, b = hi - w;  // data bytes of the word: [a, b) clamped to [0, 4)
  const uint32_t la = a <= 0 ? 0u : (a >= 4 ? 4u : (uint32_t)a);
  const uint32_t hb = b <= 0 ? 0u : (b >= 4 ? 4u : (uint32_t)b);
  if (hb <= la) return 0u;
  const uint32_t upto = hb == 4 ? 0xFFFFFFFFu : (1u << (8 * hb)) - 1u;  // bytes below hb
  const uint32_t from = ~((1u << (8 * la)) - 1u);                        // bytes from la (la < 4)
  return upto & from;
}

// A 32-bit word at virtual position v (a multiple of 4), bytes outside [off0, vbytes) read as
// zero.  A word holding a data byte is read whole: an aligned word never crosses a page, so
// the bytes next to the data are readable (they are then cleared).
__device__ __forceinline__ uint32_t load_word_checked(const Params &p, long long v) {
  const long long lo = p.off0, hi = (long long)p.vbytes;
  if (v + 4 <= lo || v >= hi) return 0u;
  const uint32_t w = ldg_word(p.base + v);
  return (v >= lo && v + 4 <= hi) ? w : w & word_keep_mask(v, lo, hi);
}

// A 16-byte chunk at virtual position c (a multiple of 16): a streaming load when it lies
// inside the data; else, if it holds a data byte, the aligned chunk is read whole (it cannot
// cross a page) and the bytes outside [off0, vbytes) are cleared; else zeros.
__device__ __forceinline__ uint4 load_chunk(const Params &p, long long c, bool inside) {
  if (inside) return ldg_stream(p.base + c);
  const long long lo = p.off0, hi = (long long)p.vbytes;
  if (c + 16 <= lo || c >= hi) return make_uint4(0u, 0u, 0u, 0u);
  uint4 v = ldg_stream(p.base + c);
  v.x &= word_keep_mask(c, lo, hi);
  v.y &= word_keep_mask(c + 4, lo, hi);
  v.z &= word_keep_mask(c + 8, lo, hi);
  v.w &= word_keep_mask(c + 12, lo, hi);
  return v;
}

// load_chunk with an L2 cache policy on the fast path.
__device__ __forceinline__ uint4 load_chunk_hint(const Params &p, long long c, bool inside,
                                                 uint64_t pol) {
  if (inside) return ldg_stream_hint(p.base + c, pol);
  return load_chunk(p, c, false);
}

// ---- decoupled look-back -----------------------------------------------------------------

// Publishes partition `part`'s aggregate (the inclusive prefix at once for partition 0).
__device__ __forceinline__ void publish_aggregate(const Params &p, uint32_t part, uint64_t agg,
                                                  uint32_t epoch) {
  if ((long long)part == p.skip_tile) return;
  const uint64_t tag = (uint64_t)epoch << ST_EPOCH_SHIFT;
  st_relaxed_u64(&p.states[part], (part == 0 ? ST_FLAG_INC : ST_FLAG_AGG) | tag | (agg & ST_VALUE_MASK));
}

// Shared memory of lookback_cta: one record per warp and poll, in two buffers that
// alternate between polls (so a poll needs a single barrier).
template <int NTH>
struct LookbackSmem {
  uint32_t first[2][NTH / 32];          // first inclusive prefix (low 16 bits), first unpublished
  unsigned long long sum[2][NTH / 32];  // the warp's states up to its first inclusive prefix
};

// Exclusive prefix of partition `part` by a CTA-wide look-back (NTH threads): each poll
// reads NTH x K predecessor states at once (thread t the K states at distances tK+1 ..
// tK+K), so a look-back that has to sum many aggregates back to the nearest inclusive prefix
// takes one round trip per NTH x K states.  Only the states between the partition and the
// nearest inclusive prefix must have been published.  Each lane sums its states up to its
// first inclusive prefix and notes an unpublished state before it; each warp records its
// first lane holding an inclusive prefix, its first lane with an unpublished state and the
// sum of its lanes up to the former; after one barrier every thread combines the records
// (the sum runs over the warps up to the first one that holds an inclusive prefix).
// Returns the exclusive prefix (in every thread) and publishes the inclusive prefix.  The
// caller must pass a barrier between two calls with the same ls.
template <int NTH, int K = 1>
__device__ __forceinline__ uint64_t lookback_cta(const Params &p, uint32_t part, uint64_t agg,
                                                 uint32_t epoch, LookbackSmem<NTH> &ls) {
  constexpr int NW = NTH / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t excl = 0;
  if (part == 0) return 0;
  long long pred = (long long)part - 1;
  uint32_t polls = 0;
  int buf = 0;
  while (true) {
    uint64_t s[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const long long idx = pred - (long long)(threadIdx.x * K + j);
      s[j] = idx >= 0 ? ld_relaxed_u64(&p.states[idx]) : ST_FLAG_INC;  // before partition 0: 0
    }
    uint64_t lsum = 0;
    bool linc = false, lbad = false;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const bool before0 = pred < (long long)(threadIdx.x * K + j);
      const bool ok = before0 || ((s[j] >> 62) != 0 && (uint32_t)((s[j] >> ST_EPOCH_SHIFT) & ST_EPOCH_MASK) == epoch);
      if (!linc) {
        lbad = lbad || !ok;
        lsum += s[j] & ST_VALUE_MASK;
        linc = ok && (s[j] >> 62) == 2;
      }
    }
    const uint32_t incm = __ballot_sync(0xffffffffu, linc);
    const uint32_t badm = __ballot_sync(0xffffffffu, lbad);
    const int li = incm ? __ffs(incm) - 1 : 32;  // the warp's first lane with an inclusive prefix
    const uint64_t v = warp_sum_u64(lane <= li ? lsum : 0ull);
    if (lane == 0) {
      const uint32_t fi = incm ? (uint32_t)(warp * 32 + li) : 0xFFFFu;
      const uint32_t fb = badm ? (uint32_t)(warp * 32 + __ffs(badm) - 1) : 0xFFFFu;
      ls.first[buf][warp] = fi | (fb << 16);
      ls.sum[buf][warp] = v;
    }
    __syncthreads();
    uint32_t first_inc = 0xFFFFu, first_bad = 0xFFFFu;
    uint64_t t = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t f = ls.first[buf][w];
      if (first_inc == 0xFFFFu) t += ls.sum[buf][w];  // warps up to the first inclusive prefix
      first_inc = (f & 0xFFFFu) < first_inc ? (f & 0xFFFFu) : first_inc;
      first_bad = (f >> 16) < first_bad ? (f >> 16) : first_bad;
    }
    buf ^= 1;
    if (first_bad <= first_inc && first_bad != 0xFFFFu) {
      // a state we need is not published yet: poll again (bounded; the count is the same in
      // every thread, so all of them leave together)
      if (++polls >= p.wait_limit) {
        if (threadIdx.x == 0) note_timeout(p.ws);
        break;
      }
      __nanosleep(64);
      continue;
    }
    excl += t;
    if (first_inc != 0xFFFFu) break;
    pred -= (long long)NTH * K;
  }
  if (threadIdx.x == 0 && (long long)part != p.skip_tile) {
    const uint64_t tag = (uint64_t)epoch << ST_EPOCH_SHIFT;
    st_relaxed_u64(&p.states[part], ST_FLAG_INC | tag | ((excl + agg) & ST_VALUE_MASK));
  }
  return excl;
}

// ---- output staging ----------------------------------------------------------------------

// Writes `cnt` staged output units that start at global unit S (all NTH threads).  Staged
// index h + k holds global unit S + k, where h = (dshift + S) & (V - 1) puts staged chunk
// boundaries on 16-byte destination boundaries.  Units at or past cap are not written.
// Whole 16-byte chunks go out with one bulk store issued (and committed as one bulk group)
// by thread 0; the ragged head and tail are written with plain stores.  Every thread that
// wrote the staging buffer must have run fence_proxy_async_smem() before the barrier that
// precedes this call.
template <typename U, int NTH>
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
    for (uint32_t i = h + threadIdx.x; i < head_end; i += NTH) gdst[i] = staging[i];
    for (uint32_t i = last_full * V + threadIdx.x; i < end; i += NTH) gdst[i] = staging[i];
  } else {
    for (uint32_t i = h + threadIdx.x; i < end; i += NTH) gdst[i] = staging[i];
  }
  if (threadIdx.x == 0) bulk_commit();
}

// ---- completion ---------------------------------------------------------------------------

// Folds this thread's smallest error position (when want_err) or count (else) into the
// workspace, then counts the CTA as done.  Returns true in exactly one CTA (the last to
// finish), after which that CTA may read the accumulated header fields.  All threads.
template <int NTH>
__device__ __forceinline__ bool fold_and_finish(const Params &p, unsigned long long v, bool want_err,
                                                unsigned long long *red, int *is_last) {
  constexpr int NW = NTH / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = want_err ? warp_min_u64(v) : warp_sum_u64(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = want_err ? NO_ERROR : 0ull;
    for (int w = 0; w < NW; ++w) a = want_err ? (red[w] < a ? red[w] : a) : a + red[w];
    if (want_err && a != NO_ERROR) atomicMin(&p.ws->errkey, a);
    if (!want_err && a) atomicAdd(&p.ws->total, a);
    __threadfence();
    const uint32_t prev = atomicAdd(&p.ws->done, 1u);
    *is_last = prev == gridDim.x - 1;
    if (*is_last) __threadfence();
  }
  __syncthreads();
  return *is_last != 0;
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
    ws->stop_tile = 0xFFFFFFFFu;
    const uint32_t e = ws->epoch + 1;
    wrap = e > ST_EPOCH_MASK;
    ws->epoch = wrap ? 1u : e;
  }
  __syncthreads();
  if (wrap) {
    for (uint32_t i = threadIdx.x; i < p.max_states; i += blockDim.x) p.states[i] = 0;
  }
  __threadfence();
}

__device__ __forceinline__ void write_result(gbu_result *r, int32_t status, uint64_t count) {
  r->status = status;
  r->reserved = 0;
  r->count = count;
}

}  // namespace gbu
