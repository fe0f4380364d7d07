// gbu_shard.cu -- one buffer split into P shards at character boundaries, and the shards'
// results combined into the result of the whole buffer.  This is the host logic of running
// one input over several streams, or over several GPUs (one shard per rank): every shard is
// an ordinary single-buffer call, and the only exchange is the one the combination needs
// (the output lengths, for the shards' output offsets, and the first error).
//
// Cut rule (Section 3 formats).  Shard k nominally starts at c_k = floor(k n / P) (balanced);
// the cut moves forward to a character start:
//   UTF-8:    the first position in [c, c+3) whose byte is not a continuation byte (10xxxxxx),
//             else c+3 (then c, c+1, c+2 are continuation bytes: at least one of them, or the
//             byte at c+3, belongs to no sequence, so an error lies at or before c+3 anyway);
//   UTF-16LE: c+1 when the word at c is a second surrogate (DC00-DFFF), else c.
// Inside a valid prefix every cut is therefore a character start, and a sequence that a cut
// splits fails in its shard with the kind and offset it has in the whole buffer (a missing
// continuation reads as TOO_SHORT at the end of a shard as before the next leading byte; a
// first surrogate ending a shard is never followed by a second one).  Hence the first shard
// with an error holds the first error of the buffer, and the shards before it are valid.
// Both rules are monotone in c, so the cuts never decrease.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbu_internal.h"
#include "gbutf.h"

namespace {

__host__ __device__ inline uint64_t nominal_cut(uint64_t n, uint64_t P, uint64_t k) {
  const uint64_t q = n / P, r = n % P;
  return q * k + (k < r ? k : r);
}

__host__ __device__ inline uint64_t cut_utf8(const uint8_t *s, uint64_t n, uint64_t c) {
  for (uint64_t j = 0; j < 3; ++j) {
    if (c + j >= n) return n;
    if ((s[c + j] & 0xC0u) != 0x80u) return c + j;
  }
  return c + 3 < n ? c + 3 : n;
}

__host__ __device__ inline uint64_t cut_utf16(const uint16_t *s, uint64_t n, uint64_t c) {
  if (c >= n) return n;
  return (s[c] & 0xFC00u) == 0xDC00u ? c + 1 : c;
}

template <bool UTF16>
__global__ void shard_cuts_kernel(const void *src, uint64_t n, uint32_t P, uint64_t *cuts) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > P) return;
  uint64_t v;
  if (k == 0) v = 0;
  else if (k == P) v = n;
  else if (UTF16) v = cut_utf16(static_cast<const uint16_t *>(src), n, nominal_cut(n, P, k));
  else v = cut_utf8(static_cast<const uint8_t *>(src), n, nominal_cut(n, P, k));
  cuts[k] = v;
}

template <bool UTF16>
int shard_cuts_launch(gbu_ctx *ctx, const void *src, uint64_t n, uint32_t P, uint64_t *cuts, gbu_stream stream) {
  if (!ctx || P < 1 || P > GBU_MAX_SHARDS || !cuts || ((uintptr_t)cuts & 7)) return GBU_BAD_ARGUMENT;
  if (n > 0 && !src) return GBU_BAD_ARGUMENT;
  if (UTF16 && ((uintptr_t)src & 1)) return GBU_BAD_ARGUMENT;
  const int dev = gbu_internal_device(ctx);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != dev) cudaSetDevice(dev);
  const uint32_t threads = 256, blocks = (P + 1 + threads - 1) / threads;
  shard_cuts_kernel<UTF16><<<blocks, threads, 0, (cudaStream_t)stream>>>(src, n, P, cuts);
  const cudaError_t e = cudaGetLastError();
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  if (e != cudaSuccess) return GBU_CUDA_ERROR;
  gbu_internal_count_launch(ctx);
  return GBU_OK;
}

template <bool UTF16>
int shard_cuts_host(const void *src, uint64_t n, uint32_t P, uint64_t *cuts) {
  if (P < 1 || P > GBU_MAX_SHARDS || !cuts || (n > 0 && !src)) return GBU_BAD_ARGUMENT;
  for (uint64_t k = 0; k <= P; ++k) {
    if (k == 0) cuts[k] = 0;
    else if (k == P) cuts[k] = n;
    else if (UTF16) cuts[k] = cut_utf16(static_cast<const uint16_t *>(src), n, nominal_cut(n, P, k));
    else cuts[k] = cut_utf8(static_cast<const uint8_t *>(src), n, nominal_cut(n, P, k));
  }
  return GBU_OK;
}

}  // namespace

extern "C" int gbu_shard_cuts_utf8(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint32_t P, uint64_t *cuts,
                                   gbu_stream stream) {
  return shard_cuts_launch<false>(ctx, src, n, P, cuts, stream);
}

extern "C" int gbu_shard_cuts_utf16le(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint32_t P, uint64_t *cuts,
                                      gbu_stream stream) {
  return shard_cuts_launch<true>(ctx, src, n, P, cuts, stream);
}

extern "C" int gbu_shard_cuts_utf8_host(const uint8_t *src, uint64_t n, uint32_t P, uint64_t *cuts) {
  return shard_cuts_host<false>(src, n, P, cuts);
}

extern "C" int gbu_shard_cuts_utf16le_host(const uint16_t *src, uint64_t n, uint32_t P, uint64_t *cuts) {
  return shard_cuts_host<true>(src, n, P, cuts);
}

extern "C" int gbu_combine_shards(const uint64_t *cuts, const gbu_result *parts, uint32_t P, gbu_result *out) {
  if (!cuts || !parts || !out || P < 1 || P > GBU_MAX_SHARDS) return GBU_BAD_ARGUMENT;
  for (uint32_t k = 0; k < P; ++k)
    if (cuts[k + 1] < cuts[k]) return GBU_BAD_ARGUMENT;
  // a shard whose call failed on the device makes the whole result that failure
  for (uint32_t k = 0; k < P; ++k) {
    const int32_t s = parts[k].status;
    if (s == GBU_TIMEOUT || s == GBU_CUDA_ERROR || s == GBU_BAD_ARGUMENT) {
      *out = gbu_result{s, 0, 0};
      return GBU_OK;
    }
  }
  // the first shard with an input error holds the buffer's first error
  for (uint32_t k = 0; k < P; ++k) {
    const int32_t s = parts[k].status;
    if (s >= GBU_HEADER_BITS && s <= GBU_SURROGATE) {
      *out = gbu_result{s, 0, cuts[k] + parts[k].count};
      return GBU_OK;
    }
  }
  uint64_t total = 0;
  bool small = false;
  for (uint32_t k = 0; k < P; ++k) {
    const int32_t s = parts[k].status;
    if (s != GBU_OK && s != GBU_OUTPUT_TOO_SMALL) return GBU_BAD_ARGUMENT;
    small = small || s == GBU_OUTPUT_TOO_SMALL;
    total += parts[k].count;
  }
  *out = gbu_result{small ? GBU_OUTPUT_TOO_SMALL : GBU_OK, 0, total};
  return GBU_OK;
}
