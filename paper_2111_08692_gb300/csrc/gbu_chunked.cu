// gbu_chunked.cu -- the resumable (chunked) form: one input that arrives in pieces (read from a
// disk or a socket into host memory) is validated or transcoded piece by piece, with the same
// results as one call on the whole input.
//
// A push sees P = carry + chunk, where the carry is the incomplete character the previous push
// held back (Section 3: at most 3 bytes of a UTF-8 sequence, or a UTF-16 first surrogate).  It
// cuts P before a trailing incomplete character -- the last non-continuation byte among P's last
// three bytes, when it is a leading byte C2-F4 whose sequence is longer than what follows it,
// or a trailing first surrogate -- and keeps that piece as the next carry.  The rest, P[0:M),
// starts and ends at character starts of the stream (when it holds no error), so the ordinary
// single-buffer call on it gives the stream's result for those units: an error at offset o of
// P[0:M) lies at stream offset (position of P[0]) + o with the same kind, and the outputs of
// consecutive pushes concatenate to the output of the whole input.  A push marked last keeps
// nothing back, so an incomplete final character fails there (TOO_SHORT, or SURROGATE for a
// first surrogate at the end).  A leading byte that is invalid in any context (C0, C1, F5-FF)
// is never held back, so it fails in the push that delivers it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "gbutf.h"

struct gbu_chunked {
  int device;
  int op;                  // GBU_OP_VALIDATE_UTF8 / _VALIDATE_UTF16LE / _CONVERT_UTF8_TO_UTF16LE / _CONVERT_UTF16LE_TO_UTF8
  bool utf16_in;
  uint32_t in_unit, out_unit;
  uint64_t max_chunk;      // units per push
  gbu_ctx *ctx;
  cudaStream_t stream;
  void *din;               // device: carry + chunk (max_chunk + 4 units)
  void *dout;              // device: the largest output of one push (transcoders)
  uint64_t out_cap;        // units of dout
  gbu_result *res_h;       // mapped pinned: the device call's result
  gbu_result *res_d;
  uint64_t *len_h;         // mapped pinned: output length of a valid prefix (after an error)
  uint64_t *len_d;
  uint8_t carry[8];        // held-back units (bytes for UTF-8, little-endian words for UTF-16)
  uint32_t carry_n;        // in units
  uint64_t pos;            // stream offset (input units) of carry[0]
  uint64_t produced;       // output units written so far
  int32_t err_status;      // sticky first error (GBU_OK while none)
  uint64_t err_offset;
  bool finished;
};

namespace {

bool is_transcode(int op) { return op == GBU_OP_CONVERT_UTF8_TO_UTF16LE || op == GBU_OP_CONVERT_UTF16LE_TO_UTF8; }

// Unit i of P = carry[0:cn) + chunk[0:n).
uint32_t p_unit(const gbu_chunked *s, const void *chunk, uint64_t i) {
  if (i < s->carry_n) {
    if (!s->utf16_in) return s->carry[i];
    return (uint32_t)s->carry[2 * i] | ((uint32_t)s->carry[2 * i + 1] << 8);
  }
  const uint64_t j = i - s->carry_n;
  if (!s->utf16_in) return static_cast<const uint8_t *>(chunk)[j];
  return static_cast<const uint16_t *>(chunk)[j];
}

// Units at the end of P (of L units) that form an incomplete character to hold back.
uint64_t tail_units(const gbu_chunked *s, const void *chunk, uint64_t L) {
  if (L == 0) return 0;
  if (s->utf16_in) {
    const uint32_t w = p_unit(s, chunk, L - 1);
    return (w & 0xFC00u) == 0xD800u ? 1 : 0;
  }
  for (uint64_t back = 1; back <= 3 && back <= L; ++back) {
    const uint32_t b = p_unit(s, chunk, L - back);
    if ((b & 0xC0u) == 0x80u) continue;  // a continuation byte: look further back
    if (b < 0xC2u || b > 0xF4u) return 0;  // ASCII, or a byte that is invalid in any context
    const uint64_t len = b >= 0xF0u ? 4 : (b >= 0xE0u ? 3 : 2);
    return back < len ? back : 0;
  }
  return 0;
}

int ensure_device(int dev) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return -1;
  if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return -1;
  return cur;
}

}  // namespace

extern "C" gbu_chunked *gbu_chunked_create(int device, int op, uint64_t max_chunk_units) {
  if (op != GBU_OP_VALIDATE_UTF8 && op != GBU_OP_VALIDATE_UTF16LE && !is_transcode(op)) return nullptr;
  if (max_chunk_units == 0 || max_chunk_units > ((uint64_t)1 << 40)) return nullptr;
  const int prev = ensure_device(device);
  if (prev < 0) return nullptr;
  gbu_chunked *s = new gbu_chunked();
  memset(s, 0, sizeof(*s));
  s->device = device;
  s->op = op;
  s->utf16_in = op == GBU_OP_VALIDATE_UTF16LE || op == GBU_OP_CONVERT_UTF16LE_TO_UTF8;
  s->in_unit = s->utf16_in ? 2 : 1;
  s->out_unit = op == GBU_OP_CONVERT_UTF8_TO_UTF16LE ? 2 : 1;
  s->max_chunk = max_chunk_units;
  const uint64_t in_max = max_chunk_units + 4;
  // worst-case output of in_max units: one word per byte (8 -> 16), three bytes per word (16 -> 8)
  s->out_cap = op == GBU_OP_CONVERT_UTF8_TO_UTF16LE ? in_max : 3 * in_max;
  bool ok = (s->ctx = gbu_create(device, in_max)) != nullptr &&
            cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&s->din, in_max * s->in_unit + 16) == cudaSuccess &&
            (!is_transcode(op) || cudaMalloc(&s->dout, s->out_cap * s->out_unit + 16) == cudaSuccess) &&
            cudaHostAlloc((void **)&s->res_h, sizeof(gbu_result), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer((void **)&s->res_d, s->res_h, 0) == cudaSuccess &&
            cudaHostAlloc((void **)&s->len_h, sizeof(uint64_t), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer((void **)&s->len_d, s->len_h, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gbu_chunked_destroy(s);
    s = nullptr;
  }
  if (prev != device) cudaSetDevice(prev);
  return s;
}

extern "C" void gbu_chunked_destroy(gbu_chunked *s) {
  if (!s) return;
  const int prev = ensure_device(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->ctx) gbu_destroy(s->ctx);
  if (s->din) cudaFree(s->din);
  if (s->dout) cudaFree(s->dout);
  if (s->res_h) cudaFreeHost(s->res_h);
  if (s->len_h) cudaFreeHost(s->len_h);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  delete s;
}

extern "C" int gbu_chunked_reset(gbu_chunked *s) {
  if (!s) return GBU_BAD_ARGUMENT;
  s->carry_n = 0;
  s->pos = 0;
  s->produced = 0;
  s->err_status = GBU_OK;
  s->err_offset = 0;
  s->finished = false;
  return GBU_OK;
}

extern "C" int gbu_chunked_push(gbu_chunked *s, const void *chunk, uint64_t n, int last, void *out,
                                uint64_t out_cap, uint64_t *out_n, gbu_result *result) {
  if (!s || !result || !out_n || n > s->max_chunk || (n > 0 && !chunk)) return GBU_BAD_ARGUMENT;
  if (s->utf16_in && ((uintptr_t)chunk & 1)) return GBU_BAD_ARGUMENT;
  if (is_transcode(s->op) && out_cap > 0 && !out) return GBU_BAD_ARGUMENT;
  if (s->finished) return GBU_BAD_ARGUMENT;
  *out_n = 0;
  const bool transcode = is_transcode(s->op);
  if (s->err_status != GBU_OK) {  // the stream already failed: later input changes nothing
    *result = gbu_result{s->err_status, 0, s->err_offset};
    s->finished = s->finished || last;
    return GBU_OK;
  }
  const uint64_t L = s->carry_n + n;
  const uint64_t tail = last ? 0 : tail_units(s, chunk, L);
  const uint64_t M = L - tail;  // units of P judged by this push
  int rc = GBU_OK;
  gbu_result r{GBU_OK, 0, 0};
  if (M > 0) {
    const int prev = ensure_device(s->device);
    if (prev < 0) return GBU_CUDA_ERROR;
    const uint64_t from_carry = s->carry_n < M ? s->carry_n : M;
    const uint64_t from_chunk = M - from_carry;
    uint8_t *din = static_cast<uint8_t *>(s->din);
    bool ok = (from_carry == 0 || cudaMemcpyAsync(din, s->carry, from_carry * s->in_unit, cudaMemcpyHostToDevice,
                                                  s->stream) == cudaSuccess) &&
              (from_chunk == 0 || cudaMemcpyAsync(din + from_carry * s->in_unit, chunk, from_chunk * s->in_unit,
                                                  cudaMemcpyHostToDevice, s->stream) == cudaSuccess);
    if (ok) {
      switch (s->op) {
        case GBU_OP_VALIDATE_UTF8:
          rc = gbu_validate_utf8(s->ctx, din, M, s->res_d, s->stream);
          break;
        case GBU_OP_VALIDATE_UTF16LE:
          rc = gbu_validate_utf16le(s->ctx, reinterpret_cast<const uint16_t *>(din), M, s->res_d, s->stream);
          break;
        case GBU_OP_CONVERT_UTF8_TO_UTF16LE:
          rc = gbu_convert_utf8_to_utf16le(s->ctx, din, M, static_cast<uint16_t *>(s->dout), s->out_cap, s->res_d,
                                           s->stream);
          break;
        default:
          rc = gbu_convert_utf16le_to_utf8(s->ctx, reinterpret_cast<const uint16_t *>(din), M,
                                           static_cast<uint8_t *>(s->dout), s->out_cap, s->res_d, s->stream);
      }
      ok = rc == GBU_OK && cudaStreamSynchronize(s->stream) == cudaSuccess;
    }
    if (ok) r = *s->res_h;
    uint64_t units = 0;  // output units of this push to hand back
    if (ok && transcode) {
      if (r.status == GBU_OK) {
        units = r.count;
      } else if (r.status >= GBU_HEADER_BITS && r.status <= GBU_SURROGATE && r.count > 0) {
        // the valid prefix P[0:count) was transcoded: its output length
        rc = s->op == GBU_OP_CONVERT_UTF8_TO_UTF16LE
                 ? gbu_utf16_length_from_utf8(s->ctx, din, r.count, s->len_d, s->stream)
                 : gbu_utf8_length_from_utf16le(s->ctx, reinterpret_cast<const uint16_t *>(din), r.count, s->len_d,
                                                s->stream);
        ok = rc == GBU_OK && cudaStreamSynchronize(s->stream) == cudaSuccess;
        if (ok) units = *s->len_h;
      }
      if (ok && units > out_cap) {
        // the caller's buffer is too small: nothing is consumed, the push can be repeated
        if (prev != s->device) cudaSetDevice(prev);
        *result = gbu_result{GBU_OUTPUT_TOO_SMALL, 0, units};
        return GBU_OK;
      }
      if (ok && units > 0)
        ok = cudaMemcpy(out, s->dout, units * s->out_unit, cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    if (prev != s->device) cudaSetDevice(prev);
    if (!ok) {
      cudaGetLastError();
      return rc != GBU_OK ? rc : GBU_CUDA_ERROR;
    }
    if (r.status == GBU_TIMEOUT) {
      *result = r;
      return GBU_OK;
    }
    *out_n = units;
    s->produced += units;
    if (r.status >= GBU_HEADER_BITS && r.status <= GBU_SURROGATE) {
      s->err_status = r.status;
      s->err_offset = s->pos + r.count;
      s->finished = last != 0;
      *result = gbu_result{s->err_status, 0, s->err_offset};
      return GBU_OK;
    }
  }
  // keep the tail: the last `tail` units of P
  uint8_t keep[8];
  for (uint64_t i = 0; i < tail; ++i) {
    const uint32_t u = p_unit(s, chunk, M + i);
    if (s->utf16_in) {
      keep[2 * i] = (uint8_t)(u & 0xFF);
      keep[2 * i + 1] = (uint8_t)(u >> 8);
    } else {
      keep[i] = (uint8_t)u;
    }
  }
  memcpy(s->carry, keep, tail * s->in_unit);
  s->carry_n = (uint32_t)tail;
  s->pos += M;
  s->finished = last != 0;
  *result = gbu_result{GBU_OK, 0, transcode ? s->produced : s->pos};
  return GBU_OK;
}
