// gbu_pipe.cu -- the host-buffer form: the six single-buffer operations on host memory, one
// synchronous call each, pipelined over the device.
//
// The input is cut into pieces at character starts; piece i runs in lane i mod S: a copy of
// its units to the device (on the lane's copy stream), the single-buffer call (its own context
// per lane) and a copy of the call's result word back (on the lane's stream).  The host retires
// pieces in order: it waits for piece i's result, queues the copy of its output to the right
// place of dst (the sum of the earlier pieces' lengths, known by then), and queues piece i + S
// in the same lane: its input copy waits only for piece i's kernel, its kernel for piece i's
// output copy.  While the host waits for one piece, the copy engines and the SMs work on the
// next ones.  The first piece with an input error decides the result,
// with its offset moved by the piece's start (pieces start at character starts, so a sequence
// that a cut meets is judged whole in the piece that holds its leading byte).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "gbutf.h"

namespace {

enum PipeOp { P_V8, P_V16, P_L16, P_L8, P_C8, P_C16 };

struct Lane {
  cudaStream_t stream = nullptr;     // the piece's kernel, result copy and output copy
  cudaStream_t in_stream = nullptr;  // the piece's input copy
  cudaEvent_t in_ready = nullptr;    // the input copy has landed
  cudaEvent_t kernel_done = nullptr; // the kernel has read din (the next input copy may start)
  cudaEvent_t done = nullptr;  // the piece's result word has reached host memory
  gbu_ctx *ctx = nullptr;
  uint8_t *din = nullptr;      // the piece's input (up to 2 x piece bytes)
  uint8_t *dout = nullptr;     // its output (up to 3 x piece + 64 bytes)
  gbu_result *dres = nullptr;  // device result word (a length is written into count)
  gbu_result *hres = nullptr;  // pinned host copy of it
  uint64_t start = 0, len = 0;  // the piece now in this lane: first unit, units
};

bool is16(PipeOp op) { return op == P_V16 || op == P_L8 || op == P_C16; }

// End of the piece that starts at `start` (units): start + piece, moved back to a character
// start.  UTF-8: back past continuation bytes (at most three; an input with a longer run is
// invalid there, and the cut stays at the nominal end).  UTF-16: back off a second surrogate
// that follows a first one.
uint64_t piece_end(const void *src, uint64_t n, uint64_t start, uint64_t piece, bool u16) {
  uint64_t e = start + piece;
  if (e >= n) return n;
  if (u16) {
    const uint16_t *s = static_cast<const uint16_t *>(src);
    if (s[e] >= 0xDC00 && s[e] <= 0xDFFF && s[e - 1] >= 0xD800 && s[e - 1] <= 0xDBFF) --e;
    return e;
  }
  const uint8_t *s = static_cast<const uint8_t *>(src);
  for (int k = 0; k < 3 && e > start + 1 && (s[e] & 0xC0) == 0x80; ++k) --e;
  if ((s[e] & 0xC0) == 0x80) e = start + piece;  // not a valid run: keep the nominal cut
  return e;
}

}  // namespace

struct gbu_pipe {
  int device;
  uint64_t piece;
  std::vector<Lane> lanes;
};

namespace {

void destroy_lanes(gbu_pipe *p) {
  for (Lane &l : p->lanes) {
    if (l.done) cudaEventDestroy(l.done);
    if (l.in_ready) cudaEventDestroy(l.in_ready);
    if (l.kernel_done) cudaEventDestroy(l.kernel_done);
    if (l.stream) cudaStreamDestroy(l.stream);
    if (l.in_stream) cudaStreamDestroy(l.in_stream);
    if (l.ctx) gbu_destroy(l.ctx);
    if (l.din) cudaFree(l.din);
    if (l.dout) cudaFree(l.dout);
    if (l.dres) cudaFree(l.dres);
    if (l.hres) cudaFreeHost(l.hres);
  }
  p->lanes.clear();
}

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" gbu_pipe *gbu_pipe_create(int device, uint64_t piece_units, int streams) {
  if (piece_units == 0) piece_units = 64ull << 20;
  if (streams == 0) streams = 3;
  if (piece_units < 4096 || piece_units > (1ull << 32) || streams < 1 || streams > 8) return nullptr;
  DeviceScope scope(device);
  gbu_pipe *p = new gbu_pipe();
  p->device = device;
  p->piece = piece_units;
  p->lanes.resize((size_t)streams);
  bool ok = true;
  for (Lane &l : p->lanes) {
    ok = ok && cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&l.in_stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&l.in_ready, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&l.kernel_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaMalloc(&l.din, 2 * piece_units) == cudaSuccess &&
         cudaMalloc(&l.dout, 3 * piece_units + 64) == cudaSuccess &&
         cudaMalloc(&l.dres, sizeof(gbu_result)) == cudaSuccess &&
         cudaHostAlloc(&l.hres, sizeof(gbu_result), cudaHostAllocDefault) == cudaSuccess;
    if (ok) ok = (l.ctx = gbu_create(device, piece_units)) != nullptr;
    if (!ok) break;
  }
  if (!ok) {
    cudaGetLastError();
    destroy_lanes(p);
    delete p;
    return nullptr;
  }
  return p;
}

extern "C" void gbu_pipe_destroy(gbu_pipe *p) {
  if (!p) return;
  DeviceScope scope(p->device);
  for (Lane &l : p->lanes) {
    if (l.stream) cudaStreamSynchronize(l.stream);
    if (l.in_stream) cudaStreamSynchronize(l.in_stream);
  }
  destroy_lanes(p);
  delete p;
}

namespace {

// The piece now in lane l: its input copy on the lane's copy stream, once the lane's previous
// kernel has read din (so input copies run ahead of the output copies the host queues later on
// the lane's stream), then the single-buffer call, the kernel_done event, the result copy and
// the done event on the lane's stream.
int enqueue_piece(PipeOp op, Lane &l, const void *src, uint64_t start, uint64_t len) {
  const uint64_t ub = is16(op) ? 2 : 1;
  l.start = start;
  l.len = len;
  if (cudaStreamWaitEvent(l.in_stream, l.kernel_done, 0) != cudaSuccess ||
      cudaMemcpyAsync(l.din, static_cast<const uint8_t *>(src) + start * ub, len * ub, cudaMemcpyHostToDevice,
                      l.in_stream) != cudaSuccess ||
      cudaEventRecord(l.in_ready, l.in_stream) != cudaSuccess ||
      cudaStreamWaitEvent(l.stream, l.in_ready, 0) != cudaSuccess)
    return GBU_CUDA_ERROR;
  int rc = GBU_OK;
  switch (op) {
    case P_V8: rc = gbu_validate_utf8(l.ctx, l.din, len, l.dres, l.stream); break;
    case P_V16:
      rc = gbu_validate_utf16le(l.ctx, reinterpret_cast<const uint16_t *>(l.din), len, l.dres, l.stream);
      break;
    case P_L16: rc = gbu_utf16_length_from_utf8(l.ctx, l.din, len, &l.dres->count, l.stream); break;
    case P_L8:
      rc = gbu_utf8_length_from_utf16le(l.ctx, reinterpret_cast<const uint16_t *>(l.din), len, &l.dres->count,
                                        l.stream);
      break;
    case P_C8:  // at most one word per byte
      rc = gbu_convert_utf8_to_utf16le(l.ctx, l.din, len, reinterpret_cast<uint16_t *>(l.dout), len, l.dres,
                                       l.stream);
      break;
    case P_C16:  // at most three bytes per word
      rc = gbu_convert_utf16le_to_utf8(l.ctx, reinterpret_cast<const uint16_t *>(l.din), len, l.dout, 3 * len,
                                       l.dres, l.stream);
      break;
  }
  if (rc != GBU_OK) return rc;
  if (cudaEventRecord(l.kernel_done, l.stream) != cudaSuccess ||
      cudaMemcpyAsync(l.hres, l.dres, sizeof(gbu_result), cudaMemcpyDeviceToHost, l.stream) != cudaSuccess ||
      cudaEventRecord(l.done, l.stream) != cudaSuccess)
    return GBU_CUDA_ERROR;
  return GBU_OK;
}

// Output units of the valid prefix of the piece in lane l (its first `units` input units),
// counted on the device from the piece's input, which is still resident.
int prefix_length(PipeOp op, Lane &l, uint64_t units, uint64_t *out) {
  int rc = op == P_C8 ? gbu_utf16_length_from_utf8(l.ctx, l.din, units, &l.dres->count, l.stream)
                      : gbu_utf8_length_from_utf16le(l.ctx, reinterpret_cast<const uint16_t *>(l.din), units,
                                                     &l.dres->count, l.stream);
  if (rc != GBU_OK) return rc;
  if (cudaMemcpyAsync(l.hres, l.dres, sizeof(gbu_result), cudaMemcpyDeviceToHost, l.stream) != cudaSuccess ||
      cudaStreamSynchronize(l.stream) != cudaSuccess)
    return GBU_CUDA_ERROR;
  *out = l.hres->count;
  return GBU_OK;
}

// Output units [from, from + units) of the piece in lane l to dst + off, clipped to cap.
int copy_out(PipeOp op, Lane &l, void *dst, uint64_t off, uint64_t units, uint64_t cap) {
  if (off >= cap) return GBU_OK;
  if (units > cap - off) units = cap - off;
  if (units == 0) return GBU_OK;
  const uint64_t ub = op == P_C8 ? 2 : 1;
  return cudaMemcpyAsync(static_cast<uint8_t *>(dst) + off * ub, l.dout, units * ub, cudaMemcpyDeviceToHost,
                         l.stream) == cudaSuccess
             ? GBU_OK
             : GBU_CUDA_ERROR;
}

int run(gbu_pipe *p, PipeOp op, const void *src, uint64_t n, void *dst, uint64_t cap, gbu_result *result) {
  const bool xcode = op == P_C8 || op == P_C16, u16 = is16(op);
  if (!p || !result || (n > 0 && !src)) return GBU_BAD_ARGUMENT;
  if (u16 && ((uintptr_t)src & 1)) return GBU_BAD_ARGUMENT;
  if (xcode && ((cap > 0 && !dst) || (op == P_C8 && ((uintptr_t)dst & 1)))) return GBU_BAD_ARGUMENT;
  DeviceScope scope(p->device);
  const size_t S = p->lanes.size();
  for (Lane &l : p->lanes) l.len = ~0ull;  // ~0: no piece in flight
  gbu_result res = {GBU_OK, 0, 0};
  uint64_t next = 0, total = 0;  // next piece's first unit; output units (or length) so far
  int rc = GBU_OK;
  bool stop = false;
  auto refill = [&](Lane &l) {
    if (rc != GBU_OK || stop || next >= n) return;
    const uint64_t e = piece_end(src, n, next, p->piece, u16);
    rc = enqueue_piece(op, l, src, next, e - next);
    next = e;
  };
  for (Lane &l : p->lanes) refill(l);
  for (size_t li = 0; rc == GBU_OK && !stop && p->lanes[li].len != ~0ull; li = (li + 1) % S) {
    Lane &l = p->lanes[li];
    if (cudaEventSynchronize(l.done) != cudaSuccess) {
      rc = GBU_CUDA_ERROR;
      break;
    }
    const gbu_result r = *l.hres;
    if (op == P_L16 || op == P_L8) {
      total += r.count;
    } else if (r.status == GBU_OK) {
      if (xcode) rc = copy_out(op, l, dst, total, r.count, cap);
      total += xcode ? r.count : l.len;
    } else {  // the first piece with an input error (or a device wait that gave up) decides
      stop = true;
      if (r.status == GBU_TIMEOUT) {
        res = {GBU_TIMEOUT, 0, 0};
        rc = gbu_reset(l.ctx);
        break;
      }
      res = {r.status, 0, l.start + r.count};
      if (xcode) {
        uint64_t plen = 0;
        rc = prefix_length(op, l, r.count, &plen);
        if (rc == GBU_OK) rc = copy_out(op, l, dst, total, plen, cap);
      }
      break;
    }
    l.len = ~0ull;
    refill(l);
  }
  // every piece still in flight ends before the call returns (the caller's buffers are free)
  for (Lane &l : p->lanes)
    if (cudaStreamSynchronize(l.in_stream) != cudaSuccess || cudaStreamSynchronize(l.stream) != cudaSuccess)
      rc = GBU_CUDA_ERROR;
  if (rc != GBU_OK) {
    cudaGetLastError();
    return rc;
  }
  if (!stop) res = {xcode && total > cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, 0, total};
  *result = res;
  return GBU_OK;
}

}  // namespace

extern "C" int gbu_pipe_validate_utf8(gbu_pipe *p, const uint8_t *src, uint64_t n, gbu_result *result) {
  return run(p, P_V8, src, n, nullptr, 0, result);
}
extern "C" int gbu_pipe_validate_utf16le(gbu_pipe *p, const uint16_t *src, uint64_t n, gbu_result *result) {
  return run(p, P_V16, src, n, nullptr, 0, result);
}
extern "C" int gbu_pipe_utf16_length_from_utf8(gbu_pipe *p, const uint8_t *src, uint64_t n, gbu_result *result) {
  return run(p, P_L16, src, n, nullptr, 0, result);
}
extern "C" int gbu_pipe_utf8_length_from_utf16le(gbu_pipe *p, const uint16_t *src, uint64_t n, gbu_result *result) {
  return run(p, P_L8, src, n, nullptr, 0, result);
}
extern "C" int gbu_pipe_convert_utf8_to_utf16le(gbu_pipe *p, const uint8_t *src, uint64_t n, uint16_t *dst,
                                                uint64_t cap, gbu_result *result) {
  return run(p, P_C8, src, n, dst, cap, result);
}
extern "C" int gbu_pipe_convert_utf16le_to_utf8(gbu_pipe *p, const uint16_t *src, uint64_t n, uint8_t *dst,
                                                uint64_t cap, gbu_result *result) {
  return run(p, P_C16, src, n, dst, cap, result);
}
