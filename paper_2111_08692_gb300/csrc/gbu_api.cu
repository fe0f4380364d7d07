// gbu_api.cu -- the C ABI declared in include/gbutf.h: contexts, argument checks, launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "gbu_device.cuh"
#include "gbu_internal.h"
#include "gbu_kernels.h"
#include "gbutf.h"

namespace {

// The six kernels, in the order gbu_launch_config reports them (K_COUNT is also the number of
// batched operations), then the UTF-16BE and UTF-32 kernels.
enum Kernel {
  K_V8 = 0, K_L8, K_C8, K_V16, K_L16, K_C16, K_COUNT,
  K_V16BE = K_COUNT, K_L16BE, K_C16BE, K_C8BE,
  K_V32, K_L8F32, K_L32, K_C32, K_C8T32,  // validate, UTF-8 length, UTF-32 length, 32 -> 8, 8 -> 32
  K_L16F32, K_L32F16, K_C32T16, K_C16T32,  // UTF-16 length, UTF-32 length of UTF-16, 32 -> 16, 16 -> 32
  K_ALL
};

const void *kernel_ptr(int k) {
  switch (k) {
    case K_V8: return gbu::stream_kernel_ptr(0);
    case K_L8: return gbu::stream_kernel_ptr(1);
    case K_V16: return gbu::stream_kernel_ptr(2);
    case K_L16: return gbu::stream_kernel_ptr(3);
    case K_C8: return gbu::utf8_to_utf16_kernel_ptr();
    case K_V16BE: return gbu::stream_kernel_ptr(4);
    case K_L16BE: return gbu::stream_kernel_ptr(5);
    case K_C16BE: return gbu::utf16be_to_utf8_kernel_ptr();
    case K_C8BE: return gbu::utf8_to_utf16be_kernel_ptr();
    case K_V32: return gbu::utf32_stream_kernel_ptr(0);
    case K_L8F32: return gbu::utf32_stream_kernel_ptr(1);
    case K_L32: return gbu::utf32_stream_kernel_ptr(2);
    case K_C32: return gbu::utf32_to_utf8_kernel_ptr();
    case K_C8T32: return gbu::utf8_to_utf32_kernel_ptr();
    case K_L16F32: return gbu::utf32_stream_kernel_ptr(3);
    case K_L32F16: return gbu::utf32_stream_kernel_ptr(4);
    case K_C32T16: return gbu::utf32_to_utf16_kernel_ptr();
    case K_C16T32: return gbu::utf16_to_utf32_kernel_ptr();
    default: return gbu::utf16_to_utf8_kernel_ptr();
  }
}
bool is_transcoder(int k) {
  return k == K_C8 || k == K_C16 || k == K_C16BE || k == K_C8BE || k == K_C32 || k == K_C8T32 || k == K_C32T16 ||
         k == K_C16T32;
}
size_t kernel_smem(int k) {
  if (k == K_C8) return gbu::utf8_to_utf16_smem_bytes();
  if (k == K_C16) return gbu::utf16_to_utf8_smem_bytes();
  if (k == K_C16BE) return gbu::utf16be_to_utf8_smem_bytes();
  if (k == K_C8BE) return gbu::utf8_to_utf16be_smem_bytes();
  if (k == K_C32) return gbu::utf32_to_utf8_smem_bytes();
  if (k == K_C8T32) return gbu::utf8_to_utf32_smem_bytes();
  if (k == K_C32T16) return gbu::utf32_to_utf16_smem_bytes();
  if (k == K_C16T32) return gbu::utf16_to_utf32_smem_bytes();
  return 0;
}
int kernel_threads(int k) { return is_transcoder(k) ? gbu::XT : gbu::STREAM_THREADS; }
uint32_t kernel_tile_bytes(int k) {
  return is_transcoder(k) ? gbu::PART_BYTES : gbu::stream_tile_bytes();
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

struct gbu_ctx {
  int device;
  uint64_t max_units;
  int num_sms;
  gbu::WsHeader *ws;   // device
  gbu_result *sync_res; // device, right after the header: the result slot of the *_sync calls
  uint64_t *sync_len;   // device, after sync_res: the length slot of the *_sync length calls
  uint64_t *states;    // device
  uint32_t max_states;
  uint32_t wait_limit;
  long long skip_tile;
  uint32_t early_exit;
  int blocks_per_sm[K_ALL];
  int batch_blocks_per_sm[K_COUNT][3];  // per batched mode and warps per CTA (4, 8, 16)
  int scan_blocks_per_sm;
  int seg_blocks_per_sm[2];             // several-string transcoders: 8 -> 16, 16 -> 8
  gbu_batch_config batch_cfg[K_COUNT];  // launch geometry of the batched kernels
  std::atomic<uint64_t> launches;
  uint64_t capture_start;               // launches when the current graph capture began
};

namespace {
int warps_index(int w) { return w == 4 ? 0 : (w == 16 ? 2 : 1); }
}  // namespace

static int init_workspace(gbu_ctx *c) {
  gbu::WsHeader h;
  memset(&h, 0, sizeof(h));
  h.epoch = 1;
  h.errkey = gbu::NO_ERROR;
  h.stop_tile = 0xFFFFFFFFu;
  if (cudaMemcpy(c->ws, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return GBU_CUDA_ERROR;
  if (cudaMemset(c->states, 0, (size_t)c->max_states * sizeof(uint64_t)) != cudaSuccess)
    return GBU_CUDA_ERROR;
  if (cudaDeviceSynchronize() != cudaSuccess) return GBU_CUDA_ERROR;
  return GBU_OK;
}

extern "C" gbu_ctx *gbu_create(int device, uint64_t max_units) {
  DeviceGuard g(device);
  gbu_ctx *c = new gbu_ctx();
  c->device = device;
  c->max_units = max_units;
  c->wait_limit = 1u << 22;
  c->skip_tile = -1;
  c->early_exit = 1;
  c->launches = 0;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  // scan states: one per transcoder partition of the largest input (UTF-32: 4 bytes per
  // unit), plus the extra partition UTF-8 inputs may use past their end
  uint64_t tiles = (4 * max_units + 64) / gbu::PART_BYTES + 4;
  // ... and one per tile of the u64 scan of up to max_units + 1 values
  const uint64_t scan_tiles = (max_units + 1) / gbu::scan_tile_items() + 2;
  if (scan_tiles > tiles) tiles = scan_tiles;
  if (tiles > 0xFFFFFFF0ull) {
    delete c;
    return nullptr;
  }
  c->max_states = (uint32_t)tiles;
  // the header, then the *_sync calls' result and length slots (one allocation)
  if (cudaMalloc(&c->ws, sizeof(gbu::WsHeader) + sizeof(gbu_result) + sizeof(uint64_t)) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  c->sync_res = reinterpret_cast<gbu_result *>(c->ws + 1);
  c->sync_len = reinterpret_cast<uint64_t *>(c->sync_res + 1);
  if (cudaMalloc(&c->states, (size_t)c->max_states * sizeof(uint64_t)) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return nullptr;
  }
  for (int k = 0; k < K_ALL; ++k) {
    const void *f = kernel_ptr(k);
    const size_t smem = kernel_smem(k);
    int bps = 0;
    if ((smem && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, f, kernel_threads(k), smem) != cudaSuccess ||
        bps < 1) {
      cudaFree(c->states);
      cudaFree(c->ws);
      delete c;
      return nullptr;
    }
    c->blocks_per_sm[k] = bps;
  }
  static const int kWarps[3] = {4, 8, 16};
  bool occ_ok = true;
  for (int m = 0; m < K_COUNT && occ_ok; ++m)
    for (int w = 0; w < 3 && occ_ok; ++w) {
      int bps = 0;
      occ_ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gbu::batch_kernel_ptr(m, kWarps[w]),
                                                             kWarps[w] * 32, 0) == cudaSuccess && bps >= 1;
      c->batch_blocks_per_sm[m][w] = bps;
    }
  occ_ok = occ_ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->scan_blocks_per_sm, gbu::scan_kernel_ptr(),
                                                                   gbu::scan_threads(), 0) == cudaSuccess &&
           c->scan_blocks_per_sm >= 1;
  for (int d = 0; d < 2 && occ_ok; ++d) {
    const void *f = d == 0 ? gbu::utf8_to_utf16_segments_kernel_ptr() : gbu::utf16_to_utf8_segments_kernel_ptr();
    const size_t smem = d == 0 ? gbu::utf8_to_utf16_segments_smem_bytes() : gbu::utf16_to_utf8_segments_smem_bytes();
    occ_ok = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->seg_blocks_per_sm[d], f, gbu::XT, smem) ==
                 cudaSuccess &&
             c->seg_blocks_per_sm[d] >= 1;
  }
  if (!occ_ok) {
    cudaFree(c->states);
    cudaFree(c->ws);
    delete c;
    return nullptr;
  }
  for (int m = 0; m < K_COUNT; ++m) c->batch_cfg[m] = gbu_batch_config{8, 64, 4096, 0};
  if (init_workspace(c) != GBU_OK) {
    cudaFree(c->states);
    cudaFree(c->ws);
    delete c;
    return nullptr;
  }
  return c;
}

extern "C" void gbu_destroy(gbu_ctx *c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaFree(c->states);
  cudaFree(c->ws);
  delete c;
}

extern "C" int gbu_reset(gbu_ctx *c) {
  if (!c) return GBU_BAD_ARGUMENT;
  DeviceGuard g(c->device);
  return init_workspace(c);
}

extern "C" void gbu_set_wait_limit(gbu_ctx *c, uint32_t rounds) {
  if (c) c->wait_limit = rounds ? rounds : 1;
}

extern "C" void gbu_debug_skip_publish(gbu_ctx *c, int64_t tile) {
  if (c) c->skip_tile = tile;
}

extern "C" void gbu_set_early_exit(gbu_ctx *c, int enable) {
  if (c) c->early_exit = enable ? 1u : 0u;
}

extern "C" uint64_t gbu_launch_count(const gbu_ctx *c) { return c ? c->launches.load() : 0; }

extern "C" int gbu_launch_config(const gbu_ctx *c, int32_t *out, int n) {
  if (!c || !out) return 0;
  constexpr int NV = K_COUNT + 5;
  int32_t v[NV];
  v[0] = c->num_sms;
  for (int k = 0; k < K_COUNT; ++k) v[1 + k] = c->blocks_per_sm[k];
  v[K_COUNT + 1] = gbu::STREAM_THREADS;
  v[K_COUNT + 2] = gbu::XT;
  v[K_COUNT + 3] = (int32_t)gbu::stream_tile_bytes();
  v[K_COUNT + 4] = (int32_t)gbu::PART_BYTES;
  const int m = n < NV ? n : NV;
  for (int i = 0; i < m; ++i) out[i] = v[i];
  return m;
}

// Builds the launch parameters of kernel k for an input of n code units.
static int make_params(gbu_ctx *c, int k, const void *src, uint64_t n, uint32_t unit_bytes,
                       bool extra_tail, gbu::Params *p) {
  if (!c) return GBU_BAD_ARGUMENT;
  if (n > c->max_units) return GBU_BAD_ARGUMENT;
  if (n > 0 && !src) return GBU_BAD_ARGUMENT;
  if (unit_bytes == 2 && ((uintptr_t)src & 1)) return GBU_BAD_ARGUMENT;
  if (unit_bytes == 4 && ((uintptr_t)src & 3)) return GBU_BAD_ARGUMENT;
  memset(p, 0, sizeof(*p));
  // the source rounded down to 16 bytes (32 for the UTF-8 <-> UTF-16LE / UTF-16BE transcoders,
  // whose lanes read 32 bytes at a time)
  const uintptr_t a = (uintptr_t)src;
  const uintptr_t amask = (k == K_C8 || k == K_C16 || k == K_C8BE || k == K_C16BE) ? 31 : 15;
  p->base = (const uint8_t *)(a & ~amask);
  p->off0 = (uint32_t)(a & amask);
  p->n = n;
  p->vbytes = p->off0 + n * unit_bytes;
  // UTF-8 validation looks at the three positions past the end (a cut sequence fails there)
  const uint64_t span = n == 0 ? 0 : p->vbytes + (extra_tail ? 3 : 0);
  const uint64_t tb = kernel_tile_bytes(k);
  const uint64_t ntiles = (span + tb - 1) / tb;
  if (ntiles > 0xFFFFFF00ull || (is_transcoder(k) && ntiles > c->max_states)) return GBU_BAD_ARGUMENT;
  p->ntiles = (uint32_t)ntiles;
  p->ws = c->ws;
  p->states = c->states;
  p->max_states = c->max_states;
  p->wait_limit = c->wait_limit;
  p->skip_tile = c->skip_tile;
  p->early_exit = c->early_exit;
  return GBU_OK;
}

// Read-only kernels deal warp tiles round-robin and never wait on another CTA; transcoders
// claim tiles from a ticket counter, so a tile only waits (in the look-back) on tiles that
// running CTAs already hold.  Neither needs the grid to be co-resident; the grid is sized to
// what fits on the device at once.
static int launch(gbu_ctx *c, int k, const gbu::Params &p, gbu_stream stream) {
  DeviceGuard g(c->device);
  uint64_t grid = (uint64_t)c->num_sms * (uint64_t)c->blocks_per_sm[k];
  const uint64_t useful = is_transcoder(k) ? p.ntiles
                                           : (p.ntiles + gbu::STREAM_THREADS / 32 - 1) / (gbu::STREAM_THREADS / 32);
  if (useful < grid) grid = useful;
  if (grid < 1) grid = 1;
  void *args[] = {(void *)&p};
  cudaError_t e = cudaLaunchKernel(kernel_ptr(k), dim3((unsigned)grid), dim3(kernel_threads(k)), args,
                                   kernel_smem(k), (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  c->launches.fetch_add(1);
  return GBU_OK;
}

static void set_dst(gbu::Params *p, void *dst, uint64_t cap, uint32_t out_unit_bytes) {
  const uintptr_t a = (uintptr_t)dst;
  p->dbase = (uint8_t *)(a & ~(uintptr_t)15);
  p->dshift = (uint32_t)((a & 15) / out_unit_bytes);
  p->cap = cap;
}

extern "C" int gbu_validate_utf8(gbu_ctx *c, const uint8_t *src, uint64_t n, gbu_result *result,
                                 gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_V8, src, n, 1, true, &p);
  if (rc != GBU_OK) return rc;
  if (!result) return GBU_BAD_ARGUMENT;
  p.result = result;
  return launch(c, K_V8, p, stream);
}

extern "C" int gbu_validate_utf16le(gbu_ctx *c, const uint16_t *src, uint64_t n, gbu_result *result,
                                    gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_V16, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result) return GBU_BAD_ARGUMENT;
  p.result = result;
  return launch(c, K_V16, p, stream);
}

extern "C" int gbu_utf16_length_from_utf8(gbu_ctx *c, const uint8_t *src, uint64_t n, uint64_t *len,
                                          gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_L8, src, n, 1, false, &p);
  if (rc != GBU_OK) return rc;
  if (!len) return GBU_BAD_ARGUMENT;
  p.len_out = len;
  return launch(c, K_L8, p, stream);
}

extern "C" int gbu_utf8_length_from_utf16le(gbu_ctx *c, const uint16_t *src, uint64_t n, uint64_t *len,
                                            gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_L16, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!len) return GBU_BAD_ARGUMENT;
  p.len_out = len;
  return launch(c, K_L16, p, stream);
}

extern "C" int gbu_convert_utf8_to_utf16le(gbu_ctx *c, const uint8_t *src, uint64_t n, uint16_t *dst,
                                           uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C8, src, n, 1, true, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst) || ((uintptr_t)dst & 1)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 2);
  return launch(c, K_C8, p, stream);
}

extern "C" int gbu_convert_utf16le_to_utf8(gbu_ctx *c, const uint16_t *src, uint64_t n, uint8_t *dst,
                                           uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C16, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 1);
  return launch(c, K_C16, p, stream);
}

// ---- host-synchronising forms ---------------------------------------------------------------

// Completes a *_sync call: rc is the launch status of the asynchronous call, which wrote its
// result (or, for a length, the length) into the context's slot on `stream`.  Copies the slot
// back and waits for the stream.
static gbu_result finish_sync(gbu_ctx *c, int rc, gbu_stream stream, bool length) {
  gbu_result r;
  r.status = rc;
  r.reserved = 0;
  r.count = 0;
  if (rc != GBU_OK) return r;
  DeviceGuard g(c->device);
  uint64_t len = 0;
  void *host = length ? (void *)&len : (void *)&r;
  const void *dev = length ? (const void *)c->sync_len : (const void *)c->sync_res;
  if (cudaMemcpyAsync(host, dev, length ? sizeof(len) : sizeof(r), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
          cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    r.status = GBU_CUDA_ERROR;
    r.reserved = 0;
    r.count = 0;
    return r;
  }
  if (length) {
    r.status = GBU_OK;
    r.count = len;
  }
  return r;
}

static gbu_result bad_argument_result() {
  gbu_result r;
  r.status = GBU_BAD_ARGUMENT;
  r.reserved = 0;
  r.count = 0;
  return r;
}

extern "C" gbu_result gbu_validate_utf8_sync(gbu_ctx *c, const uint8_t *src, uint64_t n, gbu_stream stream) {
  if (!c) return bad_argument_result();
  return finish_sync(c, gbu_validate_utf8(c, src, n, c->sync_res, stream), stream, false);
}

extern "C" gbu_result gbu_validate_utf16le_sync(gbu_ctx *c, const uint16_t *src, uint64_t n, gbu_stream stream) {
  if (!c) return bad_argument_result();
  return finish_sync(c, gbu_validate_utf16le(c, src, n, c->sync_res, stream), stream, false);
}

extern "C" gbu_result gbu_utf16_length_from_utf8_sync(gbu_ctx *c, const uint8_t *src, uint64_t n,
                                                      gbu_stream stream) {
  if (!c) return bad_argument_result();
  return finish_sync(c, gbu_utf16_length_from_utf8(c, src, n, c->sync_len, stream), stream, true);
}

extern "C" gbu_result gbu_utf8_length_from_utf16le_sync(gbu_ctx *c, const uint16_t *src, uint64_t n,
                                                        gbu_stream stream) {
  if (!c) return bad_argument_result();
  return finish_sync(c, gbu_utf8_length_from_utf16le(c, src, n, c->sync_len, stream), stream, true);
}

extern "C" gbu_result gbu_convert_utf8_to_utf16le_sync(gbu_ctx *c, const uint8_t *src, uint64_t n, uint16_t *dst,
                                                       uint64_t cap, gbu_stream stream) {
  if (!c) return bad_argument_result();
  return finish_sync(c, gbu_convert_utf8_to_utf16le(c, src, n, dst, cap, c->sync_res, stream), stream, false);
}

extern "C" gbu_result gbu_convert_utf16le_to_utf8_sync(gbu_ctx *c, const uint16_t *src, uint64_t n, uint8_t *dst,
                                                       uint64_t cap, gbu_stream stream) {
  if (!c) return bad_argument_result();
  return finish_sync(c, gbu_convert_utf16le_to_utf8(c, src, n, dst, cap, c->sync_res, stream), stream, false);
}

extern "C" int gbu_per_string_loop(gbu_ctx *c, int op, const void *src, const uint64_t *off, uint64_t B, void *dst,
                                   const uint64_t *dst_off, gbu_result *results, gbu_stream stream) {
  if (!c) return GBU_BAD_ARGUMENT;
  if (op < 0 || op >= K_COUNT || (B > 0 && (!off || !results))) return GBU_BAD_ARGUMENT;
  const bool xcode = op == GBU_OP_CONVERT_UTF8_TO_UTF16LE || op == GBU_OP_CONVERT_UTF16LE_TO_UTF8;
  if (xcode && B > 0 && !dst_off) return GBU_BAD_ARGUMENT;
  const uint8_t *s8 = static_cast<const uint8_t *>(src);
  const uint16_t *s16 = static_cast<const uint16_t *>(src);
  for (uint64_t i = 0; i < B; ++i) {
    const uint64_t a = off[i], n = off[i + 1] - off[i];
    int rc;
    switch (op) {
      case GBU_OP_VALIDATE_UTF8: rc = gbu_validate_utf8(c, s8 + a, n, results + i, stream); break;
      case GBU_OP_UTF16_LENGTH_FROM_UTF8:
        rc = gbu_utf16_length_from_utf8(c, s8 + a, n, reinterpret_cast<uint64_t *>(results) + i, stream);
        break;
      case GBU_OP_CONVERT_UTF8_TO_UTF16LE:
        rc = gbu_convert_utf8_to_utf16le(c, s8 + a, n, static_cast<uint16_t *>(dst) + dst_off[i],
                                         dst_off[i + 1] - dst_off[i], results + i, stream);
        break;
      case GBU_OP_VALIDATE_UTF16LE: rc = gbu_validate_utf16le(c, s16 + a, n, results + i, stream); break;
      case GBU_OP_UTF8_LENGTH_FROM_UTF16LE:
        rc = gbu_utf8_length_from_utf16le(c, s16 + a, n, reinterpret_cast<uint64_t *>(results) + i, stream);
        break;
      default:
        rc = gbu_convert_utf16le_to_utf8(c, s16 + a, n, static_cast<uint8_t *>(dst) + dst_off[i],
                                         dst_off[i + 1] - dst_off[i], results + i, stream);
        break;
    }
    if (rc != GBU_OK) return rc;
  }
  return GBU_OK;
}

// ---- UTF-32 ------------------------------------------------------------------------------

extern "C" int gbu_validate_utf32(gbu_ctx *c, const uint32_t *src, uint64_t n, gbu_result *result,
                                  gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_V32, src, n, 4, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result) return GBU_BAD_ARGUMENT;
  p.result = result;
  return launch(c, K_V32, p, stream);
}

extern "C" int gbu_utf8_length_from_utf32(gbu_ctx *c, const uint32_t *src, uint64_t n, uint64_t *len,
                                          gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_L8F32, src, n, 4, false, &p);
  if (rc != GBU_OK) return rc;
  if (!len) return GBU_BAD_ARGUMENT;
  p.len_out = len;
  return launch(c, K_L8F32, p, stream);
}

extern "C" int gbu_utf32_length_from_utf8(gbu_ctx *c, const uint8_t *src, uint64_t n, uint64_t *len,
                                          gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_L32, src, n, 1, false, &p);
  if (rc != GBU_OK) return rc;
  if (!len) return GBU_BAD_ARGUMENT;
  p.len_out = len;
  return launch(c, K_L32, p, stream);
}

extern "C" int gbu_convert_utf32_to_utf8(gbu_ctx *c, const uint32_t *src, uint64_t n, uint8_t *dst,
                                         uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C32, src, n, 4, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 1);
  return launch(c, K_C32, p, stream);
}

extern "C" int gbu_convert_utf8_to_utf32(gbu_ctx *c, const uint8_t *src, uint64_t n, uint32_t *dst,
                                         uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C8T32, src, n, 1, true, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst) || ((uintptr_t)dst & 3)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 4);
  return launch(c, K_C8T32, p, stream);
}

extern "C" int gbu_utf16_length_from_utf32(gbu_ctx *c, const uint32_t *src, uint64_t n, uint64_t *len,
                                           gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_L16F32, src, n, 4, false, &p);
  if (rc != GBU_OK) return rc;
  if (!len) return GBU_BAD_ARGUMENT;
  p.len_out = len;
  return launch(c, K_L16F32, p, stream);
}

extern "C" int gbu_utf32_length_from_utf16le(gbu_ctx *c, const uint16_t *src, uint64_t n, uint64_t *len,
                                             gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_L32F16, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!len) return GBU_BAD_ARGUMENT;
  p.len_out = len;
  return launch(c, K_L32F16, p, stream);
}

extern "C" int gbu_convert_utf32_to_utf16le(gbu_ctx *c, const uint32_t *src, uint64_t n, uint16_t *dst,
                                            uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C32T16, src, n, 4, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst) || ((uintptr_t)dst & 1)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 2);
  return launch(c, K_C32T16, p, stream);
}

extern "C" int gbu_convert_utf16le_to_utf32(gbu_ctx *c, const uint16_t *src, uint64_t n, uint32_t *dst,
                                            uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C16T32, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst) || ((uintptr_t)dst & 3)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 4);
  return launch(c, K_C16T32, p, stream);
}

// ---- UTF-16BE ----------------------------------------------------------------------------

extern "C" int gbu_validate_utf16be(gbu_ctx *c, const uint16_t *src, uint64_t n, gbu_result *result,
                                    gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_V16BE, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result) return GBU_BAD_ARGUMENT;
  p.result = result;
  return launch(c, K_V16BE, p, stream);
}

extern "C" int gbu_utf8_length_from_utf16be(gbu_ctx *c, const uint16_t *src, uint64_t n, uint64_t *len,
                                            gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_L16BE, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!len) return GBU_BAD_ARGUMENT;
  p.len_out = len;
  return launch(c, K_L16BE, p, stream);
}

extern "C" int gbu_convert_utf16be_to_utf8(gbu_ctx *c, const uint16_t *src, uint64_t n, uint8_t *dst,
                                           uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C16BE, src, n, 2, false, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 1);
  return launch(c, K_C16BE, p, stream);
}

extern "C" int gbu_convert_utf8_to_utf16be(gbu_ctx *c, const uint8_t *src, uint64_t n, uint16_t *dst,
                                           uint64_t cap, gbu_result *result, gbu_stream stream) {
  gbu::Params p;
  int rc = make_params(c, K_C8BE, src, n, 1, true, &p);
  if (rc != GBU_OK) return rc;
  if (!result || (cap > 0 && !dst) || ((uintptr_t)dst & 1)) return GBU_BAD_ARGUMENT;
  p.result = result;
  set_dst(&p, dst, cap, 2);
  return launch(c, K_C8BE, p, stream);
}

// ---- batched forms -----------------------------------------------------------------------

static int batch_check_config(const gbu_batch_config &b) {
  if (b.warps_per_cta != 4 && b.warps_per_cta != 8 && b.warps_per_cta != 16) return GBU_BAD_ARGUMENT;
  if (b.strings_per_claim < 1 || b.strings_per_claim > 1024) return GBU_BAD_ARGUMENT;
  if (b.long_bytes < 512) return GBU_BAD_ARGUMENT;  // at least one 512-byte warp region
  return GBU_OK;
}

// Launches batched mode m over B strings with geometry cfg.
static int batch_launch(gbu_ctx *c, int m, const gbu_batch_config &cfg, const void *src, const uint64_t *off,
                        uint64_t B, void *dst, const uint64_t *dst_off, gbu_result *results, uint64_t *lens,
                        gbu_stream stream, const gbu::StringDesc *desc = nullptr) {
  if (B == 0) return GBU_OK;  // nothing to write
  gbu::BatchParams bp;
  memset(&bp, 0, sizeof(bp));
  bp.desc = desc;
  bp.src = (const uint8_t *)src;
  bp.off = off;
  bp.B = B;
  bp.dst = (uint8_t *)dst;
  bp.dst_off = dst_off;
  bp.results = results;
  bp.lens = lens;
  bp.ws = c->ws;
  bp.grab = cfg.strings_per_claim;
  bp.long_bytes = cfg.long_bytes;
  DeviceGuard g(c->device);
  uint64_t grid = (uint64_t)c->num_sms * (uint64_t)c->batch_blocks_per_sm[m][warps_index(cfg.warps_per_cta)];
  const uint64_t claims = (B + cfg.strings_per_claim - 1) / cfg.strings_per_claim;
  if (claims < grid) grid = claims;
  if (grid < 1) grid = 1;
  void *args[] = {(void *)&bp};
  cudaError_t e = cudaLaunchKernel(gbu::batch_kernel_ptr(m, cfg.warps_per_cta), dim3((unsigned)grid),
                                   dim3(cfg.warps_per_cta * 32), args, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  c->launches.fetch_add(1);
  return GBU_OK;
}

// Argument checks shared by the batched calls.
static int batch_args(gbu_ctx *c, int m, const void *src, const uint64_t *off, uint64_t B, const void *dst,
                      const uint64_t *dst_off, const void *out) {
  if (!c || m < 0 || m >= K_COUNT) return GBU_BAD_ARGUMENT;
  if (B == 0) return GBU_OK;
  if (!src || !off || !out) return GBU_BAD_ARGUMENT;
  const bool utf16_in = m >= K_V16;
  if (utf16_in && ((uintptr_t)src & 1)) return GBU_BAD_ARGUMENT;
  if (is_transcoder(m)) {
    if (!dst || !dst_off) return GBU_BAD_ARGUMENT;
    if (m == K_C8 && ((uintptr_t)dst & 1)) return GBU_BAD_ARGUMENT;
  }
  if (((uintptr_t)off & 7) || ((uintptr_t)dst_off & 7) || ((uintptr_t)out & 7)) return GBU_BAD_ARGUMENT;
  return GBU_OK;
}

static int batch_call(gbu_ctx *c, int m, const void *src, const uint64_t *off, uint64_t B, void *dst,
                      const uint64_t *dst_off, void *out, gbu_stream stream) {
  int rc = batch_args(c, m, src, off, B, dst, dst_off, out);
  if (rc != GBU_OK) return rc;
  const bool length = m == K_L8 || m == K_L16;
  return batch_launch(c, m, c->batch_cfg[m], src, off, B, dst, dst_off, length ? nullptr : (gbu_result *)out,
                      length ? (uint64_t *)out : nullptr, stream);
}

extern "C" int gbu_validate_utf8_batched(gbu_ctx *c, const uint8_t *src, const uint64_t *off, uint64_t B,
                                         gbu_result *results, gbu_stream stream) {
  return batch_call(c, K_V8, src, off, B, nullptr, nullptr, results, stream);
}

extern "C" int gbu_validate_utf16le_batched(gbu_ctx *c, const uint16_t *src, const uint64_t *off, uint64_t B,
                                            gbu_result *results, gbu_stream stream) {
  return batch_call(c, K_V16, src, off, B, nullptr, nullptr, results, stream);
}

extern "C" int gbu_utf16_length_from_utf8_batched(gbu_ctx *c, const uint8_t *src, const uint64_t *off,
                                                  uint64_t B, uint64_t *lens, gbu_stream stream) {
  return batch_call(c, K_L8, src, off, B, nullptr, nullptr, lens, stream);
}

extern "C" int gbu_utf8_length_from_utf16le_batched(gbu_ctx *c, const uint16_t *src, const uint64_t *off,
                                                    uint64_t B, uint64_t *lens, gbu_stream stream) {
  return batch_call(c, K_L16, src, off, B, nullptr, nullptr, lens, stream);
}

extern "C" int gbu_convert_utf8_to_utf16le_batched(gbu_ctx *c, const uint8_t *src, const uint64_t *off,
                                                   uint64_t B, uint16_t *dst, const uint64_t *dst_off,
                                                   gbu_result *results, gbu_stream stream) {
  return batch_call(c, K_C8, src, off, B, dst, dst_off, results, stream);
}

extern "C" int gbu_convert_utf16le_to_utf8_batched(gbu_ctx *c, const uint16_t *src, const uint64_t *off,
                                                   uint64_t B, uint8_t *dst, const uint64_t *dst_off,
                                                   gbu_result *results, gbu_stream stream) {
  return batch_call(c, K_C16, src, off, B, dst, dst_off, results, stream);
}

extern "C" int gbu_exclusive_scan_u64(gbu_ctx *c, const uint64_t *in, uint64_t count, uint64_t *out,
                                      gbu_result *result, gbu_stream stream) {
  if (!c || !out || !result || (count > 0 && !in)) return GBU_BAD_ARGUMENT;
  if (((uintptr_t)in & 7) || ((uintptr_t)out & 7)) return GBU_BAD_ARGUMENT;
  const uint64_t tile = gbu::scan_tile_items();
  const uint64_t ntiles = (count + 1 + tile - 1) / tile;
  if (ntiles > c->max_states) return GBU_BAD_ARGUMENT;
  gbu::ScanParams sp;
  memset(&sp, 0, sizeof(sp));
  sp.in = in;
  sp.out = out;
  sp.count = count;
  sp.result = result;
  sp.lb.ntiles = (uint32_t)ntiles;
  sp.lb.ws = c->ws;
  sp.lb.states = c->states;
  sp.lb.max_states = c->max_states;
  sp.lb.wait_limit = c->wait_limit;
  sp.lb.skip_tile = c->skip_tile;
  DeviceGuard g(c->device);
  uint64_t grid = (uint64_t)c->num_sms * (uint64_t)c->scan_blocks_per_sm;
  if (ntiles < grid) grid = ntiles;
  void *args[] = {(void *)&sp};
  cudaError_t e = cudaLaunchKernel(gbu::scan_kernel_ptr(), dim3((unsigned)grid), dim3(gbu::scan_threads()),
                                   args, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  c->launches.fetch_add(1);
  return GBU_OK;
}

extern "C" int gbu_get_batch_config(const gbu_ctx *c, int op, gbu_batch_config *cfg) {
  if (!c || !cfg || op < 0 || op >= K_COUNT) return GBU_BAD_ARGUMENT;
  *cfg = c->batch_cfg[op];
  return GBU_OK;
}

extern "C" int gbu_set_batch_config(gbu_ctx *c, int op, const gbu_batch_config *cfg) {
  if (!c || !cfg || op < 0 || op >= K_COUNT) return GBU_BAD_ARGUMENT;
  const int rc = batch_check_config(*cfg);
  if (rc != GBU_OK) return rc;
  c->batch_cfg[op] = *cfg;
  return GBU_OK;
}

// Times every candidate geometry on the caller's batch (one untimed launch, then the best of
// `reps` timed launches each) and keeps the fastest in the context.  The last launch uses the
// chosen geometry, so the outputs are those of a normal call.  Synchronous.
extern "C" int gbu_tune_batched(gbu_ctx *c, int op, const void *src, const uint64_t *off, uint64_t B, void *dst,
                                const uint64_t *dst_off, void *out, int reps, gbu_stream stream,
                                gbu_batch_config *chosen) {
  int rc = batch_args(c, op, src, off, B, dst, dst_off, out);
  if (rc != GBU_OK) return rc;
  if (reps < 1) reps = 1;
  DeviceGuard g(c->device);
  const bool length = op == K_L8 || op == K_L16;
  gbu_result *results = length ? nullptr : (gbu_result *)out;
  uint64_t *lens = length ? (uint64_t *)out : nullptr;
  static const int kWarps[3] = {4, 8, 16};
  static const uint32_t kGrab[4] = {8, 32, 128, 512};
  static const uint32_t kLong[4] = {2048, 4096, 8192, 16384};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GBU_CUDA_ERROR;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GBU_CUDA_ERROR;
  }
  gbu_batch_config best = c->batch_cfg[op];
  float best_ms = -1.0f;
  rc = GBU_OK;
  for (int w = 0; w < 3 && rc == GBU_OK; ++w)
    for (int gi = 0; gi < 4 && rc == GBU_OK; ++gi)
      for (int li = 0; li < 4 && rc == GBU_OK; ++li) {
        const gbu_batch_config cand{kWarps[w], kGrab[gi], kLong[li], 0.0f};
        rc = batch_launch(c, op, cand, src, off, B, dst, dst_off, results, lens, stream);
        float t_best = -1.0f;
        for (int r = 0; r < reps && rc == GBU_OK; ++r) {
          if (cudaEventRecord(e0, (cudaStream_t)stream) != cudaSuccess) rc = GBU_CUDA_ERROR;
          if (rc == GBU_OK) rc = batch_launch(c, op, cand, src, off, B, dst, dst_off, results, lens, stream);
          if (rc == GBU_OK && cudaEventRecord(e1, (cudaStream_t)stream) != cudaSuccess) rc = GBU_CUDA_ERROR;
          float ms = 0.0f;
          if (rc == GBU_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = GBU_CUDA_ERROR;
          if (rc == GBU_OK && (t_best < 0.0f || ms < t_best)) t_best = ms;
        }
        if (rc == GBU_OK && (best_ms < 0.0f || t_best < best_ms)) {
          best_ms = t_best;
          best = cand;
        }
      }
  if (rc == GBU_OK) {
    best.tuned_ms = best_ms;
    c->batch_cfg[op] = best;
    rc = batch_launch(c, op, best, src, off, B, dst, dst_off, results, lens, stream);
    if (rc == GBU_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = GBU_CUDA_ERROR;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == GBU_OK && chosen) *chosen = best;
  return rc;
}

// ---- CUDA graphs ---------------------------------------------------------------------------

struct gbu_graph {
  int device;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  uint64_t kernels;  // library launches captured into the graph
  gbu_ctx *ctx;
};

extern "C" int gbu_graph_begin(gbu_ctx *c, gbu_stream stream) {
  if (!c || !stream) return GBU_BAD_ARGUMENT;  // the legacy default stream cannot be captured
  DeviceGuard g(c->device);
  if (cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  c->capture_start = c->launches.load();
  return GBU_OK;
}

extern "C" gbu_graph *gbu_graph_end(gbu_ctx *c, gbu_stream stream) {
  if (!c || !stream) return nullptr;
  DeviceGuard g(c->device);
  cudaGraph_t graph = nullptr;
  if (cudaStreamEndCapture((cudaStream_t)stream, &graph) != cudaSuccess || !graph) {
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return nullptr;
  }
  gbu_graph *gr = new gbu_graph{c->device, graph, exec, c->launches.load() - c->capture_start, c};
  // captured launches did not run: they are counted when the graph is launched
  c->launches.fetch_sub(gr->kernels);
  return gr;
}

extern "C" int gbu_graph_launch(gbu_graph *gr, gbu_stream stream) {
  if (!gr) return GBU_BAD_ARGUMENT;
  DeviceGuard g(gr->device);
  if (cudaGraphLaunch(gr->exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  gr->ctx->launches.fetch_add(gr->kernels);
  return GBU_OK;
}

extern "C" uint64_t gbu_graph_kernels(const gbu_graph *gr) { return gr ? gr->kernels : 0; }

extern "C" void gbu_graph_destroy(gbu_graph *gr) {
  if (!gr) return;
  DeviceGuard g(gr->device);
  cudaGraphExecDestroy(gr->exec);
  cudaGraphDestroy(gr->graph);
  delete gr;
}

// ---- library-internal entry points (gbu_internal.h) ---------------------------------------

int gbu_internal_device(const gbu_ctx *c) { return c->device; }
void gbu_internal_count_launch(gbu_ctx *c) { c->launches.fetch_add(1); }

int gbu_internal_batch_desc(gbu_ctx *c, int op, const gbu::StringDesc *desc, uint64_t B, gbu_result *results,
                            gbu_stream stream) {
  if (!c || op < 0 || op >= K_COUNT || op == K_L8 || op == K_L16) return GBU_BAD_ARGUMENT;
  if (B > 0 && (!desc || !results)) return GBU_BAD_ARGUMENT;
  return batch_launch(c, op, c->batch_cfg[op], nullptr, nullptr, B, nullptr, nullptr, results, nullptr, stream,
                      desc);
}

int gbu_internal_partitions(int op, const void *src, uint64_t n) {
  const uint64_t in_unit = op == GBU_OP_CONVERT_UTF16LE_TO_UTF8 ? 2 : 1;
  const uint64_t tail = op == GBU_OP_CONVERT_UTF8_TO_UTF16LE ? 3 : 0;  // positions judged past the end
  const uint64_t span = ((uintptr_t)src & 15) + n * in_unit + tail;
  return (int)((span + gbu::PART_BYTES - 1) / gbu::PART_BYTES);
}

int gbu_internal_convert_segments(gbu_ctx *c, int op, const gbu::StringDesc *desc, const uint32_t *pstart,
                                  uint32_t B, uint32_t ntiles, gbu::SegState *seg, gbu_result *results,
                                  gbu_stream stream) {
  if (!c || (op != K_C8 && op != K_C16)) return GBU_BAD_ARGUMENT;
  if (B == 0 || ntiles == 0) return GBU_OK;
  if (!desc || !pstart || !seg || !results || ntiles > c->max_states) return GBU_BAD_ARGUMENT;
  gbu::SegParams q;
  memset(&q, 0, sizeof(q));
  q.desc = desc;
  q.pstart = pstart;
  q.B = B;
  q.ntiles = ntiles;
  q.seg = seg;
  q.results = results;
  q.ws = c->ws;
  q.states = c->states;
  q.max_states = c->max_states;
  q.wait_limit = c->wait_limit;
  const int d = op == K_C8 ? 0 : 1;
  DeviceGuard g(c->device);
  uint64_t grid = (uint64_t)c->num_sms * (uint64_t)c->seg_blocks_per_sm[d];
  if (ntiles < grid) grid = ntiles;
  void *args[] = {(void *)&q};
  cudaError_t e = cudaLaunchKernel(
      d == 0 ? gbu::utf8_to_utf16_segments_kernel_ptr() : gbu::utf16_to_utf8_segments_kernel_ptr(), dim3((unsigned)grid),
      dim3(gbu::XT), args, d == 0 ? gbu::utf8_to_utf16_segments_smem_bytes() : gbu::utf16_to_utf8_segments_smem_bytes(),
      (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  c->launches.fetch_add(1);
  return GBU_OK;
}
