// gbu_api.cu -- the C ABI declared in include/gbutf.h: contexts, argument checks, launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "gbu_device.cuh"
#include "gbu_kernels.h"
#include "gbutf.h"

namespace {

// The six kernels, in the order gbu_launch_config reports them.
enum Kernel { K_V8 = 0, K_L8, K_C8, K_V16, K_L16, K_C16, K_COUNT };

const void *kernel_ptr(int k) {
  switch (k) {
    case K_V8: return gbu::stream_kernel_ptr(0);
    case K_L8: return gbu::stream_kernel_ptr(1);
    case K_V16: return gbu::stream_kernel_ptr(2);
    case K_L16: return gbu::stream_kernel_ptr(3);
    case K_C8: return gbu::utf8_to_utf16_kernel_ptr();
    default: return gbu::utf16_to_utf8_kernel_ptr();
  }
}
bool is_transcoder(int k) { return k == K_C8 || k == K_C16; }
size_t kernel_smem(int) { return 0; }
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
  uint64_t *states;    // device
  uint32_t max_states;
  uint32_t wait_limit;
  long long skip_tile;
  int blocks_per_sm[K_COUNT];
  std::atomic<uint64_t> launches;
};

static int init_workspace(gbu_ctx *c) {
  gbu::WsHeader h;
  memset(&h, 0, sizeof(h));
  h.epoch = 1;
  h.errkey = gbu::NO_ERROR;
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
  c->launches = 0;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  // scan states: one per transcoder partition of the largest input (UTF-16: 2 bytes per
  // unit), plus the extra partition UTF-8 inputs may use past their end
  const uint64_t tiles = (2 * max_units + 64) / gbu::PART_BYTES + 4;
  if (tiles > 0xFFFFFFF0ull) {
    delete c;
    return nullptr;
  }
  c->max_states = (uint32_t)tiles;
  if (cudaMalloc(&c->ws, sizeof(gbu::WsHeader)) != cudaSuccess) {
    delete c;
    return nullptr;
  }
  if (cudaMalloc(&c->states, (size_t)c->max_states * sizeof(uint64_t)) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return nullptr;
  }
  for (int k = 0; k < K_COUNT; ++k) {
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

extern "C" uint64_t gbu_launch_count(const gbu_ctx *c) { return c ? c->launches.load() : 0; }

extern "C" int gbu_launch_config(const gbu_ctx *c, int32_t *out, int n) {
  if (!c || !out) return 0;
  int32_t v[K_COUNT + 3];
  v[0] = c->num_sms;
  for (int k = 0; k < K_COUNT; ++k) v[1 + k] = c->blocks_per_sm[k];
  v[K_COUNT + 1] = gbu::STREAM_THREADS;
  v[K_COUNT + 2] = gbu::XT;
  const int m = n < K_COUNT + 3 ? n : K_COUNT + 3;
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
  memset(p, 0, sizeof(*p));
  const uintptr_t a = (uintptr_t)src;
  p->base = (const uint8_t *)(a & ~(uintptr_t)15);
  p->off0 = (uint32_t)(a & 15);
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
