// gbu_noalloc.cu -- gbu_convert_utf8_to_utf16le_noalloc: the UTF-8 -> UTF-16LE transcoder
// run without a context, its look-back workspace in a static device array.
//
// Some callers cannot create a context: a context allocates its workspace with cudaMalloc,
// which can synchronise the whole device (stalling every stream of a latency-bound serving
// loop), and which fails outright in a process whose device memory is already reserved by
// another allocator (a caching allocator that owns the pool).  For them this entry point
// uses a workspace that exists from module load: a file-scope __device__ array, sized for
// inputs of up to GBU_NOALLOC_MAX_UNITS bytes.  Nothing is allocated, on any call.
//
// The kernel is the context path's utf8_to_utf16_kernel with the context's default settings
// (early exit on, the same wait limit); only where its workspace lives differs.  The kernel's
// last CTA leaves the workspace ready for the next launch (ticket, done counter and
// first-error key reset, epoch advanced), so after the one-time setup below the workspace
// needs no host-side work between calls.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "gbu_device.cuh"
#include "gbu_kernels.h"
#include "gbutf.h"

namespace {

// Partition states the workspace holds: one per partition (PART_BYTES) of the input, the input's
// first byte sitting anywhere in a 32-byte block and the three positions past its end being
// judged too.
constexpr uint32_t NOALLOC_STATES = (uint32_t)(GBU_NOALLOC_MAX_UNITS / gbu::PART_BYTES) + 1u;
static_assert(((uint64_t)GBU_NOALLOC_MAX_UNITS + 31 + 3 + gbu::PART_BYTES - 1) / gbu::PART_BYTES <=
                  NOALLOC_STATES,
              "workspace too small for the stated maximum");
static_assert(sizeof(gbu::WsHeader) % 8 == 0, "header must keep the states 8-byte aligned");

constexpr size_t NOALLOC_WORDS = sizeof(gbu::WsHeader) / 8 + NOALLOC_STATES;

// [WsHeader][NOALLOC_STATES tile states]: 128 B + 8 B per partition (128 KiB for 16 KiB
// partitions and 256 MiB of input).
static __device__ __align__(256) uint64_t noalloc_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;

struct DeviceSetup {
  std::mutex mu;
  bool ready = false;           // set once the setup below has succeeded (then never cleared)
  uint64_t *scratch = nullptr;  // device address of noalloc_scratch on this device
  int grid = 0;                 // SMs x resident CTAs of the kernel
};
DeviceSetup setups[MAX_DEVICES];

// Setup on `device` (which is current): the kernel's shared-memory opt-in, the symbol's device
// address, the grid size, and the workspace's initial contents: every state word zero (epoch
// 0, never a live epoch), the header's counters zero, its epoch 1 and its first-error key
// "none".  Returns GBU_OK and marks s ready, or GBU_CUDA_ERROR and leaves s as it was, so that
// a later call tries again.  Called with s.mu held.
int setup_device(DeviceSetup &s, int device) {
  void *addr = nullptr;
  if (cudaGetSymbolAddress(&addr, noalloc_scratch) != cudaSuccess || !addr) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  int sms = 0, bps = 0;
  const size_t smem = gbu::utf8_to_utf16_smem_bytes();
  if (cudaFuncSetAttribute(gbu::utf8_to_utf16_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gbu::utf8_to_utf16_kernel_ptr(), gbu::XT, smem) !=
          cudaSuccess ||
      sms < 1 || bps < 1) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  gbu::WsHeader h;
  memset(&h, 0, sizeof(h));
  h.epoch = 1;
  h.errkey = gbu::NO_ERROR;
  h.stop_tile = 0xFFFFFFFFu;
  if (cudaMemset(addr, 0, NOALLOC_WORDS * sizeof(uint64_t)) != cudaSuccess ||
      cudaMemcpy(addr, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  s.scratch = static_cast<uint64_t *>(addr);
  s.grid = sms * bps;
  s.ready = true;
  return GBU_OK;
}

// Runs the setup of `device` unless it has succeeded before.  The setup's synchronous copies
// and device synchronise are not allowed while a stream is being captured (and would spoil
// the capture), so a call that needs the setup while `stream` is capturing returns
// GBU_CUDA_ERROR without trying; a later call outside the capture runs it.
int ensure_setup(DeviceSetup &s, int device, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(s.mu);
  if (s.ready) return GBU_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  if (cs != cudaStreamCaptureStatusNone) return GBU_CUDA_ERROR;
  return setup_device(s, device);
}

}  // namespace

extern "C" int gbu_convert_utf8_to_utf16le_noalloc(const uint8_t *src, uint64_t n, uint16_t *dst,
                                                   uint64_t cap, gbu_result *result,
                                                   gbu_stream stream) {
  if (n > GBU_NOALLOC_MAX_UNITS) return GBU_NOALLOC_TOO_LARGE;
  if ((n > 0 && !src) || !result || (cap > 0 && !dst) || ((uintptr_t)dst & 1)) return GBU_BAD_ARGUMENT;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= MAX_DEVICES) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  DeviceSetup &s = setups[device];
  const int rc = ensure_setup(s, device, (cudaStream_t)stream);
  if (rc != GBU_OK) return rc;

  gbu::Params p;
  memset(&p, 0, sizeof(p));
  const uintptr_t a = (uintptr_t)src;
  p.base = (const uint8_t *)(a & ~(uintptr_t)31);  // the kernel's lanes read 32 bytes at a time
  p.off0 = (uint32_t)(a & 31);
  p.n = n;
  p.vbytes = p.off0 + n;
  const uint64_t span = n == 0 ? 0 : p.vbytes + 3;  // the three positions past the end
  p.ntiles = (uint32_t)((span + gbu::PART_BYTES - 1) / gbu::PART_BYTES);
  p.ws = reinterpret_cast<gbu::WsHeader *>(s.scratch);
  p.states = s.scratch + sizeof(gbu::WsHeader) / 8;
  p.max_states = NOALLOC_STATES;
  p.wait_limit = 1u << 22;  // as a context's default
  p.skip_tile = -1;
  p.early_exit = 1;         // as a context's default
  p.result = result;
  const uintptr_t d = (uintptr_t)dst;
  p.dbase = (uint8_t *)(d & ~(uintptr_t)15);
  p.dshift = (uint32_t)((d & 15) / 2);
  p.cap = cap;

  uint32_t grid = (uint32_t)s.grid;
  if (p.ntiles < grid) grid = p.ntiles;
  if (grid < 1) grid = 1;
  void *args[] = {(void *)&p};
  if (cudaLaunchKernel(gbu::utf8_to_utf16_kernel_ptr(), dim3(grid), dim3(gbu::XT), args,
                       gbu::utf8_to_utf16_smem_bytes(), (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  return GBU_OK;
}
