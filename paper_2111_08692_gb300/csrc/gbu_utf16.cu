// gbu_utf16.cu -- the UTF-16LE -> UTF-8 transcoders (validating): the single-buffer kernel (the
// wide partition loop of gbu_wide.cuh with the codec of gbu_wide_utf16.cuh) and the kernel over
// several strings (the partition loop of gbu_xcode.cuh with the codec of gbu_codec_utf16.cuh).
#include <stdint.h>

#include "gbu_codec_utf16.cuh"
#include "gbu_kernels.h"
#include "gbu_wide_utf16.cuh"

namespace gbu {

__global__ void __launch_bounds__(XT, XBLOCKS) utf16_to_utf8_kernel(const Params p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(WSmem), set at launch
  WSmem<Utf16ToUtf8Wide> &sm = *reinterpret_cast<WSmem<Utf16ToUtf8Wide> *>(smem_raw);
  wtranscode<Utf16ToUtf8Wide>(p, sm, [&](uint32_t status, unsigned long long key, unsigned long long tot) {
    if (status) {
      write_result(p.result, GBU_TIMEOUT, 0);
    } else if (key != NO_ERROR) {
      uint64_t off;
      resolve_utf16_error(reinterpret_cast<const uint16_t *>(p.base + p.off0), p.n,
                          ((long long)key - (long long)p.off0) / 2, &off);
      write_result(p.result, GBU_SURROGATE, off);
    } else {
      write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
    }
  });
}

// Several strings per launch (the serving loop's large requests): one result per string.
__global__ void __launch_bounds__(XT, XBLOCKS) utf16_to_utf8_segments_kernel(const SegParams q) {
  extern __shared__ __align__(128) unsigned char smem_raw[];  // sizeof(XSmem), set at launch
  XSmem<Utf16ToUtf8> &sm = *reinterpret_cast<XSmem<Utf16ToUtf8> *>(smem_raw);
  transcode_segments<Utf16ToUtf8>(q, sm, [&](const Params &p, const SegState &st, uint32_t) {
    const uint32_t status = *(volatile uint32_t *)&p.ws->status;
    const unsigned long long key = *(volatile const unsigned long long *)&st.errkey;
    const unsigned long long tot = *(volatile const unsigned long long *)&st.total;
    if (status) {
      write_result(p.result, GBU_TIMEOUT, 0);
    } else if (key != NO_ERROR) {
      uint64_t off;
      resolve_utf16_error(reinterpret_cast<const uint16_t *>(p.base + p.off0), p.n,
                          ((long long)key - (long long)p.off0) / 2, &off);
      write_result(p.result, GBU_SURROGATE, off);
    } else {
      write_result(p.result, tot > p.cap ? GBU_OUTPUT_TOO_SMALL : GBU_OK, tot);
    }
  });
}

const void *utf16_to_utf8_kernel_ptr() { return (const void *)utf16_to_utf8_kernel; }
size_t utf16_to_utf8_smem_bytes() { return sizeof(WSmem<Utf16ToUtf8Wide>); }
size_t utf16_to_utf8_segments_smem_bytes() { return sizeof(XSmem<Utf16ToUtf8>); }

const void *utf16_to_utf8_segments_kernel_ptr() { return (const void *)utf16_to_utf8_segments_kernel; }

}  // namespace gbu
