// gbu_kernels.h -- host-visible handles of the device kernels (internal to the library).
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace gbu {

// read-only streaming kernels; mode: 0 validate_utf8, 1 utf16_length_from_utf8,
// 2 validate_utf16le, 3 utf8_length_from_utf16le, 4 validate_utf16be, 5 utf8_length_from_utf16be
const void *stream_kernel_ptr(int mode);
uint32_t stream_tile_bytes();

// transcoders (dynamic shared memory of the given size; above 48 KB it needs the
// cudaFuncAttributeMaxDynamicSharedMemorySize opt-in before the first launch)
const void *utf8_to_utf16_kernel_ptr();
const void *utf16_to_utf8_kernel_ptr();
size_t utf8_to_utf16_smem_bytes();
size_t utf16_to_utf8_smem_bytes();
// the transcoders between UTF-8 and UTF-16BE (same launch shape as the UTF-16LE ones)
const void *utf16be_to_utf8_kernel_ptr();
size_t utf16be_to_utf8_smem_bytes();
const void *utf8_to_utf16be_kernel_ptr();
size_t utf8_to_utf16be_smem_bytes();
// UTF-32: read-only kernel (mode 0 validate_utf32, 1 utf8_length_from_utf32,
// 2 utf32_length_from_utf8, 3 utf16_length_from_utf32, 4 utf32_length_from_utf16le) and the
// transcoders between UTF-32 and UTF-8 / UTF-16LE
const void *utf32_stream_kernel_ptr(int mode);
const void *utf32_to_utf8_kernel_ptr();
size_t utf32_to_utf8_smem_bytes();
const void *utf8_to_utf32_kernel_ptr();
size_t utf8_to_utf32_smem_bytes();
const void *utf32_to_utf16_kernel_ptr();
size_t utf32_to_utf16_smem_bytes();
const void *utf16_to_utf32_kernel_ptr();
size_t utf16_to_utf32_smem_bytes();
// the same transcoders over several strings per launch (SegParams)
const void *utf8_to_utf16_segments_kernel_ptr();
const void *utf16_to_utf8_segments_kernel_ptr();
size_t utf8_to_utf16_segments_smem_bytes();
size_t utf16_to_utf8_segments_smem_bytes();

// batched kernels (mode: BatchMode; nwarps: 4, 8 or 16 warps per CTA) and the u64 scan
const void *batch_kernel_ptr(int mode, int nwarps);
const void *scan_kernel_ptr();
uint32_t scan_tile_items();
int scan_threads();

}  // namespace gbu
