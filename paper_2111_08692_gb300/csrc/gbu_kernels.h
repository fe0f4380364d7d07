// gbu_kernels.h -- host-visible handles of the device kernels (internal to the library).
#pragma once

#include <stddef.h>

namespace gbu {

// mode: 0 validate, 1 length, 2 convert
size_t utf8_smem_bytes(int mode);
const void *utf8_kernel_ptr(int mode);
size_t utf16_smem_bytes(int mode);
const void *utf16_kernel_ptr(int mode);

}  // namespace gbu
