// gbu_internal.h -- entry points shared between the library's own translation units (not
// exported in include/gbutf.h).
#pragma once

#include <stdint.h>

#include "gbu_device.cuh"
#include "gbutf.h"

// Batched validation or transcoding (op: GBU_OP_VALIDATE_* or GBU_OP_CONVERT_*) over B
// strings given by device descriptors; results[i] receives string i's result.  Launches on
// `stream` with the context's batched geometry for op.
int gbu_internal_batch_desc(gbu_ctx *ctx, int op, const gbu::StringDesc *desc, uint64_t B, gbu_result *results,
                            gbu_stream stream);
