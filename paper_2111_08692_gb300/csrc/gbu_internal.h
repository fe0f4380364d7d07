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

// Launch partitions of a string of n code units at src for transcoding op
// (GBU_OP_CONVERT_*): its 64 KiB partitions, counting the three positions past the end that
// UTF-8 validation judges.
int gbu_internal_partitions(int op, const void *src, uint64_t n);

// Transcodes B strings (each n >= 1, output capacity in desc[i].cap) in one launch: string i
// owns launch partitions pstart[i] .. pstart[i+1]-1 (pstart[i+1] - pstart[i] =
// gbu_internal_partitions), ntiles = pstart[B] <= the context's states.  seg (B device
// entries) starts and is left {NO_ERROR, 0, 0}; results[i] receives string i's result.  desc,
// pstart and results may be mapped pinned host memory.
int gbu_internal_convert_segments(gbu_ctx *ctx, int op, const gbu::StringDesc *desc, const uint32_t *pstart,
                                  uint32_t B, uint32_t ntiles, gbu::SegState *seg, gbu_result *results,
                                  gbu_stream stream);

// The context's device, and the launch counter (for launches made outside gbu_api.cu).
int gbu_internal_device(const gbu_ctx *ctx);
void gbu_internal_count_launch(gbu_ctx *ctx);
