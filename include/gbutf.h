/*
 * gbutf.h -- C ABI of the GB300 (sm_103a) UTF-8 / UTF-16LE validation and transcoding library.
 *
 * The operations are the ones the paper ("Unicode at Gigabytes per Second") sets out to make
 * fast: validate UTF-8 and UTF-16, and transcode between them, always validating (Section 1
 * states the problem, Section 3 defines both formats and the six UTF-8 validity rules,
 * Section 5 states that every transcoding also validates).  The output-length functions give
 * the exact size of the other encoding (Section 3 per-character sizes).
 *
 * Conventions shared by every call:
 *   - Units.  n, cap, offsets and counts are in code units of the buffer they describe: bytes
 *     for UTF-8, 16-bit words for UTF-16LE.  Offsets and counts are 64-bit.
 *   - Memory.  src, dst, len and result pointers are DEVICE pointers owned by the caller
 *     (result may also be pinned host memory mapped into the device address space).  The
 *     library never allocates on a call; it only uses the workspace held by the context.
 *   - Alignment.  uint16_t buffers must be 2-byte aligned; any other alignment is accepted.
 *   - Streams.  Every call is asynchronous on `stream`; the result is valid once the stream
 *     has reached the call.  One context serves one stream at a time: calls made through the
 *     same context on different streams must not overlap (use one context per stream).
 *   - Return value.  GBU_OK if the work was enqueued, GBU_BAD_ARGUMENT (NULL pointer with
 *     n > 0, misaligned uint16_t pointer, n beyond the context's capacity) or GBU_CUDA_ERROR
 *     (the launch failed).  Nothing is enqueued when the return value is not GBU_OK.
 *   - n == 0 is valid: the result is {GBU_OK, 0}; result is still written (by a tiny kernel).
 *
 * Result of a validation or transcoding (gbu_result):
 *   status GBU_OK            count = n (validation) or code units written (transcoding)
 *   status 1..6              the input is invalid; count = offset of the first invalid code
 *                            unit of src (the first unit of the ill-formed sequence)
 *   status GBU_OUTPUT_TOO_SMALL  the input is valid but needs count > cap output units;
 *                            dst[0:cap] holds the first cap units of the conversion
 *   status GBU_TIMEOUT       a device-side wait gave up (see gbu_set_wait_limit); the output
 *                            and the context's workspace must be considered lost (call
 *                            gbu_reset before reusing the context)
 * On an input error, dst[0 : L] holds the conversion of the valid prefix src[0:count], where L
 * is its output length (clipped to cap); dst beyond L is unspecified but no unit at or past
 * cap is ever written.  When an input breaks several rules, the kind reported is the one the
 * bytes read so far break first in reading order: after each byte of a UTF-8 sequence the
 * values it could still encode form an interval, and the sequence is ill-formed as soon as
 * that whole interval breaks rule 4, 5 or 6; a missing continuation byte, also at the end of
 * the buffer, is GBU_TOO_SHORT.
 */
#ifndef GBUTF_H
#define GBUTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GBU_OK = 0,
  GBU_HEADER_BITS = 1,     /* rule 1: a byte whose five most significant bits are all ones */
  GBU_TOO_SHORT = 2,       /* rule 2: a leading byte without its continuation bytes        */
  GBU_TOO_LONG = 3,        /* rule 3: a continuation byte with no leading byte             */
  GBU_OVERLONG = 4,        /* rule 4: a value that a shorter sequence encodes              */
  GBU_TOO_LARGE = 5,       /* rule 5: a value of 1,114,112 (0x110000) or more              */
  GBU_SURROGATE = 6,       /* rule 6 in UTF-8 (D800-DFFF); an unpaired UTF-16 surrogate    */
  GBU_OUTPUT_TOO_SMALL = 16,
  GBU_BAD_ARGUMENT = 17,
  GBU_CUDA_ERROR = 18,
  GBU_TIMEOUT = 19,
  GBU_NOALLOC_TOO_LARGE = 20, /* n above GBU_NOALLOC_MAX_UNITS (gbu_convert_utf8_to_utf16le_noalloc) */
  GBU_CANCELLED = 21,         /* serving: the request was cancelled before admission       */
  GBU_OVER_BUDGET = 22        /* serving: the request can never fit the memory budget      */
} gbu_status;

typedef struct {
  int32_t status;   /* gbu_status */
  int32_t reserved; /* 0 */
  uint64_t count;   /* see above */
} gbu_result;       /* 16 bytes */

typedef struct gbu_ctx gbu_ctx;
typedef struct CUstream_st *gbu_stream; /* a cudaStream_t; NULL = the legacy default stream */

/* Creates a context on `device` whose workspace (tile states and counters, allocated once
 * here) serves inputs of up to max_units code units.  Returns NULL on failure. */
gbu_ctx *gbu_create(int device, uint64_t max_units);
/* Frees the context's workspace.  The caller must make sure no work using it is pending. */
void gbu_destroy(gbu_ctx *ctx);
/* Re-initialises the workspace (after GBU_TIMEOUT).  Synchronous. */
int gbu_reset(gbu_ctx *ctx);
/* Bound on each device-side spin wait, in polling rounds (default 2^22; tests use small
 * values together with gbu_debug_skip_publish to exercise the timeout path). */
void gbu_set_wait_limit(gbu_ctx *ctx, uint32_t rounds);
/* Test hook: the tile with this index never publishes its scan state, so the tiles after it
 * wait until the limit and the call reports GBU_TIMEOUT.  -1 (default) disables the hook. */
void gbu_debug_skip_publish(gbu_ctx *ctx, int64_t tile);
/* Early exit on invalid input (on by default).  The single-buffer validation calls and
 * transcoders publish the position of a flagged chunk as soon as a thread finds one; work
 * that lies wholly past it is skipped (validation stops reading, a transcoder still counts
 * and chains such a partition but does not convert it).  Results are identical either way,
 * since the first error and the output of the valid prefix never lie past a flagged chunk;
 * only the time to reach them changes.  enable = 0 scans every input to the end (used to
 * time full scans).  Not in the paper, whose kernels process blocks in order and can stop at
 * once. */
void gbu_set_early_exit(gbu_ctx *ctx, int enable);

/* UTF-8 validation (Section 3, rules 1-6). */
int gbu_validate_utf8(gbu_ctx *ctx, const uint8_t *src, uint64_t n, gbu_result *result,
                      gbu_stream stream);
/* UTF-16LE validation (Section 3: every D800-DBFF word is followed by a DC00-DFFF word and
 * every DC00-DFFF word follows a D800-DBFF word). */
int gbu_validate_utf16le(gbu_ctx *ctx, const uint16_t *src, uint64_t n, gbu_result *result,
                         gbu_stream stream);

/* Output lengths (Section 3 per-character sizes), defined for any input and computed without
 * validation: UTF-16 words = bytes that are not continuation bytes (10xxxxxx) + bytes F0-FF;
 * UTF-8 bytes = 1 per word below 0x80, 2 below 0x800, 2 per surrogate word, else 3.  Both are
 * exact for valid input.  *len is a device uint64_t. */
int gbu_utf16_length_from_utf8(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint64_t *len,
                               gbu_stream stream);
int gbu_utf8_length_from_utf16le(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint64_t *len,
                                 gbu_stream stream);

/* Validating transcoders (Section 3 formats; Section 5: transcoding includes validation).
 * dst holds cap code units of the output format. */
int gbu_convert_utf8_to_utf16le(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint16_t *dst,
                                uint64_t cap, gbu_result *result, gbu_stream stream);
int gbu_convert_utf16le_to_utf8(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint8_t *dst,
                                uint64_t cap, gbu_result *result, gbu_stream stream);

/* Host-synchronising forms of the six calls above: the same operation on the same arguments
 * (without `result`), run on `stream`, which the call then waits for; the result comes back by
 * value.  This is the problem as the paper states it (Section 1; Section 5: transcoding includes
 * validation): one call in, and out either the output length or the kind and offset of the
 * first error.
 *   validate / convert: the gbu_result the asynchronous call would have written;
 *   lengths: {GBU_OK, length}.
 * A launch failure returns {that status (GBU_BAD_ARGUMENT, GBU_CUDA_ERROR), 0}; a NULL ctx
 * returns {GBU_BAD_ARGUMENT, 0}.  The result travels through a slot of the context's workspace
 * (device memory) and one device-to-host copy, so calls on one context must not overlap, as
 * for the asynchronous calls. */
gbu_result gbu_validate_utf8_sync(gbu_ctx *ctx, const uint8_t *src, uint64_t n, gbu_stream stream);
gbu_result gbu_validate_utf16le_sync(gbu_ctx *ctx, const uint16_t *src, uint64_t n, gbu_stream stream);
gbu_result gbu_utf16_length_from_utf8_sync(gbu_ctx *ctx, const uint8_t *src, uint64_t n, gbu_stream stream);
gbu_result gbu_utf8_length_from_utf16le_sync(gbu_ctx *ctx, const uint16_t *src, uint64_t n, gbu_stream stream);
gbu_result gbu_convert_utf8_to_utf16le_sync(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint16_t *dst,
                                            uint64_t cap, gbu_stream stream);
gbu_result gbu_convert_utf16le_to_utf8_sync(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint8_t *dst,
                                            uint64_t cap, gbu_stream stream);

/* UTF-16BE: the same words as UTF-16LE (Section 3) with each word's most significant byte first
 * in memory (the byte order RFC 2781 names; no byte-order-mark sniffing).  src / dst are the
 * words as they lie in memory (2-byte aligned).  Results, units, capacities, error offsets and
 * return values are exactly those of the UTF-16LE calls on the byte-exchanged words; the UTF-16
 * length of a UTF-8 input is gbu_utf16_length_from_utf8's. */
int gbu_validate_utf16be(gbu_ctx *ctx, const uint16_t *src, uint64_t n, gbu_result *result,
                         gbu_stream stream);
int gbu_utf8_length_from_utf16be(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint64_t *len,
                                 gbu_stream stream);
int gbu_convert_utf16be_to_utf8(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint8_t *dst,
                                uint64_t cap, gbu_result *result, gbu_stream stream);
int gbu_convert_utf8_to_utf16be(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint16_t *dst,
                                uint64_t cap, gbu_result *result, gbu_stream stream);

/* UTF-32 (not in the paper, whose problem is UTF-8 and UTF-16): one 32-bit unit per value, in
 * host (little-endian) byte order, 4-byte aligned.  A unit is valid when Section 3 allows its
 * value: below 1,114,112 (rule 5; else GBU_TOO_LARGE) and outside D800-DFFF (rule 6; else
 * GBU_SURROGATE); the offset is the unit's index.  The lengths are formulas for any input: UTF-8
 * bytes by value (1 below 0x80, 2 below 0x800, 3 below 0x10000, else 4), and one UTF-32 unit per
 * UTF-8 byte that is not a continuation byte.  Transcoding validates (rules 1-6 for UTF-8
 * input); results, capacities and return values as for the UTF-16LE calls. */
int gbu_validate_utf32(gbu_ctx *ctx, const uint32_t *src, uint64_t n, gbu_result *result, gbu_stream stream);
int gbu_utf8_length_from_utf32(gbu_ctx *ctx, const uint32_t *src, uint64_t n, uint64_t *len, gbu_stream stream);
int gbu_utf32_length_from_utf8(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint64_t *len, gbu_stream stream);
int gbu_convert_utf32_to_utf8(gbu_ctx *ctx, const uint32_t *src, uint64_t n, uint8_t *dst, uint64_t cap,
                              gbu_result *result, gbu_stream stream);
int gbu_convert_utf8_to_utf32(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint32_t *dst, uint64_t cap,
                              gbu_result *result, gbu_stream stream);
/* UTF-16LE <-> UTF-32.  Lengths for any input: UTF-16 words of a UTF-32 input (1 per unit below
 * 0x10000, else 2), and UTF-32 units of a UTF-16LE input (1 per word that is not a second
 * surrogate DC00-DFFF).  The UTF-16LE input is validated by Section 3's pair rules
 * (GBU_SURROGATE at the first unpaired surrogate), the UTF-32 input as above. */
int gbu_utf16_length_from_utf32(gbu_ctx *ctx, const uint32_t *src, uint64_t n, uint64_t *len, gbu_stream stream);
int gbu_utf32_length_from_utf16le(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint64_t *len, gbu_stream stream);
int gbu_convert_utf32_to_utf16le(gbu_ctx *ctx, const uint32_t *src, uint64_t n, uint16_t *dst, uint64_t cap,
                                 gbu_result *result, gbu_stream stream);
int gbu_convert_utf16le_to_utf32(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint32_t *dst, uint64_t cap,
                                 gbu_result *result, gbu_stream stream);

/* ---- Batched forms ------------------------------------------------------------------------
 * The same six operations over B strings in ONE launch (a persistent grid; strings never wait
 * on one another).  The strings lie back to back in src; string i is src[off[i] : off[i+1]]
 * (code units of src).  off (B+1 entries), dst_off (B+1 entries), results (B entries) and
 * lens (B entries) are 8-byte-aligned DEVICE arrays.  off and dst_off must be non-decreasing
 * and inside their buffers (they are not checked; a decreasing pair reads as an empty
 * string).  Each string's result is exactly the single-buffer call's result on that string
 * alone: results[i] as for the single-buffer call (offsets relative to the string), lens[i]
 * its output length.  Transcoders write string i's output to dst[dst_off[i] : dst_off[i+1]]
 * (capacity dst_off[i+1] - dst_off[i]); dst_off is typically the exclusive scan of the
 * batched length call (gbu_exclusive_scan_u64) or a worst-case layout (n units out per UTF-8
 * unit in, 3 bytes out per UTF-16 unit in).  B == 0 enqueues nothing.  Return values as for
 * the single-buffer calls; GBU_BAD_ARGUMENT also for a NULL or misaligned array when B > 0.
 * The launch geometry is the context's per-operation gbu_batch_config (gbu_tune_batched picks
 * it by timing).  No call allocates or synchronises, so all of them can be captured in a
 * CUDA graph (gbu_graph_begin / gbu_graph_end).  Not in the paper, which handles one buffer
 * per call: this is a serving form of the same per-string operations. */
int gbu_validate_utf8_batched(gbu_ctx *ctx, const uint8_t *src, const uint64_t *off, uint64_t B,
                              gbu_result *results, gbu_stream stream);
int gbu_validate_utf16le_batched(gbu_ctx *ctx, const uint16_t *src, const uint64_t *off, uint64_t B,
                                 gbu_result *results, gbu_stream stream);
int gbu_utf16_length_from_utf8_batched(gbu_ctx *ctx, const uint8_t *src, const uint64_t *off, uint64_t B,
                                       uint64_t *lens, gbu_stream stream);
int gbu_utf8_length_from_utf16le_batched(gbu_ctx *ctx, const uint16_t *src, const uint64_t *off,
                                         uint64_t B, uint64_t *lens, gbu_stream stream);
int gbu_convert_utf8_to_utf16le_batched(gbu_ctx *ctx, const uint8_t *src, const uint64_t *off, uint64_t B,
                                        uint16_t *dst, const uint64_t *dst_off, gbu_result *results,
                                        gbu_stream stream);
int gbu_convert_utf16le_to_utf8_batched(gbu_ctx *ctx, const uint16_t *src, const uint64_t *off, uint64_t B,
                                        uint8_t *dst, const uint64_t *dst_off, gbu_result *results,
                                        gbu_stream stream);

/* out[k] = in[0] + ... + in[k-1] for k = 0 .. count (out has count + 1 entries, out[count] is
 * the total): output offsets from batched lengths.  One launch, chained by a decoupled
 * look-back (Merrill & Garland, 2016).  *result = {GBU_OK, total}; GBU_TIMEOUT as for the
 * transcoders; GBU_BAD_ARGUMENT if the total reaches 2^44 (then out is not valid).  Needs
 * count + 1 <= 4096 x (the context's tile states: max_units + 1 values always fit); returns
 * GBU_BAD_ARGUMENT beyond. */
int gbu_exclusive_scan_u64(gbu_ctx *ctx, const uint64_t *in, uint64_t count, uint64_t *out,
                           gbu_result *result, gbu_stream stream);

/* Operation codes of the batched calls (same order as gbu_launch_config). */
typedef enum {
  GBU_OP_VALIDATE_UTF8 = 0,
  GBU_OP_UTF16_LENGTH_FROM_UTF8 = 1,
  GBU_OP_CONVERT_UTF8_TO_UTF16LE = 2,
  GBU_OP_VALIDATE_UTF16LE = 3,
  GBU_OP_UTF8_LENGTH_FROM_UTF16LE = 4,
  GBU_OP_CONVERT_UTF16LE_TO_UTF8 = 5
} gbu_op;

/* The per-string alternative to a batched call, for measuring what batching saves: the same
 * B strings (input offsets off[B+1] in input code units, and for the transcoders output
 * offsets dst_off[B+1] in output code units, both in HOST memory) handled by B single-buffer
 * calls of operation `op` issued one after another from a C loop on `stream`, string i's
 * result into results[i] (device; lengths into ((uint64_t *)results)[i]).  src, dst and
 * results are device memory, as for the batched call.  Returns the first launch error, or
 * GBU_OK; B launches are made.  The paper has no counterpart: it transcodes one buffer at a
 * time (Section 5), which this loop repeats per string. */
int gbu_per_string_loop(gbu_ctx *ctx, int op, const void *src, const uint64_t *off, uint64_t B, void *dst,
                        const uint64_t *dst_off, gbu_result *results, gbu_stream stream);

/* Launch geometry of a batched operation.  A CTA of warps_per_cta warps claims
 * strings_per_claim consecutive strings at a time; each warp takes one string at a time,
 * except that strings of at least long_bytes input bytes are handled afterwards by the whole
 * CTA (warps_per_cta x 512 bytes per step). */
typedef struct {
  int32_t warps_per_cta;      /* 4, 8 or 16 (default 8) */
  uint32_t strings_per_claim; /* 1 .. 1024 (default 64) */
  uint32_t long_bytes;        /* >= 512 (default 4096) */
  float tuned_ms;             /* the tuner's best time for this geometry; 0 if set by hand */
} gbu_batch_config;

int gbu_get_batch_config(const gbu_ctx *ctx, int op, gbu_batch_config *cfg);
int gbu_set_batch_config(gbu_ctx *ctx, int op, const gbu_batch_config *cfg); /* checks ranges */
/* Autotuner: runs operation `op` on the given batch (arguments as for the batched call of
 * that operation; `out` is results or lens) for each candidate geometry (warps 4/8/16 x
 * claims of 8/32/128/512 strings x long-string thresholds of 2/4/8/16 KiB), one untimed and
 * `reps` timed launches each (CUDA events on `stream`), keeps the fastest in the context and
 * writes it to *chosen (may be NULL).  The last launch uses the chosen geometry, so the
 * outputs are valid.  Synchronous; not capturable. */
int gbu_tune_batched(gbu_ctx *ctx, int op, const void *src, const uint64_t *off, uint64_t B, void *dst,
                     const uint64_t *dst_off, void *out, int reps, gbu_stream stream,
                     gbu_batch_config *chosen);

/* ---- CUDA graphs --------------------------------------------------------------------------
 * gbu_graph_begin starts capturing `stream` (not the legacy default stream); every library
 * call made on it, by this thread, until gbu_graph_end is recorded instead of run (calls are
 * launches only: none allocates or synchronises).  gbu_graph_end instantiates the graph
 * (NULL on failure).  gbu_graph_launch replays it on any stream of the context's device; the
 * pointers and sizes captured are fixed.  The context must outlive its graphs, and the
 * one-stream-at-a-time rule of the context holds for replays too. */
typedef struct gbu_graph gbu_graph;
int gbu_graph_begin(gbu_ctx *ctx, gbu_stream stream);
gbu_graph *gbu_graph_end(gbu_ctx *ctx, gbu_stream stream);
int gbu_graph_launch(gbu_graph *graph, gbu_stream stream);
uint64_t gbu_graph_kernels(const gbu_graph *graph); /* library kernels per replay */
void gbu_graph_destroy(gbu_graph *graph);

/* ---- Serving loop --------------------------------------------------------------------------
 * Continuous batching of validation and transcoding requests on one device (not in the
 * paper, which measures one buffer at a time: this is a serving form of the same calls).
 * A scheduler thread admits requests in submission order once their scheduled arrival time
 * (server clock, gbu_server_now_ns) has passed, while an in-flight slot is free and the
 * device-memory budget covers the inputs and worst-case outputs of everything admitted;
 * outputs come from a device arena of budget_bytes allocated at creation.  Admitted small
 * requests of one operation share ONE batched launch (device descriptors); transcodings of
 * at least large_bytes of one direction share one partitioned launch (each request split into
 * 16 KiB partitions with its own look-back chain, so all SMs work on the group); large
 * validations get single-buffer launches.  Launch groups are spread over `streams`
 * CUDA streams, `groups_per_stream` in flight on each, so newly admitted work overlaps with
 * running work.  Each request's result is the one the single-buffer call gives on it.
 * Request inputs are DEVICE buffers that must stay valid until the request completes.
 * Submit requests in non-decreasing arrival order (a later arrival at the head of the queue
 * holds back the ones behind it). */
typedef struct {
  uint64_t budget_bytes;      /* device memory for inputs + outputs in flight (default 8 GiB) */
  int32_t streams;            /* CUDA streams (default 16)                                  */
  int32_t groups_per_stream;  /* launch groups in flight per stream (default 8)             */
  uint32_t max_group;         /* small requests per batched launch (default 4096)           */
  uint32_t max_large_group;   /* large transcodings per launch (default 32)                 */
  uint64_t large_bytes;       /* input bytes from which a request runs alone (default 64 KiB) */
  uint64_t max_request_units; /* largest request accepted, code units (default 16 Mi)       */
  uint32_t max_inflight;      /* admitted, not yet completed requests (default 65536)       */
  uint32_t device_rings;      /* where a launch group's request descriptors and results live:
                               * 0 = mapped pinned host memory, read and written by the kernels
                               * over the host link (no copies); 1 = device memory, with one
                               * host-to-device copy of the descriptors before the group's
                               * launches and one device-to-host copy of the results after them
                               * (default 0; see gbu_server_default_config) */
} gbu_server_config;

typedef struct {
  int32_t op;           /* GBU_OP_VALIDATE_UTF8, _VALIDATE_UTF16LE, _CONVERT_UTF8_TO_UTF16LE or
                           _CONVERT_UTF16LE_TO_UTF8 */
  int32_t flags;        /* GBU_REQ_DISCARD_OUTPUT: free the output at completion (only the
                           result is wanted) */
  const void *src;      /* device pointer, n code units */
  uint64_t n;
  uint64_t arrival_ns;  /* scheduled arrival on the server clock (0: at once) */
  uint64_t tag;         /* returned in the completion */
} gbu_request;

#define GBU_REQ_DISCARD_OUTPUT 1

typedef struct {
  uint64_t id;
  uint64_t tag;
  gbu_result result;    /* as the single-buffer call's; GBU_CANCELLED for a cancelled request */
  void *dst;            /* transcodings: device output (result.count units when GBU_OK),
                           valid until gbu_server_release(id); NULL otherwise */
  uint64_t arrival_ns, admit_ns, complete_ns;  /* server clock */
} gbu_completion;

typedef struct {
  uint64_t submitted, admitted, completed;
  uint64_t launches, groups;     /* library launches and launch groups enqueued */
  uint64_t budget_used_bytes, peak_budget_bytes;
  uint64_t inflight, pending;
} gbu_server_stats;

void gbu_server_default_config(gbu_server_config *cfg);
/* Allocates the arena, streams, contexts and pinned staging, and starts the scheduler
 * thread.  cfg NULL = defaults.  Returns NULL on failure. */
typedef struct gbu_server gbu_server;
gbu_server *gbu_server_create(int device, const gbu_server_config *cfg);
/* Stops after the admitted work is done; requests not yet admitted are dropped. */
void gbu_server_destroy(gbu_server *server);
uint64_t gbu_server_now_ns(const gbu_server *server);
/* Queues count requests; their ids are *first_id, *first_id + 1, ...  GBU_BAD_ARGUMENT (bad
 * op, NULL src with n > 0, misaligned UTF-16, n above max_request_units) or GBU_OVER_BUDGET
 * (a request larger than the whole budget): then none is queued.  Thread-safe. */
int gbu_server_submit(gbu_server *server, const gbu_request *reqs, uint64_t count, uint64_t *first_id);
/* Cancels a request not yet admitted (it completes with GBU_CANCELLED); GBU_BAD_ARGUMENT if
 * it is unknown or already admitted. */
int gbu_server_cancel(gbu_server *server, uint64_t id);
/* Moves up to max completions (oldest first) into out; returns how many.  Non-blocking. */
int gbu_server_poll(gbu_server *server, gbu_completion *out, int max);
/* Returns a completed transcoding's output buffer to the arena (and its bytes to the budget). */
int gbu_server_release(gbu_server *server, uint64_t id);
int gbu_server_get_stats(gbu_server *server, gbu_server_stats *out);
/* Copies the first `bytes` bytes of a completed, unreleased transcoding's output into host
 * memory (synchronous; for clients that want the text on the host). */
int gbu_server_copy_output(gbu_server *server, uint64_t id, void *host, uint64_t bytes);

/* The server's arena bookkeeping (first-fit offsets with coalescing; no memory behind it),
 * exported for host-side tests.  gbu_arena_alloc returns GBU_OVER_BUDGET when no free block
 * is large enough. */
typedef struct gbu_arena gbu_arena;
gbu_arena *gbu_arena_create(uint64_t capacity, uint64_t align);
int gbu_arena_alloc(gbu_arena *arena, uint64_t size, uint64_t *off);
int gbu_arena_free(gbu_arena *arena, uint64_t off);
uint64_t gbu_arena_used(const gbu_arena *arena);
uint64_t gbu_arena_largest_free(const gbu_arena *arena);
uint64_t gbu_arena_free_blocks(const gbu_arena *arena);
void gbu_arena_destroy(gbu_arena *arena);

/* Context-free, allocation-free form of gbu_convert_utf8_to_utf16le, for callers that cannot
 * allocate device memory: creating a context calls cudaMalloc, which can synchronise the
 * whole device (stalling every stream of a latency-bound serving loop) and fails where
 * another allocator already owns the device's memory.  The paper has no counterpart: it is
 * a deployment form of the same Section 3 / Section 5 transcoding, with identical results.
 *
 * The workspace is a static device array of the library (128 B + 8 B per 16 KiB partition),
 * sized for n <= GBU_NOALLOC_MAX_UNITS bytes; a larger n returns GBU_NOALLOC_TOO_LARGE and
 * enqueues nothing.  Runs on the CURRENT device, with a context's default settings (early
 * exit on), so its result and dst[0 : valid prefix] equal the context path's.  The first call
 * on each device does a one-time setup there (looks up the array's device address, queries
 * the occupancy, clears the array with synchronous copies and a device synchronise), so make
 * that first call before any stream capture: if `stream` is being captured when the setup is
 * still needed, the call returns GBU_CUDA_ERROR without touching the device, and a later call
 * outside the capture runs the setup.  A setup that fails is tried again by the next call.
 * The library never allocates on any call.
 *
 * There is ONE workspace per device, shared by every call: two calls whose kernels overlap
 * (different streams, or threads, without ordering between them) race on it and both give
 * undefined results.  Order them (one stream, or events).  Arguments, results, alignment and
 * the other return values are as for gbu_convert_utf8_to_utf16le. */
#define GBU_NOALLOC_MAX_UNITS ((uint64_t)1 << 28) /* 256 MiB of UTF-8 input */
int gbu_convert_utf8_to_utf16le_noalloc(const uint8_t *src, uint64_t n, uint16_t *dst, uint64_t cap,
                                        gbu_result *result, gbu_stream stream);

/* ---- Host-buffer form ----------------------------------------------------------------------
 * The six single-buffer operations on HOST buffers, as one synchronous call: the problem as a
 * program with its text in host memory meets it (paper §1, disk- and network-rate inputs).  The
 * input is cut into pieces of at most piece_units code units at character starts (a UTF-8 cut
 * moved back past at most three continuation bytes; a UTF-16 cut moved back off a second
 * surrogate that follows a first one), and each piece goes through a host-to-device copy, the
 * single-buffer call and a copy of its result (and output) back, in one of `streams` lanes (a
 * copy stream for the input and a stream for the kernel and the copies back), so that the
 * copies of one piece overlap the kernels and copies of the others.  The result is the
 * whole input's, as the single-buffer call would give it: the first error (its kind, and its
 * offset in the whole input: the pieces are judged in order), else the output length (units the
 * length calls count, or the transcoders write).  A transcoder writes dst[0 : length] (on an
 * input error, dst[0 : valid prefix]; past cap nothing, and the result is then
 * GBU_OUTPUT_TOO_SMALL with the full length).
 *
 * Host buffers should be pinned (cudaHostAlloc or cudaHostRegister) for the copies to overlap the
 * kernels.  A pipe owns, from creation, one context and one set of device buffers per lane
 * (2 x piece_units + 3 x piece_units + 64 bytes each) and its streams; nothing is allocated by
 * a call.  Calls on one pipe must not overlap.  Returns GBU_OK, GBU_BAD_ARGUMENT (NULL pipe,
 * result or src with n > 0; NULL dst with cap > 0; an odd uint16_t pointer) or GBU_CUDA_ERROR;
 * *result is host memory. */
typedef struct gbu_pipe gbu_pipe;
/* piece_units 4096 .. 2^32 (default when 0: 64 Mi); streams 1..8 (default when 0: 3).  NULL on failure. */
gbu_pipe *gbu_pipe_create(int device, uint64_t piece_units, int streams);
void gbu_pipe_destroy(gbu_pipe *pipe);
int gbu_pipe_validate_utf8(gbu_pipe *pipe, const uint8_t *src, uint64_t n, gbu_result *result);
int gbu_pipe_validate_utf16le(gbu_pipe *pipe, const uint16_t *src, uint64_t n, gbu_result *result);
int gbu_pipe_utf16_length_from_utf8(gbu_pipe *pipe, const uint8_t *src, uint64_t n, gbu_result *result);
int gbu_pipe_utf8_length_from_utf16le(gbu_pipe *pipe, const uint16_t *src, uint64_t n, gbu_result *result);
int gbu_pipe_convert_utf8_to_utf16le(gbu_pipe *pipe, const uint8_t *src, uint64_t n, uint16_t *dst, uint64_t cap,
                                     gbu_result *result);
int gbu_pipe_convert_utf16le_to_utf8(gbu_pipe *pipe, const uint16_t *src, uint64_t n, uint8_t *dst, uint64_t cap,
                                     gbu_result *result);

/* ---- Sharded form --------------------------------------------------------------------------
 * One buffer split into P shards at character boundaries, so that each shard can be handled by
 * an ordinary single-buffer call (on its own stream and context, or on its own GPU), and the
 * shards' results combined into the result of the whole buffer.  Not in the paper, which
 * processes one buffer on one core: this is the data-parallel split of the same Section 3
 * validation and transcoding.
 *
 * Cuts: cuts[0] = 0, cuts[P] = n, and cuts[k] (0 < k < P) is the nominal start
 * floor(k n / P) (balanced) moved forward to a character start: UTF-8, the first position in
 * [c, c+3) whose byte is not a continuation byte (10xxxxxx), else c+3; UTF-16LE, c+1 when the
 * word at c is a second surrogate (DC00-DFFF), else c.  The cuts never decrease (a shard may be
 * empty).  Inside a valid prefix every cut is a character start, and a sequence that a cut
 * splits fails in its shard with the kind and offset it has in the whole buffer, so:
 *   - validation/transcoding: the first shard (in order) with an input error holds the
 *     buffer's first error, at cuts[k] + its offset, and the shards before it are valid;
 *   - lengths: the buffer's length is the sum of the shards' lengths (the formulas are per
 *     position);
 *   - transcoding: shard k writes to dst + off[k] with capacity off[k+1] - off[k], where off is
 *     the exclusive scan of the shards' output lengths (gbu_exclusive_scan_u64) clipped to the
 *     buffer's cap; then dst[0:L] of the valid prefix is exactly the single call's output.
 * P is 1 .. GBU_MAX_SHARDS.  cuts has P + 1 entries (8-byte aligned). */
#define GBU_MAX_SHARDS 65536u
/* Cuts of a DEVICE buffer, written to the DEVICE array cuts by one small launch on `stream`. */
int gbu_shard_cuts_utf8(gbu_ctx *ctx, const uint8_t *src, uint64_t n, uint32_t P, uint64_t *cuts,
                        gbu_stream stream);
int gbu_shard_cuts_utf16le(gbu_ctx *ctx, const uint16_t *src, uint64_t n, uint32_t P, uint64_t *cuts,
                           gbu_stream stream);
/* The same cuts of a HOST buffer, computed on the host (a loader that splits text before
 * sending each shard to its GPU). */
int gbu_shard_cuts_utf8_host(const uint8_t *src, uint64_t n, uint32_t P, uint64_t *cuts);
int gbu_shard_cuts_utf16le_host(const uint16_t *src, uint64_t n, uint32_t P, uint64_t *cuts);
/* Host: combines the P shards' validation or transcoding results (host arrays; cuts as above)
 * into *out.  A shard that reported GBU_TIMEOUT (or another call failure) makes that the
 * result; else the first shard with an input error gives {kind, cuts[k] + count}; else
 * {GBU_OK, sum of counts}, or {GBU_OUTPUT_TOO_SMALL, sum of counts} if any shard ran out of
 * room.  GBU_BAD_ARGUMENT for NULL arrays, P out of range or decreasing cuts. */
int gbu_combine_shards(const uint64_t *cuts, const gbu_result *parts, uint32_t P, gbu_result *out);

/* ---- Resumable (chunked) form ----------------------------------------------------------------
 * One input that arrives in pieces (from a file or a socket, into host memory) validated or
 * transcoded piece by piece, with the same results as one call on the whole input.  Not in the
 * paper, which transcodes whole buffers; it serves the disk- and network-rate inputs its
 * introduction motivates (Section 1).  Each push sees the characters the previous push held
 * back followed by the new chunk; it holds back a trailing incomplete character (at most three
 * bytes of a UTF-8 sequence whose leading byte is C2-F4, or one UTF-16 first surrogate) and runs
 * the single-buffer call on the rest, which starts and ends at character starts.  A push with
 * last != 0 holds nothing back, so an incomplete final character fails there (GBU_TOO_SHORT, or
 * GBU_SURROGATE for a final first surrogate).
 *
 * gbu_chunked_create: op is GBU_OP_VALIDATE_UTF8, _VALIDATE_UTF16LE, _CONVERT_UTF8_TO_UTF16LE or
 * _CONVERT_UTF16LE_TO_UTF8; max_chunk_units bounds n in each push.  Allocates its context,
 * device buffers and a stream here (never on a push).  NULL on failure.
 * gbu_chunked_push: chunk = n input code units in HOST memory (any host memory); out = HOST
 * buffer of out_cap output units (transcoders; may be NULL for validation).  Synchronous.
 *   *out_n  = output units written to out by this push (the outputs of consecutive pushes
 *             concatenate to the output of the whole input);
 *   *result = {GBU_OK, input units judged so far (validation) or output units written so far
 *             (transcoding)}; or the first error {kind, offset in input units from the start of
 *             the whole input} -- sticky: later pushes return it again and write nothing; or
 *             {GBU_OUTPUT_TOO_SMALL, units needed} when out_cap is too small for this push's
 *             output (nothing was consumed: repeat the push with a larger buffer); or GBU_TIMEOUT.
 *   Return value: GBU_OK, GBU_BAD_ARGUMENT (n > max_chunk_units, NULL pointers, misaligned
 *   UTF-16, a push after the last one) or GBU_CUDA_ERROR.
 * gbu_chunked_reset starts a new input; gbu_chunked_destroy frees everything. */
typedef struct gbu_chunked gbu_chunked;
gbu_chunked *gbu_chunked_create(int device, int op, uint64_t max_chunk_units);
int gbu_chunked_push(gbu_chunked *s, const void *chunk, uint64_t n, int last, void *out, uint64_t out_cap,
                     uint64_t *out_n, gbu_result *result);
int gbu_chunked_reset(gbu_chunked *s);
void gbu_chunked_destroy(gbu_chunked *s);

/* Number of kernel launches the library made through this context so far (for accounting). */
uint64_t gbu_launch_count(const gbu_ctx *ctx);

/* Launch geometry, for diagnostics and tests: writes up to n values into out (host memory):
 * the SM count; the CTAs per SM of the kernels behind validate_utf8, utf16_length_from_utf8,
 * convert_utf8_to_utf16le, validate_utf16le, utf8_length_from_utf16le and
 * convert_utf16le_to_utf8; the threads per CTA of the read-only kernels and of the
 * transcoders; the input bytes per warp tile of the read-only kernels; the input bytes per
 * transcoder partition (the unit of the look-back).  Returns the number of values written
 * (at most 11). */
int gbu_launch_config(const gbu_ctx *ctx, int32_t *out, int n);

#ifdef __cplusplus
}
#endif
#endif /* GBUTF_H */
