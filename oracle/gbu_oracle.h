/*
 * gbu_oracle.h -- scalar CPU reference codec for UTF-8, UTF-16 (LE and BE) and UTF-32.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU-baseline leg of the
 * benchmark call this code; the CUDA library never includes, links or calls it, and this code
 * includes nothing from the CUDA library.  Its enum values are its own and are matched to the
 * library's by name in the tests.
 *
 * What it computes follows the paper's Section 3 (the UTF-8 byte layout, the six validity
 * rules, and UTF-16 surrogate pairs) and Section 5 (every transcoding also validates).
 * Offsets, counts and capacities are in code units of the input or output format: bytes for
 * UTF-8, 16-bit units for UTF-16LE and UTF-16BE, 32-bit units for UTF-32.
 *
 * Parity status of each function is stated in oracle/gbu_oracle.c.
 */
#ifndef GBU_ORACLE_H
#define GBU_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Result kinds.  The six input-error kinds name the rule of Section 3 that fails first in
 * reading order; OR_OUTPUT_TOO_SMALL means the input was valid but dst could not hold it. */
enum {
  OR_OK = 0,
  OR_HEADER_BITS = 1,   /* rule 1: a byte whose five most significant bits are all ones   */
  OR_TOO_SHORT = 2,     /* rule 2: a leading byte without enough continuation bytes        */
  OR_TOO_LONG = 3,      /* rule 3: a continuation byte with no leading byte                */
  OR_OVERLONG = 4,      /* rule 4: value too small for the sequence length                 */
  OR_TOO_LARGE = 5,     /* rule 5: value of 1,114,112 or more                              */
  OR_SURROGATE = 6,     /* rule 6 (UTF-8) or an unpaired surrogate word (UTF-16)           */
  OR_OUTPUT_TOO_SMALL = 16
};

typedef struct {
  int32_t status;   /* one of the OR_* values                                            */
  int32_t reserved; /* always 0                                                          */
  uint64_t count;   /* OK: output units; input error: offset of the first invalid unit;  */
                    /* OR_OUTPUT_TOO_SMALL: output units the whole conversion needs      */
} or_result;

/* Validation.  OK -> count = n (every input unit was checked). */
or_result or_validate_utf8(const uint8_t *src, size_t n);
or_result or_validate_utf16le(const uint16_t *src, size_t n);

/* Output-length formulas, defined for any input (no validation). */
uint64_t or_utf16_length_from_utf8(const uint8_t *src, size_t n);
uint64_t or_utf8_length_from_utf16le(const uint16_t *src, size_t n);

/* Validating transcoders.  dst may be NULL only when cap == 0.  Units are written one at a
 * time, in order, and only at indices below cap: on OR_OUTPUT_TOO_SMALL dst[0:cap] holds the
 * first cap units of the conversion; on an input error dst holds the conversion of the valid
 * prefix src[0:count] (clipped to cap). */
or_result or_convert_utf8_to_utf16le(const uint8_t *src, size_t n, uint16_t *dst, size_t cap);
or_result or_convert_utf16le_to_utf8(const uint16_t *src, size_t n, uint8_t *dst, size_t cap);

/* UTF-16BE forms (RFC 2781 byte order: each word's most significant byte first in memory).
 * src / dst hold the words as they lie in memory; results as for the UTF-16LE forms. */
or_result or_validate_utf16be(const uint16_t *src, size_t n);
uint64_t or_utf8_length_from_utf16be(const uint16_t *src, size_t n);
or_result or_convert_utf16be_to_utf8(const uint16_t *src, size_t n, uint8_t *dst, size_t cap);
or_result or_convert_utf8_to_utf16be(const uint8_t *src, size_t n, uint16_t *dst, size_t cap);

/* UTF-32 (one 32-bit unit per value, host byte order).  A unit fails as rule 5 (>= 1,114,112:
 * OR_TOO_LARGE) or rule 6 (D800-DFFF: OR_SURROGATE) at its index.  The lengths are formulas for
 * any input: UTF-8 bytes by value (1/2/3/4), and one UTF-32 unit per non-continuation byte. */
or_result or_validate_utf32(const uint32_t *src, size_t n);
uint64_t or_utf8_length_from_utf32(const uint32_t *src, size_t n);
uint64_t or_utf32_length_from_utf8(const uint8_t *src, size_t n);
or_result or_convert_utf32_to_utf8(const uint32_t *src, size_t n, uint8_t *dst, size_t cap);
or_result or_convert_utf8_to_utf32(const uint8_t *src, size_t n, uint32_t *dst, size_t cap);
/* UTF-16LE <-> UTF-32: UTF-16 words by value (1 below 0x10000, else 2), and one UTF-32 unit per
 * word that is not a second surrogate (DC00-DFFF). */
uint64_t or_utf16_length_from_utf32(const uint32_t *src, size_t n);
uint64_t or_utf32_length_from_utf16le(const uint16_t *src, size_t n);
or_result or_convert_utf32_to_utf16le(const uint32_t *src, size_t n, uint16_t *dst, size_t cap);
or_result or_convert_utf16le_to_utf32(const uint16_t *src, size_t n, uint32_t *dst, size_t cap);

/* Batched forms: a plain loop over B strings given as CSR offsets (B+1 entries, in input code
 * units).  Transcoders write string i at dst + dst_off[i] with capacity
 * dst_off[i+1] - dst_off[i]. */
void or_validate_utf8_batched(const uint8_t *src, const uint64_t *off, size_t B, or_result *res);
void or_validate_utf16le_batched(const uint16_t *src, const uint64_t *off, size_t B,
                                 or_result *res);
void or_convert_utf8_to_utf16le_batched(const uint8_t *src, const uint64_t *off, size_t B,
                                        uint16_t *dst, const uint64_t *dst_off, or_result *res);
void or_convert_utf16le_to_utf8_batched(const uint16_t *src, const uint64_t *off, size_t B,
                                        uint8_t *dst, const uint64_t *dst_off, or_result *res);

#ifdef __cplusplus
}
#endif
#endif /* GBU_ORACLE_H */
