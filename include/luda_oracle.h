/*
 * luda_oracle.h -- TEST INFRASTRUCTURE: the C ABI of liboracle.so, the plain CPU
 * compactor under oracle/ that the tests, the smoke check and the benchmark's CPU
 * baseline check libluda against. Nothing in libluda includes this header, links the
 * oracle or calls it.
 *
 * luda_oracle_compact takes the arguments of luda_compact (luda.h) and computes the same
 * compaction job (LUDA, arXiv 2004.03054, §II-A: Phase 1 unpack, Phase 2 delete and sort,
 * Phase 3 pack; §III-A: the host hands over the job's input tables and takes the new
 * tables back) with the oracle's sequential steps. Its argument structs are declared
 * again below rather than included, because the oracle shares no header with the CUDA
 * path; each has the size and field offsets of its luda.h namesake
 * (luda_oracle_input = luda_input, luda_oracle_options = luda_options,
 * luda_oracle_table = luda_table, luda_oracle_outputs = luda_outputs; a test compiles
 * both headers and checks every offset), so the very same argument values can be passed
 * to either library.
 *
 * Semantics, against luda_compact:
 *   - inputs[].data are host pointers (newest first, as for luda_compact); level is
 *     recorded only; smallest_snapshot and opts->bottommost / block_size /
 *     restart_interval / bloom_bits_per_key / target_file_size / flags mean the same.
 *   - flags: LUDA_F_STRICT_DUP (1), LUDA_F_TRACE (2, no effect here), LUDA_F_SHORT_INDEX
 *     (4), LUDA_F_FILTER_ARRAY (8), LUDA_F_COMPRESS (16). Any other bit (including the
 *     device-only test flag 32) is LUDA_ERR_INVALID_ARG (-1).
 *   - dev_alloc, dev_free, alloc_ctx, stream and tuning are ignored (no device work).
 *   - On success *out holds the new tables in oracle-owned host memory (free with
 *     luda_oracle_outputs_free), n_in_entries and n_dropped; ms_device is the wall time
 *     of the compaction on the calling host thread (ms), ms_h2d = ms_d2h = 0, stage_ms and
 *     stage_bytes are zero.
 *   - On error the status (the luda_status values: -1 invalid argument, -2 corrupt input,
 *     -3 not supported, -4 out of memory, -7 duplicate key) is returned and stored in
 *     out->status, and *out holds no tables.
 */
#ifndef LUDA_ORACLE_H
#define LUDA_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  const uint8_t* data;
  uint64_t size;
  int32_t level;
  uint64_t file_number;
} luda_oracle_input;

typedef struct {
  uint32_t block_size;
  uint32_t restart_interval;
  uint32_t bloom_bits_per_key;
  uint64_t target_file_size;
  int32_t bottommost;
  uint32_t flags;
  void* dev_alloc;
  void* dev_free;
  void* alloc_ctx;
  void* stream;
  const void* tuning;
} luda_oracle_options;

typedef struct {
  uint8_t* data;
  uint64_t size;
  uint64_t n_entries;
  uint8_t* smallest;
  uint32_t smallest_len;
  uint8_t* largest;
  uint32_t largest_len;
} luda_oracle_table;

typedef struct {
  luda_oracle_table* tables;
  uint32_t n_tables;
  int32_t status;
  uint64_t n_in_entries;
  uint64_t n_dropped;
  double ms_h2d, ms_device, ms_d2h;
  double stage_ms[8];
  uint64_t stage_bytes[8];
  void* _priv;
} luda_oracle_outputs;

int luda_oracle_compact(const luda_oracle_input* inputs, uint32_t n_inputs, int32_t level,
                        uint64_t smallest_snapshot, const luda_oracle_options* opts, luda_oracle_outputs* out);
/* Frees what luda_oracle_compact stored in *out and zeroes it. */
void luda_oracle_outputs_free(luda_oracle_outputs* out);

#ifdef __cplusplus
}
#endif
#endif /* LUDA_ORACLE_H */
