/*
 * luda.h -- C ABI of libluda.so: SSTable compaction on one NVIDIA B300 (sm_103a).
 *
 * The operation is the compaction job of LUDA (arXiv 2004.03054): decode the selected
 * input tables (§II-A Phase 1 "Unpack": verify each data block's checksum, restore full
 * keys from shared prefixes), merge and sort all pairs by internal key and drop stale
 * and deleted versions (§II-A Phase 2 "(Delete and) Sort"), then pack the survivors
 * into new tables: data blocks cut by size, shared-prefix keys, checksums, index and
 * bloom filter (§II-A Phase 3 "Pack"; §III-C kernels unpack / shared_key / encode /
 * filter). The table format is this library's written LevelDB-style format: LEB128
 * varints, prefix-compressed keys with restart points, masked CRC-32C block trailers,
 * an unshortened index, a per-table MurmurHash3 bloom filter, no block compression.
 *
 * Every step runs in this library's CUDA kernels. There is no CPU fallback: a call on a
 * machine without a usable GPU returns LUDA_ERR_CUDA.
 *
 * Conventions, all entry points:
 *   - Inputs are caller-owned and never modified. Inputs of one job are listed newest
 *     first (level-0 tables newest to oldest, then the next level's tables in key order);
 *     on identical internal keys the earlier input wins.
 *   - Outputs are library-owned until luda_outputs_free. On any error *out holds no
 *     tables (all-or-nothing), `status` holds the error, and luda_last_error_detail()
 *     names the input and byte offset when the error is in an input.
 *   - Device pointers must stay readable up to the next 16-byte boundary past their end
 *     (every cudaMalloc / PyTorch CUDA allocation is).
 *   - Calls are thread-compatible: concurrent calls must use distinct streams.
 */
#ifndef LUDA_H
#define LUDA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LUDA_API __attribute__((visibility("default")))
#else
#define LUDA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LUDA_OK = 0,
  LUDA_ERR_INVALID_ARG = -1,   /* bad option, NULL pointer, unsorted run given to luda_build */
  LUDA_ERR_CORRUPTION = -2,    /* checksum, varint, offsets, footer, magic or key order */
  LUDA_ERR_NOT_SUPPORTED = -3, /* a block type other than 0 (raw) and 1 (compressed data block, R4c),
                                  a compressed index block, or a compressed data block where the entry
                                  point does not decompress (plans, the allocation-free check) */
  LUDA_ERR_OOM = -4,           /* device or pinned host allocation failed */
  LUDA_ERR_CUDA = -5,          /* a CUDA runtime call failed (no GPU, launch error) */
  LUDA_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
  LUDA_ERR_DUPLICATE_KEY = -7, /* identical internal keys in two inputs, with LUDA_F_STRICT_DUP */
  LUDA_ERR_PLAN_MISMATCH = -8  /* a plan was re-run on inputs whose sizes changed */
} luda_status;

/* options.flags */
#define LUDA_F_STRICT_DUP 1u /* identical internal keys across inputs are an error */
#define LUDA_F_SHORT_INDEX 4u /* write shortened index keys (format variant R9s: LevelDB's bytewise separator
                                 and short successor); decoders accept either kind */
#define LUDA_F_FILTER_ARRAY 8u /* write LevelDB's filter array (format variant R10a, after the bloom filter
                                  block of an SST in LUDA §II-A and LevelDB 1.22 of §IV-A): one bloom filter
                                  per 2 KiB of data block offsets, metaindex key "filter.luda.bloom2k";
                                  compactions do not read filter blocks, so inputs may carry either kind */
#define LUDA_F_COMPRESS 16u   /* write data blocks compressed (format variant R4c, LevelDB's Snappy type in the
                                 public stream format; the paper's future work, §IV-A) when that saves an
                                 eighth: the raw blocks go to scratch, one warp per block compresses them
                                 (64-byte segments parsed one per lane), the file cut and layout use the
                                 stored sizes. Compressed INPUT blocks are read without any flag. Unknown
                                 flags are LUDA_ERR_INVALID_ARG */
#define LUDA_F_TEST_WAIT0 32u /* test only: the staged encoder's bounded waits for its shared-memory copy slots
                                 give up at once (limit 0 instead of one second), as a wait that runs out
                                 would; the call then fails with LUDA_ERR_TIMEOUT and returns no tables. The
                                 bulk copies already issued are still waited for (one second at most) before
                                 each CTA exits, so the device stays usable */
#define LUDA_F_KEEP_DECODED 64u /* keep decoded runs on the device (§III-D: data stays in GPU memory between
                                   jobs). A call with this flag keeps, for each new table it returns on the
                                   device, the table's decoded run: its records (key prefix, trailer, key and
                                   value lengths, the value's CRC-32C register, the value's address inside
                                   the table) and full keys, in one store freed together with the tables
                                   (luda_outputs_free). A later call with this flag whose inputs are ALL
                                   tables with kept runs (same data pointer and size) takes its records from
                                   the runs and runs none of the footer, index, block walk, checksum and key
                                   kernels (§II-A Phase 1 ran when the tables were written); its tables are
                                   byte for byte those of the same call without the flag. A kept run stands
                                   for the table's bytes as they were written: a caller that changes a
                                   table's bytes on the device must not pass the flag for it. Tables written
                                   compressed (LUDA_F_COMPRESS), host outputs, ranged jobs (R13) and plans
                                   neither keep nor use runs. The store takes about 48 bytes per entry plus
                                   the keys */
#define LUDA_F_TRACE 2u      /* record per-stage device times (luda_outputs.stage_ms); LUDA_TRACE=1 in the
                                environment does the same for every call. Stage boundaries always open
                                NVTX ranges "luda/<stage>" on the calling thread. */

/* One input table. For the device entry points `data` is a device pointer. */
typedef struct {
  const uint8_t* data;
  uint64_t size;
  int32_t level;        /* informational */
  uint64_t file_number; /* informational */
} luda_input;

/* Device allocator hook (e.g. PyTorch's caching allocator). NULL = cudaMallocAsync on
 * the call's stream. `stream` is a cudaStream_t. */
typedef void* (*luda_alloc_fn)(size_t bytes, void* ctx, void* stream);
typedef void (*luda_free_fn)(void* ptr, void* ctx, void* stream);

/* Launch shapes of the pipeline's kernels. They decide how the work is split over CTAs
 * and never change a byte of the output: any valid tuning gives the same tables. 0 in a
 * field means the built-in default. luda_autotune measures candidates; a caller passes
 * the winner through luda_options.tuning. */
typedef struct {
  uint32_t merge_tile;          /* records per merge CTA: 512, 1024 or 2048 (default 512) */
  uint32_t merge_ctas_per_sm;   /* grid of each merge pass, CTAs per SM: 1..32 (default 16) */
  uint32_t decode_warps;        /* warps per CTA of the key rebuild, one data block each: 1..16 (default 4) */
  uint32_t walk_threads;        /* threads per CTA of the block walk, one block each: 32..256, multiple of 32
                                   (default 256) */
  uint32_t encode_ctas_per_sm;  /* staged encoder CTAs per SM: 1..8, capped by shared memory (default: as many
                                   as fit) */
  uint32_t elem_threads;        /* threads per CTA of the per-record and per-block kernels of the drop rule,
                                   cut and layout stages: 64..1024, multiple of 32 (default 256) */
  uint32_t crc_ctas;            /* CTAs (one per SM) of the data-block checksum kernels, which run beside the
                                   other stages on a second stream: the unpack's checksum pass, and the
                                   checksums of stored compressed blocks: 1..148 (default 56) */
  uint32_t crc_warps;           /* warps per CTA of the checksum kernels of compressed blocks: 8, 16, 24 or 32
                                   (default 32; the unpack's checksum pass always has 16); fewer leave room
                                   on their SMs for the other stages' CTAs */
  uint32_t h2d_ranges;          /* luda_compact (host buffers) only: key ranges the inputs are copied in, so
                                   that the tables of the first ranges are compacted and copied back while
                                   later ranges' input bytes are still arriving (§III-D); 1 = one copy in,
                                   one compaction, one copy out; 2..64; default: one range per
                                   max(96 MiB, target_file_size) of input, at most 16. The tables are
                                   byte-identical for every value */
} luda_tuning;

/* Fills the defaults (all fields 0). */
LUDA_API void luda_tuning_default(luda_tuning* t);
/* LUDA_OK if every field is 0 or in its range, else LUDA_ERR_INVALID_ARG with the field
 * named in luda_last_error_detail. */
LUDA_API luda_status luda_tuning_check(const luda_tuning* t);

typedef struct {
  uint32_t block_size;          /* T: a data block is closed once its size reaches T (>= 1) */
  uint32_t restart_interval;    /* R: every R-th entry of a block is a restart (1..65535) */
  uint32_t bloom_bits_per_key;  /* bloom filter bits per entry (1..64); k = bpk*69/100 probes */
  uint64_t target_file_size;    /* a table is finished once its data blocks reach this (>= 1) */
  int32_t bottommost;           /* drop tombstones visible at the snapshot (single-job calls) */
  uint32_t flags;               /* LUDA_F_* */
  luda_alloc_fn dev_alloc;
  luda_free_fn dev_free;
  void* alloc_ctx;
  void* stream;                 /* cudaStream_t; NULL = the legacy default stream */
  const luda_tuning* tuning;    /* launch shapes; NULL = defaults. Read during the call (plans: during
                                   luda_plan_create) and not kept */
} luda_options;

/* Defaults: T = 4096, R = 16, bpk = 10, target = 2 MiB, not bottommost, no flags. */
LUDA_API void luda_options_default(luda_options* o);

/* One output table. `data` is a host pointer for the host entry points and a device
 * pointer for the *_device ones; `smallest`/`largest` (internal keys) are always host
 * pointers. */
typedef struct {
  uint8_t* data;
  uint64_t size;
  uint64_t n_entries;
  uint8_t* smallest;
  uint32_t smallest_len;
  uint8_t* largest;
  uint32_t largest_len;
} luda_table;

#define LUDA_N_STAGES 8

typedef struct {
  luda_table* tables;
  uint32_t n_tables;
  int32_t status;               /* luda_status of this job */
  uint64_t n_in_entries;        /* entries decoded from the inputs */
  uint64_t n_dropped;           /* entries removed by the drop rule */
  double ms_h2d, ms_device, ms_d2h;
  /* With LUDA_F_TRACE, CUDA-event times on the call's stream (ms) and algorithmic bytes
   * (a batch call reports its stages, which all its jobs share, in every job's outputs):
   *  [0] sizing (footers, index, block scan, prefix sums; includes host round trips)
   *  [1] the unpack's checksum pass (CRC-32C of every input data block and the values'
   *      CRC registers; it runs on a second stream beside stages 2-4); bytes = input data
   *      blocks with trailers
   *  [2] records and keys kernel alone      [3] order check + merge sort
   *  [4] drop rule, entry sizes, block and file cut, layout
   *  [5] encode kernel alone (block images without their CRC): bytes = output data
   *      blocks written + survivor keys and values read
   *  [6] the rest after the encoder: data block CRC trailers (assembled from the pieces'
   *      registers), joined with the filter, index, metaindex and footer kernels that ran
   *      beside the encoder
   *  [7] whole device span */
  double stage_ms[LUDA_N_STAGES];
  uint64_t stage_bytes[LUDA_N_STAGES];
  void* _priv;                  /* library bookkeeping: do not touch */
} luda_outputs;

/* ---- single compaction job ------------------------------------------------------------
 * luda_compact: inputs[].data are host pointers (pinned memory gives the fastest copies);
 *   the library copies them to the device (timed in ms_h2d), compacts, and copies the new
 *   tables back into library-owned pinned host memory (ms_d2h). A job of two or more
 *   transfer ranges (luda_tuning.h2d_ranges; by default one per 96 MiB or the target size
 *   of input, so jobs of 192 MiB and more) overlaps the two directions (§III-D): the footers and
 *   index blocks are copied and parsed first, the data blocks follow range by range (user
 *   keys chosen from the index keys so that the ranges hold about equal bytes), each range
 *   is compacted once its blocks have arrived and its finished tables are copied back
 *   while later ranges arrive. The last table of a range, back to one that starts a new
 *   user key, is compacted again with the next range, so the tables are byte-identical to
 *   those of the job in one piece. ms_device then sums the ranges' device times (and
 *   stage_ms their stages); ms_h2d and ms_d2h span each direction's copies. A job whose
 *   footers or index blocks do not parse, or whose index keys are out of order, runs in
 *   one piece (which reports the error).
 * luda_compact_device: inputs[].data are device pointers on opts->stream; the new tables
 *   stay on the device in one library-owned allocation.
 * `level` is the output level (recorded only); `smallest_snapshot` is the oldest sequence
 *   number any reader may still see ((1<<56)-1 when there are no snapshots).
 * Input data blocks may be stored compressed (type 1, format rule R4c, the public Snappy
 *   stream format; the Snappy compression the paper leaves to future work, §IV-A): their
 *   checksums are verified on the stored bytes, then they are decompressed on the device
 *   into a scratch arena (one warp per block) and sized a second time from their contents
 *   (one more host round trip, only when such blocks are present). A stream that does not
 *   decode to its announced length is LUDA_ERR_CORRUPTION. Output blocks are written
 *   compressed with LUDA_F_COMPRESS, else raw. */
LUDA_API luda_status luda_compact(const luda_input* inputs, uint32_t n_inputs, int32_t level, uint64_t smallest_snapshot,
                         const luda_options* opts, luda_outputs* out);
LUDA_API luda_status luda_compact_device(const luda_input* inputs, uint32_t n_inputs, int32_t level,
                                uint64_t smallest_snapshot, const luda_options* opts, luda_outputs* out);

/* ---- many independent jobs in one launch sequence ------------------------------------ */
typedef struct {
  const luda_input* inputs;   /* device pointers */
  uint32_t n_inputs;
  int32_t level;
  uint64_t smallest_snapshot;
  int32_t bottommost;
  /* Optional user-key range [range_lo, range_hi) (format rule R13; host pointers, NULL =
   * unbounded): the job reads only the data blocks that can hold keys of the range and
   * writes only those keys. Not supported by plans (luda_plan_create rejects it). */
  const uint8_t* range_lo;
  uint32_t range_lo_len;
  const uint8_t* range_hi;
  uint32_t range_hi_len;
} luda_job;

/* A user key (host memory). */
typedef struct {
  const uint8_t* data;
  uint32_t len;
} luda_key;

/* Compacts n_jobs jobs together: every kernel of the pipeline runs once over all jobs'
 * work. outs[j] receives job j's tables (device pointers) and status; a corrupt job fails
 * alone. Returns LUDA_OK when the batch ran (check each outs[j].status), else the error
 * that stopped the whole batch. */
LUDA_API luda_status luda_batch_compact_device(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts,
                                      luda_outputs* outs);
/* The same with host buffers (§III-A: the host hands the GPU the tables of each selected
 * job and takes the new tables back): jobs[j].inputs[].data are host pointers (pinned
 * memory gives the fastest copies). Every job's inputs are copied into one device arena
 * (one copy per input, on opts->stream; ms_h2d), all jobs run as one batch as above, and
 * the new tables of all jobs come back in one copy into library-owned pinned host memory
 * (ms_d2h): outs[j].tables[].data are host pointers. A corrupt job fails alone (its
 * outs[j].status, no tables); an error that stops the whole batch is returned and set in
 * every outs[j].status, with no tables anywhere. */
LUDA_API luda_status luda_batch_compact(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts,
                                        luda_outputs* outs);

/* ---- subcompactions (format rule R13) --------------------------------------------------
 * One job split at the strictly increasing user keys bounds[0..n_bounds) into n_bounds + 1
 * ranged jobs, run together as one batch; *out receives their tables concatenated in key
 * order (device pointers, as luda_compact_device), n_in_entries and n_dropped summed, and
 * the first failing range's status. The entries written are exactly those of the whole
 * job; only the file cut differs (each range starts its own tables). */
LUDA_API luda_status luda_subcompact_device(const luda_input* inputs, uint32_t n_inputs, int32_t level,
                                            uint64_t smallest_snapshot, const luda_key* bounds, uint32_t n_bounds,
                                            const luda_options* opts, luda_outputs* out);

/* ---- plans: a batch sized once, captured in a CUDA graph, replayed --------------------
 * luda_plan_create runs the sizing pass on the jobs' device inputs, allocates every
 * buffer and captures the whole pipeline (decode to footers, all jobs) into one CUDA
 * graph. luda_plan_run replays it on `stream`; every replay redoes all the work from the
 * input bytes and checks on the device that the sizes still match the plan
 * (LUDA_ERR_PLAN_MISMATCH otherwise). The inputs must stay valid and unchanged in size
 * for the plan's life. luda_plan_outputs gives each job's tables from the last run
 * (device pointers into the plan, valid until the next run or destroy). A job whose
 * inputs hold compressed data blocks (R4c) reports LUDA_ERR_NOT_SUPPORTED in its outputs:
 * a plan is sized from the stored blocks and does not decompress. */
typedef struct luda_plan luda_plan;
LUDA_API luda_status luda_plan_create(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts, luda_plan** plan);
LUDA_API luda_status luda_plan_run(luda_plan* plan, void* stream);
LUDA_API luda_status luda_plan_outputs(luda_plan* plan, luda_outputs* outs);
LUDA_API void luda_plan_destroy(luda_plan* plan);

/* ---- autotuner: time candidate launch shapes on a batch -------------------------------
 * For each of the n_candidates tunings, builds a plan of the jobs with opts and that
 * tuning, replays it once untimed and then `reps` times (>= 1) between CUDA events on the
 * plan's stream, and writes the median replay time in ms to ms[i] (a candidate that fails
 * gets a negative ms[i] and does not stop the others). *best receives the index of the
 * fastest candidate. Plans are built and destroyed one at a time, so the device holds one
 * plan's memory at most. opts->tuning is ignored. Returns LUDA_ERR_INVALID_ARG for an
 * invalid candidate or NULL arguments, else the first error if every candidate failed,
 * else LUDA_OK. */
LUDA_API luda_status luda_autotune(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts,
                                   const luda_tuning* candidates, uint32_t n_candidates, uint32_t reps, double* ms,
                                   uint32_t* best);

/* ---- serving: continuous batching of compaction jobs ----------------------------------
 * A server takes compaction jobs as they arise (for example from an LSM tree whose tables
 * stay resident in device memory) and runs up to n_slots of them at once, each on its own
 * CUDA stream driven by its own host thread, so that the jobs' kernels overlap on the GPU.
 * A job that a slot has taken first runs its sizing pass (footers, index, block scan);
 * it is then admitted only when the device bytes it will hold at its peak fit in
 * hbm_budget together with those of the jobs already admitted. Admission is first come,
 * first served; a job larger than the whole budget is admitted once no other job holds
 * any. The sizing pass's own buffers (well under 1% of the inputs for blocks of 4 KiB or
 * more) are not counted. A job's new tables (device memory) leave the budget when it
 * completes; the caller owns them from luda_server_wait on.
 *
 * Results do not depend on the mix: each job's tables are byte-identical to those of
 * luda_compact_device on the same inputs.
 *
 * luda_server_submit copies the job description (the luda_input array too); the input
 * tables themselves must stay valid until the job completes. luda_server_next returns the
 * ticket of a completed job that no luda_server_next has returned yet (LUDA_ERR_TIMEOUT if
 * none completes within timeout_ms; timeout_ms < 0 waits without limit).
 * luda_server_wait waits for one ticket (same timeout rule), moves its tables into *out
 * (free with luda_outputs_free) and fills *stats (may be NULL); the ticket is then gone.
 * It returns the job's status, or LUDA_ERR_TIMEOUT when the job has not completed in
 * time (the ticket then stays valid; no job itself ends with LUDA_ERR_TIMEOUT). luda_server_destroy waits for every submitted job to
 * complete, frees the tables no one collected and ends the slots' threads. Submit, next
 * and wait may be called from any host thread. */
typedef struct luda_server luda_server;

typedef struct {
  uint32_t n_slots;        /* jobs that may run at once (1..64) */
  uint64_t hbm_budget;     /* device bytes the admitted jobs may hold at once (> 0) */
  luda_options opts;       /* format options of every job; opts.stream is ignored and
                              opts.bottommost is replaced by each job's own flag */
  uint64_t prewarm_bytes;  /* device bytes allocated and freed at creation (opts.dev_alloc NULL: the
                              stream-ordered pool keeps them), so that early jobs do not wait for the
                              driver to map memory; 0 = none. Each slot also sets up its per-thread
                              state (second stream, pinned staging) before taking jobs. */
} luda_server_config;

typedef struct {
  double queue_ms;         /* submit -> a slot took the job */
  double admit_wait_ms;    /* end of sizing -> admitted */
  double run_ms;           /* a slot took the job -> completed */
  double latency_ms;       /* submit -> completed */
  uint64_t reserved_bytes; /* peak device bytes the job was admitted with */
  uint64_t input_bytes;    /* sum of the job's input table sizes */
  uint32_t slot;           /* the slot (stream) that ran it */
  uint32_t running_at_admit; /* admitted jobs, this one included, when it was admitted */
} luda_job_stats;

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t budget_peak;    /* highest sum of admitted jobs' reserved bytes */
  uint32_t running_peak;   /* most jobs admitted at once */
  uint32_t pad;
} luda_server_stats;

LUDA_API luda_status luda_server_create(const luda_server_config* cfg, luda_server** server);
LUDA_API luda_status luda_server_submit(luda_server* server, const luda_job* job, uint64_t* ticket);
/* As luda_server_submit, for a job whose input tables are in host memory (pinned memory
 * gives the fastest copies): the slot copies them to the device, compacts, and copies the
 * new tables back into library-owned pinned host memory (as luda_compact). The device
 * copy of the inputs counts against the budget. With two or more slots the copies of
 * different jobs overlap (one job's inputs going in while another's tables come out). */
LUDA_API luda_status luda_server_submit_host(luda_server* server, const luda_job* job, uint64_t* ticket);
LUDA_API luda_status luda_server_next(luda_server* server, int64_t timeout_ms, uint64_t* ticket);
LUDA_API luda_status luda_server_wait(luda_server* server, uint64_t ticket, int64_t timeout_ms, luda_outputs* out,
                                      luda_job_stats* stats);
LUDA_API luda_status luda_server_stats_get(luda_server* server, luda_server_stats* stats);
LUDA_API void luda_server_destroy(luda_server* server);

/* ---- table builder (memtable flush) ---------------------------------------------------
 * Packs one run of entries already in increasing internal-key order (user key ascending;
 * for equal user keys, sequence descending) into tables, cutting files at the target
 * size, with the same encoder as a compaction. ukeys/vals are concatenated bytes with
 * n+1 offsets; types 1 = put, 0 = delete; seqs < 2^56. Unsorted input is
 * LUDA_ERR_INVALID_ARG. luda_build takes host arrays and returns host tables;
 * luda_build_device takes device arrays and returns device tables. */
typedef struct {
  const uint8_t* ukeys;
  const uint64_t* ukoff;
  const uint64_t* seqs;
  const uint8_t* types;
  const uint8_t* vals;
  const uint64_t* voff;
  uint64_t n;
} luda_run;

LUDA_API luda_status luda_build(const luda_run* run, const luda_options* opts, luda_outputs* out);
LUDA_API luda_status luda_build_device(const luda_run* run, const luda_options* opts, luda_outputs* out);

/* ---- table check without allocation ----------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that cannot
 * allocate device memory when they need to check a table: code running inside a custom
 * allocator or memory-pool callback (a nested cudaMalloc would re-enter it), storage
 * engines that reserve all device memory at start-up, and paths that cannot afford an
 * allocation's implicit synchronisation.
 *
 * luda_check_table_noalloc runs the checks of a compaction's sizing pass on one table
 * and counts its entries, without allocating. It checks: the footer (magic, block
 * handles inside the file); the index block's CRC-32C, type byte and entry structure
 * (varints, restart array, handles of the data blocks inside the file and in order); and
 * every data block's CRC-32C, type byte and entry structure (varints, shared prefix no
 * longer than the previous key, restart array, entry and key byte counts). It does NOT
 * check what a compaction checks only after decoding the keys: the internal-key order
 * within the table and the index-key rule (each index key at or after its block's last
 * key and before the next block's first key). A table with valid checksums but two keys
 * out of order passes this check and then fails a compaction with LUDA_ERR_CORRUPTION.
 * `table` is a device pointer to `size` bytes on `stream` (a cudaStream_t, NULL = legacy
 * default), in device or managed memory of the current device (cudaPointerGetAttributes;
 * anything else, e.g. a host pointer, is LUDA_ERR_INVALID_ARG before any launch). It
 * calls no cudaMalloc, cudaFree or other allocating routine: its scratch and CRC tables
 * are static device arrays, at most LUDA_NOALLOC_STATIC_BYTES per GPU that loads the
 * library, held until the process exits; the scratch limits it to tables of at most
 * LUDA_NOALLOC_MAX_BLOCKS data blocks (larger tables: LUDA_ERR_INVALID_ARG with a
 * message naming the limit). The scratch is shared by all calls and keeps the last
 * call's contents; each call clears what it needs. Calls that overlap on the GPU race:
 * serialise them. The first call on a device (with that device current) looks up the
 * scratch with cudaGetSymbolAddress and uploads CRC tables with cudaMemcpyToSymbol;
 * make that first call before any stream capture. Returns the table's status (also in
 * out->status); on a corrupt table out->bad_offset is the byte offset of the fault. A
 * compressed data block (type 1, R4c) is checked up to its checksum and then reported as
 * LUDA_ERR_NOT_SUPPORTED: its structure is behind a decompression, which needs memory. */
#define LUDA_NOALLOC_MAX_BLOCKS 16384u
#define LUDA_NOALLOC_STATIC_BYTES (1200u * 1024u) /* scratch (block descriptors and counts) + CRC tables */

typedef struct {
  int32_t status;       /* luda_status */
  uint32_t n_blocks;    /* data blocks listed in the index */
  uint64_t n_entries;   /* entries in all data blocks (valid when status == LUDA_OK) */
  uint64_t data_bytes;  /* data block bytes including trailers (valid when LUDA_OK) */
  uint64_t bad_offset;  /* byte offset of the fault when status is an error */
} luda_table_check;

LUDA_API luda_status luda_check_table_noalloc(const uint8_t* table, uint64_t size, void* stream,
                                              luda_table_check* out);

/* Frees everything an entry point stored in *out (host and device memory). Device tables
 * the library allocated go back stream-ordered on the legacy default stream (after the work
 * queued there and on every blocking stream; no device-wide wait): work on a non-blocking
 * stream that still reads them must have completed, or been waited for, before this call.
 * With a caller's allocator (luda_options.dev_free) the memory goes to dev_free(ptr, ctx,
 * NULL). */
LUDA_API void luda_outputs_free(luda_outputs* out);

LUDA_API const char* luda_strerror(luda_status s);
/* Thread-local text for the last error of this thread's last call ("" if none). */
LUDA_API const char* luda_last_error_detail(void);
/* Library version string. */
LUDA_API const char* luda_version(void);
/* Number of CUDA kernels this library has launched in this process so far. */
LUDA_API uint64_t luda_launch_count(void);
/* Number of input tables whose records came from kept decoded runs (LUDA_F_KEEP_DECODED)
 * in this process so far. */
LUDA_API uint64_t luda_kept_inputs_used(void);

#ifdef __cplusplus
}
#endif
#endif /* LUDA_H */
