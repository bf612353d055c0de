// internal.cuh -- data structures and kernel launchers shared by the pipeline stages.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "crc.cuh"
#include "luda.h"

namespace luda {

// ---- batch description ----------------------------------------------------------------
struct DInput {
  const uint8_t* data;  // device address of the table image
  uint64_t size;
  uint32_t job;         // owning job
  uint32_t local;       // index of the input within its job (error reports)
  uint64_t idx_off;     // index block handle, set by the footer kernel
  uint64_t idx_size;
  uint32_t nblk;        // data blocks listed in the index, set by the footer kernel
  uint32_t blk_first;   // first global data-block id, set by the host
};

// Unpack: chunks of kChunk bytes (crc.cuh) per data block with piece boundaries; the walk
// records each block's chunk count when the block takes that path (kUnpChunkMax at most).
constexpr uint32_t kUnpChunkMax = 240;

struct BlockDesc {
  const uint8_t* ptr;   // block contents
  uint64_t size;        // contents size (trailer excluded)
  uint64_t off;         // offset within its input (error reports)
  uint32_t input;       // global input index
  uint32_t job;
  const uint8_t* ikey;  // the block's index key (its last internal key, checked after decode)
  uint32_t ilen;
  uint32_t pad;
};

// A job's user-key range (R13): bounds are bytes of the call's bound buffer.
struct JobRange {
  uint32_t lo_off, lo_len, hi_off, hi_len;
  uint32_t flags;  // 1: lo present, 2: hi present
};

// R13: is the user key u inside its job's range [lo, hi)?
__device__ __forceinline__ bool key_in_range(const JobRange& r, const uint8_t* bounds, const uint8_t* u, uint32_t n) {
  if ((r.flags & 1u) && cmp_user_keys(u, n, bounds + r.lo_off, r.lo_len) < 0) return false;
  if ((r.flags & 2u) && cmp_user_keys(u, n, bounds + r.hi_off, r.hi_len) >= 0) return false;
  return true;
}

struct JobDev {
  uint64_t snapshot;
  uint32_t bottommost;
  uint32_t flags;
  uint32_t rec_begin, rec_end;    // decoded records (set by the host after sizing)
  uint32_t surv_begin, surv_end;  // survivors (device)
  uint32_t blk_begin, blk_end;    // output data blocks (device)
  uint32_t file_begin, file_end;  // output tables (device)
  uint64_t n_in;                  // entries decoded
  uint64_t out_bytes;             // bytes of this job's tables (device)
  uint32_t in_first;              // first global input index of the job
  uint32_t pad;
};

struct FileDesc {
  uint64_t off;          // offset of the table image in the output arena
  uint64_t size;         // image size
  uint64_t data_size;    // data blocks with trailers
  uint64_t filter_size;  // filter contents (bitmap + k)
  uint64_t meta_off, meta_size;
  uint64_t index_off, index_size;
  uint64_t bm_word;      // first 32-bit word of this table's bitmap in the scratch
  uint32_t blk_begin, blk_end;  // output data blocks
  uint32_t ent_begin, ent_end;  // survivor positions
  uint32_t job;
  uint32_t n_filt;       // filters of the filter array (LUDA_F_FILTER_ARRAY)
  uint64_t bm_bits;      // filter bits (one filter per table)
};

struct Fmt {
  uint32_t T;       // block size threshold
  uint32_t R;       // restart interval
  uint32_t bpk;     // bloom bits per key
  uint32_t k;       // bloom probes
  uint64_t target;  // target file size
  uint32_t max_kv;  // largest internal key + value length of the inputs (0: unknown)
  uint32_t flags;   // luda_options.flags
};

// Device-side counts of the stages whose sizes only the device knows.
struct Counts {
  uint32_t n_rec;     // decoded records (host-set)
  uint32_t n_surv;    // survivors of the drop rule
  uint32_t nb;        // output data blocks
  uint32_t nf;        // output tables
  uint64_t out_bytes; // bytes of all table images
  uint64_t bm_words;  // bloom bitmap words
  uint64_t key_bytes; // gathered smallest/largest key bytes
  uint64_t in_data_bytes;   // input data blocks with trailers (block scan)
  uint64_t surv_kv_bytes;   // survivor keys + values (read by the encoder)
  uint32_t gap_surv;        // largest next(i) - i of the block cut
  uint32_t gap_blk;         // largest next(b) - b of the file cut
  uint32_t big_blocks;      // data blocks left to the CTA-per-block encoder
  uint32_t max_kv;          // largest internal key + value length in the inputs (block walk)
  uint32_t crc_next_in;     // next input data block for the checksum kernels' warps
  uint32_t crc_next_out;    // next output data block for the trailer kernels' warps
  uint32_t unp_next;        // next data block for the unpack's checksum pass
  uint32_t n_filt;          // filters of all tables' filter arrays (LUDA_F_FILTER_ARRAY)
  uint32_t comp_blocks;     // compressed input data blocks (R4c) seen by the block walk
  uint64_t comp_bytes;      // arena bytes their contents take once decompressed
};

// The filter arrays of a batch (LUDA_F_FILTER_ARRAY; base == nullptr otherwise). Filter s
// of all tables: table f owns filters [base[f], base[f + 1]); its filter i covers the data
// blocks starting in [i, i + 1) * 2 KiB of the table. boff / woff: exclusive sums of the
// filters' bytes (bitmap and k, zero when empty) and of their bitmap words; bytes: each
// filter's bytes. cap: filters the buffers hold.
constexpr uint32_t kFilterBaseLg = 11;
struct FiltArr {
  const uint64_t* base;
  const uint64_t* boff;
  const uint64_t* woff;
  const uint64_t* bytes;
  uint64_t cap;
};

// One message for the multi-warp CRC (index and filter blocks): n bytes at p (contents and
// type byte); the masked CRC is written to out, or with verify compared with the one
// stored at out (a mismatch is reported for job / local input at byte offset where).
struct CrcMsg {
  const uint8_t* p;
  uint64_t n;
  uint8_t* out;
  uint64_t where;
  uint32_t job, local;
  uint32_t verify;
  uint32_t acc;  // XOR of the chunks' shifted registers (zero when queued)
};

// Merge key of a record: the first 32 bytes of its user key as four big-endian words
// (zero-padded).
struct __align__(16) MKey {
  uint64_t h[4];
};

// Per output data block: where and what the encoder writes.
struct BlkEnc {
  uint64_t dst;       // byte offset of the block in the output arena
  uint32_t s0, m;     // first survivor, entries
  uint32_t contents;  // contents size (without the trailer)
  uint32_t job;       // job index; bit 31: outside the output arena (skip)
};

// Per survivor, in survivor order: what the encoder reads of its record.
struct EncDesc {
  uint64_t kptr;  // device address of the full internal key (key arena)
  uint64_t vptr;  // device address of the value (input table)
  uint32_t klen, vlen;
  uint32_t rec;   // the survivor's record
  uint32_t pad;
};

// Per-output-table summary copied to the host at the end.
struct FileMeta {
  uint64_t off, size, n_entries, data_size;
  uint64_t small_koff, large_koff;  // in the key gather buffer
  uint32_t small_len, large_len;
  uint32_t job;
  uint32_t max_kv;               // kept runs (LUDA_F_KEEP_DECODED): largest key + value length
  uint64_t key_first, kbytes;    // kept runs: the table's keys in the store's key arena
};

// ---- keep.cu: decoded runs kept between compactions (LUDA_F_KEEP_DECODED) ------------------
// One store per call: the survivors in output order, their full keys back to back in
// `arena` (koff: offsets, exclusive scan of klen), each value's address inside the new
// data blocks (vptr) and its CRC-32C register (vcrc).
struct KeptRecs {
  uint64_t *pfx, *tr, *koff, *vptr;
  uint32_t *klen, *vlen, *vcrc;
  uint8_t* arena;
};
// One input of a call whose records come from a kept run: survivors [first, first + count)
// of `run`, whose keys start at key_first in the run's arena; they become records
// [rec_base, rec_base + count) with keys from key_base in the call's arena.
struct KeptIn {
  KeptRecs run;
  uint64_t first, count, key_first, rec_base, key_base;
};

// ---- launch geometry --------------------------------------------------------------------
// Every launcher adds its kernel launches here (luda_launch_count).
void count_launches(uint32_t n);
// Sets the calling thread's luda_last_error_detail() text.
void set_error_detail(const char* text);

inline unsigned grid_for(uint64_t work, unsigned per_cta, unsigned max_ctas = kSms * 16) {
  uint64_t g = (work + per_cta - 1) / per_cta;
  if (g < 1) g = 1;
  if (g > max_ctas) g = max_ctas;
  return unsigned(g);
}

// ---- launch shapes (luda_tuning) ----------------------------------------------------------
// The launchers read the calling thread's current tuning; an entry point installs the
// caller's (luda_options.tuning) for its duration with a TuningScope. Defaults resolved:
struct Tuning {
  uint32_t merge_tile = 512;
  uint32_t merge_ctas_per_sm = 16;
  uint32_t decode_warps = 4;  // warps per CTA of the key rebuild (k_keys)
  uint32_t walk_threads = 256;
  uint32_t encode_ctas_per_sm = 0;  // 0: as many as shared memory allows
  uint32_t elem_threads = 256;
  uint32_t crc_ctas = 56;  // the unpack's checksum pass: the other stages run beside it on the rest
  uint32_t crc_warps = 32;
  uint32_t h2d_ranges = 0;  // luda_compact's transfer ranges (0: from the input bytes and target size)
};
const Tuning& tuning();
// Range check of a luda_tuning (0 = default); sets the error detail on failure.
bool tuning_valid(const luda_tuning* t);
class TuningScope {
 public:
  explicit TuningScope(const luda_tuning* t);  // t must be valid (or NULL)
  ~TuningScope();
  TuningScope(const TuningScope&) = delete;
  TuningScope& operator=(const TuningScope&) = delete;

 private:
  Tuning saved_;
};
// CTA size of the per-record and per-block kernels of the drop rule, cut and layout stages.
inline unsigned elem_threads() { return tuning().elem_threads; }

// Lets `kernel` use `bytes` of dynamic shared memory on the current device. The attribute
// call takes a driver lock and costs more than a small launch, so each thread remembers
// the largest size it has set per kernel and device.
void smem_optin_raw(const void* kernel, int bytes);
template <class K>
inline void smem_optin(K* kernel, uint32_t bytes) {
  smem_optin_raw(reinterpret_cast<const void*>(kernel), int(bytes));
}

// ---- scan.cu ----------------------------------------------------------------------------
uint64_t scan_temp_bytes(uint64_t n);
template <typename In, typename Out>
cudaError_t exclusive_scan(const In* in, Out* out, uint64_t cap, const uint32_t* count, void* temp,
                           cudaStream_t st);

// ---- crc_tables.cu ------------------------------------------------------------------------
bool make_crc_tables(uint32_t* slice, uint32_t* shift);
bool make_chunk_tables(uint32_t* out);

// ---- decode.cu ---------------------------------------------------------------------------
// Footers and index block checksums of n_inputs tables; msgs: n_inputs entries of scratch.
void launch_footers(DInput* in, uint32_t n_inputs, DErr* errs, CrcMsg* msgs, CrcTabs tabs, cudaStream_t st);
// launch_footers in three parts, so that the index blocks' checksums can run on another
// stream: the footers (queueing one checksum message per index block), the checksums,
// and the index block counts.
void launch_footers_read(DInput* in, uint32_t n_inputs, DErr* errs, CrcMsg* msgs, cudaStream_t st);
void launch_index_crc(CrcMsg* msgs, uint32_t n_inputs, DErr* errs, CrcTabs tabs, cudaStream_t st);
void launch_footers_finish(DInput* in, uint32_t n_inputs, DErr* errs, cudaStream_t st);
// With ranges (one JobRange per job, bound bytes in `bounds`), a block no key of its job's
// range can be in gets a null ptr (it is neither checked nor decoded).
void launch_index_entries(const DInput* in, uint32_t n_inputs, const uint32_t* in_blk_first, uint32_t n_blocks,
                          BlockDesc* blocks, DErr* errs, cudaStream_t st, const JobRange* ranges = nullptr,
                          const uint8_t* bounds = nullptr);
// The block walk's entry table: for the first kHdrMax entries of a block (blocks below
// 64 KiB), x = entry offset | value offset << 16, y = value end | shared << 16 | non-shared
// << 24 (key lengths clamped to 255; keys over 128 bytes are rebuilt by the sequential walk).
constexpr uint32_t kHdrMax = 64;
void launch_block_scan(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, uint32_t* nrec,
                       uint64_t* kbytes, DErr* errs, Counts* cnt, uint2* ent_tab, CrcTabs tabs, cudaStream_t st,
                       uint32_t* nch = nullptr);
// The two halves of launch_block_scan, for callers that run them on different streams:
// checksum and type byte (errors into verr; blocks of jobs failed in errs or verr are
// skipped), and the structure walk with entry counts.
// Input checksums. Warps take blocks from the counter *next (zero before the first
// launch); a helper launch (helper = true) on another stream adds the SMs the first launch
// left (148 - crc_ctas) and ends at once if no block is left.
void launch_block_verify(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, const DErr* errs, DErr* verr,
                         CrcTabs tabs, uint32_t* next, bool helper, cudaStream_t st);
// With nch given, nch[g] = the block's chunk count when the unpack takes it with piece
// boundaries (at most kHdrMax entries, below 64 KiB, at most kUnpChunkMax chunks), else 0.
void launch_block_walk(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, uint32_t* nrec,
                       uint64_t* kbytes, DErr* errs, Counts* cnt, uint2* ent_tab, cudaStream_t st,
                       uint64_t* ulen = nullptr, uint64_t* ures = nullptr, bool contents = false,
                       uint32_t* nch = nullptr);
// R4c: compressed data blocks (ulen[g] != kRawBlock) decompressed into dst + uoff[g], one
// warp per block; cblocks[g] (a copy of blocks[g]) then points at the contents.
constexpr uint64_t kRawBlock = ~0ull;
void launch_decompress(const BlockDesc* blocks, uint32_t n_blocks, const uint64_t* ulen, const uint64_t* uoff,
                       uint8_t* dst, uint64_t dst_cap, BlockDesc* cblocks, const DInput* in, DErr* errs,
                       cudaStream_t st);
// After decode: every data block's index key equals its last internal key.
void launch_check_index(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, const uint32_t* nrec,
                        const uint32_t* rec_first, Recs recs, const uint8_t* arena, DErr* errs, cudaStream_t st);
// link[i] = 1 when input i + 1 continues input i's sorted run (same job, disjoint and in
// order); needs the block descriptors and the inputs' blk_first.
void launch_run_links(const DInput* in, uint32_t n_inputs, const BlockDesc* blocks, const DErr* errs, uint8_t* link,
                      cudaStream_t st);
// Blocks of failed jobs and blocks not read (null ptr) hold no records.
void launch_zero_failed(const BlockDesc* blocks, uint32_t n_blocks, const DErr* errs, uint32_t* nrec,
                        uint64_t* kbytes, cudaStream_t st);
// The unpack of every data block: records and rebuilt keys, and from one read of the
// block's bytes with `verify` the block checksum and type byte (errors into verr) and each
// value's CRC register (recs.vcrc); only blocks with entries (nrec[g] > 0; with plan_nrec
// given, only when the entry and key counts match the plan) have records. chunk_first: exclusive scan of the walk's chunk counts (n_blocks + 1);
// chunkF: chunk_first[n_blocks] words; snap: 2 * (records + n_blocks) words.
struct UnpArgs {
  const BlockDesc* blocks;
  uint32_t n_blocks;
  const DInput* in;
  const uint32_t* nrec;
  const uint64_t* kbytes;
  const uint32_t* plan_nrec;
  const uint64_t* plan_kbytes;
  const uint2* ent_tab;
  const uint32_t* rec_first;
  const uint64_t* key_first;
  const uint32_t* chunk_first;
  uint32_t* chunkF;
  uint32_t* snap;
  Recs recs;
  uint8_t* arena;
  DErr* errs;
  DErr* verr;
  bool verify;
  uint32_t* next;  // block counter of the checksum pass (zero before it)
};
// Records and keys (every field but vcrc).
void launch_unpack_keys(const UnpArgs& a, cudaStream_t st);
// Checksums (with `verify`) and the value registers (vcrc), on `ctas` CTAs of one SM each;
// with half_warps each half warp folds its own block (small blocks).
void launch_unpack_crc(const UnpArgs& a, CrcTabs tabs, uint32_t ctas, bool half_warps, cudaStream_t st);
// recs.vcrc[r] = F(value of record r) for r < *n (or n_max when n is NULL), one warp per
// record (decoded records and the build path's records).
void launch_value_crc(Recs recs, const uint32_t* n, uint32_t n_max, CrcTabs tabs, cudaStream_t st);
void launch_input_ranges(const DInput* in, uint32_t n_inputs, const uint32_t* rec_first,
                         const uint64_t* key_first, uint32_t* in_rec, uint64_t* in_key, cudaStream_t st);

void launch_plan_checks(DInput* in, uint32_t n_inputs, const uint32_t* plan_nblk, DErr* errs, cudaStream_t st);
void launch_plan_check_recs(const BlockDesc* blocks, uint32_t n_blocks, const uint32_t* nrec, const uint64_t* kbytes,
                            const uint32_t* plan_nrec, const uint64_t* plan_kbytes, const DInput* in, DErr* errs,
                            cudaStream_t st);
void launch_plan_check_links(const uint8_t* link, const uint8_t* plan_link, uint32_t n_inputs, const DInput* in,
                             DErr* errs, cudaStream_t st);

// ---- sort.cu -----------------------------------------------------------------------------
struct MergeSpan {
  uint32_t a_begin;  // first position of run A (run B follows it)
  uint32_t a_len;
  uint32_t b_len;       // 0: run A is only moved to the other buffer
  uint32_t tile_first;  // first tile id of this merge
  uint32_t src;         // buffer (0/1) holding both runs; the result goes to the other
  uint32_t pad;
};
constexpr uint32_t kMergeTileMax = 2048;  // merge tiles: 512, 1024 or 2048 records

void launch_check_order(Recs recs, const uint8_t* arena, uint32_t n_rec, const DInput* in, DErr* errs,
                        cudaStream_t st);
void launch_plan_sanitize(Recs recs, uint32_t n_rec, const JobDev* jobs, uint32_t n_jobs, const DErr* errs,
                          const uint8_t* arena, cudaStream_t st);
void launch_sort_init(uint32_t* ord, MKey* okey, Recs recs, const uint8_t* arena, uint32_t n, cudaStream_t st);
// One pass of merges; ord[b] / key[b] are the two buffers, each span names its source.
void launch_merge_pass(const MergeSpan* spans, uint32_t n_spans, uint32_t n_tiles, uint32_t tile, uint32_t* ord0,
                       MKey* key0, uint32_t* ord1, MKey* key1, Recs recs, const uint8_t* arena, cudaStream_t st);
// With ranges, records whose user key is outside their job's range are dropped first.
void launch_gc_flags(const uint32_t* ord, uint32_t n_rec, const JobDev* jobs, uint32_t n_jobs, Recs recs,
                     const uint8_t* arena, uint32_t* keep, DErr* errs, cudaStream_t st,
                     const JobRange* ranges = nullptr, const uint8_t* bounds = nullptr);
void launch_gc_compact(const uint32_t* ord, const uint32_t* keep, const uint32_t* pos, uint32_t n_rec,
                       uint32_t* surv, cudaStream_t st);
void launch_job_surv(JobDev* jobs, uint32_t n_jobs, const uint32_t* pos, uint32_t n_rec, Counts* cnt,
                     cudaStream_t st);

// ---- pack.cu -----------------------------------------------------------------------------
void launch_sizes(const uint32_t* surv, const Counts* cnt, uint32_t cap, const JobDev* jobs, uint32_t n_jobs,
                  Recs recs, const uint8_t* arena, uint32_t* lcp, uint32_t* sd, uint32_t* dr, EncDesc* ed,
                  cudaStream_t st);
void launch_block_next(const uint64_t* P, const uint32_t* dr, const Counts* cnt, uint32_t cap, const JobDev* jobs,
                       uint32_t n_jobs, Fmt fmt, uint32_t* next, cudaStream_t st);
uint64_t stitch_temp_bytes(uint32_t cap);
void launch_stitch(const uint32_t* next, const uint32_t* n_dev, uint32_t cap, uint32_t* gap, const JobDev* jobs,
                   uint32_t n_jobs, bool blocks_level, uint8_t* flags, void* temp, cudaStream_t st);
void launch_compact_flags(const uint8_t* flags, const uint32_t* pos, const uint32_t* n_dev, uint32_t cap,
                          uint32_t* starts, uint32_t* total_out, cudaStream_t st);
void launch_job_blocks(JobDev* jobs, uint32_t n_jobs, const uint32_t* bpos, cudaStream_t st);
void launch_block_sizes(const uint32_t* blk_start, const Counts* cnt, uint32_t cap, const uint64_t* P,
                        const uint32_t* dr, Fmt fmt, uint64_t* bsz, uint64_t* disk, cudaStream_t st);
void launch_file_next(const uint64_t* C, const Counts* cnt, uint32_t cap, const JobDev* jobs, uint32_t n_jobs,
                      Fmt fmt, uint32_t* next, cudaStream_t st);
void launch_job_files(JobDev* jobs, uint32_t n_jobs, const uint32_t* fpos, cudaStream_t st);
void launch_block_file(const uint32_t* fpos, const Counts* cnt, uint32_t cap, uint32_t* blk_file, cudaStream_t st);
void launch_index_sizes(const uint32_t* blk_start, const uint64_t* bsz, const uint64_t* C, const uint32_t* blk_file,
                        const uint32_t* file_start, const Counts* cnt, uint32_t cap, const uint32_t* surv, Recs recs,
                        const uint8_t* arena, Fmt fmt, uint32_t* ie, cudaStream_t st);
// Filter array sizes: filters per table, then (after their scan into fa.base) each
// filter's bytes and bitmap words; sets cnt->n_filt.
void launch_filter_count(const uint32_t* file_start, const Counts* cnt, uint32_t cap, const uint64_t* C,
                         uint64_t* nfilt, cudaStream_t st);
void launch_filter_sizes(const uint64_t* fbase, const uint32_t* file_start, const uint32_t* blk_start,
                         const uint64_t* C, Counts* cnt, uint64_t slot_cap, Fmt fmt, uint64_t* fbytes,
                         uint64_t* fwords, cudaStream_t st);
void launch_file_layout(const uint32_t* file_start, const Counts* cnt, uint32_t cap, const uint32_t* blk_start,
                        const uint64_t* C, const uint64_t* IX, Fmt fmt, FiltArr fa, const JobDev* jobs,
                        uint32_t n_jobs, FileDesc* files, uint64_t* fsize, uint64_t* bmwords, cudaStream_t st);
void launch_file_offsets(FileDesc* files, Counts* cnt, uint32_t cap, const uint64_t* foff, const uint64_t* bmoff,
                         FiltArr fa, JobDev* jobs, uint32_t n_jobs, uint64_t out_cap, uint64_t bm_cap, DErr* errs,
                         cudaStream_t st);
void launch_zero_bitmap(uint32_t* bitmap, const Counts* cnt, uint64_t cap_words, cudaStream_t st);
void launch_encode(const uint32_t* blk_start, Counts* cnt, uint32_t cap, const uint32_t* blk_file,
                   const FileDesc* files, const uint64_t* C, const uint64_t* bsz, const uint32_t* surv,
                   const uint32_t* lcp, const uint32_t* sd, const uint32_t* dr, const EncDesc* ed, BlkEnc* bd,
                   Recs recs,
                   const uint8_t* arena, Fmt fmt, uint32_t max_kv, uint8_t* out, uint64_t out_cap, uint8_t* done,
                   uint32_t* big, DErr* errs, CrcTabs tabs, cudaStream_t st);
// Masked CRC trailers of the staged encoder's blocks (done[b] = 1), assembled from each
// entry's header and key delta (read back from the block) and the survivors' value
// registers (vcrc of the records).
void launch_block_trailer(const Counts* cnt, uint32_t cap, const BlkEnc* bd, const uint32_t* sd, const uint32_t* dr,
                          const EncDesc* ed, const uint32_t* vcrc, Fmt fmt, uint8_t* out, const uint8_t* done,
                          CrcTabs tabs, cudaStream_t st);
// CRC trailers of the staged encoder's blocks (done[b] = 1).
// Output block trailers; blocks taken from cnt->crc_next_out, helper launches as above.
void launch_block_crc(Counts* cnt, uint32_t cap, const uint32_t* blk_file, const FileDesc* files,
                      const uint64_t* C, const uint64_t* bsz, uint8_t* out, uint64_t out_cap, const uint8_t* done,
                      CrcTabs tabs, bool helper, cudaStream_t st);
// The blocks the staged encoder left, one CTA per block (bytes and CRC trailer).
void launch_encode_big(const uint32_t* blk_start, Counts* cnt, uint32_t cap, const uint32_t* blk_file,
                       const FileDesc* files, const uint64_t* C, const uint64_t* bsz, const uint32_t* surv,
                       const uint32_t* lcp, const uint32_t* sd, const uint32_t* dr, Recs recs, const uint8_t* arena,
                       Fmt fmt, uint8_t* out, uint64_t out_cap, const uint32_t* big, CrcTabs tabs, cudaStream_t st);
void launch_bloom(const EncDesc* ed, const Counts* cnt, uint32_t cap, const FileDesc* files, Fmt fmt,
                  const uint32_t* blk_start, const uint64_t* C, FiltArr fa, uint32_t* bitmap, uint64_t out_cap,
                  uint64_t bm_cap, cudaStream_t st);
void launch_index_write(const uint32_t* blk_start, const Counts* cnt, uint32_t cap, const uint64_t* bsz,
                        const uint64_t* C, const uint64_t* IX, const uint32_t* blk_file, const FileDesc* files,
                        const uint32_t* surv, Recs recs, const uint8_t* arena, Fmt fmt, uint8_t* out,
                        uint64_t out_cap, cudaStream_t st);
void launch_file_finish(const FileDesc* files, const Counts* cnt, uint32_t cap, const uint32_t* bitmap,
                        const uint32_t* surv, Recs recs, Fmt fmt, FiltArr fa, uint8_t* out, uint64_t out_cap,
                        CrcTabs tabs, CrcMsg* msgs, FileMeta* meta, cudaStream_t st);
// Compressed data blocks (R4c, LUDA_F_COMPRESS): scratch for the raw blocks and their
// streams, per-block offsets into both, pseudo-tables (one per job) for the raw pass.
struct PackCz {
  uint64_t *rawsz, *czsz, *Craw, *Cc;
  uint8_t* ctype;
  FileDesc* rfiles;
  uint32_t* rbf;
  uint8_t *raw, *cz;
  uint64_t raw_cap, c_cap;
};
// Raw and stream offsets of every block and the pseudo-tables (after the block sizes).
void launch_compress_blocks(PackCz z, JobDev* jobs, uint32_t n_jobs, Counts* cnt, uint32_t cap, uint64_t* bsz,
                            uint64_t* disk, void* scan_tmp, cudaStream_t st);
// After the raw pass: every block compressed, bsz/disk turned into the stored sizes.
void launch_compress(PackCz z, Counts* cnt, uint32_t cap, uint64_t* bsz, uint64_t* disk, cudaStream_t st);
// After the layout: stored bytes and type bytes into the tables; done[b] = 1 for all.
void launch_place(PackCz z, Counts* cnt, uint32_t cap, const uint32_t* blk_file, const FileDesc* files,
                  const uint64_t* C, const uint64_t* bsz, uint8_t* out, uint64_t out_cap, uint8_t* done,
                  cudaStream_t st);
void launch_key_lens(const FileMeta* meta, const Counts* cnt, uint32_t cap, uint64_t* lens, cudaStream_t st);
void launch_key_gather(FileMeta* meta, Counts* cnt, uint32_t cap, const uint64_t* koff, const FileDesc* files,
                       const uint32_t* surv, Recs recs, const uint8_t* arena, uint8_t* keybuf, cudaStream_t st);

// ---- build path (memtable flush) ----------------------------------------------------------
void launch_build_records(const uint8_t* ukeys, const uint64_t* ukoff, const uint64_t* seqs, const uint8_t* types,
                          const uint8_t* vals, const uint64_t* voff, uint32_t n, Recs recs, uint8_t* arena,
                          uint32_t* surv, DErr* err, cudaStream_t st);
void launch_build_check(Recs recs, const uint8_t* arena, uint32_t n, DErr* err, cudaStream_t st);

// CRC of messages msgs[0 .. (*count) * mult) (count may be NULL: mult messages); max_msgs
// bounds the grid.
void launch_msg_crc(CrcMsg* msgs, const uint32_t* count, uint32_t mult, uint32_t max_msgs, DErr* errs, CrcTabs tabs,
                    cudaStream_t st);

// ---- host runtime ------------------------------------------------------------------------
// Admission hook of a compaction: called once per call, after the sizing pass and before
// the large allocations, with the device bytes the call holds at its peak (sizing buffers,
// records and sort buffers, output arena). It may block; false abandons the call.
struct AdmitGate {
  uint64_t extra = 0;  // bytes the caller holds for the job besides the pipeline's own
  virtual bool admit(uint64_t bytes) = 0;
  // Around the host<->device copies of a host job (dir 0: inputs in, 1: tables out); the
  // copies are complete when copy_end is called. A server serialises each direction so
  // that one job's inputs go in while another job's tables come out.
  virtual void copy_begin(int dir) { (void)dir; }
  virtual void copy_end(int dir) { (void)dir; }
  virtual ~AdmitGate() = default;
};

// One job on opts->stream with device inputs (luda_compact_device plus an admission gate).
luda_status compact_job_device(const luda_job& job, const luda_options* opts, luda_outputs* out, AdmitGate* gate);
// One job with host inputs: copied to the device, compacted, new tables copied back into
// library-owned pinned host memory (luda_compact plus an admission gate).
// Sets up the calling thread's per-thread state (second stream and its events, the CRC
// tables of the device, the pinned staging buffer) ahead of its first job.
luda_status warm_thread();
luda_status compact_job_host(const luda_job& job, const luda_options* opts, luda_outputs* out, AdmitGate* gate);

// The kept run of a call's survivors (after the pack stage, on the call's stream): records,
// keys, value addresses in `out`, and per table key_first / kbytes / max_kv in meta.
cudaError_t launch_keep(const Counts* cnt, uint32_t cap, const EncDesc* ed, Recs recs, const FileDesc* files,
                        const BlkEnc* bd, const uint32_t* blk_file, const uint8_t* out, FileMeta* meta, KeptRecs K,
                        void* scan_tmp, cudaStream_t st);
// Records of inputs taken from kept runs (max_count: the largest input's count).
void launch_kept_gather(const KeptIn* ins, uint32_t n_inputs, uint64_t max_count, Recs recs, cudaStream_t st);

}  // namespace luda
