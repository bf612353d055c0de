// noalloc.cu -- luda_check_table_noalloc: check one input table without allocating.
//
// Some callers cannot allocate device memory at the point where they want to check a
// table: code that runs inside a custom allocator or memory-pool callback (where a
// nested cudaMalloc would re-enter the allocator), engines that reserve all device memory
// at start-up and forbid later allocations, and latency-critical paths where an
// allocation's implicit synchronisation is not acceptable. This entry point runs the
// kernels of a compaction's sizing pass -- footer, index entries, data block checksums
// and type bytes, and the block walk over every entry's varints, shared prefix and the
// restart array -- on scratch memory that lives in this file as static device arrays, so
// it calls no allocator. It stops there: the internal-key order and the index-key rule
// are checked by a compaction only after it has decoded the keys into an arena, so a
// table with valid checksums but keys out of order passes this check.
//
// Scratch: one NaScratch per device that loads the library (sizeof(NaScratch), under
// 1 MiB: LUDA_NOALLOC_MAX_BLOCKS block descriptors of 48 bytes and two per-block counts)
// plus the CRC tables (196 KiB); LUDA_NOALLOC_STATIC_BYTES bounds the sum (checked at
// compile time). It is held until the process exits. Every call reuses it and it keeps
// the last call's contents: each call clears what must start at zero (error word,
// counters) itself. Calls that overlap on the GPU (two host threads, or two streams in
// flight) share the scratch and race; callers must serialise them.
//
// Set-up: the first call on a device (with that device current) fetches the device
// addresses of the static arrays with cudaGetSymbolAddress and uploads the CRC tables
// with cudaMemcpyToSymbol. Make that first call before any stream capture.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "luda.h"

using namespace luda;

namespace {

constexpr uint32_t kNaMaxBlocks = LUDA_NOALLOC_MAX_BLOCKS;

struct NaScratch {
  DInput in;
  DErr err;
  CrcMsg msg;
  Counts cnt;
  unsigned long long entries;
  uint32_t blk_first[2];
  BlockDesc blocks[kNaMaxBlocks];
  uint32_t nrec[kNaMaxBlocks];
  uint64_t kbytes[kNaMaxBlocks];
};

static __device__ __align__(256) NaScratch g_na_scratch;
static __device__ __align__(256) uint32_t g_na_slice[1024];
static __device__ __align__(256) uint32_t g_na_shift[kShiftTables * 1024];
static_assert(sizeof(NaScratch) + sizeof(uint32_t) * (1024 + kShiftTables * 1024) <= LUDA_NOALLOC_STATIC_BYTES,
              "static device memory of the no-alloc check above its documented bound");

// Host copies used once to fill the device tables (static: no heap allocation).
uint32_t h_slice[1024];
uint32_t h_shift[kShiftTables * 1024];

struct NaDevice {
  bool ready = false;
  NaScratch* scratch = nullptr;
  CrcTabs tabs{};
};

std::mutex g_na_mu;
NaDevice g_na_dev[128];
bool g_na_tables_made = false;

__global__ void k_na_sum(const uint32_t* __restrict__ nrec, uint32_t n, unsigned long long* __restrict__ total) {
  unsigned long long s = 0;
  for (uint64_t i = gtid(); i < n; i += gstride()) s += nrec[i];
  for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  if ((threadIdx.x & 31u) == 0 && s) atomicAdd(total, s);
}

luda_status na_fail(luda_status s, luda_table_check* out, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error_detail(buf);
  if (out) out->status = s;
  return s;
}

luda_status na_setup(NaDevice** dev_out, luda_table_check* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) return na_fail(LUDA_ERR_CUDA, out, "no usable CUDA device");
  std::lock_guard<std::mutex> lk(g_na_mu);
  NaDevice& d = g_na_dev[dev];
  if (!d.ready) {
    if (!g_na_tables_made) {
      if (!make_crc_tables(h_slice, h_shift)) return na_fail(LUDA_ERR_CUDA, out, "crc table generation failed");
      g_na_tables_made = true;
    }
    void* p = nullptr;
    if ((e = cudaMemcpyToSymbol(g_na_slice, h_slice, sizeof h_slice)) != cudaSuccess ||
        (e = cudaMemcpyToSymbol(g_na_shift, h_shift, sizeof h_shift)) != cudaSuccess)
      return na_fail(LUDA_ERR_CUDA, out, "uploading crc tables: %s", cudaGetErrorString(e));
    if ((e = cudaGetSymbolAddress(&p, g_na_scratch)) != cudaSuccess)
      return na_fail(LUDA_ERR_CUDA, out, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    d.scratch = static_cast<NaScratch*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_na_slice)) != cudaSuccess)
      return na_fail(LUDA_ERR_CUDA, out, "cudaGetSymbolAddress(slice): %s", cudaGetErrorString(e));
    d.tabs.slice = static_cast<const uint32_t*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_na_shift)) != cudaSuccess)
      return na_fail(LUDA_ERR_CUDA, out, "cudaGetSymbolAddress(shift): %s", cudaGetErrorString(e));
    d.tabs.shift = static_cast<const uint32_t*>(p);
    d.ready = true;
  }
  *dev_out = &d;
  return LUDA_OK;
}

#define NA_CK(expr)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return na_fail(LUDA_ERR_CUDA, out, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" {

luda_status luda_check_table_noalloc(const uint8_t* table, uint64_t size, void* stream, luda_table_check* out) {
  set_error_detail("");
  if (!out) return na_fail(LUDA_ERR_INVALID_ARG, nullptr, "out is NULL");
  memset(out, 0, sizeof *out);
  if (!table && size) return na_fail(LUDA_ERR_INVALID_ARG, out, "table is NULL");
  if (table) {
    // device or managed memory of the current device only: a host pointer or another
    // GPU's memory would be read by the kernels below (a fault, or reads across devices)
    cudaPointerAttributes attr{};
    int cur = -1;
    NA_CK(cudaGetDevice(&cur));
    if (cudaPointerGetAttributes(&attr, table) != cudaSuccess) {
      cudaGetLastError();  // clear the sticky-free error of an unknown pointer
      return na_fail(LUDA_ERR_INVALID_ARG, out, "table is not a CUDA pointer");
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
      return na_fail(LUDA_ERR_INVALID_ARG, out, "table is not in device or managed memory (memory type %d)",
                     int(attr.type));
    if (attr.device != cur)
      return na_fail(LUDA_ERR_INVALID_ARG, out, "table is on device %d, the current device is %d", attr.device, cur);
  }
  NaDevice* dev = nullptr;
  luda_status rc = na_setup(&dev, out);
  if (rc) return rc;
  NaScratch* S = dev->scratch;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // clear what must start at zero (the scratch keeps the previous call's contents)
  NA_CK(cudaMemsetAsync(&S->err, 0, sizeof(DErr), st));
  NA_CK(cudaMemsetAsync(&S->cnt, 0, sizeof(Counts), st));
  NA_CK(cudaMemsetAsync(&S->entries, 0, sizeof(unsigned long long), st));
  DInput din{};
  din.data = table;
  din.size = size;
  NA_CK(cudaMemcpyAsync(&S->in, &din, sizeof din, cudaMemcpyHostToDevice, st));
  launch_footers(&S->in, 1, &S->err, &S->msg, dev->tabs, st);
  NA_CK(cudaGetLastError());
  NA_CK(cudaMemcpyAsync(&din, &S->in, sizeof din, cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  const uint32_t nblk = din.nblk;
  if (nblk > kNaMaxBlocks)
    return na_fail(LUDA_ERR_INVALID_ARG, out,
                   "table has %u data blocks; luda_check_table_noalloc handles at most %u (use a compaction entry "
                   "point for larger tables)",
                   nblk, kNaMaxBlocks);
  if (nblk) {
    const uint32_t first[2] = {0, nblk};
    NA_CK(cudaMemcpyAsync(S->blk_first, first, sizeof first, cudaMemcpyHostToDevice, st));
    launch_index_entries(&S->in, 1, S->blk_first, nblk, S->blocks, &S->err, st);
    launch_block_scan(S->blocks, nblk, &S->in, S->nrec, S->kbytes, &S->err, &S->cnt, nullptr, dev->tabs, st);
    k_na_sum<<<grid_for(nblk, 256, kSms), 256, 0, st>>>(S->nrec, nblk, &S->entries);
    count_launches(1);
    NA_CK(cudaGetLastError());
  }
  DErr err{};
  Counts cnt{};
  unsigned long long entries = 0;
  NA_CK(cudaMemcpyAsync(&err, &S->err, sizeof err, cudaMemcpyDeviceToHost, st));
  NA_CK(cudaMemcpyAsync(&cnt, &S->cnt, sizeof cnt, cudaMemcpyDeviceToHost, st));
  NA_CK(cudaMemcpyAsync(&entries, &S->entries, sizeof entries, cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  out->status = err.code;
  out->n_blocks = nblk;
  if (err.code == 0) {
    out->n_entries = entries;
    out->data_bytes = cnt.in_data_bytes;
    return LUDA_OK;
  }
  out->bad_offset = err.where;
  return na_fail(luda_status(err.code), out, "byte offset %llu: %s", (unsigned long long)err.where,
                 luda_strerror(luda_status(err.code)));
}

}  // extern "C"
