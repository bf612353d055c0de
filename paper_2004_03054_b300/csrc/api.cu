// api.cu -- host orchestration of the compaction pipeline and the C ABI of libluda.so.
//
// A call runs the three phases of a compaction (LUDA §II-A; Fig. 3 of §III-A without the
// host-side sort of steps 4-6, which stays on the device here) for one or many jobs:
//   sizing    footers and index blocks (one host read of per-input block counts), then
//             per-block CRC/structure checks and entry counts (one host read of per-input
//             record and key-byte totals, which size every later buffer);
//   execute   decode, merge, drop rule, sizes, block cut, file cut, layout, encode, bloom,
//             index/metaindex/footer -- launched back to back with no host round trip;
//   collect   one read of the counts, then the per-table metadata and boundary keys.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <iterator>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"
#include "luda.h"

using namespace luda;

namespace {
std::atomic<uint64_t> g_launches{0};
}

void luda::count_launches(uint32_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

thread_local char t_detail[512];

void set_detail(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_detail, sizeof t_detail, fmt, ap);
  va_end(ap);
}

}  // namespace

void luda::set_error_detail(const char* text) { snprintf(t_detail, sizeof t_detail, "%s", text); }

void luda::smem_optin_raw(const void* kernel, int bytes) {
  // The attribute belongs to the kernel on the device, not to a thread: one table for the
  // process, and the size only grows (a smaller value set by one thread would make another
  // thread's larger launch fail).
  struct Entry {
    const void* k;
    int dev, bytes;
  };
  static std::mutex mu;
  static std::vector<Entry> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  for (Entry& e : done)
    if (e.k == kernel && e.dev == dev) {
      if (bytes <= e.bytes) return;
      if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
        e.bytes = bytes;
      return;
    }
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
    done.push_back(Entry{kernel, dev, bytes});
}

// ---- launch shapes ----------------------------------------------------------------------------
namespace {
thread_local Tuning t_tuning;
}

const Tuning& luda::tuning() { return t_tuning; }

bool luda::tuning_valid(const luda_tuning* t) {
  if (!t) return true;
  const char* bad = nullptr;
  if (t->merge_tile && t->merge_tile != 512 && t->merge_tile != 1024 && t->merge_tile != 2048) bad = "merge_tile";
  else if (t->merge_ctas_per_sm > 32) bad = "merge_ctas_per_sm";
  else if (t->decode_warps > 16) bad = "decode_warps";
  else if (t->walk_threads && (t->walk_threads > 256 || t->walk_threads % 32)) bad = "walk_threads";
  else if (t->encode_ctas_per_sm > 8) bad = "encode_ctas_per_sm";
  else if (t->elem_threads && (t->elem_threads < 64 || t->elem_threads > 1024 || t->elem_threads % 32))
    bad = "elem_threads";
  else if (t->crc_ctas > kSms) bad = "crc_ctas";
  else if (t->crc_warps && (t->crc_warps < 8 || t->crc_warps > 32 || t->crc_warps % 8)) bad = "crc_warps";
  else if (t->h2d_ranges > 64) bad = "h2d_ranges";
  if (bad) set_detail("invalid tuning: %s", bad);
  return bad == nullptr;
}

luda::TuningScope::TuningScope(const luda_tuning* t) : saved_(t_tuning) {
  if (!t) return;
  if (t->merge_tile) t_tuning.merge_tile = t->merge_tile;
  if (t->merge_ctas_per_sm) t_tuning.merge_ctas_per_sm = t->merge_ctas_per_sm;
  if (t->decode_warps) t_tuning.decode_warps = t->decode_warps;
  if (t->walk_threads) t_tuning.walk_threads = t->walk_threads;
  if (t->encode_ctas_per_sm) t_tuning.encode_ctas_per_sm = t->encode_ctas_per_sm;
  if (t->elem_threads) t_tuning.elem_threads = t->elem_threads;
  if (t->crc_ctas) t_tuning.crc_ctas = t->crc_ctas;
  if (t->crc_warps) t_tuning.crc_warps = t->crc_warps;
  if (t->h2d_ranges) t_tuning.h2d_ranges = t->h2d_ranges;
}

luda::TuningScope::~TuningScope() { t_tuning = saved_; }

namespace {

// ---- per-device CRC tables ----------------------------------------------------------------
struct DevTables {
  uint32_t* slice = nullptr;
  uint32_t* shift = nullptr;
  uint32_t* chunk = nullptr;
};
std::mutex g_mu;
DevTables g_tabs[128];

luda_status get_tabs(CrcTabs* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    set_detail("no usable CUDA device");
    return LUDA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  DevTables& t = g_tabs[dev];
  if (!t.slice) {
    std::vector<uint32_t> slice(1024), shift(size_t(kShiftTables) * 1024), chunk(size_t(kChunkTables) * 1024);
    if (!make_crc_tables(slice.data(), shift.data()) || !make_chunk_tables(chunk.data())) {
      set_detail("crc table generation failed");
      return LUDA_ERR_CUDA;
    }
    uint32_t *ds = nullptr, *dh = nullptr, *dc = nullptr;
    if (cudaMalloc(&ds, slice.size() * 4) != cudaSuccess || cudaMalloc(&dh, shift.size() * 4) != cudaSuccess ||
        cudaMalloc(&dc, chunk.size() * 4) != cudaSuccess ||
        cudaMemcpy(ds, slice.data(), slice.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dh, shift.data(), shift.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dc, chunk.data(), chunk.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(ds);
      cudaFree(dh);
      cudaFree(dc);
      set_detail("could not upload crc tables: %s", cudaGetErrorString(cudaGetLastError()));
      return LUDA_ERR_CUDA;
    }
    t.slice = ds;
    t.shift = dh;
    t.chunk = dc;
    // Keep freed stream-ordered allocations cached in the device's default pool instead of
    // returning them to the driver at every synchronisation (a process-local setting).
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  out->slice = t.slice;
  out->shift = t.shift;
  out->chunk = t.chunk;
  return LUDA_OK;
}

// SMs of the unpack's checksum pass on the side stream: the other half runs the records,
// merge, drop rule and cuts beside it (74 of 148 measured best on the large job, against
// 50, 100, 120 and 148).

// ---- side stream --------------------------------------------------------------------------
// Work that does not feed the main chain of a compaction runs on a second stream of the
// calling thread: the checksums of the input data blocks (overlapping decode, merge, drop
// rule and cuts) and of the output data blocks (overlapping bloom, index and footers).
// Forks and joins are events, so the same code is captured into plans' graphs.
struct Side {
  int dev = -1;
  cudaStream_t s = nullptr;
  cudaStream_t s2 = nullptr;  // a third stream: the tables' filter, index and footer beside the encoder
  cudaEvent_t ev[7] = {};  // forks and joins: 0 input checksums, 1 their end, 2 trailers, 3 their end,
                           // 4 index block checksums, 5 filter/index/footer fork, 6 their end
};
thread_local Side t_side;

luda_status get_side(Side** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_detail("no usable CUDA device");
    return LUDA_ERR_CUDA;
  }
  Side& sd = t_side;
  if (sd.dev != dev) {
    if (sd.s) {
      cudaStreamDestroy(sd.s);
      if (sd.s2) cudaStreamDestroy(sd.s2);
      for (cudaEvent_t& e : sd.ev) cudaEventDestroy(e);
    }
    sd = Side{};
    if (cudaStreamCreateWithFlags(&sd.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sd.s2, cudaStreamNonBlocking) != cudaSuccess) {
      set_detail("cudaStreamCreateWithFlags failed");
      return LUDA_ERR_CUDA;
    }
    for (cudaEvent_t& e : sd.ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        set_detail("cudaEventCreateWithFlags failed");
        return LUDA_ERR_CUDA;
      }
    sd.dev = dev;
  }
  *out = &sd;
  return LUDA_OK;
}

// `to` waits for the work queued so far on `from` (event slot e of the side stream).
cudaError_t fork_join(Side* sd, int e, cudaStream_t from, cudaStream_t to) {
  cudaError_t r = cudaEventRecord(sd->ev[e], from);
  return r == cudaSuccess ? cudaStreamWaitEvent(to, sd->ev[e], 0) : r;
}

// ---- memory -------------------------------------------------------------------------------
struct DevMem {
  const luda_options* o;
  cudaStream_t st;
  void* get(size_t n) const {
    if (n == 0) n = 256;
    if (o && o->dev_alloc) return o->dev_alloc(n, o->alloc_ctx, st);
    void* p = nullptr;
    return cudaMallocAsync(&p, n, st) == cudaSuccess ? p : nullptr;
  }
  void put(void* p) const {
    if (!p) return;
    if (o && o->dev_free) o->dev_free(p, o->alloc_ctx, st);
    else cudaFreeAsync(p, st);
  }
};

// Bump layout over one allocation: measure, allocate, then hand out pointers.
struct Layout {
  size_t off = 0;
  uint8_t* base = nullptr;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T) + 16;
    return p;
  }
};

KeptRecs kept_layout(Layout& L, uint64_t n, uint64_t key_bytes) {
  KeptRecs K;
  K.pfx = L.take<uint64_t>(n + 1);
  K.tr = L.take<uint64_t>(n + 1);
  K.koff = L.take<uint64_t>(n + 1);
  K.vptr = L.take<uint64_t>(n + 1);
  K.klen = L.take<uint32_t>(n + 1);
  K.vlen = L.take<uint32_t>(n + 1);
  K.vcrc = L.take<uint32_t>(n + 1);
  K.arena = L.take<uint8_t>(key_bytes + 64);
  return K;
}

// ---- kept decoded runs (LUDA_F_KEEP_DECODED) -------------------------------------------------
// A store holds the kept run of one call's survivors, in the same device allocation as the
// call's tables (right after them), so that both go in one release. Each new table of the
// call registers its slice of the run under its data pointer and size; the registration
// ends when the outputs holding the tables are freed.
struct KeptStore {
  KeptRecs run{};
};
struct KeptTable {
  KeptStore* store = nullptr;  // identifies the store (for unregistering); never dereferenced by a lookup
  KeptRecs run{};              // the store's device arrays
  uint64_t size = 0;
  uint64_t first = 0, count = 0, key_first = 0, kbytes = 0;
  uint32_t max_kv = 0;
  std::vector<uint8_t> smallest, largest;  // internal keys
};
std::mutex g_kept_mu;
std::unordered_map<uintptr_t, KeptTable> g_kept;  // by the table's data pointer
std::atomic<uint64_t> g_kept_used{0};             // inputs served from kept runs

void kept_free(KeptStore* k) {
  if (!k) return;
  {
    std::lock_guard<std::mutex> lk(g_kept_mu);
    for (auto it = g_kept.begin(); it != g_kept.end();)
      it = it->second.store == k ? g_kept.erase(it) : std::next(it);
  }
  delete k;
}

// The kept runs of all n inputs (copies of their registrations), or false if one has none.
bool kept_lookup(const std::vector<DInput>& in, std::vector<KeptTable>* out) {
  std::lock_guard<std::mutex> lk(g_kept_mu);
  out->clear();
  for (const DInput& d : in) {
    auto it = g_kept.find(reinterpret_cast<uintptr_t>(d.data));
    if (it == g_kept.end() || it->second.size != d.size) return false;
    out->push_back(it->second);
  }
  return true;
}

// Internal-key order of two internal keys held on the host (user key bytes, a proper
// prefix first, then the trailer descending).
int cmp_ikey_host(const std::vector<uint8_t>& a, const std::vector<uint8_t>& b) {
  if (a.size() < 8 || b.size() < 8) return a.size() < b.size() ? -1 : (a.size() > b.size() ? 1 : 0);
  const size_t ua = a.size() - 8, ub = b.size() - 8, m = ua < ub ? ua : ub;
  const int c = m ? memcmp(a.data(), b.data(), m) : 0;
  if (c) return c < 0 ? -1 : 1;
  if (ua != ub) return ua < ub ? -1 : 1;
  uint64_t ta = 0, tb = 0;
  memcpy(&ta, a.data() + ua, 8);
  memcpy(&tb, b.data() + ub, 8);
  return ta == tb ? 0 : (ta > tb ? -1 : 1);
}

// Owner of the memory behind one or more luda_outputs (shared by the jobs of a batch).
struct Holder {
  std::atomic<int> refs{1};
  void* dev = nullptr;
  luda_free_fn dev_free = nullptr;
  void* ctx = nullptr;
  uint8_t* pinned = nullptr;
  size_t pinned_cap = 0;
  std::vector<std::pair<uint8_t*, size_t>> more_pinned;  // further pinned buffers of one result
  KeptStore* kept = nullptr;  // the kept run of the tables (LUDA_F_KEEP_DECODED)
};

// A small cache of pinned host buffers for table images (cudaHostAlloc is slow).
std::mutex g_pin_mu;
std::vector<std::pair<uint8_t*, size_t>> g_pin_free;

uint8_t* pinned_get(size_t n, size_t* cap) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (size_t i = 0; i < g_pin_free.size(); ++i)
      if (g_pin_free[i].second >= n) {
        auto pr = g_pin_free[i];
        g_pin_free.erase(g_pin_free.begin() + long(i));
        *cap = pr.second;
        return pr.first;
      }
  }
  void* p = nullptr;
  const size_t want = n < 4096 ? 4096 : n;
  if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) return nullptr;
  *cap = want;
  return static_cast<uint8_t*>(p);
}

void pinned_put(uint8_t* p, size_t cap) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.emplace_back(p, cap);
  while (g_pin_free.size() > 4) {
    cudaFreeHost(g_pin_free.front().first);
    g_pin_free.erase(g_pin_free.begin());
  }
}

void holder_release(Holder* h) {
  if (!h) return;
  if (--h->refs > 0) return;
  kept_free(h->kept);  // first: no lookup may find a table whose memory is going
  if (h->dev) {
    // stream-ordered on the legacy default stream: after the work queued there and on
    // every blocking stream, without the device-wide wait of cudaFree (which would stall
    // the other jobs of a server each time one releases its tables)
    if (h->dev_free) h->dev_free(h->dev, h->ctx, nullptr);
    else cudaFreeAsync(h->dev, cudaStreamLegacy);
  }
  pinned_put(h->pinned, h->pinned_cap);
  for (auto& pr : h->more_pinned) pinned_put(pr.first, pr.second);
  delete h;
}

struct OutPriv {
  Holder* holder;
  uint8_t* keys;
};

luda_status opts_check(const luda_options* o, Fmt* fmt) {
  if (!o) {
    set_detail("options pointer is NULL");
    return LUDA_ERR_INVALID_ARG;
  }
  if (o->block_size < 1 || o->restart_interval < 1 || o->restart_interval > 65535 || o->bloom_bits_per_key < 1 ||
      o->bloom_bits_per_key > 64 || o->target_file_size < 1) {
    set_detail("invalid options: block_size=%u restart_interval=%u bloom_bits_per_key=%u target=%llu",
               o->block_size, o->restart_interval, o->bloom_bits_per_key,
               (unsigned long long)o->target_file_size);
    return LUDA_ERR_INVALID_ARG;
  }
  if (!tuning_valid(o->tuning)) return LUDA_ERR_INVALID_ARG;
  if (o->flags & ~(LUDA_F_STRICT_DUP | LUDA_F_TRACE | LUDA_F_SHORT_INDEX | LUDA_F_FILTER_ARRAY | LUDA_F_COMPRESS |
                   LUDA_F_TEST_WAIT0 | LUDA_F_KEEP_DECODED)) {
    set_detail("unknown option flags 0x%x", o->flags);
    return LUDA_ERR_INVALID_ARG;
  }
  uint32_t k = o->bloom_bits_per_key * 69 / 100;
  if (k < 1) k = 1;
  if (k > 30) k = 30;
  *fmt = Fmt{o->block_size, o->restart_interval, o->bloom_bits_per_key, k, o->target_file_size, 0, o->flags};
  return LUDA_OK;
}

luda_status cuda_fail(cudaError_t e, const char* where) {
  set_detail("%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LUDA_ERR_OOM : LUDA_ERR_CUDA;
}

#define CK(expr)                                          \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);   \
  } while (0)

luda_status err_status(const DErr& e, uint32_t job, uint32_t n_jobs) {
  if (e.code == 0) return LUDA_OK;
  if (e.input != ~0u)
    set_detail("job %u of %u: input %u, byte offset %llu: %s", job, n_jobs, e.input, (unsigned long long)e.where,
               luda_strerror(luda_status(e.code)));
  else
    set_detail("job %u of %u: %s (position %llu)", job, n_jobs, luda_strerror(luda_status(e.code)),
               (unsigned long long)e.where);
  return luda_status(e.code);
}

// ---- pinned staging for the small host<->device transfers of one call --------------------
// Copies from and to pageable memory are staged by the driver synchronously; these go
// through one pinned buffer per host thread instead, so that a round trip is a few
// asynchronous copies and one synchronisation. take() hands out 16-byte aligned pieces
// until reset(); a request that does not fit returns NULL (the caller then uses its own
// memory) and the buffer grows at the next reset. The buffer is mapped into the device's
// address space: stage_copy moves a piece with a small kernel instead of a copy engine, so
// that a round trip does not queue behind bulk copies another stream has on the engines.
class HostStage {
 public:
  ~HostStage() {
    if (p_) cudaFreeHost(p_);
  }
  // Call only when no copy from or to the buffer is pending (after a synchronisation).
  void reset() {
    off_ = 0;
    if (want_ > cap_) {
      if (p_) cudaFreeHost(p_);
      p_ = nullptr;
      cap_ = 0;
      void* q = nullptr;
      void* d = nullptr;
      if (cudaHostAlloc(&q, want_, cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess) {
        p_ = static_cast<uint8_t*>(q);
        cap_ = want_;
        dev_ = cudaHostGetDevicePointer(&d, q, 0) == cudaSuccess ? static_cast<uint8_t*>(d) : nullptr;
      }
    }
  }
  void* take(size_t n) {
    const size_t o = (off_ + 15) & ~size_t(15);
    if (!p_ || o + n > cap_) {
      want_ = std::max(want_, std::max<size_t>(1u << 20, 2 * (o + n)));
      return nullptr;
    }
    off_ = o + n;
    return p_ + o;
  }
  // The device address of host bytes [q, q + n) when they lie in the buffer, else NULL.
  uint8_t* dev_of(const void* q, size_t n) const {
    const uint8_t* b = static_cast<const uint8_t*>(q);
    if (!dev_ || !p_ || b < p_ || n > cap_ || size_t(b - p_) > cap_ - n) return nullptr;
    return dev_ + (b - p_);
  }

 private:
  uint8_t* dev_ = nullptr;
  uint8_t* p_ = nullptr;
  size_t cap_ = 0, off_ = 0, want_ = 1u << 20;
};
thread_local HostStage t_stage;

// A copy between the device and the host stage by one small kernel (16-, 4- or 1-byte
// words, whichever the addresses and size allow).
__global__ void k_stage_copy(uint8_t* __restrict__ dst, const uint8_t* __restrict__ src, uint64_t n) {
  const uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x, step = uint64_t(gridDim.x) * blockDim.x;
  const uintptr_t a = uintptr_t(dst) | uintptr_t(src) | uintptr_t(n);
  if ((a & 15) == 0) {
    for (uint64_t i = i0; i < n / 16; i += step) reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
  } else if ((a & 3) == 0) {
    for (uint64_t i = i0; i < n / 4; i += step)
      reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(src)[i];
  } else {
    for (uint64_t i = i0; i < n; i += step) dst[i] = src[i];
  }
}

// Set while this thread runs a call whose bulk copies keep the copy engines busy.
thread_local bool t_stage_by_kernel = false;

// cudaMemcpyAsync, except that while t_stage_by_kernel is set a host-to-device or
// device-to-host copy of at most 1 MiB whose host side lies in this thread's stage runs as
// k_stage_copy on the stream. (On an idle bus the copy engine is the faster way: 0.03 ms
// per call on the 1 GiB job.)
cudaError_t stage_copy(void* dst, const void* src, size_t n, cudaMemcpyKind kind, cudaStream_t st) {
  uint8_t* hd = nullptr;
  if (t_stage_by_kernel && n && n <= (1u << 20)) {
    if (kind == cudaMemcpyHostToDevice && (hd = t_stage.dev_of(src, n))) src = hd;
    else if (kind == cudaMemcpyDeviceToHost && (hd = t_stage.dev_of(dst, n))) dst = hd;
  }
  if (!hd) return cudaMemcpyAsync(dst, src, n, kind, st);
  const uint64_t words = (n + 15) / 16;
  const unsigned grid = unsigned(std::min<uint64_t>(64, (words + 255) / 256));
  k_stage_copy<<<grid, 256, 0, st>>>(static_cast<uint8_t*>(dst), static_cast<const uint8_t*>(src), n);
  count_launches(1);
  return cudaGetLastError();
}

// ---- the pack stages, shared by compaction and build --------------------------------------
struct PackBufs {
  uint32_t *surv, *lcp, *sd, *dr, *next, *bpos, *blk_start, *fnext, *fpos, *file_start, *blk_file, *ie;
  uint8_t *sflags, *fflags, *enc_done;
  EncDesc* ed;
  BlkEnc* bd;
  CrcMsg* fmsg;
  uint32_t* big;
  uint64_t *P, *bsz, *disk, *C, *IX, *fsize, *foff, *bmw, *bmoff, *klens, *koff;
  FileDesc* files;
  FileMeta* meta;
  uint32_t* bitmap;
  uint8_t* keybuf;
  void *scan_tmp, *stitch_tmp;
  uint32_t meta_cap;  // entries of meta
  uint64_t key_cap;   // bytes of keybuf
  // filter arrays (LUDA_F_FILTER_ARRAY): per table, then per filter
  uint64_t *fcount, *fbase, *fbytes, *fwords, *fboff, *fwoff;
  uint64_t slot_cap;  // filters the buffers hold (0 without filter arrays)
  PackCz cz;          // compressed blocks (raw_cap == 0 without LUDA_F_COMPRESS)
};

// Scratch of the compressed-block pass for an output bound of out_cap bytes and at most
// cap blocks: raw blocks (each rounded to 16 bytes with a trailer's room) and their streams
// (n + n / 32 + 16 rounded, plus 16, per block).
static uint64_t cz_raw_cap(const Fmt& fmt, uint64_t out_cap, uint64_t cap) {
  return (fmt.flags & LUDA_F_COMPRESS) ? out_cap + 32 * (cap + 1) : 0;
}
static uint64_t cz_stream_cap(const Fmt& fmt, uint64_t out_cap, uint64_t cap) {
  return (fmt.flags & LUDA_F_COMPRESS) ? out_cap + out_cap / 32 + 48 * (cap + 1) : 0;
}

// Capacity of the filter arrays: a table has at most (data bytes >> 11) + 1 filters, and
// out_cap bounds all tables' bytes.
static uint64_t filter_slot_cap(const Fmt& fmt, uint64_t out_cap, uint64_t max_tables) {
  return (fmt.flags & LUDA_F_FILTER_ARRAY) ? (out_cap >> kFilterBaseLg) + max_tables + 2 : 0;
}

// Output bytes a filter array can add over one filter per table, for a job of n entries
// whose data blocks hold at most `data` bytes: a non-empty filter of m entries takes at most
// m * bpk / 8 + 10 bytes, every filter a 4-byte offset (at most data / 512 + 1 per table of
// them), and a table 6 more bytes of array offset and metaindex name.
static uint64_t filter_array_extra(const Fmt& fmt, uint64_t data, uint64_t n) {
  return (fmt.flags & LUDA_F_FILTER_ARRAY) ? (data >> (kFilterBaseLg - 3)) + 24 * n + 64 : 0;
}

void pack_layout(Layout& L, PackBufs& b, uint32_t cap, uint64_t bm_cap, uint64_t key_cap, uint64_t slot_cap,
                 uint64_t raw_cap = 0, uint64_t c_cap = 0, uint32_t n_jobs = 1) {
  b.meta_cap = cap + 1;
  b.cz = PackCz{};
  b.cz.raw_cap = raw_cap;
  b.cz.c_cap = c_cap;
  if (raw_cap) {
    b.cz.rawsz = L.take<uint64_t>(cap + 1);
    b.cz.czsz = L.take<uint64_t>(cap + 1);
    b.cz.Craw = L.take<uint64_t>(cap + 1);
    b.cz.Cc = L.take<uint64_t>(cap + 1);
    b.cz.ctype = L.take<uint8_t>(cap + 1);
    b.cz.rfiles = L.take<FileDesc>(uint64_t(n_jobs) + 1);
    b.cz.rbf = L.take<uint32_t>(cap + 1);
    b.cz.raw = L.take<uint8_t>(raw_cap + 64);
    b.cz.cz = L.take<uint8_t>(c_cap + 64);
  }
  b.key_cap = key_cap + 1;
  b.slot_cap = slot_cap;
  const uint64_t nfa = slot_cap ? cap + 1 : 1;
  b.fcount = L.take<uint64_t>(nfa);
  b.fbase = L.take<uint64_t>(nfa);
  b.fbytes = L.take<uint64_t>(slot_cap + 1);
  b.fwords = L.take<uint64_t>(slot_cap + 1);
  b.fboff = L.take<uint64_t>(slot_cap + 1);
  b.fwoff = L.take<uint64_t>(slot_cap + 1);
  b.surv = L.take<uint32_t>(cap + 1);
  b.lcp = L.take<uint32_t>(cap + 1);
  b.sd = L.take<uint32_t>(cap + 1);
  b.dr = L.take<uint32_t>(cap + 1);
  b.next = L.take<uint32_t>(cap + 1);
  b.bpos = L.take<uint32_t>(cap + 1);
  b.blk_start = L.take<uint32_t>(cap + 1);
  b.fnext = L.take<uint32_t>(cap + 1);
  b.fpos = L.take<uint32_t>(cap + 1);
  b.file_start = L.take<uint32_t>(cap + 1);
  b.blk_file = L.take<uint32_t>(cap + 1);
  b.ie = L.take<uint32_t>(cap + 1);
  b.sflags = L.take<uint8_t>(cap + 1);
  b.fflags = L.take<uint8_t>(cap + 1);
  b.enc_done = L.take<uint8_t>(cap + 1);
  b.ed = L.take<EncDesc>(cap + 1);
  b.bd = L.take<BlkEnc>(cap + 1);
  b.fmsg = L.take<CrcMsg>(3 * uint64_t(cap) + 3);
  b.big = L.take<uint32_t>(cap + 1);
  b.P = L.take<uint64_t>(cap + 1);
  b.bsz = L.take<uint64_t>(cap + 1);
  b.disk = L.take<uint64_t>(cap + 1);
  b.C = L.take<uint64_t>(cap + 1);
  b.IX = L.take<uint64_t>(cap + 1);
  b.fsize = L.take<uint64_t>(cap + 1);
  b.foff = L.take<uint64_t>(cap + 1);
  b.bmw = L.take<uint64_t>(cap + 1);
  b.bmoff = L.take<uint64_t>(cap + 1);
  b.klens = L.take<uint64_t>(cap + 1);
  b.koff = L.take<uint64_t>(cap + 1);
  b.files = L.take<FileDesc>(cap + 1);
  b.meta = L.take<FileMeta>(cap + 1);
  b.bitmap = L.take<uint32_t>(bm_cap + 1);
  b.keybuf = L.take<uint8_t>(key_cap + 1);
  b.scan_tmp = L.take<uint8_t>(scan_temp_bytes((slot_cap > cap ? slot_cap : cap) + 1));
  b.stitch_tmp = L.take<uint8_t>(stitch_temp_bytes(cap + 1));
}

// Survivors are in b.surv and cnt->n_surv is set; jobs[] hold surv ranges.
struct Trace;
void trace_mark(Trace* t, int i, cudaStream_t st);

luda_status run_pack(PackBufs& b, Counts* cnt, JobDev* jobs, uint32_t n_jobs, DErr* errs, uint32_t cap, Recs recs,
                     const uint8_t* arena, Fmt fmt, uint8_t* out, uint64_t out_cap, uint64_t bm_cap, CrcTabs tabs,
                     cudaStream_t st, Side* side, Trace* tr = nullptr) {
  launch_sizes(b.surv, cnt, cap, jobs, n_jobs, recs, arena, b.lcp, b.sd, b.dr, b.ed, st);
  CK((exclusive_scan<uint32_t, uint64_t>(b.sd, b.P, cap, &cnt->n_surv, b.scan_tmp, st)));
  launch_block_next(b.P, b.dr, cnt, cap, jobs, n_jobs, fmt, b.next, st);
  launch_stitch(b.next, &cnt->n_surv, cap, &cnt->gap_surv, jobs, n_jobs, false, b.sflags, b.stitch_tmp, st);
  CK((exclusive_scan<uint8_t, uint32_t>(b.sflags, b.bpos, cap, &cnt->n_surv, b.scan_tmp, st)));
  launch_compact_flags(b.sflags, b.bpos, &cnt->n_surv, cap, b.blk_start, &cnt->nb, st);
  launch_job_blocks(jobs, n_jobs, b.bpos, st);
  launch_block_sizes(b.blk_start, cnt, cap, b.P, b.dr, fmt, b.bsz, b.disk, st);
  if (b.cz.raw_cap) {
    // R4c: the raw blocks into scratch (the block cut used their sizes), then each block
    // compressed and its stored size taken for the file cut and the layout
    launch_compress_blocks(b.cz, jobs, n_jobs, cnt, cap, b.bsz, b.disk, b.scan_tmp, st);
    launch_encode(b.blk_start, cnt, cap, b.cz.rbf, b.cz.rfiles, b.cz.Craw, b.bsz, b.surv, b.lcp, b.sd, b.dr, b.ed,
                  b.bd, recs, arena, fmt, fmt.max_kv, b.cz.raw, b.cz.raw_cap, b.enc_done, b.big, errs, tabs, st);
    launch_encode_big(b.blk_start, cnt, cap, b.cz.rbf, b.cz.rfiles, b.cz.Craw, b.bsz, b.surv, b.lcp, b.sd, b.dr,
                      recs, arena, fmt, b.cz.raw, b.cz.raw_cap, b.big, tabs, st);
    launch_compress(b.cz, cnt, cap, b.bsz, b.disk, st);
    CK(cudaGetLastError());
  }
  CK((exclusive_scan<uint64_t, uint64_t>(b.disk, b.C, cap, &cnt->nb, b.scan_tmp, st)));
  launch_file_next(b.C, cnt, cap, jobs, n_jobs, fmt, b.fnext, st);
  launch_stitch(b.fnext, &cnt->nb, cap, &cnt->gap_blk, jobs, n_jobs, true, b.fflags, b.stitch_tmp, st);
  CK((exclusive_scan<uint8_t, uint32_t>(b.fflags, b.fpos, cap, &cnt->nb, b.scan_tmp, st)));
  launch_compact_flags(b.fflags, b.fpos, &cnt->nb, cap, b.file_start, &cnt->nf, st);
  launch_job_files(jobs, n_jobs, b.fpos, st);
  launch_block_file(b.fpos, cnt, cap, b.blk_file, st);
  launch_index_sizes(b.blk_start, b.bsz, b.C, b.blk_file, b.file_start, cnt, cap, b.surv, recs, arena, fmt, b.ie,
                     st);
  CK((exclusive_scan<uint32_t, uint64_t>(b.ie, b.IX, cap, &cnt->nb, b.scan_tmp, st)));
  FiltArr fa{};
  if (b.slot_cap) {
    // filter arrays: filters per table, each filter's bytes and bitmap words, their sums
    launch_filter_count(b.file_start, cnt, cap, b.C, b.fcount, st);
    CK((exclusive_scan<uint64_t, uint64_t>(b.fcount, b.fbase, cap, &cnt->nf, b.scan_tmp, st)));
    launch_filter_sizes(b.fbase, b.file_start, b.blk_start, b.C, cnt, b.slot_cap, fmt, b.fbytes, b.fwords, st);
    CK((exclusive_scan<uint64_t, uint64_t>(b.fbytes, b.fboff, b.slot_cap, &cnt->n_filt, b.scan_tmp, st)));
    CK((exclusive_scan<uint64_t, uint64_t>(b.fwords, b.fwoff, b.slot_cap, &cnt->n_filt, b.scan_tmp, st)));
    fa = FiltArr{b.fbase, b.fboff, b.fwoff, b.fbytes, b.slot_cap};
  }
  launch_file_layout(b.file_start, cnt, cap, b.blk_start, b.C, b.IX, fmt, fa, jobs, n_jobs, b.files, b.fsize, b.bmw,
                     st);
  CK((exclusive_scan<uint64_t, uint64_t>(b.fsize, b.foff, cap, &cnt->nf, b.scan_tmp, st)));
  CK((exclusive_scan<uint64_t, uint64_t>(b.bmw, b.bmoff, cap, &cnt->nf, b.scan_tmp, st)));
  launch_file_offsets(b.files, cnt, cap, b.foff, b.bmoff, fa, jobs, n_jobs, out_cap, bm_cap, errs, st);
  launch_zero_bitmap(b.bitmap, cnt, bm_cap, st);
  // filter, index block, metaindex, footer and table keys on the third stream, beside the
  // encoder (they read the survivors and the layout, not the data blocks)
  CK(fork_join(side, 5, st, side->s2));
  launch_bloom(b.ed, cnt, cap, b.files, fmt, b.blk_start, b.C, fa, b.bitmap, out_cap, bm_cap, side->s2);
  launch_index_write(b.blk_start, cnt, cap, b.bsz, b.C, b.IX, b.blk_file, b.files, b.surv, recs, arena, fmt, out,
                     out_cap, side->s2);
  launch_file_finish(b.files, cnt, cap, b.bitmap, b.surv, recs, fmt, fa, out, out_cap, tabs, b.fmsg, b.meta,
                     side->s2);
  launch_key_lens(b.meta, cnt, cap, b.klens, side->s2);
  CK((exclusive_scan<uint64_t, uint64_t>(b.klens, b.koff, cap, &cnt->nf, b.scan_tmp, side->s2)));
  launch_key_gather(b.meta, cnt, cap, b.koff, b.files, b.surv, recs, arena, b.keybuf, side->s2);
  CK(cudaEventRecord(side->ev[6], side->s2));
  trace_mark(tr, 7, st);
  if (b.cz.raw_cap) {
    launch_place(b.cz, cnt, cap, b.blk_file, b.files, b.C, b.bsz, out, out_cap, b.enc_done, st);
  } else {
    launch_encode(b.blk_start, cnt, cap, b.blk_file, b.files, b.C, b.bsz, b.surv, b.lcp, b.sd, b.dr, b.ed, b.bd, recs,
                  arena, fmt, fmt.max_kv, out, out_cap, b.enc_done, b.big, errs, tabs, st);
  }
  trace_mark(tr, 8, st);
  // data block trailers on the side stream (joined by the caller through event slot 3):
  // assembled from the pieces' registers, or (compressed blocks) computed from the bytes
  CK(fork_join(side, 2, st, side->s));
  if (b.cz.raw_cap)
    launch_block_crc(cnt, cap, b.blk_file, b.files, b.C, b.bsz, out, out_cap, b.enc_done, tabs, false, side->s);
  else
    launch_block_trailer(cnt, cap, b.bd, b.sd, b.dr, b.ed, recs.vcrc, fmt, out, b.enc_done, tabs, side->s);
  CK(cudaEventRecord(side->ev[3], side->s));
  if (!b.cz.raw_cap)
    launch_encode_big(b.blk_start, cnt, cap, b.blk_file, b.files, b.C, b.bsz, b.surv, b.lcp, b.sd, b.dr, recs, arena,
                      fmt, out, out_cap, b.big, tabs, st);
  CK(cudaStreamWaitEvent(st, side->ev[6], 0));
  // the SMs the trailer kernel of compressed blocks left join it for the blocks still to do
  if (b.cz.raw_cap)
    launch_block_crc(cnt, cap, b.blk_file, b.files, b.C, b.bsz, out, out_cap, b.enc_done, tabs, true, st);
  CK(cudaGetLastError());
  return LUDA_OK;
}

Recs recs_layout(Layout& L, uint32_t n) {
  Recs r;
  r.pfx = L.take<uint64_t>(n + 1);
  r.koff = L.take<uint64_t>(n + 1);
  r.klen = L.take<uint32_t>(n + 1);
  r.tr = L.take<uint64_t>(n + 1);
  r.vptr = L.take<uint64_t>(n + 1);
  r.vlen = L.take<uint32_t>(n + 1);
  r.src = L.take<uint32_t>(n + 1);
  r.vcrc = L.take<uint32_t>(n + 1);
  return r;
}

// Collect: counts -> metadata and keys -> per-job luda_outputs.
struct Collected {
  Counts cnt;
  std::vector<JobDev> jobs;
  std::vector<DErr> errs;
  std::vector<FileMeta> meta;
  std::vector<uint8_t> keys;
};

// d_errs holds 2 * (n_jobs + 1) entries: the main chain's errors, then the input checksum
// errors; a checksum error takes precedence (the inputs are verified before anything is
// read from them in the method's order).
// The counts, job records and error words come back in one round trip, together with the
// first kSpecMeta table records and kSpecKeys boundary-key bytes; only a result with more
// tables or key bytes than that needs a second one.
constexpr uint32_t kSpecMeta = 256;
constexpr uint64_t kSpecKeys = 64 * 1024;

luda_status collect(const Counts* d_cnt, const JobDev* d_jobs, const DErr* d_errs, const PackBufs& b, uint32_t n_jobs,
                    Collected* c, cudaStream_t st) {
  const size_t ne = 2 * size_t(n_jobs + 1);
  const uint32_t spec_m = std::min(kSpecMeta, b.meta_cap);
  const uint64_t spec_k = std::min(kSpecKeys, b.key_cap);
  HostStage& hs = t_stage;  // reset by the caller at the start of its call
  Counts* h_cnt = static_cast<Counts*>(hs.take(sizeof(Counts)));
  JobDev* h_jobs = static_cast<JobDev*>(hs.take(sizeof(JobDev) * n_jobs));
  DErr* h_errs = static_cast<DErr*>(hs.take(sizeof(DErr) * ne));
  FileMeta* h_meta = static_cast<FileMeta*>(hs.take(sizeof(FileMeta) * spec_m));
  uint8_t* h_keys = static_cast<uint8_t*>(hs.take(spec_k));
  const bool staged = h_cnt && h_jobs && h_errs && h_meta && h_keys;
  c->jobs.resize(n_jobs);
  c->errs.resize(ne);
  if (staged) {
    CK(stage_copy(h_cnt, d_cnt, sizeof(Counts), cudaMemcpyDeviceToHost, st));
    CK(stage_copy(h_jobs, d_jobs, sizeof(JobDev) * n_jobs, cudaMemcpyDeviceToHost, st));
    CK(stage_copy(h_errs, d_errs, sizeof(DErr) * ne, cudaMemcpyDeviceToHost, st));
    CK(stage_copy(h_meta, b.meta, sizeof(FileMeta) * spec_m, cudaMemcpyDeviceToHost, st));
    CK(stage_copy(h_keys, b.keybuf, spec_k, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->cnt = *h_cnt;
    memcpy(c->jobs.data(), h_jobs, sizeof(JobDev) * n_jobs);
    memcpy(c->errs.data(), h_errs, sizeof(DErr) * ne);
  } else {
    CK(stage_copy(&c->cnt, d_cnt, sizeof(Counts), cudaMemcpyDeviceToHost, st));
    CK(stage_copy(c->jobs.data(), d_jobs, sizeof(JobDev) * n_jobs, cudaMemcpyDeviceToHost, st));
    CK(stage_copy(c->errs.data(), d_errs, sizeof(DErr) * ne, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  for (uint32_t j = 0; j < n_jobs; ++j)
    if (c->errs[n_jobs + 1 + j].code) c->errs[j] = c->errs[n_jobs + 1 + j];
  c->errs.resize(n_jobs);
  c->meta.resize(c->cnt.nf);
  c->keys.resize(c->cnt.key_bytes + 1);
  if (!c->cnt.nf) return LUDA_OK;
  if (staged && c->cnt.nf <= spec_m && c->cnt.key_bytes <= spec_k) {
    memcpy(c->meta.data(), h_meta, sizeof(FileMeta) * c->cnt.nf);
    memcpy(c->keys.data(), h_keys, c->cnt.key_bytes);
    return LUDA_OK;
  }
  CK(stage_copy(c->meta.data(), b.meta, sizeof(FileMeta) * c->cnt.nf, cudaMemcpyDeviceToHost, st));
  CK(stage_copy(c->keys.data(), b.keybuf, c->cnt.key_bytes, cudaMemcpyDeviceToHost, st));
  return LUDA_OK;
}

void fill_outputs(const Collected& c, uint32_t n_jobs, uint8_t* out_base, Holder* h, luda_outputs* outs) {
  for (uint32_t j = 0; j < n_jobs; ++j) {
    luda_outputs& o = outs[j];
    const JobDev& jd = c.jobs[j];
    o.n_in_entries = jd.rec_end - jd.rec_begin;
    if (o.status != LUDA_OK) continue;
    const uint32_t nf = jd.file_end - jd.file_begin;
    o.n_dropped = o.n_in_entries - (jd.surv_end - jd.surv_begin);
    o.n_tables = nf;
    uint64_t kb = 0;
    for (uint32_t f = jd.file_begin; f < jd.file_end; ++f) kb += c.meta[f].small_len + c.meta[f].large_len;
    o.tables = static_cast<luda_table*>(calloc(nf ? nf : 1, sizeof(luda_table)));
    uint8_t* keys = static_cast<uint8_t*>(malloc(kb ? kb : 1));
    uint64_t kp = 0;
    for (uint32_t f = jd.file_begin; f < jd.file_end; ++f) {
      const FileMeta& m = c.meta[f];
      luda_table& t = o.tables[f - jd.file_begin];
      t.data = out_base + m.off;
      t.size = m.size;
      t.n_entries = m.n_entries;
      memcpy(keys + kp, c.keys.data() + m.small_koff, m.small_len);
      t.smallest = keys + kp;
      t.smallest_len = m.small_len;
      kp += m.small_len;
      memcpy(keys + kp, c.keys.data() + m.large_koff, m.large_len);
      t.largest = keys + kp;
      t.largest_len = m.large_len;
      kp += m.large_len;
    }
    OutPriv* p = new OutPriv{h, keys};
    ++h->refs;
    o._priv = p;
  }
}

// CUDA events at stage boundaries on the call's stream (LUDA_F_TRACE only).
// Stage boundaries also open NVTX ranges on the host ("luda/<stage>"), so a profiler's
// timeline shows which stage issued which launches; without a profiler attached they cost
// a few nanoseconds.
struct Trace {
  bool on = false;
  bool range = false;
  cudaEvent_t ev[16] = {};
  void init(bool enable) {
    on = enable;
    if (on)
      for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) on = false;
  }
  void mark(int i, cudaStream_t st) {
    if (on) cudaEventRecord(ev[i], st);
    static const char* const names[16] = {"luda/sizing", nullptr, nullptr, nullptr, "luda/decode", "luda/sort",
                                          "luda/cut",   "luda/encode", "luda/meta", nullptr, nullptr};
    if (i == 10 && range) {
      nvtxRangePop();
      range = false;
    } else if (i < 16 && names[i]) {
      if (range) nvtxRangePop();
      nvtxRangePushA(names[i]);
      range = true;
    }
  }
  double span(int a, int b) {
    float v = 0;
    if (on && cudaEventSynchronize(ev[b]) == cudaSuccess) cudaEventElapsedTime(&v, ev[a], ev[b]);
    return v;
  }
  ~Trace() {
    if (range) nvtxRangePop();
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

void trace_mark(Trace* t, int i, cudaStream_t st) {
  if (t) t->mark(i, st);
}

struct HostJob {
  const luda_input* inputs;
  uint32_t n_inputs;
  uint64_t snapshot;
  int32_t bottommost;
  const uint8_t* lo = nullptr;  // user-key range [lo, hi) (R13), host memory; null = unbounded
  uint32_t lo_len = 0;
  const uint8_t* hi = nullptr;
  uint32_t hi_len = 0;
};

HostJob host_job(const luda_job& j) {
  HostJob h{j.inputs, j.n_inputs, j.smallest_snapshot, j.bottommost};
  h.lo = j.range_lo;
  h.lo_len = j.range_lo ? j.range_lo_len : 0;
  h.hi = j.range_hi;
  h.hi_len = j.range_hi ? j.range_hi_len : 0;
  return h;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  bool on = false;
  void start(cudaStream_t st) {
    on = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    if (on) cudaEventRecord(a, st);
  }
  void stop(cudaStream_t st) {
    if (on) cudaEventRecord(b, st);
  }
  double ms() {
    float v = 0;
    if (on && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&v, a, b);
    return v;
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// ---- merge schedule ----------------------------------------------------------------------
// Runs of each job (position ranges, in order) are merged pairwise until one is left. A
// pass merges adjacent runs that sit in the same buffer, smallest pairs first and only
// pairs at most twice the smallest pair's size, so a large run (a level's tables that form
// one run) is not dragged through every pass; merged runs move to the other buffer, the
// others stay. When no adjacent pair shares a buffer the smallest run is moved across.
// At the end every job's run is brought to the buffer of the largest job.
struct MergeSched {
  uint32_t tile = 1024;  // records per merge tile (set before merge_schedule)
  std::vector<MergeSpan> spans;
  std::vector<uint32_t> pass_span0, pass_nspans, pass_ntiles;
  uint32_t max_tiles = 1;
  uint32_t final_buf = 0;
};

void merge_schedule(const std::vector<std::vector<std::pair<uint32_t, uint32_t>>>& runs_in, MergeSched* S) {
  struct R {
    uint32_t b, n, buf;
  };
  std::vector<std::vector<R>> runs(runs_in.size());
  for (size_t j = 0; j < runs_in.size(); ++j)
    for (const auto& r : runs_in[j])
      if (r.second) runs[j].push_back(R{r.first, r.second, 0});
  const uint32_t tile = S->tile;
  auto tiles_of = [tile](uint32_t n) { return (n + tile - 1) / tile; };
  auto begin_pass = [&]() { S->pass_span0.push_back(uint32_t(S->spans.size())); };
  auto end_pass = [&](uint32_t tiles) {
    S->pass_nspans.push_back(uint32_t(S->spans.size()) - S->pass_span0.back());
    S->pass_ntiles.push_back(tiles);
    if (tiles > S->max_tiles) S->max_tiles = tiles;
  };
  while (true) {
    bool more = false;
    for (auto& r : runs) more |= r.size() > 1;
    if (!more) break;
    begin_pass();
    uint32_t tiles = 0;
    for (auto& r : runs) {
      if (r.size() < 2) continue;
      std::vector<std::pair<uint64_t, size_t>> cand;
      for (size_t k = 0; k + 1 < r.size(); ++k)
        if (r[k].buf == r[k + 1].buf) cand.push_back({uint64_t(r[k].n) + r[k + 1].n, k});
      if (cand.empty()) {  // move the smallest run to the other buffer
        size_t k = 0;
        for (size_t i = 1; i < r.size(); ++i)
          if (r[i].n < r[k].n) k = i;
        S->spans.push_back(MergeSpan{r[k].b, r[k].n, 0, tiles, r[k].buf, 0});
        tiles += tiles_of(r[k].n);
        r[k].buf ^= 1u;
        continue;
      }
      std::stable_sort(cand.begin(), cand.end(),
                       [](const std::pair<uint64_t, size_t>& a, const std::pair<uint64_t, size_t>& b) {
                         return a.first < b.first;
                       });
      const uint64_t limit = 2 * cand[0].first;
      std::vector<uint8_t> first(r.size(), 0), used(r.size(), 0);
      for (const auto& c : cand) {
        if (c.first > limit) break;
        if (used[c.second] || used[c.second + 1]) continue;
        used[c.second] = used[c.second + 1] = 1;
        first[c.second] = 1;
      }
      std::vector<R> nr;
      for (size_t k = 0; k < r.size(); ++k) {
        if (first[k]) {
          S->spans.push_back(MergeSpan{r[k].b, r[k].n, r[k + 1].n, tiles, r[k].buf, 0});
          tiles += tiles_of(r[k].n + r[k + 1].n);
          nr.push_back(R{r[k].b, r[k].n + r[k + 1].n, r[k].buf ^ 1u});
          ++k;
        } else {
          nr.push_back(r[k]);
        }
      }
      r.swap(nr);
    }
    end_pass(tiles);
  }
  // one buffer for all jobs: the largest job's
  uint64_t best = 0;
  for (auto& r : runs)
    if (r.size() == 1 && r[0].n > best) {
      best = r[0].n;
      S->final_buf = r[0].buf;
    }
  bool moves = false;
  for (auto& r : runs) moves |= r.size() == 1 && r[0].buf != S->final_buf;
  if (moves) {
    begin_pass();
    uint32_t tiles = 0;
    for (auto& r : runs)
      if (r.size() == 1 && r[0].buf != S->final_buf) {
        S->spans.push_back(MergeSpan{r[0].b, r[0].n, 0, tiles, r[0].buf, 0});
        tiles += tiles_of(r[0].n);
      }
    end_pass(tiles);
  }
}

// LUDA_F_KEEP_DECODED, after the pack stage: a store for the survivors' run, filled on st.
// Null when nothing is kept: the flag is off, the tables are compressed (a compressed
// block's value has no address of its own) or go to the host, or there is no memory for
// the store (the tables are then simply not kept).
// Bytes of the store (kept_start), allocated right after the output arena so that it is
// freed with the tables in one release (0 when the call keeps nothing).
uint64_t kept_bytes(const luda_options* o, bool host_out, const Fmt& fmt, uint32_t cap, uint64_t key_bytes) {
  if (!(o->flags & LUDA_F_KEEP_DECODED) || host_out || (fmt.flags & LUDA_F_COMPRESS) || !cap) return 0;
  Layout LK;
  kept_layout(LK, cap, key_bytes);
  return LK.off;
}

luda_status kept_start(const luda_options* o, uint8_t* km, bool host_out, const PackBufs& pb,
                       const Counts* d_cnt, uint32_t cap, uint64_t key_bytes, const Recs& recs,
                       const uint8_t* d_out, cudaStream_t st, KeptStore** out) {
  *out = nullptr;
  if (!(o->flags & LUDA_F_KEEP_DECODED) || host_out || pb.cz.raw_cap || !cap || !km) return LUDA_OK;
  KeptStore* k = new KeptStore();  // its memory belongs to the output allocation
  Layout LK;
  LK.base = static_cast<uint8_t*>(km);
  k->run = kept_layout(LK, cap, key_bytes);
  const cudaError_t e =
      launch_keep(d_cnt, cap, pb.ed, recs, pb.files, pb.bd, pb.blk_file, d_out, pb.meta, k->run, pb.scan_tmp, st);
  if (e != cudaSuccess) {
    kept_free(k);
    return cuda_fail(e, "kept run");
  }
  *out = k;
  return LUDA_OK;
}

// Each new table of the finished jobs registers its slice of the store's run.
void kept_register(KeptStore* k, const Collected& col, uint32_t n_jobs, const luda_outputs* outs,
                   const uint8_t* base) {
  std::lock_guard<std::mutex> lk(g_kept_mu);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    if (outs[j].status != LUDA_OK) continue;
    const JobDev& jd = col.jobs[j];
    uint64_t first = jd.surv_begin;
    for (uint32_t f = jd.file_begin; f < jd.file_end; ++f) {
      const FileMeta& m = col.meta[f];
      KeptTable t;
      t.store = k;
      t.run = k->run;
      t.size = m.size;
      t.first = first;
      t.count = m.n_entries;
      t.key_first = m.key_first;
      t.kbytes = m.kbytes;
      t.max_kv = m.max_kv;
      t.smallest.assign(col.keys.begin() + m.small_koff, col.keys.begin() + m.small_koff + m.small_len);
      t.largest.assign(col.keys.begin() + m.large_koff, col.keys.begin() + m.large_koff + m.large_len);
      g_kept[reinterpret_cast<uintptr_t>(base + m.off)] = std::move(t);
      first += m.n_entries;
    }
  }
}

struct KeptGuard {
  KeptStore* k = nullptr;
  ~KeptGuard() { kept_free(k); }
};

// Whether the unpack's lanes fold small blocks by half warps, one block each: blocks under
// 8 KiB on average (a 5 KiB block's 36 chunks fill 64 lanes of a warp's two rounds, 48 of a
// half warp's three).
bool unpack_half(uint64_t in_bytes, uint32_t n_blocks) { return n_blocks && in_bytes / n_blocks < 8192; }

// The whole compaction for n_jobs jobs whose inputs are device pointers. On return
// outs[j] hold device (or, with host_out, pinned host) tables.
luda_status run_compaction(const HostJob* jobs, uint32_t n_jobs, const luda_options* o, cudaStream_t st,
                           luda_outputs* outs, bool host_out, double* ms_device, double* ms_d2h,
                           double* stage_ms = nullptr, uint64_t* stage_bytes = nullptr, AdmitGate* gate = nullptr,
                           std::vector<uint32_t>* blk_nrec = nullptr) {
  Fmt fmt;
  luda_status rc = opts_check(o, &fmt);
  if (rc) return rc;
  const TuningScope tuned(o->tuning);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    memset(&outs[j], 0, sizeof(luda_outputs));
    if (jobs[j].n_inputs && !jobs[j].inputs) {
      set_detail("job %u: inputs is NULL", j);
      return LUDA_ERR_INVALID_ARG;
    }
    for (uint32_t i = 0; i < jobs[j].n_inputs; ++i)
      if (!jobs[j].inputs[i].data && jobs[j].inputs[i].size) {
        set_detail("job %u input %u: data is NULL", j, i);
        return LUDA_ERR_INVALID_ARG;
      }
  }
  CrcTabs tabs;
  if ((rc = get_tabs(&tabs))) return rc;
  const DevMem mem{o, st};
  Timer tdev;
  tdev.start(st);
  Trace tr;
  // LUDA_TRACE=1 in the environment turns the stage events on as LUDA_F_TRACE does
  static const bool env_trace = [] {
    const char* v = getenv("LUDA_TRACE");
    return v && v[0] == '1';
  }();
  tr.init(((o->flags & LUDA_F_TRACE) || env_trace) && stage_ms);
  tr.mark(0, st);

  // ---- sizing: footers -------------------------------------------------------------------
  std::vector<DInput> hin;
  std::vector<uint64_t> job_in_bytes(n_jobs, 0);
  std::vector<uint32_t> job_in_first(n_jobs + 1, 0);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    job_in_first[j] = uint32_t(hin.size());
    for (uint32_t i = 0; i < jobs[j].n_inputs; ++i) {
      DInput d{};
      d.data = jobs[j].inputs[i].data;
      d.size = jobs[j].inputs[i].size;
      d.job = j;
      d.local = i;
      hin.push_back(d);
      job_in_bytes[j] += d.size;
    }
  }
  job_in_first[n_jobs] = uint32_t(hin.size());
  const uint32_t N = uint32_t(hin.size());

  // ranged jobs (R13): one JobRange per job and the bound keys back to back
  std::vector<JobRange> hranges;
  std::vector<uint8_t> hbounds;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    JobRange r{};
    if (jobs[j].lo) {
      r.flags |= 1u;
      r.lo_off = uint32_t(hbounds.size());
      r.lo_len = jobs[j].lo_len;
      hbounds.insert(hbounds.end(), jobs[j].lo, jobs[j].lo + jobs[j].lo_len);
    }
    if (jobs[j].hi) {
      r.flags |= 2u;
      r.hi_off = uint32_t(hbounds.size());
      r.hi_len = jobs[j].hi_len;
      hbounds.insert(hbounds.end(), jobs[j].hi, jobs[j].hi + jobs[j].hi_len);
    }
    hranges.push_back(r);
  }
  const bool ranged = !hbounds.empty() || std::any_of(hranges.begin(), hranges.end(),
                                                      [](const JobRange& r) { return r.flags != 0; });
  // inputs with kept decoded runs (LUDA_F_KEEP_DECODED): when every input has one, the
  // records come from the runs and none of the sizing and unpack kernels runs
  std::vector<KeptTable> kin;
  const bool cached = (o->flags & LUDA_F_KEEP_DECODED) && !ranged && N > 0 && kept_lookup(hin, &kin);
  Layout LA;
  DInput* d_in;
  DErr* d_errs;
  JobDev* d_jobs;
  uint32_t* d_in_blk_first;
  Counts* d_cnt;
  CrcMsg* d_msgs;
  uint8_t* d_link;
  JobRange* d_ranges = nullptr;
  uint8_t* d_bounds = nullptr;
  auto layA = [&](Layout& L) {
    d_in = L.take<DInput>(N + 1);
    d_errs = L.take<DErr>(2 * (n_jobs + 1));  // main chain, then input checksums
    d_jobs = L.take<JobDev>(n_jobs + 1);
    d_in_blk_first = L.take<uint32_t>(N + 1);
    d_cnt = L.take<Counts>(1);
    d_msgs = L.take<CrcMsg>(N + 1);
    d_link = L.take<uint8_t>(N + 1);
    if (ranged) {
      d_ranges = L.take<JobRange>(n_jobs + 1);
      d_bounds = L.take<uint8_t>(hbounds.size() + 32);  // word reads may pass the last key
    }
  };
  layA(LA);
  uint8_t* bufA = static_cast<uint8_t*>(mem.get(LA.off));
  if (!bufA) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  LA = Layout{};
  LA.base = bufA;
  layA(LA);
  struct Guard {
    const DevMem& m;
    std::vector<void*> ps;
    ~Guard() {
      for (void* p : ps) m.put(p);
    }
  } guard{mem, {bufA}};

  HostStage& hs = t_stage;
  hs.reset();
  // a pinned copy of a host array for an asynchronous copy (the array itself if none is left)
  auto pin = [&](const void* src, size_t n) -> const void* {
    void* q = hs.take(n);
    if (!q) return src;
    memcpy(q, src, n);
    return q;
  };
  CK(cudaMemsetAsync(d_errs, 0, sizeof(DErr) * 2 * (n_jobs + 1), st));
  CK(cudaMemsetAsync(d_cnt, 0, sizeof(Counts), st));
  if (ranged) {
    CK(stage_copy(d_ranges, pin(hranges.data(), sizeof(JobRange) * n_jobs), sizeof(JobRange) * n_jobs,
                       cudaMemcpyHostToDevice, st));
    if (!hbounds.empty())
      CK(stage_copy(d_bounds, pin(hbounds.data(), hbounds.size()), hbounds.size(), cudaMemcpyHostToDevice, st));
  }
  DInput* hin_pin = static_cast<DInput*>(hs.take(sizeof(DInput) * (N + 1)));
  if (N)
    CK(stage_copy(d_in, pin(hin.data(), sizeof(DInput) * N), sizeof(DInput) * N, cudaMemcpyHostToDevice, st));
  // the index blocks' checksums run on the side stream (their errors, like the data blocks',
  // take precedence when the results are collected) while the host sizes the job
  Side* side = nullptr;
  if ((rc = get_side(&side))) return rc;
  if (!cached) {
    launch_footers_read(d_in, N, d_errs, d_msgs, st);
    CK(fork_join(side, 4, st, side->s));
    launch_index_crc(d_msgs, N, d_errs + n_jobs + 1, tabs, side->s);
    launch_footers_finish(d_in, N, d_errs, st);
    CK(cudaGetLastError());
    if (N) CK(stage_copy(hin_pin ? hin_pin : hin.data(), d_in, sizeof(DInput) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (N && hin_pin) memcpy(hin.data(), hin_pin, sizeof(DInput) * N);
  }
  std::vector<uint32_t> in_blk_first(N + 1, 0);
  uint64_t NB64 = 0;
  for (uint32_t i = 0; i < N; ++i) {
    hin[i].blk_first = uint32_t(NB64);
    in_blk_first[i] = uint32_t(NB64);
    NB64 += hin[i].nblk;
  }
  in_blk_first[N] = uint32_t(NB64);
  if (NB64 >= (1ull << 31)) {
    set_detail("too many data blocks in one call (%llu)", (unsigned long long)NB64);
    return LUDA_ERR_INVALID_ARG;
  }
  const uint32_t NB = uint32_t(NB64);
  if (N) {
    CK(stage_copy(d_in, pin(hin.data(), sizeof(DInput) * N), sizeof(DInput) * N, cudaMemcpyHostToDevice, st));
    CK(stage_copy(d_in_blk_first, pin(in_blk_first.data(), sizeof(uint32_t) * (N + 1)),
                       sizeof(uint32_t) * (N + 1), cudaMemcpyHostToDevice, st));
  }

  // ---- sizing: block scan ------------------------------------------------------------------
  Layout LB;
  uint2* d_hdr;  // the walk's entry table
  uint32_t *d_nch, *d_chunk_first;  // the unpack's chunks per block and their offsets
  uint64_t *d_ulen, *d_ures;  // R4c: decompressed length and arena share of each block
  auto layoutB = [&](Layout& L, BlockDesc*& blocks, uint32_t*& nrec, uint64_t*& kbytes, uint32_t*& rec_first,
                     uint64_t*& key_first, uint32_t*& in_rec, uint64_t*& in_key, void*& tmp) {
    blocks = L.take<BlockDesc>(NB + 1);
    d_ulen = L.take<uint64_t>(NB + 1);
    d_ures = L.take<uint64_t>(NB + 1);
    d_hdr = L.take<uint2>(uint64_t(NB) * kHdrMax + 1);
    d_nch = L.take<uint32_t>(NB + 1);
    d_chunk_first = L.take<uint32_t>(NB + 1);
    nrec = L.take<uint32_t>(NB + 1);
    kbytes = L.take<uint64_t>(NB + 1);
    rec_first = L.take<uint32_t>(NB + 1);
    key_first = L.take<uint64_t>(NB + 1);
    in_rec = L.take<uint32_t>(N + 1);
    in_key = L.take<uint64_t>(N + 1);
    tmp = L.take<uint8_t>(scan_temp_bytes(NB + 1));
  };
  BlockDesc* d_blocks;
  uint32_t *d_nrec, *d_rec_first, *d_in_rec;
  uint64_t *d_kbytes, *d_key_first, *d_in_key;
  void* d_tmpB;
  layoutB(LB, d_blocks, d_nrec, d_kbytes, d_rec_first, d_key_first, d_in_rec, d_in_key, d_tmpB);
  uint8_t* bufB = static_cast<uint8_t*>(mem.get(LB.off));
  if (!bufB) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  guard.ps.push_back(bufB);
  LB = Layout{};
  LB.base = bufB;
  layoutB(LB, d_blocks, d_nrec, d_kbytes, d_rec_first, d_key_first, d_in_rec, d_in_key, d_tmpB);

  if (!cached) launch_index_entries(d_in, N, d_in_blk_first, NB, d_blocks, d_errs, st, d_ranges, d_bounds);
  // block contents: the stored blocks, or copies pointing at their decompressed contents
  BlockDesc* d_cb = d_blocks;
  std::vector<uint32_t> in_rec(N + 1);
  std::vector<uint64_t> in_key(N + 1);
  std::vector<DErr> herr(n_jobs + 1);
  std::vector<uint8_t> link(N + 1, 0);
  uint32_t comp_blocks = 0;
  uint64_t comp_bytes = 0;
  uint32_t n_chunks = 0;  // the unpack's chunk registers (the walk's counts summed)
  // entry counts and key bytes of every block, the inputs' record ranges and links; with
  // `contents` the blocks are contents already (the second pass after decompression)
  auto size_pass = [&](bool contents) -> luda_status {
    launch_block_walk(d_cb, NB, d_in, d_nrec, d_kbytes, d_errs, d_cnt, d_hdr, st, d_ulen, d_ures, contents, d_nch);
    if (!contents) tr.mark(2, st);
    launch_zero_failed(d_cb, NB, d_errs, d_nrec, d_kbytes, st);
    launch_run_links(d_in, N, d_cb, d_errs, d_link, st);
    CK((exclusive_scan<uint32_t, uint32_t>(d_nch, d_chunk_first, NB, nullptr, d_tmpB, st)));
    CK((exclusive_scan<uint32_t, uint32_t>(d_nrec, d_rec_first, NB, nullptr, d_tmpB, st)));
    CK((exclusive_scan<uint64_t, uint64_t>(d_kbytes, d_key_first, NB, nullptr, d_tmpB, st)));
    launch_input_ranges(d_in, N, d_rec_first, d_key_first, d_in_rec, d_in_key, st);
    CK(cudaGetLastError());
    // one pinned piece for the results (pageable vectors if the stage is full)
    uint32_t* p_rec = static_cast<uint32_t*>(hs.take(sizeof(uint32_t) * (N + 1)));
    uint64_t* p_key = static_cast<uint64_t*>(hs.take(sizeof(uint64_t) * (N + 1)));
    DErr* p_err = static_cast<DErr*>(hs.take(sizeof(DErr) * n_jobs));
    uint32_t* p_kv = static_cast<uint32_t*>(hs.take(sizeof(uint32_t)));
    uint8_t* p_link = static_cast<uint8_t*>(hs.take(N + 1));
    uint64_t* p_comp = static_cast<uint64_t*>(hs.take(2 * sizeof(uint64_t)));
    uint32_t* p_nch = static_cast<uint32_t*>(hs.take(sizeof(uint32_t)));
    const bool pinned = p_rec && p_key && p_err && p_kv && p_link && p_comp && p_nch;
    uint64_t comp[2] = {0, 0};
    if (!pinned) {
      p_rec = in_rec.data();
      p_key = in_key.data();
      p_err = herr.data();
      p_kv = &fmt.max_kv;
      p_link = link.data();
      p_comp = comp;
      p_nch = &n_chunks;
    }
    CK(stage_copy(p_rec, d_in_rec, sizeof(uint32_t) * (N + 1), cudaMemcpyDeviceToHost, st));
    CK(stage_copy(p_key, d_in_key, sizeof(uint64_t) * (N + 1), cudaMemcpyDeviceToHost, st));
    if (n_jobs) CK(stage_copy(p_err, d_errs, sizeof(DErr) * n_jobs, cudaMemcpyDeviceToHost, st));
    CK(stage_copy(p_kv, &d_cnt->max_kv, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    if (N) CK(stage_copy(p_link, d_link, N, cudaMemcpyDeviceToHost, st));
    CK(stage_copy(p_comp, &d_cnt->comp_blocks, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(stage_copy(p_comp + 1, &d_cnt->comp_bytes, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(stage_copy(p_nch, d_chunk_first + NB, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    uint32_t* p_nrec = nullptr;
    if (blk_nrec) {  // every block's entry count (0 for blocks a ranged job leaves unread)
      blk_nrec->resize(NB);
      p_nrec = static_cast<uint32_t*>(hs.take(sizeof(uint32_t) * NB));
      if (NB) CK(stage_copy(p_nrec ? p_nrec : blk_nrec->data(), d_nrec, sizeof(uint32_t) * NB, cudaMemcpyDeviceToHost, st));
    }
    if (!contents) tr.mark(3, st);
    CK(cudaStreamSynchronize(st));
    if (p_nrec && NB) memcpy(blk_nrec->data(), p_nrec, sizeof(uint32_t) * NB);
    if (pinned) {
      memcpy(in_rec.data(), p_rec, sizeof(uint32_t) * (N + 1));
      memcpy(in_key.data(), p_key, sizeof(uint64_t) * (N + 1));
      if (n_jobs) memcpy(herr.data(), p_err, sizeof(DErr) * n_jobs);
      fmt.max_kv = *p_kv;
      if (N) memcpy(link.data(), p_link, N);
      comp[0] = p_comp[0];
      comp[1] = p_comp[1];
      n_chunks = *p_nch;
    }
    comp_blocks = uint32_t(comp[0]);
    comp_bytes = comp[1];
    return LUDA_OK;
  };
  tr.mark(1, st);
  if (cached) {
    // the runs' counts, key bytes and boundary keys stand for the blocks' (records of
    // input i follow those of input i - 1; inputs i and i + 1 of one job form one sorted run
    // when i's largest key is below i + 1's smallest)
    tr.mark(2, st);
    tr.mark(3, st);
    in_rec[0] = 0;
    in_key[0] = 0;
    for (uint32_t i = 0; i < N; ++i) {
      in_rec[i + 1] = in_rec[i] + uint32_t(kin[i].count);
      in_key[i + 1] = in_key[i] + kin[i].kbytes;
      fmt.max_kv = std::max(fmt.max_kv, kin[i].max_kv);
      link[i] = i + 1 < N && hin[i].job == hin[i + 1].job && kin[i].count && kin[i + 1].count &&
                cmp_ikey_host(kin[i].largest, kin[i + 1].smallest) < 0;
    }
    if (uint64_t(in_rec[N]) != [&] {
          uint64_t t = 0;
          for (const KeptTable& k : kin) t += k.count;
          return t;
        }()) {
      set_detail("too many entries in one call");
      return LUDA_ERR_INVALID_ARG;
    }
  } else if ((rc = size_pass(false))) {
    return rc;
  }
  if (comp_blocks) {
    // R4c: the compressed blocks decompressed into one arena (each at a 16-byte multiple),
    // then the job sized again from the contents
    Layout LD;
    uint64_t* d_uoff;
    BlockDesc* d_cblocks;
    uint8_t* d_dec;
    auto layoutD = [&](Layout& L) {
      d_uoff = L.take<uint64_t>(NB + 1);
      d_cblocks = L.take<BlockDesc>(NB + 1);
      d_dec = L.take<uint8_t>(comp_bytes + 64);
    };
    layoutD(LD);
    uint8_t* bufD = static_cast<uint8_t*>(mem.get(LD.off));
    if (!bufD) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
    guard.ps.push_back(bufD);
    LD = Layout{};
    LD.base = bufD;
    layoutD(LD);
    // the stored blocks' checksums on the side stream (the unpack reads the contents),
    // joined before the results are collected
    CK(fork_join(side, 0, st, side->s));
    launch_block_verify(d_blocks, NB, d_in, d_errs, d_errs + n_jobs + 1, tabs, &d_cnt->crc_next_in, false,
                        side->s);
    CK(cudaEventRecord(side->ev[1], side->s));
    CK((exclusive_scan<uint64_t, uint64_t>(d_ures, d_uoff, NB, nullptr, d_tmpB, st)));
    CK(stage_copy(d_cblocks, d_blocks, sizeof(BlockDesc) * NB, cudaMemcpyDeviceToDevice, st));
    launch_decompress(d_blocks, NB, d_ulen, d_uoff, d_dec, comp_bytes, d_cblocks, d_in, d_errs, st);
    d_cb = d_cblocks;
    if ((rc = size_pass(true))) return rc;
  }

  const uint32_t n_rec = in_rec[N];
  const uint64_t K = in_key[N];
  std::vector<JobDev> hjobs(n_jobs);
  uint64_t out_cap = 4096, bm_cap = 64;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    JobDev& jd = hjobs[j];
    memset(&jd, 0, sizeof jd);
    jd.snapshot = jobs[j].snapshot;
    jd.bottommost = jobs[j].bottommost ? 1u : 0u;
    jd.flags = o->flags;
    jd.rec_begin = in_rec[job_in_first[j]];
    jd.rec_end = in_rec[job_in_first[j + 1]];
    jd.in_first = job_in_first[j];
    const uint64_t nj = jd.rec_end - jd.rec_begin;
    const uint64_t kj = in_key[job_in_first[j + 1]] - in_key[job_in_first[j]];
    // Output bound: data <= K + V + 24n; index <= K + 31n + 9 per table; filter, metaindex and
    // footer <= n*bpk/8 + 116 per table; tables <= n.
    out_cap += 2 * kj + job_in_bytes[j] + 200 * nj + 256;
    out_cap += filter_array_extra(fmt, 2 * kj + job_in_bytes[j] + 24 * nj, nj);
    bm_cap += nj * fmt.bpk / 32 + 5 * nj + 8;
  }
  // compressed inputs (R4c): their values take up to their decompressed bytes in the output
  out_cap += comp_bytes + (fmt.flags & LUDA_F_FILTER_ARRAY ? comp_bytes >> (kFilterBaseLg - 3) : 0);
  // merge schedule: linked inputs form one sorted run
  MergeSched ms;
  ms.tile = tuning().merge_tile;
  {
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> runs(n_jobs);
    for (uint32_t j = 0; j < n_jobs; ++j)
      for (uint32_t i = job_in_first[j]; i < job_in_first[j + 1];) {
        uint32_t e = i;
        while (e + 1 < job_in_first[j + 1] && link[e]) ++e;
        runs[j].push_back({in_rec[i], in_rec[e + 1] - in_rec[i]});
        i = e + 1;
      }
    merge_schedule(runs, &ms);
  }
  const std::vector<MergeSpan>& spans = ms.spans;
  const std::vector<uint32_t>& pass_span0 = ms.pass_span0;
  const std::vector<uint32_t>& pass_nspans = ms.pass_nspans;
  const std::vector<uint32_t>& pass_ntiles = ms.pass_ntiles;
  const uint32_t max_tiles = ms.max_tiles;

  // ---- execute -------------------------------------------------------------------------------
  const uint32_t cap = n_rec;
  const uint64_t key_cap = 2 * K + 64;
  Layout LC;
  Recs recs;
  uint8_t* d_arena;
  uint32_t *d_ord0, *d_ord1, *d_keep, *d_pos, *d_co, *d_chunkF, *d_snap;
  MKey *d_pfx0, *d_pfx1;
  MergeSpan* d_spans;
  KeptIn* d_kin;
  PackBufs pb;
  const uint64_t chunk_cap = uint64_t(n_chunks) + 16;
  auto layoutC = [&](Layout& L) {
    recs = recs_layout(L, n_rec);
    d_kin = L.take<KeptIn>(cached ? N + 1 : 1);
    d_arena = L.take<uint8_t>(K + 64);
    d_chunkF = L.take<uint32_t>(chunk_cap);
    d_snap = L.take<uint32_t>(2ull * n_rec + 2ull * NB + 2);
    d_ord0 = L.take<uint32_t>(n_rec + 1);
    d_ord1 = L.take<uint32_t>(n_rec + 1);
    d_pfx0 = L.take<MKey>(n_rec + 1);
    d_pfx1 = L.take<MKey>(n_rec + 1);
    d_keep = L.take<uint32_t>(n_rec + 1);
    d_pos = L.take<uint32_t>(n_rec + 1);
    d_co = L.take<uint32_t>(max_tiles + 1);
    d_spans = L.take<MergeSpan>(spans.size() + 1);
    pack_layout(L, pb, cap, bm_cap, key_cap, filter_slot_cap(fmt, out_cap, cap), cz_raw_cap(fmt, out_cap, cap),
                cz_stream_cap(fmt, out_cap, cap), n_jobs);
  };
  layoutC(LC);
  const uint64_t out_room = (out_cap + 255) & ~uint64_t(255);
  uint64_t keep_bytes = kept_bytes(o, host_out, fmt, cap, K);
  if (gate && !gate->admit(LA.off + LB.off + LC.off + out_room + keep_bytes + gate->extra)) {
    set_detail("the job was not admitted (server shutting down)");
    return LUDA_ERR_OOM;
  }
  uint8_t* bufC = static_cast<uint8_t*>(mem.get(LC.off));
  if (!bufC) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  guard.ps.push_back(bufC);
  LC = Layout{};
  LC.base = bufC;
  layoutC(LC);
  uint8_t* d_out = static_cast<uint8_t*>(mem.get(out_room + keep_bytes));
  if (!d_out && keep_bytes) {  // no room for the kept run: the tables alone
    cudaGetLastError();
    keep_bytes = 0;
    d_out = static_cast<uint8_t*>(mem.get(out_cap));
  }
  if (!d_out) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  bool out_owned = false;
  struct OutGuard {
    const DevMem& m;
    uint8_t* p;
    bool* owned;
    ~OutGuard() {
      if (!*owned) m.put(p);
    }
  } out_guard{mem, d_out, &out_owned};

  CK(stage_copy(&d_cnt->n_rec, pin(&n_rec, sizeof n_rec), sizeof n_rec, cudaMemcpyHostToDevice, st));
  CK(stage_copy(d_jobs, pin(hjobs.data(), sizeof(JobDev) * n_jobs), sizeof(JobDev) * n_jobs,
                     cudaMemcpyHostToDevice, st));
  if (!spans.empty())
    CK(stage_copy(d_spans, pin(spans.data(), sizeof(MergeSpan) * spans.size()), sizeof(MergeSpan) * spans.size(),
                       cudaMemcpyHostToDevice, st));

  tr.mark(4, st);
  // one read of every data block: checksum (stored blocks; compressed ones were verified on
  // their stored bytes above), records, keys and value registers
  {
    // records and keys here; the checksums (stored blocks; compressed ones were verified on
    // their stored bytes above) and the value registers on the side stream, beside the
    // merge, drop rule and cuts (joined with the data block trailers)
    UnpArgs ua{d_cb,          NB,    d_in,       d_nrec,   d_kbytes, nullptr, nullptr,
               d_hdr,         d_rec_first, d_key_first, d_chunk_first, d_chunkF, d_snap, recs,
               d_arena,       d_errs, d_errs + n_jobs + 1, comp_blocks == 0, &d_cnt->unp_next};
    if (cached) {
      // records from the kept runs, each input's keys in one copy
      tr.mark(11, st);
      tr.mark(12, st);
      std::vector<KeptIn> hk(N);
      uint64_t max_count = 0;
      for (uint32_t i = 0; i < N; ++i) {
        hk[i] = KeptIn{kin[i].run, kin[i].first, kin[i].count, kin[i].key_first, in_rec[i], in_key[i]};
        max_count = std::max(max_count, kin[i].count);
        if (kin[i].kbytes)
          CK(stage_copy(d_arena + in_key[i], kin[i].run.arena + kin[i].key_first, kin[i].kbytes,
                             cudaMemcpyDeviceToDevice, st));
      }
      CK(stage_copy(d_kin, pin(hk.data(), sizeof(KeptIn) * N), sizeof(KeptIn) * N, cudaMemcpyHostToDevice, st));
      launch_kept_gather(d_kin, N, max_count, recs, st);
      g_kept_used += N;
    } else {
      CK(fork_join(side, 0, st, side->s));
      tr.mark(11, side->s);
      uint64_t in_total = 0;
      for (uint64_t v : job_in_bytes) in_total += v;
      launch_unpack_crc(ua, tabs, tuning().crc_ctas, unpack_half(in_total, NB), side->s);
      tr.mark(12, side->s);
      launch_unpack_keys(ua, st);
    }
  }
  tr.mark(5, st);
  if (!cached) {
    // (a kept run was checked when its table was written)
    launch_check_index(d_cb, NB, d_in, d_nrec, d_rec_first, recs, d_arena, d_errs, st);
    launch_check_order(recs, d_arena, n_rec, d_in, d_errs, st);
  }
  launch_sort_init(d_ord0, d_pfx0, recs, d_arena, n_rec, st);
  for (size_t p = 0; p < pass_span0.size(); ++p)
    launch_merge_pass(d_spans + pass_span0[p], pass_nspans[p], pass_ntiles[p], ms.tile, d_ord0, d_pfx0, d_ord1,
                      d_pfx1, recs, d_arena, st);
  uint32_t* src_o = ms.final_buf ? d_ord1 : d_ord0;
  tr.mark(6, st);
  launch_gc_flags(src_o, n_rec, d_jobs, n_jobs, recs, d_arena, d_keep, d_errs, st, d_ranges, d_bounds);
  CK((exclusive_scan<uint32_t, uint32_t>(d_keep, d_pos, n_rec, nullptr, pb.scan_tmp, st)));
  launch_gc_compact(src_o, d_keep, d_pos, n_rec, pb.surv, st);
  launch_job_surv(d_jobs, n_jobs, d_pos, n_rec, d_cnt, st);
  // the SMs the stored blocks' checksum kernel left join it for the blocks still to do
  if (comp_blocks)
    launch_block_verify(d_blocks, NB, d_in, d_errs, d_errs + n_jobs + 1, tabs, &d_cnt->crc_next_in, true, st);
  CK(cudaGetLastError());
  if ((rc = run_pack(pb, d_cnt, d_jobs, n_jobs, d_errs, cap, recs, d_arena, fmt, d_out, out_cap, bm_cap, tabs, st,
                     side, &tr)))
    return rc;
  if (comp_blocks) CK(cudaStreamWaitEvent(st, side->ev[1], 0));
  CK(cudaStreamWaitEvent(st, side->ev[3], 0));
  // LUDA_F_KEEP_DECODED: the survivors kept as a sorted run for the new tables
  KeptGuard kguard;
  if ((rc = kept_start(o, keep_bytes ? d_out + out_room : nullptr, host_out, pb, d_cnt, cap, K, recs, d_out, st,
                       &kguard.k)))
    return rc;
  tr.mark(10, st);
  tdev.stop(st);

  // ---- collect -------------------------------------------------------------------------------
  Collected col;
  if ((rc = collect(d_cnt, d_jobs, d_errs, pb, n_jobs, &col, st))) return rc;
  Holder* h = new Holder();
  uint8_t* base = d_out;
  double d2h = 0;
  if (host_out) {
    h->pinned = pinned_get(col.cnt.out_bytes + 16, &h->pinned_cap);
    if (!h->pinned) {
      holder_release(h);
      return cuda_fail(cudaErrorMemoryAllocation, "pinned host allocation");
    }
    Timer t;
    if (gate) gate->copy_begin(1);
    t.start(st);
    if (col.cnt.out_bytes)
      if (stage_copy(h->pinned, d_out, col.cnt.out_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        if (gate) gate->copy_end(1);
        holder_release(h);
        return cuda_fail(cudaGetLastError(), "copy of the new tables to the host");
      }
    t.stop(st);
    d2h = t.ms();  // waits for the copy
    if (gate) gate->copy_end(1);
    base = h->pinned;
  } else {
    h->dev = d_out;
    h->dev_free = o->dev_free;
    h->ctx = o->alloc_ctx;
    out_owned = true;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    holder_release(h);
    return cuda_fail(cudaGetLastError(), "stream synchronize");
  }
  const double dev_ms = tdev.ms();
  if (ms_device) *ms_device = dev_ms;
  if (ms_d2h) *ms_d2h = d2h;
  if (tr.on) {
    stage_ms[0] = tr.span(0, 3);
    stage_ms[1] = tr.span(11, 12);  // the unpack's checksum pass (side stream, beside the later stages)
    stage_ms[2] = tr.span(4, 5);
    stage_ms[3] = tr.span(5, 6);
    stage_ms[4] = tr.span(6, 7);
    stage_ms[5] = tr.span(7, 8);
    stage_ms[6] = tr.span(8, 10);
    stage_ms[7] = tr.span(0, 10);
    uint64_t out_data = 0;
    for (const FileMeta& m : col.meta) out_data += m.data_size;
    stage_bytes[1] = col.cnt.in_data_bytes;
    stage_bytes[5] = out_data + col.cnt.surv_kv_bytes;
  }
  luda_status first = LUDA_OK;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    outs[j].status = err_status(col.errs[j], j, n_jobs);
    if (outs[j].status && !first) first = luda_status(outs[j].status);
  }
  if (kguard.k) {
    kept_register(kguard.k, col, n_jobs, outs, base);
    h->kept = kguard.k;  // freed with the tables' memory
    kguard.k = nullptr;
  }
  fill_outputs(col, n_jobs, base, h, outs);
  holder_release(h);
  if (first) {
    // keep the detail of the first failing job
    for (uint32_t j = 0; j < n_jobs; ++j)
      if (outs[j].status) {
        err_status(col.errs[j], j, n_jobs);
        break;
      }
  }
  return LUDA_OK;
}


// Build tables from one sorted run (memtable flush): records straight from the run's
// arrays, then the same pack stages as a compaction.
luda_status run_build(const luda_run* run, bool host_in, const luda_options* o, luda_outputs* out, bool host_out) {
  Fmt fmt;
  luda_status rc = opts_check(o, &fmt);
  if (rc) return rc;
  const TuningScope tuned(o->tuning);
  memset(out, 0, sizeof *out);
  if (!run) {
    set_detail("run is NULL");
    return LUDA_ERR_INVALID_ARG;
  }
  const uint64_t n64 = run->n;
  if (n64 >= (1ull << 31)) {
    set_detail("run too large (%llu entries)", (unsigned long long)n64);
    return LUDA_ERR_INVALID_ARG;
  }
  if (!run->ukoff || !run->voff || (n64 && (!run->ukeys || !run->seqs || !run->types || !run->vals))) {
    set_detail("run arrays are NULL");
    return LUDA_ERR_INVALID_ARG;
  }
  const uint32_t n = uint32_t(n64);
  CrcTabs tabs;
  if ((rc = get_tabs(&tabs))) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(o->stream);
  const DevMem mem{o, st};
  uint64_t ku = 0, vb = 0;
  if (host_in) {
    ku = run->ukoff[n];
    vb = run->voff[n];
  } else {
    CK(cudaMemcpyAsync(&ku, run->ukoff + n, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&vb, run->voff + n, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  const uint64_t K = ku + 8ull * n;
  const uint64_t out_cap = 2 * K + vb + 200ull * n + 4096 + filter_array_extra(fmt, 2 * K + vb + 24ull * n, n);
  const uint64_t bm_cap = uint64_t(n) * fmt.bpk / 32 + 5ull * n + 64;
  Layout L;
  Recs recs;
  uint8_t *arena, *h_ukeys, *h_types, *h_vals;
  uint64_t *h_ukoff, *h_seqs, *h_voff;
  DErr* d_err;
  JobDev* d_job;
  Counts* d_cnt;
  PackBufs pb;
  auto lay = [&](Layout& l) {
    recs = recs_layout(l, n);
    arena = l.take<uint8_t>(K + 64);
    d_err = l.take<DErr>(4);  // main chain and input checksums (collect's layout)
    d_job = l.take<JobDev>(1);
    d_cnt = l.take<Counts>(1);
    pack_layout(l, pb, n, bm_cap, 2 * K + 64, filter_slot_cap(fmt, out_cap, n), cz_raw_cap(fmt, out_cap, n),
                cz_stream_cap(fmt, out_cap, n), 1);
    if (host_in) {
      h_ukeys = l.take<uint8_t>(ku + 16);
      h_ukoff = l.take<uint64_t>(n + 1);
      h_seqs = l.take<uint64_t>(n + 1);
      h_types = l.take<uint8_t>(n + 1);
      h_vals = l.take<uint8_t>(vb + 16);
      h_voff = l.take<uint64_t>(n + 1);
    }
  };
  lay(L);
  uint8_t* buf = static_cast<uint8_t*>(mem.get(L.off));
  if (!buf) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  const uint64_t out_room = (out_cap + 255) & ~uint64_t(255);
  uint64_t keep_bytes = kept_bytes(o, host_out, fmt, n, K);
  uint8_t* d_out = static_cast<uint8_t*>(mem.get(out_room + keep_bytes));
  if (!d_out && keep_bytes) {  // no room for the kept run: the tables alone
    cudaGetLastError();
    keep_bytes = 0;
    d_out = static_cast<uint8_t*>(mem.get(out_cap));
  }
  if (!d_out) {
    mem.put(buf);
    return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  }
  bool out_owned = false;
  struct G {
    const DevMem& m;
    uint8_t* a;
    uint8_t* b;
    bool* owned;
    ~G() {
      m.put(a);
      if (!*owned) m.put(b);
    }
  } g{mem, buf, d_out, &out_owned};
  L = Layout{};
  L.base = buf;
  lay(L);
  const uint8_t *ukeys = run->ukeys, *types = run->types, *vals = run->vals;
  const uint64_t *ukoff = run->ukoff, *seqs = run->seqs, *voff = run->voff;
  Timer th;
  th.start(st);
  if (host_in) {
    if (ku) CK(cudaMemcpyAsync(h_ukeys, run->ukeys, ku, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h_ukoff, run->ukoff, 8ull * (n + 1), cudaMemcpyHostToDevice, st));
    if (n) {
      CK(cudaMemcpyAsync(h_seqs, run->seqs, 8ull * n, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(h_types, run->types, n, cudaMemcpyHostToDevice, st));
    }
    if (vb) CK(cudaMemcpyAsync(h_vals, run->vals, vb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h_voff, run->voff, 8ull * (n + 1), cudaMemcpyHostToDevice, st));
    ukeys = h_ukeys;
    types = h_types;
    vals = h_vals;
    ukoff = h_ukoff;
    seqs = h_seqs;
    voff = h_voff;
  }
  th.stop(st);
  Timer td;
  td.start(st);
  JobDev jd{};
  jd.rec_end = n;
  jd.surv_end = n;
  Counts hc{};
  hc.n_rec = n;
  hc.n_surv = n;
  CK(cudaMemsetAsync(d_err, 0, sizeof(DErr) * 4, st));
  CK(cudaMemcpyAsync(d_job, &jd, sizeof jd, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_cnt, &hc, sizeof hc, cudaMemcpyHostToDevice, st));
  launch_build_records(ukeys, ukoff, seqs, types, vals, voff, n, recs, arena, pb.surv, d_err, st);
  launch_build_check(recs, arena, n, d_err, st);
  launch_value_crc(recs, nullptr, n, tabs, st);
  CK(cudaGetLastError());
  Side* side = nullptr;
  if ((rc = get_side(&side))) return rc;
  if ((rc = run_pack(pb, d_cnt, d_job, 1, d_err, n, recs, arena, fmt, d_out, out_cap, bm_cap, tabs, st, side)))
    return rc;
  CK(cudaStreamWaitEvent(st, side->ev[3], 0));
  KeptGuard kguard;
  if ((rc = kept_start(o, keep_bytes ? d_out + out_room : nullptr, host_out, pb, d_cnt, n, K, recs, d_out, st,
                       &kguard.k)))
    return rc;
  td.stop(st);
  Collected col;
  t_stage.reset();  // nothing of this call was staged before (its copies are synchronous)
  if ((rc = collect(d_cnt, d_job, d_err, pb, 1, &col, st))) return rc;
  Holder* h = new Holder();
  uint8_t* base = d_out;
  double d2h = 0;
  if (host_out) {
    h->pinned = pinned_get(col.cnt.out_bytes + 16, &h->pinned_cap);
    if (!h->pinned) {
      holder_release(h);
      return cuda_fail(cudaErrorMemoryAllocation, "pinned host allocation");
    }
    Timer t;
    t.start(st);
    if (col.cnt.out_bytes) CK(cudaMemcpyAsync(h->pinned, d_out, col.cnt.out_bytes, cudaMemcpyDeviceToHost, st));
    t.stop(st);
    d2h = t.ms();
    base = h->pinned;
  } else {
    h->dev = d_out;
    h->dev_free = o->dev_free;
    h->ctx = o->alloc_ctx;
    out_owned = true;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    holder_release(h);
    return cuda_fail(cudaGetLastError(), "stream synchronize");
  }
  out->status = err_status(col.errs[0], 0, 1);
  if (kguard.k) {
    kept_register(kguard.k, col, 1, out, base);
    h->kept = kguard.k;
    kguard.k = nullptr;
  }
  fill_outputs(col, 1, base, h, out);
  holder_release(h);
  out->n_in_entries = n;
  out->n_dropped = 0;
  out->ms_h2d = host_in ? th.ms() : 0;
  out->ms_device = td.ms();
  out->ms_d2h = d2h;
  if (out->status) {
    const luda_status s = luda_status(out->status);
    luda_outputs_free(out);
    out->status = s;
    return s;
  }
  return LUDA_OK;
}


// ---- plans: sized once, captured in one CUDA graph, replayed -------------------------------
struct PlanImpl {
  int device = 0;
  cudaStream_t st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  uint32_t n_jobs = 0;
  uint64_t launches = 0;
  std::vector<void*> bufs;
  // device state the collect step reads
  Counts* d_cnt = nullptr;
  JobDev* d_jobs = nullptr;
  DErr* d_errs = nullptr;
  PackBufs pb{};
  uint8_t* d_out = nullptr;
  bool ran = false;
  ~PlanImpl() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (done) cudaEventDestroy(done);
    if (st) cudaStreamSynchronize(st);
    for (void* p : bufs) cudaFree(p);
    if (st) cudaStreamDestroy(st);
  }
};

luda_status plan_build(const luda_job* jobs, uint32_t n_jobs, const luda_options* o, PlanImpl* P) {
  Fmt fmt;
  luda_status rc = opts_check(o, &fmt);
  if (rc) return rc;
  for (uint32_t j = 0; j < n_jobs; ++j)
    if (jobs[j].range_lo || jobs[j].range_hi) {
      set_detail("job %u: ranged jobs are not supported in plans", j);
      return LUDA_ERR_INVALID_ARG;
    }
  const TuningScope tuned(o->tuning);
  CrcTabs tabs;
  if ((rc = get_tabs(&tabs))) return rc;
  CK(cudaGetDevice(&P->device));
  CK(cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming));
  cudaStream_t st = P->st;
  P->n_jobs = n_jobs;
  auto alloc = [&](size_t n) -> uint8_t* {
    void* p = nullptr;
    if (cudaMalloc(&p, n ? n : 256) != cudaSuccess) return nullptr;
    P->bufs.push_back(p);
    return static_cast<uint8_t*>(p);
  };
  // inputs
  std::vector<DInput> hin;
  std::vector<uint64_t> job_in_bytes(n_jobs, 0);
  std::vector<uint32_t> job_in_first(n_jobs + 1, 0);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    job_in_first[j] = uint32_t(hin.size());
    if (jobs[j].n_inputs && !jobs[j].inputs) {
      set_detail("job %u: inputs is NULL", j);
      return LUDA_ERR_INVALID_ARG;
    }
    for (uint32_t i = 0; i < jobs[j].n_inputs; ++i) {
      DInput d{};
      d.data = jobs[j].inputs[i].data;
      d.size = jobs[j].inputs[i].size;
      if (!d.data && d.size) {
        set_detail("job %u input %u: data is NULL", j, i);
        return LUDA_ERR_INVALID_ARG;
      }
      d.job = j;
      d.local = i;
      hin.push_back(d);
      job_in_bytes[j] += d.size;
    }
  }
  job_in_first[n_jobs] = uint32_t(hin.size());
  const uint32_t N = uint32_t(hin.size());
  Layout LA;
  DInput* d_in;
  DErr* d_errs;
  JobDev* d_jobs;
  uint32_t *d_in_blk_first, *d_plan_nblk, *d_nrec_const;
  Counts* d_cnt;
  CrcMsg* d_msgs;
  auto layA = [&](Layout& L) {
    d_in = L.take<DInput>(N + 1);
    d_errs = L.take<DErr>(2 * (n_jobs + 1));
    d_jobs = L.take<JobDev>(n_jobs + 1);
    d_in_blk_first = L.take<uint32_t>(N + 1);
    d_plan_nblk = L.take<uint32_t>(N + 1);
    d_nrec_const = L.take<uint32_t>(1);
    d_cnt = L.take<Counts>(1);
    d_msgs = L.take<CrcMsg>(N + 1);
  };
  layA(LA);
  LA.base = alloc(LA.off);
  if (!LA.base) return cuda_fail(cudaErrorMemoryAllocation, "plan allocation");
  LA.off = 0;
  layA(LA);
  CK(cudaMemsetAsync(d_errs, 0, sizeof(DErr) * 2 * (n_jobs + 1), st));
  CK(cudaMemsetAsync(d_cnt, 0, sizeof(Counts), st));
  if (N) CK(cudaMemcpyAsync(d_in, hin.data(), sizeof(DInput) * N, cudaMemcpyHostToDevice, st));
  launch_footers(d_in, N, d_errs, d_msgs, tabs, st);
  if (N) CK(cudaMemcpyAsync(hin.data(), d_in, sizeof(DInput) * N, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<uint32_t> in_blk_first(N + 1, 0), plan_nblk(N + 1, 0);
  uint64_t NB64 = 0;
  for (uint32_t i = 0; i < N; ++i) {
    hin[i].blk_first = uint32_t(NB64);
    in_blk_first[i] = uint32_t(NB64);
    plan_nblk[i] = hin[i].nblk;
    NB64 += hin[i].nblk;
  }
  in_blk_first[N] = uint32_t(NB64);
  if (NB64 >= (1ull << 31)) {
    set_detail("too many data blocks in one plan");
    return LUDA_ERR_INVALID_ARG;
  }
  const uint32_t NB = uint32_t(NB64);
  if (N) {
    CK(cudaMemcpyAsync(d_in, hin.data(), sizeof(DInput) * N, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_in_blk_first, in_blk_first.data(), sizeof(uint32_t) * (N + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_plan_nblk, plan_nblk.data(), sizeof(uint32_t) * (N + 1), cudaMemcpyHostToDevice, st));
  }
  Layout LB;
  BlockDesc* d_blocks;
  uint32_t *d_nrec, *d_rec_first, *d_in_rec, *d_plan_nrec;
  uint64_t *d_kbytes, *d_key_first, *d_in_key, *d_plan_kbytes;
  uint2* d_hdr;  // the walk's entry table
  uint32_t *d_nch, *d_chunk_first;  // the unpack's chunks per block and their offsets
  void* d_tmpB;
  uint8_t *d_link, *d_plan_link;
  auto layB = [&](Layout& L) {
    d_blocks = L.take<BlockDesc>(NB + 1);
    d_hdr = L.take<uint2>(uint64_t(NB) * kHdrMax + 1);
    d_nch = L.take<uint32_t>(NB + 1);
    d_chunk_first = L.take<uint32_t>(NB + 1);
    d_nrec = L.take<uint32_t>(NB + 1);
    d_kbytes = L.take<uint64_t>(NB + 1);
    d_plan_nrec = L.take<uint32_t>(NB + 1);
    d_plan_kbytes = L.take<uint64_t>(NB + 1);
    d_rec_first = L.take<uint32_t>(NB + 1);
    d_key_first = L.take<uint64_t>(NB + 1);
    d_in_rec = L.take<uint32_t>(N + 1);
    d_in_key = L.take<uint64_t>(N + 1);
    d_link = L.take<uint8_t>(N + 1);
    d_plan_link = L.take<uint8_t>(N + 1);
    d_tmpB = L.take<uint8_t>(scan_temp_bytes(NB + 1));
  };
  layB(LB);
  LB.base = alloc(LB.off);
  if (!LB.base) return cuda_fail(cudaErrorMemoryAllocation, "plan allocation");
  LB.off = 0;
  layB(LB);
  launch_index_entries(d_in, N, d_in_blk_first, NB, d_blocks, d_errs, st);
  launch_block_scan(d_blocks, NB, d_in, d_nrec, d_kbytes, d_errs, d_cnt, d_hdr, tabs, st, d_nch);
  CK((exclusive_scan<uint32_t, uint32_t>(d_nch, d_chunk_first, NB, nullptr, d_tmpB, st)));
  launch_zero_failed(d_blocks, NB, d_errs, d_nrec, d_kbytes, st);
  launch_run_links(d_in, N, d_blocks, d_errs, d_plan_link, st);
  if (NB) {
    CK(cudaMemcpyAsync(d_plan_nrec, d_nrec, sizeof(uint32_t) * NB, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d_plan_kbytes, d_kbytes, sizeof(uint64_t) * NB, cudaMemcpyDeviceToDevice, st));
  }
  CK((exclusive_scan<uint32_t, uint32_t>(d_nrec, d_rec_first, NB, nullptr, d_tmpB, st)));
  CK((exclusive_scan<uint64_t, uint64_t>(d_kbytes, d_key_first, NB, nullptr, d_tmpB, st)));
  launch_input_ranges(d_in, N, d_rec_first, d_key_first, d_in_rec, d_in_key, st);
  CK(cudaGetLastError());
  std::vector<uint32_t> in_rec(N + 1);
  std::vector<uint64_t> in_key(N + 1);
  std::vector<uint8_t> link(N + 1, 0);
  CK(cudaMemcpyAsync(in_rec.data(), d_in_rec, sizeof(uint32_t) * (N + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(in_key.data(), d_in_key, sizeof(uint64_t) * (N + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&fmt.max_kv, &d_cnt->max_kv, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  uint32_t n_chunks = 0;
  CK(cudaMemcpyAsync(&n_chunks, d_chunk_first + NB, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  if (N) CK(cudaMemcpyAsync(link.data(), d_plan_link, N, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint32_t n_rec = in_rec[N];
  const uint64_t K = in_key[N];
  std::vector<JobDev> hjobs(n_jobs);
  uint64_t out_cap = 4096, bm_cap = 64;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    JobDev& jd = hjobs[j];
    memset(&jd, 0, sizeof jd);
    jd.snapshot = jobs[j].smallest_snapshot;
    jd.bottommost = jobs[j].bottommost ? 1u : 0u;
    jd.flags = o->flags;
    jd.rec_begin = in_rec[job_in_first[j]];
    jd.rec_end = in_rec[job_in_first[j + 1]];
    jd.in_first = job_in_first[j];
    const uint64_t nj = jd.rec_end - jd.rec_begin;
    const uint64_t kj = in_key[job_in_first[j + 1]] - in_key[job_in_first[j]];
    out_cap += 2 * kj + job_in_bytes[j] + 200 * nj + 256;
    out_cap += filter_array_extra(fmt, 2 * kj + job_in_bytes[j] + 24 * nj, nj);
    bm_cap += nj * fmt.bpk / 32 + 5 * nj + 8;
  }
  // merge schedule (as in run_compaction); replays check that the links still hold
  MergeSched ms;
  ms.tile = tuning().merge_tile;
  {
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> runs(n_jobs);
    for (uint32_t j = 0; j < n_jobs; ++j)
      for (uint32_t i = job_in_first[j]; i < job_in_first[j + 1];) {
        uint32_t e = i;
        while (e + 1 < job_in_first[j + 1] && link[e]) ++e;
        runs[j].push_back({in_rec[i], in_rec[e + 1] - in_rec[i]});
        i = e + 1;
      }
    merge_schedule(runs, &ms);
  }
  const std::vector<MergeSpan>& spans = ms.spans;
  const std::vector<uint32_t>& pass_span0 = ms.pass_span0;
  const std::vector<uint32_t>& pass_nspans = ms.pass_nspans;
  const std::vector<uint32_t>& pass_ntiles = ms.pass_ntiles;
  const uint32_t max_tiles = ms.max_tiles;
  const uint32_t cap = n_rec;
  Layout LC;
  Recs recs;
  uint8_t* d_arena;
  uint32_t *d_ord0, *d_ord1, *d_keep, *d_pos, *d_co, *d_chunkF, *d_snap;
  MKey *d_pfx0, *d_pfx1;
  MergeSpan* d_spans;
  PackBufs pb;
  const uint64_t chunk_cap = uint64_t(n_chunks) + 16;
  auto layC = [&](Layout& L) {
    recs = recs_layout(L, n_rec);
    d_arena = L.take<uint8_t>(K + 64);
    d_chunkF = L.take<uint32_t>(chunk_cap);
    d_snap = L.take<uint32_t>(2ull * n_rec + 2ull * NB + 2);
    d_ord0 = L.take<uint32_t>(n_rec + 1);
    d_ord1 = L.take<uint32_t>(n_rec + 1);
    d_pfx0 = L.take<MKey>(n_rec + 1);
    d_pfx1 = L.take<MKey>(n_rec + 1);
    d_keep = L.take<uint32_t>(n_rec + 1);
    d_pos = L.take<uint32_t>(n_rec + 1);
    d_co = L.take<uint32_t>(max_tiles + 1);
    d_spans = L.take<MergeSpan>(spans.size() + 1);
    pack_layout(L, pb, cap, bm_cap, 2 * K + 64, filter_slot_cap(fmt, out_cap, cap), cz_raw_cap(fmt, out_cap, cap),
                cz_stream_cap(fmt, out_cap, cap), n_jobs);
  };
  layC(LC);
  LC.base = alloc(LC.off);
  if (!LC.base) return cuda_fail(cudaErrorMemoryAllocation, "plan allocation");
  LC.off = 0;
  layC(LC);
  uint8_t* d_out = alloc(out_cap);
  if (!d_out) return cuda_fail(cudaErrorMemoryAllocation, "plan allocation");
  CK(cudaMemcpyAsync(d_jobs, hjobs.data(), sizeof(JobDev) * n_jobs, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_nrec_const, &n_rec, sizeof n_rec, cudaMemcpyHostToDevice, st));
  if (!spans.empty())
    CK(cudaMemcpyAsync(d_spans, spans.data(), sizeof(MergeSpan) * spans.size(), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  // ---- capture the whole pipeline --------------------------------------------------------
  Side* side = nullptr;
  if ((rc = get_side(&side))) return rc;
  const uint64_t l0 = g_launches.load();
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  auto body = [&]() -> luda_status {
    CK(cudaMemsetAsync(d_errs, 0, sizeof(DErr) * 2 * (n_jobs + 1), st));
    CK(cudaMemsetAsync(d_cnt, 0, sizeof(Counts), st));
    CK(cudaMemcpyAsync(&d_cnt->n_rec, d_nrec_const, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    launch_footers_read(d_in, N, d_errs, d_msgs, st);
    CK(fork_join(side, 4, st, side->s));
    launch_index_crc(d_msgs, N, d_errs + n_jobs + 1, tabs, side->s);
    launch_footers_finish(d_in, N, d_errs, st);
    launch_plan_checks(d_in, N, d_plan_nblk, d_errs, st);
    launch_index_entries(d_in, N, d_in_blk_first, NB, d_blocks, d_errs, st);
    launch_block_walk(d_blocks, NB, d_in, d_nrec, d_kbytes, d_errs, d_cnt, d_hdr, st);
    launch_plan_check_recs(d_blocks, NB, d_nrec, d_kbytes, d_plan_nrec, d_plan_kbytes, d_in, d_errs, st);
    launch_run_links(d_in, N, d_blocks, d_errs, d_link, st);
    launch_plan_check_links(d_link, d_plan_link, N, d_in, d_errs, st);
    {
      // the chunk offsets are the plan's (a block with more chunks than planned takes the
      // path without boundaries)
      UnpArgs ua{d_blocks,      NB,     d_in,       d_nrec,   d_kbytes, d_plan_nrec, d_plan_kbytes,
                 d_hdr,         d_rec_first, d_key_first, d_chunk_first, d_chunkF, d_snap, recs,
                 d_arena,       d_errs, d_errs + n_jobs + 1, true, &d_cnt->unp_next};
      CK(fork_join(side, 0, st, side->s));
      uint64_t in_total = 0;
      for (const DInput& d : hin) in_total += d.size;
      launch_unpack_crc(ua, tabs, tuning().crc_ctas, unpack_half(in_total, NB), side->s);
      launch_unpack_keys(ua, st);
    }
    launch_plan_sanitize(recs, n_rec, d_jobs, n_jobs, d_errs, d_arena, st);
    launch_check_index(d_blocks, NB, d_in, d_nrec, d_rec_first, recs, d_arena, d_errs, st);
    launch_check_order(recs, d_arena, n_rec, d_in, d_errs, st);
    launch_sort_init(d_ord0, d_pfx0, recs, d_arena, n_rec, st);
    for (size_t p = 0; p < pass_span0.size(); ++p)
      launch_merge_pass(d_spans + pass_span0[p], pass_nspans[p], pass_ntiles[p], ms.tile, d_ord0, d_pfx0, d_ord1,
                        d_pfx1, recs, d_arena, st);
    uint32_t* src_o = ms.final_buf ? d_ord1 : d_ord0;
    launch_gc_flags(src_o, n_rec, d_jobs, n_jobs, recs, d_arena, d_keep, d_errs, st);
    CK((exclusive_scan<uint32_t, uint32_t>(d_keep, d_pos, n_rec, nullptr, pb.scan_tmp, st)));
    launch_gc_compact(src_o, d_keep, d_pos, n_rec, pb.surv, st);
    launch_job_surv(d_jobs, n_jobs, d_pos, n_rec, d_cnt, st);
    luda_status prc = run_pack(pb, d_cnt, d_jobs, n_jobs, d_errs, cap, recs, d_arena, fmt, d_out, out_cap, bm_cap,
                               tabs, st, side);
    if (prc) return prc;
    CK(cudaStreamWaitEvent(st, side->ev[3], 0));
    return LUDA_OK;
  };
  luda_status brc = body();
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &g);
  if (brc) {
    if (g) cudaGraphDestroy(g);
    return brc;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "stream capture");
  P->graph = g;
  CK(cudaGraphInstantiate(&P->exec, g, 0));
  P->launches = g_launches.load() - l0;
  P->d_cnt = d_cnt;
  P->d_jobs = d_jobs;
  P->d_errs = d_errs;
  P->pb = pb;
  P->d_out = d_out;
  return LUDA_OK;
}

}  // namespace

luda_status luda::warm_thread() {
  Side* side = nullptr;
  luda_status rc = get_side(&side);
  if (rc) return rc;
  CrcTabs tabs;
  if ((rc = get_tabs(&tabs))) return rc;
  t_stage.take(1);  // notes the size the stage wants
  t_stage.reset();  // allocates it
  return LUDA_OK;
}

namespace {

// ---- luda_compact with the inputs copied in key ranges (§III-D) ---------------------------
// The job is cut at user keys into ranges whose input bytes are about equal. The inputs'
// footers and index blocks are copied first and parsed on the device (the same kernels as
// the sizing stage); every input's data blocks are then copied range after range on one
// copy stream. Range r is compacted as a ranged job (R13) as soon as its blocks are on the
// device, and its finished tables go back to the host on a second copy stream while later
// ranges' input bytes still arrive. A table is finished when it was cut at the target
// size: the last table of a range (and every table back to a table that starts a new user
// key) is held back and compacted again with the next range, whose lower bound becomes
// that table's first user key. A compaction cuts its tables greedily from its first
// survivor and the drop rule works per user key, so every emitted table is byte for byte
// the table the whole compaction writes at that place.
struct Xfer {
  int dev = -1;
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t ev_in[65] = {};  // range r's input bytes have arrived
  cudaEvent_t ev_run = nullptr;  // a range's tables are written (call stream)
  cudaEvent_t t[4] = {};  // timing: copies in start / end, copies out start / end
};
thread_local Xfer t_xfer;

luda_status get_xfer(Xfer** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_detail("no usable CUDA device");
    return LUDA_ERR_CUDA;
  }
  Xfer& x = t_xfer;
  if (x.dev != dev) {
    if (x.in) {
      cudaStreamDestroy(x.in);
      cudaStreamDestroy(x.out);
      for (cudaEvent_t& e : x.ev_in) cudaEventDestroy(e);
      cudaEventDestroy(x.ev_run);
      for (cudaEvent_t& e : x.t) cudaEventDestroy(e);
    }
    x = Xfer{};
    if (cudaStreamCreateWithFlags(&x.in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&x.out, cudaStreamNonBlocking) != cudaSuccess) {
      set_detail("cudaStreamCreateWithFlags failed");
      return LUDA_ERR_CUDA;
    }
    bool ok = cudaEventCreateWithFlags(&x.ev_run, cudaEventDisableTiming) == cudaSuccess;
    for (cudaEvent_t& e : x.ev_in) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (cudaEvent_t& e : x.t) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    if (!ok) {
      set_detail("cudaEventCreateWithFlags failed");
      return LUDA_ERR_CUDA;
    }
    x.dev = dev;
  }
  *out = &x;
  return LUDA_OK;
}

// Bytewise order of two user keys (a proper prefix first), as cmp_user_keys on the device.
int cmp_user_host(const uint8_t* a, uint64_t na, const uint8_t* b, uint64_t nb) {
  const uint64_t m = na < nb ? na : nb;
  const int c = m ? memcmp(a, b, m) : 0;
  if (c) return c < 0 ? -1 : 1;
  return na == nb ? 0 : (na < nb ? -1 : 1);
}

// Bulk copies go in pieces of this size, so that the compaction's own small copies (its
// sizing round trip, the results) wait behind one piece at most, not behind a whole table.
constexpr uint64_t kXferPiece = 4ull << 20;

bool copy_pieces(void* dst, const void* src, uint64_t n, cudaMemcpyKind kind, cudaStream_t s) {
  for (uint64_t o = 0; o < n; o += kXferPiece)
    if (cudaMemcpyAsync(static_cast<uint8_t*>(dst) + o, static_cast<const uint8_t*>(src) + o,
                        std::min(kXferPiece, n - o), kind, s) != cudaSuccess)
      return false;
  return true;
}

// The plan of a job's copies: every data block's handle and index key as the index lists
// them (parsed on the device; the keys are read from the caller's host copy of the
// inputs), and each input's index block offset.
struct Plan {
  const luda_input* in = nullptr;
  uint8_t* const* dptr = nullptr;
  const BlockDesc* blk = nullptr;  // all inputs' blocks; input i's from first[i]
  std::vector<BlockDesc> own;      // the blocks when the host stage cannot hold them
  std::vector<uint32_t> first;
  std::vector<uint64_t> idx_off;
  const uint8_t* ukey(uint32_t i, uint32_t g) const { return in[i].data + (blk[g].ikey - dptr[i]); }
  uint32_t ulen(uint32_t g) const { return blk[g].ilen - 8; }
};

// Sets *bad unless every block has a handle and an index key of at least 8 bytes, and the
// blocks of each input follow one another in the file (trailers included, the last before
// the index block) with index keys in order.
__global__ void k_plan_check(const DInput* __restrict__ in, const uint32_t* __restrict__ first, uint32_t n_blocks,
                             const BlockDesc* __restrict__ b, uint32_t* bad) {
  for (uint64_t g = gtid(); g < n_blocks; g += gstride()) {
    const BlockDesc x = b[g];
    const uint32_t i = x.input;
    bool ok = x.ptr && x.ilen >= 8;
    if (ok && g > first[i]) {
      const BlockDesc p = b[g - 1];
      ok = p.ptr && p.ilen >= 8 && p.off + p.size + kTrailer <= x.off &&
           cmp_user_keys(p.ikey, p.ilen - 8, x.ikey, x.ilen - 8) <= 0;
    }
    if (ok && g + 1 == first[i + 1]) ok = x.off + x.size + kTrailer <= in[i].idx_off;
    if (!ok) atomicOr(bad, 1u);
  }
}

// The inputs' footers and index blocks copied to their places in the arena and parsed on
// the device (the sizing stage's kernels). False (and nothing reported) when a footer, an
// index block or a handle is not as a well-formed table has it, or the index keys or the
// blocks are out of order: the caller then runs the whole job in one piece, which reports
// the error.
bool plan_inputs(const luda_input* inputs, uint32_t N, uint8_t* const* dptr, cudaStream_t st, const DevMem& mem,
                 const CrcTabs& tabs, Plan* plan) {
  std::vector<DInput> hin(N);
  for (uint32_t i = 0; i < N; ++i) {
    if (inputs[i].size < kFooter) return false;
    hin[i] = DInput{};
    hin[i].data = dptr[i];
    hin[i].size = inputs[i].size;
    hin[i].local = i;
  }
  Layout L;
  DInput* d_in;
  DErr* d_errs;
  CrcMsg* d_msgs;
  uint32_t *d_first, *d_bad;
  auto lay = [&](Layout& l) {
    d_in = l.take<DInput>(N + 1);
    d_errs = l.take<DErr>(4);
    d_msgs = l.take<CrcMsg>(N + 1);
    d_first = l.take<uint32_t>(N + 1);
    d_bad = l.take<uint32_t>(1);
  };
  lay(L);
  uint8_t* buf = static_cast<uint8_t*>(mem.get(L.off));
  if (!buf) return false;
  L = Layout{};
  L.base = buf;
  lay(L);
  struct Put {
    const DevMem& m;
    std::vector<void*> ps;
    ~Put() {
      for (void* p : ps) m.put(p);
    }
  } put{mem, {buf}};
  HostStage& hs = t_stage;
  hs.reset();
  DErr herr[4];
  uint32_t hbad = 0;
  bool ok = cudaMemsetAsync(d_errs, 0, sizeof(DErr) * 4, st) == cudaSuccess &&
            cudaMemsetAsync(d_bad, 0, sizeof(uint32_t), st) == cudaSuccess;
  for (uint32_t i = 0; ok && i < N; ++i)
    ok = cudaMemcpyAsync(dptr[i] + inputs[i].size - kFooter, inputs[i].data + inputs[i].size - kFooter, kFooter,
                         cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(d_in, hin.data(), sizeof(DInput) * N, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (!ok) return false;
  launch_footers_read(d_in, N, d_errs, d_msgs, st);
  ok = cudaMemcpyAsync(hin.data(), d_in, sizeof(DInput) * N, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaMemcpyAsync(herr, d_errs, sizeof herr, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok || herr[0].code) return false;
  // the index blocks with their trailers (checksum and type byte)
  for (uint32_t i = 0; ok && i < N; ++i) {
    const uint64_t n = std::min<uint64_t>(hin[i].idx_size + 5, inputs[i].size - kFooter - hin[i].idx_off);
    ok = cudaMemcpyAsync(dptr[i] + hin[i].idx_off, inputs[i].data + hin[i].idx_off, n, cudaMemcpyHostToDevice,
                         st) == cudaSuccess;
  }
  if (!ok) return false;
  launch_index_crc(d_msgs, N, d_errs + 2, tabs, st);
  launch_footers_finish(d_in, N, d_errs, st);
  ok = cudaMemcpyAsync(hin.data(), d_in, sizeof(DInput) * N, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaMemcpyAsync(herr, d_errs, sizeof herr, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok || herr[0].code || herr[2].code) return false;
  std::vector<uint32_t>& first = plan->first;
  first.assign(N + 1, 0);
  for (uint32_t i = 0; i < N; ++i) {
    if (!hin[i].nblk) return false;
    hin[i].blk_first = first[i];
    first[i + 1] = first[i] + hin[i].nblk;
  }
  const uint32_t NB = first[N];
  BlockDesc* d_blocks = static_cast<BlockDesc*>(mem.get(sizeof(BlockDesc) * (NB + 1)));
  if (!d_blocks) return false;
  put.ps.push_back(d_blocks);
  BlockDesc* hb = static_cast<BlockDesc*>(hs.take(sizeof(BlockDesc) * NB));  // pinned: a fast copy
  if (!hb) {
    plan->own.resize(NB);
    hb = plan->own.data();
  }
  ok = cudaMemcpyAsync(d_in, hin.data(), sizeof(DInput) * N, cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(d_first, first.data(), sizeof(uint32_t) * (N + 1), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (!ok) return false;
  launch_index_entries(d_in, N, d_first, NB, d_blocks, d_errs, st, nullptr, nullptr);
  k_plan_check<<<grid_for(NB, 256), 256, 0, st>>>(d_in, d_first, NB, d_blocks, d_bad);
  count_launches(1);
  ok = cudaMemcpyAsync(hb, d_blocks, sizeof(BlockDesc) * NB, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaMemcpyAsync(herr, d_errs, sizeof herr, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaMemcpyAsync(&hbad, d_bad, sizeof hbad, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok || herr[0].code || hbad) return false;
  plan->in = inputs;
  plan->dptr = dptr;
  plan->blk = hb;
  plan->idx_off.resize(N);
  for (uint32_t i = 0; i < N; ++i) plan->idx_off[i] = hin[i].idx_off;
  return true;
}

// Range bounds (user keys in the caller's input bytes, strictly increasing, at most K - 1)
// that cut the inputs' data bytes into parts of about equal size, except the first and the
// last, which take half a part each: the first range's tables start going back sooner and
// the last range (its compaction and copy out, after all bytes are in) is short. Index keys
// are sampled about 1024 times over all inputs, each sample weighted by the data bytes
// since the previous sample of its input.
std::vector<std::pair<const uint8_t*, uint32_t>> range_bounds(const Plan& P, uint32_t K) {
  struct Sample {
    const uint8_t* k;
    uint32_t n;
    uint64_t w;
  };
  const uint32_t N = uint32_t(P.first.size()) - 1;
  const uint64_t stride = std::max<uint64_t>(1, P.first[N] / 1024);
  std::vector<Sample> smp;
  uint64_t total = 0;
  for (uint32_t i = 0; i < N; ++i) {
    uint64_t w = 0;
    for (uint32_t g = P.first[i]; g < P.first[i + 1]; ++g) {
      w += P.blk[g].size + kTrailer;
      if ((g - P.first[i] + 1) % stride == 0 || g + 1 == P.first[i + 1]) {
        smp.push_back({P.ukey(i, g), P.ulen(g), w});
        total += w;
        w = 0;
      }
    }
  }
  std::sort(smp.begin(), smp.end(),
            [](const Sample& a, const Sample& b) { return cmp_user_host(a.k, a.n, b.k, b.n) < 0; });
  // bound r (1 <= r < K) at the fraction (r - 1/2) / (K - 1) of the bytes
  auto frac = [&](uint32_t r) { return (double(r) - 0.5) / double(K - 1); };
  std::vector<std::pair<const uint8_t*, uint32_t>> out;
  uint64_t acc = 0;
  uint32_t r = 1;
  for (const Sample& s : smp) {
    acc += s.w;
    if (r < K && double(acc) >= frac(r) * double(total)) {
      if (out.empty() || cmp_user_host(out.back().first, out.back().second, s.k, s.n) < 0) out.push_back({s.k, s.n});
      while (r < K && double(acc) >= frac(r) * double(total)) ++r;
    }
  }
  return out;
}

// Where range r's copy of input i ends: after the first block whose index key reaches
// the bound (all blocks when none does), 16 bytes on for the decoders' windows, at most
// up to the index block (already on the device).
uint64_t range_copy_end(const Plan& P, uint32_t i, const std::pair<const uint8_t*, uint32_t>& bound) {
  uint32_t lo = P.first[i], hi = P.first[i + 1];  // first block with index key >= bound
  while (lo < hi) {
    const uint32_t mid = (lo + hi) / 2;
    if (cmp_user_host(P.ukey(i, mid), P.ulen(mid), bound.first, bound.second) < 0) lo = mid + 1;
    else hi = mid;
  }
  const BlockDesc& b = P.blk[lo < P.first[i + 1] ? lo : P.first[i + 1] - 1];
  return std::min(P.idx_off[i], b.off + b.size + kTrailer + 16);
}

// The default number of ranges: one per max(96 MiB, target) of input, 16 at most. Every
// range costs a compaction's fixed launches and round trips, which slow down while the
// copies fill the bus (on the 1 GiB job 6 to 16 ranges all take about 33.5 ms, 24 take 42).
uint32_t default_ranges(uint64_t in_bytes, uint64_t target) {
  const uint64_t per = std::max<uint64_t>(96ull << 20, target);
  return uint32_t(std::min<uint64_t>(16, in_bytes / per));
}

// The ranges' device memory when the caller brings no allocator: stream-ordered on the
// stream the library names, and a range's tables (released with stream NULL) on the
// copy-out stream, after their copy to the host.
void* range_alloc(size_t n, void* /*ctx*/, void* stream) {
  void* p = nullptr;
  return cudaMallocAsync(&p, n, static_cast<cudaStream_t>(stream)) == cudaSuccess ? p : nullptr;
}
void range_free(void* p, void* ctx, void* stream) {
  cudaFreeAsync(p, static_cast<cudaStream_t>(stream ? stream : ctx));
}

// luda_compact's job with its transfers overlapped by key ranges (see above). *handled is
// false when the job is left to the one-piece path (fewer than two ranges, a ranged job, a
// table the plan does not take); otherwise out holds the result.
luda_status compact_host_ranges(const luda_job& job, const luda_options* opts, luda_outputs* out, bool* handled) {
  *handled = false;
  const uint32_t N = job.n_inputs;
  if (!N || job.range_lo || job.range_hi || !tuning_valid(opts->tuning)) return LUDA_OK;
  uint64_t in_bytes = 0;
  for (uint32_t i = 0; i < N; ++i) in_bytes += job.inputs[i].size;
  uint32_t K = opts->tuning && opts->tuning->h2d_ranges ? opts->tuning->h2d_ranges
                                                         : default_ranges(in_bytes, opts->target_file_size);
  if (K < 2) return LUDA_OK;
  const cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
  const DevMem mem{opts, st};
  CrcTabs tabs;
  luda_status rc = get_tabs(&tabs);
  if (rc) return rc;
  Xfer* x = nullptr;
  if ((rc = get_xfer(&x))) return rc;
  std::vector<uint64_t> off(N + 1, 0);
  for (uint32_t i = 0; i < N; ++i) off[i + 1] = (off[i] + job.inputs[i].size + 255) & ~uint64_t(255);
  uint8_t* arena = static_cast<uint8_t*>(mem.get(off[N] + 256));
  if (!arena) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  std::vector<uint8_t*> dptr(N);
  for (uint32_t i = 0; i < N; ++i) dptr[i] = arena + off[i];
  Plan plan;
  if (!plan_inputs(job.inputs, N, dptr.data(), st, mem, tabs, &plan)) {
    mem.put(arena);
    return LUDA_OK;
  }
  const std::vector<uint64_t>& idx_off = plan.idx_off;
  const auto bounds = range_bounds(plan, K);
  if (bounds.empty()) {
    mem.put(arena);
    return LUDA_OK;
  }
  *handled = true;
  const uint32_t R = uint32_t(bounds.size()) + 1;
  // copies in: range r's part of every input (its blocks up to the first whose index key
  // reaches bound r, with 16 bytes beyond for the decoders' windows), the last range the
  // rest of the data region
  std::vector<uint64_t> done(N, 0);
  bool ok = cudaEventRecord(x->ev_run, st) == cudaSuccess && cudaStreamWaitEvent(x->in, x->ev_run, 0) == cudaSuccess &&
            cudaEventRecord(x->t[0], x->in) == cudaSuccess;
  for (uint32_t r = 0; ok && r < R; ++r) {
    for (uint32_t i = 0; ok && i < N; ++i) {
      const uint64_t e = r + 1 < R ? range_copy_end(plan, i, bounds[r]) : idx_off[i];
      if (e > done[i]) {
        ok = copy_pieces(dptr[i] + done[i], job.inputs[i].data + done[i], e - done[i], cudaMemcpyHostToDevice, x->in);
        done[i] = e;
      }
    }
    ok = ok && cudaEventRecord(x->ev_in[r], x->in) == cudaSuccess;
  }
  ok = ok && cudaEventRecord(x->t[1], x->in) == cudaSuccess;
  // the ranges: compact, emit the finished tables, copy them out on the second stream
  struct ByKernel {
    ByKernel() { t_stage_by_kernel = true; }
    ~ByKernel() { t_stage_by_kernel = false; }
  } by_kernel;
  std::vector<luda_outputs> routs(R);
  for (luda_outputs& o : routs) memset(&o, 0, sizeof o);
  std::vector<uint32_t> nrec, max_rec;
  std::vector<luda_table> emitted;  // the emitted tables, in key order (keys as offsets into ekeys)
  std::vector<uint8_t> ekeys;
  // range runs: no kept runs (their tables go to the host); each range's tables released
  // once their copy out is queued
  luda_options ro = *opts;
  ro.flags &= ~LUDA_F_KEEP_DECODED;
  if (!ro.dev_alloc) {
    ro.dev_alloc = range_alloc;
    ro.dev_free = range_free;
    ro.alloc_ctx = x->out;
  }
  std::vector<uint8_t> lo;
  bool has_lo = false;
  double ms_dev = 0;
  double sms[LUDA_N_STAGES] = {};
  uint64_t sbytes[LUDA_N_STAGES] = {};
  Holder* h = new Holder;
  const uint64_t cap0 = ((in_bytes + in_bytes / 2) | ((64ull << 20) - 1)) + 1;
  h->pinned = pinned_get(cap0, &h->pinned_cap);
  if (!h->pinned) h->pinned = pinned_get(256ull << 20, &h->pinned_cap);  // more buffers as tables come
  uint8_t* pin = h->pinned;
  uint64_t pin_left = h->pinned ? h->pinned_cap : 0, pos = 0;
  std::vector<uint8_t*> host_at;  // host address of every emitted table
  bool out_started = false;
  auto finish = [&](luda_status s) {
    cudaStreamSynchronize(x->in);
    cudaStreamSynchronize(x->out);
    for (luda_outputs& o : routs) luda_outputs_free(&o);
    mem.put(arena);
    cudaStreamSynchronize(st);
    return s;
  };
  // a failed call: no copy may still write the pinned buffers when they go back to the cache
  auto fail = [&](luda_status s) {
    cudaStreamSynchronize(x->in);
    cudaStreamSynchronize(x->out);
    holder_release(h);
    return finish(s);
  };
  if (!ok || !h->pinned) {
    const luda_status s = h->pinned ? cuda_fail(cudaGetLastError(), "copy of the inputs to the device")
                                    : cuda_fail(cudaErrorMemoryAllocation, "pinned host allocation");
    return fail(s);
  }
  for (uint32_t r = 0; r < R; ++r) {
    HostJob hj{nullptr, N, job.smallest_snapshot, job.bottommost};
    std::vector<luda_input> din(job.inputs, job.inputs + N);
    for (uint32_t i = 0; i < N; ++i) din[i].data = dptr[i];
    hj.inputs = din.data();
    static const uint8_t kEmpty = 0;
    if (has_lo) {
      hj.lo = lo.empty() ? &kEmpty : lo.data();
      hj.lo_len = uint32_t(lo.size());
    }
    if (r + 1 < R) {
      hj.hi = bounds[r].second ? bounds[r].first : &kEmpty;
      hj.hi_len = bounds[r].second;
    }
    double ms = 0;
    double rs[LUDA_N_STAGES] = {};
    uint64_t rb[LUDA_N_STAGES] = {};
    if (cudaStreamWaitEvent(st, x->ev_in[r], 0) != cudaSuccess) {
      return fail(cuda_fail(cudaGetLastError(), "stream wait"));
    }
    rc = run_compaction(&hj, 1, &ro, st, &routs[r], false, &ms, nullptr, rs, rb, nullptr, &nrec);
    if (!rc && routs[r].status) rc = luda_status(routs[r].status);
    if (rc) {
      return fail(rc);
    }
    ms_dev += ms;
    for (int k = 0; k < LUDA_N_STAGES; ++k) {
      sms[k] += rs[k];
      sbytes[k] += rb[k];
    }
    if (max_rec.size() < nrec.size()) max_rec.resize(nrec.size(), 0);
    for (size_t g = 0; g < nrec.size(); ++g) max_rec[g] = std::max(max_rec[g], nrec[g]);
    // the tables before the last one that starts a new user key are finished
    const luda_outputs& o = routs[r];
    uint32_t n_emit = o.n_tables;
    if (r + 1 < R) {
      n_emit = 0;
      for (uint32_t t = o.n_tables; t-- > 1;) {
        const luda_table& a = o.tables[t - 1];
        const luda_table& b = o.tables[t];
        if (a.largest_len >= 8 && b.smallest_len >= 8 &&
            cmp_user_host(a.largest, a.largest_len - 8, b.smallest, b.smallest_len - 8) != 0) {
          n_emit = t;
          lo.assign(b.smallest, b.smallest + b.smallest_len - 8);
          has_lo = true;
          break;
        }
      }
    }
    if (n_emit && !out_started) {
      out_started = true;
      ok = cudaEventRecord(x->t[2], x->out) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(x->ev_run, st) == cudaSuccess && cudaStreamWaitEvent(x->out, x->ev_run, 0) == cudaSuccess;
    for (uint32_t t = 0; ok && t < n_emit; ++t) {
      const luda_table& tb = o.tables[t];
      if (tb.size > pin_left) {  // another pinned buffer for the rest
        size_t c = 0;
        uint8_t* p = pinned_get(std::max<uint64_t>(2 * tb.size, 64ull << 20), &c);
        if (!p) {
          return fail(cuda_fail(cudaErrorMemoryAllocation, "pinned host allocation"));
        }
        h->more_pinned.emplace_back(p, c);
        pin = p;
        pin_left = c;
        pos = 0;
      }
      ok = copy_pieces(pin + pos, tb.data, tb.size, cudaMemcpyDeviceToHost, x->out);
      luda_table e = tb;
      e.smallest = reinterpret_cast<uint8_t*>(uintptr_t(ekeys.size()));
      ekeys.insert(ekeys.end(), tb.smallest, tb.smallest + tb.smallest_len);
      e.largest = reinterpret_cast<uint8_t*>(uintptr_t(ekeys.size()));
      ekeys.insert(ekeys.end(), tb.largest, tb.largest + tb.largest_len);
      emitted.push_back(e);
      host_at.push_back(pin + pos);
      const uint64_t adv = (tb.size + 15) & ~uint64_t(15);
      pos += adv;
      pin_left = adv < pin_left ? pin_left - adv : 0;
    }
    if (!ok) {
      return fail(cuda_fail(cudaGetLastError(), "copy of the new tables to the host"));
    }
    // with the library's allocator the tables' memory goes back on the copy-out stream, after
    // their copies; a caller's allocator gets it back at the end
    if (ro.dev_free == range_free) luda_outputs_free(&routs[r]);
  }
  // one result: the emitted tables in pinned host memory, their keys in one buffer
  if (out_started) cudaEventRecord(x->t[3], x->out);
  cudaStreamSynchronize(x->out);
  const uint32_t nt = uint32_t(emitted.size());
  uint64_t kb = 0, n_in = 0, n_out = 0;
  for (const luda_table& t : emitted) {
    kb += t.smallest_len + t.largest_len;
    n_out += t.n_entries;
  }
  for (uint32_t v : max_rec) n_in += v;
  out->tables = static_cast<luda_table*>(calloc(nt ? nt : 1, sizeof(luda_table)));
  uint8_t* keys = static_cast<uint8_t*>(malloc(kb ? kb : 1));
  uint64_t kp = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    luda_table tb = emitted[t];
    tb.data = host_at[t];
    memcpy(keys + kp, ekeys.data() + uintptr_t(emitted[t].smallest), tb.smallest_len);
    tb.smallest = keys + kp;
    kp += tb.smallest_len;
    memcpy(keys + kp, ekeys.data() + uintptr_t(emitted[t].largest), tb.largest_len);
    tb.largest = keys + kp;
    kp += tb.largest_len;
    out->tables[t] = tb;
  }
  out->n_tables = nt;
  out->n_in_entries = n_in;
  out->n_dropped = n_in - n_out;
  out->_priv = new OutPriv{h, keys};  // the result holds the holder's one reference
  float a = 0, b = 0;
  cudaStreamSynchronize(x->in);
  if (cudaEventElapsedTime(&a, x->t[0], x->t[1]) == cudaSuccess) out->ms_h2d = a;
  if (out_started && cudaEventElapsedTime(&b, x->t[2], x->t[3]) == cudaSuccess) out->ms_d2h = b;
  out->ms_device = ms_dev;
  memcpy(out->stage_ms, sms, sizeof sms);
  memcpy(out->stage_bytes, sbytes, sizeof sbytes);
  return finish(LUDA_OK);
}

}  // namespace

luda_status luda::compact_job_host(const luda_job& job, const luda_options* opts, luda_outputs* out,
                                   AdmitGate* gate) {
  t_detail[0] = 0;
  const luda_input* inputs = job.inputs;
  const uint32_t n_inputs = job.n_inputs;
  if (!out || (!inputs && n_inputs) || !opts) {
    set_detail("NULL argument");
    return LUDA_ERR_INVALID_ARG;
  }
  memset(out, 0, sizeof *out);
  if (!gate) {  // a call of its own: its copies in and out overlap by key ranges
    for (uint32_t i = 0; i < n_inputs; ++i)
      if (!inputs[i].data && inputs[i].size) {
        set_detail("input %u: data is NULL", i);
        return LUDA_ERR_INVALID_ARG;
      }
    Fmt fmt;
    luda_status rc = opts_check(opts, &fmt);
    if (rc) return rc;
    bool handled = false;
    const TuningScope tuned(opts->tuning);
    rc = compact_host_ranges(job, opts, out, &handled);
    if (handled || rc) {
      if (rc) {
        luda_outputs_free(out);
        out->status = rc;
      }
      return rc;
    }
  }
  const cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
  const DevMem mem{opts, st};
  // one device arena for all inputs, each at a 256-byte boundary
  std::vector<uint64_t> off(n_inputs + 1, 0);
  for (uint32_t i = 0; i < n_inputs; ++i) {
    if (!inputs[i].data && inputs[i].size) {
      set_detail("input %u: data is NULL", i);
      return LUDA_ERR_INVALID_ARG;
    }
    off[i + 1] = (off[i] + inputs[i].size + 255) & ~uint64_t(255);
  }
  CrcTabs tabs;
  luda_status rc = get_tabs(&tabs);
  if (rc) return rc;
  uint8_t* arena = static_cast<uint8_t*>(mem.get(off[n_inputs] + 256));
  if (!arena) return cuda_fail(cudaErrorMemoryAllocation, "device allocation");
  std::vector<luda_input> din(n_inputs);
  Timer th;
  if (gate) gate->copy_begin(0);
  th.start(st);
  for (uint32_t i = 0; i < n_inputs; ++i) {
    din[i] = inputs[i];
    din[i].data = arena + off[i];
    if (inputs[i].size &&
        cudaMemcpyAsync(arena + off[i], inputs[i].data, inputs[i].size, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      if (gate) gate->copy_end(0);
      mem.put(arena);
      return cuda_fail(cudaGetLastError(), "copy of the inputs to the device");
    }
  }
  th.stop(st);
  if (gate) {
    cudaStreamSynchronize(st);
    gate->copy_end(0);
  }
  HostJob hj = host_job(job);
  hj.inputs = din.data();
  double ms = 0, d2h = 0;
  double sms[LUDA_N_STAGES] = {};
  uint64_t sbytes[LUDA_N_STAGES] = {};
  if (gate) gate->extra = off[n_inputs] + 256;  // the device copy of the inputs counts too
  rc = run_compaction(&hj, 1, opts, st, out, true, &ms, &d2h, sms, sbytes, gate);
  const double h2d = th.ms();
  mem.put(arena);
  cudaStreamSynchronize(st);
  if (rc) {
    out->status = rc;
    return rc;
  }
  out->ms_h2d = h2d;
  out->ms_device = ms;
  out->ms_d2h = d2h;
  memcpy(out->stage_ms, sms, sizeof sms);
  memcpy(out->stage_bytes, sbytes, sizeof sbytes);
  if (out->status) {
    const luda_status s = luda_status(out->status);
    luda_outputs_free(out);
    out->status = s;
    return s;
  }
  return LUDA_OK;
}

luda_status luda::compact_job_device(const luda_job& job, const luda_options* opts, luda_outputs* out,
                                     AdmitGate* gate) {
  t_detail[0] = 0;
  if (!out || (!job.inputs && job.n_inputs) || !opts) {
    set_detail("NULL argument");
    return LUDA_ERR_INVALID_ARG;
  }
  HostJob hj = host_job(job);
  const cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
  double ms = 0;
  luda_status rc = run_compaction(&hj, 1, opts, st, out, false, &ms, nullptr, out->stage_ms, out->stage_bytes, gate);
  if (rc) {
    out->status = rc;
    return rc;
  }
  out->ms_device = ms;
  if (out->status) {
    const luda_status s = luda_status(out->status);
    luda_outputs_free(out);
    out->status = s;
    return s;
  }
  return LUDA_OK;
}

// =========================================================================================
extern "C" {

void luda_options_default(luda_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->block_size = 4096;
  o->restart_interval = 16;
  o->bloom_bits_per_key = 10;
  o->target_file_size = 2ull << 20;
}

const char* luda_strerror(luda_status s) {
  switch (s) {
    case LUDA_OK: return "ok";
    case LUDA_ERR_INVALID_ARG: return "invalid argument";
    case LUDA_ERR_CORRUPTION: return "corrupt input table";
    case LUDA_ERR_NOT_SUPPORTED: return "not supported (block type or compressed block on this path)";
    case LUDA_ERR_OOM: return "out of memory";
    case LUDA_ERR_CUDA: return "CUDA error";
    case LUDA_ERR_TIMEOUT: return "device wait timed out";
    case LUDA_ERR_DUPLICATE_KEY: return "duplicate internal key";
    case LUDA_ERR_PLAN_MISMATCH: return "plan no longer matches its inputs";
  }
  return "unknown status";
}

const char* luda_last_error_detail(void) { return t_detail; }

const char* luda_version(void) { return "luda-b300 0.1 (sm_103a)"; }

uint64_t luda_launch_count(void) { return g_launches.load(); }

uint64_t luda_kept_inputs_used(void) { return g_kept_used.load(); }

void luda_outputs_free(luda_outputs* out) {
  if (!out) return;
  OutPriv* p = static_cast<OutPriv*>(out->_priv);
  if (p) {
    free(p->keys);
    holder_release(p->holder);
    delete p;
  }
  free(out->tables);
  memset(out, 0, sizeof *out);
}

luda_status luda_batch_compact_device(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts,
                                      luda_outputs* outs) {
  t_detail[0] = 0;
  if ((!jobs && n_jobs) || !outs) {
    set_detail("jobs or outs is NULL");
    return LUDA_ERR_INVALID_ARG;
  }
  std::vector<HostJob> hj(n_jobs);
  for (uint32_t j = 0; j < n_jobs; ++j) hj[j] = host_job(jobs[j]);
  const cudaStream_t st = opts ? static_cast<cudaStream_t>(opts->stream) : nullptr;
  double ms = 0;
  double sms[LUDA_N_STAGES] = {};
  uint64_t sbytes[LUDA_N_STAGES] = {};
  luda_status rc = run_compaction(hj.data(), n_jobs, opts, st, outs, false, &ms, nullptr, sms, sbytes);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    if (rc) outs[j].status = rc;
    outs[j].ms_device = ms;
    memcpy(outs[j].stage_ms, sms, sizeof sms);  // the call's stages, shared by its jobs
    memcpy(outs[j].stage_bytes, sbytes, sizeof sbytes);
  }
  return rc;
}

luda_status luda_batch_compact(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts, luda_outputs* outs) {
  t_detail[0] = 0;
  if ((!jobs && n_jobs) || !outs || !opts) {
    set_detail("jobs, outs or opts is NULL");
    return LUDA_ERR_INVALID_ARG;
  }
  for (uint32_t j = 0; j < n_jobs; ++j) memset(&outs[j], 0, sizeof(luda_outputs));
  auto fail_all = [&](luda_status r) {  // an error that stops the batch, in every job's status
    for (uint32_t j = 0; j < n_jobs; ++j) outs[j].status = r;
    return r;
  };
  Fmt fmt;
  luda_status rc = opts_check(opts, &fmt);
  if (rc) return fail_all(rc);
  if (n_jobs == 0) return LUDA_OK;
  // one device arena for every job's inputs, each input at a 256-byte boundary
  std::vector<uint32_t> first(n_jobs + 1, 0);
  std::vector<uint64_t> off(1, 0);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    if (jobs[j].n_inputs && !jobs[j].inputs) {
      set_detail("job %u: inputs is NULL", j);
      return fail_all(LUDA_ERR_INVALID_ARG);
    }
    first[j] = uint32_t(off.size() - 1);
    for (uint32_t i = 0; i < jobs[j].n_inputs; ++i) {
      const luda_input& in = jobs[j].inputs[i];
      if (!in.data && in.size) {
        set_detail("job %u input %u: data is NULL", j, i);
        return fail_all(LUDA_ERR_INVALID_ARG);
      }
      off.push_back((off.back() + in.size + 255) & ~uint64_t(255));
    }
  }
  first[n_jobs] = uint32_t(off.size() - 1);
  const cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
  const DevMem mem{opts, st};
  CrcTabs tabs;
  if ((rc = get_tabs(&tabs))) return fail_all(rc);
  uint8_t* arena = static_cast<uint8_t*>(mem.get(off.back() + 256));
  if (!arena) return fail_all(cuda_fail(cudaErrorMemoryAllocation, "device allocation"));
  std::vector<luda_input> din(first[n_jobs] + 1);
  std::vector<HostJob> hj(n_jobs);
  Timer th;
  th.start(st);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    for (uint32_t i = 0; i < jobs[j].n_inputs; ++i) {
      const uint32_t g = first[j] + i;
      const luda_input& in = jobs[j].inputs[i];
      din[g] = in;
      din[g].data = arena + off[g];
      if (in.size && cudaMemcpyAsync(arena + off[g], in.data, in.size, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        mem.put(arena);
        return fail_all(cuda_fail(cudaGetLastError(), "copy of the inputs to the device"));
      }
    }
    hj[j] = host_job(jobs[j]);
    hj[j].inputs = din.data() + first[j];
  }
  th.stop(st);
  double ms = 0, d2h = 0;
  double sms[LUDA_N_STAGES] = {};
  uint64_t sbytes[LUDA_N_STAGES] = {};
  rc = run_compaction(hj.data(), n_jobs, opts, st, outs, true, &ms, &d2h, sms, sbytes);
  const double h2d = th.ms();
  mem.put(arena);
  cudaStreamSynchronize(st);
  for (uint32_t j = 0; j < n_jobs; ++j) {
    if (rc) outs[j].status = rc;
    outs[j].ms_h2d = h2d;
    outs[j].ms_device = ms;
    outs[j].ms_d2h = d2h;
    memcpy(outs[j].stage_ms, sms, sizeof sms);
    memcpy(outs[j].stage_bytes, sbytes, sizeof sbytes);
  }
  return rc;
}

luda_status luda_subcompact_device(const luda_input* inputs, uint32_t n_inputs, int32_t level,
                                   uint64_t smallest_snapshot, const luda_key* bounds, uint32_t n_bounds,
                                   const luda_options* opts, luda_outputs* out) {
  (void)level;
  t_detail[0] = 0;
  if (!out || (!inputs && n_inputs) || (!bounds && n_bounds) || !opts) {
    set_detail("NULL argument");
    return LUDA_ERR_INVALID_ARG;
  }
  memset(out, 0, sizeof *out);
  for (uint32_t b = 0; b < n_bounds; ++b) {
    if (!bounds[b].data && bounds[b].len) {
      set_detail("bound %u: data is NULL", b);
      return LUDA_ERR_INVALID_ARG;
    }
    if (b > 0) {
      const luda_key& x = bounds[b - 1];
      const luda_key& y = bounds[b];
      const uint32_t m = std::min(x.len, y.len);
      const int c = m ? memcmp(x.data, y.data, m) : 0;
      if (c > 0 || (c == 0 && x.len >= y.len)) {
        set_detail("bounds %u and %u are not strictly increasing", b - 1, b);
        return LUDA_ERR_INVALID_ARG;
      }
    }
  }
  static const uint8_t kEmpty = 0;
  const uint32_t K = n_bounds + 1;
  std::vector<HostJob> hj(K);
  for (uint32_t r = 0; r < K; ++r) {
    hj[r] = HostJob{inputs, n_inputs, smallest_snapshot, opts->bottommost};
    if (r > 0) {
      hj[r].lo = bounds[r - 1].len ? bounds[r - 1].data : &kEmpty;
      hj[r].lo_len = bounds[r - 1].len;
    }
    if (r + 1 < K) {
      hj[r].hi = bounds[r].len ? bounds[r].data : &kEmpty;
      hj[r].hi_len = bounds[r].len;
    }
  }
  std::vector<luda_outputs> outs(K);
  const cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
  double ms = 0;
  luda_status rc = run_compaction(hj.data(), K, opts, st, outs.data(), false, &ms, nullptr);
  if (rc) {
    out->status = rc;
    return rc;
  }
  // one result: the ranges' tables in key order; their keys are copied into one buffer and
  // the device tables stay owned by the ranges' shared holder
  luda_status first = LUDA_OK;
  uint32_t nt = 0;
  uint64_t kb = 0;
  for (const luda_outputs& o : outs) {
    if (o.status && !first) first = luda_status(o.status);
    out->n_in_entries += o.n_in_entries;
    out->n_dropped += o.n_dropped;
    nt += o.n_tables;
    for (uint32_t t = 0; t < o.n_tables; ++t) kb += o.tables[t].smallest_len + o.tables[t].largest_len;
  }
  if (first) {
    for (luda_outputs& o : outs) luda_outputs_free(&o);
    memset(out, 0, sizeof *out);
    out->status = first;
    return first;
  }
  out->tables = static_cast<luda_table*>(calloc(nt ? nt : 1, sizeof(luda_table)));
  uint8_t* keys = static_cast<uint8_t*>(malloc(kb ? kb : 1));
  Holder* holder = nullptr;
  uint64_t kp = 0;
  for (luda_outputs& o : outs) {
    OutPriv* p = static_cast<OutPriv*>(o._priv);
    if (p && !holder) {
      holder = p->holder;
      ++holder->refs;
    }
    for (uint32_t t = 0; t < o.n_tables; ++t) {
      luda_table tb = o.tables[t];
      memcpy(keys + kp, tb.smallest, tb.smallest_len);
      tb.smallest = keys + kp;
      kp += tb.smallest_len;
      memcpy(keys + kp, tb.largest, tb.largest_len);
      tb.largest = keys + kp;
      kp += tb.largest_len;
      out->tables[out->n_tables++] = tb;
    }
    luda_outputs_free(&o);
  }
  if (holder) {
    out->_priv = new OutPriv{holder, keys};
  } else {
    free(keys);
  }
  out->ms_device = ms;
  return LUDA_OK;
}

luda_status luda_compact_device(const luda_input* inputs, uint32_t n_inputs, int32_t level, uint64_t smallest_snapshot,
                                const luda_options* opts, luda_outputs* out) {
  (void)level;
  t_detail[0] = 0;
  if (!out || (!inputs && n_inputs) || !opts) {
    set_detail("NULL argument");
    return LUDA_ERR_INVALID_ARG;
  }
  HostJob hj{inputs, n_inputs, smallest_snapshot, opts->bottommost};
  const cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
  double ms = 0;
  luda_status rc = run_compaction(&hj, 1, opts, st, out, false, &ms, nullptr, out->stage_ms, out->stage_bytes);
  if (rc) {
    out->status = rc;
    return rc;
  }
  out->ms_device = ms;
  if (out->status) {
    const luda_status s = luda_status(out->status);
    luda_outputs_free(out);
    out->status = s;
    return s;
  }
  return LUDA_OK;
}

luda_status luda_compact(const luda_input* inputs, uint32_t n_inputs, int32_t level, uint64_t smallest_snapshot,
                         const luda_options* opts, luda_outputs* out) {
  if (!out || !opts) {
    t_detail[0] = 0;
    set_detail("NULL argument");
    return LUDA_ERR_INVALID_ARG;
  }
  const luda_job job{inputs, n_inputs, level, smallest_snapshot, opts->bottommost};
  return luda::compact_job_host(job, opts, out, nullptr);
}

luda_status luda_build(const luda_run* run, const luda_options* opts, luda_outputs* out) {
  t_detail[0] = 0;
  if (!out) return LUDA_ERR_INVALID_ARG;
  return run_build(run, true, opts, out, true);
}

luda_status luda_build_device(const luda_run* run, const luda_options* opts, luda_outputs* out) {
  t_detail[0] = 0;
  if (!out) return LUDA_ERR_INVALID_ARG;
  return run_build(run, false, opts, out, false);
}

luda_status luda_plan_create(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts, luda_plan** plan) {
  t_detail[0] = 0;
  if (!plan || (!jobs && n_jobs) || !opts) {
    set_detail("NULL argument");
    return LUDA_ERR_INVALID_ARG;
  }
  *plan = nullptr;
  PlanImpl* P = new PlanImpl();
  const luda_status rc = plan_build(jobs, n_jobs, opts, P);
  if (rc) {
    delete P;
    return rc;
  }
  *plan = reinterpret_cast<luda_plan*>(P);
  return LUDA_OK;
}

luda_status luda_plan_run(luda_plan* plan, void* stream) {
  t_detail[0] = 0;
  if (!plan) return LUDA_ERR_INVALID_ARG;
  PlanImpl* P = reinterpret_cast<PlanImpl*>(plan);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGraphLaunch(P->exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(P->done, st);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  g_launches.fetch_add(P->launches, std::memory_order_relaxed);
  P->ran = true;
  return LUDA_OK;
}

luda_status luda_plan_outputs(luda_plan* plan, luda_outputs* outs) {
  t_detail[0] = 0;
  if (!plan || !outs) return LUDA_ERR_INVALID_ARG;
  PlanImpl* P = reinterpret_cast<PlanImpl*>(plan);
  for (uint32_t j = 0; j < P->n_jobs; ++j) memset(&outs[j], 0, sizeof(luda_outputs));
  if (!P->ran) {
    set_detail("luda_plan_outputs before luda_plan_run");
    return LUDA_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaEventSynchronize(P->done);
  if (e != cudaSuccess) return cuda_fail(e, "waiting for the plan");
  Collected col;
  t_stage.reset();
  luda_status rc = collect(P->d_cnt, P->d_jobs, P->d_errs, P->pb, P->n_jobs, &col, P->st);
  if (rc) return rc;
  if ((e = cudaStreamSynchronize(P->st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
  Holder* h = new Holder();  // the plan owns the table memory; outputs only reference it
  luda_status first = LUDA_OK;
  for (uint32_t j = 0; j < P->n_jobs; ++j) {
    outs[j].status = err_status(col.errs[j], j, P->n_jobs);
    if (outs[j].status && !first) first = luda_status(outs[j].status);
  }
  fill_outputs(col, P->n_jobs, P->d_out, h, outs);
  holder_release(h);
  return LUDA_OK;
}

void luda_plan_destroy(luda_plan* plan) { delete reinterpret_cast<PlanImpl*>(plan); }

void luda_tuning_default(luda_tuning* t) {
  if (t) memset(t, 0, sizeof *t);
}

luda_status luda_tuning_check(const luda_tuning* t) {
  t_detail[0] = 0;
  if (!t) {
    set_detail("tuning pointer is NULL");
    return LUDA_ERR_INVALID_ARG;
  }
  return tuning_valid(t) ? LUDA_OK : LUDA_ERR_INVALID_ARG;
}

luda_status luda_autotune(const luda_job* jobs, uint32_t n_jobs, const luda_options* opts,
                          const luda_tuning* candidates, uint32_t n_candidates, uint32_t reps, double* ms,
                          uint32_t* best) {
  t_detail[0] = 0;
  if ((!jobs && n_jobs) || !opts || !candidates || !n_candidates || !reps || !ms || !best) {
    set_detail("NULL argument, no candidates or no repetitions");
    return LUDA_ERR_INVALID_ARG;
  }
  for (uint32_t c = 0; c < n_candidates; ++c)
    if (!tuning_valid(&candidates[c])) return LUDA_ERR_INVALID_ARG;
  luda_status first = LUDA_OK;
  double best_ms = -1;
  *best = 0;
  for (uint32_t c = 0; c < n_candidates; ++c) {
    ms[c] = -1;
    luda_options o = *opts;
    o.tuning = &candidates[c];
    luda_plan* plan = nullptr;
    luda_status rc = luda_plan_create(jobs, n_jobs, &o, &plan);
    std::vector<double> t;
    if (!rc) {
      PlanImpl* P = reinterpret_cast<PlanImpl*>(plan);
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaError_t e = cudaEventCreate(&e0);
      if (e == cudaSuccess) e = cudaEventCreate(&e1);
      if (e == cudaSuccess) rc = luda_plan_run(plan, P->st);  // untimed: first replay
      if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);
      for (uint32_t r = 0; r < reps && e == cudaSuccess && !rc; ++r) {
        e = cudaEventRecord(e0, P->st);
        if (e == cudaSuccess) rc = luda_plan_run(plan, P->st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, P->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float x = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
      }
      if (e != cudaSuccess && !rc) rc = cuda_fail(e, "autotune timing");
      if (!rc) {
        // a candidate whose jobs failed (a corrupt input) is not a valid measurement
        std::vector<luda_outputs> outs(n_jobs ? n_jobs : 1);
        rc = luda_plan_outputs(plan, outs.data());
        for (uint32_t j = 0; j < n_jobs && !rc; ++j)
          if (outs[j].status) rc = luda_status(outs[j].status);
        for (uint32_t j = 0; j < n_jobs; ++j) luda_outputs_free(&outs[j]);
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      luda_plan_destroy(plan);
    }
    if (rc) {
      if (!first) first = rc;
      continue;
    }
    std::sort(t.begin(), t.end());
    ms[c] = t[t.size() / 2];
    if (best_ms < 0 || ms[c] < best_ms) {
      best_ms = ms[c];
      *best = c;
    }
  }
  return best_ms < 0 ? first : LUDA_OK;
}

}  // extern "C"
