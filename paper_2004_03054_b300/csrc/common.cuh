// common.cuh -- device-side building blocks shared by the CUDA kernels of libluda.
//
// Everything here is this library's own: LEB128 varints, the internal-key order, the
// masked CRC-32C helpers and the error word the kernels report into. None of it is
// shared with the CPU oracle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace luda {

constexpr uint64_t kMagic = 0x4C55444153535431ull;  // table footer magic
constexpr uint32_t kFooter = 48;                     // footer bytes
constexpr uint32_t kTrailer = 5;                     // block trailer: type + masked crc
constexpr uint32_t kSms = 148;                       // B300 SM count (two dies x 74)

enum : int32_t {
  E_OK = 0,
  E_INVALID = -1,
  E_CORRUPT = -2,
  E_NOTSUP = -3,
  E_OOM = -4,
  E_CUDA = -5,
  E_TIMEOUT = -6,
  E_DUP = -7,
  E_PLAN = -8,
};

// Per-job error word. The first reporter wins; `input` is the job-local input index (or
// ~0u when the error is not tied to an input) and `where` a byte offset in that input.
struct DErr {
  int32_t code;
  uint32_t input;
  uint64_t where;
};

__device__ __forceinline__ void report(DErr* e, int32_t code, uint32_t input, uint64_t where) {
  if (atomicCAS(&e->code, 0, code) == 0) {
    e->input = input;
    e->where = where;
  }
}

__host__ __device__ __forceinline__ uint32_t varint_size(uint64_t v) {
  uint32_t n = 1;
  while (v >= 0x80) {
    v >>= 7;
    ++n;
  }
  return n;
}

// LEB128 decode from [p, end): at most 5 bytes for 32-bit values, 10 for 64-bit; the
// value must fit. Returns the bytes consumed, 0 when malformed.
template <int BITS>
__device__ __forceinline__ uint32_t get_varint(const uint8_t* p, const uint8_t* end, uint64_t* out) {
  constexpr int kMax = BITS == 32 ? 5 : 10;
  uint64_t v = 0;
#pragma unroll 1
  for (int i = 0; i < kMax; ++i) {
    if (p + i >= end) return 0;
    uint32_t b = p[i];
    if (BITS == 64 && i == 9 && (b & 0x7F) > 1) return 0;
    v |= uint64_t(b & 0x7F) << (7 * i);
    if (!(b & 0x80)) {
      if (BITS == 32 && v > 0xFFFFFFFFull) return 0;
      *out = v;
      return uint32_t(i + 1);
    }
  }
  return 0;
}

__device__ __forceinline__ uint32_t put_varint(uint8_t* dst, uint64_t v) {
  uint32_t i = 0;
  while (v >= 0x80) {
    dst[i++] = uint8_t(v | 0x80);
    v >>= 7;
  }
  dst[i++] = uint8_t(v);
  return i;
}

__device__ __forceinline__ uint32_t ld_u32(const uint8_t* p) {
  return uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16) | (uint32_t(p[3]) << 24);
}

__device__ __forceinline__ uint64_t ld_u64(const uint8_t* p) {
  uint64_t v = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) v |= uint64_t(p[i]) << (8 * i);
  return v;
}

__device__ __forceinline__ void st_u32(uint8_t* p, uint32_t v) {
  p[0] = uint8_t(v);
  p[1] = uint8_t(v >> 8);
  p[2] = uint8_t(v >> 16);
  p[3] = uint8_t(v >> 24);
}

// Big-endian value of the first 8 bytes of a user key, zero padded: the leading part of
// the merge key. Equal prefixes fall back to a full compare.
__device__ __forceinline__ uint64_t key_prefix(const uint8_t* k, uint32_t ulen) {
  uint64_t v = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) v = (v << 8) | (uint64_t(i) < ulen ? k[i] : 0u);
  return v;
}

// Masked CRC stored in block trailers: rotate right by 15, add a constant.
__host__ __device__ __forceinline__ uint32_t crc_mask(uint32_t c) {
  return ((c >> 15) | (c << 17)) + 0xA282EAD8u;
}
__host__ __device__ __forceinline__ uint32_t crc_unmask(uint32_t m) {
  uint32_t r = m - 0xA282EAD8u;
  return (r >> 17) | (r << 15);
}

// Records of decoded entries, structure of arrays. Index = record id. Records of a job
// are contiguous, in input order then position, so the record id is the final tie-break
// of the total order.
struct Recs {
  uint64_t* pfx;    // key_prefix of the user key
  uint64_t* koff;   // offset of the full internal key in the key arena
  uint32_t* klen;   // internal key length (user key + 8)
  uint64_t* tr;     // trailer: seq << 8 | type
  uint64_t* vptr;   // device address of the value bytes (inside an input table)
  uint32_t* vlen;
  uint32_t* src;    // batch-global input index (order check)
  uint32_t* vcrc;   // F(value): CRC-32C register after the value bytes from a zero register
};

// 8 key bytes at p as a big-endian word; bytes at index >= avail read as 0. p may have any
// alignment: two aligned 8-byte loads (the key arena is padded past its end).
__device__ __forceinline__ uint64_t key_word(const uint8_t* p, uint32_t avail) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint64_t* q = reinterpret_cast<const uint64_t*>(a & ~uintptr_t(7));
  const uint32_t sh = uint32_t(a & 7u) * 8u;
  uint64_t w = q[0];
  if (sh) w = (w >> sh) | (q[1] << (64 - sh));
  if (avail < 8) w &= avail ? (~0ull >> (64 - 8 * avail)) : 0ull;
  const uint32_t lo = uint32_t(w), hi = uint32_t(w >> 32);
  return (uint64_t(__byte_perm(lo, 0, 0x0123)) << 32) | __byte_perm(hi, 0, 0x0123);
}

// 8 bytes at p (any alignment) as a little-endian word: two aligned 8-byte loads.
__device__ __forceinline__ uint64_t le_word(const uint8_t* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint64_t* q = reinterpret_cast<const uint64_t*>(a & ~uintptr_t(7));
  const uint32_t sh = uint32_t(a & 7u) * 8u;
  const uint64_t w = q[0];
  return sh ? (w >> sh) | (q[1] << (64 - sh)) : w;
}

// Order of two user keys (memcmp over the common length, a proper prefix first); reads
// whole aligned 8-byte words around the keys (both buffers readable to 16 bytes past).
__device__ __forceinline__ int cmp_user_keys(const uint8_t* a, uint32_t la, const uint8_t* b, uint32_t lb) {
  const uint32_t m = la < lb ? la : lb;
  for (uint32_t i = 0; i < m; i += 8) {
    const uint32_t avail = m - i < 8 ? m - i : 8u;
    const uint64_t wa = key_word(a + i, avail), wb = key_word(b + i, avail);
    if (wa != wb) return wa < wb ? -1 : 1;
  }
  return la == lb ? 0 : (la < lb ? -1 : 1);
}

// Internal key order from byte `from` of the user keys on, given that the bytes before it
// are equal (zero-padded): user key bytes (8 at a time), proper prefix first, then trailer
// descending, then record id ascending (input index, then position; 0 for a == b).
__device__ __forceinline__ int cmp_tail(const Recs& r, const uint8_t* arena, uint32_t a, uint32_t b, uint32_t from,
                                        bool by_id = true) {
  const uint32_t la = r.klen[a] - 8, lb = r.klen[b] - 8;
  const uint8_t* ka = arena + r.koff[a];
  const uint8_t* kb = arena + r.koff[b];
  const uint32_t m = la < lb ? la : lb;
  for (uint32_t i = from; i < m; i += 8) {
    const uint64_t wa = key_word(ka + i, m - i), wb = key_word(kb + i, m - i);
    if (wa != wb) return wa < wb ? -1 : 1;
  }
  if (la != lb) return la < lb ? -1 : 1;
  const uint64_t ta = r.tr[a], tb = r.tr[b];
  if (ta != tb) return ta > tb ? -1 : 1;
  if (!by_id || a == b) return 0;
  return a < b ? -1 : 1;
}

// Internal key order on records: user key ascending (memcmp, proper prefix first), then
// trailer descending, then record id ascending (input index, then position).
__device__ __forceinline__ int cmp_rec(const Recs& r, const uint8_t* arena, uint32_t a, uint64_t pa, uint32_t b,
                                       uint64_t pb) {
  if (pa != pb) return pa < pb ? -1 : 1;
  if (a == b) return 0;
  return cmp_tail(r, arena, a, b, 8);
}

// User keys equal?
__device__ __forceinline__ bool same_user_key(const Recs& r, const uint8_t* arena, uint32_t a, uint32_t b) {
  if (r.pfx[a] != r.pfx[b] || r.klen[a] != r.klen[b]) return false;
  const uint32_t l = r.klen[a] - 8;
  const uint8_t* ka = arena + r.koff[a];
  const uint8_t* kb = arena + r.koff[b];
  for (uint32_t i = 8; i < l; i += 8)
    if (key_word(ka + i, l - i) != key_word(kb + i, l - i)) return false;
  return true;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Grid-stride helpers.
__device__ __forceinline__ uint64_t gtid() { return uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint64_t gstride() { return uint64_t(gridDim.x) * blockDim.x; }

}  // namespace luda
