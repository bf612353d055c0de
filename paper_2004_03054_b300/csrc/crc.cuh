// crc.cuh -- warp-parallel CRC-32C (Castagnoli) for block trailers.
//
// Block checksums are verified per data block when unpacking and computed per block when
// packing (LUDA §II-A Phases 1 and 3; §III-C "unpack" and "encode" kernels). Reflected
// polynomial 0x82F63B78, init and final XOR 0xFFFFFFFF.
//
// Method (linear-algebra view of a CRC, e.g. as used for combining CRCs of
// concatenated messages):
//   * Let F(M) be the register after feeding M into a zero register. F is linear over
//     GF(2) and F(A || B) = Z_|B|(F(A)) xor F(B), where Z_L is the linear map "feed L zero
//     bytes" (multiplication by x^{8L} modulo the polynomial).
//   * Leading zero bytes do not change F, so the message is widened to whole aligned
//     16-byte words by zero bytes in front; the trailing pad of p zero bytes is removed
//     with the inverse map Z_{-p}.
//   * Starting the register at 0xFFFFFFFF equals XOR-ing 0xFF into the first four message
//     bytes with a zero register (valid for messages of at least 4 bytes).
//   * cta_crc32c: each thread folds an equal, contiguous run of aligned words
//     (slicing-by-4 tables in shared memory); butterflies join neighbouring runs with
//     Z_{run length}, applied with four 256-entry lookup tables per shift length.
//   * warp_crc32c_u32 (data blocks): lanes take interleaved 32-byte units so that every
//     round reads 1 KiB contiguously; lane registers skip the other lanes' units with
//     Z_992 and are joined by a butterfly at the end.
// The tables are generated on the host from the polynomial (crc_tables.cu).
#pragma once

#include <cstdint>

namespace luda {

// Shift tables: index j in [0, 32) shifts by 16 << j bytes; index 32 + (p - 1) for p in
// [1, 16) applies the inverse shift by p bytes; index kShift992 shifts by 992 bytes. Each
// table: 4 x 256 words.
constexpr int kShiftPow = 32;
constexpr int kShiftInv = 15;
constexpr int kShift992 = kShiftPow + kShiftInv;  // "feed 992 zero bytes" (32-byte lane spans)
constexpr int kShiftTables = kShift992 + 1;

// Shift matrices of the unpack's 144-byte chunks (each 4 x 256 words), Z_L for L = 16, 32,
// 64, 128 (the byte-table steps of a shift below 144), 80 (the second of a chunk's two
// chains), 144 * 2^k for k < 5 (one chunk, and the lane butterfly) and 144 * 32 (the
// other lanes' chunks of a round).
constexpr uint32_t kChunk = 144;
enum : int { kCZ16, kCZ32, kCZ64, kCZ128, kCZ80, kCZ144, kCZ288, kCZ576, kCZ1152, kCZ2304, kCZ4608, kChunkTables };

struct CrcTabs {
  const uint32_t* slice;  // 4 x 256: slice[k*256 + v] = register after k+1 byte steps of v
  const uint32_t* shift;  // kShiftTables x 4 x 256
  const uint32_t* chunk;  // kChunkTables x 4 x 256 (the unpack kernel's matrices)
};

// One 4-byte step with slicing-by-4 tables in shared memory.
__device__ __forceinline__ uint32_t crc_step4(uint32_t crc, uint32_t w, const uint32_t* sT) {
  crc ^= w;
  return sT[768 + (crc & 0xFFu)] ^ sT[512 + ((crc >> 8) & 0xFFu)] ^ sT[256 + ((crc >> 16) & 0xFFu)] ^
         sT[crc >> 24];
}

__device__ __forceinline__ uint32_t crc_shift(const uint32_t* tab, uint32_t v) {
  return __ldg(tab + (v & 0xFFu)) ^ __ldg(tab + 256 + ((v >> 8) & 0xFFu)) ^
         __ldg(tab + 512 + ((v >> 16) & 0xFFu)) ^ __ldg(tab + 768 + (v >> 24));
}

// Bytes of a little-endian word at byte address q that fall outside [ps, pe) become 0;
// bytes inside [ps, ps + 4) are complemented (the register init).
__device__ __forceinline__ uint32_t crc_fix_word(uint32_t w, uintptr_t q, uintptr_t ps, uintptr_t pe) {
  uint32_t keep = 0, flip = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uintptr_t x = q + b;
    if (x >= ps && x < pe) {
      keep |= 0xFFu << (8 * b);
      if (x < ps + 4) flip |= 0xFFu << (8 * b);
    }
  }
  return (w & keep) ^ flip;
}

// Standard CRC-32C of n bytes at p computed by all NT threads of the CTA (NT = blockDim.x,
// a multiple of 32, at most 1024); same method as warp_crc32c with an NT-leaf butterfly
// (shuffles inside warps, `scratch` (>= NT/32 words of shared memory) across warps).
// Every thread must call it; every thread gets the result.
static __device__ __noinline__ uint32_t cta_crc32c(const uint8_t* p, uint64_t n, const uint32_t* sT,
                                                   const CrcTabs tabs, uint32_t* scratch) {
  const uint32_t tid = threadIdx.x, NT = blockDim.x, lane = tid & 31u, warp = tid >> 5, nw = NT >> 5;
  if (n < 16) {
    if (tid == 0) {
      uint32_t c = 0xFFFFFFFFu;
      for (uint64_t i = 0; i < n; ++i) c = sT[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
      scratch[0] = c ^ 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t r = scratch[0];
    __syncthreads();
    return r;
  }
  const uintptr_t ps = reinterpret_cast<uintptr_t>(p);
  const uintptr_t pe = ps + n;
  const uintptr_t a0 = ps & ~uintptr_t(15);
  const uintptr_t a1 = (pe + 15) & ~uintptr_t(15);
  const uint32_t pad = uint32_t(a1 - pe);
  const int64_t W = int64_t((a1 - a0) >> 4);
  uint32_t j = 0;
  while ((int64_t(NT) << j) < W) ++j;
  const int64_t cw = int64_t(1) << j;
  int64_t w0 = W - cw * int64_t(NT - tid);
  const int64_t w1 = w0 + cw;
  if (w0 < 0) w0 = 0;
  uint32_t crc = 0;
#pragma unroll 1
  for (int64_t w = w0; w < w1; ++w) {
    const uintptr_t q = a0 + (uintptr_t(w) << 4);
    uint4 v = *reinterpret_cast<const uint4*>(q);
    if (q < ps + 4 || q + 16 > pe) {
      v.x = crc_fix_word(v.x, q, ps, pe);
      v.y = crc_fix_word(v.y, q + 4, ps, pe);
      v.z = crc_fix_word(v.z, q + 8, ps, pe);
      v.w = crc_fix_word(v.w, q + 12, ps, pe);
    }
    crc = crc_step4(crc, v.x, sT);
    crc = crc_step4(crc, v.y, sT);
    crc = crc_step4(crc, v.z, sT);
    crc = crc_step4(crc, v.w, sT);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, crc, 1u << k);
    const uint32_t* tab = tabs.shift + size_t(j + k) * 1024;
    crc = (lane & (1u << k)) ? (crc_shift(tab, other) ^ crc) : (crc_shift(tab, crc) ^ other);
  }
  if (lane == 0) scratch[warp] = crc;
  __syncthreads();
  if (warp == 0) {
    crc = lane < nw ? scratch[lane] : 0u;
    for (uint32_t k = 0; (1u << k) < nw; ++k) {
      const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, crc, 1u << k);
      const uint32_t* tab = tabs.shift + size_t(j + 5 + k) * 1024;
      crc = (lane & (1u << k)) ? (crc_shift(tab, other) ^ crc) : (crc_shift(tab, crc) ^ other);
    }
    if (pad) crc = crc_shift(tabs.shift + size_t(kShiftPow + pad - 1) * 1024, crc);
    if (lane == 0) scratch[0] = crc ^ 0xFFFFFFFFu;
  }
  __syncthreads();
  const uint32_t r = scratch[0];
  __syncthreads();
  return r;
}

// ---- lane-replicated tables: conflict-free lookups ------------------------------------------
// Word (t * 256 + v) * 32 + lane holds slice[t][v], so lane l always reads bank l.
// Word (t * 256 + v) * 32 + lane holds slice[t][v]: lane l always reads bank l.
constexpr uint32_t kRepWords = 4 * 256 * 32;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- 32-byte lane spans --------------------------------------------------------------------
// Tables in shared memory, addressed with 32-bit shared-window addresses so that every
// lookup is one byte extract, one address multiply-add and one ld.shared with the table's
// offset as an immediate. tl = address of this lane's column of the lane-replicated slicing
// tables (word (t * 256 + v) * 32 + lane holds slice[t][v]); tz = address of this lane's
// copy of Z_992's four byte tables: kZCopies interleaved copies (word (t * 256 + v) *
// kZCopies + c holds copy c), lane l reading copy l mod kZCopies, so that lanes sharing a
// bank are the 32 / kZCopies lanes of one copy and conflicts stay few.
constexpr uint32_t kZCopies = 16;
constexpr uint32_t kZWords = 1024 * kZCopies;
constexpr uint32_t kRepSmem = (kRepWords + kZWords) * 4;  // bytes of shared memory for both

// One global load per table word, then its lane copies stored in rotated order, so that
// the 32 threads of a warp (consecutive words) hit 32 different banks. blockDim must be a
// multiple of 32.
__device__ __forceinline__ void load_rep_tables992(uint32_t* sTr, uint32_t* sZ, const CrcTabs tabs) {
  const uint32_t rot = threadIdx.x & 31u;
  for (uint32_t w = threadIdx.x; w < 1024; w += blockDim.x) {
    const uint32_t val = __ldg(tabs.slice + w);
    const uint32_t zv = __ldg(tabs.shift + size_t(kShift992) * 1024 + w);
    uint32_t* row = sTr + w * 32u;
#pragma unroll 8
    for (uint32_t l = 0; l < 32; ++l) row[(l + rot) & 31u] = val;
    uint32_t* zrow = sZ + w * kZCopies;
    const uint32_t zrot = (w >> 1) & (kZCopies - 1);
#pragma unroll
    for (uint32_t c = 0; c < kZCopies; ++c) zrow[(c + zrot) & (kZCopies - 1)] = zv;
  }
}

// Address of lane `lane`'s copy of the skip tables that start at sZ.
__device__ __forceinline__ uint32_t zcopy_addr(const uint32_t* sZ, uint32_t lane) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(sZ)) + (lane & (kZCopies - 1)) * 4u;
}

template <uint32_t kOff>
__device__ __forceinline__ uint32_t lds_off(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(kOff));
  return v;
}

__device__ __forceinline__ uint32_t crc_word_rep(uint32_t c, uint32_t w, uint32_t tl) {
  c ^= w;
  const uint32_t t3 = lds_off<3u * 32768u>(tl + __byte_perm(c, 0, 0x4440) * 128u);
  const uint32_t t2 = lds_off<2u * 32768u>(tl + __byte_perm(c, 0, 0x4441) * 128u);
  const uint32_t t1 = lds_off<1u * 32768u>(tl + __byte_perm(c, 0, 0x4442) * 128u);
  const uint32_t t0 = lds_off<0u>(tl + __byte_perm(c, 0, 0x4443) * 128u);
  return t3 ^ t2 ^ t1 ^ t0;
}

__device__ __forceinline__ uint32_t crc_z992(uint32_t v, uint32_t tz) {
  constexpr uint32_t kRow = kZCopies * 4u, kTab = 256u * kRow;
  return lds_off<0u>(tz + __byte_perm(v, 0, 0x4440) * kRow) ^ lds_off<kTab>(tz + __byte_perm(v, 0, 0x4441) * kRow) ^
         lds_off<2u * kTab>(tz + __byte_perm(v, 0, 0x4442) * kRow) ^
         lds_off<3u * kTab>(tz + __byte_perm(v, 0, 0x4443) * kRow);
}

__device__ __forceinline__ uint32_t crc_unit32(uint32_t acc, const uint4& x, const uint4& y, uint32_t tl) {
  acc = crc_word_rep(acc, x.x, tl);
  acc = crc_word_rep(acc, x.y, tl);
  acc = crc_word_rep(acc, x.z, tl);
  acc = crc_word_rep(acc, x.w, tl);
  acc = crc_word_rep(acc, y.x, tl);
  acc = crc_word_rep(acc, y.y, tl);
  acc = crc_word_rep(acc, y.z, tl);
  return crc_word_rep(acc, y.w, tl);
}

// Bytes of the little-endian word at offset q (from the unit base) outside [lo, hi) become
// 0; with kInit, bytes inside [lo, lo + 4) are complemented (the register init). 32-bit
// offsets.
template <bool kInit>
__device__ __forceinline__ uint32_t crc_fix_word32(uint32_t w, uint32_t q, uint32_t lo, uint32_t hi) {
  uint32_t keep = 0, flip = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t x = q + b;
    if (x >= lo && x < hi) {
      keep |= 0xFFu << (8 * b);
      if (kInit && x < lo + 4) flip |= 0xFFu << (8 * b);
    }
  }
  return (w & keep) ^ flip;
}

// Standard CRC-32C of n (< 2^32) bytes at p by one warp, 32-byte lane spans: the message is
// widened by leading zeros to U aligned 32-byte units ending at the 16-byte boundary after
// its end; in round r lane l folds unit U - 32 * (rounds - r) + l, so each round reads 1 KiB
// contiguously, and the next round's two 16-byte loads are issued before this round's
// arithmetic. Between rounds a lane register moves past the other lanes' 992 bytes with
// Z_992; the lanes are joined with Z_{32 * 2^k} (k < 5), the trailing pad is removed with
// the inverse shift. Only 16-byte words inside [p & ~15, end rounded up] are loaded.
// kInit = false starts from a zero register instead of 0xFFFFFFFF and kFinal = false skips
// the final complement (for chunks of one message: the first chunk carries the init, the
// register of the whole message is complemented once after joining).
template <bool kInit = true, bool kFinal = true>
static __device__ __noinline__ uint32_t warp_crc32c_u32(const uint8_t* p, uint64_t n, uint32_t tl, uint32_t tz,
                                                        const CrcTabs tabs) {
  const uint32_t lane = threadIdx.x & 31u;
  if (n < 16) {
    uint32_t c = kInit ? 0xFFFFFFFFu : 0u;
    if (lane == 0)
      for (uint64_t i = 0; i < n; ++i) c = lds_off<0u>(tl + ((c ^ p[i]) & 0xFFu) * 128u) ^ (c >> 8);
    c = __shfl_sync(0xFFFFFFFFu, c, 0);
    return kFinal ? c ^ 0xFFFFFFFFu : c;
  }
  const uintptr_t ps = reinterpret_cast<uintptr_t>(p);
  const uintptr_t pe = ps + n;
  const uintptr_t a1 = (pe + 15) & ~uintptr_t(15);
  const uint32_t pad = uint32_t(a1 - pe);
  const uint32_t U = uint32_t((((a1 - (ps & ~uintptr_t(15))) >> 4) + 1) >> 1);
  const uintptr_t base = a1 - uintptr_t(U) * 32u;  // p & ~15, or 16 bytes before it
  const uint32_t lo = uint32_t(ps - base), hi = uint32_t(pe - base), lo16 = lo & ~15u;
  const uint32_t rounds = (U + 31) >> 5;
  // unit of this lane in round 0 (negative: leading zero unit, skipped)
  int32_t u = int32_t(U) - int32_t(32 * rounds) + int32_t(lane);
  auto load = [&](int32_t uu, uint4& x, uint4& y) {
    x = make_uint4(0, 0, 0, 0);
    y = x;
    if (uu < 0) return;
    const uint32_t q = uint32_t(uu) * 32u;
    const uint4* a = reinterpret_cast<const uint4*>(base + q);
    if (q >= lo16) x = a[0];
    y = a[1];
  };
  uint4 x0, y0, x1, y1;
  load(u, x0, y0);
  uint32_t acc = 0;
  for (uint32_t r = 0; r < rounds; ++r, u += 32) {
    if (r + 1 < rounds) load(u + 32, x1, y1);
    if (u >= 0) {
      const uint32_t q = uint32_t(u) * 32u;
      if (q < lo + 4 || q + 32 > hi) {
        x0.x = crc_fix_word32<kInit>(x0.x, q, lo, hi);
        x0.y = crc_fix_word32<kInit>(x0.y, q + 4, lo, hi);
        x0.z = crc_fix_word32<kInit>(x0.z, q + 8, lo, hi);
        x0.w = crc_fix_word32<kInit>(x0.w, q + 12, lo, hi);
        y0.x = crc_fix_word32<kInit>(y0.x, q + 16, lo, hi);
        y0.y = crc_fix_word32<kInit>(y0.y, q + 20, lo, hi);
        y0.z = crc_fix_word32<kInit>(y0.z, q + 24, lo, hi);
        y0.w = crc_fix_word32<kInit>(y0.w, q + 28, lo, hi);
      }
      acc = crc_unit32(crc_z992(acc, tz), x0, y0, tl);
    }
    x0 = x1;
    y0 = y1;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, acc, 1u << k);
    const uint32_t* tab = tabs.shift + size_t(k + 1) * 1024;
    acc = (lane & (1u << k)) ? (crc_shift(tab, other) ^ acc) : (crc_shift(tab, acc) ^ other);
  }
  if (pad) acc = crc_shift(tabs.shift + size_t(kShiftPow + pad - 1) * 1024, acc);
  return kFinal ? acc ^ 0xFFFFFFFFu : acc;
}

// Z_L(v): the register v moved past L zero bytes (L mod 16 single-byte steps, then the
// power-of-two shift tables for L / 16).
__device__ __forceinline__ uint32_t crc_zeros(uint32_t v, uint64_t L, const CrcTabs& tabs) {
  for (uint32_t r = uint32_t(L & 15u); r; --r) v = __ldg(tabs.slice + (v & 0xFFu)) ^ (v >> 8);
  uint64_t q = L >> 4;
  for (uint32_t j = 0; q; ++j, q >>= 1)
    if (q & 1u) v = crc_shift(tabs.shift + size_t(j) * 1024, v);
  return v;
}

// ---- CRCs assembled from pieces --------------------------------------------------------------
// A data block's checksum is assembled from the registers of its pieces: with F(M) the
// register after feeding M into a zero register, F(A || B) = Z_|B|(F(A)) xor F(B), and the
// standard CRC of a message M of n bytes is ~(Z_n(0xFFFFFFFF) xor F(M)). The value of every
// record carries F(value) from the pass that read it, so the encoder's blocks need only
// the few header and key bytes fed directly plus one shift per piece.

// One byte step of the register (T0: the first 256 words of the slicing table).
__device__ __forceinline__ uint32_t crc_byte(uint32_t c, uint32_t b, const uint32_t* T0) {
  return T0[(c ^ b) & 0xFFu] ^ (c >> 8);
}

// One matrix of four byte tables (1024 words) applied to v.
__device__ __forceinline__ uint32_t crc_mat(const uint32_t* t, uint32_t v) {
  return t[v & 0xFFu] ^ t[256 + ((v >> 8) & 0xFFu)] ^ t[512 + ((v >> 16) & 0xFFu)] ^ t[768 + (v >> 24)];
}

// Z_L(v) from tables in shared memory: L mod 16 zero-byte steps with T0, then for every
// set bit j of L / 16 the matrix Z_{16 * 2^j} stored at sZ + j * 1024 (2^nz > L / 16).
__device__ __forceinline__ uint32_t crc_zeros_s(uint32_t v, uint32_t L, const uint32_t* T0, const uint32_t* sZ) {
  for (uint32_t r = L & 15u; r; --r) v = T0[v & 0xFFu] ^ (v >> 8);
  uint32_t q = L >> 4;
  for (uint32_t j = 0; q; ++j, q >>= 1)
    if (q & 1u) v = crc_mat(sZ + j * 1024u, v);
  return v;
}

// Stage the slicing table into shared memory (1024 words), whole CTA.
__device__ __forceinline__ void load_slice_table(uint32_t* sT, const CrcTabs tabs) {
  for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) sT[i] = __ldg(tabs.slice + i);
}

}  // namespace luda
