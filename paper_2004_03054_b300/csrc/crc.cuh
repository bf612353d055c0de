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
//   * Each lane folds an equal, contiguous run of aligned words (slicing-by-4 tables in
//     shared memory); a 5-level butterfly joins neighbouring runs with Z_{run length},
//     applied with four 256-entry lookup tables per shift length.
// The tables are generated on the host from the polynomial (crc_tables.cu).
#pragma once

#include <cstdint>

namespace luda {

// Shift tables: index j in [0, 32) shifts by 16 << j bytes; index 32 + (p - 1) for p in
// [1, 16) applies the inverse shift by p bytes. Each table: 4 x 256 words.
constexpr int kShiftPow = 32;
constexpr int kShiftInv = 15;
constexpr int kShift496 = kShiftPow + kShiftInv;  // "feed 496 zero bytes" (interleaved rounds)
constexpr int kShiftTables = kShift496 + 1;

struct CrcTabs {
  const uint32_t* slice;  // 4 x 256: slice[k*256 + v] = register after k+1 byte steps of v
  const uint32_t* shift;  // kShiftTables x 4 x 256
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

// Standard CRC-32C of the n bytes at p (generic address: global or shared memory).
// All 32 lanes of the warp must call it with the same arguments; every lane gets the
// result. The 16-byte words that contain p[0..n) are read whole (bytes outside are
// ignored), so the memory around the range must be readable to the next 16-byte bounds.
// `sT` is the slicing table (1024 words) staged in shared memory by the caller.
static __device__ __noinline__ uint32_t warp_crc32c(const uint8_t* p, uint64_t n, const uint32_t* sT, const CrcTabs tabs) {
  const uint32_t lane = threadIdx.x & 31u;
  if (n < 16) {  // short message: lane 0 alone, byte at a time
    uint32_t c = 0xFFFFFFFFu;
    if (lane == 0)
      for (uint64_t i = 0; i < n; ++i) c = sT[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    c = __shfl_sync(0xFFFFFFFFu, c, 0);
    return c ^ 0xFFFFFFFFu;
  }
  const uintptr_t ps = reinterpret_cast<uintptr_t>(p);
  const uintptr_t pe = ps + n;
  const uintptr_t a0 = ps & ~uintptr_t(15);
  const uintptr_t a1 = (pe + 15) & ~uintptr_t(15);
  const uint32_t pad = uint32_t(a1 - pe);
  const int64_t W = int64_t((a1 - a0) >> 4);
  uint32_t j = 0;
  while ((int64_t(32) << j) < W) ++j;
  const int64_t cw = int64_t(1) << j;
  int64_t w0 = W - cw * int64_t(32 - lane);
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
  if (pad) crc = crc_shift(tabs.shift + size_t(kShiftPow + pad - 1) * 1024, crc);
  return crc ^ 0xFFFFFFFFu;
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
// Word (t * 256 + v) * 32 + lane holds slice[t][v]: lane l always reads bank l.
constexpr uint32_t kRepWords = 4 * 256 * 32;

__device__ __forceinline__ void load_rep_tables(uint32_t* sTr, uint32_t* sZ, const CrcTabs tabs) {
  for (uint32_t i = threadIdx.x; i < kRepWords; i += blockDim.x) sTr[i] = __ldg(tabs.slice + (i >> 5));
  for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) sZ[i] = __ldg(tabs.shift + size_t(kShift496) * 1024 + i);
}

// Shared-memory word at a 32-bit shared-window byte address.
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One 4-byte step; tb = shared address of this lane's column (sTr + lane). Byte b of the
// register indexes row b of table 3 - b: word (t * 256 + v) * 32 + lane.
__device__ __forceinline__ uint32_t crc_step4r(uint32_t crc, uint32_t w, uint32_t tb) {
  crc ^= w;
  const uint32_t b0 = __byte_perm(crc, 0, 0x4440), b1 = __byte_perm(crc, 0, 0x4441);
  const uint32_t b2 = __byte_perm(crc, 0, 0x4442), b3 = __byte_perm(crc, 0, 0x4443);
  return lds32(tb + 98304u + b0 * 128u) ^ lds32(tb + 65536u + b1 * 128u) ^ lds32(tb + 32768u + b2 * 128u) ^
         lds32(tb + b3 * 128u);
}

// Z_496 applied through its four byte tables at shared address zb.
__device__ __forceinline__ uint32_t crc_shift_s(uint32_t zb, uint32_t v) {
  return lds32(zb + (v & 0xFFu) * 4u) ^ lds32(zb + 1024u + ((v >> 8) & 0xFFu) * 4u) ^
         lds32(zb + 2048u + ((v >> 16) & 0xFFu) * 4u) ^ lds32(zb + 3072u + (v >> 24) * 4u);
}

// Fold one 16-byte chunk into a lane register.
__device__ __forceinline__ uint32_t crc_chunk(uint32_t acc, uint4 v, uint32_t tb) {
  acc = crc_step4r(acc, v.x, tb);
  acc = crc_step4r(acc, v.y, tb);
  acc = crc_step4r(acc, v.z, tb);
  return crc_step4r(acc, v.w, tb);
}

// Join the 32 lane registers of an interleaved CRC (lane l holds chunks ending 31 - l chunks
// before the message end) and finish: remove the trailing pad, final XOR.
__device__ __forceinline__ uint32_t crc_il_finish(uint32_t acc, uint32_t pad, const CrcTabs tabs, uint32_t lane,
                                                  uint32_t extra = 0) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, acc, 1u << k);
    const uint32_t* tab = tabs.shift + size_t(k) * 1024;
    acc = (lane & (1u << k)) ? (crc_shift(tab, other) ^ acc) : (crc_shift(tab, acc) ^ other);
  }
  acc ^= extra;  // contributions folded in separately, already aligned to the message end
  if (pad) acc = crc_shift(tabs.shift + size_t(kShiftPow + pad - 1) * 1024, acc);
  return acc ^ 0xFFFFFFFFu;
}

// Z_{16 d}(v): move a register past 16 d zero bytes (binary decomposition of d).
__device__ __forceinline__ uint32_t crc_shift16(uint32_t v, uint64_t d, const CrcTabs tabs) {
  for (uint32_t j = 0; d; ++j, d >>= 1)
    if (d & 1) v = crc_shift(tabs.shift + size_t(j) * 1024, v);
  return v;
}

// Standard CRC-32C of n bytes at p by one warp, interleaved: in round r lane l folds the
// 16-byte aligned chunk W - 32 * (rounds - r) + l, so each round reads 512 contiguous bytes
// (coalesced). Between rounds a lane register moves past the other lanes' 496 bytes with
// Z_496 (register after 496 zero bytes). Tables: sTr lane-replicated slicing-by-4, sZ = Z_496.
static __device__ __noinline__ uint32_t warp_crc32c_il(const uint8_t* p, uint64_t n, uint32_t tb0, uint32_t zb,
                                                       const CrcTabs tabs) {
  // tb0: shared address of the replicated slicing tables, zb: of the Z_496 table
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t tb = tb0 + lane * 4u;
  if (n < 16) {
    uint32_t c = 0xFFFFFFFFu;
    if (lane == 0)
      for (uint64_t i = 0; i < n; ++i) c = lds32(tb0 + ((c ^ p[i]) & 0xFFu) * 128u) ^ (c >> 8);
    c = __shfl_sync(0xFFFFFFFFu, c, 0);
    return c ^ 0xFFFFFFFFu;
  }
  const uintptr_t ps = reinterpret_cast<uintptr_t>(p);
  const uintptr_t pe = ps + n;
  const uintptr_t a0 = ps & ~uintptr_t(15);
  const uintptr_t a1 = (pe + 15) & ~uintptr_t(15);
  const uint32_t pad = uint32_t(a1 - pe);
  const int64_t W = int64_t((a1 - a0) >> 4);
  const int64_t rounds = (W + 31) >> 5;
  uint32_t acc = 0;
  int64_t c = W - 32 * rounds + lane;
  for (int64_t r = 0; r < rounds; r += 2, c += 64) {
    const int64_t c2 = c + 32;
    uint4 v1 = make_uint4(0, 0, 0, 0), v2 = make_uint4(0, 0, 0, 0);
    const uintptr_t q1 = a0 + (uintptr_t(c) << 4), q2 = a0 + (uintptr_t(c2) << 4);
    if (c >= 0) v1 = *reinterpret_cast<const uint4*>(q1);
    if (r + 1 < rounds && c2 >= 0) v2 = *reinterpret_cast<const uint4*>(q2);
    if (c >= 0) {
      if (q1 < ps + 4 || q1 + 16 > pe) {
        v1.x = crc_fix_word(v1.x, q1, ps, pe);
        v1.y = crc_fix_word(v1.y, q1 + 4, ps, pe);
        v1.z = crc_fix_word(v1.z, q1 + 8, ps, pe);
        v1.w = crc_fix_word(v1.w, q1 + 12, ps, pe);
      }
      acc = crc_chunk(r ? crc_shift_s(zb, acc) : acc, v1, tb);
    }
    if (r + 1 < rounds) {
      if (c2 >= 0) {
        if (q2 < ps + 4 || q2 + 16 > pe) {
          v2.x = crc_fix_word(v2.x, q2, ps, pe);
          v2.y = crc_fix_word(v2.y, q2 + 4, ps, pe);
          v2.z = crc_fix_word(v2.z, q2 + 8, ps, pe);
          v2.w = crc_fix_word(v2.w, q2 + 12, ps, pe);
        }
        acc = crc_chunk(crc_shift_s(zb, acc), v2, tb);
      }
    }
  }
  return crc_il_finish(acc, pad, tabs, lane);
}

// Stage the slicing table into shared memory (1024 words), whole CTA.
__device__ __forceinline__ void load_slice_table(uint32_t* sT, const CrcTabs tabs) {
  for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) sT[i] = __ldg(tabs.slice + i);
}

}  // namespace luda
