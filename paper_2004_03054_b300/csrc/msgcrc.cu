// msgcrc.cu -- CRC-32C of a few large messages: index and filter blocks (§II-A; LUDA
// §III-C "filter" kernel writes them, every block carries a checksum).
//
// A message is cut into at most kMsgMaxChunks chunks of at least 4 KiB, and every chunk of
// every message goes to its own warp, so a handful of quarter-megabyte blocks spread over
// the whole GPU (a fixed number of chunk slots per message keeps the mapping free of any
// prefix sum; empty slots are skipped). A warp computes its chunk's register without the
// final complement, the first chunk from the init register 0xFFFFFFFF and the others from
// a zero register, moves it past the bytes that follow the chunk in the message and XORs it
// into the message's accumulator. By linearity over GF(2) the accumulator is then the
// register of the whole message,
//   XOR_c Z_{bytes after chunk c}(R(chunk c)),
// where Z_L moves a register past L zero bytes; a second kernel complements it and writes
// (or checks) the masked trailer.
#include <cstdint>

#include "internal.cuh"

namespace luda {

namespace {

constexpr int kMsgWarps = 32;
constexpr uint32_t kMsgMaxChunks = 64;
constexpr uint32_t kMsgSmem = kRepSmem;

__device__ __forceinline__ uint64_t msg_chunk(uint64_t n) {
  const uint64_t c = (n + kMsgMaxChunks - 1) / kMsgMaxChunks;
  return c < 4096 ? 4096 : (c + 15) & ~uint64_t(15);
}

// Warp w of the grid takes slot w: message w / kMsgMaxChunks, chunk w % kMsgMaxChunks.
__global__ void __launch_bounds__(kMsgWarps * 32, 1) k_msg_chunks(CrcMsg* __restrict__ msgs,
                                                                  const uint32_t* __restrict__ count, uint32_t mult,
                                                                  CrcTabs tabs) {
  extern __shared__ uint32_t s_msg[];
  load_rep_tables992(s_msg, s_msg + kRepWords, tabs);
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t tl = smem_addr(s_msg) + lane * 4u, tz = zcopy_addr(s_msg + kRepWords, lane);
  const uint64_t n_slots = uint64_t((count ? *count : 1u) * mult) * kMsgMaxChunks;
  const uint64_t warps = gstride() / 32;
  for (uint64_t w = gtid() / 32; w < n_slots; w += warps) {
    const uint32_t m = uint32_t(w / kMsgMaxChunks), c = uint32_t(w % kMsgMaxChunks);
    const CrcMsg M = msgs[m];
    if (M.p == nullptr) continue;
    const uint64_t chunk = msg_chunk(M.n);
    const uint64_t a = uint64_t(c) * chunk;
    if (a >= M.n) continue;
    const uint64_t len = M.n - a < chunk ? M.n - a : chunk;
    const uint32_t raw = c == 0 ? warp_crc32c_u32<true, false>(M.p, len, tl, tz, tabs)
                                : warp_crc32c_u32<false, false>(M.p + a, len, tl, tz, tabs);
    if (lane == 0) atomicXor(&msgs[m].acc, crc_zeros(raw, M.n - a - len, tabs));
  }
}

__global__ void k_msg_finish(const CrcMsg* __restrict__ msgs, const uint32_t* __restrict__ count, uint32_t mult,
                             DErr* errs, CrcTabs tabs) {
  const uint32_t n_msgs = (count ? *count : 1u) * mult;
  for (uint64_t m = gtid(); m < n_msgs; m += gstride()) {
    const CrcMsg M = msgs[m];
    if (M.p == nullptr) continue;
    const uint32_t crc = M.acc ^ 0xFFFFFFFFu;
    if (M.verify) {
      if (crc_unmask(ld_u32(M.out)) != crc) report(errs + M.job, E_CORRUPT, M.local, M.where);
    } else {
      st_u32(M.out, crc_mask(crc));
    }
  }
}

}  // namespace

void launch_msg_crc(CrcMsg* msgs, const uint32_t* count, uint32_t mult, uint32_t max_msgs, DErr* errs, CrcTabs tabs,
                    cudaStream_t st) {
  if (!max_msgs) return;
  smem_optin(k_msg_chunks, kMsgSmem);
  k_msg_chunks<<<kSms, kMsgWarps * 32, kMsgSmem, st>>>(msgs, count, mult, tabs);
  k_msg_finish<<<grid_for(max_msgs, 128, kSms), 128, 0, st>>>(msgs, count, mult, errs, tabs);
  count_launches(2);
}

}  // namespace luda
