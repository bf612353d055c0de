// decode.cu -- Phase 1 "Unpack" (LUDA §II-A; §III-C "unpack" kernel, Fig. 4a).
//
// Per input table: parse the footer and verify the index block. Per data block (there
// are no data dependencies among data blocks, §III-C): verify the trailer CRC and the
// block structure, count entries, then restore every full key from the shared prefixes
// into a key arena and emit one record per entry. Values are not copied: a record keeps
// the device address of its value inside the input table, so values move exactly once,
// from the input straight into the output block (the paper's "lazy value movement" of
// §III-D taken one step further).
#include <cstdint>

#include "internal.cuh"

namespace luda {

namespace {

__device__ __forceinline__ bool handle_ok(uint64_t off, uint64_t size, uint64_t limit) {
  return off <= limit && size <= limit - off && uint64_t(kTrailer) <= limit - off - size;
}

// One thread per input: parse the footer (magic, metaindex and index handles) and queue the
// index block (contents and type byte) for the multi-warp checksum.
__global__ void k_footers(DInput* in, uint32_t n_inputs, DErr* errs, CrcMsg* msgs) {
  for (uint64_t i = gtid(); i < n_inputs; i += gstride()) {
    const uint8_t* f = in[i].data;
    const uint64_t size = in[i].size;
    DErr* e = errs + in[i].job;
    const uint32_t local = in[i].local;
    uint64_t ioff = 0, isize = 0;
    int ok = 0;
    if (size >= kFooter && ld_u64(f + size - 8) == kMagic) {
      const uint8_t* p = f + size - kFooter;
      const uint8_t* end = p + 40;
      uint64_t moff = 0, msize = 0;
      uint32_t a = get_varint<64>(p, end, &moff);
      if (a) a = (p += a, get_varint<64>(p, end, &msize));
      if (a) a = (p += a, get_varint<64>(p, end, &ioff));
      if (a) a = (p += a, get_varint<64>(p, end, &isize));
      const uint64_t limit = size - kFooter;
      ok = a && handle_ok(moff, msize, limit) && handle_ok(ioff, isize, limit);
    }
    CrcMsg m{};
    if (ok) {
      m.p = f + ioff;
      m.n = isize + 1;
      m.out = const_cast<uint8_t*>(f + ioff + isize + 1);
      m.where = ioff;
      m.job = in[i].job;
      m.local = local;
      m.verify = 1;
    } else {
      report(e, E_CORRUPT, local, size);
      ioff = isize = 0;
    }
    msgs[i] = m;
    in[i].idx_off = ioff;
    in[i].idx_size = isize;
    in[i].nblk = ok ? 1u : 0u;  // provisional: footer parsed
  }
}

// After the index checksums: type byte and restart count give the number of data blocks.
__global__ void k_footers_finish(DInput* in, uint32_t n_inputs, DErr* errs) {
  for (uint64_t i = gtid(); i < n_inputs; i += gstride()) {
    const DInput d = in[i];
    uint32_t nblk = 0;
    if (d.nblk && *(volatile int32_t*)&errs[d.job].code == 0) {
      const uint8_t* f = d.data;
      if (f[d.idx_off + d.idx_size] != 0) {
        report(errs + d.job, E_NOTSUP, d.local, d.idx_off);
      } else {
        const uint64_t nr = d.idx_size >= 4 ? ld_u32(f + d.idx_off + d.idx_size - 4) : 0;
        if (nr >= 1 && nr <= (d.idx_size - 4) / 4) nblk = uint32_t(nr);
        else report(errs + d.job, E_CORRUPT, d.local, d.idx_off);
      }
    }
    in[i].nblk = nblk;
  }
}

// Index entry k of input d (restart interval 1, so every entry starts a restart segment
// and all decode independently): its key and block handle; false when malformed.
__device__ bool index_entry(const DInput& d, uint32_t k, const uint8_t** key, uint32_t* klen, uint64_t* off,
                            uint64_t* size) {
  const uint8_t* ib = d.data + d.idx_off;
  const uint64_t rstart = d.idx_size - 4 - 4ull * d.nblk;
  const uint64_t s = ld_u32(ib + rstart + 4ull * k);
  const uint64_t e = k + 1 < d.nblk ? ld_u32(ib + rstart + 4ull * (k + 1)) : rstart;
  if ((k == 0 && s != 0) || s >= e || e > rstart) return false;
  const uint8_t* p = ib + s;
  const uint8_t* end = ib + e;
  uint64_t shared = 0, nonshared = 0, vlen = 0;
  uint32_t a = get_varint<32>(p, end, &shared);
  if (a) a = (p += a, get_varint<32>(p, end, &nonshared));
  if (a) a = (p += a, get_varint<32>(p, end, &vlen));
  if (a) p += a;
  if (!(a && shared == 0 && nonshared <= uint64_t(end - p) && vlen <= uint64_t(end - p) - nonshared)) return false;
  *key = p;
  *klen = uint32_t(nonshared);
  p += nonshared;
  if (p + vlen != end) return false;
  const uint8_t* vend = p + vlen;
  uint32_t b = get_varint<64>(p, vend, off);
  if (b) b = (p += b, get_varint<64>(p, vend, size));
  return b && p + b == vend && handle_ok(*off, *size, d.size - kFooter);
}

// One thread per data block: its index entry gives the block handle. A block of a ranged
// job (R13) that cannot hold keys of the range (its index key's user key is below lo, or
// the previous block's is at or above hi) is left unread (null ptr).
__global__ void k_index_entries(const DInput* __restrict__ in, uint32_t n_inputs,
                                const uint32_t* __restrict__ in_blk_first, uint32_t n_blocks,
                                BlockDesc* __restrict__ blocks, DErr* errs, const JobRange* __restrict__ ranges,
                                const uint8_t* __restrict__ bounds) {
  for (uint64_t g = gtid(); g < n_blocks; g += gstride()) {
    uint32_t lo = 0, hi = n_inputs;  // last input with blk_first <= g
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (in_blk_first[mid] <= g) lo = mid;
      else hi = mid;
    }
    const DInput d = in[lo];
    const uint32_t k = uint32_t(g - in_blk_first[lo]);
    BlockDesc out{nullptr, 0, 0, lo, d.job, nullptr, 0, 0};
    if (k >= d.nblk) {  // only when a replayed plan sees fewer blocks than it was sized for
      report(errs + d.job, E_PLAN, d.local, d.idx_off);
      blocks[g] = out;
      continue;
    }
    const uint8_t* ikey = nullptr;
    uint32_t ilen = 0;
    uint64_t off = 0, size = 0;
    if (index_entry(d, k, &ikey, &ilen, &off, &size)) {
      bool read = true;
      if (ranges && ranges[d.job].flags) {
        const JobRange r = ranges[d.job];
        if ((r.flags & 1u) && ilen >= 8 && cmp_user_keys(ikey, ilen - 8, bounds + r.lo_off, r.lo_len) < 0)
          read = false;
        const uint8_t* pk;
        uint32_t pl;
        uint64_t po, ps;
        if (read && k > 0 && (r.flags & 2u) && index_entry(d, k - 1, &pk, &pl, &po, &ps) && pl >= 8 &&
            cmp_user_keys(pk, pl - 8, bounds + r.hi_off, r.hi_len) >= 0)
          read = false;
      }
      if (read) {
        out.ptr = d.data + off;
        out.size = size;
        out.off = off;
        out.ikey = ikey;
        out.ilen = ilen;
      }
    } else {
      const uint64_t rstart = d.idx_size - 4 - 4ull * d.nblk;
      report(errs + d.job, E_CORRUPT, d.local, d.idx_off + rstart + 4ull * k);
    }
    blocks[g] = out;
  }
}

// ---- block scan: checksum verify and structure walk ----------------------------------------
// k_block_verify: one warp per data block recomputes the CRC-32C of contents || type byte
// (32-byte lane spans, lane-replicated tables, 1024-thread CTAs, one per SM) and checks
// the type byte. k_block_walk: one thread per data block walks the restart segments in
// order (the entries' offsets depend on the previous entries' headers, so a block's walk is
// sequential; blocks run in parallel), checks the structure, counts entries and key bytes
// and records the first kHdrMax entry offsets for the decoder. Each header is read from one
// 16-byte window (two aligned 8-byte loads; tables are readable up to 16 bytes past any
// entry, since at least the trailer and footer follow every data block).
constexpr int kVerifyWarps = 32;
constexpr uint32_t kVerifySmem = kRepSmem;

__global__ void __launch_bounds__(kVerifyWarps * 32, 1) k_block_verify(const BlockDesc* __restrict__ blocks,
                                                                       uint32_t n_blocks,
                                                                       const DInput* __restrict__ in,
                                                                       const DErr* errs, DErr* verr, CrcTabs tabs,
                                                                       uint32_t* __restrict__ next) {
  extern __shared__ uint32_t s_ver[];
  __shared__ uint32_t s_go;  // one decision for the whole CTA
  if (threadIdx.x == 0) s_go = *(volatile uint32_t*)next < n_blocks;
  __syncthreads();
  if (!s_go) return;  // a helper launch with nothing left
  load_rep_tables992(s_ver, s_ver + kRepWords, tabs);
  __syncthreads();
  const uint32_t lane = lane_id();
  const uint32_t tl = smem_addr(s_ver) + lane * 4u, tz = zcopy_addr(s_ver + kRepWords, lane);
  for (;;) {
    uint32_t g = 0;
    if (lane == 0) g = atomicAdd(next, 1u);
    g = __shfl_sync(0xFFFFFFFFu, g, 0);
    if (g >= n_blocks) break;
    const BlockDesc b = blocks[g];
    DErr* e = verr + b.job;
    if (b.ptr == nullptr || *(volatile const int32_t*)&errs[b.job].code != 0 || *(volatile int32_t*)&e->code != 0)
      continue;
    const uint32_t got = warp_crc32c_u32(b.ptr, b.size + 1, tl, tz, tabs);
    if (lane == 0) {
      const uint32_t want = crc_unmask(ld_u32(b.ptr + b.size + 1));
      if (got != want) report(e, E_CORRUPT, in[b.input].local, b.off);
      else if (b.ptr[b.size] > 1) report(e, E_NOTSUP, in[b.input].local, b.off);  // 1: compressed (R4c)
    }
  }
}

// Byte i (< 16) of the 16-byte window w0 | w1 << 64.
__device__ __forceinline__ uint32_t win_byte(uint64_t w0, uint64_t w1, uint32_t i) {
  return uint32_t((i < 8 ? w0 >> (8 * i) : w1 >> (8 * (i - 8))) & 0xFFu);
}

// Parses the three varint32 header fields of the entry at p (p < end). Returns the header
// length, or 0 on a malformed or out-of-range varint.
__device__ __forceinline__ uint32_t read_header(const uint8_t* p, const uint8_t* end, uint32_t* f) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(7);
  const uint32_t o = uint32_t(reinterpret_cast<uintptr_t>(p) & 7u);
  const uint64_t u0 = *reinterpret_cast<const uint64_t*>(a), u1 = *reinterpret_cast<const uint64_t*>(a + 8);
  const uint64_t w0 = o ? (u0 >> (8 * o)) | (u1 << (64 - 8 * o)) : u0;
  const uint64_t w1 = u1 >> (8 * o);
  const uint32_t have = 16u - o;  // window bytes starting at p
  const uint64_t room = uint64_t(end - p);
  uint32_t pos = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint64_t v = 0;
    uint32_t i = 0;
    for (;; ++i) {
      if (i == 5 || pos >= room) return 0;
      const uint32_t byte = pos < have ? win_byte(w0, w1, pos) : p[pos];
      ++pos;
      v |= uint64_t(byte & 0x7Fu) << (7 * i);
      if (!(byte & 0x80u)) break;
    }
    if (v > 0xFFFFFFFFull) return 0;
    f[k] = uint32_t(v);
  }
  return pos;
}

// Stored blocks: a compressed one (type 1, R4c) is not walked here; with ulen given its
// decompressed length goes to ulen[g] and its arena share (16-byte multiple) to ures[g]
// (kRawBlock and 0 for the others), without ulen it is not supported. With `contents` the
// blocks are contents (decompressed or raw), the type byte is not read, and the stored
// bytes were counted already.
__global__ void __launch_bounds__(256) k_block_walk(const BlockDesc* __restrict__ blocks, uint32_t n_blocks,
                                                    const DInput* __restrict__ in, uint32_t* __restrict__ nrec,
                                                    uint64_t* __restrict__ kbytes, DErr* errs, Counts* counts,
                                                    uint2* __restrict__ ent_tab, uint64_t* __restrict__ ulen,
                                                    uint64_t* __restrict__ ures, bool contents,
                                                    uint32_t* __restrict__ nch) {
  unsigned long long data_bytes = 0, comp_bytes = 0;
  uint32_t max_kv = 0, comp = 0;
  for (uint64_t g = gtid(); g < n_blocks; g += gstride()) {
    const BlockDesc b = blocks[g];
    DErr* e = errs + b.job;
    uint32_t cnt = 0;
    uint64_t kb = 0;
    if (!contents && ulen) {
      ulen[g] = kRawBlock;
      ures[g] = 0;
    }
    if (b.ptr != nullptr && *(volatile int32_t*)&e->code == 0) {
      if (!contents) data_bytes += b.size + kTrailer;
      if (!contents && b.ptr[b.size] == 1) {
        // the stream's length header: a varint32 inside the stored bytes
        uint64_t n = 0;
        uint32_t sh = 0, k = 0;
        bool ok = false;
        for (; k < 5 && k < b.size; ++k) {
          const uint8_t c = b.ptr[k];
          n |= uint64_t(c & 0x7Fu) << sh;
          sh += 7;
          if (!(c & 0x80u)) {
            ok = n <= 0xFFFFFFFFull;
            break;
          }
        }
        if (!ulen) {
          report(e, E_NOTSUP, in[b.input].local, b.off);
        } else if (!ok) {
          report(e, E_CORRUPT, in[b.input].local, b.off);
        } else {
          ulen[g] = n;
          ures[g] = ((n + 15) & ~15ull) + 16;
          comp_bytes += ures[g];
          comp += 1;
        }
        nrec[g] = 0;
        kbytes[g] = 0;
        if (nch) nch[g] = 0;
        continue;
      }
      const uint64_t nr = b.size >= 4 ? ld_u32(b.ptr + b.size - 4) : 0;
      bool bad = !(nr >= 1 && nr <= (b.size - 4) / 4);
      if (!bad) {
        const uint64_t rstart = b.size - 4 - 4 * nr;
        const uint8_t* rs = b.ptr + rstart;
        uint2* ents = ent_tab && b.size < 65536 ? ent_tab + g * kHdrMax : nullptr;
        uint64_t s = ld_u32(rs);
        bad = s != 0;
        for (uint64_t k = 0; k < nr && !bad; ++k) {
          const uint64_t en = k + 1 < nr ? ld_u32(rs + 4 * (k + 1)) : rstart;
          if (s >= en || en > rstart) {
            bad = true;
            break;
          }
          const uint8_t* p = b.ptr + s;
          const uint8_t* end = b.ptr + en;
          uint64_t prev = 0;
          bool first = true;
          while (p < end) {
            const uint32_t off = uint32_t(p - b.ptr);
            uint32_t f[3];
            const uint32_t hl = read_header(p, end, f);
            if (!hl) {
              bad = true;
              break;
            }
            p += hl;
            const uint64_t shared = f[0], nonshared = f[1], vlen = f[2];
            if ((first && shared != 0) || shared > prev || nonshared > uint64_t(end - p) ||
                vlen > uint64_t(end - p) - nonshared || shared + nonshared < 8) {
              bad = true;
              break;
            }
            if (ents && cnt < kHdrMax) {
              // entry start, value start and end; shared and non-shared key bytes (at most 255
              // each here: longer keys are rebuilt by the sequential walk anyway)
              const uint32_t vs = uint32_t(p - b.ptr) + uint32_t(nonshared);
              ents[cnt] = make_uint2(off | (vs << 16), (vs + uint32_t(vlen)) | (min(uint32_t(shared), 255u) << 16) |
                                                           (min(uint32_t(nonshared), 255u) << 24));
            }
            p += nonshared + vlen;
            prev = shared + nonshared;
            max_kv = max(max_kv, uint32_t(prev + vlen));
            first = false;
            cnt += 1;
            kb += prev;
          }
          s = en;
        }
      }
      if (bad) {
        report(e, E_CORRUPT, in[b.input].local, b.off);
        cnt = 0;
        kb = 0;
      }
    }
    nrec[g] = cnt;
    kbytes[g] = kb;
    if (nch) {
      // chunks of the unpack's boundary path: the message (contents and type byte) widened
      // to 16-byte words, in kChunk-byte chunks
      const uintptr_t ps = reinterpret_cast<uintptr_t>(b.ptr), a1 = (ps + b.size + 1 + 15) & ~uintptr_t(15);
      const uint64_t U = (a1 - (ps & ~uintptr_t(15)) + kChunk - 1) / kChunk;
      nch[g] = cnt > 0 && cnt <= kHdrMax && b.size < 65536 && U <= kUnpChunkMax ? uint32_t(U) : 0u;
    }
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    data_bytes += __shfl_xor_sync(0xFFFFFFFFu, data_bytes, d);
    comp_bytes += __shfl_xor_sync(0xFFFFFFFFu, comp_bytes, d);
    comp += __shfl_xor_sync(0xFFFFFFFFu, comp, d);
  }
  if ((threadIdx.x & 31u) == 0 && data_bytes)
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts->in_data_bytes), data_bytes);
  if ((threadIdx.x & 31u) == 0 && comp) {
    atomicAdd(&counts->comp_blocks, comp);
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts->comp_bytes), comp_bytes);
  }
  max_kv = __reduce_max_sync(0xFFFFFFFFu, max_kv);
  if ((threadIdx.x & 31u) == 0 && max_kv) atomicMax(&counts->max_kv, max_kv);
}

// Keys of at most 32 * kDecSlots = 128 bytes are rebuilt with lanes as byte positions; a
// block with longer keys (or too many entries for the walk's table) is decoded by one lane
// walking its restart segments in order (decode_walk).
constexpr uint32_t kDecSlots = 4;  // key bytes per lane: 128-byte keys
constexpr uint32_t kKeyBatch = 4;  // entries whose key bytes k_keys loads at once

__device__ void decode_walk(const BlockDesc& b, uint64_t rec, uint64_t kpos, const Recs& recs, uint8_t* arena, bool* bad) {
  const uint64_t nr = ld_u32(b.ptr + b.size - 4);
  const uint64_t rstart = b.size - 4 - 4 * nr;
  const uint8_t* rs = b.ptr + rstart;
  for (uint64_t k = 0; k < nr; ++k) {
    const uint8_t* p = b.ptr + ld_u32(rs + 4 * k);
    const uint8_t* end = b.ptr + (k + 1 < nr ? ld_u32(rs + 4 * (k + 1)) : rstart);
    uint64_t prev_kpos = 0;
    while (p < end) {
      uint64_t shared, nonshared, vlen;
      p += get_varint<32>(p, end, &shared);
      p += get_varint<32>(p, end, &nonshared);
      p += get_varint<32>(p, end, &vlen);
      uint8_t* kd = arena + kpos;
      for (uint64_t t = 0; t < shared; ++t) kd[t] = arena[prev_kpos + t];
      for (uint64_t t = 0; t < nonshared; ++t) kd[shared + t] = p[t];
      p += nonshared;
      const uint32_t klen = uint32_t(shared + nonshared);
      const uint64_t tr = ld_u64(kd + klen - 8);
      if ((tr & 0xFF) > 1) *bad = true;
      recs.pfx[rec] = key_prefix(kd, klen - 8);
      recs.koff[rec] = kpos;
      recs.klen[rec] = klen;
      recs.tr[rec] = tr;
      recs.vptr[rec] = reinterpret_cast<uint64_t>(p);
      recs.vlen[rec] = uint32_t(vlen);
      recs.src[rec] = b.input;
      p += vlen;
      prev_kpos = kpos;
      kpos += klen;
      ++rec;
    }
  }
}

// F(value) of every record: one warp per record, 32-byte lane spans over the value from a
// zero register, without the final complement (the piece the encoder's trailers reuse).
__global__ void __launch_bounds__(kVerifyWarps * 32, 1) k_value_crc(Recs recs, const uint32_t* __restrict__ n_dev,
                                                                    uint32_t n_max, CrcTabs tabs) {
  extern __shared__ uint32_t s_vc[];
  load_rep_tables992(s_vc, s_vc + kRepWords, tabs);
  __syncthreads();
  const uint32_t n = n_dev ? *n_dev : n_max;
  const uint32_t lane = lane_id();
  const uint32_t tl = smem_addr(s_vc) + lane * 4u, tz = zcopy_addr(s_vc + kRepWords, lane);
  const uint64_t warps = gstride() / 32;
  for (uint64_t r = gtid() / 32; r < n; r += warps) {
    const uint32_t c = warp_crc32c_u32<false, false>(reinterpret_cast<const uint8_t*>(recs.vptr[r]), recs.vlen[r],
                                                      tl, tz, tabs);
    if (lane == 0) recs.vcrc[r] = c;
  }
}

// ---- unpack: records and keys; checksums and value registers from one read of each block ----
// One warp per data block in every kernel (§III-C "unpack": blocks are independent).
//
// k_keys (main stream). Lane per entry from the walk's entry table: the records' value and
// key fields; the keys are rebuilt with lanes as byte positions (the shared prefix carried
// in registers, the delta read from the block) into a per-warp buffer in shared memory and
// the key arena. Blocks the table does not cover are decoded by one lane walking them.
//
// k_unpack (second stream, beside the merge, drop rule and cuts; a work counter hands out
// blocks). The block's message (contents and type byte, n bytes) is cut into chunks of
// kChunk = 144 bytes that end at the 16-byte boundary after its end (bytes outside the
// message read as zero); in round r lane l folds chunk U - 32 * (rounds - r) + l with two
// independent registers (the chunk's first 64 bytes and its last 80, joined by Z_80), and
// keeps Z_{32 * kChunk}-weighted sums of its chunks; a butterfly joins the lanes
// (Z_{kChunk * 2^k}). With the first four message bytes complemented (the register's
// initial value), the result equals Z_pad of the complemented stored CRC when the block is
// intact. For a block with at most kHdrMax entries the walk's entry table gives the pieces
// of the message (each entry's header with key delta, its value, and the restart array
// with num_restarts and the type byte), and the pass stores, per chunk, its register
// (chunkF) and, per piece boundary, the register of its chunk's bytes before the
// boundary's 16-byte word (snap). For other blocks each value's register is computed by
// the whole warp on its own.
//
// k_vcrc (second stream, after k_unpack; blocks with boundaries). A half warp per block, a lane per entry: the
// prefix register at a boundary is its word's register advanced by the word's bytes before
// it; F(value) = S(end) xor Z_len(S(start)) inside one chunk, the chunks in between joined
// by Z_kChunk (Horner). Only the trailers of the new data blocks read the value registers.
constexpr uint32_t kUnpWarps = 16;
constexpr uint32_t kUnpBndMax = 2 * kHdrMax + 2;  // piece boundaries: two per entry, the tail, the end
constexpr uint32_t kSkStride = 11;                // words of a lane's slot (odd: lanes hit distinct banks)
struct UnpWarp {
  uint32_t bnd[2][kUnpBndMax];  // piece boundaries (message offsets, ascending) of the warp's block, or of
                                // each half warp's block
  uint32_t sk[32 * kSkStride];  // per lane of a round: its chunk's registers before each 16-byte word, then
                                // the first chain's register
};
constexpr uint32_t kUnpSmem = kRepWords * 4 + kChunkTables * 4096 + kUnpWarps * uint32_t(sizeof(UnpWarp));
static_assert(kUnpSmem <= 227u * 1024u, "unpack shared memory");

// Byte step with this lane's column of the lane-replicated slicing tables.
__device__ __forceinline__ uint32_t crc_byte_rep(uint32_t c, uint32_t b, uint32_t tl) {
  return lds_off<0u>(tl + ((c ^ b) & 0xFFu) * 128u) ^ (c >> 8);
}

// Z_L(v) for L < 256: L mod 16 zero bytes (four at a time with the slicing tables, then
// single bytes), then Z_16, Z_32, Z_64, Z_128 (sC: the chunk matrices in shared memory).
__device__ __forceinline__ uint32_t unp_zeros(uint32_t v, uint32_t L, uint32_t tl, const uint32_t* sC) {
  uint32_t r = L & 15u;
  for (; r >= 4; r -= 4) v = crc_word_rep(v, 0u, tl);
  for (; r; --r) v = crc_byte_rep(v, 0u, tl);
  const uint32_t q = L >> 4;
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j)
    if (q & (1u << j)) v = crc_mat(sC + (kCZ16 + j) * 1024u, v);
  return v;
}

// Message geometry: chunks of kChunk bytes ending at a1 = end rounded up to 16.
struct UnpGeo {
  uintptr_t ps, pe, a1, lo16;
  uint32_t U, pad;
  int32_t x0;  // message offset of chunk 0's first byte (<= 0)
};

__device__ __forceinline__ UnpGeo unp_geo(const uint8_t* p, uint32_t n) {
  UnpGeo G;
  G.ps = reinterpret_cast<uintptr_t>(p);
  G.pe = G.ps + n;
  G.a1 = (G.pe + 15) & ~uintptr_t(15);
  G.lo16 = G.ps & ~uintptr_t(15);
  G.pad = uint32_t(G.a1 - G.pe);
  G.U = uint32_t((G.a1 - G.lo16 + kChunk - 1) / kChunk);
  G.x0 = int32_t(int64_t(G.a1) - int64_t(kChunk) * int64_t(G.U) - int64_t(G.ps));
  return G;
}

// Bytes of the little-endian word at address q outside [ps, pe) become 0.
__device__ __forceinline__ uint32_t unp_mask(uint32_t w, uintptr_t q, uintptr_t ps, uintptr_t pe) {
  uint32_t keep = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b)
    if (q + b >= ps && q + b < pe) keep |= 0xFFu << (8 * b);
  return w & keep;
}

__device__ __forceinline__ uint4 unp_mask4(uint4 x, uintptr_t q, uintptr_t ps, uintptr_t pe) {
  if (q < ps || q + 16 > pe) {
    x.x = unp_mask(x.x, q, ps, pe);
    x.y = unp_mask(x.y, q + 4, ps, pe);
    x.z = unp_mask(x.z, q + 8, ps, pe);
    x.w = unp_mask(x.w, q + 12, ps, pe);
  }
  return x;
}

constexpr int kChunkW = int(kChunk / 16);  // 16-byte words of a chunk

// The words of chunk c (c < 0: zeros); only 16-byte words holding message bytes are read,
// and bytes outside the message read as 0.
__device__ __forceinline__ void unp_load(const UnpGeo G, int32_t c, uint4 (&w)[kChunkW]) {
  const uintptr_t base = G.a1 - uintptr_t(kChunk) * uintptr_t(int64_t(G.U) - c);
  if (c >= 0 && base >= G.ps && base + kChunk <= G.pe) {
    const uint4* q = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int t = 0; t < kChunkW; ++t) w[t] = q[t];
    return;
  }
#pragma unroll
  for (int t = 0; t < kChunkW; ++t) {
    const uintptr_t q = base + 16u * t;
    w[t] = make_uint4(0, 0, 0, 0);
    if (c >= 0 && q >= G.lo16) w[t] = unp_mask4(*reinterpret_cast<const uint4*>(q), q, G.ps, G.pe);
  }
}

__device__ __forceinline__ uint32_t crc_quad_rep(uint32_t S, const uint4 v, uint32_t tl) {
  S = crc_word_rep(S, v.x, tl);
  S = crc_word_rep(S, v.y, tl);
  S = crc_word_rep(S, v.z, tl);
  return crc_word_rep(S, v.w, tl);
}

// Lanes take a block in groups of GW: the whole warp (GW = 32), or each half warp its own
// block (GW = 16: for small blocks, whose last round would leave most of a warp idle).
template <uint32_t GW>
__device__ __forceinline__ uint32_t grp_mask() {
  return GW == 32 ? 0xFFFFFFFFu : (0xFFFFu << (lane_id() & 16u));
}

// Folds every chunk of the message: returns this lane's Z_{GW * kChunk}-weighted sum of its
// chunks' registers. With nb > 0 boundaries (W->bnd set), each chunk's register goes to
// chF[c] and, for each boundary inside the chunk, the register of the chunk's bytes before
// the boundary's 16-byte word to snap[i]: after each round the lanes leave their chunks'
// word registers in W->sk and then take the round's boundaries one per lane. With `init`,
// the sum is that of the message with its first four bytes complemented (the standard
// register's initial value 0xFFFFFFFF). The next round's chunks are prefetched into L2
// while a round is folded.
template <uint32_t GW>
__device__ __forceinline__ uint32_t unp_fold(const UnpGeo G, UnpWarp* W, const uint32_t* bnd, uint32_t nb,
                                             uint32_t* chF, uint32_t* snap, uint32_t tl, const uint32_t* sC,
                                             bool init) {
  const uint32_t lane = lane_id(), gl = lane & (GW - 1), gb = lane & ~(GW - 1), gm = grp_mask<GW>();
  const uint32_t rounds = (G.U + GW - 1) / GW;
  uint32_t acc = 0, bnext = 0;  // bnext: the first boundary of the round (uniform in the group)
  uint32_t* slot = W ? W->sk + lane * kSkStride : nullptr;
  for (uint32_t r = 0; r < rounds; ++r) {
    const int32_t c = int32_t(G.U) - int32_t(GW * (rounds - r)) + int32_t(gl);
    if (gl == 0 && r + 1 < rounds) {
      const uintptr_t lo = G.a1 - uintptr_t(kChunk) * uintptr_t(GW * (rounds - r - 1));
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(GW * kChunk) : "memory");
    }
    uint4 cur[kChunkW];
    unp_load(G, c, cur);
    if (c >= 0) {
      // two chains: words 0..3 (64 bytes) and 4..8 (80 bytes); Sk[j]: register before word j
      uint32_t SA = 0, SB = 0, Sk[kChunkW];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        if (j < 4) {
          Sk[j] = SA;
          SA = crc_quad_rep(SA, cur[j], tl);
        }
        Sk[4 + j] = SB;
        SB = crc_quad_rep(SB, cur[4 + j], tl);
      }
      uint32_t S = crc_mat(sC + kCZ80 * 1024u, SA) ^ SB;
      const int32_t xc = G.x0 + int32_t(kChunk) * c;  // message offset of the chunk
      if (nb) {
        chF[c] = S;
#pragma unroll
        for (int j = 0; j < kChunkW; ++j) slot[j] = Sk[j];
        slot[kChunkW] = SA;
      }
      if (init && xc < 4) {
        // bytes 0..3 of the message complemented: F(0xFFFFFFFF) shifted to the end of the
        // chunk, or (bytes split between chunks) Z_{kChunk - 1 - r}(F(0xFF)) per byte at offset r
        const int32_t r0 = -xc;
        if (r0 >= 0 && r0 + 4 <= int32_t(kChunk)) {
          S ^= unp_zeros(crc_word_rep(0u, 0xFFFFFFFFu, tl), uint32_t(int32_t(kChunk) - 4 - r0), tl, sC);
        } else {
          const uint32_t ff = crc_byte_rep(0u, 0xFFu, tl);
          for (int32_t q = 0; q < 4; ++q) {
            const int32_t rr = q - xc;
            if (rr >= 0 && rr < int32_t(kChunk)) S ^= unp_zeros(ff, uint32_t(int32_t(kChunk) - 1 - rr), tl, sC);
          }
        }
      }
      acc = crc_mat(sC + (GW == 32 ? kCZ4608 : kCZ2304) * 1024u, acc) ^ S;  // the group's other chunks of the round
    }
    if (nb) {
      // the boundaries inside this round's chunks (cr0 .. cr0 + GW - 1), one per lane; they
      // ascend, so the lanes that find one form a prefix. A boundary at the message's
      // padded end (chunk U) lies in no chunk and is never taken.
      __syncwarp(gm);
      const int32_t cr0 = int32_t(G.U) - int32_t(GW * (rounds - r));
      for (;;) {
        const uint32_t bi = bnext + gl;
        int32_t o = 0, cb = 0;
        bool mine = false;
        if (bi < nb) {
          o = int32_t(bnd[bi]) - G.x0;  // offset from chunk 0's first byte
          cb = o / int32_t(kChunk);
          mine = cb < cr0 + int32_t(GW);
        }
        const uint32_t took = __popc(__ballot_sync(gm, mine));
        if (mine) {
          const uint32_t* sl = W->sk + (gb + uint32_t(cb - cr0)) * kSkStride;
          const uint32_t k = uint32_t(o - int32_t(kChunk) * cb) >> 4;
          uint32_t sv = sl[k];
          // a word of the second chain: its register follows the first chain's bytes
          if (k >= 4) sv ^= unp_zeros(sl[kChunkW], 16u * (k - 4), tl, sC);
          snap[bi] = sv;
        }
        bnext += took;
        if (took < GW) break;
      }
      __syncwarp(gm);
    }
  }
  return acc;
}

// Z_pad(F(message)) from the group's sums (every lane gets it): a butterfly with Z_{kChunk * 2^k}.
template <uint32_t GW>
__device__ __forceinline__ uint32_t unp_join(uint32_t acc, const uint32_t* sC) {
  const uint32_t lane = lane_id(), gm = grp_mask<GW>();
#pragma unroll
  for (int k = 0; k < (GW == 32 ? 5 : 4); ++k) {
    const uint32_t other = __shfl_xor_sync(gm, acc, 1u << k);
    const uint32_t* tab = sC + (kCZ144 + k) * 1024u;
    acc = (lane & (1u << k)) ? (crc_mat(tab, other) ^ acc) : (crc_mat(tab, acc) ^ other);
  }
  return acc;
}

// F(p[0 .. n)) by the lane group (no boundaries; the pad removed with Z_{-pad}).
template <uint32_t GW>
__device__ __noinline__ uint32_t unp_range(const uint8_t* p, uint32_t n, uint32_t tl, const uint32_t* sC,
                                           const CrcTabs tabs) {
  if (n == 0) return 0;
  const UnpGeo G = unp_geo(p, n);
  uint32_t acc = unp_join<GW>(unp_fold<GW>(G, nullptr, nullptr, 0, nullptr, nullptr, tl, sC, false), sC);
  if (G.pad) acc = crc_shift(tabs.shift + size_t(kShiftPow + G.pad - 1) * 1024, acc);
  return acc;
}

// Entry count of block g as the unpack takes it: zero when a replayed plan's counts differ.
__device__ __forceinline__ uint32_t unp_entries(const UnpArgs& A, uint64_t g) {
  const uint32_t nent = A.nrec[g];
  if (A.plan_nrec && (nent != A.plan_nrec[g] || A.kbytes[g] != A.plan_kbytes[g])) return 0;
  return nent;
}

// Whether block g takes the boundary path (both kernels decide alike).
__device__ __forceinline__ bool unp_fast(const UnpArgs& A, const BlockDesc& b, uint64_t g, uint32_t nent,
                                         const UnpGeo& G) {
  return nent > 0 && nent <= kHdrMax && b.size < 65536 && G.U <= A.chunk_first[g + 1] - A.chunk_first[g];
}

template <uint32_t GW>
__global__ void __launch_bounds__(kUnpWarps * 32, 1) k_unpack(const UnpArgs A, CrcTabs tabs) {
  extern __shared__ __align__(16) uint32_t s_unp[];
  uint32_t* sTr = s_unp;
  uint32_t* sC = s_unp + kRepWords;
  UnpWarp* Wall = reinterpret_cast<UnpWarp*>(sC + kChunkTables * 1024);
  {
    const uint32_t rot = threadIdx.x & 31u;
    for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) {
      const uint32_t val = __ldg(tabs.slice + i);
      uint32_t* row = sTr + i * 32u;
#pragma unroll 8
      for (uint32_t l = 0; l < 32; ++l) row[(l + rot) & 31u] = val;
    }
    for (uint32_t i = threadIdx.x; i < kChunkTables * 1024; i += blockDim.x) sC[i] = __ldg(tabs.chunk + i);
  }
  __syncthreads();
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t gl = lane & (GW - 1), gb = lane & ~(GW - 1), gm = grp_mask<GW>();
  UnpWarp* W = Wall + warp;
  uint32_t* bnd = W->bnd[gb ? 1 : 0];  // the group's boundary list
  const uint32_t tl = smem_addr(sTr) + lane * 4u;
  uint32_t gnext = 0;
  if (gl == 0) gnext = atomicAdd(A.next, 1u);
  for (;;) {
    const uint64_t g = __shfl_sync(gm, gnext, gb);
    if (g >= A.n_blocks) break;
    // the group's next block is claimed now, so that the claim's round trip overlaps this block
    if (gl == 0) gnext = atomicAdd(A.next, 1u);
    const BlockDesc b = A.blocks[g];
    if (b.ptr == nullptr) continue;
    // the stored trailer and type byte are loaded before the fold, their round trip beside it
    uint32_t stored = 0, btype = 0;
    if (A.verify && gl == 0) {
      stored = ld_u32(b.ptr + b.size + 1);
      btype = b.ptr[b.size];
    }
    const uint32_t nent = unp_entries(A, g);
    if (!A.verify && nent == 0) continue;
    const uint64_t rec0 = A.rec_first[g];
    const uint32_t n = uint32_t(b.size) + 1;  // contents and type byte
    const UnpGeo G = unp_geo(b.ptr, n);
    const bool fast = unp_fast(A, b, g, nent, G);
    const uint32_t nb = fast ? 2 * nent + 2 : 0;
    if (fast) {
      // piece boundaries from the walk's entry table
#pragma unroll
      for (int h = 0; h < int(kHdrMax / GW); ++h) {
        const uint32_t k = gl + GW * h;
        if (k < nent) {
          const uint2 t = A.ent_tab[g * kHdrMax + k];
          bnd[2 * k] = t.x & 0xFFFFu;
          bnd[2 * k + 1] = t.x >> 16;
          if (k == nent - 1) {
            bnd[2 * nent] = t.y & 0xFFFFu;  // the restart array
            bnd[2 * nent + 1] = n;
          }
        }
      }
      __syncwarp(gm);
    }
    uint32_t acc = 0;
    if (fast || A.verify)
      acc = unp_fold<GW>(G, W, bnd, nb, A.chunkF + A.chunk_first[g], A.snap + 2 * (rec0 + g), tl, sC, A.verify);
    if (A.verify) {
      const uint32_t got = unp_join<GW>(acc, sC);
      if (gl == 0) {
        const uint32_t want = unp_zeros(~crc_unmask(stored), G.pad, tl, sC);
        DErr* ve = A.verr + b.job;
        if (got != want) report(ve, E_CORRUPT, A.in[b.input].local, b.off);
        else if (btype > 1) report(ve, E_NOTSUP, A.in[b.input].local, b.off);  // 1: compressed (R4c)
      }
    }
    if (nent == 0 || fast) {
      __syncwarp(gm);  // the group's shared arrays are reused by its next block
      continue;
    }
    // a block without boundaries: each value's register on its own; the values from the
    // entry table, or (blocks the table does not cover) from the group's first lane walking
    // the block
    const bool tab = nent <= kHdrMax && b.size < 65536;
    const uint64_t nr = ld_u32(b.ptr + b.size - 4);
    const uint64_t rstart = b.size - 4 - 4 * nr;
    const uint8_t *p = nullptr, *end = nullptr;  // the first lane's walk position
    uint64_t seg = 0;
    for (uint32_t k = 0; k < nent; ++k) {
      uint64_t vp = 0;
      uint32_t vl = 0;
      if (tab) {
        const uint2 t = A.ent_tab[g * kHdrMax + k];
        vp = reinterpret_cast<uint64_t>(b.ptr + (t.x >> 16));
        vl = (t.y & 0xFFFFu) - (t.x >> 16);
      } else if (gl == 0) {
        // the walk validated the block: next entry, crossing into the next restart segment
        while (p >= end) {
          p = b.ptr + ld_u32(b.ptr + rstart + 4 * seg);
          end = b.ptr + (seg + 1 < nr ? ld_u32(b.ptr + rstart + 4 * (seg + 1)) : rstart);
          ++seg;
        }
        uint64_t shared, nonshared, vlen;
        p += get_varint<32>(p, end, &shared);
        p += get_varint<32>(p, end, &nonshared);
        p += get_varint<32>(p, end, &vlen);
        p += nonshared;
        vp = reinterpret_cast<uint64_t>(p);
        vl = uint32_t(vlen);
        p += vlen;
      }
      vp = __shfl_sync(gm, vp, gb);
      vl = __shfl_sync(gm, vl, gb);
      const uint32_t v = unp_range<GW>(reinterpret_cast<const uint8_t*>(vp), vl, tl, sC, tabs);
      if (gl == 0) A.recs.vcrc[rec0 + k] = v;
    }
    __syncwarp(gm);
  }
}

// ---- k_vcrc and k_keys ----------------------------------------------------------------------------
constexpr uint32_t kPostWarps = 8;
constexpr uint32_t kPostZ = kCZ144 + 1;  // the chunk matrices kCZ16 .. kCZ144
constexpr uint32_t kPostSmem = (1024 + kPostZ * 1024) * 4;
// k_keys: luda_tuning.decode_warps warps per CTA, rounded up to 2, 4, 8 or 16

// Z_L(v) for L < 256 with the slicing table sT and the matrices sZ (Z_16 .. Z_128) in shared
// memory: whole zero words, single zero bytes, then the matrices.
__device__ __forceinline__ uint32_t post_zeros(uint32_t v, uint32_t L, const uint32_t* sT, const uint32_t* sZ) {
  uint32_t r = L & 15u;
  for (; r >= 4; r -= 4) v = crc_step4(v, 0u, sT);
  for (; r; --r) v = sT[v & 0xFFu] ^ (v >> 8);
  const uint32_t q = L >> 4;
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j)
    if (q & (1u << j)) v = crc_mat(sZ + (kCZ16 + j) * 1024u, v);
  return v;
}

// Register v advanced by the first q (< 16) bytes of the 16-byte word at address w (bytes
// outside the message as 0): whole 4-byte words, then single bytes.
__device__ __forceinline__ uint32_t post_feed(uint32_t v, const UnpGeo& G, uintptr_t w, uint32_t q,
                                              const uint32_t* sT) {
  if (q == 0) return v;
  const uint4 x = unp_mask4(*reinterpret_cast<const uint4*>(w), w, G.ps, G.pe);
  const uint32_t words[4] = {x.x, x.y, x.z, x.w};
  uint32_t t = 0;
#pragma unroll
  for (uint32_t j = 0; j < 3; ++j)
    if (t + 4 <= q) {
      v = crc_step4(v, words[j], sT);
      t += 4;
    }
  const uint32_t last = t == 0 ? words[0] : t == 4 ? words[1] : t == 8 ? words[2] : words[3];
  for (uint32_t i = 0; t + i < q; ++i) v = sT[(v ^ (last >> (8 * i))) & 0xFFu] ^ (v >> 8);
  return v;
}

__global__ void __launch_bounds__(kPostWarps * 32) k_vcrc(const UnpArgs A, CrcTabs tabs) {
  extern __shared__ __align__(16) uint32_t s_post[];
  uint32_t* sT = s_post;
  uint32_t* sZ = s_post + 1024;
  for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) sT[i] = __ldg(tabs.slice + i);
  for (uint32_t i = threadIdx.x; i < kPostZ * 1024; i += blockDim.x) sZ[i] = __ldg(tabs.chunk + i);
  __syncthreads();
  const uint32_t* sZ144 = sZ + kCZ144 * 1024u;
  // a half warp per block (most blocks hold at most 16 entries, a lane each); the lanes
  // work on their own, without warp-wide operations
  const uint32_t hl = lane_id() & 15u;
  const uint64_t halves = gstride() / 16;
  for (uint64_t g = gtid() / 16; g < A.n_blocks; g += halves) {
    const BlockDesc b = A.blocks[g];
    if (b.ptr == nullptr) continue;
    const uint32_t nent = unp_entries(A, g);
    const UnpGeo G = unp_geo(b.ptr, uint32_t(b.size) + 1);
    if (!unp_fast(A, b, g, nent, G)) continue;
    const uint64_t rec0 = A.rec_first[g];
    const uint32_t* chF = A.chunkF + A.chunk_first[g];
    const uint32_t* snap = A.snap + 2 * (rec0 + g);
    const uintptr_t base0 = G.a1 - uintptr_t(kChunk) * uintptr_t(G.U);  // chunk 0's first byte
    for (uint32_t k = hl; k < nent; k += 16) {
      const uint2 t = A.ent_tab[g * kHdrMax + k];
      const uint32_t vs = t.x >> 16, ve = t.y & 0xFFFFu;
      uint32_t F = 0;
      if (vs < ve) {
        // prefix registers at the value's start (boundary 2k + 1) and end (boundary 2k + 2)
        const uint32_t ao = uint32_t(int32_t(vs) - G.x0), zo = uint32_t(int32_t(ve) - G.x0);
        const uint32_t ca = ao / kChunk, ra = ao - kChunk * ca;
        const uint32_t cb = (zo - 1) / kChunk, rb = zo - kChunk * cb;
        const uint32_t Pa = post_feed(snap[2 * k + 1], G, base0 + (ao & ~15u), ao & 15u, sT);
        const uint32_t Pb = rb == kChunk ? chF[cb] : post_feed(snap[2 * k + 2], G, base0 + (zo & ~15u), zo & 15u, sT);
        if (ca == cb) {
          F = Pb ^ post_zeros(Pa, rb - ra, sT, sZ);
        } else {
          uint32_t x = chF[ca] ^ post_zeros(Pa, kChunk - ra, sT, sZ);
          for (uint32_t c = ca + 1; c < cb; ++c) x = crc_mat(sZ144, x) ^ chF[c];
          F = post_zeros(x, rb, sT, sZ) ^ Pb;
        }
      }
      A.recs.vcrc[rec0 + k] = F;
    }
  }
}

__device__ __forceinline__ void keys_body(const UnpArgs& A) {
  const uint32_t lane = lane_id();
  const uint64_t warps = gstride() / 32;
  for (uint64_t g = gtid() / 32; g < A.n_blocks; g += warps) {
    const BlockDesc b = A.blocks[g];
    if (b.ptr == nullptr) continue;
    const uint32_t nent = unp_entries(A, g);
    if (nent == 0) continue;
    const uint64_t rec0 = A.rec_first[g], key0 = A.key_first[g];
    bool tab = nent <= kHdrMax && b.size < 65536;
    // lane per entry (entries lane and lane + 32): record fields
    uint32_t sh[2] = {0, 0}, kl[2] = {0, 0}, dp[2] = {0, 0};
    if (tab) {
      bool long_key = false;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k = lane + 32 * h;
        if (k < nent) {
          const uint2 t = A.ent_tab[g * kHdrMax + k];
          const uint32_t vs = t.x >> 16, ve = t.y & 0xFFFFu, ns = t.y >> 24;
          sh[h] = (t.y >> 16) & 0xFFu;
          kl[h] = sh[h] + ns;
          dp[h] = vs - ns;
          long_key |= kl[h] > 32 * kDecSlots;
          A.recs.vptr[rec0 + k] = reinterpret_cast<uint64_t>(b.ptr + vs);
          A.recs.vlen[rec0 + k] = ve - vs;
          A.recs.klen[rec0 + k] = kl[h];
          A.recs.src[rec0 + k] = b.input;
        }
      }
      tab = !__any_sync(0xFFFFFFFFu, long_key);
    }
    bool bad = false;
    if (!tab) {
      if (lane == 0) decode_walk(b, rec0, key0, A.recs, A.arena, &bad);
    } else {
      // key offsets: exclusive scan of key lengths over the (up to 64) entries
      uint32_t x0 = kl[0], x1 = kl[1];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o0 = __shfl_up_sync(0xFFFFFFFFu, x0, d), o1 = __shfl_up_sync(0xFFFFFFFFu, x1, d);
        if (lane >= uint32_t(d)) {
          x0 += o0;
          x1 += o1;
        }
      }
      const uint32_t tot0 = __shfl_sync(0xFFFFFFFFu, x0, 31);
      const uint32_t ko[2] = {x0 - kl[0], tot0 + x1 - kl[1]};
      // lane t keeps byte t (t + 32, ...) of the current key: the shared prefix carried from
      // the previous key, the rest read from the key delta. The delta bytes of kKeyBatch
      // entries are loaded together (they do not depend on one another), byte s of a lane's
      // share of entry i in byte s of d[i]; then the keys are rebuilt in order.
      uint32_t cur = 0;
      for (uint32_t kb = 0; kb < nent; kb += kKeyBatch) {
        uint32_t d[kKeyBatch];
#pragma unroll
        for (uint32_t i = 0; i < kKeyBatch; ++i) {
          const uint32_t k = kb + i, src = k & 31u, h = (k >> 5) & 1u;
          const uint32_t shared = __shfl_sync(0xFFFFFFFFu, h ? sh[1] : sh[0], src);
          const uint32_t klen = __shfl_sync(0xFFFFFFFFu, h ? kl[1] : kl[0], src);
          const uint32_t dpos = __shfl_sync(0xFFFFFFFFu, h ? dp[1] : dp[0], src);
          d[i] = 0;
          if (k < nent) {
#pragma unroll
            for (uint32_t s = 0; s < kDecSlots; ++s) {
              const uint32_t t = lane + 32 * s;
              if (t < klen && t >= shared) d[i] |= uint32_t(__ldg(b.ptr + dpos + t - shared)) << (8 * s);
            }
          }
        }
#pragma unroll
        for (uint32_t i = 0; i < kKeyBatch; ++i) {
          const uint32_t k = kb + i, src = k & 31u, h = (k >> 5) & 1u;
          const uint32_t shared = __shfl_sync(0xFFFFFFFFu, h ? sh[1] : sh[0], src);
          const uint32_t klen = __shfl_sync(0xFFFFFFFFu, h ? kl[1] : kl[0], src);
          const uint32_t kof = __shfl_sync(0xFFFFFFFFu, h ? ko[1] : ko[0], src);
          if (k < nent) {
            uint8_t* kd = A.arena + key0 + kof;
#pragma unroll
            for (uint32_t s = 0; s < kDecSlots; ++s) {
              const uint32_t t = lane + 32 * s;
              if (t < klen) {
                if (t >= shared) cur = (cur & ~(0xFFu << (8 * s))) | (d[i] & (0xFFu << (8 * s)));
                kd[t] = uint8_t(cur >> (8 * s));
              }
            }
          }
        }
      }
      __syncwarp();  // the warp's key bytes are visible to all its lanes
      // per entry (lane): user-key prefix and trailer read back from the rebuilt key
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k = lane + 32 * h;
        if (k < nent) {
          const uint8_t* kd = A.arena + key0 + ko[h];
          const uint32_t ul = kl[h] - 8;
          const uint64_t tr = le_word(kd + ul);
          if ((tr & 0xFF) > 1) bad = true;
          A.recs.pfx[rec0 + k] = key_word(kd, ul < 8 ? ul : 8u);
          A.recs.tr[rec0 + k] = tr;
          A.recs.koff[rec0 + k] = key0 + ko[h];
        }
      }
    }
    bad = __any_sync(0xFFFFFFFFu, bad);
    if (bad && lane == 0) report(A.errs + b.job, E_CORRUPT, A.in[b.input].local, b.off);
  }
}

// k_keys with W warps per CTA, sized for about 36 resident warps per SM (it waits on memory
// most of the time, so resident warps count more than registers).
template <uint32_t W>
__global__ void __launch_bounds__(W * 32, 36 / W) k_keys(const UnpArgs A) {
  keys_body(A);
}

// Internal-key order of two full internal keys (user key bytes, proper prefix first, then
// the trailer descending).
__device__ int cmp_ikey_bytes(const uint8_t* a, uint32_t la, const uint8_t* b, uint32_t lb) {
  const uint32_t ua = la - 8, ub = lb - 8, m = ua < ub ? ua : ub;
  for (uint32_t i = 0; i < m; i += 8) {
    const uint32_t avail = m - i < 8 ? m - i : 8u;
    const uint64_t wa = key_word(a + i, avail), wb = key_word(b + i, avail);
    if (wa != wb) return wa < wb ? -1 : 1;
  }
  if (ua != ub) return ua < ub ? -1 : 1;
  const uint64_t ta = le_word(a + ua), tb = le_word(b + ub);
  return ta == tb ? 0 : (ta > tb ? -1 : 1);
}

// R9: a data block's index key is an internal key at or above the block's last key, and
// below the first key of the next data block of the same table.
__global__ void k_check_index(const BlockDesc* __restrict__ blocks, uint32_t n_blocks, const DInput* __restrict__ in,
                              const uint32_t* __restrict__ nrec, const uint32_t* __restrict__ rec_first, Recs recs,
                              const uint8_t* __restrict__ arena, DErr* errs) {
  for (uint64_t g = gtid(); g < n_blocks; g += gstride()) {
    const BlockDesc b = blocks[g];
    if (b.ptr == nullptr || nrec[g] == 0 || *(volatile int32_t*)&errs[b.job].code != 0) continue;
    const uint32_t last = rec_first[g] + nrec[g] - 1;
    bool ok = b.ilen >= 8 && cmp_ikey_bytes(arena + recs.koff[last], recs.klen[last], b.ikey, b.ilen) <= 0;
    if (ok && g + 1 < n_blocks && blocks[g + 1].input == b.input && nrec[g + 1] > 0) {
      const uint32_t first = rec_first[g + 1];
      ok = cmp_ikey_bytes(b.ikey, b.ilen, arena + recs.koff[first], recs.klen[first]) < 0;
    }
    if (!ok) report(errs + b.job, E_CORRUPT, in[b.input].local, b.off);
  }
}

// One thread per input: link[i] = 1 when input i + 1 belongs to the same job and all its
// keys follow all of input i's (its first key, read from its first data block, is above
// input i's last index key, which is at or above its last key). Linked inputs form one sorted
// run for the merge. The index keys are checked against the data after decode, and each
// input's own order by the order check, so a link never rests on an unchecked key.
__global__ void k_run_links(const DInput* __restrict__ in, uint32_t n_inputs, const BlockDesc* __restrict__ blocks,
                            const DErr* errs, uint8_t* __restrict__ link) {
  for (uint64_t i = gtid(); i < n_inputs; i += gstride()) {
    uint8_t l = 0;
    if (i + 1 < n_inputs) {
      const DInput a = in[i], c = in[i + 1];
      if (a.job == c.job && a.nblk && c.nblk && errs[a.job].code == 0) {
        const BlockDesc la = blocks[a.blk_first + a.nblk - 1], fc = blocks[c.blk_first];
        if (la.ptr && fc.ptr && la.ilen >= 8) {
          uint32_t f[3];
          const uint32_t hl = read_header(fc.ptr, fc.ptr + fc.size, f);
          if (hl && f[0] == 0 && f[1] >= 8 && f[1] <= fc.size - hl)
            l = cmp_ikey_bytes(la.ikey, la.ilen, fc.ptr + hl, f[1]) < 0;
        }
      }
    }
    link[i] = l;
  }
}

__global__ void k_zero_failed(const BlockDesc* __restrict__ blocks, uint32_t n_blocks, const DErr* __restrict__ errs,
                              uint32_t* __restrict__ nrec, uint64_t* __restrict__ kbytes) {
  for (uint64_t g = gtid(); g < n_blocks; g += gstride())
    if (errs[blocks[g].job].code != 0 || blocks[g].ptr == nullptr) {
      nrec[g] = 0;
      kbytes[g] = 0;
    }
}

__global__ void k_input_ranges(const DInput* __restrict__ in, uint32_t n_inputs, const uint32_t* __restrict__ rec_first,
                               const uint64_t* __restrict__ key_first, uint32_t* __restrict__ in_rec,
                               uint64_t* __restrict__ in_key) {
  for (uint64_t i = gtid(); i <= n_inputs; i += gstride()) {
    const uint32_t blk =
        i < n_inputs ? in[i].blk_first : (n_inputs ? in[n_inputs - 1].blk_first + in[n_inputs - 1].nblk : 0);
    in_rec[i] = rec_first[blk];
    in_key[i] = key_first[blk];
  }
}

// Plans: a replay must see the block counts the plan was sized for.
__global__ void k_plan_check_blocks(DInput* in, uint32_t n_inputs, const uint32_t* __restrict__ plan_nblk, DErr* errs) {
  for (uint64_t i = gtid(); i < n_inputs; i += gstride())
    if (in[i].nblk != plan_nblk[i]) {
      report(errs + in[i].job, E_PLAN, in[i].local, in[i].size);
      in[i].nblk = 0;
    }
}

// ... and the entry and key-byte counts of every block.
__global__ void k_plan_check_recs(const BlockDesc* __restrict__ blocks, uint32_t n_blocks,
                                  const uint32_t* __restrict__ nrec, const uint64_t* __restrict__ kbytes,
                                  const uint32_t* __restrict__ plan_nrec, const uint64_t* __restrict__ plan_kbytes,
                                  const DInput* __restrict__ in, DErr* errs) {
  for (uint64_t g = gtid(); g < n_blocks; g += gstride())
    if (nrec[g] != plan_nrec[g] || kbytes[g] != plan_kbytes[g])
      report(errs + blocks[g].job, E_PLAN, in[blocks[g].input].local, blocks[g].off);
}

// Replay: an input that continued the previous input's run when the plan was made must
// still do so (the captured merge schedule relies on it).
__global__ void k_plan_check_links(const uint8_t* __restrict__ link, const uint8_t* __restrict__ plan_link,
                                   uint32_t n_inputs, const DInput* __restrict__ in, DErr* errs) {
  for (uint64_t i = gtid(); i < n_inputs; i += gstride())
    if (plan_link[i] && !link[i]) report(errs + in[i].job, E_PLAN, in[i].local, 0);
}

}  // namespace

void launch_plan_check_links(const uint8_t* link, const uint8_t* plan_link, uint32_t n_inputs, const DInput* in,
                             DErr* errs, cudaStream_t st) {
  if (!n_inputs) return;
  k_plan_check_links<<<grid_for(n_inputs, 128), 128, 0, st>>>(link, plan_link, n_inputs, in, errs);
  count_launches(1);
}

void launch_plan_checks(DInput* in, uint32_t n_inputs, const uint32_t* plan_nblk, DErr* errs, cudaStream_t st) {
  if (!n_inputs) return;
  k_plan_check_blocks<<<grid_for(n_inputs, 128), 128, 0, st>>>(in, n_inputs, plan_nblk, errs);
  count_launches(1);
}

void launch_plan_check_recs(const BlockDesc* blocks, uint32_t n_blocks, const uint32_t* nrec, const uint64_t* kbytes,
                            const uint32_t* plan_nrec, const uint64_t* plan_kbytes, const DInput* in, DErr* errs,
                            cudaStream_t st) {
  if (!n_blocks) return;
  k_plan_check_recs<<<grid_for(n_blocks, 256), 256, 0, st>>>(blocks, n_blocks, nrec, kbytes, plan_nrec, plan_kbytes,
                                                             in, errs);
  count_launches(1);
}

void launch_footers_read(DInput* in, uint32_t n_inputs, DErr* errs, CrcMsg* msgs, cudaStream_t st) {
  if (!n_inputs) return;
  k_footers<<<grid_for(n_inputs, 128), 128, 0, st>>>(in, n_inputs, errs, msgs);
  count_launches(1);
}

void launch_index_crc(CrcMsg* msgs, uint32_t n_inputs, DErr* errs, CrcTabs tabs, cudaStream_t st) {
  if (!n_inputs) return;
  launch_msg_crc(msgs, nullptr, n_inputs, n_inputs, errs, tabs, st);
}

void launch_footers_finish(DInput* in, uint32_t n_inputs, DErr* errs, cudaStream_t st) {
  if (!n_inputs) return;
  k_footers_finish<<<grid_for(n_inputs, 128), 128, 0, st>>>(in, n_inputs, errs);
  count_launches(1);
}

void launch_footers(DInput* in, uint32_t n_inputs, DErr* errs, CrcMsg* msgs, CrcTabs tabs, cudaStream_t st) {
  launch_footers_read(in, n_inputs, errs, msgs, st);
  launch_index_crc(msgs, n_inputs, errs, tabs, st);
  launch_footers_finish(in, n_inputs, errs, st);
}

void launch_index_entries(const DInput* in, uint32_t n_inputs, const uint32_t* in_blk_first, uint32_t n_blocks,
                          BlockDesc* blocks, DErr* errs, cudaStream_t st, const JobRange* ranges,
                          const uint8_t* bounds) {
  if (!n_blocks) return;
  k_index_entries<<<grid_for(n_blocks, 256), 256, 0, st>>>(in, n_inputs, in_blk_first, n_blocks, blocks, errs,
                                                           ranges, bounds);
  count_launches(1);
}

void launch_block_verify(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, const DErr* errs, DErr* verr,
                         CrcTabs tabs, uint32_t* next, bool helper, cudaStream_t st) {
  const uint32_t ctas = helper ? kSms - tuning().crc_ctas : tuning().crc_ctas;
  if (!n_blocks || !ctas) return;
  smem_optin(k_block_verify, kVerifySmem);
  const unsigned w = tuning().crc_warps;
  const unsigned g = grid_for(n_blocks, w, ctas);
  k_block_verify<<<g, w * 32, kVerifySmem, st>>>(blocks, n_blocks, in, errs, verr, tabs, next);
  count_launches(1);
}

void launch_block_walk(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, uint32_t* nrec,
                       uint64_t* kbytes, DErr* errs, Counts* cnt, uint2* ent_tab, cudaStream_t st,
                       uint64_t* ulen, uint64_t* ures, bool contents, uint32_t* nch) {
  if (!n_blocks) return;
  const unsigned t = tuning().walk_threads;
  k_block_walk<<<grid_for(n_blocks, t), t, 0, st>>>(blocks, n_blocks, in, nrec, kbytes, errs, cnt, ent_tab, ulen,
                                                    ures, contents, nch);
  count_launches(1);
}

// R4c, one warp per compressed block, several elements per step. The stream's next 128
// bytes sit in registers (lane l holds bytes 4l..4l+3 of the window; a byte is one
// shuffle away). Each step, lane l reads the element header that would start at p + l and
// where the element after it would start; the true element starts are the chain from p
// (one shuffle per element), their output positions a warp scan of their lengths. The
// marked elements of at most 64 bytes whose source lies wholly before the step's first
// output byte (literals, and copies reaching back past it) are then written at once, each
// by its own lane; the others (long literals, copies of bytes this step writes) follow in
// order, the warp's lanes covering an element's bytes. A copy of offset d and length L
// writes out[w + i] = out[w - d + i mod d] for i < L (its own output repeats with period
// d, so every byte comes from the d bytes before w). Any element that runs past the
// stream, copies from before the output or writes past the announced length, or a total
// other than it, is CORRUPTION; the block's contents pointer stays null then.
__global__ void __launch_bounds__(256) k_decompress(const BlockDesc* __restrict__ blocks, uint32_t n_blocks,
                                                    const uint64_t* __restrict__ ulen,
                                                    const uint64_t* __restrict__ uoff, uint8_t* __restrict__ dst,
                                                    uint64_t dst_cap, BlockDesc* __restrict__ cblocks,
                                                    const DInput* __restrict__ in, DErr* errs) {
  const uint32_t lane = lane_id();
  const uint64_t warps = gstride() / 32;
  for (uint64_t g = gtid() / 32; g < n_blocks; g += warps) {
    const uint64_t n64 = ulen[g];
    if (n64 == kRawBlock) continue;
    const BlockDesc b = blocks[g];
    DErr* e = errs + b.job;
    if (b.ptr == nullptr || *(volatile int32_t*)&e->code != 0) continue;
    // positions fit 32 bits: the length header is a varint32, a block's stored size too
    bool ok = uoff[g] + n64 <= dst_cap && b.size < 0xFFFFFFFFull;
    const uint32_t n = uint32_t(n64), S = uint32_t(b.size);
    uint8_t* out = dst + uoff[g];
    const uint8_t* src = b.ptr;
    uint32_t p = 0;
    while (p < S && (src[p] & 0x80u)) ++p;  // the length header (checked by the block walk)
    ++p;
    uint32_t wb = 0, word = 0;
    bool have = false;
    auto byte_at = [&](uint32_t q) -> uint32_t {  // q in [wb, wb + 128)
      const uint32_t r = q - wb;
      return (__shfl_sync(0xFFFFFFFFu, word, r >> 2) >> ((r & 3u) * 8)) & 0xFFu;
    };
    uint32_t w = 0;
    while (ok && p < S) {
      if (!have || p + 37 > wb + 128) {  // the window covers every header starting below p + 32
        wb = p;
        word = 0;
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
          const uint32_t q = wb + 4 * lane + k;
          if (q < S) word |= uint32_t(src[q]) << (8 * k);
        }
        have = true;
      }
      // the element that would start at q = p + lane
      const uint32_t q = p + lane;
      const uint32_t tag = byte_at(q < S ? q : p);
      const uint32_t kind = tag & 3u;
      uint32_t hl = kind == 0 ? 1u : (kind == 1 ? 2u : (kind == 2 ? 3u : 5u));
      uint32_t nb = 0;
      if (kind == 0 && (tag >> 2) >= 60) {
        nb = (tag >> 2) - 59;
        hl = 1 + nb;
      }
      uint32_t x[4];
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k) x[k] = byte_at(q + 1 + k);  // q + 4 < p + 36: in the window
      uint64_t len = 0;
      uint32_t arg = 0;
      if (kind == 0) {
        len = tag >> 2;
        if (nb) {
          len = 0;
#pragma unroll
          for (uint32_t k = 0; k < 4; ++k)
            if (k < nb) len |= uint64_t(x[k]) << (8 * k);
        }
        len += 1;
      } else if (kind == 1) {
        len = 4 + ((tag >> 2) & 7u);
        arg = ((tag >> 5) << 8) | x[0];
      } else {
        len = 1 + (tag >> 2);
        arg = x[0] | x[1] << 8;
        if (kind == 3) arg |= x[2] << 16 | x[3] << 24;
      }
      // header and literal bytes inside the stream; where the next element would start
      const bool fits = q < S && hl <= S - q && (kind != 0 || len <= uint64_t(S - q - hl));
      const uint64_t nx = uint64_t(q) + hl + (kind == 0 ? len : 0);
      const uint32_t nxt = fits && nx < uint64_t(p) + 32 ? uint32_t(nx - p) : 32u;
      // the chain of true element starts from p
      uint32_t marks = 0, cur = 0, last = 0;
      bool broken = false;
      while (cur < 32 && p + cur < S) {
        marks |= 1u << cur;
        last = cur;
        if (!__shfl_sync(0xFFFFFFFFu, fits ? 1u : 0u, cur)) {
          broken = true;
          break;
        }
        cur = __shfl_sync(0xFFFFFFFFu, nxt, cur);
      }
      if (broken) {
        ok = false;
        break;
      }
      const bool mine = (marks >> lane) & 1u;
      // output positions of the marked elements
      const uint64_t ml = mine ? len : 0;
      uint64_t xs = ml;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, xs, d);
        if (lane >= uint32_t(d)) xs += y;
      }
      const uint64_t total = __shfl_sync(0xFFFFFFFFu, xs, 31);
      const uint64_t wl = uint64_t(w) + xs - ml;
      const bool bad = mine && (wl + len > n || (kind != 0 && (arg == 0 || arg > wl)));
      if (__any_sync(0xFFFFFFFFu, bad)) {
        ok = false;
        break;
      }
      // elements that read nothing this step writes, at most 64 bytes: each lane its own
      const uint32_t ew = uint32_t(wl), el = uint32_t(len);
      const bool solo = mine && el <= 64 && (kind == 0 || (arg >= el ? ew - arg + el <= w : ew - arg + arg <= w));
      if (solo) {
        if (kind == 0) {
          const uint32_t from = q + hl;
          for (uint32_t k = 0; k < el; ++k) out[ew + k] = src[from + k];
        } else if (arg >= el) {
          for (uint32_t k = 0; k < el; ++k) out[ew + k] = out[ew - arg + k];
        } else {
          for (uint32_t k = 0; k < el; ++k) out[ew + k] = out[ew - arg + k % arg];
        }
      }
      __syncwarp();
      // the rest, in order
      uint32_t todo = marks & ~__ballot_sync(0xFFFFFFFFu, solo);
      while (todo) {
        const uint32_t l = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint32_t ek = __shfl_sync(0xFFFFFFFFu, kind, l);
        const uint32_t tl = __shfl_sync(0xFFFFFFFFu, el, l);
        const uint32_t tw = __shfl_sync(0xFFFFFFFFu, ew, l);
        if (ek == 0) {
          const uint32_t from = p + l + __shfl_sync(0xFFFFFFFFu, hl, l);
          for (uint32_t k = lane; k < tl; k += 32) out[tw + k] = src[from + k];
        } else {
          const uint32_t d = __shfl_sync(0xFFFFFFFFu, arg, l);
          if (d >= tl) {
            if (lane < tl) out[tw + lane] = out[tw - d + lane];
            if (lane + 32 < tl) out[tw + lane + 32] = out[tw - d + lane + 32];
          } else {  // overlapping: a pattern of d < tl <= 64 bytes
            if (lane < tl) out[tw + lane] = out[tw - d + lane % d];
            if (lane + 32 < tl) out[tw + lane + 32] = out[tw - d + (lane + 32) % d];
          }
        }
        __syncwarp();
      }
      w += uint32_t(total);
      p = uint32_t(__shfl_sync(0xFFFFFFFFu, nx, last));
    }
    if (ok && w != n) ok = false;
    if (lane == 0) {
      if (ok) {
        cblocks[g].ptr = out;
        cblocks[g].size = n;
      } else {
        cblocks[g].ptr = nullptr;
        report(e, E_CORRUPT, in[b.input].local, b.off);
      }
    }
  }
}

void launch_decompress(const BlockDesc* blocks, uint32_t n_blocks, const uint64_t* ulen, const uint64_t* uoff,
                       uint8_t* dst, uint64_t dst_cap, BlockDesc* cblocks, const DInput* in, DErr* errs,
                       cudaStream_t st) {
  if (!n_blocks) return;
  k_decompress<<<grid_for(uint64_t(n_blocks) * 32, 256), 256, 0, st>>>(blocks, n_blocks, ulen, uoff, dst, dst_cap,
                                                                      cblocks, in, errs);
  count_launches(1);
}

void launch_block_scan(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, uint32_t* nrec,
                       uint64_t* kbytes, DErr* errs, Counts* cnt, uint2* ent_tab, CrcTabs tabs, cudaStream_t st,
                       uint32_t* nch) {
  launch_block_verify(blocks, n_blocks, in, errs, errs, tabs, &cnt->crc_next_in, false, st);
  launch_block_verify(blocks, n_blocks, in, errs, errs, tabs, &cnt->crc_next_in, true, st);
  launch_block_walk(blocks, n_blocks, in, nrec, kbytes, errs, cnt, ent_tab, st, nullptr, nullptr, false, nch);
}

void launch_value_crc(Recs recs, const uint32_t* n, uint32_t n_max, CrcTabs tabs, cudaStream_t st) {
  if (!n_max) return;
  smem_optin(k_value_crc, kVerifySmem);
  k_value_crc<<<kSms, kVerifyWarps * 32, kVerifySmem, st>>>(recs, n, n_max, tabs);
  count_launches(1);
}

void launch_unpack_keys(const UnpArgs& a, cudaStream_t st) {
  if (!a.n_blocks) return;
  const uint32_t w = tuning().decode_warps;
  if (w <= 2) k_keys<2><<<grid_for(a.n_blocks, 2), 64, 0, st>>>(a);
  else if (w <= 4) k_keys<4><<<grid_for(a.n_blocks, 4), 128, 0, st>>>(a);
  else if (w <= 8) k_keys<8><<<grid_for(a.n_blocks, 8), 256, 0, st>>>(a);
  else k_keys<16><<<grid_for(a.n_blocks, 16), 512, 0, st>>>(a);
  count_launches(1);
}

void launch_unpack_crc(const UnpArgs& a, CrcTabs tabs, uint32_t ctas, bool half_warps, cudaStream_t st) {
  if (!a.n_blocks) return;
  if (half_warps) {
    smem_optin(k_unpack<16>, kUnpSmem);
    k_unpack<16><<<ctas, kUnpWarps * 32, kUnpSmem, st>>>(a, tabs);
  } else {
    smem_optin(k_unpack<32>, kUnpSmem);
    k_unpack<32><<<ctas, kUnpWarps * 32, kUnpSmem, st>>>(a, tabs);
  }
  smem_optin(k_vcrc, kPostSmem);
  k_vcrc<<<grid_for(a.n_blocks, kPostWarps, kSms * 8), kPostWarps * 32, kPostSmem, st>>>(a, tabs);
  count_launches(2);
}

void launch_check_index(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, const uint32_t* nrec,
                        const uint32_t* rec_first, Recs recs, const uint8_t* arena, DErr* errs, cudaStream_t st) {
  if (!n_blocks) return;
  k_check_index<<<grid_for(n_blocks, 256), 256, 0, st>>>(blocks, n_blocks, in, nrec, rec_first, recs, arena, errs);
  count_launches(1);
}

void launch_run_links(const DInput* in, uint32_t n_inputs, const BlockDesc* blocks, const DErr* errs, uint8_t* link,
                      cudaStream_t st) {
  if (!n_inputs) return;
  k_run_links<<<grid_for(n_inputs, 128), 128, 0, st>>>(in, n_inputs, blocks, errs, link);
  count_launches(1);
}

void launch_zero_failed(const BlockDesc* blocks, uint32_t n_blocks, const DErr* errs, uint32_t* nrec,
                        uint64_t* kbytes, cudaStream_t st) {
  if (!n_blocks) return;
  k_zero_failed<<<grid_for(n_blocks, 256), 256, 0, st>>>(blocks, n_blocks, errs, nrec, kbytes); count_launches(1);
}

void launch_input_ranges(const DInput* in, uint32_t n_inputs, const uint32_t* rec_first, const uint64_t* key_first,
                         uint32_t* in_rec, uint64_t* in_key, cudaStream_t st) {
  k_input_ranges<<<grid_for(n_inputs + 1, 256), 256, 0, st>>>(in, n_inputs, rec_first, key_first, in_rec, in_key); count_launches(1);
}

}  // namespace luda
