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
                                                    uint16_t* __restrict__ hdr_tab, uint64_t* __restrict__ ulen,
                                                    uint64_t* __restrict__ ures, bool contents) {
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
        continue;
      }
      const uint64_t nr = b.size >= 4 ? ld_u32(b.ptr + b.size - 4) : 0;
      bool bad = !(nr >= 1 && nr <= (b.size - 4) / 4);
      if (!bad) {
        const uint64_t rstart = b.size - 4 - 4 * nr;
        const uint8_t* rs = b.ptr + rstart;
        uint16_t* offs = b.size < 65536 ? hdr_tab + g * kHdrMax : nullptr;
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
            if (offs && cnt < kHdrMax) offs[cnt] = uint16_t(p - b.ptr);
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

// One warp per data block. With the block's entry offsets from the scan (at most kHdrMax
// entries, keys of at most 128 bytes), all headers are parsed at once (lane per entry)
// and the keys are rebuilt entry by entry with lanes as byte positions: lane t keeps byte
// t (t + 32, ...) of the current key in registers, takes the new bytes from the entry's
// key delta, and stores the whole key with coalesced byte stores. Other blocks are
// decoded by lane 0 alone, walking the segments in order.
constexpr uint32_t kDecSlots = 4;  // key bytes per lane: 128-byte keys

__device__ void decode_walk(const BlockDesc& b, uint64_t rec, uint64_t kpos, Recs& recs, uint8_t* arena, bool* bad) {
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

__global__ void __launch_bounds__(512) k_decode(const BlockDesc* __restrict__ blocks, uint32_t n_blocks,
                                                const DInput* __restrict__ in, const uint32_t* __restrict__ nrec,
                                                const uint16_t* __restrict__ hdr_tab,
                                                const uint32_t* __restrict__ rec_first,
                                                const uint64_t* __restrict__ key_first, Recs recs,
                                                uint8_t* __restrict__ arena, DErr* errs) {
  const uint32_t lane = lane_id();
  const uint64_t warps = gstride() / 32;
  for (uint64_t g = gtid() / 32; g < n_blocks; g += warps) {
    const BlockDesc b = blocks[g];
    DErr* e = errs + b.job;
    if (b.ptr == nullptr || *(volatile int32_t*)&e->code != 0) continue;
    const uint32_t nent = nrec[g];
    const uint64_t rec0 = rec_first[g], key0 = key_first[g];
    bool bad = false;
    bool tab = nent <= kHdrMax && b.size < 65536;
    // lane-per-entry header parse (entries lane and lane + 32)
    uint32_t sh[2] = {0, 0}, ns[2] = {0, 0}, kl[2] = {0, 0}, dp[2] = {0, 0};
    if (tab) {
      bool long_key = false;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k = lane + 32 * h;
        if (k < nent) {
          // the walk already validated this header (16-byte window read)
          const uint8_t* p = b.ptr + hdr_tab[g * kHdrMax + k];
          uint32_t f[3] = {0, 0, 0};
          p += read_header(p, b.ptr + b.size, f);
          sh[h] = f[0];
          ns[h] = f[1];
          kl[h] = f[0] + f[1];
          dp[h] = uint32_t(p - b.ptr);
          long_key |= kl[h] > 32 * kDecSlots;
          recs.vptr[rec0 + k] = reinterpret_cast<uint64_t>(p + f[1]);
          recs.vlen[rec0 + k] = f[2];
          recs.klen[rec0 + k] = kl[h];
          recs.src[rec0 + k] = b.input;
        }
      }
      tab = !__any_sync(0xFFFFFFFFu, long_key);
    }
    if (!tab) {
      if (lane == 0) decode_walk(b, rec0, key0, recs, arena, &bad);
      bad = __any_sync(0xFFFFFFFFu, bad);
      if (bad && lane == 0) report(e, E_CORRUPT, in[b.input].local, b.off);
      continue;
    }
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
    uint8_t cur[kDecSlots] = {0, 0, 0, 0};
    for (uint32_t k = 0; k < nent; ++k) {
      const uint32_t src = k & 31u, h = k >> 5;
      const uint32_t shared = __shfl_sync(0xFFFFFFFFu, h ? sh[1] : sh[0], src);
      const uint32_t klen = __shfl_sync(0xFFFFFFFFu, h ? kl[1] : kl[0], src);
      const uint32_t dpos = __shfl_sync(0xFFFFFFFFu, h ? dp[1] : dp[0], src);
      const uint32_t kof = __shfl_sync(0xFFFFFFFFu, h ? ko[1] : ko[0], src);
      uint8_t* kd = arena + key0 + kof;
#pragma unroll
      for (uint32_t s = 0; s < kDecSlots; ++s) {
        const uint32_t t = lane + 32 * s;
        if (t < klen) {
          if (t >= shared) cur[s] = b.ptr[dpos + t - shared];
          kd[t] = cur[s];
        }
      }
    }
    __syncwarp();  // the warp's key bytes are visible to all its lanes
    // per entry (lane): user-key prefix and trailer read back from the rebuilt key
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t k = lane + 32 * h;
      if (k < nent) {
        const uint8_t* kd = arena + key0 + ko[h];
        const uint32_t ul = kl[h] - 8;
        const uint64_t pf = key_word(kd, ul < 8 ? ul : 8u);
        const uint64_t tr = le_word(kd + ul);
        if ((tr & 0xFF) > 1) bad = true;
        recs.pfx[rec0 + k] = pf;
        recs.tr[rec0 + k] = tr;
        recs.koff[rec0 + k] = key0 + ko[h];
      }
    }
    bad = __any_sync(0xFFFFFFFFu, bad);
    if (bad && lane == 0) report(e, E_CORRUPT, in[b.input].local, b.off);
  }
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
                       uint64_t* kbytes, DErr* errs, Counts* cnt, uint16_t* hdr_tab, cudaStream_t st,
                       uint64_t* ulen, uint64_t* ures, bool contents) {
  if (!n_blocks) return;
  const unsigned t = tuning().walk_threads;
  k_block_walk<<<grid_for(n_blocks, t), t, 0, st>>>(blocks, n_blocks, in, nrec, kbytes, errs, cnt, hdr_tab, ulen,
                                                    ures, contents);
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
                       uint64_t* kbytes, DErr* errs, Counts* cnt, uint16_t* hdr_tab, CrcTabs tabs, cudaStream_t st) {
  launch_block_verify(blocks, n_blocks, in, errs, errs, tabs, &cnt->crc_next_in, false, st);
  launch_block_verify(blocks, n_blocks, in, errs, errs, tabs, &cnt->crc_next_in, true, st);
  launch_block_walk(blocks, n_blocks, in, nrec, kbytes, errs, cnt, hdr_tab, st);
}

void launch_decode(const BlockDesc* blocks, uint32_t n_blocks, const DInput* in, const uint32_t* nrec,
                   const uint16_t* hdr_tab, const uint32_t* rec_first, const uint64_t* key_first, Recs recs,
                   uint8_t* arena, DErr* errs, cudaStream_t st) {
  if (!n_blocks) return;
  const unsigned w = tuning().decode_warps;
  k_decode<<<grid_for(n_blocks, w), w * 32, 0, st>>>(blocks, n_blocks, in, nrec, hdr_tab, rec_first, key_first, recs,
                                                  arena, errs);
  count_launches(1);
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
