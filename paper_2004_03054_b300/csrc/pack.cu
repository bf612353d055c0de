// pack.cu -- Phase 3 "Pack" (LUDA §II-A; §III-C "shared_key", "encode" and "filter"
// kernels, Fig. 4b).
//
//   sizes      per survivor: shared prefix with its predecessor (the prefix-compressed key)
//              and its encoded size in delta form and in restart form
//   block cut  the greedy builder rule "close the block once its size estimate reaches
//              the block size" made parallel: next(i) (where a block starting at entry i
//              ends) for every i from prefix sums, then the chain 0, next(0), ... is
//              stitched tile by tile (speculate each tile's entry, fix mispredictions)
//   file cut   the same over blocks with the target file size
//   encode     one CTA per data block: headers, key deltas, values gathered straight from
//              the input tables, restart array, CRC trailer; no data exchange between
//              blocks (§III-C)
//   filter     per-table bloom bitmap built with atomics, then written with its trailer
//   index, metaindex, footer per table.
#include <cstdint>

#include "internal.cuh"

namespace luda {

namespace {

__device__ __forceinline__ uint32_t job_of_surv(const JobDev* jobs, uint32_t n_jobs, uint32_t s) {
  uint32_t lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jobs[mid].surv_begin <= s) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t job_of_block(const JobDev* jobs, uint32_t n_jobs, uint32_t b) {
  uint32_t lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jobs[mid].blk_begin <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_sizes(const uint32_t* __restrict__ surv, const Counts* __restrict__ cnt,
                        const JobDev* __restrict__ jobs, uint32_t n_jobs, Recs recs, const uint8_t* __restrict__ arena,
                        uint32_t* __restrict__ lcp, uint32_t* __restrict__ sd, uint32_t* __restrict__ dr,
                        EncDesc* __restrict__ ed) {
  const uint32_t n = cnt->n_surv;
  uint64_t kv = 0;
  for (uint64_t s = gtid(); s < n; s += gstride()) {
    const uint32_t j = job_of_surv(jobs, n_jobs, uint32_t(s));
    const uint32_t x = surv[s];
    const uint32_t klen = recs.klen[x], vlen = recs.vlen[x];
    uint32_t l = 0;
    if (s > jobs[j].surv_begin) {
      // common prefix of the two internal keys, 8 bytes at a time
      const uint32_t y = surv[s - 1];
      const uint32_t m = min(klen, recs.klen[y]);
      const uint8_t* a = arena + recs.koff[x];
      const uint8_t* b = arena + recs.koff[y];
      while (l < m) {
        const uint32_t avail = m - l < 8 ? m - l : 8u;
        const uint64_t d = key_word(a + l, avail) ^ key_word(b + l, avail);
        if (d) {
          l += uint32_t(__clzll(d)) >> 3;
          break;
        }
        l += avail;
      }
    }
    const uint32_t d = varint_size(l) + varint_size(klen - l) + varint_size(vlen) + (klen - l) + vlen;
    const uint32_t r = 1 + varint_size(klen) + varint_size(vlen) + klen + vlen;
    lcp[s] = l;
    sd[s] = d;
    dr[s] = r - d;
    ed[s] = EncDesc{reinterpret_cast<uint64_t>(arena + recs.koff[x]), recs.vptr[x], klen, vlen, x, 0u};
    kv += klen + vlen;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) kv += __shfl_xor_sync(0xFFFFFFFFu, kv, o);
  if ((threadIdx.x & 31u) == 0 && kv)
    atomicAdd(reinterpret_cast<unsigned long long*>(&const_cast<Counts*>(cnt)->surv_kv_bytes),
              (unsigned long long)kv);
}

// next(i) = 1 + min{j >= i : E(i, j) >= T}, capped at the job's end, with
// E(i, j) = P[j+1] - P[i] + sum of dr over the restarts i, i+R, ... <= j + 4*ceil((j-i+1)/R) + 4.
__global__ void k_block_next(const uint64_t* __restrict__ P, const uint32_t* __restrict__ dr,
                             const Counts* __restrict__ cnt, const JobDev* __restrict__ jobs, uint32_t n_jobs, Fmt fmt,
                             uint32_t* __restrict__ next) {
  const uint64_t T = fmt.T, R = fmt.R;
  const uint32_t n = cnt->n_surv;
  for (uint64_t i = gtid(); i < n; i += gstride()) {
    const uint64_t e = jobs[job_of_surv(jobs, n_jobs, uint32_t(i))].surv_end;
    const uint64_t base = P[i];
    uint64_t rs = 0;
    uint64_t res = e;
    for (uint64_t g = 0;; ++g) {
      const uint64_t gs = i + g * R;
      rs += dr[gs];
      const uint64_t ge = min(gs + R, e) - 1;
      const uint64_t fixed = rs + 4 * (g + 1) + 4 - base;
      if (P[ge + 1] + fixed >= T) {
        uint64_t j = gs;
        while (P[j + 1] + fixed < T) ++j;
        res = j + 1;
        break;
      }
      if (ge + 1 >= e) break;
    }
    next[i] = uint32_t(res);
  }
}

// ---- chain stitching --------------------------------------------------------------------
// The cut points are the chain 0, next(0), next(next(0)), ... over a next[] array with
// next(i) > i, capped at each job's end (so every job start is on the chain). Exact and
// parallel without any convergence assumption:
//   window path (largest step G = max(next(i) - i) <= kWinMax): the first chain node of
//     tile t lies in [L_t, L_t + G). Each tile walks its chain from every one of those W
//     candidates (one thread each, tile's next[] in shared memory) and records where it
//     leaves the tile; one CTA then composes the tiles in order with table lookups in
//     shared memory; finally every tile marks its chain from its true entry.
//   walk path (G > kWinMax, e.g. the file cut over blocks): the chain is walked per job,
//     jobs in parallel; such chains have few nodes.
constexpr uint32_t kStitchTile = 2048;
constexpr uint32_t kWinMax = 256;

__device__ __forceinline__ uint32_t win_of(uint32_t gap) { return max(32u, (gap + 31u) & ~31u); }

__global__ void __launch_bounds__(256) k_max_gap(const uint32_t* __restrict__ next, const uint32_t* __restrict__ n_dev,
                                                 uint32_t* __restrict__ gap) {
  __shared__ uint32_t s_max[8];
  const uint32_t n = *n_dev;
  uint32_t g = 0;
  for (uint64_t i = gtid(); i < n; i += gstride()) g = max(g, next[i] - uint32_t(i));
  g = __reduce_max_sync(0xFFFFFFFFu, g);
  if ((threadIdx.x & 31u) == 0) s_max[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x < 32) {
    g = threadIdx.x < 8 ? s_max[threadIdx.x] : 0u;
    g = __reduce_max_sync(0xFFFFFFFFu, g);
    if (threadIdx.x == 0 && g) atomicMax(gap, g);
  }
}

__global__ void __launch_bounds__(256) k_stitch_win(const uint32_t* __restrict__ next,
                                                    const uint32_t* __restrict__ n_dev,
                                                    const uint32_t* __restrict__ gap,
                                                    uint32_t* __restrict__ exitw) {
  __shared__ uint32_t s_next[kStitchTile];
  if (*gap > kWinMax) return;
  const uint32_t n = *n_dev, W = win_of(*gap);
  const uint32_t n_tiles = (n + kStitchTile - 1) / kStitchTile;
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint32_t L = t * kStitchTile, U = min(n, L + kStitchTile);
    for (uint32_t i = threadIdx.x; i < U - L; i += blockDim.x) s_next[i] = next[L + i];
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < W; k += blockDim.x) {
      uint32_t x = L + k;
      while (x < U) x = s_next[x - L];
      exitw[uint64_t(t) * kWinMax + k] = x;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_stitch_combine(const uint32_t* __restrict__ exitw,
                                                        const uint32_t* __restrict__ n_dev,
                                                        const uint32_t* __restrict__ gap,
                                                        uint32_t* __restrict__ entry,
                                                        const uint32_t* __restrict__ done) {
  constexpr uint32_t kWords = 12000;  // rows held in shared memory
  __shared__ uint32_t s_rows[kWords];
  __shared__ uint32_t s_cur;
  if (*gap > kWinMax || *done) return;
  const uint32_t n = *n_dev, W = win_of(*gap);
  const uint32_t n_tiles = (n + kStitchTile - 1) / kStitchTile;
  const uint32_t per = kWords / W;
  if (threadIdx.x == 0) s_cur = 0;
  for (uint32_t t0 = 0; t0 < n_tiles; t0 += per) {
    const uint32_t tn = min(per, n_tiles - t0);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tn * W; i += blockDim.x) {
      const uint32_t r = i / W, k = i - r * W;
      s_rows[i] = exitw[uint64_t(t0 + r) * kWinMax + k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t c = s_cur;
      for (uint32_t r = 0; r < tn; ++r) {
        const uint32_t L = (t0 + r) * kStitchTile;
        entry[t0 + r] = c;
        if (c < n) c = s_rows[r * W + (c - L)];
      }
      s_cur = c;
    }
  }
}

// Parallel composition of the tiles (when all W-entry tables fit in shared memory): tile
// t's table f_t maps the chain's entry offset in tile t to its entry offset in tile t + 1
// (W: the chain has ended). Doubling (Hillis-Steele over function composition) turns
// f_t into f_t o f_{t-1} o ... o f_0 in log2(tiles) rounds; tile t's entry is then
// f_{t-1} o ... o f_0 applied to offset 0. Falls back to the sequential walk (all threads
// return without writing, k_stitch_combine runs) when the tables do not fit.
constexpr uint32_t kCombWords = 24576;
constexpr uint32_t kCombSmem = 2 * kCombWords * 4;

__global__ void __launch_bounds__(1024) k_stitch_compose(const uint32_t* __restrict__ exitw,
                                                         const uint32_t* __restrict__ n_dev,
                                                         const uint32_t* __restrict__ gap,
                                                         uint32_t* __restrict__ entry,
                                                         uint32_t* __restrict__ done) {
  extern __shared__ uint32_t s_comp[];
  if (*gap > kWinMax) return;
  const uint32_t n = *n_dev, W = win_of(*gap);
  const uint32_t n_tiles = (n + kStitchTile - 1) / kStitchTile;
  if (uint64_t(n_tiles) * W > kCombWords) {
    if (threadIdx.x == 0) *done = 0;
    return;
  }
  uint32_t* A = s_comp;
  uint32_t* B = s_comp + kCombWords;
  for (uint32_t i = threadIdx.x; i < n_tiles * W; i += blockDim.x) {
    const uint32_t t = i / W, k = i - t * W;
    const uint32_t x = exitw[uint64_t(t) * kWinMax + k];
    const uint32_t next_l = (t + 1) * kStitchTile;
    A[i] = x < n ? x - next_l : W;  // offset in tile t + 1, or W: ended
  }
  __syncthreads();
  for (uint32_t d = 1; d < n_tiles; d <<= 1) {
    for (uint32_t i = threadIdx.x; i < n_tiles * W; i += blockDim.x) {
      const uint32_t t = i / W;
      if (t < d) {
        B[i] = A[i];
      } else {
        const uint32_t v = A[(t - d) * W + (i - t * W)];  // through tiles t-2d+1 .. t-d
        B[i] = v < W ? A[t * W + v] : W;
      }
    }
    __syncthreads();
    uint32_t* tmp = A;
    A = B;
    B = tmp;
  }
  for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    if (t == 0) {
      entry[0] = 0;
    } else {
      const uint32_t v = A[(t - 1) * W];
      entry[t] = v < W ? t * kStitchTile + v : n;
    }
  }
  if (threadIdx.x == 0) *done = 1;
}

__global__ void __launch_bounds__(128) k_stitch_mark(const uint32_t* __restrict__ next,
                                                     const uint32_t* __restrict__ n_dev,
                                                     const uint32_t* __restrict__ gap,
                                                     const uint32_t* __restrict__ entry,
                                                     uint8_t* __restrict__ flags) {
  __shared__ uint32_t s_next[kStitchTile];
  __shared__ uint8_t s_flag[kStitchTile];
  if (*gap > kWinMax) return;
  const uint32_t n = *n_dev;
  const uint32_t n_tiles = (n + kStitchTile - 1) / kStitchTile;
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint32_t L = t * kStitchTile, U = min(n, L + kStitchTile);
    for (uint32_t i = threadIdx.x; i < U - L; i += blockDim.x) {
      s_next[i] = next[L + i];
      s_flag[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t x = entry[t];
      while (x < U) {
        s_flag[x - L] = 1;
        x = s_next[x - L];
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < U - L; i += blockDim.x) flags[L + i] = s_flag[i];
    __syncthreads();
  }
}

// Walk path: one warp per job; lane 0 follows the chain over global next[].
__global__ void k_stitch_walk(const uint32_t* __restrict__ next, const uint32_t* __restrict__ gap,
                              const JobDev* __restrict__ jobs, uint32_t n_jobs, bool blocks_level,
                              uint8_t* __restrict__ flags) {
  if (*gap <= kWinMax) return;
  const uint64_t warps = gstride() / 32;
  for (uint64_t j = gtid() / 32; j < n_jobs; j += warps) {
    const uint32_t b = blocks_level ? jobs[j].blk_begin : jobs[j].surv_begin;
    const uint32_t e = blocks_level ? jobs[j].blk_end : jobs[j].surv_end;
    if (lane_id() == 0) {  // flags were cleared by the caller
      uint32_t x = b;
      while (x < e) {
        flags[x] = 1;
        x = next[x];
      }
    }
  }
}

// starts[pos[i]] = i for flagged i, starts[total] = n; *total_out = total.
__global__ void k_compact_flags(const uint8_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                                const uint32_t* __restrict__ n_dev, uint32_t* __restrict__ starts,
                                uint32_t* __restrict__ total_out) {
  const uint32_t n = *n_dev;
  for (uint64_t i = gtid(); i < n; i += gstride())
    if (flags[i]) starts[pos[i]] = uint32_t(i);
  if (gtid() == 0) {
    starts[pos[n]] = n;
    *total_out = pos[n];
  }
}

__global__ void k_job_blocks(JobDev* jobs, uint32_t n_jobs, const uint32_t* __restrict__ bpos) {
  for (uint64_t j = gtid(); j < n_jobs; j += gstride()) {
    jobs[j].blk_begin = bpos[jobs[j].surv_begin];
    jobs[j].blk_end = bpos[jobs[j].surv_end];
  }
}

__global__ void k_job_files(JobDev* jobs, uint32_t n_jobs, const uint32_t* __restrict__ fpos) {
  for (uint64_t j = gtid(); j < n_jobs; j += gstride()) {
    jobs[j].file_begin = fpos[jobs[j].blk_begin];
    jobs[j].file_end = fpos[jobs[j].blk_end];
  }
}

// Contents size of block [s, e): exact, equal to the builder's estimate at its close.
__global__ void k_block_sizes(const uint32_t* __restrict__ start, const Counts* __restrict__ cnt,
                              const uint64_t* __restrict__ P, const uint32_t* __restrict__ dr, Fmt fmt,
                              uint64_t* __restrict__ bsz, uint64_t* __restrict__ disk) {
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) {
    const uint32_t s = start[b], e = start[b + 1];
    uint64_t sz = P[e] - P[s];
    uint64_t nr = 0;
    for (uint64_t k = s; k < e; k += fmt.R, ++nr) sz += dr[k];
    sz += 4 * nr + 4;
    bsz[b] = sz;
    disk[b] = sz + kTrailer;
  }
}

// File cut: a table ends after the block that brings its data bytes to >= target.
__global__ void k_file_next(const uint64_t* __restrict__ C, const Counts* __restrict__ cnt,
                            const JobDev* __restrict__ jobs, uint32_t n_jobs, Fmt fmt, uint32_t* __restrict__ next) {
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) {
    const uint32_t be = jobs[job_of_block(jobs, n_jobs, uint32_t(b))].blk_end;
    const uint64_t base = C[b];
    uint32_t lo = uint32_t(b), hi = be;  // first b' in [b, be) with C[b'+1] - base >= target
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (C[mid + 1] - base >= fmt.target) hi = mid;
      else lo = mid + 1;
    }
    next[b] = lo < be ? lo + 1 : be;
  }
}

__global__ void k_block_file(const uint32_t* __restrict__ fpos, const Counts* __restrict__ cnt,
                             uint32_t* __restrict__ blk_file) {
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) blk_file[b] = fpos[b + 1] - 1;
}

// R9s: the length L of block b's shortened index user key (its bytes are a[0..L-1) and
// a[L-1] + 1, then the trailer of the largest sequence number with type put), or 0 when
// the block keeps its full last key. a = user key of the block's last key (ua bytes); nb =
// user key of the next block's first key in the same table (ub bytes), or nullptr for the
// table's last block. The first differing byte is found 8 bytes at a time.
__device__ uint32_t short_index_len(const uint8_t* a, uint32_t ua, const uint8_t* nb, uint32_t ub) {
  if (nb) {
    const uint32_t m = ua < ub ? ua : ub;
    uint32_t d = m;
    for (uint32_t i = 0; i < m; i += 8) {
      const uint32_t avail = m - i < 8 ? m - i : 8u;
      const uint64_t x = key_word(a + i, avail) ^ key_word(nb + i, avail);
      if (x) {
        d = i + (uint32_t(__clzll(x)) >> 3);
        break;
      }
    }
    return d < m && uint32_t(a[d]) + 1 < uint32_t(nb[d]) && d + 1 < ua ? d + 1 : 0u;
  }
  uint32_t d = 0;
  while (d < ua && a[d] == 0xFF) ++d;
  return d + 1 < ua ? d + 1 : 0u;
}

// Index key of block b: its length, and (with dst) its bytes.
__device__ __forceinline__ uint32_t index_key_of(uint64_t b, uint32_t fb1, const uint32_t* __restrict__ start,
                                                 const uint32_t* __restrict__ surv, const Recs& recs,
                                                 const uint8_t* __restrict__ arena, uint32_t flags, uint8_t* dst) {
  const uint32_t x = surv[start[b + 1] - 1];
  const uint32_t klen = recs.klen[x];
  const uint8_t* k = arena + recs.koff[x];
  uint32_t L = 0;
  if (flags & LUDA_F_SHORT_INDEX) {
    const uint8_t* nk = nullptr;
    uint32_t nl = 0;
    if (b + 1 < fb1) {
      const uint32_t y = surv[start[b + 1]];
      nk = arena + recs.koff[y];
      nl = recs.klen[y] - 8;
    }
    L = short_index_len(k, klen - 8, nk, nl);
  }
  if (!L) {
    if (dst)
      for (uint32_t t = 0; t < klen; ++t) dst[t] = k[t];
    return klen;
  }
  if (dst) {
    for (uint32_t t = 0; t + 1 < L; ++t) dst[t] = k[t];
    dst[L - 1] = uint8_t(k[L - 1] + 1);
    dst[L] = 1;  // trailer (2^56 - 1) << 8 | 1, little-endian
    for (uint32_t t = 1; t < 8; ++t) dst[L + t] = 0xFF;
  }
  return L + 8;
}

__global__ void k_index_sizes(const uint32_t* __restrict__ start, const uint64_t* __restrict__ bsz,
                              const uint64_t* __restrict__ C, const uint32_t* __restrict__ blk_file,
                              const uint32_t* __restrict__ file_start, const Counts* __restrict__ cnt,
                              const uint32_t* __restrict__ surv, Recs recs, const uint8_t* __restrict__ arena,
                              uint32_t flags, uint32_t* __restrict__ ie) {
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) {
    const uint32_t f = blk_file[b];
    const uint32_t fb0 = file_start[f], fb1 = file_start[f + 1];
    const uint64_t off = C[b] - C[fb0];
    const uint32_t klen = index_key_of(b, fb1, start, surv, recs, arena, flags, nullptr);
    const uint32_t hlen = varint_size(off) + varint_size(bsz[b]);
    ie[b] = 1 + varint_size(klen) + varint_size(hlen) + klen + hlen;
  }
}

// Largest i in [0, n) with a[i] <= v (a ascending, a[0] <= v).
template <typename T>
__device__ __forceinline__ uint32_t last_le(const T* __restrict__ a, uint32_t n, T v) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---- filter array (R10a) ----------------------------------------------------------------
// Filters of table f: max(D >> 11, (o_last >> 11) + 1), D = end of its data blocks, o_last =
// offset of its last data block.
__global__ void k_filter_count(const uint32_t* __restrict__ file_start, const Counts* __restrict__ cnt,
                               const uint64_t* __restrict__ C, uint64_t* __restrict__ nfilt) {
  const uint32_t nf = cnt->nf;
  for (uint64_t f = gtid(); f < nf; f += gstride()) {
    const uint32_t fb0 = file_start[f], fb1 = file_start[f + 1];
    const uint64_t a = (C[fb1] - C[fb0]) >> kFilterBaseLg, b = ((C[fb1 - 1] - C[fb0]) >> kFilterBaseLg) + 1;
    nfilt[f] = a > b ? a : b;
  }
}

// One thread per filter: the entries of the table's blocks that start in the filter's
// window (blocks are in offset order, so a range found by two binary searches), its bytes
// (bitmap and k; none when empty) and bitmap words. Filters past slot_cap are left to the
// capacity check of k_file_offsets.
__global__ void k_filter_sizes(const uint64_t* __restrict__ fbase, const uint32_t* __restrict__ file_start,
                               const uint32_t* __restrict__ start, const uint64_t* __restrict__ C, Counts* cnt,
                               uint64_t slot_cap, Fmt fmt, uint64_t* __restrict__ fbytes,
                               uint64_t* __restrict__ fwords) {
  const uint32_t nf = cnt->nf;
  const uint64_t total = fbase[nf], n = total < slot_cap ? total : slot_cap;
  if (gtid() == 0) cnt->n_filt = uint32_t(n);
  for (uint64_t s = gtid(); s < n; s += gstride()) {
    const uint32_t f = last_le<uint64_t>(fbase, nf, s);
    const uint32_t fb0 = file_start[f], fb1 = file_start[f + 1];
    const uint64_t w0 = C[fb0] + ((s - fbase[f]) << kFilterBaseLg), w1 = w0 + (1ull << kFilterBaseLg);
    uint32_t lo = fb0, hi = fb1;  // first block at or after w0
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (C[mid] < w0) lo = mid + 1;
      else hi = mid;
    }
    uint32_t lo2 = lo, hi2 = fb1;  // first block at or after w1
    while (lo2 < hi2) {
      const uint32_t mid = (lo2 + hi2) >> 1;
      if (C[mid] < w1) lo2 = mid + 1;
      else hi2 = mid;
    }
    const uint64_t keys = start[lo2] - start[lo];
    uint64_t bits = keys * fmt.bpk;
    if (bits < 64) bits = 64;
    const uint64_t bytes = keys ? (bits + 7) / 8 : 0;
    fbytes[s] = keys ? bytes + 1 : 0;
    fwords[s] = (bytes + 3) / 4;
  }
}

__global__ void k_file_layout(const uint32_t* __restrict__ file_start, const Counts* __restrict__ cnt,
                              const uint32_t* __restrict__ start,
                              const uint64_t* __restrict__ C, const uint64_t* __restrict__ IX, Fmt fmt,
                              FiltArr fa, const JobDev* __restrict__ jobs, uint32_t n_jobs,
                              FileDesc* __restrict__ files, uint64_t* __restrict__ fsize,
                              uint64_t* __restrict__ bmwords) {
  const uint32_t nf = cnt->nf;
  const bool fits = fa.base && fa.base[nf] <= fa.cap;
  for (uint64_t f = gtid(); f < nf; f += gstride()) {
    const uint32_t fb0 = file_start[f], fb1 = file_start[f + 1];
    const uint32_t e0 = start[fb0], e1 = start[fb1];
    FileDesc d{};
    d.blk_begin = fb0;
    d.blk_end = fb1;
    d.ent_begin = e0;
    d.ent_end = e1;
    d.job = job_of_block(jobs, n_jobs, fb0);
    d.data_size = C[fb1] - C[fb0];
    uint64_t words;
    if (fa.base) {
      // filter array: the filters, their u32 offsets, the array's offset, base_lg
      const uint64_t s0 = fits ? fa.base[f] : 0, s1 = fits ? fa.base[f + 1] : 0;
      d.n_filt = uint32_t(s1 - s0);
      d.filter_size = (fa.boff[s1] - fa.boff[s0]) + 4 * (s1 - s0) + 5;
      words = fa.woff[s1] - fa.woff[s0];
    } else {
      uint64_t bits = uint64_t(e1 - e0) * fmt.bpk;
      if (bits < 64) bits = 64;
      const uint64_t bytes = (bits + 7) / 8;
      d.bm_bits = bytes * 8;
      d.filter_size = bytes + 1;
      words = (bytes + 3) / 4;
    }
    const uint32_t hf = varint_size(d.data_size) + varint_size(d.filter_size);
    d.meta_size = 3 + (fa.base ? 19 : 17) + hf + 8;
    d.meta_off = d.data_size + d.filter_size + kTrailer;
    d.index_size = (IX[fb1] - IX[fb0]) + 4ull * (fb1 - fb0) + 4;
    d.index_off = d.meta_off + d.meta_size + kTrailer;
    d.size = d.index_off + d.index_size + kTrailer + kFooter;
    files[f] = d;
    fsize[f] = d.size;
    bmwords[f] = words;
  }
}

__global__ void k_file_offsets(FileDesc* files, Counts* cnt, const uint64_t* __restrict__ foff,
                               const uint64_t* __restrict__ bmoff, FiltArr fa, JobDev* jobs, uint32_t n_jobs,
                               uint64_t out_cap, uint64_t bm_cap, DErr* errs) {
  const uint32_t nf = cnt->nf;
  for (uint64_t f = gtid(); f < nf; f += gstride()) {
    files[f].off = foff[f];
    files[f].bm_word = bmoff[f];
  }
  for (uint64_t j = gtid(); j < n_jobs; j += gstride()) {
    jobs[j].out_bytes = foff[jobs[j].file_end] - foff[jobs[j].file_begin];
    if (foff[nf] > out_cap || bmoff[nf] > bm_cap || (fa.base && fa.base[nf] > fa.cap))
      report(errs + j, E_OOM, ~0u, foff[nf]);
  }
  if (gtid() == 0) {
    cnt->out_bytes = foff[nf];
    cnt->bm_words = bmoff[nf];
  }
}

__global__ void k_zero_words(uint32_t* __restrict__ w, const Counts* __restrict__ cnt, uint64_t cap) {
  const uint64_t n = cnt->bm_words < cap ? cnt->bm_words : cap;
  for (uint64_t i = gtid(); i < n; i += gstride()) w[i] = 0;
}

// ---- encode -------------------------------------------------------------------------------
// One CTA per data block. The block image is assembled in shared memory at the same
// 16-byte phase as its destination, so the final store is whole aligned 16-byte words
// (bytes only at the two ragged ends). Values are gathered from the input tables with
// aligned 4-byte loads joined by funnel shifts; the CRC trailer is computed by the whole
// CTA from shared memory. A block larger than the shared buffer is written straight to
// global memory instead (same bytes).
constexpr int kEncThreads = 256;
constexpr uint32_t kEncBuf = 64 * 1024;

// Copy n bytes from global src (any alignment) to dst (any alignment), one warp.
__device__ __forceinline__ void warp_copy(uint8_t* dst, const uint8_t* src, uint32_t n, uint32_t lane) {
  uint32_t head = (4u - (uint32_t(reinterpret_cast<uintptr_t>(dst)) & 3u)) & 3u;
  if (head > n) head = n;
  if (lane < head) dst[lane] = src[lane];
  const uint32_t nw = (n - head) >> 2;
  const uint8_t* s = src + head;
  uint32_t* d = reinterpret_cast<uint32_t*>(dst + head);
  const uint32_t sh = (uint32_t(reinterpret_cast<uintptr_t>(s)) & 3u) * 8u;
  const uint32_t* sa = reinterpret_cast<const uint32_t*>(reinterpret_cast<uintptr_t>(s) & ~uintptr_t(3));
  if (sh == 0) {
    for (uint32_t k = lane; k < nw; k += 32) d[k] = __ldg(sa + k);
  } else {
    for (uint32_t k = lane; k < nw; k += 32) d[k] = __funnelshift_r(__ldg(sa + k), __ldg(sa + k + 1), sh);
  }
  const uint32_t done = head + 4 * nw;
  if (lane < n - done) dst[done + lane] = src[done + lane];
}

__global__ void __launch_bounds__(kEncThreads) k_encode_big(const uint32_t* __restrict__ start,
                                                        const Counts* __restrict__ cnt,
                                                        const uint32_t* __restrict__ blk_file,
                                                        const FileDesc* __restrict__ files,
                                                        const uint64_t* __restrict__ C, const uint64_t* __restrict__ bsz,
                                                        const uint32_t* __restrict__ surv,
                                                        const uint32_t* __restrict__ lcp,
                                                        const uint32_t* __restrict__ sd,
                                                        const uint32_t* __restrict__ dr, Recs recs,
                                                        const uint8_t* __restrict__ arena, Fmt fmt,
                                                        uint8_t* __restrict__ out, uint64_t out_cap,
                                                        const uint32_t* __restrict__ big, CrcTabs tabs) {
  if (blockIdx.x >= cnt->big_blocks) return;
  extern __shared__ uint4 s_dyn[];
  __shared__ uint32_t sT[1024];
  __shared__ uint32_t s_off[kEncThreads];
  __shared__ uint32_t s_wsum[kEncThreads / 32];
  __shared__ uint32_t s_scratch[kEncThreads / 32];
  load_slice_table(sT, tabs);
  __syncthreads();
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  constexpr uint32_t nwarps = kEncThreads / 32;
  const uint32_t R = fmt.R;
  const uint32_t n_big = cnt->big_blocks;
  for (uint32_t i = blockIdx.x; i < n_big; i += gridDim.x) {
    const uint32_t b = big[i];
    const uint32_t s = start[b], e = start[b + 1], m = e - s;
    const FileDesc F = files[blk_file[b]];
    if (F.off + F.size > out_cap) continue;
    uint8_t* dst = out + F.off + (C[b] - C[F.blk_begin]);
    const uint64_t contents = bsz[b];
    const uint32_t nr = (m + R - 1) / R;
    const uint64_t rbase = contents - 4ull * nr - 4;
    const uint32_t phase = uint32_t(reinterpret_cast<uintptr_t>(dst) & 15u);
    const bool in_smem = contents + kTrailer + 16 <= kEncBuf;
    uint8_t* img = in_smem ? reinterpret_cast<uint8_t*>(s_dyn) + phase : dst;
    uint32_t base = 0;
    for (uint32_t r0 = 0; r0 < m; r0 += kEncThreads) {
      const uint32_t k = r0 + tid;
      uint32_t sz = 0;
      if (k < m) sz = sd[s + k] + ((k % R) == 0 ? dr[s + k] : 0u);
      uint32_t x = sz;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= uint32_t(d)) x += o;
      }
      if (lane == 31) s_wsum[warp] = x;
      __syncthreads();
      uint32_t before = 0, total = 0;
#pragma unroll
      for (uint32_t w = 0; w < nwarps; ++w) {
        const uint32_t v = s_wsum[w];
        before += w < warp ? v : 0u;
        total += v;
      }
      s_off[tid] = base + before + x - sz;
      __syncthreads();
      const uint32_t cnt_r = min(uint32_t(kEncThreads), m - r0);
      for (uint32_t kk = warp; kk < cnt_r; kk += nwarps) {
        const uint32_t kb = r0 + kk;
        const uint32_t xi = surv[s + kb];
        const uint32_t klen = recs.klen[xi], vlen = recs.vlen[xi];
        const bool restart = (kb % R) == 0;
        const uint32_t shared = restart ? 0u : lcp[s + kb];
        const uint32_t nonshared = klen - shared;
        const uint32_t eoff = s_off[kk];
        uint8_t* ep = img + eoff;
        const uint32_t h = varint_size(shared) + varint_size(nonshared) + varint_size(vlen);
        if (lane == 0) {
          uint32_t q = put_varint(ep, shared);
          q += put_varint(ep + q, nonshared);
          put_varint(ep + q, vlen);
          if (restart) st_u32(img + rbase + 4ull * (kb / R), eoff);
        }
        const uint8_t* ks = arena + recs.koff[xi] + shared;
        for (uint32_t t = lane; t < nonshared; t += 32) ep[h + t] = ks[t];
        warp_copy(ep + h + nonshared, reinterpret_cast<const uint8_t*>(recs.vptr[xi]), vlen, lane);
      }
      base += total;
      __syncthreads();
    }
    if (tid == 0) {
      st_u32(img + contents - 4, nr);
      img[contents] = 0;
    }
    __syncthreads();
    const uint32_t crc = cta_crc32c(img, contents + 1, sT, tabs, s_scratch);
    if (tid == 0) st_u32(img + contents + 1, crc_mask(crc));
    __syncthreads();
    if (in_smem) {
      // aligned 16-byte words of [dst, dst + len) at the same phase in shared memory
      const uint64_t len = contents + kTrailer;
      const uint64_t nq = (phase + len + 15) >> 4;
      uint4* gq = reinterpret_cast<uint4*>(dst - phase);
      for (uint64_t q = tid; q < nq; q += kEncThreads) {
        const uint64_t lo = q * 16, hi = lo + 16;
        if (lo >= phase && hi <= phase + len) {
          gq[q] = s_dyn[q];
        } else {
          const uint8_t* sb = reinterpret_cast<const uint8_t*>(s_dyn);
          uint8_t* gb = dst - phase;
          for (uint64_t i = lo; i < hi; ++i)
            if (i >= phase && i < phase + len) gb[i] = sb[i];
        }
      }
      __syncthreads();
    }
  }
}


// ---- staged encoder (TMA) -------------------------------------------------------------------
// A CTA encodes data blocks b = blockIdx.x, + gridDim.x, ... with one producer warp and
// kStgConsumers consumer warps, two staging slots in flight:
//   producer: one lane per entry reads the survivor's descriptor (survivor order,
//     coalesced) and its shared-prefix length; a warp scan places every entry in the block
//     and in the slot's staging buffer; each entry's key delta and value are fetched into
//     the staging buffer by bulk asynchronous copies (cp.async.bulk, completion counted
//     in bytes on the slot's "full" mbarrier) as whole aligned 16-byte ranges. It refills
//     a slot once the consumers release it on the slot's "empty" mbarrier.
//   consumers: assemble the block image in shared memory at its destination's 16-byte
//     phase: headers, key deltas, value edges, restart array and type byte bytewise; every
//     16-byte image word inside one value comes from the staging buffer with funnel
//     shifts (one warp per entry). The aligned middle of the image leaves in one bulk
//     store (cp.async.bulk shared -> global); the ragged ends with byte stores.
// Blocks with more than kStgMaxEnt entries or larger than the buffers go to k_encode_big.
// The CRC trailer is assembled afterwards by k_block_trailer.
constexpr uint32_t kStgConsumers = 8;
constexpr uint32_t kStgThreads = 32 * (kStgConsumers + 1);
constexpr uint32_t kStgCons = 32 * kStgConsumers;  // consumer threads
constexpr uint32_t kStgMaxEnt = 128;

struct StgEnt {
  uint32_t eoff;  // entry offset in the block
  uint32_t shr, nsh, vlen;
  uint32_t ks;    // staging offset of the key delta's first byte
  uint32_t vs;    // staging offset of the value's first byte
  uint32_t vb;    // block offset of the value's first byte
  uint32_t pad;
};

struct StgInfo {     // one slot's block, written by the producer before "full" completes
  uint64_t dst;      // block start in the output
  uint32_t b, m;
  uint32_t contents, phase;
  uint32_t state;    // 1 staged, 2 nothing to do (sent to k_encode_big or out of range)
  uint32_t pad;
};

// shared memory: 4 mbarriers | 2 StgInfo | entries [2][kStgMaxEnt] | sources [2][kStgMaxEnt]
constexpr uint32_t kStgOffInfo = 32;
constexpr uint32_t kStgOffEnt = kStgOffInfo + 2 * 32;
constexpr uint32_t kStgOffSrc = kStgOffEnt + 2 * kStgMaxEnt * 32;
constexpr uint32_t kStgHead = kStgOffSrc + 2 * kStgMaxEnt * 16;

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity: false once limit_ns have passed. A
// zero limit gives up without looking at the barrier (the test-only LUDA_F_TEST_WAIT0).
constexpr uint64_t kWaitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (limit_ns == 0) return false;
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(a, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bytes [sh, sh + 16) of the 32 bytes a || b, with selects (no divergent branches).
__device__ __forceinline__ uint4 shift32(uint4 a, uint4 b, uint32_t sh) {
  const bool s2 = (sh & 8u) != 0, s1 = (sh & 4u) != 0;
  const uint32_t x0 = s2 ? a.z : a.x, x1 = s2 ? a.w : a.y, x2 = s2 ? b.x : a.z;
  const uint32_t x3 = s2 ? b.y : a.w, x4 = s2 ? b.z : b.x, x5 = s2 ? b.w : b.y;
  const uint32_t y0 = s1 ? x1 : x0, y1 = s1 ? x2 : x1, y2 = s1 ? x3 : x2, y3 = s1 ? x4 : x3, y4 = s1 ? x5 : x4;
  const uint32_t bs = (sh & 3u) * 8u;
  return make_uint4(__funnelshift_r(y0, y1, bs), __funnelshift_r(y1, y2, bs), __funnelshift_r(y2, y3, bs),
                    __funnelshift_r(y3, y4, bs));
}

__device__ __forceinline__ uint32_t hdr_len(uint32_t shr, uint32_t nsh, uint32_t vlen) {
  return varint_size(shr) + varint_size(nsh) + varint_size(vlen);
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kStgCons) : "memory"); }
// Barrier of the consumer threads that also ANDs a predicate across them.
__device__ __forceinline__ bool consumers_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"(uint32_t(v)), "n"(kStgCons)
      : "memory");
  return r != 0;
}

// Per block: destination offset, entries and size for the encoder (one thread per block).
__global__ void k_block_enc(const uint32_t* __restrict__ start, const Counts* __restrict__ cnt,
                            const uint32_t* __restrict__ blk_file, const FileDesc* __restrict__ files,
                            const uint64_t* __restrict__ C, const uint64_t* __restrict__ bsz, uint64_t out_cap,
                            BlkEnc* __restrict__ bd) {
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) {
    const FileDesc F = files[blk_file[b]];
    BlkEnc d;
    d.dst = F.off + (C[b] - C[F.blk_begin]);
    d.s0 = start[b];
    d.m = start[b + 1] - d.s0;
    d.contents = uint32_t(bsz[b]);
    d.job = F.job | (F.off + F.size > out_cap ? 0x80000000u : 0u);
    bd[b] = d;
  }
}

__global__ void __launch_bounds__(kStgThreads) k_encode_stg(Counts* __restrict__ cnt,
                                                            const BlkEnc* __restrict__ bd,
                                                            const uint32_t* __restrict__ lcp,
                                                            const EncDesc* __restrict__ ed, Fmt fmt,
                                                            uint8_t* __restrict__ out, uint64_t out_cap,
                                                            uint8_t* __restrict__ done, uint32_t* __restrict__ big,
                                                            DErr* errs, uint32_t S, uint32_t I) {
  extern __shared__ __align__(128) uint8_t s_stg[];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t sbase = smem_addr(s_stg);
  // mbarriers: full[0], full[1], empty[0], empty[1]
  auto full = [&](uint32_t sl) { return sbase + 8 * sl; };
  auto empty = [&](uint32_t sl) { return sbase + 16 + 8 * sl; };
  StgInfo* info = reinterpret_cast<StgInfo*>(s_stg + kStgOffInfo);
  StgEnt* ents = reinterpret_cast<StgEnt*>(s_stg + kStgOffEnt);
  uint64_t* srcs = reinterpret_cast<uint64_t*>(s_stg + kStgOffSrc);
  uint8_t* stage = s_stg + ((kStgHead + 127) & ~127u);  // [2][S]
  uint8_t* img = stage + 2 * size_t(S);                  // [I + 16]
  const uint32_t stage_a = smem_addr(stage), img_a = smem_addr(img);
  const uint32_t R = fmt.R;
  // limit of the waits for a copy slot; the drain at the end always allows kWaitNs
  const uint64_t slot_wait_ns = (fmt.flags & LUDA_F_TEST_WAIT0) ? 0 : kWaitNs;
  const uint32_t nb = cnt->nb;
  if (tid == 0) {
    mbar_init(full(0), 1);
    mbar_init(full(1), 1);
    mbar_init(empty(0), 1);
    mbar_init(empty(1), 1);
    fence_proxy_async();
  }
  __syncthreads();

  __shared__ uint32_t s_fills[2], s_used[2];
  if (warp == 0) {
    // ---------------- producer ----------------
    uint32_t j = 0;
    BlkEnc pre{};  // lane l holds the descriptor of block b + l * gridDim.x of the current batch of 32
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x, ++j) {
      const uint32_t sl = j & 1u;
      if ((j & 31u) == 0) {
        const uint64_t bl = uint64_t(b) + uint64_t(lane) * gridDim.x;
        if (bl < nb) pre = bd[bl];
      }
      const uint32_t src_lane = j & 31u;
      BlkEnc D;
      D.dst = __shfl_sync(0xFFFFFFFFu, pre.dst, src_lane);
      D.s0 = __shfl_sync(0xFFFFFFFFu, pre.s0, src_lane);
      D.m = __shfl_sync(0xFFFFFFFFu, pre.m, src_lane);
      D.contents = __shfl_sync(0xFFFFFFFFu, pre.contents, src_lane);
      D.job = __shfl_sync(0xFFFFFFFFu, pre.job, src_lane);
      // the block's first 32 entry descriptors start loading before the slot is free
      EncDesc pd{};
      uint32_t plcp = 0;
      if ((D.job & 0x80000000u) == 0 && D.m <= kStgMaxEnt && lane < D.m) {
        pd = ed[D.s0 + lane];
        plcp = lcp[D.s0 + lane];
      }
      if (j >= 2 && !mbar_wait(empty(sl), ((j >> 1) - 1) & 1u, slot_wait_ns)) {
        if (lane == 0) report(errs + (D.job & 0x7FFFFFFFu), E_TIMEOUT, 0, b);
        break;
      }
      StgInfo inf{};
      const uint32_t s0 = D.s0, m = D.m;
      inf.b = b;
      inf.m = m;
      inf.contents = D.contents;
      uint8_t* dst = out + D.dst;
      inf.dst = reinterpret_cast<uint64_t>(dst);
      inf.phase = uint32_t(reinterpret_cast<uintptr_t>(dst) & 15u);
      inf.state = 2;
      const bool in_range = (D.job & 0x80000000u) == 0;
      bool fits = in_range && m <= kStgMaxEnt && inf.phase + inf.contents + 1 <= I;
      uint32_t ce = 0, cs = 0;  // running entry / staging offsets
      StgEnt* E = ents + sl * kStgMaxEnt;
      uint64_t* SRC = srcs + sl * 2 * kStgMaxEnt;
      for (uint32_t k0 = 0; fits && k0 < m; k0 += 32) {
        const uint32_t k = k0 + lane;
        uint32_t esz = 0, ssz = 0, shr = 0, nsh = 0, vlen = 0, kc = 0;
        uint64_t kp = 0, vp = 0;
        if (k < m) {
          const EncDesc d = k0 == 0 ? pd : ed[s0 + k];
          shr = (k % R) == 0 ? 0u : (k0 == 0 ? plcp : lcp[s0 + k]);
          nsh = d.klen - shr;
          vlen = d.vlen;
          kp = d.kptr + shr;
          vp = d.vptr;
          kc = nsh ? uint32_t(((kp + nsh + 15) & ~uint64_t(15)) - (kp & ~uint64_t(15))) : 0u;
          const uint32_t vc = vlen ? uint32_t(((vp + vlen + 15) & ~uint64_t(15)) - (vp & ~uint64_t(15))) : 0u;
          esz = hdr_len(shr, nsh, vlen) + nsh + vlen;
          ssz = kc + vc;
        }
        uint32_t xe = esz, xs = ssz;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t oe = __shfl_up_sync(0xFFFFFFFFu, xe, d), os = __shfl_up_sync(0xFFFFFFFFu, xs, d);
          if (lane >= uint32_t(d)) {
            xe += oe;
            xs += os;
          }
        }
        if (k < m) {
          StgEnt e;
          e.eoff = ce + xe - esz;
          const uint32_t soff = cs + xs - ssz;
          e.shr = shr;
          e.nsh = nsh;
          e.vlen = vlen;
          e.ks = soff + uint32_t(kp & 15u);
          e.vs = soff + kc + uint32_t(vp & 15u);
          e.vb = e.eoff + esz - vlen;
          e.pad = 0;
          E[k] = e;
          SRC[2 * k] = kp;
          SRC[2 * k + 1] = vp;
        }
        ce += __shfl_sync(0xFFFFFFFFu, xe, 31);
        cs += __shfl_sync(0xFFFFFFFFu, xs, 31);
        fits = cs <= S;
      }
      if (fits) inf.state = 1;
      if (lane == 0) {
        if (!fits) {
          done[b] = 0;
          if (in_range) big[atomicAdd(&cnt->big_blocks, 1u)] = b;
        }
        info[sl] = inf;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(full(sl), fits ? cs : 0u);
      __syncwarp();
      if (fits) {
        const uint32_t dst0 = stage_a + sl * S;
        for (uint32_t k = lane; k < m; k += 32) {
          const StgEnt e = E[k];
          const uint64_t kp = SRC[2 * k], vp = SRC[2 * k + 1];
          const uint32_t kb = uint32_t(kp & 15u), vb = uint32_t(vp & 15u);
          if (e.nsh) {
            const uint32_t kc = (kb + e.nsh + 15) & ~15u;
            bulk_load(dst0 + e.ks - kb, reinterpret_cast<const void*>(kp - kb), kc, full(sl));
          }
          if (e.vlen) {
            const uint32_t vc = (vb + e.vlen + 15) & ~15u;
            bulk_load(dst0 + e.vs - vb, reinterpret_cast<const void*>(vp - vb), vc, full(sl));
          }
        }
      }
    }
    if (lane == 0) {
      s_fills[0] = (j + 1) >> 1;  // fills of slot 0 and slot 1
      s_fills[1] = j >> 1;
    }
  }

  // ---------------- consumers ----------------
  const uint32_t ct = tid - 32, cw = warp - 1;  // consumer thread / warp index
  uint32_t j = 0;
  for (uint32_t b = blockIdx.x; warp != 0 && b < nb; b += gridDim.x, ++j) {
    const uint32_t sl = j & 1u;
    if (!consumers_all(mbar_wait(full(sl), (j >> 1) & 1u, slot_wait_ns))) {
      if (ct == 0) report(errs + (bd[b].job & 0x7FFFFFFFu), E_TIMEOUT, 0, b);
      break;
    }
    const StgInfo inf = info[sl];
    if (inf.state == 1) {
      if (ct == 0) bulk_wait_read_all();  // the previous image has left shared memory
      consumers_sync();
      const StgEnt* E = ents + sl * kStgMaxEnt;
      const uint8_t* stg = stage + sl * size_t(S);
      const uint32_t P = inf.phase, m = inf.m;
      const uint32_t contents = inf.contents, msg = contents + 1;
      const uint32_t nr = (m + R - 1) / R;
      const uint32_t rbase = contents - 4 - 4 * nr;
      if (ct < m) {  // headers
        const StgEnt e = E[ct];
        uint8_t* p = img + P + e.eoff;
        uint32_t q = put_varint(p, e.shr);
        q += put_varint(p + q, e.nsh);
        put_varint(p + q, e.vlen);
      }
      // key delta and value: one warp per entry; 16-byte image words inside the value from
      // the staging buffer with funnel shifts, the value's ragged ends and the key bytewise
      for (uint32_t k = cw; k < m; k += kStgConsumers) {
        const StgEnt e = E[k];
        const uint32_t v0 = P + e.vb, v1 = v0 + e.vlen;  // image positions of the value
        const uint32_t kd = v0 - e.nsh;
        for (uint32_t t = lane; t < e.nsh; t += 32) img[kd + t] = stg[e.ks + t];
        const uint32_t h1 = min((v0 + 15) & ~15u, v1), t0 = max(v1 & ~15u, h1);
        if (lane < h1 - v0) img[v0 + lane] = stg[e.vs + lane];
        if (lane < v1 - t0) img[t0 + lane] = stg[e.vs + (t0 - v0) + lane];
        const uint32_t dsrc = e.vs - v0;  // staging offset = image position + dsrc
        for (uint32_t w = h1 + 16 * lane; w + 16 <= t0; w += 512) {
          const uint32_t src = w + dsrc;
          const uint4* q = reinterpret_cast<const uint4*>(stg + (src & ~15u));
          const uint32_t sh = src & 15u;
          const uint4 u0 = q[0];
          *reinterpret_cast<uint4*>(img + w) = sh ? shift32(u0, q[1], sh) : u0;
        }
      }
      for (uint32_t t = ct; t < 4 * nr; t += kStgCons)  // restart array
        img[P + rbase + t] = uint8_t(E[(t >> 2) * R].eoff >> (8 * (t & 3u)));
      if (ct < 4) img[P + contents - 4 + ct] = uint8_t(nr >> (8 * ct));
      if (ct == 4) img[P + contents] = 0;
      fence_proxy_async();
      consumers_sync();  // image complete; the slot's staging buffer is no longer read
      if (ct == 0) mbar_arrive(empty(sl));
      // store: aligned middle in bulk, ragged ends bytewise
      const uint32_t i0 = (P + 15) & ~15u, i1 = (P + msg) & ~15u;
      uint8_t* g = reinterpret_cast<uint8_t*>(inf.dst) - P;  // 16-byte aligned
      if (i1 > i0) {
        if (ct == 0) {
          bulk_store(g + i0, img_a + i0, i1 - i0);
          bulk_commit();
        }
        if (ct >= 32 && ct < 32 + (i0 - P)) g[P + (ct - 32)] = img[P + (ct - 32)];
        if (ct >= 64 && ct < 64 + (P + msg - i1)) g[i1 + (ct - 64)] = img[i1 + (ct - 64)];
      } else {
        for (uint32_t t = ct; t < msg; t += kStgCons) g[P + t] = img[P + t];
      }
      if (ct == 0) done[inf.b] = 1;
    } else {
      consumers_sync();  // every consumer has read the slot's info
      if (ct == 0) mbar_arrive(empty(sl));
    }
  }
  if (tid == 32) {
    bulk_wait_all();
    s_used[0] = (j + 1) >> 1;  // slots consumed (or abandoned) by the consumers
    s_used[1] = j >> 1;
  }
  __syncthreads();
  // after a timeout, let copies still in flight land before the CTA exits (bounded)
  if (tid == 0)
    for (uint32_t sl = 0; sl < 2; ++sl)
      if (s_fills[sl] > s_used[sl]) mbar_wait(full(sl), (s_fills[sl] - 1) & 1u);
}

// Masked CRC-32C trailers of the blocks k_encode wrote (done[b] = 1): one warp per block,
// the block re-read from global memory (mostly L2).
constexpr int kCrcWarps = 32;
constexpr uint32_t kCrcSmem = kRepSmem;

__global__ void __launch_bounds__(kCrcWarps * 32, 1) k_block_crc(Counts* __restrict__ cnt,
                                                                  const uint32_t* __restrict__ blk_file,
                                                                  const FileDesc* __restrict__ files,
                                                                  const uint64_t* __restrict__ C,
                                                                  const uint64_t* __restrict__ bsz,
                                                                  uint8_t* __restrict__ out, uint64_t out_cap,
                                                                  const uint8_t* __restrict__ done, CrcTabs tabs) {
  extern __shared__ uint32_t s_crc[];
  __shared__ uint32_t s_go;  // one decision for the whole CTA
  const uint32_t nb = cnt->nb;
  uint32_t* next = &cnt->crc_next_out;
  if (threadIdx.x == 0) s_go = *(volatile uint32_t*)next < nb;
  __syncthreads();
  if (!s_go) return;  // a helper launch with nothing left
  load_rep_tables992(s_crc, s_crc + kRepWords, tabs);
  __syncthreads();
  const uint32_t lane = lane_id();
  const uint32_t tl = smem_addr(s_crc) + lane * 4u, tz = zcopy_addr(s_crc + kRepWords, lane);
  for (;;) {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(next, 1u);
    b = __shfl_sync(0xFFFFFFFFu, b, 0);
    if (b >= nb) break;
    if (!done[b]) continue;
    const FileDesc F = files[blk_file[b]];
    if (F.off + F.size > out_cap) continue;
    uint8_t* dst = out + F.off + (C[b] - C[F.blk_begin]);
    const uint64_t contents = bsz[b];
    const uint32_t crc = warp_crc32c_u32(dst, contents + 1, tl, tz, tabs);
    if (lane == 0) st_u32(dst + contents + 1, crc_mask(crc));
  }
}

// ---- data block trailers ----------------------------------------------------------------------
// Masked CRC-32C trailer of every block the staged encoder wrote (done[b] = 1), assembled
// from pieces (F linear, F(A || B) = Z_|B|(F(A)) xor F(B)): entry k contributes
// Z_{n - end_k}(Z_{vlen_k}(h_k) xor F(value_k)), with h_k the register of the entry's
// header and key delta read back from the block, restart word r (the offset of entry r * R)
// Z_{n - end of the word}(F(word)), num_restarts and the type byte Z_1(F(num_restarts)), and
// the register's initial value Z_n(0xFFFFFFFF), where n = contents + 1 is the message
// length and end_k the end offset of entry k. One warp per block, one lane per entry; the
// entry offsets come from a warp scan of the entry sizes. The shift matrices Z_{16 * 2^j}
// and the slicing table sit in shared memory.
constexpr uint32_t kTrlZ = 13;  // Z_{16 * 2^j} for j < 13: messages of at most 64 KiB
constexpr uint32_t kTrlSmem = (1024 + kTrlZ * 1024) * 4;
constexpr uint32_t kTrlThreads = 1024;
constexpr uint32_t kTrlWords = 24;  // header and key-delta words loaded at once (keys up to about 80 bytes)

__global__ void __launch_bounds__(kTrlThreads) k_block_trailer(const Counts* __restrict__ cnt,
                                                               const BlkEnc* __restrict__ bd,
                                                               const uint32_t* __restrict__ sd,
                                                               const uint32_t* __restrict__ dr,
                                                               const EncDesc* __restrict__ ed,
                                                               const uint32_t* __restrict__ vcrc, Fmt fmt,
                                                               uint8_t* __restrict__ out,
                                                               const uint8_t* __restrict__ done, CrcTabs tabs) {
  extern __shared__ uint32_t s_trl[];
  for (uint32_t i = threadIdx.x; i < 1024 + kTrlZ * 1024; i += blockDim.x)
    s_trl[i] = i < 1024 ? __ldg(tabs.slice + i) : __ldg(tabs.shift + (i - 1024));
  __syncthreads();
  const uint32_t* sT = s_trl;
  const uint32_t* sZ = s_trl + 1024;
  // a half warp per block: most blocks hold at most 16 entries (a lane each)
  const uint32_t hl = lane_id() & 15u, R = fmt.R, nb = cnt->nb;
  const uint32_t hmask = 0xFFFFu << (lane_id() & 16u);
  const uint64_t halves = gstride() / 16;
  for (uint64_t b = gtid() / 16; b < nb; b += halves) {
    if (!done[b]) continue;
    const BlkEnc D = bd[b];
    if (D.job & 0x80000000u) continue;  // outside the output arena (never staged)
    const uint32_t m = D.m, msg = D.contents + 1, nr = (m + R - 1) / R, rbase = D.contents - 4 - 4 * nr;
    uint32_t acc = 0, carry = 0;
    for (uint32_t k0 = 0; k0 < m; k0 += 16) {
      const uint32_t k = k0 + hl;
      const bool restart = k % R == 0;
      uint32_t esz = 0;
      if (k < m) esz = sd[D.s0 + k] + (restart ? dr[D.s0 + k] : 0u);
      uint32_t x = esz;
#pragma unroll
      for (int d = 1; d < 16; d <<= 1) {
        const uint32_t o = __shfl_up_sync(hmask, x, d, 16);
        if (hl >= uint32_t(d)) x += o;
      }
      if (k < m) {
        const uint32_t eoff = carry + x - esz;
        const EncDesc e = ed[D.s0 + k];
        // header and key delta: bytes [a, z) of the output, aligned words (the bytes before
        // a zeroed: leading zeros leave a zero register unchanged), then single bytes; the
        // words of up to kTrlWords are all loaded before the register is advanced
        const uint64_t a = D.dst + eoff, z = a + esz - e.vlen;
        uint32_t h = 0;
        uint64_t q = a & ~uint64_t(3);
        const uint32_t nw = uint32_t((z - q) >> 2);
        if (nw <= kTrlWords) {
          uint32_t wv[kTrlWords];
#pragma unroll
          for (uint32_t i = 0; i < kTrlWords; ++i)
            wv[i] = i < nw ? *reinterpret_cast<const uint32_t*>(out + q + 4 * i) : 0u;
          if (nw) wv[0] &= ~0u << (8 * uint32_t(a - q));
#pragma unroll
          for (uint32_t i = 0; i < kTrlWords; ++i)
            if (i < nw) h = crc_step4(h, wv[i], sT);
          q += 4ull * nw;
        } else {
          for (; q + 4 <= z; q += 4) {
            uint32_t w = *reinterpret_cast<const uint32_t*>(out + q);
            if (q < a) w &= ~0u << (8 * uint32_t(a - q));
            h = crc_step4(h, w, sT);
          }
        }
        for (q = q > a ? q : a; q < z; ++q) h = crc_byte(h, out[q], sT);
        const uint32_t g = crc_zeros_s(h, e.vlen, sT, sZ) ^ vcrc[e.rec];
        acc ^= crc_zeros_s(g, msg - (eoff + esz), sT, sZ);
        if (restart) acc ^= crc_zeros_s(crc_step4(0u, eoff, sT), msg - (rbase + 4 * (k / R) + 4), sT, sZ);
      }
      carry += __shfl_sync(hmask, x, 15, 16);
    }
    if (hl == 0) acc ^= crc_zeros_s(crc_step4(0u, nr, sT), 1, sT, sZ) ^ crc_zeros_s(0xFFFFFFFFu, msg, sT, sZ);
#pragma unroll
    for (int d = 8; d; d >>= 1) acc ^= __shfl_xor_sync(hmask, acc, d, 16);
    if (hl < 4) out[D.dst + D.contents + 1 + hl] = uint8_t(crc_mask(acc ^ 0xFFFFFFFFu) >> (8 * hl));
  }
}

// ---- compressed data blocks (R4c) ------------------------------------------------------------
// With LUDA_F_COMPRESS the encoders first write every block's raw contents into a scratch
// arena (block b at Craw[b], one pseudo-table per job), k_compress compresses each block
// into a second scratch (block b at Cc[b]) and turns bsz/disk into the stored sizes (the
// block cut used the raw ones), the file cut and layout run on the stored sizes, and
// k_place copies each block's stored bytes and type byte into its table; the trailer
// checksums then cover the stored bytes.

// Scratch shares: raw block with room for a trailer, and the compressor's bound (a 64-byte
// segment of literals takes at most 66 bytes; a copy never takes more than it covers; the
// length header at most 5), both 16-byte multiples.
__global__ void k_raw_sizes(const Counts* __restrict__ cnt, const uint64_t* __restrict__ bsz,
                            uint64_t* __restrict__ rawsz, uint64_t* __restrict__ czsz) {
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) {
    const uint64_t n = bsz[b];
    rawsz[b] = (n + kTrailer + 15) & ~15ull;
    czsz[b] = ((n + n / 32 + 16 + 15) & ~15ull) + 16;
  }
}

__global__ void k_raw_files(const JobDev* __restrict__ jobs, uint32_t n_jobs, const Counts* __restrict__ cnt,
                            const uint64_t* __restrict__ Craw, FileDesc* __restrict__ rfiles,
                            uint32_t* __restrict__ rbf) {
  for (uint64_t j = gtid(); j < n_jobs; j += gstride()) {
    FileDesc F{};
    F.blk_begin = jobs[j].blk_begin;
    F.blk_end = jobs[j].blk_end;
    F.off = Craw[F.blk_begin];
    F.size = Craw[F.blk_end] - F.off;
    F.job = uint32_t(j);
    rfiles[j] = F;
  }
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) rbf[b] = job_of_block(jobs, n_jobs, uint32_t(b));
}

constexpr uint32_t kCzTab = 4096;      // hash table entries (12-bit hash)
constexpr uint32_t kCzWin = 32 * 64;   // positions per window: one 64-byte segment per lane
constexpr uint32_t kCzStage = 72;      // staging bytes per lane (a segment's elements: at most 66)
constexpr uint32_t kCzWinOut = 32 * 66 + 64;  // a window's stream, joined before its coalesced store
// Positions as Pos (16 bits for blocks below 65535 bytes: smaller tables, more warps per
// SM; 32 bits for larger blocks), kWarps warps per CTA.
template <typename Pos>
__host__ __device__ constexpr uint32_t cz_warp_smem() {
  return (kCzTab + kCzWin) * uint32_t(sizeof(Pos)) + 32 * kCzStage + kCzWinOut;
}
constexpr uint32_t kCzSmallMax = 65534;  // largest block for 16-bit positions (65535: none)
constexpr uint32_t kCzWarps16 = 2, kCzWarps32 = 4;
// Blocks up to kCzCopyMax bytes go to k_compress_copy, which reads a shared-memory copy.
constexpr uint32_t kCzCopy = 18 * 1024;
constexpr uint32_t kCzCopyMax = kCzCopy - 16;
constexpr uint32_t kCzCopyWarps = 1;
__host__ __device__ constexpr uint32_t cz_copy_smem() {
  return kCzTab * 2 + kCzWin * 2 + (kCzWin / 32) * 4 + kCzWinOut + kCzCopy;
}
static_assert(cz_copy_smem() % 16 == 0, "16-byte aligned shares");

// The little-endian word at in + q, from the two aligned words around it (`in` is 16-byte
// aligned and its block's scratch share extends at least 4 bytes past any word read).
__device__ __forceinline__ uint32_t ld4_at(const uint8_t* __restrict__ in, uint64_t q) {
  const uint32_t* a = reinterpret_cast<const uint32_t*>(in + (q & ~uint64_t(3)));
  return __funnelshift_r(__ldg(a), __ldg(a + 1), uint32_t(q & 3u) * 8u);
}

// One warp per block. Per window of 2048 positions: the warp steps through it 32
// positions at a time (lane = position) to find cand(i), the latest earlier position with
// the same 12-bit hash (within the step by matching hashes across lanes, else from the
// table of earlier steps, which the last lane of each hash then updates); then each lane
// parses its own 64-byte segment from the window's candidates into its staging bytes, and
// the segments are written out in order after a warp scan of their sizes. The block is
// kept compressed (type 1) when the stream is shorter than raw - raw / 8.
template <typename Pos, uint32_t kWarps>
__global__ void __launch_bounds__(kWarps * 32) k_compress(const Counts* __restrict__ cnt,
                                                            const uint64_t* __restrict__ Craw,
                                                            const uint64_t* __restrict__ Cc,
                                                            uint64_t* __restrict__ bsz, uint64_t* __restrict__ disk,
                                                            const uint8_t* __restrict__ raw, uint64_t raw_cap,
                                                            uint8_t* __restrict__ cz, uint64_t c_cap,
                                                            uint8_t* __restrict__ ctype) {
  extern __shared__ __align__(16) uint8_t s_cz[];
  constexpr bool kSmall = sizeof(Pos) == 2;
  constexpr uint32_t kCzNone = kSmall ? 0xFFFFu : 0xFFFFFFFFu;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  Pos* tab = reinterpret_cast<Pos*>(s_cz + warp * cz_warp_smem<Pos>());
  Pos* cw = tab + kCzTab;
  uint8_t* const stage0 = reinterpret_cast<uint8_t*>(cw + kCzWin);
  uint8_t* stage = stage0 + lane * kCzStage;
  uint8_t* const wout = stage0 + 32 * kCzStage;
  const uint32_t nb = cnt->nb;
  const uint64_t warps = gstride() / 32;
  for (uint64_t b = gtid() / 32; b < nb; b += warps) {
    const uint64_t n = bsz[b];
    if (kSmall ? (n <= kCzCopyMax || n > kCzSmallMax) : n <= kCzSmallMax) continue;  // another kernel takes it
    const uint64_t cbound = n + n / 32 + 16;
    if (Craw[b] + n > raw_cap || Cc[b] + cbound > c_cap) {
      if (lane == 0) ctype[b] = 0;
      continue;
    }
    const uint8_t* in = raw + Craw[b];
    uint8_t* o = cz + Cc[b];
    for (uint32_t k = lane; k < kCzTab; k += 32) tab[k] = Pos(kCzNone);
    uint32_t total = 0;  // stream bytes so far: the length header, then the segments
    {
      uint64_t v = n;
      while (v >= 0x80) {
        if (lane == 0) o[total] = uint8_t(v | 0x80);
        v >>= 7;
        ++total;
      }
      if (lane == 0) o[total] = uint8_t(v);
      ++total;
    }
    __syncwarp();
    for (uint64_t wb = 0; wb < n; wb += kCzWin) {
      const uint64_t we = wb + kCzWin < n ? wb + kCzWin : n;
      for (uint64_t base = wb; base < we; base += 32) {
        const uint64_t p = base + lane;
        const bool valid = p + 4 <= n;
        const uint32_t h = valid ? (ld4_at(in, p) * 2654435761u) >> 20 : kCzTab + lane;
        const uint32_t m = __match_any_sync(0xFFFFFFFFu, h);
        const uint32_t lower = m & ((1u << lane) - 1u);
        uint32_t c = kCzNone;
        if (valid) c = lower ? uint32_t(base) + (31u - __clz(lower)) : uint32_t(tab[h]);
        __syncwarp();
        if (valid && (m >> lane) == 1u) tab[h] = Pos(p);
        __syncwarp();
        if (p < we) cw[p - wb] = Pos(c);
      }
      __syncwarp();
      // this lane's segment [s0, e)
      const uint64_t s0 = wb + 64ull * lane;
      uint32_t sz = 0;
      if (s0 < n) {
        const uint64_t e = s0 + 64 < n ? s0 + 64 : n;
        uint64_t i = s0, lit = s0;
        auto literal = [&](uint64_t from, uint64_t to) {
          const uint32_t len = uint32_t(to - from), v = len - 1;
          if (v < 60) {
            stage[sz++] = uint8_t(v << 2);
          } else {
            stage[sz++] = uint8_t(60u << 2);
            stage[sz++] = uint8_t(v);
          }
          for (uint64_t k = from; k < to; ++k) stage[sz++] = in[k];
        };
        while (i < e) {
          const uint32_t c = uint32_t(cw[i - wb]);
          bool ok = e - i >= 4 && c != kCzNone && i - c < 65536;
          if (ok) ok = ld4_at(in, c) == ld4_at(in, i);
          if (ok) {
            uint64_t L = 4;
            while (i + L < e && in[c + L] == in[i + L]) ++L;
            if (i > lit) literal(lit, i);
            const uint64_t off = i - c;
            if (L <= 11 && off < 2048) {
              stage[sz++] = uint8_t(1u | uint32_t(L - 4) << 2 | uint32_t(off >> 8) << 5);
              stage[sz++] = uint8_t(off);
            } else {
              stage[sz++] = uint8_t(2u | uint32_t(L - 1) << 2);
              stage[sz++] = uint8_t(off);
              stage[sz++] = uint8_t(off >> 8);
            }
            i += L;
            lit = i;
          } else {
            ++i;
          }
        }
        if (e > lit) literal(lit, e);
      }
      // segments in order
      uint32_t x = sz;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= uint32_t(d)) x += y;
      }
      // the segments joined in shared memory, then stored by consecutive lanes
      const uint32_t at = x - sz, wsum = __shfl_sync(0xFFFFFFFFu, x, 31);
      for (uint32_t k = 0; k < sz; ++k) wout[at + k] = stage[k];
      __syncwarp();
      for (uint32_t k = lane; k < wsum; k += 32) o[total + k] = wout[k];
      total += wsum;
      __syncwarp();
    }
    if (lane == 0) {
      const bool keep = total < n - n / 8;
      ctype[b] = keep ? 1 : 0;
      bsz[b] = keep ? total : n;
      disk[b] = bsz[b] + kTrailer;
    }
  }
}

// The little-endian word at byte q of a block copy in shared memory (the copy extends at
// least 8 bytes past any word read).
__device__ __forceinline__ uint32_t ld4s(const uint8_t* in, uint32_t q) {
  const uint32_t* a = reinterpret_cast<const uint32_t*>(in + (q & ~3u));
  return __funnelshift_r(a[0], a[1], (q & 3u) * 8u);
}

// k_compress for blocks of at most kCzCopyMax bytes, with the same output: the warp first
// copies its block into shared memory. The candidate search also decides, for every
// position, whether a copy can start there (a candidate, whose first four bytes equal the
// position's, inside the position's segment), as one bit per position; each lane then
// parses its segment by jumping from one such position to the next, once to size its
// elements and once, after a warp scan of the sizes, to write them into the window's
// stream. The next step's word, hash and match are taken while a step updates the table.
__global__ void __launch_bounds__(kCzCopyWarps * 32) k_compress_copy(const Counts* __restrict__ cnt,
                                                                    const uint64_t* __restrict__ Craw,
                                                                    const uint64_t* __restrict__ Cc,
                                                                    uint64_t* __restrict__ bsz, uint64_t* __restrict__ disk,
                                                                    const uint8_t* __restrict__ raw, uint64_t raw_cap,
                                                                    uint8_t* __restrict__ cz, uint64_t c_cap,
                                                                    uint8_t* __restrict__ ctype) {
  extern __shared__ __align__(16) uint8_t s_cz[];
  constexpr uint32_t kNone = 0xFFFFu;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint16_t* tab = reinterpret_cast<uint16_t*>(s_cz + warp * cz_copy_smem());
  uint16_t* cw = tab + kCzTab;
  uint32_t* okm = reinterpret_cast<uint32_t*>(cw + kCzWin);  // bit j of word k: position wb + 32k + j
  uint8_t* const wout = reinterpret_cast<uint8_t*>(okm + kCzWin / 32);
  uint8_t* const in = wout + kCzWinOut;
  const uint32_t nb = cnt->nb;
  const uint64_t warps = gstride() / 32;
  for (uint64_t b = gtid() / 32; b < nb; b += warps) {
    const uint64_t n64 = bsz[b];
    if (n64 > kCzCopyMax) continue;  // k_compress takes it
    const uint32_t n = uint32_t(n64);
    const uint64_t cbound = n64 + n64 / 32 + 16;
    if (Craw[b] + n64 > raw_cap || Cc[b] + cbound > c_cap) {
      if (lane == 0) ctype[b] = 0;
      continue;
    }
    {
      // the block into shared memory, 16 bytes per lane and step (its scratch share is a
      // 16-byte multiple at a 16-byte boundary)
      const uint4* src = reinterpret_cast<const uint4*>(raw + Craw[b]);
      uint4* dst = reinterpret_cast<uint4*>(in);
      for (uint32_t k = lane; k < (n + 15) / 16; k += 32) dst[k] = __ldg(src + k);
    }
    uint8_t* o = cz + Cc[b];
    for (uint32_t k = lane; k < kCzTab; k += 32) tab[k] = uint16_t(kNone);
    uint32_t total = 0;  // stream bytes so far: the length header, then the segments
    {
      uint32_t v = n;
      while (v >= 0x80) {
        if (lane == 0) o[total] = uint8_t(v | 0x80);
        v >>= 7;
        ++total;
      }
      if (lane == 0) o[total] = uint8_t(v);
      ++total;
    }
    __syncwarp();
    for (uint32_t wb = 0; wb < n; wb += kCzWin) {
      const uint32_t we = wb + kCzWin < n ? wb + kCzWin : n;
      uint32_t p = wb + lane;
      bool valid = p + 4 <= n;
      uint32_t w = valid ? ld4s(in, p) : 0u;
      uint32_t h = valid ? (w * 2654435761u) >> 20 : kCzTab + lane;
      uint32_t m = __match_any_sync(0xFFFFFFFFu, h);
      for (uint32_t base = wb; base < we; base += 32) {
        const uint32_t pn = p + 32;
        const bool vn = base + 32 < we && pn + 4 <= n;
        const uint32_t wn = vn ? ld4s(in, pn) : 0u;
        const uint32_t hn = vn ? (wn * 2654435761u) >> 20 : kCzTab + lane;
        const uint32_t mn = __match_any_sync(0xFFFFFFFFu, hn);
        const uint32_t lower = m & ((1u << lane) - 1u);
        const uint32_t src = lower ? 31u - __clz(lower) : lane;
        const uint32_t wl = __shfl_sync(0xFFFFFFFFu, w, src);
        uint32_t c = kNone;
        if (valid) c = lower ? base + src : uint32_t(tab[h]);
        __syncwarp();
        if (valid && (m >> lane) == 1u) tab[h] = uint16_t(p);
        __syncwarp();
        const uint32_t send = wb + ((p - wb) & ~63u) + 64u;  // the end of p's segment
        const bool ok = valid && p < we && c != kNone && p + 4 <= (send < n ? send : n) &&
                        (lower ? wl : ld4s(in, c)) == w;
        if (p < we) cw[p - wb] = uint16_t(c);
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, ok);
        if (lane == 0) okm[(base - wb) >> 5] = bits;
        p = pn;
        valid = vn;
        w = wn;
        h = hn;
        m = mn;
      }
      __syncwarp();
      // this lane's segment [s0, e): sized, then (after the scan) written at its offset
      const uint32_t s0 = wb + 64u * lane;
      const uint32_t e = s0 + 64u < n ? s0 + 64u : n;
      uint64_t mask = 0;
      if (s0 < n) {
        const uint32_t k0 = (s0 - wb) >> 5;
        mask = uint64_t(okm[k0]) | (uint64_t(okm[k0 + 1]) << 32);
        if (e - s0 < 64) mask &= (1ull << (e - s0)) - 1;  // words past the window are stale
      }
      uint32_t at = 0, sz = 0;
      for (int pass = 0; pass < 2; ++pass) {
        uint8_t* q = wout + at;
        uint32_t put = 0;
        auto literal = [&](uint32_t from, uint32_t to) {
          const uint32_t len = to - from, v = len - 1;
          if (v < 60) {
            if (pass) q[put] = uint8_t(v << 2);
            put += 1;
          } else {
            if (pass) {
              q[put] = uint8_t(60u << 2);
              q[put + 1] = uint8_t(v);
            }
            put += 2;
          }
          if (pass) {
            uint32_t k = from;
            for (; k + 4 <= to; k += 4) {
              const uint32_t x = ld4s(in, k);
              q[put] = uint8_t(x);
              q[put + 1] = uint8_t(x >> 8);
              q[put + 2] = uint8_t(x >> 16);
              q[put + 3] = uint8_t(x >> 24);
              put += 4;
            }
            for (; k < to; ++k) q[put++] = in[k];
          } else {
            put += len;
          }
        };
        if (s0 < n) {
          uint32_t i = s0, lit = s0;
          while (i < e) {
            const uint32_t oi = i - s0;
            const uint64_t rem = mask >> oi << oi;  // copies can start at these positions >= i
            if (!rem) break;
            i = s0 + uint32_t(__ffsll(static_cast<long long>(rem)) - 1);
            const uint32_t c = cw[i - wb];
            uint32_t L = 4;
            while (i + L < e && in[c + L] == in[i + L]) ++L;
            if (i > lit) literal(lit, i);
            const uint32_t off = i - c;
            if (L <= 11 && off < 2048) {
              if (pass) {
                q[put] = uint8_t(1u | (L - 4) << 2 | (off >> 8) << 5);
                q[put + 1] = uint8_t(off);
              }
              put += 2;
            } else {
              if (pass) {
                q[put] = uint8_t(2u | (L - 1) << 2);
                q[put + 1] = uint8_t(off);
                q[put + 2] = uint8_t(off >> 8);
              }
              put += 3;
            }
            i += L;
            lit = i;
          }
          if (e > lit) literal(lit, e);
        }
        if (pass == 0) {
          sz = put;
          uint32_t x = sz;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= uint32_t(d)) x += y;
          }
          at = x - sz;
        }
      }
      __syncwarp();
      const uint32_t wsum = __shfl_sync(0xFFFFFFFFu, at + sz, 31);
      for (uint32_t k = lane; k < wsum; k += 32) o[total + k] = wout[k];
      total += wsum;
      __syncwarp();
    }
    if (lane == 0) {
      const bool keep = total < n - n / 8;
      ctype[b] = keep ? 1 : 0;
      bsz[b] = keep ? total : n;
      disk[b] = bsz[b] + kTrailer;
    }
  }
}

// One warp per block: its stored bytes (compressed or raw) and type byte into its table.
__global__ void k_place(const Counts* __restrict__ cnt, const uint32_t* __restrict__ blk_file,
                        const FileDesc* __restrict__ files, const uint64_t* __restrict__ C,
                        const uint64_t* __restrict__ bsz, const uint64_t* __restrict__ Craw,
                        const uint64_t* __restrict__ Cc, const uint8_t* __restrict__ raw,
                        const uint8_t* __restrict__ cz, const uint8_t* __restrict__ ctype,
                        uint8_t* __restrict__ out, uint64_t out_cap, uint8_t* __restrict__ done) {
  const uint32_t lane = lane_id(), nb = cnt->nb;
  const uint64_t warps = gstride() / 32;
  for (uint64_t b = gtid() / 32; b < nb; b += warps) {
    const FileDesc F = files[blk_file[b]];
    if (F.off + F.size > out_cap) continue;
    uint8_t* dst = out + F.off + (C[b] - C[F.blk_begin]);
    const uint8_t t = ctype[b];
    const uint8_t* src = t ? cz + Cc[b] : raw + Craw[b];
    const uint64_t n = bsz[b];
    for (uint64_t k = lane; k < n; k += 32) dst[k] = src[k];
    if (lane == 0) {
      dst[n] = t;
      done[b] = 1;
    }
  }
}

// MurmurHash3 x86_32 (Appleby, public domain), from its published description.
__device__ __forceinline__ uint32_t rotl(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

__device__ uint32_t murmur3_32(const uint8_t* p, uint32_t n, uint32_t seed) {
  const uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
  uint32_t h = seed;
  const uint32_t nb = n >> 2;
  for (uint32_t i = 0; i < nb; ++i) {
    uint32_t k = ld_u32(p + 4 * i);
    k *= c1;
    k = rotl(k, 15);
    k *= c2;
    h ^= k;
    h = rotl(h, 13);
    h = h * 5u + 0xe6546b64u;
  }
  const uint8_t* t = p + 4 * nb;
  uint32_t k = 0;
  switch (n & 3) {
    case 3: k ^= uint32_t(t[2]) << 16; [[fallthrough]];
    case 2: k ^= uint32_t(t[1]) << 8; [[fallthrough]];
    case 1:
      k ^= t[0];
      k *= c1;
      k = rotl(k, 15);
      k *= c2;
      h ^= k;
  }
  h ^= n;
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__global__ void k_bloom(const EncDesc* __restrict__ ed, const Counts* __restrict__ cnt,
                        const FileDesc* __restrict__ files, Fmt fmt, const uint32_t* __restrict__ start,
                        const uint64_t* __restrict__ C, FiltArr fa, uint32_t* __restrict__ bitmap,
                        uint64_t out_cap, uint64_t bm_cap) {
  const uint32_t n = cnt->n_surv, nf = cnt->nf;
  if (cnt->out_bytes > out_cap || cnt->bm_words > bm_cap) return;
  if (fa.base && fa.base[nf] > fa.cap) return;
  for (uint64_t s = gtid(); s < n; s += gstride()) {
    uint32_t lo = 0, hi = nf;  // the table holding survivor s
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (files[mid].ent_begin <= s) lo = mid;
      else hi = mid;
    }
    const FileDesc F = files[lo];
    const EncDesc e = ed[s];
    uint32_t h = murmur3_32(reinterpret_cast<const uint8_t*>(e.kptr), e.klen - 8, 0);
    const uint32_t d = (h >> 17) | (h << 15);
    uint32_t* bm = bitmap + F.bm_word;
    uint64_t nbits = F.bm_bits;
    if (fa.base) {  // the filter of the 2 KiB window the entry's block starts in
      const uint32_t b = F.blk_begin + last_le<uint32_t>(start + F.blk_begin, F.blk_end - F.blk_begin, uint32_t(s));
      const uint64_t slot = fa.base[lo] + ((C[b] - C[F.blk_begin]) >> kFilterBaseLg);
      bm = bitmap + fa.woff[slot];
      nbits = (fa.bytes[slot] - 1) * 8;
    }
    for (uint32_t j = 0; j < fmt.k; ++j) {
      const uint64_t bit = h % nbits;
      atomicOr(bm + (bit >> 5), 1u << (bit & 31));
      h += d;
    }
  }
}

__global__ void k_index_write(const uint32_t* __restrict__ start, const Counts* __restrict__ cnt,
                              const uint64_t* __restrict__ bsz,
                              const uint64_t* __restrict__ C, const uint64_t* __restrict__ IX,
                              const uint32_t* __restrict__ blk_file, const FileDesc* __restrict__ files,
                              const uint32_t* __restrict__ surv, Recs recs, const uint8_t* __restrict__ arena,
                              uint32_t flags, uint8_t* __restrict__ out, uint64_t out_cap) {
  const uint32_t nb = cnt->nb;
  for (uint64_t b = gtid(); b < nb; b += gstride()) {
    const FileDesc F = files[blk_file[b]];
    if (F.off + F.size > out_cap) continue;
    uint8_t* ib = out + F.off + F.index_off;
    const uint32_t fb0 = F.blk_begin, fb1 = F.blk_end;
    const uint64_t eoff = IX[b] - IX[fb0];
    const uint32_t klen = index_key_of(b, fb1, start, surv, recs, arena, flags, nullptr);
    const uint64_t off = C[b] - C[fb0], size = bsz[b];
    const uint32_t hlen = varint_size(off) + varint_size(size);
    uint8_t* p = ib + eoff;
    *p++ = 0;
    p += put_varint(p, klen);
    p += put_varint(p, hlen);
    index_key_of(b, fb1, start, surv, recs, arena, flags, p);
    p += klen;
    p += put_varint(p, off);
    put_varint(p, size);
    st_u32(ib + (IX[fb1] - IX[fb0]) + 4ull * (b - fb0), uint32_t(eoff));
  }
}

// Filter bitmaps into the tables: one thread per 32-bit bitmap word of all tables.
__global__ void k_filter_copy(const FileDesc* __restrict__ files, const Counts* __restrict__ cnt, FiltArr fa,
                              const uint32_t* __restrict__ bitmap, uint8_t* __restrict__ out, uint64_t out_cap) {
  const uint32_t nf = cnt->nf;
  const uint64_t nw = cnt->bm_words;
  if (fa.base) {
    // filter array: word w of filter s, at the filter's offset in its table's filter block
    const uint32_t ns = cnt->n_filt;
    if (fa.base[nf] > fa.cap) return;
    for (uint64_t w = gtid(); w < nw; w += gstride()) {
      const uint32_t s = last_le<uint64_t>(fa.woff, ns, w);
      const uint32_t f = last_le<uint64_t>(fa.base, nf, s);
      const FileDesc F = files[f];
      if (F.off + F.size > out_cap) continue;
      const uint64_t i = 4 * (w - fa.woff[s]), bytes = fa.bytes[s] - 1;
      if (fa.bytes[s] == 0 || i >= bytes) continue;
      const uint32_t v = bitmap[w];
      uint8_t* fp = out + F.off + F.data_size + (fa.boff[s] - fa.boff[fa.base[f]]) + i;
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k)
        if (i + k < bytes) fp[k] = uint8_t(v >> (8 * k));
    }
    return;
  }
  for (uint64_t w = gtid(); w < nw; w += gstride()) {
    uint32_t lo = 0, hi = nf;  // last table whose bitmap starts at or before w
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (files[mid].bm_word <= w) lo = mid;
      else hi = mid;
    }
    const FileDesc F = files[lo];
    if (F.off + F.size > out_cap) continue;
    const uint64_t i = 4 * (w - F.bm_word), bytes = F.filter_size - 1;
    if (i >= bytes) continue;
    const uint32_t v = bitmap[w];
    uint8_t* fp = out + F.off + F.data_size + i;
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (i + k < bytes) fp[k] = uint8_t(v >> (8 * k));
  }
}

// Filter array, one thread per filter: its probe count byte (when not empty) and its entry
// in the table's offset array.
__global__ void k_filter_tail(const FileDesc* __restrict__ files, const Counts* __restrict__ cnt, FiltArr fa, Fmt fmt,
                              uint8_t* __restrict__ out, uint64_t out_cap) {
  const uint32_t nf = cnt->nf, ns = cnt->n_filt;
  if (fa.base[nf] > fa.cap) return;
  for (uint64_t s = gtid(); s < ns; s += gstride()) {
    const uint32_t f = last_le<uint64_t>(fa.base, nf, s);
    const FileDesc F = files[f];
    if (F.off + F.size > out_cap) continue;
    const uint64_t s0 = fa.base[f], rel = fa.boff[s] - fa.boff[s0];
    uint8_t* fp = out + F.off + F.data_size;
    if (fa.bytes[s]) fp[rel + fa.bytes[s] - 1] = uint8_t(fmt.k);
    st_u32(fp + (fa.boff[fa.base[f + 1]] - fa.boff[s0]) + 4 * (s - s0), uint32_t(rel));
  }
}

// One thread per table: probe count byte, metaindex, index restart count, footer, the three
// block checksums queued for the multi-warp CRC, and the table's summary.
__global__ void k_file_finish(const FileDesc* __restrict__ files, const Counts* __restrict__ cnt,
                              const uint32_t* __restrict__ surv, Recs recs, Fmt fmt, uint8_t* __restrict__ out,
                              uint64_t out_cap, CrcMsg* __restrict__ msgs, FileMeta* __restrict__ meta) {
  const uint32_t nf = cnt->nf;
  for (uint64_t f = gtid(); f < nf; f += gstride()) {
    const FileDesc F = files[f];
    if (F.off + F.size > out_cap) {
      msgs[3 * f] = msgs[3 * f + 1] = msgs[3 * f + 2] = CrcMsg{};
      continue;
    }
    uint8_t* base = out + F.off;
    uint8_t* fp = base + F.data_size;
    const bool array = (fmt.flags & LUDA_F_FILTER_ARRAY) != 0;
    if (array) {  // the offset array's position, then base_lg
      st_u32(fp + F.filter_size - 5, uint32_t(F.filter_size - 5 - 4ull * F.n_filt));
      fp[F.filter_size - 1] = uint8_t(kFilterBaseLg);
    } else {
      fp[F.filter_size - 1] = uint8_t(fmt.k);
    }
    fp[F.filter_size] = 0;
    // metaindex: one entry "filter.luda.bloom" (or "filter.luda.bloom2k" for a filter
    // array) -> filter handle, restart interval 1
    uint8_t* mp = base + F.meta_off;
    uint8_t hbuf[20];
    uint32_t hl = put_varint(hbuf, F.data_size);
    hl += put_varint(hbuf + hl, F.filter_size);
    uint32_t q = 0;
    const char name[] = "filter.luda.bloom2k";
    const uint32_t name_len = array ? 19 : 17;
    mp[q++] = 0;
    mp[q++] = uint8_t(name_len);
    mp[q++] = uint8_t(hl);
    for (uint32_t i = 0; i < name_len; ++i) mp[q++] = uint8_t(name[i]);
    for (uint32_t i = 0; i < hl; ++i) mp[q++] = hbuf[i];
    st_u32(mp + q, 0);
    st_u32(mp + q + 4, 1);
    mp[F.meta_size] = 0;
    // index block: restart count and type
    uint8_t* ip = base + F.index_off;
    st_u32(ip + F.index_size - 4, F.blk_end - F.blk_begin);
    ip[F.index_size] = 0;
    // block checksums: filter, metaindex, index
    CrcMsg m{};
    m.p = fp;
    m.n = F.filter_size + 1;
    m.out = fp + F.filter_size + 1;
    msgs[3 * f] = m;
    m.p = base + F.meta_off;
    m.n = F.meta_size + 1;
    m.out = base + F.meta_off + F.meta_size + 1;
    msgs[3 * f + 1] = m;
    m.p = base + F.index_off;
    m.n = F.index_size + 1;
    m.out = base + F.index_off + F.index_size + 1;
    msgs[3 * f + 2] = m;
    uint8_t* ft = base + F.size - kFooter;
    q = put_varint(ft, F.meta_off);
    q += put_varint(ft + q, F.meta_size);
    q += put_varint(ft + q, F.index_off);
    q += put_varint(ft + q, F.index_size);
    while (q < 40) ft[q++] = 0;
    for (int i = 0; i < 8; ++i) ft[40 + i] = uint8_t(kMagic >> (8 * i));
    FileMeta mt{};
    mt.off = F.off;
    mt.size = F.size;
    mt.n_entries = F.ent_end - F.ent_begin;
    mt.data_size = F.data_size;
    mt.small_len = recs.klen[surv[F.ent_begin]];
    mt.large_len = recs.klen[surv[F.ent_end - 1]];
    mt.job = F.job;
    meta[f] = mt;
  }
}

__global__ void k_key_lens(const FileMeta* __restrict__ meta, const Counts* __restrict__ cnt,
                           uint64_t* __restrict__ lens) {
  const uint32_t nf = cnt->nf;
  for (uint64_t f = gtid(); f < nf; f += gstride()) lens[f] = uint64_t(meta[f].small_len) + meta[f].large_len;
}

__global__ void k_key_gather(FileMeta* meta, Counts* cnt, const uint64_t* __restrict__ koff,
                             const FileDesc* __restrict__ files, const uint32_t* __restrict__ surv, Recs recs,
                             const uint8_t* __restrict__ arena, uint8_t* __restrict__ keybuf) {
  const uint32_t nf = cnt->nf;
  if (gtid() == 0) cnt->key_bytes = koff[nf];
  for (uint64_t f = gtid(); f < nf; f += gstride()) {
    const FileDesc F = files[f];
    const uint32_t a = surv[F.ent_begin], z = surv[F.ent_end - 1];
    const uint64_t o = koff[f];
    const uint32_t la = recs.klen[a], lz = recs.klen[z];
    for (uint32_t i = 0; i < la; ++i) keybuf[o + i] = arena[recs.koff[a] + i];
    for (uint32_t i = 0; i < lz; ++i) keybuf[o + la + i] = arena[recs.koff[z] + i];
    meta[f].small_koff = o;
    meta[f].large_koff = o + la;
  }
}

// ---- build path ------------------------------------------------------------------------
__global__ void k_build_records(const uint8_t* __restrict__ ukeys, const uint64_t* __restrict__ ukoff,
                                const uint64_t* __restrict__ seqs, const uint8_t* __restrict__ types,
                                const uint8_t* __restrict__ vals, const uint64_t* __restrict__ voff, uint32_t n,
                                Recs recs, uint8_t* __restrict__ arena, uint32_t* __restrict__ surv, DErr* err) {
  const uint64_t uend = ukoff[n], vend = voff[n];
  for (uint64_t i = gtid(); i < n; i += gstride()) {
    uint64_t u0 = ukoff[i], ulen = ukoff[i + 1] - u0;
    uint64_t v0 = voff[i], vlen = voff[i + 1] - v0;
    const uint64_t seq = seqs[i];
    const uint32_t ty = types[i];
    if (seq >= (1ull << 56) || ty > 1) report(err, E_INVALID, ~0u, i);
    // offsets that are not ascending inside [0, total] fail the call; the record then
    // stays inside the buffers (empty user key and value)
    if (ukoff[i + 1] < u0 || ukoff[i + 1] > uend || voff[i + 1] < v0 || voff[i + 1] > vend ||
        ulen > 0xFFFFFF00ull || vlen > 0xFFFFFFFFull) {
      report(err, E_INVALID, ~0u, i);
      u0 = ulen = v0 = vlen = 0;
    }
    const uint64_t kpos = u0 + 8 * i;
    const uint64_t tr = (seq << 8) | (ty & 0xFFu);
    uint8_t* kd = arena + kpos;
    for (uint64_t t = 0; t < ulen; ++t) kd[t] = ukeys[u0 + t];
    for (int t = 0; t < 8; ++t) kd[ulen + t] = uint8_t(tr >> (8 * t));
    recs.pfx[i] = key_prefix(kd, uint32_t(ulen));
    recs.koff[i] = kpos;
    recs.klen[i] = uint32_t(ulen + 8);
    recs.tr[i] = tr;
    recs.vptr[i] = reinterpret_cast<uint64_t>(vals + v0);
    recs.vlen[i] = uint32_t(vlen);
    recs.src[i] = 0;
    surv[i] = uint32_t(i);
  }
}

__global__ void k_build_check(Recs recs, const uint8_t* __restrict__ arena, uint32_t n, DErr* err) {
  for (uint64_t i = gtid() + 1; i < n; i += gstride()) {
    const uint32_t a = uint32_t(i - 1), b = uint32_t(i);
    // strictly increasing internal keys
    int c;
    const uint64_t pa = recs.pfx[a], pb = recs.pfx[b];
    if (pa != pb) {
      c = pa < pb ? -1 : 1;
    } else {
      const uint32_t la = recs.klen[a] - 8, lb = recs.klen[b] - 8;
      const uint8_t* ka = arena + recs.koff[a];
      const uint8_t* kb = arena + recs.koff[b];
      const uint32_t m = la < lb ? la : lb;
      c = 0;
      for (uint32_t t = 8; t < m && !c; ++t)
        if (ka[t] != kb[t]) c = ka[t] < kb[t] ? -1 : 1;
      if (!c && la != lb) c = la < lb ? -1 : 1;
      if (!c) {
        const uint64_t ta = recs.tr[a], tb = recs.tr[b];
        c = ta == tb ? 0 : (ta > tb ? -1 : 1);
      }
    }
    if (c >= 0) report(err, E_INVALID, ~0u, i);
  }
}

}  // namespace

void launch_sizes(const uint32_t* surv, const Counts* cnt, uint32_t cap, const JobDev* jobs, uint32_t n_jobs,
                  Recs recs, const uint8_t* arena, uint32_t* lcp, uint32_t* sd, uint32_t* dr, EncDesc* ed,
                  cudaStream_t st) {
  if (!cap) return;
  k_sizes<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(surv, cnt, jobs, n_jobs, recs, arena, lcp, sd, dr, ed); count_launches(1);
}

void launch_block_next(const uint64_t* P, const uint32_t* dr, const Counts* cnt, uint32_t cap, const JobDev* jobs,
                       uint32_t n_jobs, Fmt fmt, uint32_t* next, cudaStream_t st) {
  if (!cap) return;
  k_block_next<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(P, dr, cnt, jobs, n_jobs, fmt, next); count_launches(1);
}

uint64_t stitch_temp_bytes(uint32_t cap) {
  const uint64_t tiles = (uint64_t(cap) + kStitchTile - 1) / kStitchTile;
  return (tiles * kWinMax + tiles + 64) * sizeof(uint32_t) + 256;
}

void launch_stitch(const uint32_t* next, const uint32_t* n_dev, uint32_t cap, uint32_t* gap, const JobDev* jobs,
                   uint32_t n_jobs, bool blocks_level, uint8_t* flags, void* temp, cudaStream_t st) {
  if (!cap) return;
  const uint32_t tiles = (cap + kStitchTile - 1) / kStitchTile;
  uint32_t* exitw = static_cast<uint32_t*>(temp);
  uint32_t* entry = exitw + uint64_t(tiles) * kWinMax;
  uint32_t* done = entry + tiles + 1;
  k_max_gap<<<grid_for(cap, 256, kSms * 2), 256, 0, st>>>(next, n_dev, gap); count_launches(1);
  cudaMemsetAsync(flags, 0, cap + 1, st);  // the walk path sets only the chain's flags
  k_stitch_win<<<grid_for(tiles, 1, kSms * 8), 256, 0, st>>>(next, n_dev, gap, exitw); count_launches(1);
  smem_optin(k_stitch_compose, kCombSmem);
  k_stitch_compose<<<1, 1024, kCombSmem, st>>>(exitw, n_dev, gap, entry, done);
  k_stitch_combine<<<1, 256, 0, st>>>(exitw, n_dev, gap, entry, done); count_launches(2);
  k_stitch_mark<<<grid_for(tiles, 1, kSms * 8), 128, 0, st>>>(next, n_dev, gap, entry, flags); count_launches(1);
  k_stitch_walk<<<grid_for(n_jobs, 8, kSms * 8), 256, 0, st>>>(next, gap, jobs, n_jobs, blocks_level, flags);
  count_launches(1);
}

void launch_compact_flags(const uint8_t* flags, const uint32_t* pos, const uint32_t* n_dev, uint32_t cap,
                          uint32_t* starts, uint32_t* total_out, cudaStream_t st) {
  k_compact_flags<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(flags, pos, n_dev, starts, total_out); count_launches(1);
}

void launch_job_blocks(JobDev* jobs, uint32_t n_jobs, const uint32_t* bpos, cudaStream_t st) {
  k_job_blocks<<<grid_for(n_jobs, 128), 128, 0, st>>>(jobs, n_jobs, bpos); count_launches(1);
}

void launch_block_sizes(const uint32_t* blk_start, const Counts* cnt, uint32_t cap, const uint64_t* P,
                        const uint32_t* dr, Fmt fmt, uint64_t* bsz, uint64_t* disk, cudaStream_t st) {
  if (!cap) return;
  k_block_sizes<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(blk_start, cnt, P, dr, fmt, bsz, disk); count_launches(1);
}

void launch_file_next(const uint64_t* C, const Counts* cnt, uint32_t cap, const JobDev* jobs, uint32_t n_jobs,
                      Fmt fmt, uint32_t* next, cudaStream_t st) {
  if (!cap) return;
  k_file_next<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(C, cnt, jobs, n_jobs, fmt, next); count_launches(1);
}

void launch_job_files(JobDev* jobs, uint32_t n_jobs, const uint32_t* fpos, cudaStream_t st) {
  k_job_files<<<grid_for(n_jobs, 128), 128, 0, st>>>(jobs, n_jobs, fpos); count_launches(1);
}

void launch_block_file(const uint32_t* fpos, const Counts* cnt, uint32_t cap, uint32_t* blk_file, cudaStream_t st) {
  if (!cap) return;
  k_block_file<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(fpos, cnt, blk_file); count_launches(1);
}

void launch_index_sizes(const uint32_t* blk_start, const uint64_t* bsz, const uint64_t* C, const uint32_t* blk_file,
                        const uint32_t* file_start, const Counts* cnt, uint32_t cap, const uint32_t* surv, Recs recs,
                        const uint8_t* arena, Fmt fmt, uint32_t* ie, cudaStream_t st) {
  if (!cap) return;
  k_index_sizes<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(blk_start, bsz, C, blk_file, file_start,
                                                                           cnt, surv, recs, arena, fmt.flags, ie);
  count_launches(1);
}

void launch_filter_count(const uint32_t* file_start, const Counts* cnt, uint32_t cap, const uint64_t* C,
                         uint64_t* nfilt, cudaStream_t st) {
  if (!cap) return;
  k_filter_count<<<grid_for(cap, 128), 128, 0, st>>>(file_start, cnt, C, nfilt); count_launches(1);
}

void launch_filter_sizes(const uint64_t* fbase, const uint32_t* file_start, const uint32_t* blk_start,
                         const uint64_t* C, Counts* cnt, uint64_t slot_cap, Fmt fmt, uint64_t* fbytes,
                         uint64_t* fwords, cudaStream_t st) {
  k_filter_sizes<<<grid_for(slot_cap ? slot_cap : 1, 256), 256, 0, st>>>(fbase, file_start, blk_start, C, cnt,
                                                                        slot_cap, fmt, fbytes, fwords);
  count_launches(1);
}

void launch_file_layout(const uint32_t* file_start, const Counts* cnt, uint32_t cap, const uint32_t* blk_start,
                        const uint64_t* C, const uint64_t* IX, Fmt fmt, FiltArr fa, const JobDev* jobs,
                        uint32_t n_jobs, FileDesc* files, uint64_t* fsize, uint64_t* bmwords, cudaStream_t st) {
  if (!cap) return;
  k_file_layout<<<grid_for(cap, 128), 128, 0, st>>>(file_start, cnt, blk_start, C, IX, fmt, fa, jobs, n_jobs, files,
                                                    fsize, bmwords); count_launches(1);
}

void launch_file_offsets(FileDesc* files, Counts* cnt, uint32_t cap, const uint64_t* foff, const uint64_t* bmoff,
                         FiltArr fa, JobDev* jobs, uint32_t n_jobs, uint64_t out_cap, uint64_t bm_cap, DErr* errs,
                         cudaStream_t st) {
  k_file_offsets<<<grid_for(cap > n_jobs ? cap : n_jobs, 128), 128, 0, st>>>(files, cnt, foff, bmoff, fa, jobs,
                                                                             n_jobs, out_cap, bm_cap, errs);
  count_launches(1);
}

void launch_zero_bitmap(uint32_t* bitmap, const Counts* cnt, uint64_t cap_words, cudaStream_t st) {
  if (!cap_words) return;
  k_zero_words<<<grid_for(cap_words, 256), 256, 0, st>>>(bitmap, cnt, cap_words); count_launches(1);
}

// Buffer bytes of the staged encoder. A block's contents are below T plus its last entry,
// and an entry is at most key + value + 11 bytes (max_kv: largest key + value length of the
// inputs, 0 when unknown); staging adds up to 30 bytes of alignment per entry.
static void stg_sizes(uint32_t T, uint32_t max_kv, uint32_t* S, uint32_t* I) {
  uint64_t img = uint64_t(T) + (max_kv ? uint64_t(max_kv) + 11 : uint64_t(T)) + 64;
  uint64_t stage = img + (T / 4 > 1024 ? T / 4 : 1024);
  img = (img + 127) & ~uint64_t(127);
  stage = (stage + 127) & ~uint64_t(127);
  *I = uint32_t(img > 64 * 1024 ? 64 * 1024 : img);
  *S = uint32_t(stage > 64 * 1024 ? 64 * 1024 : stage);
}

void launch_encode(const uint32_t* blk_start, Counts* cnt, uint32_t cap, const uint32_t* blk_file,
                   const FileDesc* files, const uint64_t* C, const uint64_t* bsz, const uint32_t* surv,
                   const uint32_t* lcp, const uint32_t* sd, const uint32_t* dr, const EncDesc* ed, BlkEnc* bd,
                   Recs recs, const uint8_t* arena, Fmt fmt, uint32_t max_kv, uint8_t* out, uint64_t out_cap,
                   uint8_t* done, uint32_t* big, DErr* errs, CrcTabs tabs, cudaStream_t st) {
  if (!cap) return;
  uint32_t S, I;
  stg_sizes(fmt.T, max_kv, &S, &I);
  const uint32_t smem = ((kStgHead + 127) & ~127u) + 2 * S + I + 16;
  uint32_t per_sm = (227u * 1024u) / (smem + 1024u);
  per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
  if (tuning().encode_ctas_per_sm && tuning().encode_ctas_per_sm < per_sm) per_sm = tuning().encode_ctas_per_sm;
  smem_optin(k_encode_stg, smem);
  k_block_enc<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(blk_start, cnt, blk_file, files, C, bsz, out_cap, bd);
  k_encode_stg<<<kSms * per_sm, kStgThreads, smem, st>>>(cnt, bd, lcp, ed, fmt, out, out_cap, done, big, errs, S, I);
  count_launches(2);
}

void launch_block_crc(Counts* cnt, uint32_t cap, const uint32_t* blk_file, const FileDesc* files,
                      const uint64_t* C, const uint64_t* bsz, uint8_t* out, uint64_t out_cap, const uint8_t* done,
                      CrcTabs tabs, bool helper, cudaStream_t st) {
  const uint32_t ctas = helper ? kSms - tuning().crc_ctas : tuning().crc_ctas;
  if (!cap || !ctas) return;
  smem_optin(k_block_crc, kCrcSmem);
  k_block_crc<<<ctas, tuning().crc_warps * 32, kCrcSmem, st>>>(cnt, blk_file, files, C, bsz, out, out_cap, done,
                                                                tabs);
  count_launches(1);
}

void launch_block_trailer(const Counts* cnt, uint32_t cap, const BlkEnc* bd, const uint32_t* sd, const uint32_t* dr,
                          const EncDesc* ed, const uint32_t* vcrc, Fmt fmt, uint8_t* out, const uint8_t* done,
                          CrcTabs tabs, cudaStream_t st) {
  if (!cap) return;
  smem_optin(k_block_trailer, kTrlSmem);
  k_block_trailer<<<kSms, kTrlThreads, kTrlSmem, st>>>(cnt, bd, sd, dr, ed, vcrc, fmt, out, done, tabs);
  count_launches(1);
}

void launch_encode_big(const uint32_t* blk_start, Counts* cnt, uint32_t cap, const uint32_t* blk_file,
                       const FileDesc* files, const uint64_t* C, const uint64_t* bsz, const uint32_t* surv,
                       const uint32_t* lcp, const uint32_t* sd, const uint32_t* dr, Recs recs, const uint8_t* arena,
                       Fmt fmt, uint8_t* out, uint64_t out_cap, const uint32_t* big, CrcTabs tabs, cudaStream_t st) {
  if (!cap) return;
  smem_optin(k_encode_big, kEncBuf);
  k_encode_big<<<kSms, kEncThreads, kEncBuf, st>>>(blk_start, cnt, blk_file, files, C, bsz, surv, lcp, sd, dr, recs,
                                                   arena, fmt, out, out_cap, big, tabs);
  count_launches(1);
}

void launch_bloom(const EncDesc* ed, const Counts* cnt, uint32_t cap, const FileDesc* files, Fmt fmt,
                  const uint32_t* blk_start, const uint64_t* C, FiltArr fa, uint32_t* bitmap, uint64_t out_cap,
                  uint64_t bm_cap, cudaStream_t st) {
  if (!cap) return;
  k_bloom<<<grid_for(cap, elem_threads()), elem_threads(), 0, st>>>(ed, cnt, files, fmt, blk_start, C, fa, bitmap,
                                                                     out_cap, bm_cap);
  count_launches(1);
}

void launch_index_write(const uint32_t* blk_start, const Counts* cnt, uint32_t cap, const uint64_t* bsz,
                        const uint64_t* C, const uint64_t* IX, const uint32_t* blk_file, const FileDesc* files,
                        const uint32_t* surv, Recs recs, const uint8_t* arena, Fmt fmt, uint8_t* out,
                        uint64_t out_cap, cudaStream_t st) {
  if (!cap) return;
  k_index_write<<<grid_for(cap, 128), 128, 0, st>>>(blk_start, cnt, bsz, C, IX, blk_file, files, surv, recs, arena,
                                                    fmt.flags, out, out_cap);
  count_launches(1);
}

void launch_file_finish(const FileDesc* files, const Counts* cnt, uint32_t cap, const uint32_t* bitmap,
                        const uint32_t* surv, Recs recs, Fmt fmt, FiltArr fa, uint8_t* out, uint64_t out_cap,
                        CrcTabs tabs, CrcMsg* msgs, FileMeta* meta, cudaStream_t st) {
  if (!cap) return;
  k_filter_copy<<<kSms * 4, 256, 0, st>>>(files, cnt, fa, bitmap, out, out_cap);
  if (fa.base) {
    k_filter_tail<<<grid_for(fa.cap ? fa.cap : 1, 256), 256, 0, st>>>(files, cnt, fa, fmt, out, out_cap);
    count_launches(1);
  }
  k_file_finish<<<grid_for(cap, 128, kSms), 128, 0, st>>>(files, cnt, surv, recs, fmt, out, out_cap, msgs, meta);
  count_launches(2);
  launch_msg_crc(msgs, &cnt->nf, 3, 3 * cap, nullptr, tabs, st);
}

void launch_key_lens(const FileMeta* meta, const Counts* cnt, uint32_t cap, uint64_t* lens, cudaStream_t st) {
  if (!cap) return;
  k_key_lens<<<grid_for(cap, 128), 128, 0, st>>>(meta, cnt, lens); count_launches(1);
}

void launch_key_gather(FileMeta* meta, Counts* cnt, uint32_t cap, const uint64_t* koff, const FileDesc* files,
                       const uint32_t* surv, Recs recs, const uint8_t* arena, uint8_t* keybuf, cudaStream_t st) {
  k_key_gather<<<grid_for(cap ? cap : 1, 128), 128, 0, st>>>(meta, cnt, koff, files, surv, recs, arena, keybuf); count_launches(1);
}

void launch_build_records(const uint8_t* ukeys, const uint64_t* ukoff, const uint64_t* seqs, const uint8_t* types,
                          const uint8_t* vals, const uint64_t* voff, uint32_t n, Recs recs, uint8_t* arena,
                          uint32_t* surv, DErr* err, cudaStream_t st) {
  if (!n) return;
  k_build_records<<<grid_for(n, 256), 256, 0, st>>>(ukeys, ukoff, seqs, types, vals, voff, n, recs, arena, surv, err); count_launches(1);
}

void launch_build_check(Recs recs, const uint8_t* arena, uint32_t n, DErr* err, cudaStream_t st) {
  if (n < 2) return;
  k_build_check<<<grid_for(n, 256), 256, 0, st>>>(recs, arena, n, err); count_launches(1);
}

void launch_compress_blocks(PackCz z, JobDev* jobs, uint32_t n_jobs, Counts* cnt, uint32_t cap, uint64_t* bsz,
                            uint64_t* disk, void* scan_tmp, cudaStream_t st) {
  if (!cap) return;
  k_raw_sizes<<<grid_for(cap, 256), 256, 0, st>>>(cnt, bsz, z.rawsz, z.czsz);
  count_launches(1);
  exclusive_scan<uint64_t, uint64_t>(z.rawsz, z.Craw, cap, &cnt->nb, scan_tmp, st);
  exclusive_scan<uint64_t, uint64_t>(z.czsz, z.Cc, cap, &cnt->nb, scan_tmp, st);
  k_raw_files<<<grid_for(cap > n_jobs ? cap : n_jobs, 256), 256, 0, st>>>(jobs, n_jobs, cnt, z.Craw, z.rfiles, z.rbf);
  count_launches(1);
}

void launch_compress(PackCz z, Counts* cnt, uint32_t cap, uint64_t* bsz, uint64_t* disk, cudaStream_t st) {
  if (!cap) return;
  // blocks below 64 KiB (nearly all) with 16-bit positions, the others with 32-bit ones
  constexpr uint32_t s16 = kCzWarps16 * cz_warp_smem<uint16_t>(), s32 = kCzWarps32 * cz_warp_smem<uint32_t>();
  constexpr uint32_t scp = kCzCopyWarps * cz_copy_smem();
  smem_optin(k_compress_copy, scp);
  smem_optin(k_compress<uint16_t, kCzWarps16>, s16);
  smem_optin(k_compress<uint32_t, kCzWarps32>, s32);
  k_compress_copy<<<grid_for(uint64_t(cap) * 32, kCzCopyWarps * 32), kCzCopyWarps * 32, scp, st>>>(
      cnt, z.Craw, z.Cc, bsz, disk, z.raw, z.raw_cap, z.cz, z.c_cap, z.ctype);
  k_compress<uint16_t, kCzWarps16><<<grid_for(uint64_t(cap) * 32, kCzWarps16 * 32), kCzWarps16 * 32, s16, st>>>(
      cnt, z.Craw, z.Cc, bsz, disk, z.raw, z.raw_cap, z.cz, z.c_cap, z.ctype);
  k_compress<uint32_t, kCzWarps32><<<grid_for(uint64_t(cap) * 32, kCzWarps32 * 32), kCzWarps32 * 32, s32, st>>>(
      cnt, z.Craw, z.Cc, bsz, disk, z.raw, z.raw_cap, z.cz, z.c_cap, z.ctype);
  count_launches(3);
}

void launch_place(PackCz z, Counts* cnt, uint32_t cap, const uint32_t* blk_file, const FileDesc* files,
                  const uint64_t* C, const uint64_t* bsz, uint8_t* out, uint64_t out_cap, uint8_t* done,
                  cudaStream_t st) {
  if (!cap) return;
  k_place<<<grid_for(uint64_t(cap) * 32, 256), 256, 0, st>>>(cnt, blk_file, files, C, bsz, z.Craw, z.Cc, z.raw,
                                                             z.cz, z.ctype, out, out_cap, done);
  count_launches(1);
}

}  // namespace luda
