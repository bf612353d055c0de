// sort.cu -- Phase 2 "(Delete and) Sort" (LUDA §II-A; §III-C, §III-D).
//
// Every input table is already a sorted run (and consecutive inputs whose key ranges do
// not overlap form one run), so the total order is reached by merging runs pairwise
// (merge path: each output tile finds its split of the two runs, then merges it in shared
// memory). Runs that a pass does not merge stay in their buffer. The paper sorted
// <K, V_offset> tuples on the host because it found no fast GPU sort for them (§III-D
// "Cooperative Sort"); here the tuples (record id plus a 32-byte key head) never leave the
// device.
//
// The drop rule then keeps entry i unless a newer version of the same user key is
// visible at the smallest snapshot S, or it is a tombstone visible at S in a bottommost
// job (LevelDB's compaction rule: seq_{i-1} <= S for the same user key, or DEL with
// seq_i <= S and bottommost).
#include <cstdint>

#include "internal.cuh"

namespace luda {

namespace {

// Internal-key compare without the record-id tie-break (strict order inside an input).
__device__ __forceinline__ int cmp_ikey(const Recs& r, const uint8_t* arena, uint32_t a, uint32_t b) {
  const uint64_t pa = r.pfx[a], pb = r.pfx[b];
  if (pa != pb) return pa < pb ? -1 : 1;
  return cmp_tail(r, arena, a, b, 8, false);
}

// Merge key: the first 32 bytes of the user key (big-endian words, zero-padded); ties on
// it are resolved from the key arena.
__device__ __forceinline__ int cmp_mkey(const Recs& r, const uint8_t* arena, uint32_t a, const MKey& ka, uint32_t b,
                                        const MKey& kb) {
#pragma unroll
  for (int w = 0; w < 4; ++w)
    if (ka.h[w] != kb.h[w]) return ka.h[w] < kb.h[w] ? -1 : 1;
  if (a == b) return 0;
  return cmp_tail(r, arena, a, b, 32);
}

__global__ void k_check_order(Recs recs, const uint8_t* __restrict__ arena, uint32_t n_rec,
                              const DInput* __restrict__ in, DErr* errs) {
  for (uint64_t i = gtid() + 1; i < n_rec; i += gstride()) {
    const uint32_t s = recs.src[i];
    if (s != recs.src[i - 1]) continue;
    if (cmp_ikey(recs, arena, uint32_t(i - 1), uint32_t(i)) >= 0) {
      const DInput d = in[s];
      report(errs + d.job, E_CORRUPT, d.local, 0);
    }
  }
}

__global__ void k_sort_init(uint32_t* __restrict__ ord, MKey* __restrict__ okey, Recs recs,
                            const uint8_t* __restrict__ arena, uint32_t n) {
  for (uint64_t i = gtid(); i < n; i += gstride()) {
    ord[i] = uint32_t(i);
    const uint32_t ul = recs.klen[i] - 8;
    const uint8_t* k = arena + recs.koff[i];
    MKey m;
    m.h[0] = recs.pfx[i];
#pragma unroll
    for (uint32_t w = 1; w < 4; ++w) m.h[w] = key_word(k + 8 * w, ul > 8 * w ? ul - 8 * w : 0u);
    okey[i] = m;
  }
}

constexpr int kMergeThreads = 128;

// Co-rank of output position d in the merge of A and B, found by the whole CTA: while the
// candidate range is wider than the CTA, every thread tests one of kMergeThreads evenly
// spaced split points ("A[i] goes before B[d-1-i]" is true up to the answer, then false)
// and the count of true tests narrows the range (about three rounds for a million
// elements, instead of twenty dependent steps of a binary search).
__device__ uint32_t corank_cta(uint32_t d, const uint32_t* A, const MKey* Ak, uint32_t na, const uint32_t* B,
                               const MKey* Bk, uint32_t nb, const Recs& recs, const uint8_t* arena) {
  uint32_t lo = d > nb ? d - nb : 0;
  uint32_t hi = d < na ? d : na;
  const uint32_t t = threadIdx.x;
  while (hi > lo) {
    const uint32_t span = hi - lo;
    if (span <= uint32_t(kMergeThreads)) {
      const uint32_t i = lo + t;
      bool p = false;
      if (t < span) p = cmp_mkey(recs, arena, A[i], Ak[i], B[d - i - 1], Bk[d - i - 1]) < 0;
      return lo + uint32_t(__syncthreads_count(p));
    }
    const uint32_t step = (span + kMergeThreads) / (kMergeThreads + 1);
    const uint32_t i = lo + (t + 1) * step - 1;
    bool p = false;
    if (i < hi) p = cmp_mkey(recs, arena, A[i], Ak[i], B[d - i - 1], Bk[d - i - 1]) < 0;
    const uint32_t c = uint32_t(__syncthreads_count(p));
    // tests 0..c-1 were true: the answer is past test c-1; test c (if any) was false or
    // past hi: the answer is at most its index
    const uint32_t nlo = c ? lo + c * step : lo;
    if (c < uint32_t(kMergeThreads)) {
      const uint32_t nhi = lo + (c + 1) * step - 1;
      hi = nhi < hi ? nhi : hi;
    }
    lo = nlo;
  }
  return lo;
}

// Co-rank inside shared memory (binary search, one thread).
__device__ __forceinline__ uint32_t corank_smem(uint32_t d, const uint32_t* A, const MKey* Ak, uint32_t na,
                                                const uint32_t* B, const MKey* Bk, uint32_t nb, const Recs& recs,
                                                const uint8_t* arena) {
  uint32_t lo = d > nb ? d - nb : 0;
  uint32_t hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t bj = d - mid - 1;
    if (cmp_mkey(recs, arena, A[mid], Ak[mid], B[bj], Bk[bj]) < 0) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t find_span(const MergeSpan* spans, uint32_t n_spans, uint32_t tile) {
  uint32_t lo = 0, hi = n_spans;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (spans[mid].tile_first <= tile) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One CTA per output tile of kTile elements: co-rank both ends of the tile, stage the
// tile's parts of A and B in shared memory (keys first, 16-byte aligned, then the ids),
// then each thread co-ranks its kTile / kMergeThreads outputs there and merges them.
template <uint32_t kTile>
__global__ void __launch_bounds__(kMergeThreads) k_merge(const MergeSpan* __restrict__ spans, uint32_t n_spans,
                                                         uint32_t n_tiles, uint32_t* ord0, MKey* key0, uint32_t* ord1,
                                                         MKey* key1, Recs recs, const uint8_t* __restrict__ arena) {
  constexpr uint32_t kItems = kTile / kMergeThreads;
  extern __shared__ uint4 s_merge[];
  MKey* s_key = reinterpret_cast<MKey*>(s_merge);
  uint32_t* s_ord = reinterpret_cast<uint32_t*>(s_key + kTile);
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const MergeSpan sp = spans[find_span(spans, n_spans, t)];
    const uint32_t* src_ord = sp.src ? ord1 : ord0;
    const MKey* src_key = sp.src ? key1 : key0;
    uint32_t* dst_ord = sp.src ? ord0 : ord1;
    MKey* dst_key = sp.src ? key0 : key1;
    const uint32_t total = sp.a_len + sp.b_len;
    const uint32_t d0 = (t - sp.tile_first) * kTile;
    const uint32_t d1 = min(d0 + kTile, total);
    const uint32_t* A = src_ord + sp.a_begin;
    const MKey* Ak = src_key + sp.a_begin;
    const uint32_t* B = A + sp.a_len;
    const MKey* Bk = Ak + sp.a_len;
    const uint32_t i0 = corank_cta(d0, A, Ak, sp.a_len, B, Bk, sp.b_len, recs, arena);
    const uint32_t i1 = d1 == total ? sp.a_len : corank_cta(d1, A, Ak, sp.a_len, B, Bk, sp.b_len, recs, arena);
    const uint32_t j0 = d0 - i0, j1 = d1 - i1;
    const uint32_t na = i1 - i0, nb = j1 - j0;
    {
      // all of a thread's loads first, then the shared stores (one memory latency per tile)
      uint32_t ro[kItems];
      MKey rk[kItems];
#pragma unroll
      for (uint32_t k = 0; k < kItems; ++k) {
        const uint32_t x = threadIdx.x + k * kMergeThreads;
        if (x < na + nb) {
          const uint32_t src = x < na ? i0 + x : sp.a_len + j0 + (x - na);
          ro[k] = A[src];
          rk[k] = Ak[src];
        }
      }
#pragma unroll
      for (uint32_t k = 0; k < kItems; ++k) {
        const uint32_t x = threadIdx.x + k * kMergeThreads;
        if (x < na + nb) {
          s_ord[x] = ro[k];
          s_key[x] = rk[k];
        }
      }
    }
    __syncthreads();
    const uint32_t dd = threadIdx.x * kItems;
    if (dd < na + nb) {
      const uint32_t ia = corank_smem(dd, s_ord, s_key, na, s_ord + na, s_key + na, nb, recs, arena);
      uint32_t a = ia, ib = dd - ia;
      const uint32_t cnt = min(kItems, na + nb - dd);
      uint32_t out = sp.a_begin + d0 + dd;
      for (uint32_t k = 0; k < cnt; ++k, ++out) {
        bool take_a;
        if (a >= na) take_a = false;
        else if (ib >= nb) take_a = true;
        else take_a = cmp_mkey(recs, arena, s_ord[a], s_key[a], s_ord[na + ib], s_key[na + ib]) < 0;
        const uint32_t x = take_a ? a++ : na + ib++;
        dst_ord[out] = s_ord[x];
        dst_key[out] = s_key[x];
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ uint32_t find_job(const JobDev* jobs, uint32_t n_jobs, uint32_t p, bool by_surv) {
  uint32_t lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((by_surv ? jobs[mid].surv_begin : jobs[mid].rec_begin) <= p) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_gc_flags(const uint32_t* __restrict__ ord, uint32_t n_rec, const JobDev* __restrict__ jobs,
                           uint32_t n_jobs, Recs recs, const uint8_t* __restrict__ arena, uint32_t* __restrict__ keep,
                           DErr* errs, const JobRange* __restrict__ ranges, const uint8_t* __restrict__ bounds) {
  for (uint64_t p = gtid(); p < n_rec; p += gstride()) {
    const uint32_t j = find_job(jobs, n_jobs, uint32_t(p), false);
    const JobDev job = jobs[j];
    if (*(volatile int32_t*)&errs[j].code != 0) {
      keep[p] = 0;
      continue;
    }
    const uint32_t x = ord[p];
    const uint64_t tr = recs.tr[x];
    const uint64_t S = job.snapshot;
    bool drop = false;
    if (ranges && ranges[j].flags && !key_in_range(ranges[j], bounds, arena + recs.koff[x], recs.klen[x] - 8)) {
      keep[p] = 0;  // R13: only keys of the job's range are written
      continue;
    }
    if (p > job.rec_begin) {
      const uint32_t y = ord[p - 1];
      if (same_user_key(recs, arena, y, x)) {
        const uint64_t tp = recs.tr[y];
        if ((tp >> 8) <= S) drop = true;
        if ((job.flags & 1u) && tp == tr) report(errs + j, E_DUP, ~0u, p);
      }
    }
    if (!drop && (tr & 0xFF) == 0 && (tr >> 8) <= S && job.bottommost) drop = true;
    keep[p] = drop ? 0u : 1u;
  }
}

__global__ void k_gc_compact(const uint32_t* __restrict__ ord, const uint32_t* __restrict__ keep,
                             const uint32_t* __restrict__ pos, uint32_t n_rec, uint32_t* __restrict__ surv) {
  for (uint64_t p = gtid(); p < n_rec; p += gstride())
    if (keep[p]) surv[pos[p]] = ord[p];
}

__global__ void k_job_surv(JobDev* jobs, uint32_t n_jobs, const uint32_t* __restrict__ pos, uint32_t n_rec,
                           Counts* cnt) {
  for (uint64_t j = gtid(); j < n_jobs; j += gstride()) {
    jobs[j].surv_begin = pos[jobs[j].rec_begin];
    jobs[j].surv_end = pos[jobs[j].rec_end];
  }
  if (gtid() == 0) cnt->n_surv = pos[n_rec];
}

// Plans: records of a job that failed before decode are left undefined; give them a
// harmless value (an 8-byte key at arena offset 0, no value) so later kernels stay in bounds.
__global__ void k_plan_sanitize(Recs recs, uint32_t n_rec, const JobDev* __restrict__ jobs, uint32_t n_jobs,
                                const DErr* errs, const uint8_t* __restrict__ arena) {
  for (uint64_t p = gtid(); p < n_rec; p += gstride()) {
    const uint32_t j = find_job(jobs, n_jobs, uint32_t(p), false);
    if (errs[j].code == 0) continue;
    recs.pfx[p] = 0;
    recs.koff[p] = 0;
    recs.klen[p] = 8;
    recs.tr[p] = 0;
    recs.vptr[p] = reinterpret_cast<uint64_t>(arena);
    recs.vlen[p] = 0;
    recs.src[p] = jobs[j].in_first;
  }
}

}  // namespace

void launch_plan_sanitize(Recs recs, uint32_t n_rec, const JobDev* jobs, uint32_t n_jobs, const DErr* errs,
                          const uint8_t* arena, cudaStream_t st) {
  if (!n_rec) return;
  k_plan_sanitize<<<grid_for(n_rec, 256), 256, 0, st>>>(recs, n_rec, jobs, n_jobs, errs, arena);
  count_launches(1);
}

void launch_check_order(Recs recs, const uint8_t* arena, uint32_t n_rec, const DInput* in, DErr* errs,
                        cudaStream_t st) {
  if (n_rec < 2) return;
  k_check_order<<<grid_for(n_rec, elem_threads()), elem_threads(), 0, st>>>(recs, arena, n_rec, in, errs); count_launches(1);
}

void launch_sort_init(uint32_t* ord, MKey* okey, Recs recs, const uint8_t* arena, uint32_t n, cudaStream_t st) {
  if (!n) return;
  k_sort_init<<<grid_for(n, elem_threads()), elem_threads(), 0, st>>>(ord, okey, recs, arena, n); count_launches(1);
}

template <uint32_t kTile>
void merge_pass_t(const MergeSpan* spans, uint32_t n_spans, uint32_t n_tiles, uint32_t* ord0, MKey* key0,
                  uint32_t* ord1, MKey* key1, Recs recs, const uint8_t* arena, cudaStream_t st) {
  constexpr uint32_t smem = kTile * (sizeof(MKey) + sizeof(uint32_t));
  if (smem > 48u * 1024u) smem_optin(k_merge<kTile>, smem);
  k_merge<kTile><<<grid_for(n_tiles, 1, kSms * tuning().merge_ctas_per_sm), kMergeThreads, smem, st>>>(
      spans, n_spans, n_tiles, ord0, key0, ord1, key1, recs, arena);
}

void launch_merge_pass(const MergeSpan* spans, uint32_t n_spans, uint32_t n_tiles, uint32_t tile, uint32_t* ord0,
                       MKey* key0, uint32_t* ord1, MKey* key1, Recs recs, const uint8_t* arena, cudaStream_t st) {
  if (!n_tiles) return;
  switch (tile) {
    case 512: merge_pass_t<512>(spans, n_spans, n_tiles, ord0, key0, ord1, key1, recs, arena, st); break;
    case 2048: merge_pass_t<2048>(spans, n_spans, n_tiles, ord0, key0, ord1, key1, recs, arena, st); break;
    default: merge_pass_t<1024>(spans, n_spans, n_tiles, ord0, key0, ord1, key1, recs, arena, st); break;
  }
  count_launches(1);
}

void launch_gc_flags(const uint32_t* ord, uint32_t n_rec, const JobDev* jobs, uint32_t n_jobs, Recs recs,
                     const uint8_t* arena, uint32_t* keep, DErr* errs, cudaStream_t st, const JobRange* ranges,
                     const uint8_t* bounds) {
  if (!n_rec) return;
  k_gc_flags<<<grid_for(n_rec, elem_threads()), elem_threads(), 0, st>>>(ord, n_rec, jobs, n_jobs, recs, arena, keep,
                                                                         errs, ranges, bounds);
  count_launches(1);
}

void launch_gc_compact(const uint32_t* ord, const uint32_t* keep, const uint32_t* pos, uint32_t n_rec,
                       uint32_t* surv, cudaStream_t st) {
  if (!n_rec) return;
  k_gc_compact<<<grid_for(n_rec, elem_threads()), elem_threads(), 0, st>>>(ord, keep, pos, n_rec, surv); count_launches(1);
}

void launch_job_surv(JobDev* jobs, uint32_t n_jobs, const uint32_t* pos, uint32_t n_rec, Counts* cnt,
                     cudaStream_t st) {
  k_job_surv<<<grid_for(n_jobs, 128), 128, 0, st>>>(jobs, n_jobs, pos, n_rec, cnt); count_launches(1);
}

}  // namespace luda
