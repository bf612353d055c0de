// sort.cu -- Phase 2 "(Delete and) Sort" (LUDA §II-A; §III-C, §III-D).
//
// Every input table is already a sorted run, so the total order is reached by merging
// runs pairwise (merge path: each output tile finds its split of the two runs by binary
// search, then merges it in shared memory). The paper sorted <K, V_offset> tuples on the
// host because it found no fast GPU sort for them (§III-D "Cooperative Sort"); here the
// tuples (record id plus an 8-byte key prefix) never leave the device.
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

// Merge key: the first 16 bytes of the user key (big-endian words, zero-padded); ties on
// it are resolved from the key arena.
__device__ __forceinline__ int cmp_mkey(const Recs& r, const uint8_t* arena, uint32_t a, const MKey& ka, uint32_t b,
                                        const MKey& kb) {
  if (ka.h0 != kb.h0) return ka.h0 < kb.h0 ? -1 : 1;
  if (ka.h1 != kb.h1) return ka.h1 < kb.h1 ? -1 : 1;
  if (a == b) return 0;
  return cmp_tail(r, arena, a, b, 16);
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
    okey[i] = MKey{recs.pfx[i], key_word(arena + recs.koff[i] + 8, ul > 8 ? ul - 8 : 0u)};
  }
}

// Co-rank of output position d in the merge of A (len na) and B (len nb): the number of
// A elements among the first d outputs.
__device__ __forceinline__ uint32_t corank(uint32_t d, const uint32_t* A, const MKey* Ap, uint32_t na,
                                           const uint32_t* B, const MKey* Bp, uint32_t nb, const Recs& recs,
                                           const uint8_t* arena) {
  uint32_t lo = d > nb ? d - nb : 0;
  uint32_t hi = d < na ? d : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t bj = d - mid - 1;
    if (cmp_mkey(recs, arena, A[mid], Ap[mid], B[bj], Bp[bj]) < 0) lo = mid + 1;
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

__global__ void k_merge_partition(const MergeSpan* __restrict__ spans, uint32_t n_spans, uint32_t n_tiles,
                                  uint32_t* __restrict__ co, const uint32_t* __restrict__ ord,
                                  const MKey* __restrict__ pfx, Recs recs, const uint8_t* __restrict__ arena) {
  for (uint64_t t = gtid(); t < n_tiles; t += gstride()) {
    const MergeSpan sp = spans[find_span(spans, n_spans, uint32_t(t))];
    const uint32_t d = uint32_t(t - sp.tile_first) * kMergeTile;
    const uint32_t* A = ord + sp.a_begin;
    co[t] = corank(d, A, pfx + sp.a_begin, sp.a_len, A + sp.a_len, pfx + sp.a_begin + sp.a_len, sp.b_len, recs,
                   arena);
  }
}

constexpr int kMergeThreads = 128;
constexpr int kMergeItems = kMergeTile / kMergeThreads;

__global__ void __launch_bounds__(kMergeThreads) k_merge_tiles(const MergeSpan* __restrict__ spans, uint32_t n_spans,
                                                               uint32_t n_tiles, const uint32_t* __restrict__ co,
                                                               const uint32_t* __restrict__ src_ord,
                                                               const MKey* __restrict__ src_pfx,
                                                               uint32_t* __restrict__ dst_ord,
                                                               MKey* __restrict__ dst_pfx, Recs recs,
                                                               const uint8_t* __restrict__ arena) {
  __shared__ uint32_t s_ord[kMergeTile];
  __shared__ MKey s_pfx[kMergeTile];
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint32_t si = find_span(spans, n_spans, t);
    const MergeSpan sp = spans[si];
    const uint32_t total = sp.a_len + sp.b_len;
    const uint32_t d0 = (t - sp.tile_first) * kMergeTile;
    const uint32_t d1 = min(d0 + kMergeTile, total);
    const uint32_t last_tile = (si + 1 < n_spans ? spans[si + 1].tile_first : n_tiles) - 1;
    const uint32_t i0 = co[t];
    const uint32_t i1 = t < last_tile ? co[t + 1] : sp.a_len;
    const uint32_t j0 = d0 - i0, j1 = d1 - i1;
    const uint32_t na = i1 - i0, nb = j1 - j0;
    const uint32_t a_base = sp.a_begin + i0, b_base = sp.a_begin + sp.a_len + j0;
    for (uint32_t x = threadIdx.x; x < na + nb; x += blockDim.x) {
      const uint32_t src = x < na ? a_base + x : b_base + (x - na);
      s_ord[x] = src_ord[src];
      s_pfx[x] = src_pfx[src];
    }
    __syncthreads();
    const uint32_t dd = threadIdx.x * kMergeItems;
    if (dd < na + nb) {
      const uint32_t ia = corank(dd, s_ord, s_pfx, na, s_ord + na, s_pfx + na, nb, recs, arena);
      uint32_t ib = dd - ia;
      uint32_t a = ia;
      const uint32_t cnt = min(uint32_t(kMergeItems), na + nb - dd);
      uint32_t out = sp.a_begin + d0 + dd;
      for (uint32_t k = 0; k < cnt; ++k, ++out) {
        bool take_a;
        if (a >= na) take_a = false;
        else if (ib >= nb) take_a = true;
        else take_a = cmp_mkey(recs, arena, s_ord[a], s_pfx[a], s_ord[na + ib], s_pfx[na + ib]) < 0;
        if (take_a) {
          dst_ord[out] = s_ord[a];
          dst_pfx[out] = s_pfx[a];
          ++a;
        } else {
          dst_ord[out] = s_ord[na + ib];
          dst_pfx[out] = s_pfx[na + ib];
          ++ib;
        }
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
                           DErr* errs) {
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
  k_check_order<<<grid_for(n_rec, 256), 256, 0, st>>>(recs, arena, n_rec, in, errs); count_launches(1);
}

void launch_sort_init(uint32_t* ord, MKey* okey, Recs recs, const uint8_t* arena, uint32_t n, cudaStream_t st) {
  if (!n) return;
  k_sort_init<<<grid_for(n, 256), 256, 0, st>>>(ord, okey, recs, arena, n); count_launches(1);
}

void launch_merge_pass(const MergeSpan* spans, uint32_t n_spans, uint32_t n_tiles, uint32_t* corank_buf,
                       const uint32_t* src_ord, const MKey* src_pfx, uint32_t* dst_ord, MKey* dst_pfx,
                       Recs recs, const uint8_t* arena, cudaStream_t st) {
  if (!n_tiles) return;
  k_merge_partition<<<grid_for(n_tiles, 128), 128, 0, st>>>(spans, n_spans, n_tiles, corank_buf, src_ord, src_pfx,
                                                            recs, arena); count_launches(1);
  k_merge_tiles<<<grid_for(n_tiles, 1, kSms * 8), kMergeThreads, 0, st>>>(spans, n_spans, n_tiles, corank_buf,
                                                                          src_ord, src_pfx, dst_ord, dst_pfx, recs,
                                                                          arena); count_launches(1);
}

void launch_gc_flags(const uint32_t* ord, uint32_t n_rec, const JobDev* jobs, uint32_t n_jobs, Recs recs,
                     const uint8_t* arena, uint32_t* keep, DErr* errs, cudaStream_t st) {
  if (!n_rec) return;
  k_gc_flags<<<grid_for(n_rec, 256), 256, 0, st>>>(ord, n_rec, jobs, n_jobs, recs, arena, keep, errs); count_launches(1);
}

void launch_gc_compact(const uint32_t* ord, const uint32_t* keep, const uint32_t* pos, uint32_t n_rec,
                       uint32_t* surv, cudaStream_t st) {
  if (!n_rec) return;
  k_gc_compact<<<grid_for(n_rec, 256), 256, 0, st>>>(ord, keep, pos, n_rec, surv); count_launches(1);
}

void launch_job_surv(JobDev* jobs, uint32_t n_jobs, const uint32_t* pos, uint32_t n_rec, Counts* cnt,
                     cudaStream_t st) {
  k_job_surv<<<grid_for(n_jobs, 128), 128, 0, st>>>(jobs, n_jobs, pos, n_rec, cnt); count_launches(1);
}

}  // namespace luda
