// keep.cu -- decoded runs kept on the device between compactions (LUDA §III-D: data stays
// in GPU memory so that it is not moved again between jobs).
//
// When a compaction or a table build runs with LUDA_F_KEEP_DECODED, the survivors it has
// just written are kept as a sorted run: each survivor's record (key prefix, trailer, key
// and value lengths, the value's CRC-32C register), its full internal key (in output
// order, in the store's own key arena) and the address of its value inside the new data
// blocks (read back from the written blocks). A later compaction whose inputs are all
// tables with kept runs takes its records from the stores: one gather kernel and one key
// copy per input replace the footer, index, block walk, checksum and key kernels (§II-A
// Phase 1 runs once per table, when the table is written).
#include <cstdint>

#include "internal.cuh"

namespace luda {

namespace {

// store.klen of every survivor (the key lengths the key offsets are scanned from)
__global__ void k_keep_lens(const Counts* __restrict__ cnt, const EncDesc* __restrict__ ed, KeptRecs K) {
  const uint32_t n = cnt->n_surv;
  for (uint64_t s = gtid(); s < n; s += gstride()) K.klen[s] = ed[s].klen;
}

// Every survivor's record and full internal key into the store (output order).
__global__ void k_keep_recs(const Counts* __restrict__ cnt, const EncDesc* __restrict__ ed, Recs recs, KeptRecs K) {
  const uint32_t n = cnt->n_surv;
  for (uint64_t s = gtid(); s < n; s += gstride()) {
    const EncDesc e = ed[s];
    K.pfx[s] = recs.pfx[e.rec];
    K.tr[s] = recs.tr[e.rec];
    K.vlen[s] = e.vlen;
    K.vcrc[s] = recs.vcrc[e.rec];
    const uint8_t* src = reinterpret_cast<const uint8_t*>(e.kptr);
    uint8_t* dst = K.arena + K.koff[s];
    for (uint32_t i = 0; i < e.klen; ++i) dst[i] = src[i];
  }
}

// Per new table: where its keys start in the store and how many bytes they take; the
// largest key + value length starts at 0 (k_keep_values raises it).
__global__ void k_keep_files(const Counts* __restrict__ cnt, const FileDesc* __restrict__ files, KeptRecs K,
                             FileMeta* __restrict__ meta) {
  const uint32_t nf = cnt->nf;
  for (uint64_t f = gtid(); f < nf; f += gstride()) {
    const FileDesc F = files[f];
    meta[f].key_first = K.koff[F.ent_begin];
    meta[f].kbytes = K.koff[F.ent_end] - K.koff[F.ent_begin];
    meta[f].max_kv = 0;
  }
}

// The address of every survivor's value inside its data block: a warp per written block,
// its first lane walking the entries (three varints, the key delta, the value); the
// block's largest key + value length raises its table's max_kv.
__global__ void k_keep_values(const Counts* __restrict__ cnt, const BlkEnc* __restrict__ bd,
                              const uint32_t* __restrict__ blk_file, const uint8_t* __restrict__ out, KeptRecs K,
                              FileMeta* __restrict__ meta) {
  const uint32_t nb = cnt->nb;
  const uint64_t warps = gstride() / 32;
  for (uint64_t b = gtid() / 32; b < nb; b += warps) {
    if ((threadIdx.x & 31u) != 0) continue;
    const BlkEnc d = bd[b];
    if (d.job & 0x80000000u) continue;  // outside the arena: the job fails
    const uint8_t* p = out + d.dst;
    const uint8_t* end = p + d.contents;
    uint32_t mkv = 0;
    for (uint32_t j = 0; j < d.m && p < end; ++j) {
      uint64_t shared = 0, nonshared = 0, vlen = 0;
      p += get_varint<32>(p, end, &shared);
      p += get_varint<32>(p, end, &nonshared);
      p += get_varint<32>(p, end, &vlen);
      K.vptr[d.s0 + j] = reinterpret_cast<uint64_t>(p + nonshared);
      const uint64_t kv = shared + nonshared + vlen;
      mkv = kv > mkv ? uint32_t(kv) : mkv;
      p += nonshared + vlen;
    }
    atomicMax(&meta[blk_file[b]].max_kv, mkv);
  }
}

// The records of input blockIdx.y from its kept run: fields copied, the key offset moved
// to where the input's keys are copied in the call's arena, the input index set.
__global__ void k_kept_gather(const KeptIn* __restrict__ ins, Recs recs) {
  const KeptIn I = ins[blockIdx.y];
  for (uint64_t r = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < I.count;
       r += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t s = I.first + r, d = I.rec_base + r;
    recs.pfx[d] = I.run.pfx[s];
    recs.tr[d] = I.run.tr[s];
    recs.klen[d] = I.run.klen[s];
    recs.vlen[d] = I.run.vlen[s];
    recs.vptr[d] = I.run.vptr[s];
    recs.vcrc[d] = I.run.vcrc[s];
    recs.koff[d] = I.key_base + (I.run.koff[s] - I.key_first);
    recs.src[d] = blockIdx.y;
  }
}

}  // namespace

cudaError_t launch_keep(const Counts* cnt, uint32_t cap, const EncDesc* ed, Recs recs, const FileDesc* files,
                        const BlkEnc* bd, const uint32_t* blk_file, const uint8_t* out, FileMeta* meta, KeptRecs K,
                        void* scan_tmp, cudaStream_t st) {
  if (!cap) return cudaSuccess;
  k_keep_lens<<<grid_for(cap, 256), 256, 0, st>>>(cnt, ed, K);
  cudaError_t e = exclusive_scan<uint32_t, uint64_t>(K.klen, K.koff, cap, &cnt->n_surv, scan_tmp, st);
  if (e != cudaSuccess) return e;
  k_keep_recs<<<grid_for(cap, 256), 256, 0, st>>>(cnt, ed, recs, K);
  k_keep_files<<<grid_for(cap, 128, kSms), 128, 0, st>>>(cnt, files, K, meta);
  k_keep_values<<<grid_for(uint64_t(cap) * 32, 256), 256, 0, st>>>(cnt, bd, blk_file, out, K, meta);
  count_launches(4);
  return cudaGetLastError();
}

void launch_kept_gather(const KeptIn* ins, uint32_t n_inputs, uint64_t max_count, Recs recs, cudaStream_t st) {
  if (!n_inputs || !max_count) return;
  const uint32_t x = uint32_t(max_count < 256ull * kSms * 4 ? (max_count + 255) / 256 : kSms * 4);
  k_kept_gather<<<dim3(x, n_inputs), 256, 0, st>>>(ins, recs);
  count_launches(1);
}

}  // namespace luda
