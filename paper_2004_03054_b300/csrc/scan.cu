// scan.cu -- device-wide exclusive prefix sums (reduce, then down-sweep; the tile sums are
// scanned recursively only when there are many tiles).
//
// out[i] = in[0] + ... + in[i-1] for i in [0, n], so out[n] is the total. Used for record
// offsets, survivor positions, block starts, byte offsets of blocks and files.
#include <cstdint>

#include "internal.cuh"

namespace luda {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = uint64_t(kScanThreads) * kScanItems;

uint64_t tiles_of(uint64_t n) { return (n + kScanTile - 1) / kScanTile; }

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T o = __shfl_up_sync(0xFFFFFFFFu, v, d);
    if (lane >= uint32_t(d)) v += o;
  }
  return v;
}

// Exclusive scan of one value per thread across the CTA; returns the CTA total too.
template <typename T>
__device__ __forceinline__ T cta_excl_scan(T v, T* total) {
  __shared__ T warp_sums[kScanThreads / 32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const T incl = warp_incl_scan(v);
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
    s = warp_incl_scan(s);
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const T before = warp ? warp_sums[warp - 1] : T(0);
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + incl - v;
}

template <typename In>
__global__ void __launch_bounds__(kScanThreads) k_tile_reduce(const In* __restrict__ in, uint64_t cap,
                                                              const uint32_t* __restrict__ count,
                                                              uint64_t* __restrict__ sums) {
  const uint64_t n = count ? *count : cap;
  const uint64_t base = uint64_t(blockIdx.x) * kScanTile + uint64_t(threadIdx.x) * kScanItems;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += uint64_t(in[base + k]);
  uint64_t total;
  cta_excl_scan<uint64_t>(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename In, typename Out>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const In* __restrict__ in, uint64_t cap,
                                                            const uint32_t* __restrict__ count,
                                                            Out* __restrict__ out,
                                                            const uint64_t* __restrict__ offsets) {
  const uint64_t n = count ? *count : cap;
  if (n == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = Out(0);
    return;
  }
  if (uint64_t(blockIdx.x) * kScanTile >= n) return;
  const uint64_t base = uint64_t(blockIdx.x) * kScanTile + uint64_t(threadIdx.x) * kScanItems;
  Out v[kScanItems];
  Out s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? Out(in[base + k]) : Out(0);
    s += v[k];
  }
  Out total;
  Out run = cta_excl_scan<Out>(s, &total) + (offsets ? Out(offsets[blockIdx.x]) : Out(0));
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (base < n && base + kScanItems >= n) out[n] = run;  // the thread holding the last item
}

// As k_tile_scan, with the tile's offset summed from the tile sums by the CTA itself (one
// launch fewer than scanning the sums; used while the tile count is small).
template <typename In, typename Out>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan_sums(const In* __restrict__ in, uint64_t cap,
                                                                 const uint32_t* __restrict__ count,
                                                                 Out* __restrict__ out,
                                                                 const uint64_t* __restrict__ sums) {
  const uint64_t n = count ? *count : cap;
  if (n == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = Out(0);
    return;
  }
  if (uint64_t(blockIdx.x) * kScanTile >= n) return;
  uint64_t part = 0;
  for (uint32_t i = threadIdx.x; i < blockIdx.x; i += kScanThreads) part += sums[i];
  uint64_t offset;
  cta_excl_scan<uint64_t>(part, &offset);
  const uint64_t base = uint64_t(blockIdx.x) * kScanTile + uint64_t(threadIdx.x) * kScanItems;
  Out v[kScanItems];
  Out s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? Out(in[base + k]) : Out(0);
    s += v[k];
  }
  Out total;
  Out run = cta_excl_scan<Out>(s, &total) + Out(offset);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (base < n && base + kScanItems >= n) out[n] = run;
}

constexpr uint64_t kScanFusedTiles = 2048;

}  // namespace

uint64_t scan_temp_bytes(uint64_t n) {
  uint64_t bytes = 0;
  while (n > kScanTile) {
    const uint64_t t = tiles_of(n);
    bytes += (2 * t + 1) * sizeof(uint64_t);
    n = t;
  }
  return bytes + 256;
}

// n = *count when `count` is given (a device-side element count <= cap), else cap. Grids
// are sized by cap; tiles past n do nothing, so the cost follows n.
template <typename In, typename Out>
cudaError_t exclusive_scan(const In* in, Out* out, uint64_t cap, const uint32_t* count, void* temp,
                           cudaStream_t st) {
  if (cap == 0) return cudaMemsetAsync(out, 0, sizeof(Out), st);
  const uint64_t t = tiles_of(cap);
  if (t == 1) {
    k_tile_scan<In, Out><<<1, kScanThreads, 0, st>>>(in, cap, count, out, nullptr); count_launches(1);
    return cudaGetLastError();
  }
  uint64_t* sums = static_cast<uint64_t*>(temp);
  uint64_t* offs = sums + t;
  void* rest = offs + t + 1;
  k_tile_reduce<In><<<unsigned(t), kScanThreads, 0, st>>>(in, cap, count, sums); count_launches(1);
  if (t <= kScanFusedTiles) {
    k_tile_scan_sums<In, Out><<<unsigned(t), kScanThreads, 0, st>>>(in, cap, count, out, sums);
    count_launches(1);
    return cudaGetLastError();
  }
  cudaError_t e = exclusive_scan<uint64_t, uint64_t>(sums, offs, t, nullptr, rest, st);
  if (e != cudaSuccess) return e;
  k_tile_scan<In, Out><<<unsigned(t), kScanThreads, 0, st>>>(in, cap, count, out, offs); count_launches(1);
  return cudaGetLastError();
}

template cudaError_t exclusive_scan<uint8_t, uint32_t>(const uint8_t*, uint32_t*, uint64_t, const uint32_t*, void*,
                                                       cudaStream_t);
template cudaError_t exclusive_scan<uint32_t, uint32_t>(const uint32_t*, uint32_t*, uint64_t, const uint32_t*, void*,
                                                        cudaStream_t);
template cudaError_t exclusive_scan<uint32_t, uint64_t>(const uint32_t*, uint64_t*, uint64_t, const uint32_t*, void*,
                                                        cudaStream_t);
template cudaError_t exclusive_scan<uint64_t, uint64_t>(const uint64_t*, uint64_t*, uint64_t, const uint32_t*, void*,
                                                        cudaStream_t);

}  // namespace luda
