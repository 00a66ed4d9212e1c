// Exclusive prefix sum over device arrays (the `scan` instruction of the
// paper's APM table, Sec. 3.2).  Reduce-then-scan: per-tile sums, a recursive
// scan of the tile sums, and a per-tile block scan that adds the tile offset.
// No inter-block waiting, so no spin loops.
#pragma once
#include "common.cuh"

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class Ti, class To>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const Ti* __restrict__ in, u64 n, To* __restrict__ partial) {
  __shared__ To sm[kScanThreads / 32 + 1];
  const u64 base = (u64)blockIdx.x * kScanTile;
  To s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    u64 idx = base + (u64)i * kScanThreads + threadIdx.x;
    if (idx < n) s += (To)in[idx];
  }
  To total;
  block_exclusive_sum<To>(s, sm, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// out[i] = carry[tile] + sum(in[tile_base .. i)); in and out may alias.
template <class Ti, class To>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const Ti* in, To* out, u64 n, const To* __restrict__ carry,
                                                           To* __restrict__ total_out) {
  __shared__ To sm[kScanThreads / 32 + 1];
  const u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
  To v[kScanItems];
  To s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    u64 idx = base + i;
    v[i] = idx < n ? (To)in[idx] : To(0);
    s += v[i];
  }
  To total;
  To ex = block_exclusive_sum<To>(s, sm, &total);
  To c = carry ? carry[blockIdx.x] : To(0);
  ex += c;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    u64 idx = base + i;
    if (idx < n) out[idx] = ex;
    ex += v[i];
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = c + total;
}

// kernels launched by exclusive_scan for n elements
inline int scan_launches(u64 n) {
  if (n == 0) return 0;
  u64 tiles = (n + kScanTile - 1) / kScanTile;
  return tiles == 1 ? 1 : 2 + scan_launches(tiles);
}

// scratch elements (of To) needed to scan n elements
inline u64 scan_scratch_elems(u64 n) {
  u64 s = 0;
  while (n > (u64)kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    s += n + 1;
  }
  return s + 1;
}

// Exclusive scan in -> out (may alias) of n elements; *total_dev (device) gets
// the sum.  `scratch` holds scan_scratch_elems(n) elements of To.
template <class Ti, class To>
void exclusive_scan(const Ti* in, To* out, u64 n, To* total_dev, To* scratch, cudaStream_t st) {
  if (n == 0) {
    if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(To), st);
    return;
  }
  u64 tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_scan_apply<Ti, To><<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, total_dev);
    return;
  }
  To* partial = scratch;
  k_scan_reduce<Ti, To><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, partial);
  exclusive_scan<To, To>(partial, partial, tiles, nullptr, scratch + tiles + 1, st);
  k_scan_apply<Ti, To><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, partial, total_dev);
}
