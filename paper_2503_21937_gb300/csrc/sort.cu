// LSD radix sort of packed keys with an optional payload (the `sort`
// instruction of the paper's APM table, Sec. 3.2; used on candidate tuples in
// the Stratum rule of the appendix).
//
// One pass per RB-bit digit, least significant first.  Each pass:
//   1. upsweep: per 4096-key tile, a digit histogram in shared memory;
//   2. scan of the digit-major histogram matrix -> each (digit, tile) output base;
//   3. scatter: each warp ranks its 512 keys stably with __match_any_sync
//      (keys with equal digits in one 32-key round get consecutive ranks in lane
//      order; a per-warp running count carries ranks across rounds), warps are
//      combined per digit in shared memory, and every key is written to
//      base + rank.  Rank order = input order, so each pass is stable.
// No block waits on another block.
#include "kernels.h"
#include "scan.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;                        // 32-key rounds per warp
constexpr int kWarpKeys = 32 * kSortRounds;            // 512
constexpr int kSortTile = kWarpKeys * kSortWarps;      // 4096

struct NoPay {};

template <class K, int RB>
__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const K* __restrict__ keys, u64 n, int shift,
                                                                u32* __restrict__ hist, u64 ntiles) {
  constexpr int D = 1 << RB;
  __shared__ u32 h[D];
  for (int d = threadIdx.x; d < D; d += kSortThreads) h[d] = 0;
  __syncthreads();
  const u64 base = (u64)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    u64 idx = base + i;
    if (idx < n) atomicAdd(&h[(u32)((keys[idx] >> shift) & (K)(D - 1))], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < D; d += kSortThreads) hist[(u64)d * ntiles + blockIdx.x] = h[d];
}

template <class K, class P, int RB>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const K* __restrict__ keys, const P* __restrict__ pay,
                                                                K* __restrict__ okeys, P* __restrict__ opay, u64 n,
                                                                int shift, const u32* __restrict__ offs, u64 ntiles) {
  constexpr int D = 1 << RB;
  constexpr bool kPay = !std::is_same<P, NoPay>::value;
  __shared__ u32 wh[kSortWarps][D];
  for (int i = threadIdx.x; i < kSortWarps * D; i += kSortThreads) (&wh[0][0])[i] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 lt_mask = (1u << lane) - 1u;
  const u64 wbase = (u64)blockIdx.x * kSortTile + (u64)warp * kWarpKeys;
  K k[kSortRounds];
  P p[kSortRounds];
  u32 rank[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; r++) {
    const u64 idx = wbase + (u64)r * 32 + lane;
    const bool valid = idx < n;
    k[r] = valid ? keys[idx] : K(0);
    if constexpr (kPay) {
      if (valid) p[r] = pay[idx];
    }
    const u32 d = valid ? (u32)((k[r] >> shift) & (K)(D - 1)) : (u32)D;
    const u32 peers = __match_any_sync(0xFFFFFFFFu, d);
    u32 base = 0;
    if (valid) base = wh[warp][d];
    rank[r] = base + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && (__ffs(peers) - 1) == lane) wh[warp][d] = base + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps (tile-local offset of each warp's run)
  for (int d = threadIdx.x; d < D; d += kSortThreads) {
    u32 s = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) {
      u32 c = wh[w][d];
      wh[w][d] = s;
      s += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; r++) {
    const u64 idx = wbase + (u64)r * 32 + lane;
    if (idx < n) {
      const u32 d = (u32)((k[r] >> shift) & (K)(D - 1));
      const u64 pos = (u64)offs[(u64)d * ntiles + blockIdx.x] + wh[warp][d] + rank[r];
      okeys[pos] = k[r];
      if constexpr (kPay) opay[pos] = p[r];
    }
  }
}

template <class K, class P, int RB>
void sort_impl(void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, void* scratch, cudaStream_t st) {
  constexpr int D = 1 << RB;
  if (n <= 1 || bits <= 0) return;
  const u64 ntiles = (n + kSortTile - 1) / kSortTile;
  u32* hist = reinterpret_cast<u32*>(scratch);
  u32* scan_ws = hist + (u64)D * ntiles + 1;
  K* src_k = reinterpret_cast<K*>(*keys);
  K* dst_k = reinterpret_cast<K*>(ktmp);
  P* src_p = reinterpret_cast<P*>(*pay);
  P* dst_p = reinterpret_cast<P*>(ptmp);
  constexpr double kb = sizeof(K), pb = std::is_same<P, NoPay>::value ? 0 : sizeof(P);
  for (int shift = 0; shift < bits; shift += RB) {
    {
      ProfScope ps("radix_upsweep", n * kb + (double)D * ntiles * 4, st);
      k_radix_upsweep<K, RB><<<(unsigned)ntiles, kSortThreads, 0, st>>>(src_k, n, shift, hist, ntiles);
    }
    {
      ProfScope ps("radix_digit_scan", (double)D * ntiles * 8, st);
      exclusive_scan<u32, u32>(hist, hist, (u64)D * ntiles, nullptr, scan_ws, st);
    }
    {
      ProfScope ps("radix_scatter", 2.0 * n * (kb + pb) + (double)D * ntiles * 4, st);
      k_radix_scatter<K, P, RB><<<(unsigned)ntiles, kSortThreads, 0, st>>>(src_k, src_p, dst_k, dst_p, n, shift, hist, ntiles);
    }
    std::swap(src_k, dst_k);
    std::swap(src_p, dst_p);
  }
  *keys = src_k;
  *pay = src_p;
}

template <class K, class P>
void sort_rb(int rb, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, void* scratch, cudaStream_t st) {
  switch (rb) {
    case 4: sort_impl<K, P, 4>(keys, pay, ktmp, ptmp, n, bits, scratch, st); break;
    case 6: sort_impl<K, P, 6>(keys, pay, ktmp, ptmp, n, bits, scratch, st); break;
    default: sort_impl<K, P, 8>(keys, pay, ktmp, ptmp, n, bits, scratch, st); break;
  }
}

}  // namespace

int sort_supported_radix_bits(int rb) { return (rb == 4 || rb == 6 || rb == 8) ? rb : 8; }

size_t sort_scratch_bytes(u64 n, int rb) {
  rb = sort_supported_radix_bits(rb);
  const u64 ntiles = (n + kSortTile - 1) / kSortTile;
  const u64 h = ((u64)1 << rb) * ntiles;
  return (h + 1 + scan_scratch_elems(h) + 64) * sizeof(u32);
}

void sort_pairs(int key64, int pay_bytes, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, int rb,
                void* scratch, cudaStream_t st) {
  rb = sort_supported_radix_bits(rb);
  if (key64) {
    if (pay_bytes == 0) sort_rb<u64, NoPay>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st);
    else if (pay_bytes == 4) sort_rb<u64, u32>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st);
    else sort_rb<u64, u64>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st);
  } else {
    if (pay_bytes == 0) sort_rb<u32, NoPay>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st);
    else if (pay_bytes == 4) sort_rb<u32, u32>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st);
    else sort_rb<u32, u64>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st);
  }
}

int sort_kernel_launches(u64 n, int bits, int rb) {
  if (n <= 1 || bits <= 0) return 0;
  rb = sort_supported_radix_bits(rb);
  const u64 ntiles = (n + kSortTile - 1) / kSortTile;
  const u64 h = ((u64)1 << rb) * ntiles;
  int scan = 0;
  for (u64 m = h;; m = (m + kScanTile - 1) / kScanTile) {
    if ((m + kScanTile - 1) / kScanTile <= 1) { scan += 1; break; }
    scan += 2;
  }
  const int passes = (bits + rb - 1) / rb;
  return passes * (2 + scan);
}
