// LSD radix sort of packed keys with an optional payload (the `sort`
// instruction of the paper's APM table, Sec. 3.2; used on candidate tuples in
// the Stratum rule of the appendix).
//
// One pass per RB-bit digit, least significant first.  Each pass:
//   1. upsweep: per 4096-key tile, a digit histogram (per-warp shared-memory
//      counters);
//   2. scan of the digit-major histogram matrix -> each (digit, tile) output base;
//   3. scatter: each warp ranks its keys stably with a ballot multisplit (keys
//      with equal digits in one 32-key round -- found by intersecting one ballot
//      per digit bit -- get consecutive ranks in lane order; a
//      per-warp running count carries ranks across rounds), warps are combined
//      per digit, the tile is reordered by digit in shared memory, and each
//      digit's run is stored to consecutive global addresses.  Rank order =
//      input order, so each pass is stable.
// No block waits on another block.
#include "kernels.h"
#include "scan.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMinSortTile = kSortThreads * 16;

struct NoPay {};

// keys per thread (4096-key tiles)
template <class K, class P>
struct SortCfg {
  static constexpr int kPayBytes = std::is_same<P, NoPay>::value ? 0 : (int)sizeof(P);
  static constexpr int kItems = 16;
  static constexpr int kTile = kSortThreads * kItems;
  static constexpr int kSmem = kTile * ((int)sizeof(K) + kPayBytes);
};

template <class K, class P, int RB>
__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const K* __restrict__ keys, u64 n, int shift,
                                                                u32* __restrict__ hist, u64 ntiles,
                                                                const u64* __restrict__ n_dev) {
  constexpr int D = 1 << RB;
  if (n_dev) {
    n = *n_dev < n ? *n_dev : n;  // tiles past it count nothing
    if (n == 0) return;           // nothing to sort: the scatter will not read the histograms
  }
  constexpr int IT = SortCfg<K, P>::kItems;
  __shared__ u32 h[kSortWarps][D];
  for (int i = threadIdx.x; i < kSortWarps * D; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const u64 tbase = (u64)blockIdx.x * SortCfg<K, P>::kTile;
  K k[IT];
#pragma unroll
  for (int r = 0; r < IT; r++) {  // issue every load before the first use
    const u64 idx = tbase + (u64)r * kSortThreads + threadIdx.x;
    k[r] = idx < n ? keys[idx] : K(0);
  }
#pragma unroll
  for (int r = 0; r < IT; r++) {
    const u64 idx = tbase + (u64)r * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[warp][(u32)((k[r] >> shift) & (K)(D - 1))], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < D; d += kSortThreads) {
    u32 t = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) t += h[w][d];
    hist[(u64)d * ntiles + blockIdx.x] = t;
  }
}

// Lanes of this warp holding the same RB-bit digit (and a valid key): the
// intersection over the digit's bits of the ballot of lanes agreeing on that bit.
template <int RB>
LOB_DEV u32 same_digit_lanes(u32 d, bool valid) {
  u32 m = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
  for (int b = 0; b < RB; b++) {
    const bool bit = (d >> b) & 1u;
    const u32 v = __ballot_sync(0xFFFFFFFFu, bit);
    m &= bit ? v : ~v;
  }
  return m;
}

// One LSD pass.  Warp w ranks its 32*IT keys (in input order) per digit with a
// ballot multisplit; the tile's keys are then placed in shared memory in
// (digit, input order) order and written out run by run, so each digit's run
// of the tile goes to consecutive global addresses (coalesced stores).
template <class K, class P, int RB>
__global__ void __launch_bounds__(kSortThreads, 2) k_radix_scatter(const K* __restrict__ keys, const P* __restrict__ pay,
                                                                   K* __restrict__ okeys, P* __restrict__ opay, u64 n,
                                                                   int shift, const u32* __restrict__ offs, u64 ntiles,
                                                                   const u64* __restrict__ n_dev) {
  constexpr int D = 1 << RB;
  if (n_dev) n = *n_dev < n ? *n_dev : n;
  if ((u64)blockIdx.x * SortCfg<K, P>::kTile >= n) return;  // a tile past a device-resident count
  constexpr int IT = SortCfg<K, P>::kItems;
  constexpr int TILE = SortCfg<K, P>::kTile;
  constexpr bool kPay = !std::is_same<P, NoPay>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw);
  P* sp = reinterpret_cast<P*>(sk + TILE);
  __shared__ u32 wh[kSortWarps][D];
  __shared__ u32 dstart[D];
  __shared__ u32 gbase[D];
  __shared__ u32 sm[kSortThreads / 32 + 1];
  for (int i = threadIdx.x; i < kSortWarps * D; i += kSortThreads) (&wh[0][0])[i] = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 lt_mask = (1u << lane) - 1u;
  const u64 tbase = (u64)blockIdx.x * TILE;
  const int tile_n = (int)min((u64)TILE, n - tbase);
  const int wofs = warp * 32 * IT;  // this warp's first key within the tile
  const K* kin = keys + tbase + wofs;
  K k[IT];
  P p[IT];
  u32 rank[IT];
#pragma unroll
  for (int r = 0; r < IT; r++) {  // issue every load before the ranking starts
    const int o = r * 32 + lane;
    const bool valid = wofs + o < tile_n;
    k[r] = valid ? kin[o] : K(0);
    if constexpr (kPay) {
      if (valid) p[r] = pay[tbase + wofs + o];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IT; r++) {
    const bool valid = wofs + r * 32 + lane < tile_n;
    const u32 d = valid ? (u32)((k[r] >> shift) & (K)(D - 1)) : 0u;
    const u32 peers = same_digit_lanes<RB>(d, valid);
    u32 base = 0;
    if (valid) base = wh[warp][d];
    rank[r] = base + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && (__ffs(peers) - 1) == lane) wh[warp][d] = base + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive offsets of the warps, tile total
  for (int d = threadIdx.x; d < D; d += kSortThreads) {
    u32 s = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) {
      const u32 c = wh[w][d];
      wh[w][d] = s;
      s += c;
    }
    dstart[d] = s;
  }
  __syncthreads();
  {
    const u32 t = threadIdx.x < D ? dstart[threadIdx.x] : 0u;
    u32 tot;
    const u32 ex = block_exclusive_sum<u32>(t, sm, &tot);
    if (threadIdx.x < D) {
      dstart[threadIdx.x] = ex;
      gbase[threadIdx.x] = offs[(u64)threadIdx.x * ntiles + blockIdx.x];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IT; r++) {
    if (wofs + r * 32 + lane < tile_n) {
      const u32 d = (u32)((k[r] >> shift) & (K)(D - 1));
      const u32 lp = dstart[d] + wh[warp][d] + rank[r];
      sk[lp] = k[r];
      if constexpr (kPay) sp[lp] = p[r];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
    const K key = sk[i];
    const u32 d = (u32)((key >> shift) & (K)(D - 1));
    const u64 pos = (u64)gbase[d] + (u32)(i - dstart[d]);
    okeys[pos] = key;
    if constexpr (kPay) opay[pos] = sp[i];
  }
}

template <class K, class P, int RB>
void sort_impl(void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, void* scratch, cudaStream_t st,
               const u64* n_dev) {
  constexpr int D = 1 << RB;
  constexpr int TILE = SortCfg<K, P>::kTile;
  constexpr int SMEM = SortCfg<K, P>::kSmem;
  if (n <= 1 || bits <= 0) return;
  const u64 ntiles = (n + TILE - 1) / TILE;
  allow_dynamic_smem(k_radix_scatter<K, P, RB>, SMEM);
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
      k_radix_upsweep<K, P, RB><<<(unsigned)ntiles, kSortThreads, 0, st>>>(src_k, n, shift, hist, ntiles, n_dev);
    }
    {
      ProfScope ps("radix_digit_scan", (double)D * ntiles * 8, st);
      exclusive_scan<u32, u32>(hist, hist, (u64)D * ntiles, nullptr, scan_ws, st);
    }
    {
      ProfScope ps("radix_scatter", 2.0 * n * (kb + pb) + (double)D * ntiles * 4, st);
      k_radix_scatter<K, P, RB><<<(unsigned)ntiles, kSortThreads, SMEM, st>>>(src_k, src_p, dst_k, dst_p, n, shift, hist,
                                                                               ntiles, n_dev);
    }
    std::swap(src_k, dst_k);
    std::swap(src_p, dst_p);
  }
  *keys = src_k;
  *pay = src_p;
}

template <class K, class P>
void sort_rb(int rb, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, void* scratch, cudaStream_t st,
             const u64* n_dev) {
  switch (rb) {
    case 4: sort_impl<K, P, 4>(keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev); break;
    case 6: sort_impl<K, P, 6>(keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev); break;
    default: sort_impl<K, P, 8>(keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev); break;
  }
}


// ---------------------------------------------------------------------------
// Single-pass-per-digit variant (decoupled look-back, after Adinets and
// Merrill, "Onesweep", 2022): the global digit histograms of every pass come
// from one read of the keys; each pass is then one kernel whose tiles take
// dynamic ids, publish their per-digit counts, and obtain their per-digit
// output offsets by walking back over the published state of earlier tiles.
// A tile waits only on tiles that started before it, so the walk always ends;
// every wait is still bounded, and giving up sets *err (the host then reports
// a timeout instead of returning unsorted data).
// ---------------------------------------------------------------------------
constexpr u64 kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62, kValMask = (1ull << 62) - 1;
constexpr u32 kSpinLimit = 1u << 22;

template <class K, int RB>
__global__ void __launch_bounds__(256) k_onesweep_hist(const K* __restrict__ keys, u64 n, int passes,
                                                       unsigned long long* __restrict__ ghist) {
  constexpr int D = 1 << RB;
  __shared__ u32 h[8][D];
  for (int i = threadIdx.x; i < 8 * D; i += 256) (&h[0][0])[i] = 0;
  __syncthreads();
  const u64 stride = (u64)gridDim.x * 256 * 4;
  for (u64 base = (u64)blockIdx.x * 256 * 4; base < n; base += stride) {
    K k[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const u64 idx = base + (u64)j * 256 + threadIdx.x;
      k[j] = idx < n ? keys[idx] : K(0);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      if (base + (u64)j * 256 + threadIdx.x >= n) continue;
      for (int p = 0; p < passes; p++) atomicAdd(&h[p][(u32)((k[j] >> (p * RB)) & (K)(D - 1))], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * D; i += 256) {
    const u32 c = (&h[0][0])[i];
    if (c) atomicAdd(ghist + i, (unsigned long long)c);
  }
}

// exclusive scan of each pass's D digit counts (one block, one thread per digit)
template <int RB>
__global__ void k_onesweep_starts(unsigned long long* ghist, int passes) {
  constexpr int D = 1 << RB;
  __shared__ u64 sm[256 / 32 + 1];
  for (int p = 0; p < passes; p++) {
    const u64 v = threadIdx.x < D ? ghist[p * D + threadIdx.x] : 0ull;
    u64 tot;
    const u64 ex = block_exclusive_sum<u64>(v, sm, &tot);
    if (threadIdx.x < D) ghist[p * D + threadIdx.x] = ex;
  }
}

template <class K, class P, int RB>
__global__ void __launch_bounds__(kSortThreads, 2) k_onesweep_scatter(const K* __restrict__ keys, const P* __restrict__ pay,
                                                                      K* __restrict__ okeys, P* __restrict__ opay, u64 n,
                                                                      int shift, const unsigned long long* __restrict__ gstart,
                                                                      unsigned long long* status, u32* tile_counter,
                                                                      u32* err) {
  constexpr int D = 1 << RB;
  constexpr int IT = SortCfg<K, P>::kItems;
  constexpr int TILE = SortCfg<K, P>::kTile;
  constexpr bool kPay = !std::is_same<P, NoPay>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw);
  P* sp = reinterpret_cast<P*>(sk + TILE);
  __shared__ u32 wh[kSortWarps][D];
  __shared__ u32 dstart[D];
  __shared__ u64 gbase[D];
  __shared__ u32 sm[kSortThreads / 32 + 1];
  __shared__ u32 s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
  for (int i = threadIdx.x; i < kSortWarps * D; i += kSortThreads) (&wh[0][0])[i] = 0;
  __syncthreads();
  const u64 tile = s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 lt_mask = (1u << lane) - 1u;
  const u64 tbase = tile * TILE;
  const int tile_n = (int)min((u64)TILE, n - tbase);
  const int wofs = warp * 32 * IT;
  const K* kin = keys + tbase + wofs;
  K k[IT];
  P p[IT];
  u32 rank[IT];
#pragma unroll
  for (int r = 0; r < IT; r++) {
    const int o = r * 32 + lane;
    const bool valid = wofs + o < tile_n;
    k[r] = valid ? kin[o] : K(0);
    if constexpr (kPay) {
      if (valid) p[r] = pay[tbase + wofs + o];
    }
  }
#pragma unroll
  for (int r = 0; r < IT; r++) {
    const bool valid = wofs + r * 32 + lane < tile_n;
    const u32 d = valid ? (u32)((k[r] >> shift) & (K)(D - 1)) : 0u;
    const u32 peers = same_digit_lanes<RB>(d, valid);
    u32 base = 0;
    if (valid) base = wh[warp][d];
    rank[r] = base + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && (__ffs(peers) - 1) == lane) wh[warp][d] = base + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int d = threadIdx.x; d < D; d += kSortThreads) {
    u32 s = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) {
      const u32 c = wh[w][d];
      wh[w][d] = s;
      s += c;
    }
    dstart[d] = s;
  }
  __syncthreads();
  if (threadIdx.x < D) {  // publish this tile's count of digit d, then look back for its prefix
    const int d = threadIdx.x;
    const u64 cnt = dstart[d];
    volatile unsigned long long* st = status;
    u64 excl = 0;
    if (tile == 0) {
      st[d] = kFlagPrefix | cnt;
    } else {
      st[tile * D + d] = kFlagAgg | cnt;
      u64 i = tile - 1;
      u32 spins = 0;
      for (;;) {
        const u64 v = st[i * D + d];
        const u64 flag = v & ~kValMask;
        if (flag == 0) {
          if (++spins > kSpinLimit) {
            atomicExch(err, 1u);
            break;
          }
          __nanosleep(32);
          continue;
        }
        excl += v & kValMask;
        if (flag == kFlagPrefix || i == 0) break;
        i--;
      }
      st[tile * D + d] = kFlagPrefix | (excl + cnt);
    }
    gbase[d] = gstart[d] + excl;
  }
  {
    const u32 t = threadIdx.x < D ? dstart[threadIdx.x] : 0u;
    u32 tot;
    const u32 ex = block_exclusive_sum<u32>(t, sm, &tot);
    if (threadIdx.x < D) dstart[threadIdx.x] = ex;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IT; r++) {
    if (wofs + r * 32 + lane < tile_n) {
      const u32 d = (u32)((k[r] >> shift) & (K)(D - 1));
      const u32 lp = dstart[d] + wh[warp][d] + rank[r];
      sk[lp] = k[r];
      if constexpr (kPay) sp[lp] = p[r];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
    const K key = sk[i];
    const u32 d = (u32)((key >> shift) & (K)(D - 1));
    const u64 pos = gbase[d] + (u32)(i - dstart[d]);
    okeys[pos] = key;
    if constexpr (kPay) opay[pos] = sp[i];
  }
}

template <class K, class P, int RB>
void onesweep_impl(void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, void* scratch, u32* err,
                   cudaStream_t st) {
  constexpr int D = 1 << RB;
  constexpr int TILE = SortCfg<K, P>::kTile;
  constexpr int SMEM = SortCfg<K, P>::kSmem;
  if (n <= 1 || bits <= 0) return;
  const int passes = (bits + RB - 1) / RB;
  const u64 ntiles = (n + TILE - 1) / TILE;
  allow_dynamic_smem(k_onesweep_scatter<K, P, RB>, SMEM);
  unsigned long long* ghist = reinterpret_cast<unsigned long long*>(scratch);
  u32* counters = reinterpret_cast<u32*>(ghist + 8 * D);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(counters + 64);
  cudaMemsetAsync(scratch, 0, 8 * D * sizeof(u64) + 64 * sizeof(u32), st);
  constexpr double kb = sizeof(K), pb = std::is_same<P, NoPay>::value ? 0 : sizeof(P);
  {
    ProfScope ps("radix_histogram", n * kb, st);
    u64 blocks = (n + 1023) / 1024;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    k_onesweep_hist<K, RB><<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const K*>(*keys), n, passes, ghist);
    k_onesweep_starts<RB><<<1, 256, 0, st>>>(ghist, passes);
  }
  K* src_k = reinterpret_cast<K*>(*keys);
  K* dst_k = reinterpret_cast<K*>(ktmp);
  P* src_p = reinterpret_cast<P*>(*pay);
  P* dst_p = reinterpret_cast<P*>(ptmp);
  for (int pass = 0; pass < passes; pass++) {
    cudaMemsetAsync(status, 0, ntiles * D * sizeof(u64), st);
    ProfScope ps("radix_scatter", 2.0 * n * (kb + pb), st);
    k_onesweep_scatter<K, P, RB><<<(unsigned)ntiles, kSortThreads, SMEM, st>>>(
        src_k, src_p, dst_k, dst_p, n, pass * RB, ghist + (u64)pass * D, status, counters + pass, err);
    std::swap(src_k, dst_k);
    std::swap(src_p, dst_p);
  }
  *keys = src_k;
  *pay = src_p;
}

template <class K, class P>
void onesweep_rb(int rb, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, void* scratch, u32* err,
                 cudaStream_t st) {
  switch (rb) {
    case 4: onesweep_impl<K, P, 4>(keys, pay, ktmp, ptmp, n, bits, scratch, err, st); break;
    case 6: onesweep_impl<K, P, 6>(keys, pay, ktmp, ptmp, n, bits, scratch, err, st); break;
    default: onesweep_impl<K, P, 8>(keys, pay, ktmp, ptmp, n, bits, scratch, err, st); break;
  }
}

}  // namespace

int sort_supported_radix_bits(int rb) { return (rb == 4 || rb == 6 || rb == 8) ? rb : 8; }

size_t sort_onesweep_scratch_bytes(u64 n, int rb) {
  rb = sort_supported_radix_bits(rb);
  const u64 ntiles = (n + kMinSortTile - 1) / kMinSortTile;
  return 8 * 256 * sizeof(u64) + 64 * sizeof(u32) + ntiles * ((u64)1 << rb) * sizeof(u64) + 256;
}

void sort_pairs_onesweep(int key64, int pay_bytes, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits,
                         int rb, void* scratch, u32* err, cudaStream_t st) {
  rb = sort_supported_radix_bits(rb);
  if (key64) {
    if (pay_bytes == 0) onesweep_rb<u64, NoPay>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, err, st);
    else if (pay_bytes == 4) onesweep_rb<u64, u32>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, err, st);
    else onesweep_rb<u64, u64>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, err, st);
  } else {
    if (pay_bytes == 0) onesweep_rb<u32, NoPay>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, err, st);
    else if (pay_bytes == 4) onesweep_rb<u32, u32>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, err, st);
    else onesweep_rb<u32, u64>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, err, st);
  }
}

int sort_onesweep_launches(u64 n, int bits, int rb) {
  if (n <= 1 || bits <= 0) return 0;
  rb = sort_supported_radix_bits(rb);
  const int passes = (bits + rb - 1) / rb;
  return 2 + passes;
}


size_t sort_scratch_bytes(u64 n, int rb) {
  rb = sort_supported_radix_bits(rb);
  const u64 ntiles = (n + kMinSortTile - 1) / kMinSortTile;
  const u64 h = ((u64)1 << rb) * ntiles;
  return (h + 1 + scan_scratch_elems(h) + 64) * sizeof(u32);
}

void sort_pairs(int key64, int pay_bytes, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, int rb,
                void* scratch, cudaStream_t st, const u64* n_dev) {
  rb = sort_supported_radix_bits(rb);
  if (key64) {
    if (pay_bytes == 0) sort_rb<u64, NoPay>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev);
    else if (pay_bytes == 4) sort_rb<u64, u32>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev);
    else sort_rb<u64, u64>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev);
  } else {
    if (pay_bytes == 0) sort_rb<u32, NoPay>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev);
    else if (pay_bytes == 4) sort_rb<u32, u32>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev);
    else sort_rb<u32, u64>(rb, keys, pay, ktmp, ptmp, n, bits, scratch, st, n_dev);
  }
}

int sort_kernel_launches(u64 n, int bits, int rb) {
  if (n <= 1 || bits <= 0) return 0;
  rb = sort_supported_radix_bits(rb);
  const u64 ntiles = (n + kMinSortTile - 1) / kMinSortTile;
  const u64 h = ((u64)1 << rb) * ntiles;
  int scan = 0;
  for (u64 m = h;; m = (m + kScanTile - 1) / kScanTile) {
    if ((m + kScanTile - 1) / kScanTile <= 1) { scan += 1; break; }
    scan += 2;
  }
  const int passes = (bits + rb - 1) / rb;
  return passes * (2 + scan);
}
