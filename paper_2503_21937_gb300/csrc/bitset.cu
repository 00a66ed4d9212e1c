// Sorted key lists read out of membership bitmaps (unit semiring).
//
// A relation whose packed key has at most 34 bits keeps a membership bitmap
// (bit k set <=> key k is a fact).  The bitmap is itself the relation in key
// order, so the facts one iteration added -- the bits set in the bitmap but not
// in the copy taken when the iteration started -- come out already sorted by
// reading both bitmaps once: no candidate list, sort, unique or difference is
// needed for them (Sec. 3.2's sort / unique / difference on candidate tuples,
// computed here as a set difference of two bitmaps).
//
// Each 256-thread tile owns 4096 consecutive words; a first pass counts the
// tile's bits, an exclusive scan places the tiles, and a second pass writes the
// tile's keys in increasing order from its scanned offset.
#include "kernels.h"
#include "scan.cuh"

namespace {

constexpr int kSliceWords = 16;
constexpr u64 kBitTileWords = 256 * kSliceWords;

// this thread's 16 words of a, masked by ~b when kDiff
template <bool kDiff>
LOB_DEV void load_slice(const u32* __restrict__ a, const u32* __restrict__ b, u64 w0, u64 nwords, u32 (&x)[kSliceWords]) {
  if (w0 + kSliceWords <= nwords) {
    const uint4* A = reinterpret_cast<const uint4*>(a + w0);
#pragma unroll
    for (int j = 0; j < kSliceWords / 4; j++) {
      const uint4 v = A[j];
      x[4 * j] = v.x; x[4 * j + 1] = v.y; x[4 * j + 2] = v.z; x[4 * j + 3] = v.w;
    }
    if constexpr (kDiff) {
      const uint4* B = reinterpret_cast<const uint4*>(b + w0);
#pragma unroll
      for (int j = 0; j < kSliceWords / 4; j++) {
        const uint4 v = B[j];
        x[4 * j] &= ~v.x; x[4 * j + 1] &= ~v.y; x[4 * j + 2] &= ~v.z; x[4 * j + 3] &= ~v.w;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < kSliceWords; j++) {
      const u64 w = w0 + j;
      x[j] = w < nwords ? (kDiff ? a[w] & ~b[w] : a[w]) : 0u;
    }
  }
}

template <bool kDiff>
__global__ void __launch_bounds__(256) k_bits_count(const u32* __restrict__ a, const u32* __restrict__ b, u64 nwords,
                                                    u64 ntiles, u64* __restrict__ tile_cnt) {
  __shared__ u32 part[256 / 32];
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    u32 x[kSliceWords];
    load_slice<kDiff>(a, b, t * kBitTileWords + (u64)threadIdx.x * kSliceWords, nwords, x);
    u32 c = 0;
#pragma unroll
    for (int j = 0; j < kSliceWords; j++) c += __popc(x[j]);
    c = warp_inclusive_sum(c);
    if ((threadIdx.x & 31) == 31) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      u64 s = 0;
      for (int w = 0; w < 256 / 32; w++) s += part[w];
      tile_cnt[t] = s;
    }
    __syncthreads();
  }
}

// Extraction: warp w of a tile owns the tile's words [w*512, (w+1)*512), held
// lane-strided (lane l has words i*32 + l, i < 16) so every load and the
// catch-up store of the copy are coalesced.  The warp walks its 16 batches of
// 32 words in order: a warp scan of the batch's bit counts places each lane's
// keys in the warp's shared-memory stage, and the warp then stores the batch's
// keys to consecutive global addresses.
constexpr int kWarpWords = kBitTileWords / 8;
constexpr int kBatches = kWarpWords / 32;

template <class K, bool kDiff>
__global__ void __launch_bounds__(256) k_bits_extract(const u32* __restrict__ a, u32* __restrict__ b, u64 nwords,
                                                      u64 ntiles, const u64* __restrict__ tile_off, K* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* stage = reinterpret_cast<K*>(smem_raw) + (threadIdx.x >> 5) * 1024;
  __shared__ u64 wbase[256 / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const u64 wf = t * kBitTileWords + (u64)warp * kWarpWords;  // this warp's first word
    u32 x[kBatches], av[kBatches];
    u32 c = 0;
#pragma unroll
    for (int i = 0; i < kBatches; i++) {
      const u64 w = wf + (u64)i * 32 + lane;
      av[i] = w < nwords ? a[w] : 0u;
      x[i] = av[i];
    }
    if constexpr (kDiff) {
#pragma unroll
      for (int i = 0; i < kBatches; i++) {
        const u64 w = wf + (u64)i * 32 + lane;
        x[i] &= w < nwords ? ~b[w] : 0u;
      }
    }
#pragma unroll
    for (int i = 0; i < kBatches; i++) c += __popc(x[i]);
    c = warp_inclusive_sum(c);
    if (lane == 31) wbase[warp] = c;
    __syncthreads();
    u64 base = tile_off[t];
    for (int v = 0; v < warp; v++) base += wbase[v];
    __syncthreads();  // wbase is rewritten by the next tile
#pragma unroll
    for (int i = 0; i < kBatches; i++) {
      const u32 m0 = x[i];
      const u32 cnt = __popc(m0);
      const u32 inc = warp_inclusive_sum(cnt);
      const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
      if (!tot) continue;
      u32 pos = inc - cnt;
      const K kw = (K)((wf + (u64)i * 32 + lane) << 5);
      for (u32 m = m0; m; m &= m - 1) stage[pos++] = kw | (K)(__ffs(m) - 1);
      __syncwarp();
      for (u32 q = lane; q < tot; q += 32) out[base + q] = stage[q];
      __syncwarp();
      base += tot;
    }
    if constexpr (kDiff) {  // the start-of-iteration copy catches up (b is a subset of a)
#pragma unroll
      for (int i = 0; i < kBatches; i++)
        if (x[i]) b[wf + (u64)i * 32 + lane] = av[i];
    }
  }
}

// Dense (+)-accumulation read-out (tagged semirings): the touched bitmap `a`
// lists the keys that received candidates this iteration and acc[key] holds
// their (+)-reduced candidate tag.  Reading both in key order yields the
// iteration's unique candidates already sorted, with their reduced tags -- the
// result of Sec. 3.2's sort + unique<(+)> over the candidate tuples, without
// materialising or sorting the candidates.  Each read slot is reset to 0 and
// each bitmap word cleared, ready for the next iteration.  Same tiling as
// k_bits_extract; the warp stages keys and tags side by side.
template <class K, class C>
__global__ void __launch_bounds__(256) k_dense_extract(u32* __restrict__ a, u64 nwords, u64 ntiles,
                                                       const u64* __restrict__ tile_off, C* __restrict__ acc,
                                                       K* __restrict__ out, C* __restrict__ otags, u64 cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tstage = reinterpret_cast<C*>(smem_raw) + (threadIdx.x >> 5) * 1024;
  K* stage = reinterpret_cast<K*>(reinterpret_cast<C*>(smem_raw) + 8 * 1024) + (threadIdx.x >> 5) * 1024;
  __shared__ u64 wbase[256 / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const u64 wf = t * kBitTileWords + (u64)warp * kWarpWords;
    u32 x[kBatches];
    u32 c = 0;
#pragma unroll
    for (int i = 0; i < kBatches; i++) {
      const u64 w = wf + (u64)i * 32 + lane;
      x[i] = w < nwords ? a[w] : 0u;
      c += __popc(x[i]);
    }
    c = warp_inclusive_sum(c);
    if (lane == 31) wbase[warp] = c;
    __syncthreads();
    u64 base = tile_off[t];
    for (int v = 0; v < warp; v++) base += wbase[v];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kBatches; i++) {
      const u32 m0 = x[i];
      const u32 cnt = __popc(m0);
      const u32 inc = warp_inclusive_sum(cnt);
      const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
      if (!tot) continue;
      u32 pos = inc - cnt;
      const u64 kw = (wf + (u64)i * 32 + lane) << 5;
      for (u32 m = m0; m; m &= m - 1) {
        const u64 key = kw | (u64)(__ffs(m) - 1);
        tstage[pos] = acc[key];
        acc[key] = C(0);
        stage[pos++] = (K)key;
      }
      __syncwarp();
      for (u32 q = lane; q < tot; q += 32) {
        if (base + q >= cap) break;  // beyond the output's capacity: only the resets happen
        out[base + q] = stage[q];
        otags[base + q] = tstage[q];
      }
      __syncwarp();
      base += tot;
      if (m0) a[wf + (u64)i * 32 + lane] = 0u;
    }
  }
}

// candidates written by other producers (projections, general join steps)
// folded into the dense accumulator; all-ones keys (dropped rows) are skipped
template <class Sem>
__global__ void k_dense_fold(const void* __restrict__ keys, int key64, const typename Sem::Cand* __restrict__ tags, u64 n,
                             void* __restrict__ acc, u32* __restrict__ bm) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 k = load_key(keys, key64, i);
    if (k == invalid_of(key64)) continue;
    dense_add<Sem>(acc, k, tags[i]);
    touch_bit(bm, k);
  }
}

u64 bit_words(u64 nbits) { return (nbits + 31) / 32; }
u64 bit_tiles(u64 nbits) { return (bit_words(nbits) + kBitTileWords - 1) / kBitTileWords; }
unsigned bit_grid(u64 ntiles) { return (unsigned)(ntiles < 152ull * 16 ? ntiles : 152ull * 16); }

}  // namespace

size_t bits_scratch_bytes(u64 nbits) {
  const u64 nt = bit_tiles(nbits);
  return (2 * nt + scan_scratch_elems(nt) + 8) * sizeof(u64);
}

int bits_count(const u32* a, const u32* b, u64 nbits, void* scratch, u64* total_dev, cudaStream_t st) {
  const u64 nw = bit_words(nbits), nt = bit_tiles(nbits);
  u64* tile_cnt = reinterpret_cast<u64*>(scratch);
  u64* tile_off = tile_cnt + nt;
  u64* ws = tile_off + nt;
  {
    ProfScope ps("bitmap_count", nw * (b ? 8.0 : 4.0), st);
    if (b) k_bits_count<true><<<bit_grid(nt), 256, 0, st>>>(a, b, nw, nt, tile_cnt);
    else k_bits_count<false><<<bit_grid(nt), 256, 0, st>>>(a, nullptr, nw, nt, tile_cnt);
  }
  exclusive_scan<u64, u64>(tile_cnt, tile_off, nt, total_dev, ws, st);
  return 1 + scan_launches(nt);
}

void bits_extract(const u32* a, u32* b, u64 nbits, int key64, void* out, u64 n_out, void* scratch, cudaStream_t st) {
  const u64 nw = bit_words(nbits), nt = bit_tiles(nbits);
  const u64* tile_off = reinterpret_cast<const u64*>(scratch) + nt;
  ProfScope ps("bitmap_extract", nw * (b ? 8.0 : 4.0) + n_out * (key64 ? 8.0 : 4.0), st);
  const unsigned g = bit_grid(nt);
  const int sm32 = 8 * 1024 * 4, sm64 = 8 * 1024 * 8;  // one 1024-key stage per warp
  if (key64) {
    if (b) allow_dynamic_smem(k_bits_extract<u64, true>, sm64);
    else allow_dynamic_smem(k_bits_extract<u64, false>, sm64);
    if (b) k_bits_extract<u64, true><<<g, 256, sm64, st>>>(a, b, nw, nt, tile_off, reinterpret_cast<u64*>(out));
    else k_bits_extract<u64, false><<<g, 256, sm64, st>>>(a, nullptr, nw, nt, tile_off, reinterpret_cast<u64*>(out));
  } else {
    if (b) k_bits_extract<u32, true><<<g, 256, sm32, st>>>(a, b, nw, nt, tile_off, reinterpret_cast<u32*>(out));
    else k_bits_extract<u32, false><<<g, 256, sm32, st>>>(a, nullptr, nw, nt, tile_off, reinterpret_cast<u32*>(out));
  }
}

// ---------------------------------------------------------------------------
// dense (+)-accumulation (host side)
// ---------------------------------------------------------------------------
namespace {
template <class K, class C>
void dense_extract_t(u32* a, u64 nbits, void* acc, void* out, void* otags, void* scratch, cudaStream_t st, u64 cap) {
  const u64 nw = bit_words(nbits), nt = bit_tiles(nbits);
  const u64* tile_off = reinterpret_cast<const u64*>(scratch) + nt;
  const int smem = 8 * 1024 * (int)(sizeof(K) + sizeof(C));
  allow_dynamic_smem(k_dense_extract<K, C>, smem);
  k_dense_extract<K, C><<<bit_grid(nt), 256, smem, st>>>(a, nw, nt, tile_off, reinterpret_cast<C*>(acc),
                                                         reinterpret_cast<K*>(out), reinterpret_cast<C*>(otags), cap);
}
template <class Sem>
void dense_fold_t(const void* keys, int key64, const void* tags, u64 n, void* acc, u32* bm, cudaStream_t st) {
  u64 b = (n + 255) / 256;
  if (b > 152ull * 16) b = 152ull * 16;
  k_dense_fold<Sem><<<(unsigned)(b ? b : 1), 256, 0, st>>>(keys, key64, reinterpret_cast<const typename Sem::Cand*>(tags),
                                                           n, acc, bm);
}
}  // namespace

int dense_cand_bytes(int sem) { return sem == SR_MAX_MIN ? 4 : 8; }

void dense_extract(int sem, int key64, u32* touched, void* acc, u64 nbits, void* okeys, void* otags, u64 n_out,
                   void* scratch, cudaStream_t st, u64 cap) {
  const double cb = dense_cand_bytes(sem), kb = key64 ? 8 : 4;
  ProfScope ps("dense_extract", bit_words(nbits) * 4.0 + n_out * (2.0 * cb + kb + cb), st);
  if (sem == SR_MAX_MIN) {
    if (key64) dense_extract_t<u64, float>(touched, nbits, acc, okeys, otags, scratch, st, cap);
    else dense_extract_t<u32, float>(touched, nbits, acc, okeys, otags, scratch, st, cap);
  } else {
    if (key64) dense_extract_t<u64, u64>(touched, nbits, acc, okeys, otags, scratch, st, cap);
    else dense_extract_t<u32, u64>(touched, nbits, acc, okeys, otags, scratch, st, cap);
  }
}

void dense_fold(int sem, int key64, const void* keys, const void* tags, u64 n, void* acc, u32* touched, cudaStream_t st) {
  ProfScope ps("dense_fold", n * ((key64 ? 8.0 : 4.0) + 2.0 * dense_cand_bytes(sem) + 4.0), st);
  if (!n) return;
  switch (sem) {
    case SR_MAX_MIN: dense_fold_t<SemMaxMin>(keys, key64, tags, n, acc, touched, st); break;
    case SR_DIFF_MAX_MIN: dense_fold_t<SemDiffMaxMin>(keys, key64, tags, n, acc, touched, st); break;
    default: dense_fold_t<SemAddMult>(keys, key64, tags, n, acc, touched, st); break;
  }
}
