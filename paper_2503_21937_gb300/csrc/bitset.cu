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
// Each 256-thread tile owns 4096 consecutive words (16 per thread); a first
// pass counts the tile's bits, an exclusive scan places the tiles, and a second
// pass writes every thread's keys in increasing order from its scanned offset.
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

template <class K, bool kDiff>
__global__ void __launch_bounds__(256) k_bits_extract(const u32* __restrict__ a, u32* __restrict__ b, u64 nwords,
                                                      u64 ntiles, const u64* __restrict__ tile_off, K* __restrict__ out) {
  __shared__ u32 sm[256 / 32 + 1];
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const u64 w0 = t * kBitTileWords + (u64)threadIdx.x * kSliceWords;
    u32 x[kSliceWords];
    load_slice<kDiff>(a, b, w0, nwords, x);
    u32 c = 0;
#pragma unroll
    for (int j = 0; j < kSliceWords; j++) c += __popc(x[j]);
    u32 tot;
    const u32 ex = block_exclusive_sum<u32>(c, sm, &tot);
    u64 o = tile_off[t] + ex;
#pragma unroll
    for (int j = 0; j < kSliceWords; j++) {
      u32 m = x[j];
      const K base = (K)((w0 + j) << 5);
      while (m) {
        out[o++] = base | (K)(__ffs(m) - 1);
        m &= m - 1;
      }
    }
    if constexpr (kDiff) {  // the start-of-iteration copy catches up with the bitmap
#pragma unroll
      for (int j = 0; j < kSliceWords; j++)
        if (x[j]) b[w0 + j] |= x[j];
    }
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
  if (key64) {
    if (b) k_bits_extract<u64, true><<<g, 256, 0, st>>>(a, b, nw, nt, tile_off, reinterpret_cast<u64*>(out));
    else k_bits_extract<u64, false><<<g, 256, 0, st>>>(a, nullptr, nw, nt, tile_off, reinterpret_cast<u64*>(out));
  } else {
    if (b) k_bits_extract<u32, true><<<g, 256, 0, st>>>(a, b, nw, nt, tile_off, reinterpret_cast<u32*>(out));
    else k_bits_extract<u32, false><<<g, 256, 0, st>>>(a, nullptr, nw, nt, tile_off, reinterpret_cast<u32*>(out));
  }
}
