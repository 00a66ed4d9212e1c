// Join pipeline kernels: the APM instructions count / join / gather and
// gather<(x)> of Sec. 3.2 and the appendix's join_impl rule, re-designed as
//   count:  per input row, the [lo, hi) range of matching rows of a sorted
//           relation view, found through a dense offset table or binary search;
//   scan:   exclusive prefix sum of the counts (scan.cuh);
//   emit:   load-balanced expansion -- each 2048-output tile finds the input
//           row of every output by a shared-memory max-scan of row starts, so
//           a skewed row (a hub vertex) is spread over many tiles -- fused
//           with the gather of the matched columns, the projection to the
//           head, the selection filters and the tag product (x).
// The index is a relation view sorted by its join columns, so the matches of
// a row are one contiguous range (the paper's hash index maps keys to row
// indices; a sorted view gives the same lookup and coalesced emission).
#include "kernels.h"

#include "join_common.cuh"

namespace {

template <class Sem>
__global__ void __launch_bounds__(256) k_join_count(const __grid_constant__ StepParams P) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < P.n_in; r += stride) {
    u32 val[kMaxSlots];
    u32 sample;
    typename Sem::Cand tag;
    u64 lo = 0, hi = 0;
    if (read_input<Sem>(P, r, val, sample, tag)) probe_range(P, val, sample, lo, hi);
    P.cnt[r] = (u32)(hi - lo);
    P.lo[r] = lo;
  }
}

__global__ void k_lbs_partition(const u64* __restrict__ off, u64 n_in, u64 j_begin, u64 total, u64 ntiles,
                                u64* __restrict__ part) {
  const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t > ntiles) return;
  const u64 j = t == ntiles ? j_begin + total - 1 : j_begin + t * (u64)kEmitTile;
  part[t] = upper_bound_dev<u64>(off, 0, n_in, j) - 1;
}

template <class Sem>
__global__ void __launch_bounds__(256) k_join_emit(const __grid_constant__ StepParams P, const u64* __restrict__ part) {
  typedef typename Sem::Stored S;
  constexpr int kItems = kEmitTile / 256;
  __shared__ u32 row_of[kEmitTile];
  __shared__ u32 sm[256 / 32 + 1];
  const u64 j0 = P.j_begin + (u64)blockIdx.x * kEmitTile;
  const u64 j_end = P.j_begin + P.total;
  const u64 r0 = part[blockIdx.x];
  const u64 r_end = part[blockIdx.x + 1];
  for (int i = threadIdx.x; i < kEmitTile; i += 256) row_of[i] = 0;
  __syncthreads();
  for (u64 r = r0 + 1 + threadIdx.x; r <= r_end; r += 256) {
    const u64 o = P.off[r];
    if (o < j0 + kEmitTile) atomicMax(&row_of[o - j0], (u32)(r - r0));
  }
  __syncthreads();
  // inclusive max-scan: tile position -> input row (relative to r0)
  u32 loc[kItems];
  u32 m = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    const u32 x = row_of[threadIdx.x * kItems + i];
    m = x > m ? x : m;
    loc[i] = m;
  }
  const u32 inc = block_inclusive_max<u32>(m, sm);
  // exclusive prefix of thread maxima = inclusive of the previous thread
  __shared__ u32 th_inc[256];
  th_inc[threadIdx.x] = inc;
  __syncthreads();
  const u32 ex = threadIdx.x ? th_inc[threadIdx.x - 1] : 0u;
#pragma unroll
  for (int i = 0; i < kItems; i++) row_of[threadIdx.x * kItems + i] = loc[i] > ex ? loc[i] : ex;
  __syncthreads();
#pragma unroll 1
  for (int i = 0; i < kItems; i++) {
    const u64 j = j0 + (u64)i * 256 + threadIdx.x;
    if (j >= j_end) break;
    const u64 r = r0 + row_of[j - j0];
    const u64 v = P.lo[r] + (j - P.off[r]);
    u32 val[kMaxSlots];
    u32 sample;
    typename Sem::Cand tag;
    read_input<Sem>(P, r, val, sample, tag);
    bool ok = P.v_stamp_mode == STAMP_NONE || stamp_ok(P.v_stamp[v], P.v_stamp_mode, P.v_stamp_val);
    const u64 vk = load_key(P.v_keys, P.v_lay.key64, v);
#pragma unroll
    for (int c = 0; c < kMaxArity; c++) {
      if (c >= P.v_lay.arity) break;
      if (c >= P.prefix_len && ok) ok = apply_act(P.v_act[c], (u32)field_of(vk, P.v_lay.shift[c], P.v_lay.width[c]), val);
    }
    for (int f = 0; f < P.n_filters && ok; f++) ok = eval_filter(P, P.filters[f], val);
    if constexpr (std::is_same<Sem, SemTop1>::value) {
      if (ok) tag = top1_union(P.top1, tag, reinterpret_cast<const S*>(P.v_tags)[v]);
    } else if constexpr (Sem::kTags) {
      tag = Sem::mul(tag, Sem::from_stored(reinterpret_cast<const S*>(P.v_tags)[v]));
    }
    write_output<Sem>(P, P.out_base + (j - P.j_begin), ok, val, sample, tag);
  }
}

// Emission with the membership filter (unit semiring): candidates whose bit was
// already set (a known fact, or a candidate emitted earlier) are dropped; the
// survivors of a tile are written contiguously at a block-reserved offset.
__global__ void __launch_bounds__(256) k_join_emit_filtered(const __grid_constant__ StepParams P,
                                                           const u64* __restrict__ part) {
  typedef SemUnit Sem;
  constexpr int kItems = kEmitTile / 256;
  __shared__ u32 row_of[kEmitTile];
  __shared__ u32 sm[256 / 32 + 1];
  __shared__ u32 th_inc[256];
  __shared__ u64 block_base;
  const u64 j0 = P.j_begin + (u64)blockIdx.x * kEmitTile;
  const u64 j_end = P.j_begin + P.total;
  const u64 r0 = part[blockIdx.x];
  const u64 r_end = part[blockIdx.x + 1];
  for (int i = threadIdx.x; i < kEmitTile; i += 256) row_of[i] = 0;
  __syncthreads();
  for (u64 r = r0 + 1 + threadIdx.x; r <= r_end; r += 256) {
    const u64 o = P.off[r];
    if (o < j0 + kEmitTile) atomicMax(&row_of[o - j0], (u32)(r - r0));
  }
  __syncthreads();
  u32 loc[kItems];
  u32 m = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    const u32 x = row_of[threadIdx.x * kItems + i];
    m = x > m ? x : m;
    loc[i] = m;
  }
  const u32 inc = block_inclusive_max<u32>(m, sm);
  th_inc[threadIdx.x] = inc;
  __syncthreads();
  const u32 ex = threadIdx.x ? th_inc[threadIdx.x - 1] : 0u;
#pragma unroll
  for (int i = 0; i < kItems; i++) row_of[threadIdx.x * kItems + i] = loc[i] > ex ? loc[i] : ex;
  __syncthreads();
  u64 kept[kItems];
  u32 nkeep = 0;
  const Layout& L = P.out_lay;
#pragma unroll 1
  for (int i = 0; i < kItems; i++) {
    const u64 j = j0 + (u64)i * 256 + threadIdx.x;
    if (j >= j_end) break;
    const u64 r = r0 + row_of[j - j0];
    const u64 v = P.lo[r] + (j - P.off[r]);
    u32 val[kMaxSlots];
    u32 sample;
    typename Sem::Cand tag;
    read_input<Sem>(P, r, val, sample, tag);
    bool ok = P.v_stamp_mode == STAMP_NONE || stamp_ok(P.v_stamp[v], P.v_stamp_mode, P.v_stamp_val);
    const u64 vk = load_key(P.v_keys, P.v_lay.key64, v);
    for (int c = 0; c < P.v_lay.arity; c++)
      if (c >= P.prefix_len && ok) ok = apply_act(P.v_act[c], (u32)field_of(vk, P.v_lay.shift[c], P.v_lay.width[c]), val);
    for (int f = 0; f < P.n_filters && ok; f++) ok = eval_filter(P, P.filters[f], val);
    if (!ok) continue;
    u64 key = L.swidth ? (u64)sample << L.sshift : 0ull;
    for (int c = 0; c < L.arity && ok; c++) {
      u32 x;
      ok = head_value(P, c, val, x);
      key |= (u64)x << L.shift[c];
    }
    if (!ok) continue;
    const u32 bit = 1u << (u32)(key & 31u);
    if (atomicOr(P.bitmap + (key >> 5), bit) & bit) continue;
    kept[nkeep++] = key;
  }
  u32 tot;
  const u32 mine = block_exclusive_sum<u32>(nkeep, sm, &tot);
  if (threadIdx.x == 0) block_base = tot ? atomicAdd(reinterpret_cast<unsigned long long*>(P.out_count), (u64)tot) : 0ull;
  __syncthreads();
  const u64 base = P.out_base + block_base + mine;
  for (u32 q = 0; q < nkeep; q++) store_key(P.out_keys, L.key64, base + q, kept[q]);
}

__global__ void k_bitmap_set(const void* __restrict__ keys, int key64, u64 n, u32* __restrict__ bm) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 k = load_key(keys, key64, i);
    atomicOr(bm + (k >> 5), 1u << (u32)(k & 31u));
  }
}

template <class Sem>
__global__ void __launch_bounds__(256) k_project(const __grid_constant__ StepParams P) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < P.n_in; r += stride) {
    u32 val[kMaxSlots];
    u32 sample;
    typename Sem::Cand tag = Sem::one();
    const bool ok = read_input<Sem>(P, r, val, sample, tag);
    write_output<Sem>(P, P.out_base + r, ok, val, sample, tag);
  }
}

__global__ void k_dense_index(const void* __restrict__ keys, int key64, u64 n, int rs, u64* __restrict__ offs, u64 domain,
                              const u64* __restrict__ n_dev, const u64* __restrict__ changed_dev,
                              void* const* __restrict__ keys_pp) {
  if (changed_dev && *changed_dev == 0) return;  // the view did not change: its index still holds
  if (n_dev) n = *n_dev < n ? *n_dev : n;
  if (keys_pp) keys = keys_pp[0];
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x; p <= domain; p += stride)
    offs[p] = p == domain ? n : lower_bound_any(keys, key64, n, p << rs);
}

struct Perm {
  int p[kMaxArity];
};

__global__ void k_repack(Layout from, Perm pf, Layout to, Perm pt, const void* __restrict__ in, void* __restrict__ out, u64 n,
                         const u64* __restrict__ n_dev, void* const* __restrict__ in_pp) {
  if (n_dev) n = *n_dev < n ? *n_dev : n;
  if (in_pp) in = in_pp[0];
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 k = load_key(in, from.key64, i);
    u32 rel[kMaxArity];
    for (int j = 0; j < from.arity; j++) rel[pf.p[j]] = (u32)field_of(k, from.shift[j], from.width[j]);
    u64 o = from.swidth ? field_of(k, from.sshift, from.swidth) << to.sshift : 0ull;
    for (int j = 0; j < to.arity; j++) o |= (u64)rel[pt.p[j]] << to.shift[j];
    store_key(out, to.key64, i, o);
  }
}

__global__ void k_pack_rows(Layout L, const u32* __restrict__ cols, u64 stride_c, const u32* __restrict__ samples, u64 n,
                            void* __restrict__ keys, u32* __restrict__ rows) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    u64 k = (L.swidth && samples) ? (u64)samples[i] << L.sshift : 0ull;
    for (int j = 0; j < L.arity; j++) k |= (u64)cols[(u64)j * stride_c + i] << L.shift[j];
    store_key(keys, L.key64, i, k);
    rows[i] = (u32)i;
  }
}

template <class Sem>
__global__ void k_read_rows(Layout L, Perm perm, const void* __restrict__ keys, const void* __restrict__ tags, u64 n,
                            u32* __restrict__ cols, u64 stride_c, float* __restrict__ otags, u32* __restrict__ samples) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 k = load_key(keys, L.key64, i);
    for (int j = 0; j < L.arity; j++) cols[(u64)perm.p[j] * stride_c + i] = (u32)field_of(k, L.shift[j], L.width[j]);
    if (samples) samples[i] = L.swidth ? (u32)field_of(k, L.sshift, L.swidth) : 0u;
    if (otags) {
      float t = 1.0f;
      if constexpr (std::is_same<Sem, SemDiffMaxMin>::value || std::is_same<Sem, SemTop1>::value)
        t = dmm_value(reinterpret_cast<const u64*>(tags)[i]);
      else if constexpr (Sem::kTags) t = reinterpret_cast<const float*>(tags)[i];
      otags[i] = t;
    }
  }
}

__global__ void k_reduce_max(const u32* __restrict__ a, u64 n, u32* __restrict__ out) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  u32 m = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) m = max(m, a[i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

inline unsigned grid_for(u64 n, int threads = 256) {
  u64 b = (n + threads - 1) / threads;
  const u64 cap = 152ull * 16;  // enough resident blocks to fill every SM
  if (b > cap) b = cap;
  return (unsigned)(b ? b : 1);
}

template <template <class> class Launch, class... A>
void by_sem(int sem, A&&... a) {
  switch (sem) {
    case SR_UNIT: Launch<SemUnit>::go(a...); break;
    case SR_MAX_MIN: Launch<SemMaxMin>::go(a...); break;
    case SR_DIFF_MAX_MIN: Launch<SemDiffMaxMin>::go(a...); break;
    case SR_TOP1: Launch<SemTop1>::go(a...); break;
    default: Launch<SemAddMult>::go(a...); break;
  }
}

template <class Sem> struct CountL {
  static void go(const StepParams& P, cudaStream_t st) { k_join_count<Sem><<<grid_for(P.n_in), 256, 0, st>>>(P); }
};
template <class Sem> struct EmitL {
  static void go(const StepParams& P, const u64* part, cudaStream_t st) {
    const u64 tiles = (P.total + kEmitTile - 1) / kEmitTile;
    if (std::is_same<Sem, SemUnit>::value && P.bitmap && P.out_packed)
      k_join_emit_filtered<<<(unsigned)tiles, 256, 0, st>>>(P, part);
    else
      k_join_emit<Sem><<<(unsigned)tiles, 256, 0, st>>>(P, part);
  }
};
template <class Sem> struct ProjL {
  static void go(const StepParams& P, cudaStream_t st) { k_project<Sem><<<grid_for(P.n_in), 256, 0, st>>>(P); }
};
template <class Sem> struct ReadL {
  static void go(const Layout& L, const Perm& p, const void* keys, const void* tags, u64 n, u32* cols, u64 stride,
                 float* otags, u32* samples, cudaStream_t st) {
    k_read_rows<Sem><<<grid_for(n), 256, 0, st>>>(L, p, keys, tags, n, cols, stride, otags, samples);
  }
};

}  // namespace

static double input_row_bytes(int sem, const StepParams& P) {
  const double tb = sem == SR_UNIT ? 0 : (sem == SR_MAX_MIN ? 4 : 8);
  if (P.in_packed) return (P.in_lay.key64 ? 8 : 4) + (sem == SR_UNIT ? 0 : (sem == SR_DIFF_MAX_MIN || sem == SR_TOP1 ? 8 : 4));
  return 4.0 * (P.n_in_cols + 1) + tb;
}
static double output_row_bytes(int sem, const StepParams& P) {
  const double tb = sem == SR_UNIT ? 0 : (sem == SR_MAX_MIN ? 4 : 8);
  if (P.out_packed) return (P.out_lay.key64 ? 8 : 4) + tb;
  return 4.0 * (P.n_out_cols + 1) + tb;
}

void join_count(int sem, const StepParams& P, cudaStream_t st) {
  // read each input row once, two index words per row, write count + lo
  ProfScope ps("join_count", P.n_in * (input_row_bytes(sem, P) + 16.0 + 12.0), st);
  if (P.n_in) by_sem<CountL>(sem, P, st);
}

void lbs_partition(const u64* off, u64 n_in, u64 j_begin, u64 total, u64* part, cudaStream_t st) {
  const u64 ntiles = (total + kEmitTile - 1) / kEmitTile;
  ProfScope ps("join_partition", (ntiles + 1) * 8.0, st);
  k_lbs_partition<<<(unsigned)((ntiles + 1 + 255) / 256), 256, 0, st>>>(off, n_in, j_begin, total, ntiles, part);
}

void join_emit(int sem, const StepParams& P, const u64* part, cudaStream_t st) {
  // read the input rows and their offsets once, each matched view row once,
  // write every output row once
  const double vb = (P.v_lay.key64 ? 8 : 4) + (sem == SR_UNIT ? 0 : (sem == SR_DIFF_MAX_MIN || sem == SR_TOP1 ? 8 : 4));
  ProfScope ps("join_emit", P.n_in * (input_row_bytes(sem, P) + 16.0) + P.total * (vb + output_row_bytes(sem, P)), st);
  if (P.total) by_sem<EmitL>(sem, P, part, st);
}

void project_rows(int sem, const StepParams& P, cudaStream_t st) {
  ProfScope ps("project", P.n_in * (input_row_bytes(sem, P) + output_row_bytes(sem, P)), st);
  if (P.n_in) by_sem<ProjL>(sem, P, st);
}

void build_dense_index(const Layout& L, int prefix_len, const void* keys, u64 n, u64* offs, u64 domain, cudaStream_t st,
                       const u64* n_dev, const u64* changed_dev, void* const* keys_pp) {
  ProfScope ps("index_build", (domain + 1) * 8.0 + n * (L.key64 ? 8.0 : 4.0), st);
  k_dense_index<<<grid_for(domain + 1), 256, 0, st>>>(keys, L.key64, n, rest_shift(L, prefix_len), offs, domain, n_dev,
                                                     changed_dev, keys_pp);
}

// Insert every distinct prefix of a sorted view, by the first row of its run.
__global__ void k_hash_build(const void* __restrict__ keys, int key64, u64 n, int rs, HashSlot* __restrict__ tab, int bits) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 mask = (1ull << bits) - 1;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 pv = shr64(load_key(keys, key64, i), rs);
    if (i > 0 && shr64(load_key(keys, key64, i - 1), rs) == pv) continue;
    const u64 klo = shl64(pv, rs), khi = klo + shl64(1ull, rs);
    const u64 hi = (khi <= klo || rs >= 64) ? n : lower_bound_any(keys, key64, n, khi);
    u64 sl = hash_home(pv, bits);
    for (u64 t = 0; t <= mask; t++) {  // at most one pass over the table (load factor <= 1/2)
      const unsigned long long old = atomicCAS(&tab[sl].key, 0ull, (unsigned long long)(pv + 1));
      if (old == 0ull) {
        tab[sl].lo = (u32)i;
        tab[sl].cnt = (u32)(hi - i);
        break;
      }
      sl = (sl + 1) & mask;
    }
  }
}

void build_hash_index(const Layout& L, int prefix_len, const void* keys, u64 n, void* table, int bits, cudaStream_t st) {
  ProfScope ps("index_build", n * (L.key64 ? 8.0 : 4.0) + 16.0 * (double)(1ull << bits), st);
  if (n) k_hash_build<<<grid_for(n), 256, 0, st>>>(keys, L.key64, n, rest_shift(L, prefix_len),
                                                   reinterpret_cast<HashSlot*>(table), bits);
}

__global__ void k_copy_words(const u32* __restrict__ in, u32* __restrict__ out, u64 n_words, const u64* __restrict__ n_dev,
                             u32 words_per_elem, void* const* __restrict__ in_pp) {
  if (n_dev) n_words = (*n_dev * words_per_elem < n_words) ? *n_dev * words_per_elem : n_words;
  if (in_pp) in = reinterpret_cast<const u32*>(in_pp[0]);
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += stride) out[i] = in[i];
}

void copy_elems(void* dst, const void* src, u64 n, int elem_bytes, const u64* n_dev, cudaStream_t st, void* const* src_pp) {
  const u64 w = n * (u64)(elem_bytes / 4);
  if (!w) return;
  k_copy_words<<<grid_for(w), 256, 0, st>>>(reinterpret_cast<const u32*>(src), reinterpret_cast<u32*>(dst), w, n_dev,
                                            (u32)(elem_bytes / 4), src_pp);
}

void repack_keys(const Layout& from, const int* perm_from, const Layout& to, const int* perm_to, const void* in, void* out,
                 u64 n, cudaStream_t st, const u64* n_dev, void* const* in_pp) {
  if (!n) return;
  ProfScope ps("view_repack", n * ((from.key64 ? 8.0 : 4.0) + (to.key64 ? 8.0 : 4.0)), st);
  Perm a, b;
  for (int j = 0; j < kMaxArity; j++) {
    a.p[j] = j < from.arity ? perm_from[j] : 0;
    b.p[j] = j < to.arity ? perm_to[j] : 0;
  }
  k_repack<<<grid_for(n), 256, 0, st>>>(from, a, to, b, in, out, n, n_dev, in_pp);
}

void pack_rows(const Layout& L, const u32* cols, u64 stride, const u32* samples, u64 n, void* keys, u32* rows,
               cudaStream_t st) {
  ProfScope ps("load_pack", n * (4.0 * L.arity + (samples ? 4.0 : 0.0) + (L.key64 ? 8.0 : 4.0) + 4.0), st);
  if (n) k_pack_rows<<<grid_for(n), 256, 0, st>>>(L, cols, stride, samples, n, keys, rows);
}

void read_rows(int sem, const Layout& L, const int* perm, const void* keys, const void* tags, u64 n, u32* cols,
               u64 stride, float* otags, u32* samples, cudaStream_t st) {
  if (!n) return;
  Perm p;
  for (int j = 0; j < kMaxArity; j++) p.p[j] = j < L.arity ? perm[j] : 0;
  by_sem<ReadL>(sem, L, p, keys, tags, n, cols, stride, otags, samples, st);
}

void bitmap_set_keys(const void* keys, int key64, u64 n, u32* bitmap, cudaStream_t st) {
  ProfScope ps("bitmap_build", n * (key64 ? 8.0 : 4.0), st);
  if (n) k_bitmap_set<<<grid_for(n), 256, 0, st>>>(keys, key64, n, bitmap);
}

void reduce_max_u32(const u32* a, u64 n, u32* out_dev, cudaStream_t st) {
  cudaMemsetAsync(out_dev, 0, sizeof(u32), st);
  if (n) k_reduce_max<<<grid_for(n), 256, 0, st>>>(a, n, out_dev);
}
