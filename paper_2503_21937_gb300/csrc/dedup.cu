// unique<(+)>, the delta-versus-full difference and the merge of the new facts
// into the full relation (APM `unique` and `merge`, Sec. 3.2; the appendix's
// Stratum rule), plus the load-time normalisation of input facts.
#include "kernels.h"
#include "scan.cuh"

namespace {

// ---------------------------------------------------------------------------
// unique: collapse runs of equal keys of a sorted array, (+)-reducing tags
// ---------------------------------------------------------------------------
constexpr int kUThreads = 256;
constexpr int kUItems = 16;
constexpr int kUTile = kUThreads * kUItems;

template <class K>
LOB_DEV bool is_head(const K* keys, u64 idx, K k) {
  return k != invalid_key<K>() && (idx == 0 || keys[idx - 1] != k);
}

// Both unique kernels walk a 4096-key tile in 16 rounds of 256 consecutive
// keys (coalesced loads); element i is a run head when it differs from i-1.
template <class K>
__global__ void __launch_bounds__(kUThreads) k_unique_count(const K* __restrict__ keys, u64 n, u64* __restrict__ tile_cnt) {
  __shared__ u64 sm[kUThreads / 32 + 1];
  const u64 base = (u64)blockIdx.x * kUTile;
  K cur[kUItems], prev[kUItems];
#pragma unroll
  for (int i = 0; i < kUItems; i++) {  // all loads first
    const u64 idx = base + (u64)i * kUThreads + threadIdx.x;
    cur[i] = idx < n ? keys[idx] : invalid_key<K>();
    prev[i] = (idx < n && idx > 0) ? keys[idx - 1] : invalid_key<K>();
  }
  u64 c = 0;
#pragma unroll
  for (int i = 0; i < kUItems; i++) {
    const u64 idx = base + (u64)i * kUThreads + threadIdx.x;
    c += idx < n && cur[i] != invalid_key<K>() && (idx == 0 || prev[i] != cur[i]);
  }
  u64 total;
  block_exclusive_sum<u64>(c, sm, &total);
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = total;
}

template <class K, class Sem>
__global__ void __launch_bounds__(kUThreads) k_unique_write(const K* __restrict__ keys, const typename Sem::Cand* __restrict__ tags,
                                                            u64 n, const u64* __restrict__ tile_off, K* __restrict__ okeys,
                                                            typename Sem::Cand* __restrict__ otags) {
  __shared__ u32 wsum[kUThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u64 base = (u64)blockIdx.x * kUTile;
  u64 o = tile_off[blockIdx.x];
  K cur[kUItems];
  u32 heads = 0;
#pragma unroll
  for (int i = 0; i < kUItems; i++) {  // all loads first
    const u64 idx = base + (u64)i * kUThreads + threadIdx.x;
    cur[i] = idx < n ? keys[idx] : invalid_key<K>();
    const K pv = (idx < n && idx > 0) ? keys[idx - 1] : invalid_key<K>();
    heads |= (u32)(idx < n && cur[i] != invalid_key<K>() && (idx == 0 || pv != cur[i])) << i;
  }
#pragma unroll 1
  for (int i = 0; i < kUItems; i++) {
    const u64 idx = base + (u64)i * kUThreads + threadIdx.x;
    const K k = cur[i];
    const bool head = heads >> i & 1u;
    const u32 bal = __ballot_sync(0xFFFFFFFFu, head);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    u32 before = 0, round = 0;
#pragma unroll
    for (int w = 0; w < kUThreads / 32; w++) {
      const u32 c = wsum[w];
      before += w < warp ? c : 0u;
      round += c;
    }
    if (head) {
      const u64 pos = o + before + __popc(bal & ((1u << lane) - 1u));
      okeys[pos] = k;
      if constexpr (Sem::kTags) {
        typename Sem::Cand acc = tags[idx];
        for (u64 j = idx + 1; j < n && keys[j] == k; j++) acc = Sem::add(acc, tags[j]);
        otags[pos] = acc;
      }
    }
    o += round;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// delta-vs-full difference fused with the merge (merge path over F and U)
// ---------------------------------------------------------------------------
constexpr int kMThreads = 256;
constexpr int kMItems = 8;
constexpr int kMTile = kMThreads * kMItems;

// a = number of A elements among the first d merged elements (A first on ties)
template <class K>
__global__ void k_merge_path(const K* __restrict__ A, u64 na, const K* __restrict__ B, u64 nb, u64 nparts,
                             u64* __restrict__ apart, const u64* __restrict__ na_dev = nullptr,
                             const u64* __restrict__ nb_dev = nullptr, void* const* a_pp = nullptr,
                             int skip_empty = 0) {
  if (na_dev) na = *na_dev < na ? *na_dev : na;  // device-resident sizes, capped by the launch's capacities
  if (nb_dev) nb = *nb_dev < nb ? *nb_dev : nb;
  if (skip_empty && nb == 0) return;
  if (a_pp) A = reinterpret_cast<const K*>(a_pp[0]);
  const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nparts) return;
  const u64 d = min(t * (u64)kMTile, na + nb);
  u64 lo = d > nb ? d - nb : 0, hi = min(d, na);
  while (lo < hi) {
    u64 mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - mid - 1]) lo = mid + 1; else hi = mid;
  }
  apart[t] = lo;
}

template <class K>
struct MergeTile {
  u64 d0, a0, b0, na_t, nb_t;
};

// Stage one merge-path tile of A and B in shared memory.  A partition that is
// not monotone (which only unsorted input can produce) sets *err and yields an
// empty tile instead of an out-of-range read.
template <class K>
LOB_DEV MergeTile<K> load_merge_tile(const K* A, u64 na, const K* B, u64 nb, const u64* apart, K* sk, u64* err) {
  MergeTile<K> t;
  t.d0 = (u64)blockIdx.x * kMTile;
  if (t.d0 >= na + nb) {  // a tile past a device-resident total: empty
    t.a0 = na;
    t.b0 = nb;
    t.na_t = t.nb_t = 0;
    return t;
  }
  const u64 d1 = min(t.d0 + kMTile, na + nb);
  t.a0 = apart[blockIdx.x];
  const u64 a1 = apart[blockIdx.x + 1];
  t.b0 = t.d0 - t.a0;
  const u64 b1 = d1 - a1;
  if (a1 < t.a0 || b1 < t.b0 || a1 > na || b1 > nb || (a1 - t.a0) + (b1 - t.b0) > (u64)kMTile) {
    if (threadIdx.x == 0 && err) atomicExch(err, 1ull);
    t.a0 = min(t.a0, na);
    t.b0 = min(t.b0, nb);
    t.na_t = t.nb_t = 0;
    __syncthreads();
    return t;
  }
  t.na_t = a1 - t.a0;
  t.nb_t = b1 - t.b0;
  K v[kMItems];
  const u64 nt = t.na_t + t.nb_t;
#pragma unroll
  for (int j = 0; j < kMItems; j++) {  // coalesced, all loads in flight together
    const u64 i = (u64)j * kMThreads + threadIdx.x;
    v[j] = i < t.na_t ? A[t.a0 + i] : (i < nt ? B[t.b0 + (i - t.na_t)] : K(0));
  }
#pragma unroll
  for (int j = 0; j < kMItems; j++) {
    const u64 i = (u64)j * kMThreads + threadIdx.x;
    if (i < nt) sk[i] = v[j];
  }
  __syncthreads();
  return t;
}

// local merge path inside the staged tile
template <class K>
LOB_DEV u64 local_path(const K* sA, u64 na, const K* sB, u64 nb, u64 d) {
  u64 lo = d > nb ? d - nb : 0, hi = min(d, na);
  while (lo < hi) {
    u64 mid = (lo + hi) >> 1;
    if (sA[mid] <= sB[d - mid - 1]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <class K, class Sem>
struct MergeCtx {
  const K* fk; const typename Sem::Stored* ft; const u32* fs; u64 nf;
  const K* uk; const void* ut; u64 nu; int u_stored;
  K* ok; typename Sem::Stored* ot; u32* os;
  K* rk; typename Sem::Stored* rt;
  u32 stamp;
  u64* err;
  const u64* nf_dev; const u64* nu_dev;  // device-resident sizes (nf, nu are then capacities)
  const u64* stamp_dev;                  // device-resident stamp base (stamp is then added to it)
  u64 rcap;                              // R entries past it are not written (0: no limit)
  void* const* f_pp; void* const* o_pp; void* const* r_pp;  // device-resident buffer pointers
  int skip_empty;
};

template <class K, class Sem>
LOB_DEV MergeCtx<K, Sem> resolve_sizes(MergeCtx<K, Sem> c) {
  if (c.nf_dev) c.nf = *c.nf_dev < c.nf ? *c.nf_dev : c.nf;
  if (c.nu_dev) c.nu = *c.nu_dev < c.nu ? *c.nu_dev : c.nu;
  if (c.stamp_dev) c.stamp = (u32)*c.stamp_dev + c.stamp;
  if (c.f_pp) {
    c.fk = reinterpret_cast<const K*>(c.f_pp[0]);
    c.ft = reinterpret_cast<const typename Sem::Stored*>(c.f_pp[1]);
    c.fs = reinterpret_cast<const u32*>(c.f_pp[2]);
  }
  if (c.o_pp) {
    c.ok = reinterpret_cast<K*>(c.o_pp[0]);
    c.ot = reinterpret_cast<typename Sem::Stored*>(c.o_pp[1]);
    c.os = reinterpret_cast<u32*>(c.o_pp[2]);
  }
  if (c.r_pp) {
    c.rk = reinterpret_cast<K*>(c.r_pp[0]);
    c.rt = reinterpret_cast<typename Sem::Stored*>(c.r_pp[1]);
  }
  return c;
}

template <class Sem>
LOB_DEV typename Sem::Stored u_tag_stored(const void* ut, int u_stored, u64 i) {
  if (u_stored) return reinterpret_cast<const typename Sem::Stored*>(ut)[i];
  return Sem::store(reinterpret_cast<const typename Sem::Cand*>(ut)[i]);
}

template <class Sem>
LOB_DEV u32 u_clamp_bit(const void* ut, int u_stored, u64 i) {
  if constexpr (std::is_same<Sem, SemAddMult>::value) {
    if (!u_stored && reinterpret_cast<const double*>(ut)[i] > 1.0) return 0x80000000u;
  }
  return 0u;
}

// Walk this thread's merged items.  For each item calls f(isA, local a, local b, dup, improved).
template <class K, class Sem, class F>
LOB_DEV void walk_items(const MergeCtx<K, Sem>& c, const MergeTile<K>& t, const K* sk, F&& f) {
  const K* sA = sk;
  const K* sB = sk + t.na_t;
  const u64 nt = t.na_t + t.nb_t;
  const u64 diag = min((u64)threadIdx.x * kMItems, nt);
  u64 ai = local_path(sA, t.na_t, sB, t.nb_t, diag);
  u64 bi = diag - ai;
  bool have_last = false;
  K last = K(0);
  if (ai > 0) { have_last = true; last = sA[ai - 1]; }
  else if (t.a0 > 0) { have_last = true; last = c.fk[t.a0 - 1]; }
  for (int s = 0; s < kMItems && ai + bi < nt; s++) {
    const bool takeA = ai < t.na_t && (bi >= t.nb_t || sA[ai] <= sB[bi]);
    if (takeA) {
      last = sA[ai];
      have_last = true;
      f(true, ai, bi, false, false);
      ai++;
    } else {
      const bool dup = have_last && last == sB[bi];
      bool improved = false;
      if (dup && Sem::kIdempotent && Sem::kTags) {
        improved = Sem::better(u_tag_stored<Sem>(c.ut, c.u_stored, t.b0 + bi), c.ft[t.a0 + ai - 1]);
      }
      f(false, ai, bi, dup, improved);
      bi++;
    }
  }
}

template <class K, class Sem>
__global__ void __launch_bounds__(kMThreads) k_diffmerge_count(MergeCtx<K, Sem> c0, const u64* __restrict__ apart,
                                                               u64* __restrict__ tile_dup, u64* __restrict__ tile_r) {
  const MergeCtx<K, Sem> c = resolve_sizes(c0);
  if (c.skip_empty && c.nu == 0) {  // nothing to merge: zero counts, so the totals read 0
    if (threadIdx.x == 0) {
      tile_dup[blockIdx.x] = 0;
      tile_r[blockIdx.x] = 0;
    }
    return;
  }
  __shared__ K sk[kMTile];
  __shared__ u64 sm[kMThreads / 32 + 1];
  MergeTile<K> t = load_merge_tile(c.fk, c.nf, c.uk, c.nu, apart, sk, c.err);
  u64 ndup = 0, nr = 0;
  walk_items(c, t, sk, [&](bool isA, u64, u64, bool dup, bool improved) {
    if (!isA) {
      ndup += dup;
      nr += (!dup) || improved;
    }
  });
  u64 tot;
  block_exclusive_sum<u64>(ndup, sm, &tot);
  if (threadIdx.x == 0) tile_dup[blockIdx.x] = tot;
  block_exclusive_sum<u64>(nr, sm, &tot);
  if (threadIdx.x == 0) tile_r[blockIdx.x] = tot;
}

template <class K, class Sem>
__global__ void __launch_bounds__(kMThreads) k_diffmerge_write(MergeCtx<K, Sem> c0, const u64* __restrict__ apart,
                                                               const u64* __restrict__ dup_off, const u64* __restrict__ r_off) {
  const MergeCtx<K, Sem> c = resolve_sizes(c0);
  if (c.skip_empty && c.nu == 0) return;
  __shared__ K sk[kMTile];
  __shared__ u64 sm[kMThreads / 32 + 1];
  MergeTile<K> t = load_merge_tile(c.fk, c.nf, c.uk, c.nu, apart, sk, (u64*)nullptr);
  u64 ndup = 0, nr = 0;
  walk_items(c, t, sk, [&](bool isA, u64, u64, bool dup, bool improved) {
    if (!isA) {
      ndup += dup;
      nr += (!dup) || improved;
    }
  });
  u64 tot;
  u64 dups_before = dup_off[blockIdx.x] + block_exclusive_sum<u64>(ndup, sm, &tot);
  u64 rpos = r_off[blockIdx.x] + block_exclusive_sum<u64>(nr, sm, &tot);
  const K* sA = sk;
  const K* sB = sk + t.na_t;
  walk_items(c, t, sk, [&](bool isA, u64 ai, u64 bi, bool dup, bool improved) {
    const u64 d = t.d0 + ai + bi;
    if (isA) {
      const u64 ga = t.a0 + ai;
      const u64 pos = d - dups_before;
      const K k = sA[ai];
      c.ok[pos] = k;
      if constexpr (Sem::kTags) {
        typename Sem::Stored tag = c.ft[ga];
        u32 st = c.fs ? c.fs[ga] : 0u;
        if (Sem::kIdempotent) {
          // an equal U element comes right after this one in merge order
          const u64 gb = t.b0 + bi;
          const bool next_eq = bi < t.nb_t ? (sB[bi] == k) : (gb < c.nu && c.uk[gb] == k);
          if (next_eq) {
            typename Sem::Stored ut = u_tag_stored<Sem>(c.ut, c.u_stored, gb);
            if (Sem::better(ut, tag)) { tag = ut; st = c.stamp; }
          }
        }
        c.ot[pos] = tag;
        if (c.os) c.os[pos] = st;
      } else {
        if (c.os) c.os[pos] = c.fs ? c.fs[ga] : 0u;
      }
    } else {
      const u64 gb = t.b0 + bi;
      const K k = sB[bi];
      if (!dup) {
        const u64 pos = d - dups_before;
        c.ok[pos] = k;
        if constexpr (Sem::kTags) c.ot[pos] = u_tag_stored<Sem>(c.ut, c.u_stored, gb);
        if (c.os) c.os[pos] = c.stamp | u_clamp_bit<Sem>(c.ut, c.u_stored, gb);
      } else {
        dups_before++;
      }
      if (!dup || improved) {
        if (c.rk && (!c.rcap || rpos < c.rcap)) {
          c.rk[rpos] = k;
          if constexpr (Sem::kTags) c.rt[rpos] = u_tag_stored<Sem>(c.ut, c.u_stored, gb);
        }
        rpos++;
      }
    }
  });
}

// ---------------------------------------------------------------------------
// combine: merge two sorted distinct-key lists, (+)-combining shared keys
// (accumulates the unique candidates of several chunks of one iteration)
// ---------------------------------------------------------------------------
template <class K, class F>
LOB_DEV void walk_merge(const K* A, const MergeTile<K>& t, const K* sk, F&& f) {
  const K* sA = sk;
  const K* sB = sk + t.na_t;
  const u64 nt = t.na_t + t.nb_t;
  const u64 diag = min((u64)threadIdx.x * kMItems, nt);
  u64 ai = local_path(sA, t.na_t, sB, t.nb_t, diag);
  u64 bi = diag - ai;
  bool have_last = false;
  K last = K(0);
  if (ai > 0) { have_last = true; last = sA[ai - 1]; }
  else if (t.a0 > 0) { have_last = true; last = A[t.a0 - 1]; }
  for (int s = 0; s < kMItems && ai + bi < nt; s++) {
    if (ai < t.na_t && (bi >= t.nb_t || sA[ai] <= sB[bi])) {
      last = sA[ai];
      have_last = true;
      f(true, ai, bi, false);
      ai++;
    } else {
      f(false, ai, bi, have_last && last == sB[bi]);
      bi++;
    }
  }
}

template <class K>
__global__ void __launch_bounds__(kMThreads) k_combine_count(const K* __restrict__ A, u64 na, const K* __restrict__ B, u64 nb,
                                                             const u64* __restrict__ apart, u64* __restrict__ tile_dup,
                                                             u64* err) {
  __shared__ K sk[kMTile];
  __shared__ u64 sm[kMThreads / 32 + 1];
  MergeTile<K> t = load_merge_tile(A, na, B, nb, apart, sk, err);
  u64 ndup = 0;
  walk_merge(A, t, sk, [&](bool isA, u64, u64, bool dup) { ndup += (!isA) && dup; });
  u64 tot;
  block_exclusive_sum<u64>(ndup, sm, &tot);
  if (threadIdx.x == 0) tile_dup[blockIdx.x] = tot;
}

template <class K, class Sem>
__global__ void __launch_bounds__(kMThreads) k_combine_write(const K* __restrict__ A, const typename Sem::Cand* __restrict__ at,
                                                             u64 na, const K* __restrict__ B,
                                                             const typename Sem::Cand* __restrict__ bt, u64 nb,
                                                             const u64* __restrict__ apart, const u64* __restrict__ dup_off,
                                                             K* __restrict__ ok, typename Sem::Cand* __restrict__ ot) {
  __shared__ K sk[kMTile];
  __shared__ u64 sm[kMThreads / 32 + 1];
  MergeTile<K> t = load_merge_tile(A, na, B, nb, apart, sk, (u64*)nullptr);
  u64 ndup = 0;
  walk_merge(A, t, sk, [&](bool isA, u64, u64, bool dup) { ndup += (!isA) && dup; });
  u64 tot;
  u64 dups_before = dup_off[blockIdx.x] + block_exclusive_sum<u64>(ndup, sm, &tot);
  const K* sA = sk;
  const K* sB = sk + t.na_t;
  walk_merge(A, t, sk, [&](bool isA, u64 ai, u64 bi, bool dup) {
    const u64 d = t.d0 + ai + bi;
    if (isA) {
      const u64 pos = d - dups_before;
      const K k = sA[ai];
      ok[pos] = k;
      if constexpr (Sem::kTags) {
        typename Sem::Cand tag = at[t.a0 + ai];
        const u64 gb = t.b0 + bi;
        const bool next_eq = bi < t.nb_t ? (sB[bi] == k) : (gb < nb && B[gb] == k);
        if (next_eq) tag = Sem::add(tag, bt[gb]);
        ot[pos] = tag;
      }
    } else if (dup) {
      dups_before++;
    } else {
      const u64 pos = d - dups_before;
      ok[pos] = sB[bi];
      if constexpr (Sem::kTags) ot[pos] = bt[t.b0 + bi];
    }
  });
}

template <class K, class Sem>
void combine_impl(const void* a, const void* at, u64 na, const void* b, const void* bt, u64 nb, void* o, void* ot,
                  u64* count_dev, void* scratch, cudaStream_t st) {
  typedef typename Sem::Cand C;
  const u64 tiles = (na + nb + kMTile - 1) / kMTile;
  u64* apart = reinterpret_cast<u64*>(scratch);
  u64* tdup = apart + tiles + 1;
  u64* ws = tdup + tiles + 1;
  cudaMemsetAsync(count_dev + 1, 0, sizeof(u64), st);
  const double kb = sizeof(K), cb = Sem::kTags ? sizeof(C) : 0;
  { ProfScope ps("merge_path", (tiles + 1) * 8.0, st);
    k_merge_path<K><<<(unsigned)((tiles + 1 + 255) / 256), 256, 0, st>>>((const K*)a, na, (const K*)b, nb, tiles + 1, apart); }
  { ProfScope ps("combine_count", (na + nb) * kb, st);
    k_combine_count<K><<<(unsigned)tiles, kMThreads, 0, st>>>((const K*)a, na, (const K*)b, nb, apart, tdup, count_dev + 1); }
  exclusive_scan<u64, u64>(tdup, tdup, tiles, count_dev, ws, st);
  { ProfScope ps("combine_write", 2.0 * (na + nb) * (kb + cb), st);
    k_combine_write<K, Sem><<<(unsigned)tiles, kMThreads, 0, st>>>((const K*)a, (const C*)at, na, (const K*)b, (const C*)bt,
                                                                   nb, apart, tdup, (K*)o, (C*)ot); }
}

// ---------------------------------------------------------------------------
// merge of two sorted key lists that share no key: output position = a + b
// ---------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(kMThreads) k_merge_nodup(const K* __restrict__ A, u64 na, const K* __restrict__ B, u64 nb,
                                                           const u64* __restrict__ apart, K* __restrict__ out) {
  __shared__ K sk[kMTile];
  MergeTile<K> t = load_merge_tile(A, na, B, nb, apart, sk, (u64*)nullptr);
  const K* sA = sk;
  const K* sB = sk + t.na_t;
  const u64 nt = t.na_t + t.nb_t;
  const u64 diag = min((u64)threadIdx.x * kMItems, nt);
  u64 ai = local_path(sA, t.na_t, sB, t.nb_t, diag);
  u64 bi = diag - ai;
  // each thread merges its run of at most kMItems outputs into registers; the
  // tile is then written back through shared memory with coalesced stores
  K v[kMItems];
  int m = 0;
  for (int s = 0; s < kMItems && ai + bi < nt; s++) {
    if (ai < t.na_t && (bi >= t.nb_t || sA[ai] <= sB[bi])) v[m++] = sA[ai++];
    else v[m++] = sB[bi++];
  }
  __syncthreads();
  for (int s = 0; s < m; s++) sk[diag + s] = v[s];
  __syncthreads();
  for (u64 i = threadIdx.x; i < nt; i += kMThreads) out[t.d0 + i] = sk[i];
}

// ---------------------------------------------------------------------------
// load: sorted (key, row) pairs -> unique facts, tags (+)-merged over the rows
// ---------------------------------------------------------------------------
template <class Sem>
LOB_DEV typename Sem::Cand row_tag(const float* raw, u64 row, u32 id_base, int differentiable) {
  if constexpr (std::is_same<Sem, SemDiffMaxMin>::value) {
    float v = raw ? raw[row] : 1.0f;
    return dmm_pack(v, differentiable ? id_base + (u32)row : 0xFFFFFFFFu);
  } else if constexpr (std::is_same<Sem, SemTop1>::value) {
    // a row with a probability is the proof {its id}, whose arena entry sits at
    // word 1 + 2 id; a row without one has the empty proof (word 0, probability 1)
    if (!raw || !differentiable) return SemTop1::one();
    return ((u64)__float_as_uint(raw[row]) << 32) | (u64)(1u + 2u * (id_base + (u32)row));
  } else if constexpr (std::is_same<Sem, SemUnit>::value) {
    return 1u;
  } else {
    return (typename Sem::Cand)(raw ? raw[row] : 1.0f);
  }
}

template <class K, class Sem>
__global__ void __launch_bounds__(kUThreads) k_load_write(const K* __restrict__ keys, const u32* __restrict__ rows, u64 n,
                                                          const float* __restrict__ raw, u32 id_base, int differentiable,
                                                          const u64* __restrict__ tile_off, K* __restrict__ okeys,
                                                          typename Sem::Stored* __restrict__ otags, u32* __restrict__ ostamp,
                                                          float* __restrict__ row_factor) {
  __shared__ u64 sm[kUThreads / 32 + 1];
  const u64 base = (u64)blockIdx.x * kUTile + (u64)threadIdx.x * kUItems;
  u32 heads = 0;
#pragma unroll
  for (int i = 0; i < kUItems; i++) {
    u64 idx = base + i;
    if (idx < n && is_head(keys, idx, keys[idx])) heads |= 1u << i;
  }
  u64 total;
  u64 o = tile_off[blockIdx.x] + block_exclusive_sum<u64>((u64)__popc(heads), sm, &total);
#pragma unroll 1
  for (int i = 0; i < kUItems; i++) {
    if (!(heads >> i & 1u)) continue;
    const u64 idx = base + i;
    const K k = keys[idx];
    okeys[o] = k;
    if (ostamp) ostamp[o] = 0u;
    if constexpr (Sem::kTags) {
      typename Sem::Cand acc = row_tag<Sem>(raw, rows[idx], id_base, differentiable);
      u64 j = idx + 1;
      for (; j < n && keys[j] == k; j++) acc = Sem::add(acc, row_tag<Sem>(raw, rows[j], id_base, differentiable));
      otags[o] = Sem::store(acc);
      if (row_factor) {
        float f = 1.0f;
        if constexpr (std::is_same<Sem, SemAddMult>::value) f = acc > 1.0 ? 0.0f : 1.0f;
        for (u64 q = idx; q < j; q++) row_factor[rows[q]] = f;
      }
    }
    o++;
  }
}

template <class Sem>
void dispatch_unique(int key64, const void* keys, const void* tags, u64 n, void* okeys, void* otags, u64* count_dev,
                     void* scratch, cudaStream_t st) {
  const u64 tiles = (n + kUTile - 1) / kUTile;
  u64* tile = reinterpret_cast<u64*>(scratch);
  u64* ws = tile + tiles + 1;
  typedef typename Sem::Cand C;
  const double kb = key64 ? 8 : 4, cb = Sem::kTags ? sizeof(C) : 0;
  if (key64) {
    { ProfScope ps("unique_count", n * kb, st);
      k_unique_count<u64><<<(unsigned)tiles, kUThreads, 0, st>>>((const u64*)keys, n, tile); }
    { ProfScope ps("unique_scan", tiles * 16.0, st); exclusive_scan<u64, u64>(tile, tile, tiles, count_dev, ws, st); }
    { ProfScope ps("unique_write", n * (kb + cb), st);
      k_unique_write<u64, Sem><<<(unsigned)tiles, kUThreads, 0, st>>>((const u64*)keys, (const C*)tags, n, tile, (u64*)okeys, (C*)otags); }
  } else {
    { ProfScope ps("unique_count", n * kb, st);
      k_unique_count<u32><<<(unsigned)tiles, kUThreads, 0, st>>>((const u32*)keys, n, tile); }
    { ProfScope ps("unique_scan", tiles * 16.0, st); exclusive_scan<u64, u64>(tile, tile, tiles, count_dev, ws, st); }
    { ProfScope ps("unique_write", n * (kb + cb), st);
      k_unique_write<u32, Sem><<<(unsigned)tiles, kUThreads, 0, st>>>((const u32*)keys, (const C*)tags, n, tile, (u32*)okeys, (C*)otags); }
  }
}

template <class K, class Sem>
void merge_impl(const MergeArgs& a, void* scratch, cudaStream_t st) {
  const u64 tot = a.nf + a.nu;
  const u64 tiles = (tot + kMTile - 1) / kMTile;
  u64* apart = reinterpret_cast<u64*>(scratch);
  u64* tdup = apart + tiles + 1;
  u64* tr = tdup + tiles + 1;
  u64* ws = tr + tiles + 1;
  MergeCtx<K, Sem> c{};
  c.fk = (const K*)a.fkeys; c.ft = (const typename Sem::Stored*)a.ftags; c.fs = a.fstamp; c.nf = a.nf;
  c.uk = (const K*)a.ukeys; c.ut = a.utags; c.nu = a.nu; c.u_stored = a.u_stored;
  c.ok = (K*)a.okeys; c.ot = (typename Sem::Stored*)a.otags; c.os = a.ostamp;
  c.rk = (K*)a.rkeys; c.rt = (typename Sem::Stored*)a.rtags;
  c.stamp = a.stamp;
  // counts_dev[2]: set by a merge tile whose partition is not monotone (the
  // inputs were not sorted distinct keys); cleared here so that every call
  // reports only its own inputs
  c.err = a.counts_dev + 2;
  c.nf_dev = a.nf_dev;
  c.nu_dev = a.nu_dev;
  c.stamp_dev = a.stamp_dev;
  c.rcap = a.rcap;
  c.f_pp = a.f_pp;
  c.o_pp = a.o_pp;
  c.r_pp = a.r_pp;
  c.skip_empty = a.skip_empty;
  cudaMemsetAsync(c.err, 0, sizeof(u64), st);
  const double kb = sizeof(K), sb = Sem::kTags ? sizeof(typename Sem::Stored) : 0, ub = a.u_stored ? sb : (Sem::kTags ? sizeof(typename Sem::Cand) : 0);
  const double fsb = a.fstamp ? 4 : 0;
  { ProfScope ps("merge_path", (tiles + 1) * 8.0, st);
    k_merge_path<K><<<(unsigned)((tiles + 1 + 255) / 256), 256, 0, st>>>(c.fk, a.nf, c.uk, a.nu, tiles + 1, apart,
                                                                          a.nf_dev, a.nu_dev, a.f_pp, a.skip_empty); }
  { ProfScope ps("diffmerge_count", (a.nf + a.nu) * kb, st);
    k_diffmerge_count<K, Sem><<<(unsigned)tiles, kMThreads, 0, st>>>(c, apart, tdup, tr); }
  { ProfScope ps("diffmerge_scan", tiles * 32.0, st);
    exclusive_scan<u64, u64>(tdup, tdup, tiles, a.counts_dev, ws, st);
    exclusive_scan<u64, u64>(tr, tr, tiles, a.counts_dev + 1, ws, st); }
  // algorithmic: read F and U once; write F' (<= nf + nu rows) and R (<= nu rows)
  { ProfScope ps("diffmerge_write", a.nf * (kb + sb + fsb) + a.nu * (kb + ub) + (a.nf + a.nu) * (kb + sb + fsb) +
                                        (a.rkeys ? a.nu * (kb + sb) : 0.0), st);
    k_diffmerge_write<K, Sem><<<(unsigned)tiles, kMThreads, 0, st>>>(c, apart, tdup, tr); }
}

template <class K, class Sem>
void load_impl(const LoadUniqueArgs& a, void* scratch, cudaStream_t st) {
  const u64 tiles = (a.n + kUTile - 1) / kUTile;
  u64* tile = reinterpret_cast<u64*>(scratch);
  u64* ws = tile + tiles + 1;
  k_unique_count<K><<<(unsigned)tiles, kUThreads, 0, st>>>((const K*)a.keys, a.n, tile);
  exclusive_scan<u64, u64>(tile, tile, tiles, a.count_dev, ws, st);
  k_load_write<K, Sem><<<(unsigned)tiles, kUThreads, 0, st>>>((const K*)a.keys, a.rows, a.n, a.raw_tags, a.id_base,
                                                             a.differentiable, tile, (K*)a.okeys,
                                                             (typename Sem::Stored*)a.otags, a.ostamp, a.row_factor);
}

}  // namespace

size_t unique_scratch_bytes(u64 n) {
  const u64 tiles = (n + kUTile - 1) / kUTile;
  return (tiles + 1 + scan_scratch_elems(tiles) + 8) * sizeof(u64);
}

void unique_run(int sem, int key64, const void* keys, const void* tags, u64 n, void* okeys, void* otags, u64* count_dev,
                void* scratch, cudaStream_t st) {
  if (n == 0) {
    cudaMemsetAsync(count_dev, 0, sizeof(u64), st);
    return;
  }
  switch (sem) {
    case SR_UNIT: dispatch_unique<SemUnit>(key64, keys, tags, n, okeys, otags, count_dev, scratch, st); break;
    case SR_MAX_MIN: dispatch_unique<SemMaxMin>(key64, keys, tags, n, okeys, otags, count_dev, scratch, st); break;
    case SR_DIFF_MAX_MIN: dispatch_unique<SemDiffMaxMin>(key64, keys, tags, n, okeys, otags, count_dev, scratch, st); break;
    case SR_TOP1: dispatch_unique<SemTop1>(key64, keys, tags, n, okeys, otags, count_dev, scratch, st); break;
    default: dispatch_unique<SemAddMult>(key64, keys, tags, n, okeys, otags, count_dev, scratch, st); break;
  }
}

size_t merge_scratch_bytes(u64 nf, u64 nu) {
  const u64 tiles = (nf + nu + kMTile - 1) / kMTile;
  return (3 * (tiles + 1) + scan_scratch_elems(tiles) + 8) * sizeof(u64);
}

void diff_merge(const MergeArgs& a, void* scratch, cudaStream_t st) {
  if (a.nu == 0) return;
  const int sem = a.sem;
#define LOB_MERGE(K)                                                              \
  switch (sem) {                                                                  \
    case SR_UNIT: merge_impl<K, SemUnit>(a, scratch, st); break;                  \
    case SR_MAX_MIN: merge_impl<K, SemMaxMin>(a, scratch, st); break;             \
    case SR_DIFF_MAX_MIN: merge_impl<K, SemDiffMaxMin>(a, scratch, st); break;    \
    case SR_TOP1: merge_impl<K, SemTop1>(a, scratch, st); break;                  \
    default: merge_impl<K, SemAddMult>(a, scratch, st); break;                    \
  }
  if (a.key64) { LOB_MERGE(u64) } else { LOB_MERGE(u32) }
#undef LOB_MERGE
}

size_t merge_nodup_scratch_bytes(u64 na, u64 nb) { return ((na + nb) / kMTile + 8) * sizeof(u64); }

void merge_nodup(int key64, const void* a, u64 na, const void* b, u64 nb, void* out, void* scratch, cudaStream_t st) {
  const u64 tiles = (na + nb + kMTile - 1) / kMTile;
  if (!tiles) return;
  u64* apart = reinterpret_cast<u64*>(scratch);
  const double kb = key64 ? 8 : 4;
  ProfScope ps("merge_nodup", 2.0 * (na + nb) * kb, st);
  if (key64) {
    k_merge_path<u64><<<(unsigned)((tiles + 1 + 255) / 256), 256, 0, st>>>((const u64*)a, na, (const u64*)b, nb, tiles + 1, apart);
    k_merge_nodup<u64><<<(unsigned)tiles, kMThreads, 0, st>>>((const u64*)a, na, (const u64*)b, nb, apart, (u64*)out);
  } else {
    k_merge_path<u32><<<(unsigned)((tiles + 1 + 255) / 256), 256, 0, st>>>((const u32*)a, na, (const u32*)b, nb, tiles + 1, apart);
    k_merge_nodup<u32><<<(unsigned)tiles, kMThreads, 0, st>>>((const u32*)a, na, (const u32*)b, nb, apart, (u32*)out);
  }
}

size_t combine_scratch_bytes(u64 na, u64 nb) {
  const u64 tiles = (na + nb + kMTile - 1) / kMTile;
  return (2 * (tiles + 1) + scan_scratch_elems(tiles) + 8) * sizeof(u64);
}

// count_dev[0] = number of distinct keys written (na + nb - shared keys)
void combine_merge(int sem, int key64, const void* akeys, const void* atags, u64 na, const void* bkeys,
                   const void* btags, u64 nb, void* okeys, void* otags, u64* count_dev, void* scratch, cudaStream_t st) {
#define LOB_COMB(K)                                                                                                   \
  switch (sem) {                                                                                                      \
    case SR_UNIT: combine_impl<K, SemUnit>(akeys, atags, na, bkeys, btags, nb, okeys, otags, count_dev, scratch, st); break; \
    case SR_MAX_MIN: combine_impl<K, SemMaxMin>(akeys, atags, na, bkeys, btags, nb, okeys, otags, count_dev, scratch, st); break; \
    case SR_DIFF_MAX_MIN: combine_impl<K, SemDiffMaxMin>(akeys, atags, na, bkeys, btags, nb, okeys, otags, count_dev, scratch, st); break; \
    case SR_TOP1: combine_impl<K, SemTop1>(akeys, atags, na, bkeys, btags, nb, okeys, otags, count_dev, scratch, st); break; \
    default: combine_impl<K, SemAddMult>(akeys, atags, na, bkeys, btags, nb, okeys, otags, count_dev, scratch, st); break; \
  }
  if (key64) { LOB_COMB(u64) } else { LOB_COMB(u32) }
#undef LOB_COMB
}

void load_unique(const LoadUniqueArgs& a, void* scratch, cudaStream_t st) {
  if (a.n == 0) {
    cudaMemsetAsync(a.count_dev, 0, sizeof(u64), st);
    return;
  }
#define LOB_LOAD(K)                                                            \
  switch (a.sem) {                                                             \
    case SR_UNIT: load_impl<K, SemUnit>(a, scratch, st); break;                \
    case SR_MAX_MIN: load_impl<K, SemMaxMin>(a, scratch, st); break;           \
    case SR_DIFF_MAX_MIN: load_impl<K, SemDiffMaxMin>(a, scratch, st); break;  \
    case SR_TOP1: load_impl<K, SemTop1>(a, scratch, st); break;                \
    default: load_impl<K, SemAddMult>(a, scratch, st); break;                  \
  }
  if (a.key64) { LOB_LOAD(u64) } else { LOB_LOAD(u32) }
#undef LOB_LOAD
}
