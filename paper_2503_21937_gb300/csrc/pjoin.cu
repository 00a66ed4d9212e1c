// Packed join pipeline: the same count / emit steps as join.cu, specialised
// for rules whose intermediate bindings fit one 64-bit word.
//
// Every rule variable lives in a bit field of either the input word (a packed
// relation key, or a packed binding row of the previous step) or the matched
// view key.  The plan compiles each step into operand lists -- (word, shift,
// width) or a constant -- for the probe prefix, the equality / inequality
// checks and the output word, so the kernels only shift, mask, compare and OR
// values held in registers.  A dropped binding row is the all-ones word (no
// field is ever all ones, so no valid row is).
#include <algorithm>

#include "pjoin.h"

namespace {

LOB_DEV u64 pick(const POperand& o, u64 wi, u64 wv) {
  if (o.word == 2) return o.cval;
  const u64 w = o.word ? wv : wi;
  return (w >> o.shift) & (o.width >= 64 ? ~0ull : ((1ull << o.width) - 1ull));
}

LOB_DEV u64 load_word(const void* p, int w64, u64 i) {
  return w64 ? reinterpret_cast<const u64*>(p)[i] : (u64)reinterpret_cast<const u32*>(p)[i];
}

LOB_DEV bool checks_ok(const PCheck* c, int n, u64 wi, u64 wv) {
  bool ok = true;
#pragma unroll 4
  for (int q = 0; q < n; q++) ok = ok && ((pick(c[q].a, wi, wv) == pick(c[q].b, wi, wv)) == (c[q].eq != 0));
  return ok;
}

LOB_DEV u64 compose(const PField* f, int n, u64 wi, u64 wv) {
  u64 o = 0;
#pragma unroll 4
  for (int q = 0; q < n; q++) o |= pick(f[q].op, wi, wv) << f[q].shift;
  return o;
}

// input row r: its word, or false when the row is dropped / filtered
template <class Sem>
LOB_DEV bool input_row(const PStep& P, const PPtrs& Q, u64 r, u64& wi, typename Sem::Cand& tag) {
  if (P.in_stamp_mode != STAMP_NONE) {
    u32 s = P.in_stamp[r] & 0x7FFFFFFFu;
    if (P.in_stamp_mode == STAMP_LT ? !(s < P.in_stamp_val) : s != P.in_stamp_val) return false;
  }
  wi = load_word(Q.in_words, P.in_w64, r);
  if (wi == (P.in_w64 ? ~0ull : 0xFFFFFFFFull)) return false;
  if (!checks_ok(P.in_checks, P.n_in_checks, wi, 0)) return false;
  if constexpr (Sem::kTags) {
    if (P.in_packed) tag = Sem::from_stored(reinterpret_cast<const typename Sem::Stored*>(Q.in_tags)[r]);
    else tag = reinterpret_cast<const typename Sem::Cand*>(Q.in_tags)[r];
  } else {
    tag = Sem::one();
  }
  return true;
}

LOB_DEV u64 lower_bound_w(const void* keys, int key64, u64 n, u64 x) {
  u64 lo = 0, hi = n;
  if (key64) {
    const u64* a = reinterpret_cast<const u64*>(keys);
    while (lo < hi) { const u64 m = (lo + hi) >> 1; if (a[m] < x) lo = m + 1; else hi = m; }
  } else {
    if (x > 0xFFFFFFFFull) return n;
    const u32* a = reinterpret_cast<const u32*>(keys);
    const u32 y = (u32)x;
    while (lo < hi) { const u64 m = (lo + hi) >> 1; if (a[m] < y) lo = m + 1; else hi = m; }
  }
  return lo;
}

LOB_DEV u64 row_off(const PStep& P, u64 r) { return P.blk_off[r / kLocRows] + P.loc[r]; }

template <class Sem, int kFilter>
__global__ void __launch_bounds__(256) k_pemit(const __grid_constant__ PStep P, const u64* __restrict__ part) {
  typedef typename Sem::Stored S;
  typedef typename Sem::Cand C;
  constexpr int kItems = kEmitTile / 256;
  __shared__ __align__(16) u32 row_of[kEmitTile];
  __shared__ u32 sm[256 / 32 + 1];
  __shared__ u32 th_inc[256];
  __shared__ u64 block_base;
  // tiles of kEmitTile outputs; a block takes tiles blockIdx.x, + gridDim.x, ...
  // (one tile per block when the grid has one block per tile)
  const u64 j_end = P.j_begin + dev_size(P.total, P.total_dev);
  const PPtrs Q = resolve_ptrs(P);
  for (u64 tile = blockIdx.x;; tile += gridDim.x) {
  const u64 j0 = P.j_begin + tile * kEmitTile;
  if (j0 >= j_end) break;
  const u64 r0 = part[tile];
  const u64 r_end = part[tile + 1];
  for (int i = threadIdx.x; i < kEmitTile; i += 256) row_of[i] = 0;
  __syncthreads();
  for (u64 r = r0 + 1 + threadIdx.x; r <= r_end; r += 256) {
    const u64 o = row_off(P, r);
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
  const u64 invalid_out = P.out_w64 ? ~0ull : 0xFFFFFFFFull;
  const u32 vsv = P.stamp_dev ? (u32)*P.stamp_dev + P.v_stamp_val : P.v_stamp_val;
  u64 kept[kFilter == 1 ? kItems : 1];
  u32 nkeep = 0;
#pragma unroll 2
  for (int i = 0; i < kItems; i++) {
    const u64 j = j0 + (u64)i * 256 + threadIdx.x;
    if (j >= j_end) break;
    const u64 r = r0 + row_of[j - j0];
    const u64 v = (u64)P.lo32[r] + (j - row_off(P, r));
    u64 wi;
    C tag;
    input_row<Sem>(P, Q, r, wi, tag);
    const u64 wv = load_word(Q.v_keys, P.v_key64, v);
    bool ok = P.v_stamp_mode == STAMP_NONE ||
              (P.v_stamp_mode == STAMP_LT ? (Q.v_stamp[v] & 0x7FFFFFFFu) < vsv : (Q.v_stamp[v] & 0x7FFFFFFFu) == vsv);
    ok = ok && checks_ok(P.checks, P.n_checks, wi, wv);
    const u64 w = ok ? compose(P.out, P.n_out, wi, wv) : invalid_out;
    if constexpr (kFilter == 3) {
      if (!ok) continue;
      dense_add<Sem>(P.acc, w, Sem::mul(tag, Sem::from_stored(reinterpret_cast<const S*>(Q.v_tags)[v])));
      touch_bit(P.bitmap, w);
    } else if constexpr (kFilter) {
      if (!ok) continue;
      const u32 bit = 1u << (u32)(w & 31u);
      u32* word = P.bitmap + (w >> 5);
      if constexpr (kFilter == 2) {  // bitmap only: set the bit, no old value needed
        atomicOr(word, bit);
        continue;
      }
      if (*reinterpret_cast<volatile u32*>(word) & bit) continue;  // a known fact: no atomic needed
      if (atomicOr(word, bit) & bit) continue;
      if constexpr (kFilter == 1) kept[nkeep++] = w;
    } else {
      const u64 o = P.out_base + (j - P.j_begin);
      if (P.out_w64) reinterpret_cast<u64*>(P.out_words)[o] = w;
      else reinterpret_cast<u32*>(P.out_words)[o] = (u32)w;
      if constexpr (Sem::kTags) reinterpret_cast<C*>(P.out_tags)[o] = Sem::mul(tag, Sem::from_stored(reinterpret_cast<const S*>(Q.v_tags)[v]));
    }
  }
  if constexpr (kFilter == 1) {
    // compact the tile's survivors in shared memory (reusing row_of), then
    // store them with consecutive threads writing consecutive words
    u32 tot;
    const u32 mine = block_exclusive_sum<u32>(nkeep, sm, &tot);
    if (threadIdx.x == 0) block_base = tot ? atomicAdd(reinterpret_cast<unsigned long long*>(P.out_count), (u64)tot) : 0ull;
    __syncthreads();
    const u64 base = P.out_base + block_base;
    if (P.out_w64) {
      u64* stage = reinterpret_cast<u64*>(row_of);  // kEmitTile u32 = kEmitTile / 2 u64 slots
      for (u32 c0 = 0; c0 < tot; c0 += kEmitTile / 2) {
        for (u32 q = 0; q < nkeep; q++) {
          const u32 pos = mine + q;
          if (pos >= c0 && pos < c0 + kEmitTile / 2) stage[pos - c0] = kept[q];
        }
        __syncthreads();
        const u32 lim = min(tot - c0, (u32)(kEmitTile / 2));
        for (u32 i = threadIdx.x; i < lim; i += 256) reinterpret_cast<u64*>(P.out_words)[base + c0 + i] = stage[i];
        __syncthreads();
      }
    } else {
      for (u32 q = 0; q < nkeep; q++) row_of[mine + q] = (u32)kept[q];
      __syncthreads();
      for (u32 i = threadIdx.x; i < tot; i += 256) reinterpret_cast<u32*>(P.out_words)[base + i] = row_of[i];
    }
  }
  __syncthreads();  // shared memory is reused by the block's next tile
  }
}

template <class Sem>
__global__ void __launch_bounds__(256) k_pproject(const __grid_constant__ PStep P) {
  typedef typename Sem::Cand C;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 invalid_out = P.out_w64 ? ~0ull : 0xFFFFFFFFull;
  const PPtrs Q = resolve_ptrs(P);
  for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < P.n_in; r += stride) {
    u64 wi;
    C tag = Sem::one();
    const bool ok = input_row<Sem>(P, Q, r, wi, tag);
    const u64 w = ok ? compose(P.out, P.n_out, wi, 0) : invalid_out;
    const u64 o = P.out_base + r;
    if (P.out_w64) reinterpret_cast<u64*>(P.out_words)[o] = w;
    else reinterpret_cast<u32*>(P.out_words)[o] = (u32)w;
    if constexpr (Sem::kTags) reinterpret_cast<C*>(P.out_tags)[o] = tag;
  }
}


// ---------------------------------------------------------------------------
// Specialised emission: the numbers of output fields (NOUT) and of checks
// (NCHK) are compile-time, so operand descriptors live in registers and every
// field costs a select, two shifts, a mask and an OR.  Each thread's outputs are
// processed in phases -- all row lookups, then all row-offset / match-start /
// input-word loads, then all matched-key loads, then the arithmetic -- so a
// thread keeps many independent loads in flight instead of one dependent chain.
// ---------------------------------------------------------------------------
struct RegOp {
  u64 mask;
  u32 cval;
  uint8_t shift, word;
};

LOB_DEV RegOp reg_op(const POperand& o) {
  RegOp r;
  r.mask = o.width >= 64 ? ~0ull : ((1ull << o.width) - 1ull);
  r.shift = o.shift;
  r.word = o.word;
  r.cval = o.cval;
  return r;
}
LOB_DEV u64 reg_pick(const RegOp& o, u64 wi, u64 wv) {
  return o.word == 2 ? (u64)o.cval : (((o.word ? wv : wi) >> o.shift) & o.mask);
}

template <class Sem, int kFilter, int NOUT, int NCHK>
__global__ void __launch_bounds__(256) k_pemit_fast(const __grid_constant__ PStep P, const u64* __restrict__ part) {
  typedef typename Sem::Stored S;
  typedef typename Sem::Cand C;
  constexpr int kItems = kEmitTile / 256;
  __shared__ __align__(16) u32 row_of[kEmitTile];
  __shared__ u32 sm[256 / 32 + 1];
  __shared__ u32 th_inc[256];
  __shared__ u64 block_base;
  // tiles of kEmitTile outputs; a block takes tiles blockIdx.x, + gridDim.x, ...
  // (one tile per block when the grid has one block per tile)
  const u64 j_end = P.j_begin + dev_size(P.total, P.total_dev);
  const PPtrs Q = resolve_ptrs(P);
  for (u64 tile = blockIdx.x;; tile += gridDim.x) {
  const u64 j0 = P.j_begin + tile * kEmitTile;
  if (j0 >= j_end) break;
  const u64 r0 = part[tile];
  const u64 r_end = part[tile + 1];
  for (int i = threadIdx.x; i < kEmitTile; i += 256) row_of[i] = 0;
  __syncthreads();
  for (u64 r = r0 + 1 + threadIdx.x; r <= r_end; r += 256) {
    const u64 o = row_off(P, r);
    if (o < j0 + kEmitTile) atomicMax(&row_of[o - j0], (u32)(r - r0));
  }
  __syncthreads();
  {
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
  }
  __syncthreads();
  RegOp out_op[NOUT];
  u32 out_sh[NOUT];
#pragma unroll
  for (int q = 0; q < NOUT; q++) {
    out_op[q] = reg_op(P.out[q].op);
    out_sh[q] = P.out[q].shift;
  }
  RegOp ca[NCHK > 0 ? NCHK : 1], cb[NCHK > 0 ? NCHK : 1];
  bool ceq[NCHK > 0 ? NCHK : 1];
#pragma unroll
  for (int q = 0; q < NCHK; q++) {
    ca[q] = reg_op(P.checks[q].a);
    cb[q] = reg_op(P.checks[q].b);
    ceq[q] = P.checks[q].eq != 0;
  }
  const u64 invalid_out = P.out_w64 ? ~0ull : 0xFFFFFFFFull;
  const u64 invalid_in = P.in_w64 ? ~0ull : 0xFFFFFFFFull;
  const u32 vsv = P.stamp_dev ? (u32)*P.stamp_dev + P.v_stamp_val : P.v_stamp_val;
  u64 kept[kFilter == 1 ? kItems : 1];
  u32 nkeep = 0;
  constexpr int B = kFilter == 2 ? 4 : 2;  // outputs whose loads are issued together (keeps registers, and occupancy, up)
#pragma unroll 1
  for (int i0 = 0; i0 < kItems; i0 += B) {
    u32 rr[B];
    u64 offv[B], wi[B], wv[B];
    u32 lov[B];
#pragma unroll
    for (int b = 0; b < B; b++) {
      const u64 j = j0 + (u64)(i0 + b) * 256 + threadIdx.x;
      rr[b] = j < j_end ? row_of[j - j0] : 0u;
    }
#pragma unroll
    for (int b = 0; b < B; b++) {
      const u64 r = r0 + rr[b];
      offv[b] = row_off(P, r);
      lov[b] = P.lo32[r];
      wi[b] = load_word(Q.in_words, P.in_w64, r);
    }
#pragma unroll
    for (int b = 0; b < B; b++) {
      const u64 j = j0 + (u64)(i0 + b) * 256 + threadIdx.x;
      wv[b] = j < j_end ? load_word(Q.v_keys, P.v_key64, (u64)lov[b] + (j - offv[b])) : 0ull;
    }
#pragma unroll
    for (int b = 0; b < B; b++) {
      const u64 j = j0 + (u64)(i0 + b) * 256 + threadIdx.x;
      if (j >= j_end) continue;
      bool ok = wi[b] != invalid_in;
      if (P.n_in_checks) ok = ok && checks_ok(P.in_checks, P.n_in_checks, wi[b], 0);
      const u64 v = (u64)lov[b] + (j - offv[b]);
      if (P.v_stamp_mode != STAMP_NONE) {
        const u32 st = Q.v_stamp[v] & 0x7FFFFFFFu;
        ok = ok && (P.v_stamp_mode == STAMP_LT ? st < vsv : st == vsv);
      }
#pragma unroll
      for (int q = 0; q < NCHK; q++) ok = ok && ((reg_pick(ca[q], wi[b], wv[b]) == reg_pick(cb[q], wi[b], wv[b])) == ceq[q]);
      u64 w = 0;
#pragma unroll
      for (int q = 0; q < NOUT; q++) w |= reg_pick(out_op[q], wi[b], wv[b]) << out_sh[q];
      if constexpr (kFilter == 3) {
        if (!ok) continue;
        const u64 r = r0 + rr[b];
        const C tag = P.in_packed ? Sem::from_stored(reinterpret_cast<const S*>(Q.in_tags)[r])
                                  : reinterpret_cast<const C*>(Q.in_tags)[r];
        dense_add<Sem>(P.acc, w, Sem::mul(tag, Sem::from_stored(reinterpret_cast<const S*>(Q.v_tags)[v])));
        touch_bit(P.bitmap, w);
      } else if constexpr (kFilter) {
        if (!ok) continue;
        const u32 bit = 1u << (u32)(w & 31u);
        u32* word = P.bitmap + (w >> 5);
        if constexpr (kFilter == 2) {  // bitmap only: set the bit, no old value needed
          atomicOr(word, bit);
          continue;
        }
        if (*reinterpret_cast<volatile u32*>(word) & bit) continue;
        if (atomicOr(word, bit) & bit) continue;
        if constexpr (kFilter == 1) kept[nkeep++] = w;
      } else {
        const u64 o = P.out_base + (j - P.j_begin);
        if (!ok) w = invalid_out;
        if (P.out_w64) reinterpret_cast<u64*>(P.out_words)[o] = w;
        else reinterpret_cast<u32*>(P.out_words)[o] = (u32)w;
        if constexpr (Sem::kTags) {
          const u64 r = r0 + rr[b];
          C tag = P.in_packed ? Sem::from_stored(reinterpret_cast<const S*>(Q.in_tags)[r])
                              : reinterpret_cast<const C*>(Q.in_tags)[r];
          reinterpret_cast<C*>(P.out_tags)[o] = Sem::mul(tag, Sem::from_stored(reinterpret_cast<const S*>(Q.v_tags)[v]));
        }
      }
    }
  }
  if constexpr (kFilter == 1) {
    u32 tot;
    const u32 mine = block_exclusive_sum<u32>(nkeep, sm, &tot);
    if (threadIdx.x == 0) block_base = tot ? atomicAdd(reinterpret_cast<unsigned long long*>(P.out_count), (u64)tot) : 0ull;
    __syncthreads();
    const u64 base = P.out_base + block_base;
    if (P.out_w64) {
      u64* stage = reinterpret_cast<u64*>(row_of);
      for (u32 c0 = 0; c0 < tot; c0 += kEmitTile / 2) {
        for (u32 q = 0; q < nkeep; q++) {
          const u32 pos = mine + q;
          if (pos >= c0 && pos < c0 + kEmitTile / 2) stage[pos - c0] = kept[q];
        }
        __syncthreads();
        const u32 lim = min(tot - c0, (u32)(kEmitTile / 2));
        for (u32 i = threadIdx.x; i < lim; i += 256) reinterpret_cast<u64*>(P.out_words)[base + c0 + i] = stage[i];
        __syncthreads();
      }
    } else {
      for (u32 q = 0; q < nkeep; q++) row_of[mine + q] = (u32)kept[q];
      __syncthreads();
      for (u32 i = threadIdx.x; i < tot; i += 256) reinterpret_cast<u32*>(P.out_words)[base + i] = row_of[i];
    }
  }
  __syncthreads();  // shared memory is reused by the block's next tile
  }
}

// Count: the matches of every input row in the probed view (lo32: first matched
// view row) and the row's output offset within its block of kLocRows rows
// (loc), plus one total per block (blk_cnt).  Each thread takes four
// consecutive rows, so the block's local offsets come from one block scan and
// no pass over per-row counts is needed afterwards.  NPRE > 0: dense index
// probed with NPRE prefix fields held in registers; NPRE == 0: any index.
template <int NPRE>
__global__ void __launch_bounds__(256) k_pcount_loc(const __grid_constant__ PStep P, u64 n_blk) {
  __shared__ u64 sm64[256 / 32 + 1];
  constexpr int NP = NPRE > 0 ? NPRE : 1;
  RegOp pre[NP];
  u32 psh[NP], plim[NP];
#pragma unroll
  for (int q = 0; q < NPRE; q++) {
    pre[q] = reg_op(P.prefix[q].op);
    psh[q] = P.prefix[q].shift;
    plim[q] = P.prefix[q].limit_bits;
  }
  const u64 invalid_in = P.in_w64 ? ~0ull : 0xFFFFFFFFull;
  const PPtrs Q = resolve_ptrs(P);
  const bool vec_in = (reinterpret_cast<uintptr_t>(Q.in_words) & 15) == 0;
  const u64 n_in = dev_size(P.n_in, P.n_in_dev);  // blocks past it get count 0
  for (u64 b = blockIdx.x; b < n_blk; b += gridDim.x) {
    if (b * kLocRows >= n_in) {
      if (threadIdx.x == 0) P.blk_cnt[b] = 0;
      continue;
    }
    const u64 r0 = b * kLocRows + (u64)threadIdx.x * 4;
    const bool full = r0 + 4 <= n_in;
    u64 w[4];
    if (full && vec_in) {
      if (P.in_w64) {
        const ulonglong2 x = reinterpret_cast<const ulonglong2*>(Q.in_words)[r0 / 2];
        const ulonglong2 y = reinterpret_cast<const ulonglong2*>(Q.in_words)[r0 / 2 + 1];
        w[0] = x.x; w[1] = x.y; w[2] = y.x; w[3] = y.y;
      } else {
        const uint4 x = reinterpret_cast<const uint4*>(Q.in_words)[r0 / 4];
        w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++) w[i] = r0 + i < n_in ? load_word(Q.in_words, P.in_w64, r0 + i) : invalid_in;
    }
    u32 c[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      c[i] = 0;
      lo[i] = 0;
      bool ok = w[i] != invalid_in;
      if (ok && P.in_stamp_mode != STAMP_NONE) {
        const u32 st = P.in_stamp[r0 + i] & 0x7FFFFFFFu;
        ok = P.in_stamp_mode == STAMP_LT ? st < P.in_stamp_val : st == P.in_stamp_val;
      }
      if (ok && P.n_in_checks) ok = checks_ok(P.in_checks, P.n_in_checks, w[i], 0);
      u64 pv = 0;
      if constexpr (NPRE > 0) {
#pragma unroll
        for (int q = 0; q < NPRE; q++) {
          const u64 x = reg_pick(pre[q], w[i], 0);
          ok = ok && !(plim[q] < 64 && (x >> plim[q]));
          pv |= x << psh[q];
        }
        if (ok) {
          const u64 l = P.dense_offs[pv];
          c[i] = (u32)(P.dense_offs[pv + 1] - l);
          lo[i] = (u32)l;
        }
      } else {
        for (int q = 0; q < P.n_prefix; q++) {
          const u64 x = pick(P.prefix[q].op, w[i], 0);
          ok = ok && !(P.prefix[q].limit_bits < 64 && (x >> P.prefix[q].limit_bits));
          pv |= x << P.prefix[q].shift;
        }
        if (ok) {
          u64 l, h;
          if (P.index_mode == INDEX_DENSE) {
            l = P.dense_offs[pv];
            h = P.dense_offs[pv + 1];
          } else if (P.index_mode == INDEX_HASH) {
            hash_find(reinterpret_cast<const HashSlot*>(P.dense_offs), P.hash_bits, pv, l, h);
          } else {
            const u64 vn = dev_size(P.v_n, P.v_n_dev);
            if (P.whole_view) {
              l = 0;
              h = vn;
            } else {
              const u64 klo = pv << P.rest_shift;
              const u64 khi = klo + (1ull << P.rest_shift);
              l = lower_bound_w(Q.v_keys, P.v_key64, vn, klo);
              h = khi < klo ? vn : lower_bound_w(Q.v_keys, P.v_key64, vn, khi);
            }
          }
          c[i] = (u32)(h - l);
          lo[i] = (u32)l;
        }
      }
    }
    u64 tot;
    const u64 ex = block_exclusive_sum<u64>((u64)c[0] + c[1] + c[2] + c[3], sm64, &tot);
    u32 lc[4];
    u32 run = (u32)ex;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      lc[i] = run;
      run += c[i];
    }
    if (full) {
      reinterpret_cast<uint4*>(P.loc)[r0 / 4] = make_uint4(lc[0], lc[1], lc[2], lc[3]);
      reinterpret_cast<uint4*>(P.lo32)[r0 / 4] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (r0 + i < n_in) {
          P.loc[r0 + i] = lc[i];
          P.lo32[r0 + i] = lo[i];
        }
    }
    if (threadIdx.x == 0) {
      P.blk_cnt[b] = tot;
      if (tot >> 32) atomicOr(P.err, kErrLocOverflow);
    }
  }
}

// partition of outputs [j_begin, j_begin + total) into tiles of kEmitTile:
// part[t] = the last row whose first output is at or before the tile's start
__global__ void k_ppartition(const __grid_constant__ PStep P, u64 n_blk, u64 ntiles, u64* __restrict__ part) {
  const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 total = dev_size(P.total, P.total_dev);
  const u64 n_in = dev_size(P.n_in, P.n_in_dev);
  if (P.total_dev) {  // device-resident total: the tiles it needs, out of the launch's
    if (!total) return;
    ntiles = (total + kEmitTile - 1) / kEmitTile;
  }
  if (t > ntiles) return;
  const u64 j = t == ntiles ? P.j_begin + total - 1 : P.j_begin + t * (u64)kEmitTile;
  const u64 b = upper_bound_dev<u64>(P.blk_off, 0, n_blk, j) - 1;
  const u64 lo = b * kLocRows;
  const u64 hi = lo + kLocRows < n_in ? lo + kLocRows : n_in;
  part[t] = upper_bound_dev<u32>(P.loc, lo, hi, (u32)(j - P.blk_off[b])) - 1;
}

// ---------------------------------------------------------------------------
// Warp-balanced expansion (unit semiring, where the order of a step's outputs
// does not matter).  A warp takes 32 consecutive input rows, one per lane,
// probes them, and scans the lanes' match counts; it then produces the rows'
// outputs in rounds of 32, lane l taking output t = round * 32 + l, whose row
// is found by a binary search over the lanes' scanned counts with shuffles.
// No per-row arrays, no partition and no block barriers.  kMode 0: binding
// words stored at positions claimed per warp with one atomicAdd (the step's
// total is counted first, for the allocation); kMode 2: last step, every
// output only sets its membership bit (a non-returning atomic OR).
// ---------------------------------------------------------------------------
LOB_DEV u32 probe_row(const PStep& P, u64 r, u64& wi, u32& lo) {
  lo = 0;
  wi = 0;
  if (r >= P.n_in) return 0;
  wi = load_word(P.in_words, P.in_w64, r);
  if (wi == (P.in_w64 ? ~0ull : 0xFFFFFFFFull)) return 0;
  if (P.in_stamp_mode != STAMP_NONE) {
    const u32 st = P.in_stamp[r] & 0x7FFFFFFFu;
    if (P.in_stamp_mode == STAMP_LT ? !(st < P.in_stamp_val) : st != P.in_stamp_val) return 0;
  }
  if (P.n_in_checks && !checks_ok(P.in_checks, P.n_in_checks, wi, 0)) return 0;
  u64 pv = 0;
  for (int q = 0; q < P.n_prefix; q++) {
    const u64 x = pick(P.prefix[q].op, wi, 0);
    if (P.prefix[q].limit_bits < 64 && (x >> P.prefix[q].limit_bits)) return 0;
    pv |= x << P.prefix[q].shift;
  }
  u64 l, h;
  if (P.index_mode == INDEX_DENSE) {
    l = P.dense_offs[pv];
    h = P.dense_offs[pv + 1];
  } else if (P.index_mode == INDEX_HASH) {
    hash_find(reinterpret_cast<const HashSlot*>(P.dense_offs), P.hash_bits, pv, l, h);
  } else if (P.whole_view) {
    l = 0;
    h = P.v_n;
  } else {
    const u64 klo = pv << P.rest_shift;
    const u64 khi = klo + (1ull << P.rest_shift);
    l = lower_bound_w(P.v_keys, P.v_key64, P.v_n, klo);
    h = khi < klo ? P.v_n : lower_bound_w(P.v_keys, P.v_key64, P.v_n, khi);
  }
  lo = (u32)l;
  return (u32)(h - l);
}

// Row blocks of the warp steps: 1024 rows, taken by a CTA as four rounds of
// 256 (warp w of round i owns rows i*256 + w*32 .. +31, one per lane).
constexpr u64 kWarpBlockRows = 1024;

// outputs per row block (placement of an intermediate step's binding words)
__global__ void __launch_bounds__(256) k_pwarp_count(const __grid_constant__ PStep P, u64* __restrict__ blk_cnt,
                                                     u64 n_blk) {
  __shared__ u64 part[256 / 32];
  for (u64 b = blockIdx.x; b < n_blk; b += gridDim.x) {
    u64 c = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      u64 wi;
      u32 lo;
      c += probe_row(P, b * kWarpBlockRows + (u64)i * 256 + threadIdx.x, wi, lo);
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      u64 t = 0;
      for (int w = 0; w < 256 / 32; w++) t += part[w];
      blk_cnt[b] = t;
    }
    __syncthreads();
  }
}

// the outputs of one 32-row group: lane l takes outputs l, l + 32, ...
template <int kMode, int NOUT, int NCHK>
LOB_DEV void warp_expand(const PStep& P, const RegOp* out_op, const u32* out_sh, const RegOp* ca, const RegOp* cb,
                         const bool* ceq, u64 wi, u32 lo, u32 ex, u32 tot, u64 base) {
  const int lane = threadIdx.x & 31;
  for (u32 t0 = 0; t0 < tot; t0 += 32) {
    const u32 t = t0 + lane;
    int src = 0;  // the last lane whose outputs start at or before t
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const u32 e = __shfl_sync(0xFFFFFFFFu, ex, src + step);
      if (e <= t) src += step;
    }
    const u64 wr = __shfl_sync(0xFFFFFFFFu, wi, src);
    const u32 lr = __shfl_sync(0xFFFFFFFFu, lo, src);
    const u32 er = __shfl_sync(0xFFFFFFFFu, ex, src);
    if (t >= tot) continue;
    const u64 v = (u64)lr + (t - er);
    const u64 wv = load_word(P.v_keys, P.v_key64, v);
    bool ok = true;
    if (P.v_stamp_mode != STAMP_NONE) {
      const u32 st = P.v_stamp[v] & 0x7FFFFFFFu;
      ok = P.v_stamp_mode == STAMP_LT ? st < P.v_stamp_val : st == P.v_stamp_val;
    }
#pragma unroll
    for (int q = 0; q < NCHK; q++) ok = ok && ((reg_pick(ca[q], wr, wv) == reg_pick(cb[q], wr, wv)) == ceq[q]);
    u64 w = 0;
#pragma unroll
    for (int q = 0; q < NOUT; q++) w |= reg_pick(out_op[q], wr, wv) << out_sh[q];
    if constexpr (kMode == 2) {
      if (ok) atomicOr(P.bitmap + (w >> 5), 1u << (u32)(w & 31u));
    } else {
      if (!ok) w = P.out_w64 ? ~0ull : 0xFFFFFFFFull;
      const u64 o = base + t;
      if (P.out_w64) reinterpret_cast<u64*>(P.out_words)[o] = w;
      else reinterpret_cast<u32*>(P.out_words)[o] = (u32)w;
    }
  }
}

// kMode 0: binding words, row block b's outputs from blk_off[b] on, its groups
// in (round, warp) order.  kMode 2: bitmap bits only; *emitted counts outputs.
template <int kMode, int NOUT, int NCHK>
__global__ void __launch_bounds__(256) k_pwarp_emit(const __grid_constant__ PStep P, const u64* __restrict__ blk_off,
                                                    u64 n_blk, unsigned long long* emitted) {
  RegOp out_op[NOUT];
  u32 out_sh[NOUT];
#pragma unroll
  for (int q = 0; q < NOUT; q++) {
    out_op[q] = reg_op(P.out[q].op);
    out_sh[q] = P.out[q].shift;
  }
  RegOp ca[NCHK > 0 ? NCHK : 1], cb[NCHK > 0 ? NCHK : 1];
  bool ceq[NCHK > 0 ? NCHK : 1];
#pragma unroll
  for (int q = 0; q < NCHK; q++) {
    ca[q] = reg_op(P.checks[q].a);
    cb[q] = reg_op(P.checks[q].b);
    ceq[q] = P.checks[q].eq != 0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (kMode == 2) {
    const u64 nwarps = (u64)gridDim.x * (blockDim.x / 32);
    u64 mine = 0;
    for (u64 g = (u64)blockIdx.x * (blockDim.x / 32) + warp; g * 32 < P.n_in; g += nwarps) {
      u64 wi;
      u32 lo;
      const u32 c = probe_row(P, g * 32 + lane, wi, lo);
      const u32 inc = warp_inclusive_sum(c);
      const u32 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
      if (!tot) continue;
      mine += tot;
      warp_expand<2, NOUT, NCHK>(P, out_op, out_sh, ca, cb, ceq, wi, lo, inc - c, tot, 0);
    }
    if (lane == 0 && mine) atomicAdd(emitted, (unsigned long long)mine);
  } else {
    __shared__ u32 gsum[32];
    for (u64 b = blockIdx.x; b < n_blk; b += gridDim.x) {
      u64 wi[4];
      u32 lo[4], ex[4], tot[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const u32 c = probe_row(P, b * kWarpBlockRows + (u64)i * 256 + warp * 32 + lane, wi[i], lo[i]);
        const u32 inc = warp_inclusive_sum(c);
        ex[i] = inc - c;
        tot[i] = __shfl_sync(0xFFFFFFFFu, inc, 31);
        if (lane == 0) gsum[i * 8 + warp] = tot[i];
      }
      __syncthreads();
      if (warp == 0) {  // exclusive scan of the 32 group totals, in (round, warp) order
        const u32 v = gsum[lane];
        const u32 inc = warp_inclusive_sum(v);
        __syncwarp();
        gsum[lane] = inc - v;
      }
      __syncthreads();
      const u64 bbase = blk_off[b];
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (tot[i]) warp_expand<0, NOUT, NCHK>(P, out_op, out_sh, ca, cb, ceq, wi[i], lo[i], ex[i], tot[i], bbase + gsum[i * 8 + warp]);
      __syncthreads();  // gsum is rewritten by the next block
    }
  }
}

// Backward emission (see pjoin.h): one tile of kEmitTile outputs per block,
// located like the forward emission's.
template <int NOUT, int NCHK>
__global__ void __launch_bounds__(256) k_pbwd_emit(const __grid_constant__ PStep P, const __grid_constant__ PBwd B,
                                                   const u64* __restrict__ part) {
  constexpr int kItems = kEmitTile / 256;
  __shared__ __align__(16) u32 row_of[kEmitTile];
  __shared__ u32 sm[256 / 32 + 1];
  __shared__ u32 th_inc[256];
  const u64 j0 = P.j_begin + (u64)blockIdx.x * kEmitTile;
  const u64 j_end = P.j_begin + P.total;
  if (j0 >= j_end) return;
  const u64 r0 = part[blockIdx.x];
  const u64 r_end = part[blockIdx.x + 1];
  for (int i = threadIdx.x; i < kEmitTile; i += 256) row_of[i] = 0;
  __syncthreads();
  for (u64 r = r0 + 1 + threadIdx.x; r <= r_end; r += 256) {
    const u64 o = row_off(P, r);
    if (o < j0 + kEmitTile) atomicMax(&row_of[o - j0], (u32)(r - r0));
  }
  __syncthreads();
  {
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
  }
  __syncthreads();
  RegOp out_op[NOUT];
  u32 out_sh[NOUT];
#pragma unroll
  for (int q = 0; q < NOUT; q++) {
    out_op[q] = reg_op(P.out[q].op);
    out_sh[q] = P.out[q].shift;
  }
  RegOp ca[NCHK > 0 ? NCHK : 1], cb[NCHK > 0 ? NCHK : 1];
  bool ceq[NCHK > 0 ? NCHK : 1];
#pragma unroll
  for (int q = 0; q < NCHK; q++) {
    ca[q] = reg_op(P.checks[q].a);
    cb[q] = reg_op(P.checks[q].b);
    ceq[q] = P.checks[q].eq != 0;
  }
  const u64 invalid_in = P.in_w64 ? ~0ull : 0xFFFFFFFFull;
  const u64 invalid_out = P.out_w64 ? ~0ull : 0xFFFFFFFFull;
  const int nf_in = B.packed_source ? 1 : B.n_in_facts;
#pragma unroll 1
  for (int i = 0; i < kItems; i++) {
    const u64 j = j0 + (u64)i * 256 + threadIdx.x;
    if (j >= j_end) break;
    const u64 r = r0 + row_of[j - j0];
    const u64 v = (u64)P.lo32[r] + (j - row_off(P, r));
    const u64 wi = load_word(P.in_words, P.in_w64, r);
    const u64 wv = load_word(P.v_keys, P.v_key64, v);
    bool ok = wi != invalid_in;
    if (P.n_in_checks) ok = ok && checks_ok(P.in_checks, P.n_in_checks, wi, 0);
    if (P.v_stamp_mode != STAMP_NONE) {
      const u32 st = P.v_stamp[v] & 0x7FFFFFFFu;
      ok = ok && (P.v_stamp_mode == STAMP_LT ? st < P.v_stamp_val : st == P.v_stamp_val);
    }
#pragma unroll
    for (int q = 0; q < NCHK; q++) ok = ok && ((reg_pick(ca[q], wi, wv) == reg_pick(cb[q], wi, wv)) == ceq[q]);
    u64 w = 0;
#pragma unroll
    for (int q = 0; q < NOUT; q++) w |= reg_pick(out_op[q], wi, wv) << out_sh[q];
    const u32 vrow = B.v_prow ? B.v_prow[v] : (u32)v;
    if (!B.last) {  // the binding word (dropped: all ones) and the rows of the facts so far
      const u64 o = j - P.j_begin;
      if (P.out_w64) reinterpret_cast<u64*>(P.out_words)[o] = ok ? w : invalid_out;
      else reinterpret_cast<u32*>(P.out_words)[o] = (u32)(ok ? w : invalid_out);
      for (int q = 0; q < nf_in; q++) B.out_rows[q][o] = B.packed_source ? (u32)r : B.in_rows[q][r];
      B.out_rows[nf_in][o] = vrow;
      continue;
    }
    if (!ok) continue;
    if (!((B.h_new[w >> 5] >> (w & 31)) & 1u)) continue;  // the head was not new (or was clamped) in this iteration
    u64 hj;
    if (B.h_row) {
      hj = B.h_row[w];
    } else {
      u64 lo = 0, hi = B.h_n;
      if (B.h_key64) {
        const u64* a = reinterpret_cast<const u64*>(B.h_keys);
        while (lo < hi) { const u64 m = (lo + hi) >> 1; if (a[m] < w) lo = m + 1; else hi = m; }
      } else {
        const u32* a = reinterpret_cast<const u32*>(B.h_keys);
        while (lo < hi) { const u64 m = (lo + hi) >> 1; if (a[m] < (u32)w) lo = m + 1; else hi = m; }
      }
      hj = lo;
    }
    const double adj = B.h_adj[hj];
    if (adj == 0.0) continue;
    u32 rows[kMaxArity + 1];
    float tags[kMaxArity + 1];
    for (int q = 0; q < nf_in; q++) rows[q] = B.packed_source ? (u32)r : B.in_rows[q][r];
    rows[nf_in] = vrow;
    const int nf = nf_in + 1;
    for (int q = 0; q < nf; q++) tags[q] = B.fact_tags[q][rows[q]];
    for (int q = 0; q < nf; q++) {
      if (!B.fact_adj[q]) continue;
      double c = adj;
      for (int l = 0; l < nf; l++)
        if (l != q) c *= (double)tags[l];
      atomicAdd(B.fact_adj[q] + rows[q], c);
    }
  }
}

// ---------------------------------------------------------------------------
// Fused cross-product step (unit semiring, bitmap-only last step).  When both
// probes of a two-probe arm are keyed by the delta row alone -- same
// generation's sg(x,y) :- parent(a,x), sg(a,b), parent(b,y), where children(a)
// and children(b) depend only on (a, b) -- a warp probes both views for 32
// delta rows, scans the lanes' product counts |A| * |B|, and expands the
// products in rounds of 32 (lane l takes output t; its row is found by a
// binary search over the scanned counts, its pair (i, j) by one division),
// setting each output's membership bit.  No binding words, no count pass.
// Operands: word 0 the delta row, 1 the key matched in view A, 3 the key
// matched in view B, 2 a constant.
// ---------------------------------------------------------------------------
LOB_DEV u64 reg_pick3(const RegOp& o, u64 wi, u64 wa, u64 wb) {
  if (o.word == 2) return (u64)o.cval;
  const u64 w = o.word == 0 ? wi : (o.word == 1 ? wa : wb);
  return (w >> o.shift) & o.mask;
}

// match range of view B for input word wi (B's prefix operands read wi only)
LOB_DEV u32 probe_b(const PStep& B, u64 wi, u32& lo) {
  u64 pv = 0;
  lo = 0;
  for (int q = 0; q < B.n_prefix; q++) {
    const u64 x = pick(B.prefix[q].op, wi, 0);
    if (B.prefix[q].limit_bits < 64 && (x >> B.prefix[q].limit_bits)) return 0;
    pv |= x << B.prefix[q].shift;
  }
  u64 l, h;
  if (B.index_mode == INDEX_DENSE) {
    l = B.dense_offs[pv];
    h = B.dense_offs[pv + 1];
  } else if (B.index_mode == INDEX_HASH) {
    hash_find(reinterpret_cast<const HashSlot*>(B.dense_offs), B.hash_bits, pv, l, h);
  } else if (B.whole_view) {
    l = 0;
    h = B.v_n;
  } else {
    const u64 klo = pv << B.rest_shift;
    const u64 khi = klo + (1ull << B.rest_shift);
    l = lower_bound_w(B.v_keys, B.v_key64, B.v_n, klo);
    h = khi < klo ? B.v_n : lower_bound_w(B.v_keys, B.v_key64, B.v_n, khi);
  }
  lo = (u32)l;
  return (u32)(h - l);
}

template <int NOUT, int NCHKA, int NCHKB>
__global__ void __launch_bounds__(256) k_pwarp_cross(const __grid_constant__ PStep A, const __grid_constant__ PStep B,
                                                     unsigned long long* emitted) {
  RegOp out_op[NOUT];
  u32 out_sh[NOUT];
#pragma unroll
  for (int q = 0; q < NOUT; q++) {
    out_op[q] = reg_op(B.out[q].op);
    out_sh[q] = B.out[q].shift;
  }
  RegOp aa[NCHKA > 0 ? NCHKA : 1], ab[NCHKA > 0 ? NCHKA : 1], ba[NCHKB > 0 ? NCHKB : 1], bb[NCHKB > 0 ? NCHKB : 1];
  bool aeq[NCHKA > 0 ? NCHKA : 1], beq[NCHKB > 0 ? NCHKB : 1];
#pragma unroll
  for (int q = 0; q < NCHKA; q++) {
    aa[q] = reg_op(A.checks[q].a);
    ab[q] = reg_op(A.checks[q].b);
    aeq[q] = A.checks[q].eq != 0;
  }
#pragma unroll
  for (int q = 0; q < NCHKB; q++) {
    ba[q] = reg_op(B.checks[q].a);
    bb[q] = reg_op(B.checks[q].b);
    beq[q] = B.checks[q].eq != 0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u64 nwarps = (u64)gridDim.x * (blockDim.x / 32);
  u64 mine = 0;
  for (u64 g = (u64)blockIdx.x * (blockDim.x / 32) + warp; g * 32 < A.n_in; g += nwarps) {
    u64 wi;
    u32 loa, lob = 0, cb = 0;
    const u32 ca = probe_row(A, g * 32 + lane, wi, loa);
    if (ca) cb = probe_b(B, wi, lob);
    const u64 c = (u64)ca * cb;
    const u64 inc = warp_inclusive_sum(c);
    const u64 ex = inc - c;
    const u64 tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    if (!tot) continue;
    mine += tot;
    if (tot <= 0xFFFFFFFFull) {
      // the warp's products fit 32 bits: 32-bit scan values, and the division
      // u / |B| by a per-row reciprocal m = ceil(2^32 / |B|): umulhi(u, m) is
      // floor(u / |B|) or one more, fixed by one multiply-compare
      const u32 ex32 = (u32)ex, tot32 = (u32)tot;
      const u32 rcp = cb > 1 ? 0xFFFFFFFFu / cb + 1u : 0u;
      for (u32 t0 = 0; t0 < tot32; t0 += 32) {
        const u32 t = t0 + (u32)lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const u32 e = __shfl_sync(0xFFFFFFFFu, ex32, src + step);
          if (e <= t) src += step;
        }
        const u64 wr = __shfl_sync(0xFFFFFFFFu, wi, src);
        const u32 la = __shfl_sync(0xFFFFFFFFu, loa, src);
        const u32 lb = __shfl_sync(0xFFFFFFFFu, lob, src);
        const u32 nb = __shfl_sync(0xFFFFFFFFu, cb, src);
        const u32 er = __shfl_sync(0xFFFFFFFFu, ex32, src);
        const u32 m = __shfl_sync(0xFFFFFFFFu, rcp, src);
        if (t >= tot32) continue;
        const u32 u = t - er;
        u32 i = nb == 1 ? u : __umulhi(u, m);
        if ((u64)i * nb > u) i--;
        const u32 j = u - i * nb;
        const u64 wa = load_word(A.v_keys, A.v_key64, (u64)la + i);
        const u64 wb = load_word(B.v_keys, B.v_key64, (u64)lb + j);
        bool ok = true;
#pragma unroll
        for (int q = 0; q < NCHKA; q++) ok = ok && ((reg_pick3(aa[q], wr, wa, 0) == reg_pick3(ab[q], wr, wa, 0)) == aeq[q]);
#pragma unroll
        for (int q = 0; q < NCHKB; q++) ok = ok && ((reg_pick3(ba[q], wr, wa, wb) == reg_pick3(bb[q], wr, wa, wb)) == beq[q]);
        u64 w = 0;
#pragma unroll
        for (int q = 0; q < NOUT; q++) w |= reg_pick3(out_op[q], wr, wa, wb) << out_sh[q];
        if (ok) atomicOr(B.bitmap + (w >> 5), 1u << (u32)(w & 31u));
      }
      continue;
    }
    for (u64 t0 = 0; t0 < tot; t0 += 32) {
      const u64 t = t0 + lane;
      int src = 0;
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const u64 e = __shfl_sync(0xFFFFFFFFu, ex, src + step);
        if (e <= t) src += step;
      }
      const u64 wr = __shfl_sync(0xFFFFFFFFu, wi, src);
      const u32 la = __shfl_sync(0xFFFFFFFFu, loa, src);
      const u32 lb = __shfl_sync(0xFFFFFFFFu, lob, src);
      const u32 nb = __shfl_sync(0xFFFFFFFFu, cb, src);
      const u64 er = __shfl_sync(0xFFFFFFFFu, ex, src);
      if (t >= tot) continue;
      const u32 u = (u32)(t - er);
      const u32 i = u / nb, j = u - i * nb;
      const u64 wa = load_word(A.v_keys, A.v_key64, (u64)la + i);
      const u64 wb = load_word(B.v_keys, B.v_key64, (u64)lb + j);
      bool ok = true;
#pragma unroll
      for (int q = 0; q < NCHKA; q++) ok = ok && ((reg_pick3(aa[q], wr, wa, 0) == reg_pick3(ab[q], wr, wa, 0)) == aeq[q]);
#pragma unroll
      for (int q = 0; q < NCHKB; q++) ok = ok && ((reg_pick3(ba[q], wr, wa, wb) == reg_pick3(bb[q], wr, wa, wb)) == beq[q]);
      u64 w = 0;
#pragma unroll
      for (int q = 0; q < NOUT; q++) w |= reg_pick3(out_op[q], wr, wa, wb) << out_sh[q];
      if (ok) atomicOr(B.bitmap + (w >> 5), 1u << (u32)(w & 31u));
    }
  }
  if (lane == 0 && mine) atomicAdd(emitted, (unsigned long long)mine);
}

unsigned grid_n(u64 n) {
  u64 b = (n + 255) / 256;
  if (b > 152ull * 16) b = 152ull * 16;
  return (unsigned)(b ? b : 1);
}

double row_bytes(int sem, int w64, bool packed_in) {
  const double t = sem == SR_UNIT ? 0 : (packed_in ? (sem == SR_DIFF_MAX_MIN ? 8 : 4) : (sem == SR_MAX_MIN ? 4 : 8));
  return (w64 ? 8 : 4) + t;
}

template <template <class> class L, class... A>
void by_sem_p(int sem, A&&... a) {
  switch (sem) {
    case SR_UNIT: L<SemUnit>::go(a...); break;
    case SR_MAX_MIN: L<SemMaxMin>::go(a...); break;
    case SR_DIFF_MAX_MIN: L<SemDiffMaxMin>::go(a...); break;
    default: L<SemAddMult>::go(a...); break;
  }
}
template <class Sem, int F, int NO, int NC>
void launch_fast(const PStep& P, const u64* part, unsigned tiles, cudaStream_t st) {
  k_pemit_fast<Sem, F, NO, NC><<<tiles, 256, 0, st>>>(P, part);
}
template <class Sem, int F>
bool try_fast(const PStep& P, const u64* part, unsigned tiles, cudaStream_t st) {
  const int no = P.n_out, nc = P.n_checks;
#define LOB_FAST(NO, NC) if (no == NO && nc == NC) { launch_fast<Sem, F, NO, NC>(P, part, tiles, st); return true; }
  LOB_FAST(1, 0) LOB_FAST(2, 0) LOB_FAST(3, 0) LOB_FAST(4, 0)
  LOB_FAST(1, 1) LOB_FAST(2, 1) LOB_FAST(3, 1) LOB_FAST(4, 1)
#undef LOB_FAST
  return false;
}
template <class Sem> struct PEmitL {
  static void go(const PStep& P, const u64* part, cudaStream_t st) {
    // one block per tile; with a device-resident total, a fixed grid of
    // blocks walks the tiles the total needs (P.total is then a capacity)
    const u64 ntile = (P.total + kEmitTile - 1) / kEmitTile;
    const u64 tiles = P.total_dev ? std::min<u64>(ntile, 152ull * 8) : ntile;
    // membership filter: 1 = new facts also written out, 2 = bitmap only;
    // 3 = dense (+)-accumulation of tagged outputs
    if (!std::is_same<Sem, SemUnit>::value && P.acc) {
      if (!try_fast<Sem, 3>(P, part, (unsigned)tiles, st)) k_pemit<Sem, 3><<<(unsigned)tiles, 256, 0, st>>>(P, part);
    } else if (std::is_same<Sem, SemUnit>::value && P.bitmap && P.out_words) {
      if (!try_fast<SemUnit, 1>(P, part, (unsigned)tiles, st))
        k_pemit<SemUnit, 1><<<(unsigned)tiles, 256, 0, st>>>(P, part);
    } else if (std::is_same<Sem, SemUnit>::value && P.bitmap) {
      if (!try_fast<SemUnit, 2>(P, part, (unsigned)tiles, st))
        k_pemit<SemUnit, 2><<<(unsigned)tiles, 256, 0, st>>>(P, part);
    } else if (!try_fast<Sem, 0>(P, part, (unsigned)tiles, st)) {
      k_pemit<Sem, 0><<<(unsigned)tiles, 256, 0, st>>>(P, part);
    }
  }
};
template <int M>
bool try_warp(const PStep& P, unsigned grid, const u64* blk_off, u64 n_blk, unsigned long long* emitted, cudaStream_t st) {
  const int no = P.n_out, nc = P.n_checks;
#define LOB_WARP(NO, NC) if (no == NO && nc == NC) { k_pwarp_emit<M, NO, NC><<<grid, 256, 0, st>>>(P, blk_off, n_blk, emitted); return true; }
  LOB_WARP(1, 0) LOB_WARP(2, 0) LOB_WARP(3, 0) LOB_WARP(4, 0)
  LOB_WARP(1, 1) LOB_WARP(2, 1) LOB_WARP(3, 1) LOB_WARP(4, 1)
#undef LOB_WARP
  return false;
}
template <class Sem> struct PProjL {
  static void go(const PStep& P, cudaStream_t st) { k_pproject<Sem><<<grid_n(P.n_in), 256, 0, st>>>(P); }
};

}  // namespace

void pjoin_count(int sem, const PStep& P, cudaStream_t st) {
  const u64 n_blk = pjoin_loc_blocks(P.n_in);
  // input rows read, per-row offsets and match starts written (the index is
  // read per distinct probe key, mostly from L2)
  ProfScope ps("join_count", P.n_in * (row_bytes(sem, P.in_w64, P.in_packed) + 8.0) + n_blk * 8.0, st);
  if (!P.n_in) return;
  const unsigned g = (unsigned)(n_blk < 152ull * 64 ? n_blk : 152ull * 64);
  if (P.index_mode == INDEX_DENSE && P.n_prefix == 1) k_pcount_loc<1><<<g, 256, 0, st>>>(P, n_blk);
  else if (P.index_mode == INDEX_DENSE && P.n_prefix == 2) k_pcount_loc<2><<<g, 256, 0, st>>>(P, n_blk);
  else if (P.index_mode == INDEX_DENSE && P.n_prefix == 3) k_pcount_loc<3><<<g, 256, 0, st>>>(P, n_blk);
  else k_pcount_loc<0><<<g, 256, 0, st>>>(P, n_blk);
}

void pjoin_partition(const PStep& P, u64 ntiles, u64* part, cudaStream_t st) {
  ProfScope ps("join_partition", (ntiles + 1) * 8.0, st);
  k_ppartition<<<(unsigned)((ntiles + 1 + 255) / 256), 256, 0, st>>>(P, pjoin_loc_blocks(P.n_in), ntiles, part);
}

void pjoin_emit(int sem, const PStep& P, const u64* part, cudaStream_t st) {
  // read the input rows and their offsets once and each matched view key once;
  // write each output (a membership-bitmap word per output in bitmap-only mode)
  const double vb = (P.v_key64 ? 8 : 4) + (sem == SR_UNIT ? 0 : (sem == SR_DIFF_MAX_MIN ? 8 : 4));
  // an output is written as a word (+ tag), or as a bitmap word, or as a
  // (+)-accumulation into its dense slot plus its bitmap word
  const double ob = P.acc ? (sem == SR_MAX_MIN ? 4.0 : 8.0) + 4.0 : (P.out_words ? row_bytes(sem, P.out_w64, false) : 4.0);
  ProfScope ps("join_emit", P.n_in * (row_bytes(sem, P.in_w64, P.in_packed) + 8.0) + P.total * (vb + ob), st);
  if (P.total) by_sem_p<PEmitL>(sem, P, part, st);
}

void pjoin_backward_emit(const PStep& P, const PBwd& B, const u64* part, cudaStream_t st) {
  if (!P.total) return;
  const u64 tiles = (P.total + kEmitTile - 1) / kEmitTile;
  const int nf = (B.packed_source ? 1 : B.n_in_facts) + 1;
  const double vb = (P.v_key64 ? 8 : 4) + 4.0;
  // per output: the matched key and stamp; an intermediate step writes its word
  // and carried rows, the last step probes the new-head bitmap
  ProfScope ps("bwd_emit", P.n_in * ((P.in_w64 ? 8.0 : 4.0) + 8.0) +
                               P.total * (vb + (B.last ? 4.0 : (P.out_w64 ? 8.0 : 4.0) + 4.0 * nf)), st);
  const int no = P.n_out, nc = P.n_checks;
#define LOB_BWD(NO, NC) if (no == NO && nc == NC) { k_pbwd_emit<NO, NC><<<(unsigned)tiles, 256, 0, st>>>(P, B, part); return; }
  LOB_BWD(1, 0) LOB_BWD(2, 0) LOB_BWD(3, 0) LOB_BWD(4, 0) LOB_BWD(5, 0)
  LOB_BWD(1, 1) LOB_BWD(2, 1) LOB_BWD(3, 1) LOB_BWD(4, 1) LOB_BWD(5, 1)
  LOB_BWD(1, 2) LOB_BWD(2, 2) LOB_BWD(3, 2) LOB_BWD(4, 2) LOB_BWD(5, 2)
#undef LOB_BWD
}

bool pjoin_backward_supported(const PStep& P) { return P.n_out >= 1 && P.n_out <= 5 && P.n_checks <= 2; }

void pjoin_project(int sem, const PStep& P, cudaStream_t st) {
  ProfScope ps("project", P.n_in * (row_bytes(sem, P.in_w64, P.in_packed) + row_bytes(sem, P.out_w64, false)), st);
  if (P.n_in) by_sem_p<PProjL>(sem, P, st);
}

bool pjoin_cross_supported(const PStep& A, const PStep& B) {
  return A.n_checks <= 1 && B.n_checks <= 1 && B.n_out >= 1 && B.n_out <= 4;
}

void pjoin_warp_cross_bitmap(const PStep& A, const PStep& B, u64* emitted_dev, cudaStream_t st) {
  // the outputs' bytes (two matched keys and a bitmap word each) are added by
  // the caller once their number is known
  ProfScope ps("join_emit", A.n_in * (A.in_w64 ? 8.0 : 4.0), st);
  if (!A.n_in) return;
  auto* em = reinterpret_cast<unsigned long long*>(emitted_dev);
  const unsigned g = grid_n(A.n_in);
  const int no = B.n_out, ca = A.n_checks, cb = B.n_checks;
#define LOB_CROSS(NO, CA, CB) \
  if (no == NO && ca == CA && cb == CB) { k_pwarp_cross<NO, CA, CB><<<g, 256, 0, st>>>(A, B, em); return; }
  LOB_CROSS(1, 0, 0) LOB_CROSS(2, 0, 0) LOB_CROSS(3, 0, 0) LOB_CROSS(4, 0, 0)
  LOB_CROSS(1, 1, 0) LOB_CROSS(2, 1, 0) LOB_CROSS(3, 1, 0) LOB_CROSS(4, 1, 0)
  LOB_CROSS(1, 0, 1) LOB_CROSS(2, 0, 1) LOB_CROSS(3, 0, 1) LOB_CROSS(4, 0, 1)
  LOB_CROSS(1, 1, 1) LOB_CROSS(2, 1, 1) LOB_CROSS(3, 1, 1) LOB_CROSS(4, 1, 1)
#undef LOB_CROSS
}

bool pjoin_warp_supported(int sem, const PStep& P) {
  return sem == SR_UNIT && P.n_out >= 1 && P.n_out <= 4 && P.n_checks <= 1;
}

u64 pjoin_warp_blocks(u64 n_in) { return (n_in + kWarpBlockRows - 1) / kWarpBlockRows; }

void pjoin_warp_count(const PStep& P, u64* blk_cnt, cudaStream_t st) {
  const u64 n_blk = pjoin_warp_blocks(P.n_in);
  ProfScope ps("join_count", P.n_in * (P.in_w64 ? 8.0 : 4.0) + n_blk * 8.0, st);
  if (n_blk) k_pwarp_count<<<(unsigned)(n_blk < 152ull * 16 ? n_blk : 152ull * 16), 256, 0, st>>>(P, blk_cnt, n_blk);
}

void pjoin_warp_emit(const PStep& P, u64 total, const u64* blk_off, cudaStream_t st) {
  const double vb = P.v_key64 ? 8 : 4;
  ProfScope ps("join_emit", P.n_in * (P.in_w64 ? 8.0 : 4.0) + total * (vb + (P.out_w64 ? 8 : 4)), st);
  const u64 n_blk = pjoin_warp_blocks(P.n_in);
  if (n_blk) try_warp<0>(P, (unsigned)(n_blk < 152ull * 16 ? n_blk : 152ull * 16), blk_off, n_blk, nullptr, st);
}

void pjoin_warp_bitmap(const PStep& P, u64* emitted_dev, cudaStream_t st) {
  // the outputs' bytes (a matched key read and a bitmap word per output) are
  // added by the caller once their number is known
  ProfScope ps("join_emit", P.n_in * (P.in_w64 ? 8.0 : 4.0), st);
  if (!P.n_in) return;
  try_warp<2>(P, grid_n(P.n_in), nullptr, 0, reinterpret_cast<unsigned long long*>(emitted_dev), st);
}
