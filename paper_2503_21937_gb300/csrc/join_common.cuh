// Device helpers shared by the forward join kernels and the backward replay:
// decoding an input row into rule variables, looking up the matching range of a
// sorted relation view, applying filters and writing outputs.
#pragma once
#include "kernels.h"

LOB_DEV bool apply_act(const ColAct& a, u32 v, u32* val) {
  if (a.op == OP_BIND) {
    val[a.slot] = v;
    return true;
  }
  if (a.op == OP_CHECK_SLOT) return val[a.slot] == v;
  return v == a.cnst;
}

// Run bytecode program `prog` of P on the row's variables; false when a
// division by zero drops the row.
LOB_DEV bool bc_run(const StepParams& P, int prog, const u32* val, u32& out) {
  u32 st[kBcStack];
  int sp = 0;
  const int b = P.prog_off[prog], n = P.prog_len[prog];
  for (int i = 0; i < n; i++) {
    const BcIns I = P.code[b + i];
    if (I.op == BC_VAR) {
      st[sp++] = val[I.slot];
    } else if (I.op == BC_CONST) {
      st[sp++] = I.imm;
    } else {
      const u32 y = st[--sp];
      const u32 x = st[sp - 1];
      u32 r;
      switch (I.op) {
        case BC_ADD: r = x + y; break;
        case BC_SUB: r = x - y; break;
        case BC_MUL: r = x * y; break;
        case BC_DIV:
          if (y == 0) return false;
          r = x / y;
          break;
        case BC_EQ: r = x == y; break;
        case BC_NE: r = x != y; break;
        case BC_LT: r = x < y; break;
        case BC_LE: r = x <= y; break;
        case BC_GT: r = x > y; break;
        default: r = x >= y; break;
      }
      st[sp - 1] = r;
    }
  }
  out = st[0];
  return true;
}

LOB_DEV bool eval_filter(const StepParams& P, const FilterP& f, const u32* val) {
  if (f.prog) {
    u32 r;
    return bc_run(P, f.prog - 1, val, r) && r != 0u;
  }
  u32 a = f.a_slot >= 0 ? val[f.a_slot] : f.a_const;
  u32 b = f.b_slot >= 0 ? val[f.b_slot] : f.b_const;
  return (a == b) == (f.eq != 0);
}

// Value of head column j; false drops the row (a division by zero, or a
// computed value of 2^32 - 1, which the keys reserve).
LOB_DEV bool head_value(const StepParams& P, int j, const u32* val, u32& x) {
  if (P.head_prog[j]) return bc_run(P, P.head_prog[j] - 1, val, x) && x != 0xFFFFFFFFu;
  x = P.head_slot[j] >= 0 ? val[P.head_slot[j]] : P.head_const[j];
  return true;
}

LOB_DEV bool stamp_ok(u32 s, int mode, u32 v) {
  s &= 0x7FFFFFFFu;
  return mode == STAMP_LT ? s < v : s == v;
}

template <class Sem>
LOB_DEV bool read_input(const StepParams& P, u64 r, u32* val, u32& sample, typename Sem::Cand& tag) {
  typedef typename Sem::Stored S;
  typedef typename Sem::Cand C;
  if (P.in_packed) {
    if (P.in_stamp_mode != STAMP_NONE && !stamp_ok(P.in_stamp[r], P.in_stamp_mode, P.in_stamp_val)) return false;
    const u64 key = load_key(P.in_keys, P.in_lay.key64, r);
    sample = P.in_lay.swidth ? (u32)field_of(key, P.in_lay.sshift, P.in_lay.swidth) : 0u;
#pragma unroll
    for (int j = 0; j < kMaxArity; j++) {
      if (j >= P.in_lay.arity) break;
      if (!apply_act(P.in_act[j], (u32)field_of(key, P.in_lay.shift[j], P.in_lay.width[j]), val)) return false;
    }
    for (int f = 0; f < P.n_in_filters; f++)
      if (!eval_filter(P, P.in_filters[f], val)) return false;
    if constexpr (Sem::kTags) tag = Sem::from_stored(reinterpret_cast<const S*>(P.in_tags)[r]);
    else tag = Sem::one();
  } else {
    sample = P.in_sample[r];
    if (sample == 0xFFFFFFFFu) return false;
    for (int k = 0; k < P.n_in_cols; k++) val[P.in_slot[k]] = P.in_cols[k][r];
    if constexpr (Sem::kTags) tag = reinterpret_cast<const C*>(P.in_tags)[r];
    else tag = Sem::one();
  }
  return true;
}

template <class K>
LOB_DEV u64 lower_bound_keys(const K* a, u64 n, K x) {
  u64 lo = 0, hi = n;
  while (lo < hi) {
    u64 mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

LOB_DEV u64 lower_bound_any(const void* keys, int key64, u64 n, u64 x) {
  if (key64) return lower_bound_keys(reinterpret_cast<const u64*>(keys), n, x);
  if (x > 0xFFFFFFFFull) return n;
  return lower_bound_keys(reinterpret_cast<const u32*>(keys), n, (u32)x);
}

// range of view rows whose first prefix_len view columns (and sample) match
LOB_DEV bool probe_range(const StepParams& P, const u32* val, u32 sample, u64& lo, u64& hi) {
  const Layout& L = P.v_lay;
  const int p = P.prefix_len;
  if (p == 0 && L.swidth == 0) {
    lo = 0;
    hi = P.v_n;
    return hi > 0;
  }
  const int rs = rest_shift(L, p);
  u64 pv = 0;
  if (L.swidth) {
    if ((u64)sample >> L.swidth) return false;
    pv |= (u64)sample << (L.sshift - rs);
  }
  for (int j = 0; j < p; j++) {
    const u32 x = P.prefix_slot[j] >= 0 ? val[P.prefix_slot[j]] : P.prefix_const[j];
    if (L.width[j] < 32 && (x >> L.width[j])) return false;
    pv |= (u64)x << (L.shift[j] - rs);
  }
  if (P.index_mode == INDEX_DENSE) {
    lo = P.dense_offs[pv];
    hi = P.dense_offs[pv + 1];
  } else if (P.index_mode == INDEX_HASH) {
    hash_find(reinterpret_cast<const HashSlot*>(P.dense_offs), P.hash_bits, pv, lo, hi);
  } else {
    const u64 klo = pv << rs;
    const u64 khi = klo + (1ull << rs);
    lo = lower_bound_any(P.v_keys, L.key64, P.v_n, klo);
    hi = khi < klo ? P.v_n : lower_bound_any(P.v_keys, L.key64, P.v_n, khi);
  }
  return hi > lo;
}

template <class Sem>
LOB_DEV void write_output(const StepParams& P, u64 o, bool ok, const u32* val, u32 sample, typename Sem::Cand tag) {
  typedef typename Sem::Cand C;
  if (P.out_packed) {
    const Layout& L = P.out_lay;
    u64 key = L.swidth ? (u64)sample << L.sshift : 0ull;
#pragma unroll
    for (int j = 0; j < kMaxArity; j++) {
      if (j >= L.arity || !ok) break;
      u32 x;
      ok = head_value(P, j, val, x);
      key |= (u64)x << L.shift[j];
    }
    if (!ok) key = invalid_of(L.key64);
    store_key(P.out_keys, L.key64, o, key);
  } else {
    P.out_sample[o] = ok ? sample : 0xFFFFFFFFu;
    if (ok)
      for (int k = 0; k < P.n_out_cols; k++) P.out_cols[k][o] = val[P.out_slot[k]];
  }
  if constexpr (Sem::kTags) reinterpret_cast<C*>(P.out_tags)[o] = tag;
}

