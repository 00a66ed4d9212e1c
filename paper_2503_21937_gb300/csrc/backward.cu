// Reverse-mode gradients of the differentiable semirings (Sec. 3.4: the
// differentiable versions of max-min-prob and add-mult-prob).
//
// diff-max-min: a tag is (v, id) where id is the input row that bounds v, so
//   d tag_o / d p_id = 1 and the backward pass is one scatter of each output's
//   gradient to its id.
// diff-add-mult: a fact h first derived in iteration k has
//   tag(h) = min(1, sum over the groundings g of iteration k with head h of
//                   prod over g's body facts of their tags),
//   so d tag(h) / d tag(f) = [sum <= 1] * (product of the other body tags) for
//   every body fact f of every such grounding.  Iterations are replayed in
//   reverse: all adjoints flowing into a fact of iteration k come from facts of
//   later iterations, so they are complete when iteration k is replayed.  Each
//   replay re-runs iteration k's semi-naive arms on the final relations with
//   stamp filters (delta = stamp k-1, full = stamp < k, old = stamp < k-1;
//   when k begins a stratum after the first, delta = stamp < k: every fact),
//   recomputing the groundings instead of storing them, and pushes
//   adjoint(h) * (product of the other tags) to every body fact with FP64
//   atomics.  Loaded facts finally pass their adjoints to the caller's input
//   rows (times the derivative of the clamped merge of duplicate rows).
#include <algorithm>
#include <cstring>

#include "engine.h"
#include "pjoin.h"
#include "join_common.cuh"
#include "scan.cuh"

namespace {

struct BwdParams {
  int packed_source;                 // step input is the stamp-filtered delta view (fact 0 = that row)
  int n_in_facts;                    // facts carried by a binding-table input
  const u32* in_fact_row[kMaxArity];
  const float* in_fact_tag[kMaxArity];
  const u32* v_prow;                 // probed view row -> primary row (null: primary view)
  u32* out_fact_row[kMaxArity];      // intermediate steps: facts carried forward
  float* out_fact_tag[kMaxArity];
  int last;
  const void* h_keys; int h_key64; u64 h_n; const u32* h_stamp; const double* h_adj; u32 k;
  const u32* h_row;                  // dense key -> row of the head relation (0xFFFFFFFF: absent), or null
  const u32* h_new;                  // bitmap of the head keys first derived, unclamped, in iteration k (or null)
  double* fact_adj[kMaxArity];       // adjoint array of the relation of fact m (null: no adjoint needed)
  int n_facts;                       // body facts of a grounding at the last step
};

// adjoint of the head of a grounding emitted in iteration B.k, or 0 when the
// head was not new in that iteration or its (+) was clamped
LOB_DEV double head_adjoint(const BwdParams& B, u64 key) {
  u64 j;
  if (B.h_row) {
    j = B.h_row[key];
    if (j == 0xFFFFFFFFull) return 0.0;
  } else if (B.h_key64) {
    j = lower_bound_dev<u64>(reinterpret_cast<const u64*>(B.h_keys), 0, B.h_n, key);
    if (j >= B.h_n || reinterpret_cast<const u64*>(B.h_keys)[j] != key) return 0.0;
  } else {
    j = lower_bound_dev<u32>(reinterpret_cast<const u32*>(B.h_keys), 0, B.h_n, (u32)key);
    if (j >= B.h_n || reinterpret_cast<const u32*>(B.h_keys)[j] != (u32)key) return 0.0;
  }
  const u32 st = B.h_stamp[j];
  if ((st & 0x7FFFFFFFu) != B.k || (st & 0x80000000u)) return 0.0;
  return B.h_adj[j];
}

// the head key of a grounding; false when a computed head value drops it
LOB_DEV bool head_key(const StepParams& P, const u32* val, u32 sample, u64& key) {
  const Layout& L = P.out_lay;
  key = L.swidth ? (u64)sample << L.sshift : 0ull;
  for (int j = 0; j < L.arity; j++) {
    u32 x;
    if (!head_value(P, j, val, x)) return false;
    key |= (u64)x << L.shift[j];
  }
  return true;
}

__global__ void __launch_bounds__(256) k_bwd_emit(const __grid_constant__ StepParams P, const __grid_constant__ BwdParams B,
                                                 const u64* __restrict__ part) {
  typedef SemAddMult Sem;
  constexpr int kItems = kEmitTile / 256;
  __shared__ u32 row_of[kEmitTile];
  __shared__ u32 sm[256 / 32 + 1];
  __shared__ u32 th_inc[256];
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
#pragma unroll 1
  for (int i = 0; i < kItems; i++) {
    const u64 j = j0 + (u64)i * 256 + threadIdx.x;
    if (j >= j_end) break;
    const u64 r = r0 + row_of[j - j0];
    const u64 v = P.lo[r] + (j - P.off[r]);
    u32 val[kMaxSlots];
    u32 sample;
    double tag;
    read_input<Sem>(P, r, val, sample, tag);
    bool ok = P.v_stamp_mode == STAMP_NONE || stamp_ok(P.v_stamp[v], P.v_stamp_mode, P.v_stamp_val);
    const u64 vk = load_key(P.v_keys, P.v_lay.key64, v);
    for (int c = 0; c < P.v_lay.arity; c++)
      if (c >= P.prefix_len && ok) ok = apply_act(P.v_act[c], (u32)field_of(vk, P.v_lay.shift[c], P.v_lay.width[c]), val);
    for (int f = 0; f < P.n_filters && ok; f++) ok = eval_filter(P, P.filters[f], val);
    if (B.last) {
      if (!ok) continue;
      u64 hk;
      if (!head_key(P, val, sample, hk)) continue;
      // most groundings re-derive a head that existed before iteration k: one
      // bit of the iteration's new-head bitmap rules them out
      if (B.h_new && !((B.h_new[hk >> 5] >> (hk & 31)) & 1u)) continue;
      const double a = head_adjoint(B, hk);
      if (a == 0.0) continue;
      u32 rows[kMaxArity + 1];
      float tags[kMaxArity + 1];
      int nf = 0;
      if (B.packed_source) {
        rows[nf] = (u32)r;
        tags[nf++] = reinterpret_cast<const float*>(P.in_tags)[r];
      } else {
        for (int q = 0; q < B.n_in_facts; q++) {
          rows[nf] = B.in_fact_row[q][r];
          tags[nf++] = B.in_fact_tag[q][r];
        }
      }
      rows[nf] = B.v_prow ? B.v_prow[v] : (u32)v;
      tags[nf++] = reinterpret_cast<const float*>(P.v_tags)[v];
      for (int q = 0; q < nf; q++) {
        if (!B.fact_adj[q]) continue;
        double c = a;
        for (int l = 0; l < nf; l++)
          if (l != q) c *= (double)tags[l];
        atomicAdd(B.fact_adj[q] + rows[q], c);
      }
      continue;
    }
    // facts of the grounding so far, carried to the next step
    u32 rows[kMaxArity + 1];
    float tags[kMaxArity + 1];
    int nf = 0;
    if (B.packed_source) {
      rows[nf] = (u32)r;
      tags[nf++] = reinterpret_cast<const float*>(P.in_tags)[r];
    } else {
      for (int q = 0; q < B.n_in_facts; q++) {
        rows[nf] = B.in_fact_row[q][r];
        tags[nf++] = B.in_fact_tag[q][r];
      }
    }
    rows[nf] = B.v_prow ? B.v_prow[v] : (u32)v;
    tags[nf++] = reinterpret_cast<const float*>(P.v_tags)[v];
    tag = Sem::mul(tag, (double)tags[nf - 1]);
    const u64 o = j - P.j_begin;
    write_output<Sem>(P, P.out_base + o, ok, val, sample, tag);
    for (int q = 0; q < nf; q++) {
      B.out_fact_row[q][o] = rows[q];
      B.out_fact_tag[q][o] = tags[q];
    }
  }
}

// single-atom rules: each delta row is the only body fact of its grounding
__global__ void k_bwd_project(const __grid_constant__ StepParams P, const __grid_constant__ BwdParams B) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < P.n_in; r += stride) {
    u32 val[kMaxSlots];
    u32 sample;
    double tag;
    if (!read_input<SemAddMult>(P, r, val, sample, tag)) continue;
    u64 hk;
    if (!head_key(P, val, sample, hk)) continue;
    if (B.h_new && !((B.h_new[hk >> 5] >> (hk & 31)) & 1u)) continue;
    const double a = head_adjoint(B, hk);
    if (a != 0.0 && B.fact_adj[0]) atomicAdd(B.fact_adj[0] + r, a);
  }
}

__global__ void k_locate(const void* __restrict__ keys, int key64, u64 n, const void* __restrict__ q, u64 nq,
                         u32* __restrict__ out) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += stride) {
    if (key64) out[i] = (u32)lower_bound_dev<u64>(reinterpret_cast<const u64*>(keys), 0, n, reinterpret_cast<const u64*>(q)[i]);
    else out[i] = (u32)lower_bound_dev<u32>(reinterpret_cast<const u32*>(keys), 0, n, reinterpret_cast<const u32*>(q)[i]);
  }
}

// dense key -> row map of a sorted relation (every other slot stays all ones)
__global__ void k_dense_rows(const void* __restrict__ keys, int key64, u64 n, u32* __restrict__ map) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) map[load_key(keys, key64, i)] = (u32)i;
}

// bits of the facts first derived, with an unclamped (+), in iteration k
__global__ void k_mark_new(const void* __restrict__ keys, int key64, const u32* __restrict__ stamps, u64 n, u32 k,
                           u32* __restrict__ bm) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (stamps[i] == k) {
      const u64 key = load_key(keys, key64, i);
      atomicOr(bm + (key >> 5), 1u << (u32)(key & 31u));
    }
}

__global__ void k_f32_to_f64(const float* __restrict__ a, u64 n, double* __restrict__ out) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (double)a[i];
}

// loaded rows: grad[q] += adjoint(fact of row q) * d(merged tag)/d(row tag)
__global__ void k_bwd_inputs(const void* __restrict__ keys, int key64, u64 n, const void* __restrict__ row_keys,
                             const float* __restrict__ factor, const double* __restrict__ adj, u64 nrows,
                             float* __restrict__ grad) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < nrows; q += stride) {
    u64 j;
    if (key64) j = lower_bound_dev<u64>(reinterpret_cast<const u64*>(keys), 0, n, reinterpret_cast<const u64*>(row_keys)[q]);
    else j = lower_bound_dev<u32>(reinterpret_cast<const u32*>(keys), 0, n, reinterpret_cast<const u32*>(row_keys)[q]);
    grad[q] += (float)(adj[j] * (double)factor[q]);
  }
}

constexpr int kMaxGradRels = 64;
struct GradTable {
  int n;
  u32 base[kMaxGradRels];
  u32 count[kMaxGradRels];
  float* grad[kMaxGradRels];
};

__global__ void k_dmm_scatter(const u64* __restrict__ tags, const float* __restrict__ g, u64 n, GradTable T) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u32 id = dmm_id(tags[i]);
    if (id == 0xFFFFFFFFu) continue;
    for (int k = 0; k < T.n; k++)
      if (id >= T.base[k] && id - T.base[k] < T.count[k]) {
        if (T.grad[k]) atomicAdd(T.grad[k] + (id - T.base[k]), g[i]);
        break;
      }
  }
}

unsigned grid_for_n(u64 n) {
  u64 b = (n + 255) / 256;
  if (b > 152ull * 16) b = 152ull * 16;
  return (unsigned)(b ? b : 1);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct BwdState {
  std::vector<DevBuf> adj;                   // per relation, f64, primary view order
  std::vector<DevBuf> hrow;                  // per derived relation with a small key space: dense key -> row
  std::vector<DevBuf> hnew;                  // and its bitmap of the facts new in the iteration being replayed
  std::vector<std::vector<DevBuf>> prow;     // per relation, per view (index 0 unused)
};

void free_state(lob_engine& e, BwdState& S) {
  for (auto& b : S.adj) e.release(b);
  for (auto& b : S.hrow) e.release(b);
  for (auto& b : S.hnew) e.release(b);
  for (auto& v : S.prow)
    for (auto& b : v) e.release(b);
}

void fill_filters_b(const RuleAst& R, const std::vector<int>& fs, FilterP* out, int& n) {
  n = 0;
  for (int f : fs) {
    const FilterAst& F = R.filters[f];
    FilterP p{};
    p.a_slot = F.a.var ? (int8_t)F.a.v : (int8_t)-1;
    p.a_const = F.a.var ? 0 : F.a.v;
    p.b_slot = F.b.var ? (int8_t)F.b.v : (int8_t)-1;
    p.b_const = F.b.var ? 0 : F.b.v;
    p.eq = F.eq ? 1 : 0;
    p.prog = (uint8_t)F.prog;
    out[n++] = p;
  }
}

// The stamp filter that selects iteration k's recent set from a relation's
// facts: those first derived in iteration k - 1, or, when k begins a stratum
// after the first (every fact recent), all facts derived before k.
void set_delta_stamps(const lob_engine& e, u32 k, int& mode, u32& val) {
  if (begins_stratum(e.stratum_begin, k)) {
    mode = STAMP_LT;
    val = k;
  } else {
    mode = STAMP_EQ;
    val = k - 1;
  }
}

void replay_arm(lob_engine& e, BwdState& S, const RulePlan& rp, const ArmPlan& A, u32 k) {
  const RuleAst& R = rp.ast;
  RelSt& D = e.rels[R.body[A.delta].rel];
  RelSt& H = e.rels[R.head.rel];
  ViewSt& DV = D.views[0];
  ViewSt& HV = H.views[0];
  StepParams P;
  std::memset(&P, 0, sizeof(P));
  P.in_packed = 1;
  P.in_keys = DV.keys.p;
  P.in_lay = DV.lay;
  std::copy(A.steps[0].act, A.steps[0].act + kMaxArity, P.in_act);
  P.in_tags = DV.tags.p;
  P.in_stamp = DV.stamps.as<u32>();
  set_delta_stamps(e, k, P.in_stamp_mode, P.in_stamp_val);
  P.n_in = DV.n;
  fill_filters_b(R, A.steps[0].filters, P.in_filters, P.n_in_filters);
  P.out_lay = HV.lay;
  for (int j = 0; j < kMaxArity; j++) { P.head_slot[j] = -1; P.head_const[j] = 0; }
  for (size_t c = 0; c < R.head.args.size(); c++) {
    if (R.head.args[c].var) P.head_slot[c] = (int8_t)R.head.args[c].v;
    else P.head_const[c] = R.head.args[c].v;
  }
  set_rule_code(R, P);
  BwdParams B;
  std::memset(&B, 0, sizeof(B));
  B.packed_source = 1;
  B.h_keys = HV.keys.p;
  B.h_key64 = HV.lay.key64;
  B.h_n = HV.n;
  B.h_stamp = HV.stamps.as<u32>();
  B.h_adj = S.adj[R.head.rel].as<double>();
  B.h_row = S.hrow[R.head.rel].as<u32>();
  B.h_new = S.hnew[R.head.rel].as<u32>();
  B.k = k;
  // adjoints are kept for derived relations and for tagged inputs; an untagged
  // input fact (tag 1, not differentiable) needs none
  auto adj_of = [&](u32 rel) -> double* {
    const RelSt& q = e.rels[rel];
    return q.idb || q.in_has_tags ? S.adj[rel].as<double>() : nullptr;
  };
  B.fact_adj[0] = adj_of(R.body[A.delta].rel);
  for (size_t s = 1; s < A.steps.size(); s++) B.fact_adj[s] = adj_of(R.body[A.steps[s].atom].rel);
  B.n_facts = (int)A.steps.size();
  if (A.steps.size() == 1) {
    B.last = 1;
    ProfScope ps("bwd_project", P.n_in * (16.0 + 12.0), e.stream);
    k_bwd_project<<<grid_for_n(P.n_in), 256, 0, e.stream>>>(P, B);
    e.after_launch("backward project");
    e.launches++;
    return;
  }
  int side = 0;
  for (size_t s = 1; s < A.steps.size(); s++) {
    const StepPlan& SP = A.steps[s];
    const bool last = s + 1 == A.steps.size();
    RelSt& V = e.rels[R.body[SP.atom].rel];
    ViewSt& W = V.views[SP.view];
    if (!W.n) return;
    engine_ensure_index(e, W, SP.prefix_len);
    IndexSt& I = W.index[SP.prefix_len];
    P.has_probe = 1;
    P.v_keys = W.keys.p;
    P.v_lay = W.lay;
    P.v_tags = W.tags.p;
    P.v_stamp = W.stamps.as<u32>();
    P.v_n = W.n;
    P.v_stamp_mode = STAMP_LT;
    P.v_stamp_val = SP.probe_old ? k - 1 : k;
    P.prefix_len = SP.prefix_len;
    std::copy(SP.prefix_slot, SP.prefix_slot + kMaxArity, P.prefix_slot);
    std::copy(SP.prefix_const, SP.prefix_const + kMaxArity, P.prefix_const);
    std::copy(SP.act, SP.act + kMaxArity, P.v_act);
    P.index_mode = I.mode;
    P.dense_offs = I.offs.as<u64>();
    P.dense_domain = I.domain;
    P.hash_bits = I.hash_bits;
    fill_filters_b(R, SP.filters, P.filters, P.n_filters);
    B.v_prow = SP.view ? S.prow[R.body[SP.atom].rel][SP.view].as<u32>() : nullptr;
    e.ensure(e.cnt, P.n_in * 4);
    e.ensure(e.lo, P.n_in * 8);
    e.ensure(e.off, (P.n_in + 1) * 8);
    P.cnt = e.cnt.as<u32>();
    P.lo = e.lo.as<u64>();
    join_count(SR_ADD_MULT, P, e.stream);
    e.after_launch("backward count");
    e.ensure(e.scratch, scan_scratch_elems(P.n_in) * 8 + 64);
    exclusive_scan<u32, u64>(e.cnt.as<u32>(), e.off.as<u64>(), P.n_in, e.counts.as<u64>(), e.scratch.as<u64>(), e.stream);
    e.after_launch("backward scan");
    e.launches += 1 + scan_launches(P.n_in);
    const u64 total = e.read_u64(e.counts.as<u64>());
    if (!total) return;
    const int out_side = side ^ 1;
    B.last = last;
    const int nf = (int)s + 1;  // facts after this step
    if (!last) {
      P.out_packed = 0;
      P.n_out_cols = (int)SP.live.size();
      for (int q = 0; q < P.n_out_cols; q++) {
        e.ensure(e.bind[out_side][q], total * 4);
        P.out_slot[q] = (int8_t)SP.live[q];
        P.out_cols[q] = e.bind[out_side][q].as<u32>();
      }
      e.ensure(e.bind[out_side][kMaxSlots], total * 4);
      P.out_sample = e.bind[out_side][kMaxSlots].as<u32>();
      e.ensure(e.bind[out_side][kMaxSlots + 1], total * 8);
      P.out_tags = e.bind[out_side][kMaxSlots + 1].p;
      P.out_base = 0;
      for (int q = 0; q < nf; q++) {
        e.ensure(e.bfact[out_side][2 * q], total * 4);
        e.ensure(e.bfact[out_side][2 * q + 1], total * 4);
        B.out_fact_row[q] = e.bfact[out_side][2 * q].as<u32>();
        B.out_fact_tag[q] = e.bfact[out_side][2 * q + 1].as<float>();
      }
    }
    const u64 ntiles = (total + kEmitTile - 1) / kEmitTile;
    e.ensure(e.part, (ntiles + 1) * 8);
    lbs_partition(e.off.as<u64>(), P.n_in, 0, total, e.part.as<u64>(), e.stream);
    P.off = e.off.as<u64>();
    P.total = total;
    P.j_begin = 0;
    {
      // per grounding: its input row and matched fact read; an intermediate
      // row (+ carried facts) written, or the head's adjoint looked up and one
      // adjoint pushed per body fact
      const double per = last ? 8.0 + 4.0 + 8.0 + 8.0 * nf : 8.0 + 4.0 + 16.0 + 8.0 * nf;
      ProfScope ps("bwd_emit", P.n_in * 24.0 + total * per, e.stream);
      k_bwd_emit<<<(unsigned)ntiles, 256, 0, e.stream>>>(P, B, e.part.as<u64>());
    }
    e.after_launch("backward emit");
    e.launches += 2;
    if (last) return;
    side = out_side;
    P.in_packed = 0;
    P.in_stamp_mode = STAMP_NONE;
    P.n_in = total;
    P.n_in_cols = (int)std::min(SP.live.size(), (size_t)kMaxSlots);
    for (int q = 0; q < P.n_in_cols; q++) {
      P.in_slot[q] = (int8_t)SP.live[q];
      P.in_cols[q] = e.bind[side][q].as<u32>();
    }
    P.in_sample = e.bind[side][kMaxSlots].as<u32>();
    P.in_tags = e.bind[side][kMaxSlots + 1].p;
    P.n_in_filters = 0;
    B.packed_source = 0;
    B.n_in_facts = nf;
    for (int q = 0; q < nf; q++) {
      B.in_fact_row[q] = e.bfact[side][2 * q].as<u32>();
      B.in_fact_tag[q] = e.bfact[side][2 * q + 1].as<float>();
    }
  }
}

// The same replay on the packed kernels (pjoin.cu): returns false when the arm
// is not a packed pipeline of at least one probe, or its head has no dense
// key map, and the general replay runs instead.
bool replay_arm_packed(lob_engine& e, BwdState& S, const RulePlan& rp, const ArmPlan& A, u32 k) {
  if (!e.opt_packed_backward || !A.packed.ok || A.steps.size() < 2) return false;
  for (const PStep& T : A.packed.steps)
    if (!pjoin_backward_supported(T)) return false;
  const RuleAst& R = rp.ast;
  const u32 hrel = R.head.rel;
  if (!S.hnew[hrel].p || !S.hrow[hrel].p) return false;
  RelSt& D = e.rels[R.body[A.delta].rel];
  ViewSt& DV = D.views[0];
  RelSt& H = e.rels[hrel];
  auto adj_of = [&](u32 rel) -> double* {
    const RelSt& q = e.rels[rel];
    return q.idb || q.in_has_tags ? S.adj[rel].as<double>() : nullptr;
  };
  PBwd B;
  std::memset(&B, 0, sizeof(B));
  B.packed_source = 1;
  B.h_new = S.hnew[hrel].as<u32>();
  B.h_row = S.hrow[hrel].as<u32>();
  B.h_keys = H.views[0].keys.p;
  B.h_key64 = H.views[0].lay.key64;
  B.h_n = H.views[0].n;
  B.h_adj = S.adj[hrel].as<double>();
  B.fact_tags[0] = DV.tags.as<float>();
  B.fact_adj[0] = adj_of(R.body[A.delta].rel);
  for (size_t s = 1; s < A.steps.size(); s++) {
    const u32 rel = R.body[A.steps[s].atom].rel;
    B.fact_tags[s] = e.rels[rel].views[0].tags.as<float>();
    B.fact_adj[s] = adj_of(rel);
  }
  const void* in_words = DV.keys.p;
  u64 n_in = DV.n;
  int side = 0;
  for (size_t s = 1; s < A.steps.size(); s++) {
    const StepPlan& SP = A.steps[s];
    const bool last = s + 1 == A.steps.size();
    const u32 vrel = R.body[SP.atom].rel;
    ViewSt& W = e.rels[vrel].views[SP.view];
    if (!W.n || !n_in) return true;
    engine_ensure_index(e, W, SP.prefix_len);
    PStep P = A.packed.steps[s - 1];
    P.in_words = in_words;
    P.in_tags = nullptr;
    P.n_in = n_in;
    if (s == 1) {  // the delta atom: the recent set of iteration k
      P.in_stamp = DV.stamps.as<u32>();
      set_delta_stamps(e, k, P.in_stamp_mode, P.in_stamp_val);
    } else {
      P.in_stamp_mode = STAMP_NONE;
    }
    P.v_keys = W.keys.p;
    P.v_key64 = W.lay.key64;
    P.v_tags = W.tags.p;
    P.v_stamp = W.stamps.as<u32>();
    P.v_n = W.n;
    P.v_stamp_mode = STAMP_LT;
    P.v_stamp_val = SP.probe_old ? k - 1 : k;
    const IndexSt& I = W.index[SP.prefix_len];
    P.index_mode = I.mode;
    P.dense_offs = I.offs.as<u64>();
    P.hash_bits = I.hash_bits;
    const u64 n_blk = pjoin_loc_blocks(n_in);
    e.ensure(e.cnt, n_in * 4);
    e.ensure(e.lo, n_in * 4);
    e.ensure(e.off, n_blk * 16);
    P.loc = e.cnt.as<u32>();
    P.lo32 = e.lo.as<u32>();
    P.blk_cnt = e.off.as<u64>() + n_blk;
    P.blk_off = e.off.as<u64>();
    P.err = reinterpret_cast<u32*>(e.counts.as<u64>() + 1);
    e.check(cudaMemsetAsync(P.err, 0, sizeof(u64), e.stream), "join error word");
    pjoin_count(SR_ADD_MULT, P, e.stream);
    e.after_launch("backward count");
    e.ensure(e.scratch, scan_scratch_elems(n_blk) * 8 + 64);
    exclusive_scan<u64, u64>(P.blk_cnt, e.off.as<u64>(), n_blk, e.counts.as<u64>(), e.scratch.as<u64>(), e.stream);
    e.after_launch("backward scan");
    e.launches += 1 + scan_launches(n_blk);
    e.check(cudaMemcpyAsync(e.pinned, e.counts.as<u64>(), 16, cudaMemcpyDeviceToHost, e.stream), "join total");
    e.sync();
    if (e.pinned[1] & kErrLocOverflow)
      throw LobError(LOB_E_ARG, "join step: 1024 consecutive input rows have 2^32 or more matches");
    const u64 total = e.pinned[0];
    if (!total) return true;
    B.last = last;
    B.v_prow = SP.view ? S.prow[vrel][SP.view].as<u32>() : nullptr;
    const int nf_in = B.packed_source ? 1 : B.n_in_facts;
    const int out_side = side ^ 1;
    if (!last) {
      e.ensure(e.bind[out_side][0], total * (P.out_w64 ? 8 : 4));
      P.out_words = e.bind[out_side][0].p;
      for (int q = 0; q <= nf_in; q++) {
        e.ensure(e.bfact[out_side][q], total * 4);
        B.out_rows[q] = e.bfact[out_side][q].as<u32>();
      }
    }
    const u64 ntiles = (total + kEmitTile - 1) / kEmitTile;
    e.ensure(e.part, (ntiles + 1) * 8);
    P.total = total;
    P.j_begin = 0;
    pjoin_partition(P, ntiles, e.part.as<u64>(), e.stream);
    pjoin_backward_emit(P, B, e.part.as<u64>(), e.stream);
    e.after_launch("backward emit");
    e.launches += 2;
    if (last) return true;
    side = out_side;
    in_words = e.bind[side][0].p;
    n_in = total;
    B.packed_source = 0;
    B.n_in_facts = nf_in + 1;
    for (int q = 0; q < B.n_in_facts; q++) B.in_rows[q] = e.bfact[side][q].as<u32>();
  }
  return true;
}

}  // namespace

int backward_impl(lob_engine* e, u32 out_rel, const float* grad_tags, float* const* grad_inputs, int mem) {
  if (!e->ran_diff) throw LobError(LOB_E_STATE, "lob_backward needs a completed LOB_DIFF_* run");
  if (out_rel >= e->rels.size()) throw LobError(LOB_E_UNKNOWN_REL, "unknown relation id");
  if (mem != LOB_MEM_HOST && mem != LOB_MEM_DEVICE) throw LobError(LOB_E_ARG, "bad mem");
  if (!grad_inputs) throw LobError(LOB_E_ARG, "null grad_inputs");
  RelSt& O = e->rels[out_rel];
  const u64 n_out = O.views[0].n;
  if (n_out && !grad_tags) throw LobError(LOB_E_ARG, "null grad_tags");
  const size_t nrel = e->rels.size();
  // device views of the caller's buffers
  DevBuf g, gin_all;
  std::vector<float*> gin(nrel, nullptr);
  const float* gdev = grad_tags;
  if (mem == LOB_MEM_HOST) {
    e->ensure(g, std::max<u64>(n_out, 1) * 4);
    if (n_out) e->check(cudaMemcpyAsync(g.p, grad_tags, n_out * 4, cudaMemcpyHostToDevice, e->stream), "grad in");
    gdev = g.as<float>();
    u64 tot = 0;
    for (size_t k = 0; k < nrel; k++)
      if (grad_inputs[k]) tot += e->rels[k].n_in;
    e->ensure(gin_all, std::max<u64>(tot, 1) * 4);
    u64 off = 0;
    for (size_t k = 0; k < nrel; k++)
      if (grad_inputs[k]) {
        gin[k] = gin_all.as<float>() + off;
        if (e->rels[k].n_in)
          e->check(cudaMemcpyAsync(gin[k], grad_inputs[k], e->rels[k].n_in * 4, cudaMemcpyHostToDevice, e->stream),
                   "grad inputs in");
        off += e->rels[k].n_in;
      }
  } else {
    for (size_t k = 0; k < nrel; k++) gin[k] = grad_inputs[k];
  }
  if (e->semiring == LOB_DIFF_MAX_MIN) {
    if (nrel > (size_t)kMaxGradRels) throw LobError(LOB_E_ARG, "more than 64 relations");
    GradTable T{};
    T.n = (int)nrel;
    for (size_t k = 0; k < nrel; k++) {
      T.base[k] = e->rels[k].id_base;
      T.count[k] = (u32)e->rels[k].n_in;
      T.grad[k] = gin[k];
    }
    if (n_out) {
      k_dmm_scatter<<<grid_for_n(n_out), 256, 0, e->stream>>>(O.views[0].tags.as<u64>(), gdev, n_out, T);
      e->after_launch("max-min backward");
    }
  } else if (e->semiring == LOB_DIFF_TOP1_PROOFS) {
    // each output's probability is the product over its proof: its gradient
    // goes to every input fact of the proof (top1.cu)
    if (nrel > (size_t)kTop1GradRels) throw LobError(LOB_E_ARG, "more than 64 relations");
    Top1GradTable T{};
    T.n = (int)nrel;
    for (size_t k = 0; k < nrel; k++) {
      T.base[k] = e->rels[k].id_base;
      T.count[k] = (u32)e->rels[k].n_in;
      T.grad[k] = gin[k];
    }
    top1_grad_scatter(O.views[0].tags.as<u64>(), gdev, n_out, e->arena.as<u32>(), e->top1_prob.as<float>(), T, e->stream);
    e->after_launch("top-1-proofs backward");
  } else {
    BwdState S;
    try {
      S.adj.resize(nrel);
      S.hrow.resize(nrel);
      S.hnew.resize(nrel);
      S.prow.resize(nrel);
      for (size_t k = 0; k < nrel; k++) {
        RelSt& r = e->rels[k];
        const u64 n = r.views[0].n;
        const Layout& L = r.views[0].lay;
        if (r.idb && n && L.bits <= e->opt_acc_bits) {  // heads are found by one load instead of a binary search
          const u64 slots = 1ull << L.bits;
          e->ensure(S.hrow[k], slots * 4);
          e->check(cudaMemsetAsync(S.hrow[k].p, 0xFF, slots * 4, e->stream), "head rows");
          k_dense_rows<<<grid_for_n(n), 256, 0, e->stream>>>(r.views[0].keys.p, L.key64, n, S.hrow[k].as<u32>());
          e->after_launch("head rows");
          e->ensure(S.hnew[k], std::max<u64>(16, slots / 8));
        }
        e->ensure(S.adj[k], std::max<u64>(n, 1) * 8);
        e->check(cudaMemsetAsync(S.adj[k].p, 0, std::max<u64>(n, 1) * 8, e->stream), "adjoint init");
        if (n > 0xFFFFFFFFull) throw LobError(LOB_E_ARG, "backward supports relations below 2^32 facts");
        S.prow[k].resize(r.views.size());
        for (size_t vi = 1; vi < r.views.size(); vi++) {
          ViewSt& W = r.views[vi];
          if (!W.n) continue;
          const int kb = r.views[0].lay.key64 ? 8 : 4;
          e->ensure(e->tmp_keys, W.n * kb);
          repack_keys(W.lay, W.perm, r.views[0].lay, r.views[0].perm, W.keys.p, e->tmp_keys.p, W.n, e->stream);
          e->ensure(S.prow[k][vi], W.n * 4);
          k_locate<<<grid_for_n(W.n), 256, 0, e->stream>>>(r.views[0].keys.p, r.views[0].lay.key64, r.views[0].n,
                                                             e->tmp_keys.p, W.n, S.prow[k][vi].as<u32>());
          e->after_launch("view rows");
        }
      }
      if (n_out) {
        k_f32_to_f64<<<grid_for_n(n_out), 256, 0, e->stream>>>(gdev, n_out, S.adj[out_rel].as<double>());
        e->after_launch("adjoint seed");
      }
      // Only relations out_rel depends on carry adjoints: rules with another
      // head contribute nothing and are not replayed.
      std::vector<char> needed(nrel, 0);
      needed[out_rel] = 1;
      for (bool grew = true; grew;) {
        grew = false;
        for (auto& p : e->plans)
          if (needed[p.ast.head.rel])
            for (auto& a : p.ast.body)
              if (!needed[a.rel]) needed[a.rel] = grew = true;
      }
      // facts first derived in iteration k (the recent set at the start of k + 1,
      // unless k + 1 began a stratum: then iteration k, its stratum's last, found none)
      auto new_in = [&](u32 k, u32 rel) -> u64 {
        if (begins_stratum(e->stratum_begin, k + 1)) return 0;
        return k < e->iter_counts.size() ? e->iter_counts[k][rel].second : e->rels[rel].n_recent;
      };
      for (u32 k = e->last_iter; k >= 1; k--) {
        for (size_t q = 0; q < nrel; q++) {  // the heads new in iteration k
          if (!S.hnew[q].p || !needed[q] || !new_in(k, (u32)q)) continue;
          RelSt& r = e->rels[q];
          e->check(cudaMemsetAsync(S.hnew[q].p, 0, S.hnew[q].cap, e->stream), "new heads");
          k_mark_new<<<grid_for_n(r.views[0].n), 256, 0, e->stream>>>(r.views[0].keys.p, r.views[0].lay.key64,
                                                                      r.views[0].stamps.as<u32>(), r.views[0].n, k,
                                                                      S.hnew[q].as<u32>());
          e->after_launch("new heads");
        }
        const int stratum = stratum_of_iter(e->stratum_begin, k);
        for (auto& p : e->plans)
          for (auto& A : p.arms) {
            if (p.stratum != stratum) continue;  // the rule did not run in iteration k
            if (!needed[p.ast.head.rel] || !new_in(k, p.ast.head.rel)) continue;  // no adjoint can flow here
            const auto& cnt = e->iter_counts[k - 1];  // (total, recent) per relation at the start of iteration k
            if (!cnt[p.ast.body[A.delta].rel].second) continue;
            bool skip = false;
            for (u32 b : A.before_rels)
              if (cnt[b].first == cnt[b].second) { skip = true; break; }
            if (skip) continue;
            if (!replay_arm_packed(*e, S, p, A, k)) replay_arm(*e, S, p, A, k);
          }
      }
      for (size_t k = 0; k < nrel; k++) {
        RelSt& r = e->rels[k];
        if (!gin[k] || !r.n_in || !r.views[0].n) continue;
        k_bwd_inputs<<<grid_for_n(r.n_in), 256, 0, e->stream>>>(r.views[0].keys.p, r.views[0].lay.key64, r.views[0].n,
                                                                 r.row_keys.p, r.row_factor.as<float>(),
                                                                 S.adj[k].as<double>(), r.n_in, gin[k]);
        e->after_launch("input gradients");
      }
    } catch (...) {
      free_state(*e, S);
      throw;
    }
    free_state(*e, S);
  }
  if (mem == LOB_MEM_HOST) {
    for (size_t k = 0; k < nrel; k++)
      if (grad_inputs[k] && e->rels[k].n_in)
        e->check(cudaMemcpyAsync(grad_inputs[k], gin[k], e->rels[k].n_in * 4, cudaMemcpyDeviceToHost, e->stream),
                 "grad inputs out");
  }
  e->sync();
  e->release(g);
  e->release(gin_all);
  return LOB_OK;
}
