// C ABI, memory management, planning and the semi-naive iteration driver.
//
// Per iteration k (Algorithm 1; the appendix's Join and Stratum rules):
//   1. every rule arm whose delta relation has recent facts runs its join
//      pipeline (count -> scan -> emit, one step per body atom) and appends
//      candidate head tuples (packed keys + tags) to the head's buffer;
//   2. per head relation: radix sort, unique with (+), then one fused pass that
//      drops candidates already in the full relation F (or keeps them when
//      their tag improves, for idempotent (+)), merges the rest into F and
//      writes them as the next recent set; secondary sorted views of the
//      relation receive the same new facts;
//   3. stop when no relation has recent facts; a program of several strata
//      runs them in order, each to this stop (assign_strata).
#include <algorithm>
#include <cstring>
#include <functional>

#include "engine.h"
#include "scan.cuh"

RuleAst parse_rule(const lob_engine& e, const char* text);
bool valid_ident(const char* s);
int backward_impl(lob_engine* e, u32 out_rel, const float* grad_tags, float* const* grad_inputs, int mem);

static thread_local std::string g_create_err;
thread_local KernelProfiler* g_prof = nullptr;

// ---------------------------------------------------------------------------
// per-kernel CUDA-event timing
// ---------------------------------------------------------------------------
cudaEvent_t EngineProfiler::take() {
  if (pool.empty()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) throw LobError(LOB_E_CUDA, "cudaEventCreate failed");
    return ev;
  }
  cudaEvent_t ev = pool.back();
  pool.pop_back();
  return ev;
}
void EngineProfiler::begin(const char* name, cudaStream_t st) {
  cudaEvent_t a = take();
  cudaEventRecord(a, st);
  open.push_back({name, a});
}
void EngineProfiler::end(const char* name, double bytes, cudaStream_t st) {
  if (open.empty()) return;
  cudaEvent_t b = take();
  cudaEventRecord(b, st);
  Open o = open.back();
  open.pop_back();
  done.push_back({name, o.a, b, bytes});
}
void EngineProfiler::add_last_bytes(double bytes) {
  if (!done.empty()) done.back().bytes += bytes;
}
void EngineProfiler::flush() {
  for (auto& d : done) {
    cudaEventSynchronize(d.b);
    float ms = 0;
    cudaEventElapsedTime(&ms, d.a, d.b);
    ProfAgg& g = agg[d.name];
    g.launches++;
    g.ms += ms;
    g.bytes += d.bytes;
    pool.push_back(d.a);
    pool.push_back(d.b);
  }
  done.clear();
}
EngineProfiler::~EngineProfiler() {
  for (auto& d : done) { cudaEventDestroy(d.a); cudaEventDestroy(d.b); }
  for (auto& o : open) cudaEventDestroy(o.a);
  for (auto ev : pool) cudaEventDestroy(ev);
}

// ---------------------------------------------------------------------------
// memory and errors
// ---------------------------------------------------------------------------
void lob_engine::check(cudaError_t c, const char* what) {
  if (c != cudaSuccess) {
    cudaGetLastError();
    if (c == cudaErrorMemoryAllocation) throw LobError(LOB_E_OOM, std::string(what) + ": out of device memory");
    throw LobError(LOB_E_CUDA, std::string(what) + ": " + cudaGetErrorString(c));
  }
}

void lob_engine::after_launch(const char* what) {
  check(cudaGetLastError(), what);
  if (opt_sync_check) check(cudaStreamSynchronize(stream), what);
}

void* lob_engine::dalloc(size_t bytes) {
  if (!bytes) return nullptr;
  void* p = nullptr;
  if (custom_alloc) {
    p = alloc.alloc(bytes, stream, alloc.ctx);
  } else if (cudaMallocFromPoolAsync(&p, bytes, pool, stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) throw LobError(LOB_E_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  live_bytes += bytes;
  peak_bytes = std::max(peak_bytes, live_bytes);
  return p;
}

void lob_engine::dfree(void* p, size_t bytes) {
  if (!p) return;
  if (custom_alloc) alloc.release(p, bytes, stream, alloc.ctx);
  else cudaFreeAsync(p, stream);
  live_bytes -= bytes;
}

// Grow-only buffers reused across iterations (Sec. 4.1, buffer reuse): a
// buffer is replaced only when a request exceeds its capacity, with slack.
void lob_engine::ensure(DevBuf& b, size_t bytes, bool keep) {
  if (b.cap >= bytes) return;
  size_t cap = std::max(bytes, b.cap + b.cap / 2);
  cap = (cap + 255) & ~(size_t)255;
  void* p = dalloc(cap);
  if (keep && b.p) check(cudaMemcpyAsync(p, b.p, b.cap, cudaMemcpyDeviceToDevice, stream), "grow copy");
  dfree(b.p, b.cap);
  b.p = p;
  b.cap = cap;
}

void lob_engine::release(DevBuf& b) {
  dfree(b.p, b.cap);
  b.p = nullptr;
  b.cap = 0;
}

u64 lob_engine::read_u64(const u64* dev) {
  check(cudaMemcpyAsync(pinned, dev, sizeof(u64), cudaMemcpyDeviceToHost, stream), "readback");
  check(cudaStreamSynchronize(stream), "readback sync");
  host_syncs++;
  return pinned[0];
}

void lob_engine::sync() {
  check(cudaStreamSynchronize(stream), "synchronize");
  host_syncs++;
}

static void release_view(lob_engine& e, ViewSt& v) {
  for (DevBuf* b : {&v.keys, &v.tags, &v.stamps, &v.keys2, &v.tags2, &v.stamps2}) e.release(*b);
  for (auto& kv : v.index) e.release(kv.second.offs);
  v.index.clear();
  v.n = 0;
}

static void release_derived(lob_engine& e) {
  for (auto& r : e.rels) {
    for (auto& v : r.views) release_view(e, v);
    r.views.clear();
    for (DevBuf* b : {&r.rkeys, &r.rtags, &r.nkeys, &r.ntags, &r.ckeys, &r.ctags, &r.ckeys2, &r.ctags2, &r.row_factor,
                      &r.row_keys, &r.akeys, &r.atags, &r.akeys2, &r.atags2, &r.bitmap, &r.prev_bitmap, &r.dacc,
                      &r.dtouched})
      e.release(*b);
    r.extract = r.touched = r.keys_stale = r.dense = false;
    r.n_recent = r.n_next = r.n_cand = r.n_acc = 0;
    r.flushed = false;
    r.filter_on = false;
    r.last_cand = r.last_new = r.cand_iter = 0;
  }
  for (DevBuf* b : {&e.arena, &e.top1_state, &e.top1_prob}) e.release(*b);
  e.arena_tail = e.arena_cap = 0;
  e.plans.clear();
}

void lob_engine::release_all() {
  release_derived(*this);
  for (auto& r : rels) {
    for (auto& b : r.in_cols) release(b);
    release(r.in_tags);
    release(r.in_samples);
  }
  for (DevBuf* b : {&scratch, &cnt, &lo, &off, &part, &counts, &tmp_keys, &tmp_tags, &tmp_keys2, &tmp_tags2}) release(*b);
  for (auto& side : bind)
    for (auto& b : side) release(b);
  for (auto& side : bfact)
    for (auto& b : side) release(b);
}

// ---------------------------------------------------------------------------
// layouts and planning
// ---------------------------------------------------------------------------
static int bitlen(u64 x) { return x ? 64 - __builtin_clzll(x) : 0; }


static void make_layout(const lob_engine& e, const RelSt& r, const int* perm, Layout& L) {
  std::memset(&L, 0, sizeof(L));
  L.arity = (int)r.arity;
  int sh = 0;
  for (int j = (int)r.arity - 1; j >= 0; j--) {
    L.width[j] = r.width[perm[j]];
    L.shift[j] = sh;
    sh += L.width[j];
  }
  L.sshift = sh;
  L.swidth = e.swidth;
  L.bits = sh + e.swidth;
  L.key64 = L.bits > 32;
  if (L.bits > 64)
    throw LobError(LOB_E_KEY_WIDTH, "relation '" + r.name + "' needs " + std::to_string(L.bits) +
                                        " key bits (sample id + columns); at most 64 are supported");
}

static int find_view(lob_engine& e, RelSt& r, const int* perm) {
  for (size_t i = 0; i < r.views.size(); i++)
    if (std::equal(perm, perm + r.arity, r.views[i].perm)) return (int)i;
  ViewSt v;
  std::copy(perm, perm + r.arity, v.perm);
  make_layout(e, r, perm, v.lay);
  r.views.push_back(std::move(v));
  return (int)r.views.size() - 1;
}

static ArmPlan plan_arm(lob_engine& e, const RuleAst& R, int delta, bool idempotent) {
  ArmPlan A;
  A.delta = delta;
  for (int i = 0; i < delta; i++) A.before_rels.push_back(R.body[i].rel);
  const int nv = (int)R.var_names.size();
  std::vector<char> bound(nv, 0), used(R.body.size(), 0);
  std::vector<std::vector<char>> bound_after;
  {  // source: the delta atom read from the recent set (primary layout)
    StepPlan s;
    s.atom = delta;
    s.view = 0;
    const AtomAst& a = R.body[delta];
    for (size_t c = 0; c < a.args.size(); c++) {
      const Term& t = a.args[c];
      ColAct act{};
      if (!t.var) { act.op = OP_CHECK_CONST; act.cnst = t.v; act.slot = -1; }
      else if (!bound[t.v]) { act.op = OP_BIND; act.slot = (int8_t)t.v; bound[t.v] = 1; }
      else { act.op = OP_CHECK_SLOT; act.slot = (int8_t)t.v; }
      s.act[c] = act;
    }
    used[delta] = 1;
    A.steps.push_back(s);
    bound_after.push_back(bound);
  }
  // Greedy join order: next the atom with the most bound columns; on a tie an
  // input relation (fixed size, static index) before a derived one, then the
  // smaller input relation, then body order.
  for (size_t n_used = 1; n_used < R.body.size(); n_used++) {
    int best = -1, best_b = -1, best_edb = -1;
    u64 best_n = 0;
    for (size_t i = 0; i < R.body.size(); i++) {
      if (used[i]) continue;
      int b = 0;
      for (auto& t : R.body[i].args) b += (!t.var || bound[t.v]);
      const RelSt& cand = e.rels[R.body[i].rel];
      const int edb = cand.idb ? 0 : 1;
      const u64 n = cand.n_in;
      const bool better = b > best_b || (b == best_b && (edb > best_edb || (edb == best_edb && edb && n < best_n)));
      if (better) { best_b = b; best = (int)i; best_edb = edb; best_n = n; }
    }
    const AtomAst& a = R.body[best];
    RelSt& rel = e.rels[a.rel];
    int perm[kMaxArity];
    int np = 0;
    for (size_t c = 0; c < a.args.size(); c++)
      if (!a.args[c].var || bound[a.args[c].v]) perm[np++] = (int)c;
    const int prefix = np;
    for (size_t c = 0; c < a.args.size(); c++)
      if (a.args[c].var && !bound[a.args[c].v]) perm[np++] = (int)c;
    StepPlan s;
    s.atom = best;
    s.view = find_view(e, rel, perm);
    rel.views[s.view].probed = true;
    s.prefix_len = prefix;
    for (int j = 0; j < kMaxArity; j++) { s.prefix_slot[j] = -1; s.prefix_const[j] = 0; s.act[j] = ColAct{}; }
    for (int j = 0; j < prefix; j++) {
      const Term& t = a.args[perm[j]];
      if (t.var) s.prefix_slot[j] = (int8_t)t.v;
      else s.prefix_const[j] = t.v;
    }
    for (int j = prefix; j < (int)a.args.size(); j++) {
      const Term& t = a.args[perm[j]];
      ColAct act{};
      act.slot = (int8_t)t.v;
      if (!bound[t.v]) { act.op = OP_BIND; bound[t.v] = 1; }
      else act.op = OP_CHECK_SLOT;
      s.act[j] = act;
    }
    s.probe_old = best < delta && !idempotent && rel.idb;
    used[best] = 1;
    A.steps.push_back(s);
    bound_after.push_back(bound);
  }
  // filters at the first step that binds all their variables
  for (size_t f = 0; f < R.filters.size(); f++) {
    const FilterAst& F = R.filters[f];
    for (size_t s = 0; s < A.steps.size(); s++) {
      bool ok = (!F.a.var || bound_after[s][F.a.v]) && (!F.b.var || bound_after[s][F.b.v]);
      for (u32 v : F.vars) ok = ok && bound_after[s][v];
      if (ok) { A.steps[s].filters.push_back((int)f); break; }
    }
  }
  // live variables after each non-final step
  for (size_t s = 0; s + 1 < A.steps.size(); s++) {
    std::vector<char> need(nv, 0);
    for (size_t q = s + 1; q < A.steps.size(); q++) {
      for (auto& t : R.body[A.steps[q].atom].args)
        if (t.var) need[t.v] = 1;
      for (int f : A.steps[q].filters) {
        if (R.filters[f].a.var) need[R.filters[f].a.v] = 1;
        if (R.filters[f].b.var) need[R.filters[f].b.v] = 1;
        for (u32 v : R.filters[f].vars) need[v] = 1;
      }
    }
    for (auto& t : R.head.args)
      if (t.var) need[t.v] = 1;
    for (u32 v : R.head_vars) need[v] = 1;
    for (int v = 0; v < nv; v++)
      if (need[v] && bound_after[s][v]) A.steps[s].live.push_back(v);
  }
  return A;
}

// ---------------------------------------------------------------------------
// packed-word compilation of an arm (see pjoin.cu)
// ---------------------------------------------------------------------------
static POperand op_field(int word, int shift, int width) {
  POperand o{};
  o.word = (uint8_t)word;
  o.shift = (uint8_t)shift;
  o.width = (uint8_t)width;
  return o;
}
static POperand op_const(u32 c) {
  POperand o{};
  o.word = 2;
  o.cval = c;
  return o;
}

static PackedArm compile_packed(lob_engine& e, const RuleAst& R, const ArmPlan& A) {
  PackedArm out;
  const int nv = (int)R.var_names.size();
  std::vector<POperand> loc(nv, op_const(0));
  auto term_op = [&](const Term& t) { return t.var ? loc[t.v] : op_const(t.v); };
  auto add_check = [&](PCheck* arr, int& n, POperand a, POperand b, bool eq) {
    if (n >= kMaxPChecks) return false;
    PCheck c{};
    c.a = a;
    c.b = b;
    c.eq = eq ? 1 : 0;
    arr[n++] = c;
    return true;
  };
  PStep cur;
  std::memset(&cur, 0, sizeof(cur));
  // source atom: the delta relation's primary layout
  const RelSt& D = e.rels[R.body[A.delta].rel];
  const Layout& L0 = D.views[0].lay;
  cur.in_packed = 1;
  cur.in_w64 = L0.key64;
  std::vector<char> bound(nv, 0);
  for (size_t c = 0; c < R.body[A.delta].args.size(); c++) {
    const Term& t = R.body[A.delta].args[c];
    const POperand f = op_field(0, L0.shift[c], L0.width[c]);
    if (!t.var) { if (!add_check(cur.in_checks, cur.n_in_checks, f, op_const(t.v), true)) return out; }
    else if (bound[t.v]) { if (!add_check(cur.in_checks, cur.n_in_checks, f, loc[t.v], true)) return out; }
    else { loc[t.v] = f; bound[t.v] = 1; }
  }
  for (int f : A.steps[0].filters) {
    const FilterAst& F = R.filters[f];
    if (!add_check(cur.in_checks, cur.n_in_checks, term_op(F.a), term_op(F.b), F.eq)) return out;
  }
  POperand sample = L0.swidth ? op_field(0, L0.sshift, L0.swidth) : op_const(0);
  const Layout& HL = e.rels[R.head.rel].views[0].lay;
  auto head_fields = [&](PStep& P) {
    P.n_out = 0;
    for (size_t c = 0; c < R.head.args.size(); c++) {
      PField f{};
      f.op = term_op(R.head.args[c]);
      f.shift = (uint8_t)HL.shift[c];
      P.out[P.n_out++] = f;
    }
    if (HL.swidth) {
      PField f{};
      f.op = sample;
      f.shift = (uint8_t)HL.sshift;
      P.out[P.n_out++] = f;
    }
    P.out_w64 = HL.key64;
  };
  if (A.steps.size() == 1) {
    head_fields(cur);
    out.steps.push_back(cur);
    out.ok = true;
    return out;
  }
  for (size_t s = 1; s < A.steps.size(); s++) {
    const StepPlan& S = A.steps[s];
    const AtomAst& atom = R.body[S.atom];
    const ViewSt& W = e.rels[atom.rel].views[S.view];
    const Layout& WL = W.lay;
    const int rs = rest_shift(WL, S.prefix_len);
    cur.n_prefix = 0;
    if (WL.swidth) {
      PField f{};
      f.op = sample;
      f.shift = (uint8_t)(WL.sshift - rs);
      f.limit_bits = (uint8_t)WL.swidth;
      cur.prefix[cur.n_prefix++] = f;
    }
    for (int j = 0; j < S.prefix_len; j++) {
      PField f{};
      f.op = term_op(atom.args[W.perm[j]]);
      f.shift = (uint8_t)(WL.shift[j] - rs);
      f.limit_bits = (uint8_t)WL.width[j];
      cur.prefix[cur.n_prefix++] = f;
    }
    cur.rest_shift = rs >= 64 ? 0 : rs;
    cur.whole_view = S.prefix_len == 0 && WL.swidth == 0;
    cur.n_checks = 0;
    for (int j = S.prefix_len; j < (int)atom.args.size(); j++) {
      const Term& t = atom.args[W.perm[j]];
      const POperand f = op_field(1, WL.shift[j], WL.width[j]);
      const ColAct& act = S.act[j];
      if (act.op == OP_BIND) loc[t.v] = f;
      else if (!add_check(cur.checks, cur.n_checks, f, act.op == OP_CHECK_CONST ? op_const(act.cnst) : loc[t.v], true))
        return out;
    }
    for (int f : S.filters) {
      const FilterAst& F = R.filters[f];
      if (!add_check(cur.checks, cur.n_checks, term_op(F.a), term_op(F.b), F.eq)) return out;
    }
    const bool last = s + 1 == A.steps.size();
    if (last) {
      head_fields(cur);
      out.steps.push_back(cur);
      break;
    }
    // binding word of the live variables (and the sample id) for the next step
    int acc = 0;
    cur.n_out = 0;
    std::vector<POperand> next(nv, op_const(0));
    for (int v : S.live) {
      PField f{};
      f.op = loc[v];
      f.shift = (uint8_t)acc;
      cur.out[cur.n_out++] = f;
      next[v] = op_field(0, acc, loc[v].width);
      acc += loc[v].width;
      if (cur.n_out >= kMaxPFields) return out;
    }
    POperand next_sample = op_const(0);
    if (WL.swidth) {
      PField f{};
      f.op = sample;
      f.shift = (uint8_t)acc;
      cur.out[cur.n_out++] = f;
      next_sample = op_field(0, acc, WL.swidth);
      acc += WL.swidth;
    }
    if (acc > 64 || acc == 0) return out;
    cur.out_w64 = acc > 32;
    out.steps.push_back(cur);
    // the next step reads this binding word
    PStep nxt;
    std::memset(&nxt, 0, sizeof(nxt));
    nxt.in_packed = 0;
    nxt.in_w64 = cur.out_w64;
    loc = next;
    sample = next_sample;
    cur = nxt;
  }
  out.ok = true;
  return out;
}

// The fused cross-product form of a two-probe arm whose second probe's prefix
// is bound by the delta atom alone (see pjoin_warp_cross_bitmap).
static void compile_cross(lob_engine& e, const RuleAst& R, const ArmPlan& A, PackedArm& out) {
  if (!out.ok || A.steps.size() != 3) return;
  const int nv = (int)R.var_names.size();
  std::vector<POperand> loc(nv, op_const(0));
  std::vector<char> src(nv, 0);
  const Layout& L0 = e.rels[R.body[A.delta].rel].views[0].lay;
  for (size_t c = 0; c < R.body[A.delta].args.size(); c++) {
    const Term& t = R.body[A.delta].args[c];
    if (t.var && !src[t.v]) {
      loc[t.v] = op_field(0, L0.shift[c], L0.width[c]);
      src[t.v] = 1;
    }
  }
  const POperand sample = L0.swidth ? op_field(0, L0.sshift, L0.swidth) : op_const(0);
  const StepPlan& S1 = A.steps[1];
  const ViewSt& W1 = e.rels[R.body[S1.atom].rel].views[S1.view];
  for (int j = S1.prefix_len; j < (int)R.body[S1.atom].args.size(); j++)
    if (S1.act[j].op == OP_BIND) loc[R.body[S1.atom].args[W1.perm[j]].v] = op_field(1, W1.lay.shift[j], W1.lay.width[j]);
  const StepPlan& S2 = A.steps[2];
  const AtomAst& atom = R.body[S2.atom];
  const ViewSt& W2 = e.rels[atom.rel].views[S2.view];
  const Layout& WL = W2.lay;
  for (int j = 0; j < S2.prefix_len; j++) {
    const Term& t = atom.args[W2.perm[j]];
    if (t.var && !src[t.v]) return;  // keyed by a variable the first probe binds: no cross product
  }
  PStep P;
  std::memset(&P, 0, sizeof(P));
  const int rs = rest_shift(WL, S2.prefix_len);
  auto term_op = [&](const Term& t) { return t.var ? loc[t.v] : op_const(t.v); };
  if (WL.swidth) {
    PField f{};
    f.op = sample;
    f.shift = (uint8_t)(WL.sshift - rs);
    f.limit_bits = (uint8_t)WL.swidth;
    P.prefix[P.n_prefix++] = f;
  }
  for (int j = 0; j < S2.prefix_len; j++) {
    PField f{};
    f.op = term_op(atom.args[W2.perm[j]]);
    f.shift = (uint8_t)(WL.shift[j] - rs);
    f.limit_bits = (uint8_t)WL.width[j];
    P.prefix[P.n_prefix++] = f;
  }
  P.rest_shift = rs >= 64 ? 0 : rs;
  P.whole_view = S2.prefix_len == 0 && WL.swidth == 0;
  for (int j = S2.prefix_len; j < (int)atom.args.size(); j++) {
    const Term& t = atom.args[W2.perm[j]];
    const POperand f = op_field(3, WL.shift[j], WL.width[j]);
    const ColAct& act = S2.act[j];
    if (act.op == OP_BIND) {
      loc[t.v] = f;
    } else {
      if (P.n_checks >= kMaxPChecks) return;
      PCheck c{};
      c.a = f;
      c.b = act.op == OP_CHECK_CONST ? op_const(act.cnst) : loc[t.v];
      c.eq = 1;
      P.checks[P.n_checks++] = c;
    }
  }
  for (int f : S2.filters) {
    if (P.n_checks >= kMaxPChecks) return;
    PCheck c{};
    c.a = term_op(R.filters[f].a);
    c.b = term_op(R.filters[f].b);
    c.eq = R.filters[f].eq ? 1 : 0;
    P.checks[P.n_checks++] = c;
  }
  const Layout& HL = e.rels[R.head.rel].views[0].lay;
  for (size_t c = 0; c < R.head.args.size(); c++) {
    PField f{};
    f.op = term_op(R.head.args[c]);
    f.shift = (uint8_t)HL.shift[c];
    P.out[P.n_out++] = f;
  }
  if (HL.swidth) {
    PField f{};
    f.op = sample;
    f.shift = (uint8_t)HL.sshift;
    P.out[P.n_out++] = f;
  }
  P.out_w64 = HL.key64;
  if (!pjoin_cross_supported(out.steps[0], P)) return;
  out.cross = P;
  out.cross_ok = true;
}

// Strata (Sec. 3.1: a RAM program is a sequence of strata; Algorithm 1 runs
// each to its fixpoint before the next).  Derived relations that depend on one
// another, directly or through others, form a component; a component's level
// is 0 when its rules read no derived relation outside it, else one more than
// the highest level among the components they read.  Components of one level
// never read each other, so they share a stratum (one semi-naive loop); the
// levels run in increasing order.  Only semirings whose result depends on that
// order (sem_strata) are split; the others keep every rule in one loop.
static void assign_strata(lob_engine& e, int sem) {
  e.n_strata = 1;
  for (auto& p : e.plans) p.stratum = 0;
  if (!sem_strata(sem)) return;
  const size_t n = e.rels.size();
  std::vector<std::vector<char>> dep(n, std::vector<char>(n, 0));  // dep[h][b]: h reads b
  for (auto& p : e.plans)
    for (auto& a : p.ast.body)
      if (e.rels[a.rel].idb) dep[p.ast.head.rel][a.rel] = 1;
  for (size_t m = 0; m < n; m++)
    for (size_t h = 0; h < n; h++)
      if (dep[h][m])
        for (size_t b = 0; b < n; b++) dep[h][b] |= dep[m][b];
  std::vector<int> level(n, 0);
  for (size_t round = 0; round <= n; round++) {
    bool changed = false;
    for (size_t h = 0; h < n; h++) {
      if (!e.rels[h].idb) continue;
      int lv = 0;
      for (size_t b = 0; b < n; b++)
        if (dep[h][b] && !dep[b][h]) lv = std::max(lv, level[b] + 1);  // b lies in a lower component
      for (size_t b = 0; b < n; b++)  // the component shares one level
        if (dep[h][b] && dep[b][h]) lv = std::max(lv, level[b]);
      if (lv != level[h]) {
        level[h] = lv;
        changed = true;
      }
    }
    if (!changed) break;
  }
  for (auto& p : e.plans) {
    p.stratum = level[p.ast.head.rel];
    e.n_strata = std::max(e.n_strata, p.stratum + 1);
  }
}

static void prepare(lob_engine& e, int sem) {
  release_derived(e);
  e.semiring = sem;
  // column widths: bitlen(max + 1) of the loaded values, so that no field ever
  // holds its all-ones value (the all-ones key marks dropped candidates)
  u32* dmax = reinterpret_cast<u32*>(e.counts.p) + 32;
  bool any_samples = false;
  u32 max_sample = 0;
  for (auto& r : e.rels) {
    for (u32 c = 0; c < r.arity; c++) {
      u32 m = 0;
      if (r.n_in) {
        reduce_max_u32(r.in_cols[0].as<u32>() + (u64)c * r.in_cap, r.n_in, dmax, e.stream);
        e.after_launch("column max");
        m = (u32)(e.read_u64(reinterpret_cast<u64*>(dmax)) & 0xFFFFFFFFull);
      }
      r.width[c] = r.n_in ? std::max(1, bitlen((u64)m + 1)) : 1;
    }
    if (r.in_has_samples && r.n_in) {
      reduce_max_u32(r.in_samples.as<u32>(), r.n_in, dmax, e.stream);
      e.after_launch("sample max");
      max_sample = std::max(max_sample, (u32)(e.read_u64(reinterpret_cast<u64*>(dmax)) & 0xFFFFFFFFull));
      any_samples = true;
    }
  }
  e.swidth = any_samples ? bitlen((u64)max_sample + 1) : 0;
  for (auto& r : e.rels) r.idb = false;
  for (auto& R : e.rules) e.rels[R.head.rel].idb = true;
  for (bool changed = true; changed;) {
    changed = false;
    for (auto& R : e.rules) {
      RelSt& h = e.rels[R.head.rel];
      for (size_t c = 0; c < R.head.args.size(); c++) {
        const Term& t = R.head.args[c];
        int need = 1;
        if (c < R.head_prog.size() && R.head_prog[c]) need = 32;  // computed: any u32 but 2^32 - 1
        else if (!t.var) need = bitlen((u64)t.v + 1);
        else
          for (auto& a : R.body)
            for (size_t q = 0; q < a.args.size(); q++)
              if (a.args[q].var && a.args[q].v == t.v) need = std::max(need, e.rels[a.rel].width[q]);
        if (need > h.width[c]) { h.width[c] = need; changed = true; }
      }
    }
  }
  for (auto& r : e.rels) {
    int id[kMaxArity];
    for (int j = 0; j < kMaxArity; j++) id[j] = j;
    find_view(e, r, id);
  }
  const bool idem = sem_idempotent(sem);
  for (auto& R : e.rules) {
    RulePlan p;
    p.ast = R;
    for (size_t i = 0; i < R.body.size(); i++) p.arms.push_back(plan_arm(e, R, (int)i, idem));
    e.plans.push_back(std::move(p));
  }
  assign_strata(e, sem);
  // A secondary view is merged every iteration only if an arm whose delta
  // relation can have recent facts after iteration 1 (a rule head) probes it;
  // arms whose delta is a plain input relation run in iteration 1 only.  The
  // add-mult runs keep every view current (their views carry stamps).
  for (auto& p : e.plans)
    for (auto& A : p.arms) {
      const bool late = e.rels[p.ast.body[A.delta].rel].idb || sem_stamps(sem);
      for (size_t s = 1; s < A.steps.size(); s++)
        if (late) {
          ViewSt& W = e.rels[p.ast.body[A.steps[s].atom].rel].views[A.steps[s].view];
          W.maintained = true;
          W.probed_late = true;
        }
    }
  for (auto& p : e.plans)
    for (auto& A : p.arms) {
      // top-1-proofs joins form unions of proofs, and computed head arguments
      // and comparison filters run bytecode: general steps only
      A.packed = e.opt_packed_join && !sem_top1(sem) && !p.ast.computes() ? compile_packed(e, p.ast, A) : PackedArm{};
      if (sem == SR_UNIT) compile_cross(e, p.ast, A, A.packed);
    }
}

// ---------------------------------------------------------------------------
// loading facts into the full relations (stamp 0) and the first recent sets
// ---------------------------------------------------------------------------
static void scratch_at_least(lob_engine& e, size_t bytes) { e.ensure(e.scratch, bytes); }

// error word of the look-back sort (set by a kernel whose bounded wait gave up)
static u32* sort_err(lob_engine& e) { return reinterpret_cast<u32*>(e.counts.as<u64>() + 15); }

// Radix sort with the engine's chosen algorithm: reduce-then-scan passes by
// default, or one kernel per pass with decoupled look-back (option sort_algo=1).
static void engine_sort(lob_engine& e, int key64, int pay_bytes, void** keys, void** pay, void* ktmp, void* ptmp, u64 n,
                        int bits) {
  const int rb = sort_supported_radix_bits(e.opt_radix_bits);
  const bool onesweep = e.opt_sort_algo == 1 && (bits + rb - 1) / rb <= 8;
  if (onesweep) {
    scratch_at_least(e, sort_onesweep_scratch_bytes(n, rb));
    sort_pairs_onesweep(key64, pay_bytes, keys, pay, ktmp, ptmp, n, bits, rb, e.scratch.p, sort_err(e), e.stream);
    e.launches += sort_onesweep_launches(n, bits, rb);
  } else {
    scratch_at_least(e, sort_scratch_bytes(n, rb));
    sort_pairs(key64, pay_bytes, keys, pay, ktmp, ptmp, n, bits, rb, e.scratch.p, e.stream);
    e.launches += sort_kernel_launches(n, bits, rb);
  }
}

// Re-encode n primary-layout facts into view `v`'s layout and sort them.
// Returns pointers (into the engine's tmp buffers) to the sorted keys and tags.
static std::pair<void*, void*> sort_view_rows(lob_engine& e, RelSt& r, ViewSt& v, const void* pkeys, const void* ptags,
                                              u64 n) {
  const int sem = e.semiring;
  const int kb = v.lay.key64 ? 8 : 4, sb = stored_bytes(sem);
  e.ensure(e.tmp_keys, n * kb);
  e.ensure(e.tmp_keys2, n * kb);
  if (sb) {
    e.ensure(e.tmp_tags, n * sb);
    e.ensure(e.tmp_tags2, n * sb);
    e.check(cudaMemcpyAsync(e.tmp_tags.p, ptags, n * sb, cudaMemcpyDeviceToDevice, e.stream), "copy tags");
  }
  repack_keys(r.views[0].lay, r.views[0].perm, v.lay, v.perm, pkeys, e.tmp_keys.p, n, e.stream);
  e.after_launch("repack");
  void* k = e.tmp_keys.p;
  void* t = e.tmp_tags.p;
  engine_sort(e, v.lay.key64, sb, &k, &t, e.tmp_keys2.p, e.tmp_tags2.p, n, v.lay.bits);
  e.after_launch("view sort");
  e.launches += 1;
  return {k, t};
}

// top-1-proofs: the proof arena (empty proof + one singleton proof per
// input-fact id) and the probability of every id
constexpr u64 kArenaMaxWords = 0xFFFFFFFFull;  // tags address words with 32 bits
static void top1_setup(lob_engine& e, u64 n_ids) {
  const u64 base_words = 1 + 2 * n_ids;
  if (base_words > kArenaMaxWords) throw LobError(LOB_E_ARG, "top-1-proofs: more than 2^31 - 1 loaded rows");
  const u64 words = std::min(kArenaMaxWords, base_words + e.opt_arena_words);
  e.ensure(e.arena, words * 4);
  e.arena_cap = std::min<u64>(kArenaMaxWords, e.arena.cap / 4);
  top1_init_arena(e.arena.as<u32>(), n_ids, e.stream);
  e.after_launch("proof arena");
  e.ensure(e.top1_prob, std::max<u64>(n_ids, 1) * 4);
  for (auto& r : e.rels) {
    if (!r.n_in) continue;
    float* dst = e.top1_prob.as<float>() + r.id_base;
    if (r.in_has_tags)
      e.check(cudaMemcpyAsync(dst, r.in_tags.p, r.n_in * 4, cudaMemcpyDeviceToDevice, e.stream), "fact probabilities");
    else
      fill_f32(dst, r.n_in, 1.0f, e.stream);
  }
  e.ensure(e.top1_state, 16);
  e.check(cudaMemsetAsync(e.top1_state.p, 0, 16, e.stream), "proof arena state");
  set_u64_dev(e.top1_state.as<unsigned long long>(), base_words, e.stream);
  e.arena_tail = base_words;
  e.launches += 3;
}

static Top1Arena top1_desc(lob_engine& e) {
  Top1Arena A{};
  A.words = e.arena.as<u32>();
  A.tail = e.top1_state.as<unsigned long long>();
  A.cap = e.arena_cap;
  A.prob = e.top1_prob.as<float>();
  A.proof_cap = (u32)e.opt_proof_cap;
  A.err = reinterpret_cast<u32*>(e.top1_state.as<u64>() + 1);
  return A;
}

// After a top-1-proofs join emission: a union longer than the proof cap is an
// error; when the arena ran out, it grows (keeping the proofs before this
// step) and the step runs again from the same tail.  Emission is idempotent:
// every output has a fixed position.
static void top1_after_emit(lob_engine& e, int sem, StepParams& P, const u64* part) {
  for (;;) {
    e.check(cudaMemcpyAsync(e.pinned, e.top1_state.p, 16, cudaMemcpyDeviceToHost, e.stream), "proof arena state");
    e.sync();
    const u64 tail = e.pinned[0];
    if (e.pinned[1] & 1)
      throw LobError(LOB_E_CAPACITY, "top-1-proofs: a proof is longer than the proof cap (option proof_cap)");
    if (tail <= e.arena_cap) {
      e.arena_tail = tail;
      return;
    }
    if (e.arena_cap >= kArenaMaxWords) throw LobError(LOB_E_CAPACITY, "top-1-proofs: the proof arena needs 2^32 words");
    const u64 want = std::min(kArenaMaxWords, std::max(2 * e.arena_cap, tail + tail / 2));
    e.ensure(e.arena, want * 4, true);
    e.arena_cap = std::min<u64>(kArenaMaxWords, e.arena.cap / 4);
    set_u64_dev(e.top1_state.as<unsigned long long>(), e.arena_tail, e.stream);
    P.top1 = top1_desc(e);
    join_emit(sem, P, part, e.stream);
    e.after_launch("join emit (proof arena grown)");
    e.launches += 2;
  }
}

static void load_facts(lob_engine& e) {
  const int sem = e.semiring;
  const int ks = sem_kernel(sem);
  const int sb = stored_bytes(sem);
  const bool stamps = sem_stamps(sem);
  u64 id_base = 0;
  for (auto& r : e.rels) {
    r.id_base = (u32)id_base;
    id_base += r.n_in;
    if (id_base > 0xFFFFFFFEull) throw LobError(LOB_E_ARG, "more than 2^32-2 loaded rows");
    ViewSt& V = r.views[0];
    const u64 n = r.n_in;
    V.n = 0;
    r.n_recent = 0;
    if (!n) continue;
    const int kb = V.lay.key64 ? 8 : 4;
    e.ensure(e.tmp_keys, n * kb);
    e.ensure(e.tmp_keys2, n * kb);
    e.ensure(e.tmp_tags, n * 4);
    e.ensure(e.tmp_tags2, n * 4);
    pack_rows(V.lay, r.in_cols[0].as<u32>(), r.in_cap, r.in_has_samples ? r.in_samples.as<u32>() : nullptr, n,
              e.tmp_keys.p, e.tmp_tags.as<u32>(), e.stream);
    e.after_launch("pack rows");
    e.launches++;
    if (sem == SR_DIFF_ADD_MULT) {
      e.ensure(r.row_keys, n * kb);
      e.check(cudaMemcpyAsync(r.row_keys.p, e.tmp_keys.p, n * kb, cudaMemcpyDeviceToDevice, e.stream), "row keys");
      e.ensure(r.row_factor, n * 4);
    }
    void* k = e.tmp_keys.p;
    void* rows = e.tmp_tags.p;
    engine_sort(e, V.lay.key64, 4, &k, &rows, e.tmp_keys2.p, e.tmp_tags2.p, n, V.lay.bits);
    e.after_launch("load sort");
    e.ensure(V.keys, n * kb);
    if (sb) e.ensure(V.tags, n * sb);
    if (stamps) e.ensure(V.stamps, n * 4);
    LoadUniqueArgs a{};
    a.sem = ks;
    a.key64 = V.lay.key64;
    a.keys = k;
    a.rows = reinterpret_cast<const u32*>(rows);
    a.n = n;
    a.raw_tags = r.in_has_tags ? r.in_tags.as<float>() : nullptr;
    a.id_base = r.id_base;
    a.differentiable = r.in_has_tags;
    a.okeys = V.keys.p;
    a.otags = V.tags.p;
    a.ostamp = stamps ? V.stamps.as<u32>() : nullptr;
    a.row_factor = sem == SR_DIFF_ADD_MULT ? r.row_factor.as<float>() : nullptr;
    a.count_dev = e.counts.as<u64>();
    scratch_at_least(e, unique_scratch_bytes(n));
    load_unique(a, e.scratch.p, e.stream);
    e.after_launch("load unique");
    e.launches += 2 + scan_launches((n + 4095) / 4096);
    V.n = e.read_u64(e.counts.as<u64>());
    // recent = all loaded facts (Algorithm 1 starts with stable empty, recent = F_T)
    e.ensure(r.rkeys, V.n * kb);
    e.check(cudaMemcpyAsync(r.rkeys.p, V.keys.p, V.n * kb, cudaMemcpyDeviceToDevice, e.stream), "recent keys");
    if (sb) {
      e.ensure(r.rtags, V.n * sb);
      e.check(cudaMemcpyAsync(r.rtags.p, V.tags.p, V.n * sb, cudaMemcpyDeviceToDevice, e.stream), "recent tags");
    }
    r.n_recent = V.n;
    for (size_t vi = 1; vi < r.views.size(); vi++) {
      ViewSt& W = r.views[vi];
      auto kt = sort_view_rows(e, r, W, V.keys.p, V.tags.p, V.n);
      const int wkb = W.lay.key64 ? 8 : 4;
      e.ensure(W.keys, V.n * wkb);
      e.check(cudaMemcpyAsync(W.keys.p, kt.first, V.n * wkb, cudaMemcpyDeviceToDevice, e.stream), "view keys");
      if (sb) {
        e.ensure(W.tags, V.n * sb);
        e.check(cudaMemcpyAsync(W.tags.p, kt.second, V.n * sb, cudaMemcpyDeviceToDevice, e.stream), "view tags");
      }
      W.n = V.n;
      if (stamps) {
        e.ensure(W.stamps, V.n * 4);
        e.check(cudaMemsetAsync(W.stamps.p, 0, V.n * 4, e.stream), "stamps");
      }
    }
  }
  if (sem_top1(sem)) top1_setup(e, id_base);
}

// ---------------------------------------------------------------------------
// one iteration
// ---------------------------------------------------------------------------
static void ensure_index(lob_engine& e, ViewSt& v, int prefix) {
  IndexSt& I = v.index[prefix];
  if (I.valid) return;
  const Layout& L = v.lay;
  if (prefix == 0 && L.swidth == 0) {
    I.mode = INDEX_BSEARCH;
    I.valid = true;
    return;
  }
  const int dbits = L.bits - rest_shift(L, prefix);
  bool dense = dbits <= e.opt_dense_bits;
  if (e.opt_join_index == 1) dense = dbits <= 30;
  if (e.opt_join_index >= 2) dense = false;
  if (e.opt_join_index == 3 && v.n < (1ull << 31)) {
    // hash index of the view's distinct prefixes (Sec. 5.1): at least
    // opt_hash_slots slots per row, so the load factor is at most 1 / opt_hash_slots
    int bits = 4;
    while ((1ull << bits) < (u64)e.opt_hash_slots * std::max<u64>(v.n, 1)) bits++;
    I.mode = INDEX_HASH;
    I.hash_bits = bits;
    I.domain = 1ull << bits;
    e.ensure(I.offs, I.domain * sizeof(HashSlot));
    e.check(cudaMemsetAsync(I.offs.p, 0, I.domain * sizeof(HashSlot), e.stream), "hash index");
    build_hash_index(L, prefix, v.keys.p, v.n, I.offs.p, bits, e.stream);
    e.after_launch("hash index");
    e.launches++;
    I.valid = true;
    return;
  }
  if (dense) {
    I.mode = INDEX_DENSE;
    I.domain = 1ull << dbits;
    e.ensure(I.offs, (I.domain + 1) * 8);
    build_dense_index(L, prefix, v.keys.p, v.n, I.offs.as<u64>(), I.domain, e.stream);
    e.after_launch("dense index");
    e.launches++;
  } else {
    I.mode = INDEX_BSEARCH;
  }
  I.valid = true;
}

// Re-derive a secondary view from the primary view (tags as payload).
static void rebuild_view(lob_engine& e, RelSt& r, ViewSt& W) {
  const ViewSt& V = r.views[0];
  const int sb = stored_bytes(e.semiring), kb = W.lay.key64 ? 8 : 4;
  if (sem_stamps(e.semiring)) throw LobError(LOB_E_STATE, "stale view in a stamped run");
  W.n = V.n;
  if (V.n) {
    auto kt = sort_view_rows(e, r, W, V.keys.p, V.tags.p, V.n);
    e.ensure(W.keys, V.n * kb);
    e.check(cudaMemcpyAsync(W.keys.p, kt.first, V.n * kb, cudaMemcpyDeviceToDevice, e.stream), "view keys");
    if (sb) {
      e.ensure(W.tags, V.n * sb);
      e.check(cudaMemcpyAsync(W.tags.p, kt.second, V.n * sb, cudaMemcpyDeviceToDevice, e.stream), "view tags");
    }
  }
  W.stale = false;
  for (auto& kv : W.index) kv.second.valid = false;
}

void engine_ensure_index(lob_engine& e, ViewSt& v, int prefix) { ensure_index(e, v, prefix); }

static void fill_filters(const RuleAst& R, const std::vector<int>& fs, FilterP* out, int& n) {
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

// the rule's bytecode programs (computed head arguments, comparison filters)
void set_rule_code(const RuleAst& R, StepParams& P) {
  for (int j = 0; j < kMaxArity; j++) P.head_prog[j] = 0;
  for (size_t c = 0; c < R.head_prog.size() && c < (size_t)kMaxArity; c++) P.head_prog[c] = (uint8_t)R.head_prog[c];
  for (size_t k = 0; k < R.progs.size(); k++) {
    P.prog_off[k] = (uint8_t)R.progs[k].first;
    P.prog_len[k] = (uint8_t)R.progs[k].second;
  }
  std::copy(R.code.begin(), R.code.end(), P.code);
}

static void set_head_output(lob_engine& e, const RuleAst& R, StepParams& P, RelSt& H) {
  P.out_packed = 1;
  P.out_lay = H.views[0].lay;
  for (int j = 0; j < kMaxArity; j++) { P.head_slot[j] = -1; P.head_const[j] = 0; }
  for (size_t c = 0; c < R.head.args.size(); c++) {
    if (R.head.args[c].var) P.head_slot[c] = (int8_t)R.head.args[c].v;
    else P.head_const[c] = R.head.args[c].v;
  }
  P.out_keys = H.ckeys.p;
  P.out_tags = H.ctags.p;
  P.out_base = H.n_cand;
}

static void ensure_cand(lob_engine& e, RelSt& H, u64 extra) {
  const int kb = H.views[0].lay.key64 ? 8 : 4;
  const int cb = cand_bytes(e.semiring);
  e.ensure(H.ckeys, (H.n_cand + extra) * kb, true);
  if (cb) e.ensure(H.ctags, (H.n_cand + extra) * cb, true);
}

// Sort + unique the candidates gathered so far and (+)-combine them into the
// iteration's accumulator, so that no sort ever sees more than opt_max_cand keys.
static void flush_candidates(lob_engine& e, RelSt& H) {
  const u64 n = H.n_cand;
  if (H.dense) {  // dense accumulation: candidates are (+)-added into their slots
    dense_fold(sem_kernel(e.semiring), H.views[0].lay.key64, H.ckeys.p, H.ctags.p, n, H.dacc.p, H.dtouched.as<u32>(),
               e.stream);
    e.after_launch("dense fold");
    e.launches += n ? 1 : 0;
    H.n_cand = 0;
    if (n) H.touched = true;
    return;
  }
  if (H.extract) {  // bitmap delta mode: candidates only need their bits set
    bitmap_set_keys(H.ckeys.p, H.views[0].lay.key64, n, H.bitmap.as<u32>(), e.stream);
    e.after_launch("bitmap");
    e.launches += n ? 1 : 0;
    H.n_cand = 0;
    if (n) H.touched = true;  // the iteration's read-out must run even if no candidates follow
    return;
  }
  H.flushed = true;
  if (!n) return;
  const int ks = sem_kernel(e.semiring);
  const Layout& L = H.views[0].lay;
  const int kb = L.key64 ? 8 : 4, cb = cand_bytes(e.semiring);
  if (n > e.opt_max_cand || n >= (1ull << 32)) throw LobError(LOB_E_CUDA, "internal error: candidate chunk too large");
  e.ensure(H.ckeys2, n * kb);
  if (cb) e.ensure(H.ctags2, n * cb);
  void* keys = H.ckeys.p;
  void* tags = H.ctags.p;
  engine_sort(e, L.key64, cb, &keys, &tags, H.ckeys2.p, H.ctags2.p, n, L.bits);
  e.after_launch("chunk sort");
  void* ukeys = keys == H.ckeys.p ? H.ckeys2.p : H.ckeys.p;
  void* utags = tags == H.ctags.p ? H.ctags2.p : H.ctags.p;
  scratch_at_least(e, unique_scratch_bytes(n));
  unique_run(ks, L.key64, keys, tags, n, ukeys, utags, e.counts.as<u64>() + 1, e.scratch.p, e.stream);
  e.after_launch("chunk unique");
  e.launches += 2 + scan_launches((n + 4095) / 4096);
  const u64 nu = e.read_u64(e.counts.as<u64>() + 1);
  H.n_cand = 0;
  if (!nu) return;
  if (!H.n_acc) {
    e.ensure(H.akeys, nu * kb);
    e.check(cudaMemcpyAsync(H.akeys.p, ukeys, nu * kb, cudaMemcpyDeviceToDevice, e.stream), "accumulate");
    if (cb) {
      e.ensure(H.atags, nu * cb);
      e.check(cudaMemcpyAsync(H.atags.p, utags, nu * cb, cudaMemcpyDeviceToDevice, e.stream), "accumulate");
    }
    H.n_acc = nu;
    return;
  }
  e.ensure(H.akeys2, (H.n_acc + nu) * kb);
  if (cb) e.ensure(H.atags2, (H.n_acc + nu) * cb);
  scratch_at_least(e, combine_scratch_bytes(H.n_acc, nu));
  combine_merge(ks, L.key64, H.akeys.p, H.atags.p, H.n_acc, ukeys, utags, nu, H.akeys2.p, H.atags2.p,
                e.counts.as<u64>() + 6, e.scratch.p, e.stream);
  e.after_launch("accumulate");
  e.launches += 3 + scan_launches((H.n_acc + nu + 2047) / 2048);
  e.check(cudaMemcpyAsync(e.pinned, e.counts.as<u64>() + 6, 16, cudaMemcpyDeviceToHost, e.stream), "counts");
  e.sync();
  if (e.pinned[1]) throw LobError(LOB_E_CUDA, "internal error: unsorted input to the candidate accumulator");
  H.n_acc = H.n_acc + nu - e.pinned[0];  // keys present in both lists collapse to one
  std::swap(H.akeys, H.akeys2);
  std::swap(H.atags, H.atags2);
}

// Run one semi-naive arm of a rule for iteration k.  Δ-atom rows are the
// recent facts of the delta relation (or, with `src_stamp`, the rows of its
// primary view carrying that stamp).
static void run_arm(lob_engine& e, const RulePlan& rp, const ArmPlan& A, u32 k) {
  const RuleAst& R = rp.ast;
  RelSt& D = e.rels[R.body[A.delta].rel];
  RelSt& H = e.rels[R.head.rel];
  const int sem = sem_kernel(e.semiring);
  const int cb = cand_bytes(e.semiring);
  if (!D.n_recent) return;
  StepParams P;
  std::memset(&P, 0, sizeof(P));
  const bool top1 = sem_top1(e.semiring);
  if (top1) P.top1 = top1_desc(e);
  set_rule_code(R, P);
  P.in_packed = 1;
  P.in_keys = D.rkeys.p;
  P.in_lay = D.views[0].lay;
  std::copy(A.steps[0].act, A.steps[0].act + kMaxArity, P.in_act);
  P.in_tags = D.rtags.p;
  P.n_in = D.n_recent;
  fill_filters(R, A.steps[0].filters, P.in_filters, P.n_in_filters);
  if (A.steps.size() == 1) {  // one output row per delta row, in chunks of at most opt_max_cand
    const u64 n = P.n_in;
    const int kb = P.in_lay.key64 ? 8 : 4, sb = stored_bytes(e.semiring);
    for (u64 rb = 0; rb < n; rb += e.opt_max_cand) {
      const u64 sub = std::min(e.opt_max_cand, n - rb);
      if (H.n_cand + sub > e.opt_max_cand) flush_candidates(e, H);
      ensure_cand(e, H, sub);
      set_head_output(e, R, P, H);
      P.in_keys = static_cast<const char*>(D.rkeys.p) + rb * kb;
      P.in_tags = sb ? static_cast<const char*>(D.rtags.p) + rb * sb : nullptr;
      P.n_in = sub;
      project_rows(sem, P, e.stream);
      e.after_launch("project");
      e.launches++;
      H.n_cand += sub;
      H.cand_iter += sub;
      H.unfiltered = true;
      e.cand_emitted += sub;
    }
    return;
  }
  int side = 0;
  for (size_t s = 1; s < A.steps.size(); s++) {
    const StepPlan& S = A.steps[s];
    const bool last = s + 1 == A.steps.size();
    RelSt& V = e.rels[R.body[S.atom].rel];
    ViewSt& W = V.views[S.view];
    if (W.stale) rebuild_view(e, V, W);
    if (!W.n) return;
    ensure_index(e, W, S.prefix_len);
    P.has_probe = 1;
    P.v_keys = W.keys.p;
    P.v_lay = W.lay;
    P.v_tags = W.tags.p;
    P.v_stamp = W.stamps.as<u32>();
    P.v_n = W.n;
    P.v_stamp_mode = STAMP_NONE;
    if (S.probe_old) {  // facts older than the previous iteration's recent set
      P.v_stamp_mode = STAMP_LT;
      P.v_stamp_val = k - 1;
    }
    P.prefix_len = S.prefix_len;
    std::copy(S.prefix_slot, S.prefix_slot + kMaxArity, P.prefix_slot);
    std::copy(S.prefix_const, S.prefix_const + kMaxArity, P.prefix_const);
    std::copy(S.act, S.act + kMaxArity, P.v_act);
    const IndexSt& I = W.index[S.prefix_len];
    P.index_mode = I.mode;
    P.dense_offs = I.offs.as<u64>();
    P.dense_domain = I.domain;
    P.hash_bits = I.hash_bits;
    fill_filters(R, S.filters, P.filters, P.n_filters);
    // count -> scan
    e.ensure(e.cnt, P.n_in * 4);
    e.ensure(e.lo, P.n_in * 8);
    e.ensure(e.off, (P.n_in + 1) * 8);
    P.cnt = e.cnt.as<u32>();
    P.lo = e.lo.as<u64>();
    join_count(sem, P, e.stream);
    e.after_launch("join count");
    scratch_at_least(e, scan_scratch_elems(P.n_in) * 8 + 64);
    {
      ProfScope ps("join_scan", P.n_in * 12.0, e.stream);
      exclusive_scan<u32, u64>(e.cnt.as<u32>(), e.off.as<u64>(), P.n_in, e.counts.as<u64>(), e.scratch.as<u64>(), e.stream);
    }
    e.after_launch("join scan");
    e.launches += 1 + scan_launches(P.n_in);
    const u64 total = e.read_u64(e.counts.as<u64>());
    if (!total) return;
    // outputs
    const int out_side = side ^ 1;
    if (last) {  // candidates, emitted in sub-ranges of at most opt_max_cand outputs
      P.off = e.off.as<u64>();
      for (u64 jb = 0; jb < total; jb += e.opt_max_cand) {
        const u64 sub = std::min(e.opt_max_cand, total - jb);
        if (H.n_cand + sub > e.opt_max_cand) flush_candidates(e, H);
        ensure_cand(e, H, sub);
        set_head_output(e, R, P, H);
        const u64 nt = (sub + kEmitTile - 1) / kEmitTile;
        e.ensure(e.part, (nt + 1) * 8);
        lbs_partition(e.off.as<u64>(), P.n_in, jb, sub, e.part.as<u64>(), e.stream);
        P.total = sub;
        P.j_begin = jb;
        if (H.filter_on) {
          P.bitmap = H.bitmap.as<u32>();
          P.out_count = e.counts.as<u64>() + 14;
          e.check(cudaMemsetAsync(P.out_count, 0, sizeof(u64), e.stream), "filter count");
        }
        join_emit(sem, P, e.part.as<u64>(), e.stream);
        e.after_launch("join emit");
        e.launches += 2;
        if (top1) top1_after_emit(e, sem, P, e.part.as<u64>());
        const u64 written = H.filter_on ? e.read_u64(e.counts.as<u64>() + 14) : sub;
        P.bitmap = nullptr;
        P.out_count = nullptr;
        H.n_cand += written;
        H.cand_iter += sub;
        e.cand_emitted += sub;
      }
      return;
    } else {
      P.out_packed = 0;
      P.n_out_cols = (int)S.live.size();
      for (size_t q = 0; q < S.live.size(); q++) {
        e.ensure(e.bind[out_side][q], total * 4);
        P.out_slot[q] = (int8_t)S.live[q];
        P.out_cols[q] = e.bind[out_side][q].as<u32>();
      }
      e.ensure(e.bind[out_side][kMaxSlots], total * 4);
      P.out_sample = e.bind[out_side][kMaxSlots].as<u32>();
      if (cb) e.ensure(e.bind[out_side][kMaxSlots + 1], total * cb);
      P.out_tags = e.bind[out_side][kMaxSlots + 1].p;
      P.out_base = 0;
    }
    const u64 ntiles = (total + kEmitTile - 1) / kEmitTile;
    e.ensure(e.part, (ntiles + 1) * 8);
    lbs_partition(e.off.as<u64>(), P.n_in, 0, total, e.part.as<u64>(), e.stream);
    P.off = e.off.as<u64>();
    P.total = total;
    P.j_begin = 0;
    join_emit(sem, P, e.part.as<u64>(), e.stream);
    e.after_launch("join emit");
    e.launches += 2;
    if (top1) top1_after_emit(e, sem, P, e.part.as<u64>());
    // the binding table becomes the next step's input
    side = out_side;
    P.in_packed = 0;
    P.n_in = total;
    P.n_in_cols = (int)std::min(S.live.size(), (size_t)kMaxSlots);
    for (int q = 0; q < P.n_in_cols; q++) {
      P.in_slot[q] = (int8_t)S.live[q];
      P.in_cols[q] = e.bind[side][q].as<u32>();
    }
    P.in_sample = e.bind[side][kMaxSlots].as<u32>();
    P.in_tags = e.bind[side][kMaxSlots + 1].p;
    P.n_in_filters = 0;
  }
}

// Secondary views of H receive the nr new / improved facts now in H.nkeys.
static void update_secondary_views(lob_engine& e, RelSt& H, u32 k, u64 nr) {
  if (!nr) return;
  const int sem = e.semiring;
  const int ks = sem_kernel(sem);
  const int sb = stored_bytes(sem);
  const bool stamps = sem_stamps(sem);
  for (size_t vi = 1; vi < H.views.size(); vi++) {
    ViewSt& W = H.views[vi];
    if (!W.maintained) {
      W.stale = true;
      continue;
    }
    const int kb = W.lay.key64 ? 8 : 4;
    auto kt = sort_view_rows(e, H, W, H.nkeys.p, H.ntags.p, nr);
    e.ensure(W.keys2, (W.n + nr) * kb);
    if (sb) e.ensure(W.tags2, (W.n + nr) * sb);
    if (stamps) e.ensure(W.stamps2, (W.n + nr) * 4);
    MergeArgs M2{};
    M2.sem = ks;
    M2.key64 = W.lay.key64;
    M2.fkeys = W.keys.p; M2.ftags = W.tags.p; M2.fstamp = stamps ? W.stamps.as<u32>() : nullptr; M2.nf = W.n;
    M2.ukeys = kt.first; M2.utags = kt.second; M2.nu = nr; M2.u_stored = 1;
    M2.okeys = W.keys2.p; M2.otags = W.tags2.p; M2.ostamp = stamps ? W.stamps2.as<u32>() : nullptr;
    M2.rkeys = nullptr; M2.rtags = nullptr;
    M2.stamp = k;
    M2.counts_dev = e.counts.as<u64>() + 9;
    scratch_at_least(e, merge_scratch_bytes(W.n, nr));
    diff_merge(M2, e.scratch.p, e.stream);
    e.after_launch("view merge");
    e.launches += 3 + 2 * scan_launches((W.n + nr + 2047) / 2048);
    e.check(cudaMemcpyAsync(e.pinned, e.counts.as<u64>() + 9, 24, cudaMemcpyDeviceToHost, e.stream), "counts");
    e.sync();
    if (e.pinned[2]) throw LobError(LOB_E_CUDA, "internal error: unsorted input to a view merge");
    const u64 d2 = e.pinned[0];
    W.n = W.n + nr - d2;
    if (H.dense) note_loop_cap(e, "v" + std::to_string(&H - &e.rels[0]) + "." + std::to_string(vi), W.n);
    std::swap(W.keys, W.keys2);
    std::swap(W.tags, W.tags2);
    std::swap(W.stamps, W.stamps2);
    for (auto& kv : W.index) kv.second.valid = false;
  }
}

// The same arm on the packed-word kernels (compile_packed).
static void run_arm_packed(lob_engine& e, const RulePlan& rp, const ArmPlan& A, u32 k) {
  const RuleAst& R = rp.ast;
  RelSt& D = e.rels[R.body[A.delta].rel];
  RelSt& H = e.rels[R.head.rel];
  const int sem = sem_kernel(e.semiring);
  const int cb = cand_bytes(e.semiring), sb = stored_bytes(e.semiring);
  if (!D.n_recent) return;
  if (A.steps.size() == 1) {  // projection, in chunks of at most opt_max_cand rows
    PStep P = A.packed.steps[0];
    const int kb = D.views[0].lay.key64 ? 8 : 4;
    for (u64 rb = 0; rb < D.n_recent; rb += e.opt_max_cand) {
      const u64 sub = std::min(e.opt_max_cand, D.n_recent - rb);
      if (H.n_cand + sub > e.opt_max_cand) flush_candidates(e, H);
      ensure_cand(e, H, sub);
      P.in_words = static_cast<const char*>(D.rkeys.p) + rb * kb;
      P.in_tags = sb ? static_cast<const char*>(D.rtags.p) + rb * sb : nullptr;
      P.n_in = sub;
      P.out_words = H.ckeys.p;
      P.out_tags = H.ctags.p;
      P.out_base = H.n_cand;
      pjoin_project(sem, P, e.stream);
      e.after_launch("project");
      e.launches++;
      H.n_cand += sub;
      H.cand_iter += sub;
      H.unfiltered = true;
      e.cand_emitted += sub;
    }
    return;
  }
  if (A.packed.cross_ok && e.opt_cross_join && e.opt_warp_join && H.extract) {
    // both probes keyed by the delta row: one pass over the products
    const StepPlan& S1 = A.steps[1];
    const StepPlan& S2 = A.steps[2];
    RelSt& V1 = e.rels[R.body[S1.atom].rel];
    RelSt& V2 = e.rels[R.body[S2.atom].rel];
    ViewSt& W1 = V1.views[S1.view];
    ViewSt& W2 = V2.views[S2.view];
    if (W1.stale) rebuild_view(e, V1, W1);
    if (W2.stale) rebuild_view(e, V2, W2);
    if (W1.n < (1ull << 27) && W2.n < (1ull << 27)) {
      if (!W1.n || !W2.n) return;
      ensure_index(e, W1, S1.prefix_len);
      ensure_index(e, W2, S2.prefix_len);
      PStep PA = A.packed.steps[0];
      PA.in_words = D.rkeys.p;
      PA.in_tags = nullptr;
      PA.n_in = D.n_recent;
      PA.v_keys = W1.keys.p;
      PA.v_key64 = W1.lay.key64;
      PA.v_n = W1.n;
      PA.v_stamp_mode = STAMP_NONE;
      PA.index_mode = W1.index[S1.prefix_len].mode;
      PA.dense_offs = W1.index[S1.prefix_len].offs.as<u64>();
      PA.hash_bits = W1.index[S1.prefix_len].hash_bits;
      PStep PB = A.packed.cross;
      PB.v_keys = W2.keys.p;
      PB.v_key64 = W2.lay.key64;
      PB.v_n = W2.n;
      PB.index_mode = W2.index[S2.prefix_len].mode;
      PB.dense_offs = W2.index[S2.prefix_len].offs.as<u64>();
      PB.hash_bits = W2.index[S2.prefix_len].hash_bits;
      PB.bitmap = H.bitmap.as<u32>();
      H.touched = true;
      const u64 before = g_prof ? e.read_u64(e.counts.as<u64>() + 13) : 0;
      pjoin_warp_cross_bitmap(PA, PB, e.counts.as<u64>() + 13, e.stream);
      e.after_launch("join emit");
      e.launches++;
      if (g_prof) {
        const u64 outs = e.read_u64(e.counts.as<u64>() + 13) - before;
        g_prof->add_last_bytes(outs * ((W1.lay.key64 ? 8.0 : 4.0) + (W2.lay.key64 ? 8.0 : 4.0) + 4.0));
      }
      return;
    }
  }
  const void* in_words = D.rkeys.p;
  const void* in_tags = D.rtags.p;
  u64 n_in = D.n_recent;
  int side = 0;
  for (size_t s = 1; s < A.steps.size(); s++) {
    const StepPlan& S = A.steps[s];
    const bool last = s + 1 == A.steps.size();
    RelSt& V = e.rels[R.body[S.atom].rel];
    ViewSt& W = V.views[S.view];
    if (W.stale) rebuild_view(e, V, W);
    if (!W.n) return;
    ensure_index(e, W, S.prefix_len);
    PStep P = A.packed.steps[s - 1];
    P.in_words = in_words;
    P.in_tags = in_tags;
    P.n_in = n_in;
    P.v_keys = W.keys.p;
    P.v_key64 = W.lay.key64;
    P.v_tags = W.tags.p;
    P.v_stamp = W.stamps.as<u32>();
    P.v_n = W.n;
    P.v_stamp_mode = S.probe_old ? STAMP_LT : STAMP_NONE;
    P.v_stamp_val = k - 1;
    const IndexSt& I = W.index[S.prefix_len];
    P.index_mode = I.mode;
    P.dense_offs = I.offs.as<u64>();
    P.hash_bits = I.hash_bits;
    // unit semiring: warp-balanced steps.  Views below 2^27 rows keep a 32-row
    // group's outputs, and views below 2^22 rows a 1024-row block's outputs,
    // under 2^32.
    const bool warp = e.opt_warp_join && pjoin_warp_supported(sem, P) && W.n < (1ull << 27);
    if (last && warp && H.extract) {  // one pass: probe, expand, set bits
      H.touched = true;
      P.out_words = nullptr;
      P.bitmap = H.bitmap.as<u32>();
      const u64 before = g_prof ? e.read_u64(e.counts.as<u64>() + 13) : 0;
      pjoin_warp_bitmap(P, e.counts.as<u64>() + 13, e.stream);
      e.after_launch("join emit");
      e.launches++;
      if (g_prof) {
        const u64 outs = e.read_u64(e.counts.as<u64>() + 13) - before;
        g_prof->add_last_bytes(outs * ((P.v_key64 ? 8.0 : 4.0) + 4.0));
      }
      return;
    }
    if (!last && warp && e.opt_warp_join == 1 && W.n < (1ull << 22)) {  // binding words placed per block of input rows
      const u64 n_blk = pjoin_warp_blocks(n_in);
      e.ensure(e.off, n_blk * 16);
      pjoin_warp_count(P, e.off.as<u64>() + n_blk, e.stream);
      e.after_launch("join count");
      scratch_at_least(e, scan_scratch_elems(n_blk) * 8 + 64);
      {
        ProfScope ps("join_scan", n_blk * 16.0, e.stream);
        exclusive_scan<u64, u64>(e.off.as<u64>() + n_blk, e.off.as<u64>(), n_blk, e.counts.as<u64>(), e.scratch.as<u64>(),
                                 e.stream);
      }
      e.after_launch("join scan");
      e.launches += 1 + scan_launches(n_blk);
      const u64 total = e.read_u64(e.counts.as<u64>());
      if (!total) return;
      const int out_side = side ^ 1;
      const int wb = P.out_w64 ? 8 : 4;
      e.ensure(e.bind[out_side][0], total * wb);
      P.out_words = e.bind[out_side][0].p;
      P.out_tags = nullptr;
      P.out_base = 0;
      pjoin_warp_emit(P, total, e.off.as<u64>(), e.stream);
      e.after_launch("join emit");
      e.launches++;
      side = out_side;
      in_words = e.bind[side][0].p;
      in_tags = nullptr;
      n_in = total;
      continue;
    }
    const u64 n_blk = pjoin_loc_blocks(n_in);
    e.ensure(e.cnt, n_in * 4);
    e.ensure(e.lo, n_in * 4);
    e.ensure(e.off, n_blk * 16);
    P.loc = e.cnt.as<u32>();
    P.lo32 = e.lo.as<u32>();
    P.blk_cnt = e.off.as<u64>() + n_blk;
    P.blk_off = e.off.as<u64>();
    P.err = reinterpret_cast<u32*>(e.counts.as<u64>() + 1);
    if (W.n > 0xFFFFFFFFull) throw LobError(LOB_E_ARG, "packed join needs views below 2^32 rows");
    e.check(cudaMemsetAsync(P.err, 0, sizeof(u64), e.stream), "join error word");
    pjoin_count(sem, P, e.stream);
    e.after_launch("join count");
    scratch_at_least(e, scan_scratch_elems(n_blk) * 8 + 64);
    {
      ProfScope ps("join_scan", n_blk * 16.0, e.stream);
      exclusive_scan<u64, u64>(P.blk_cnt, e.off.as<u64>(), n_blk, e.counts.as<u64>(), e.scratch.as<u64>(), e.stream);
    }
    e.after_launch("join scan");
    e.launches += 1 + scan_launches(n_blk);
    e.check(cudaMemcpyAsync(e.pinned, e.counts.as<u64>(), 16, cudaMemcpyDeviceToHost, e.stream), "join total");
    e.sync();
    if (e.pinned[1] & kErrLocOverflow)
      throw LobError(LOB_E_ARG, "join step: 1024 consecutive input rows have 2^32 or more matches");
    const u64 total = e.pinned[0];
    if (!total) return;
    note_loop_cap(e, "tiles", (total + kEmitTile - 1) / kEmitTile);
    if (!last) note_loop_cap(e, "bind", total);
    if (last && H.extract) {  // new facts only set their bits in the membership bitmap
      H.touched = true;
      P.out_words = nullptr;
      P.out_tags = nullptr;
      P.out_base = 0;
      P.out_count = nullptr;
      P.bitmap = H.bitmap.as<u32>();
      for (u64 jb = 0; jb < total; jb += e.opt_max_cand) {
        const u64 sub = std::min(e.opt_max_cand, total - jb);
        const u64 nt = (sub + kEmitTile - 1) / kEmitTile;
        e.ensure(e.part, (nt + 1) * 8);
        P.total = sub;
        P.j_begin = jb;
        pjoin_partition(P, nt, e.part.as<u64>(), e.stream);
        pjoin_emit(sem, P, e.part.as<u64>(), e.stream);
        e.after_launch("join emit");
        e.launches += 2;
        H.cand_iter += sub;
        e.cand_emitted += sub;
      }
      return;
    }
    if (last && H.dense) {  // outputs (+)-added into the head's dense accumulator
      H.touched = true;
      P.out_words = nullptr;
      P.out_tags = nullptr;
      P.out_base = 0;
      P.out_count = nullptr;
      P.bitmap = H.dtouched.as<u32>();
      P.acc = H.dacc.p;
      for (u64 jb = 0; jb < total; jb += e.opt_max_cand) {
        const u64 sub = std::min(e.opt_max_cand, total - jb);
        const u64 nt = (sub + kEmitTile - 1) / kEmitTile;
        e.ensure(e.part, (nt + 1) * 8);
        P.total = sub;
        P.j_begin = jb;
        pjoin_partition(P, nt, e.part.as<u64>(), e.stream);
        pjoin_emit(sem, P, e.part.as<u64>(), e.stream);
        e.after_launch("join emit");
        e.launches += 2;
        H.cand_iter += sub;
        e.cand_emitted += sub;
      }
      return;
    }
    if (last) {  // candidates, in sub-ranges of at most opt_max_cand outputs
      for (u64 jb = 0; jb < total; jb += e.opt_max_cand) {
        const u64 sub = std::min(e.opt_max_cand, total - jb);
        if (H.n_cand + sub > e.opt_max_cand) flush_candidates(e, H);
        ensure_cand(e, H, sub);
        P.out_words = H.ckeys.p;
        P.out_tags = H.ctags.p;
        P.out_base = H.n_cand;
        const u64 nt = (sub + kEmitTile - 1) / kEmitTile;
        e.ensure(e.part, (nt + 1) * 8);
        P.total = sub;
        P.j_begin = jb;
        pjoin_partition(P, nt, e.part.as<u64>(), e.stream);
        P.bitmap = nullptr;
        P.out_count = nullptr;
        if (H.filter_on) {
          P.bitmap = H.bitmap.as<u32>();
          P.out_count = e.counts.as<u64>() + 14;
          e.check(cudaMemsetAsync(P.out_count, 0, sizeof(u64), e.stream), "filter count");
        }
        pjoin_emit(sem, P, e.part.as<u64>(), e.stream);
        e.after_launch("join emit");
        e.launches += 2;
        const u64 written = H.filter_on ? e.read_u64(e.counts.as<u64>() + 14) : sub;
        H.n_cand += written;
        H.cand_iter += sub;
        e.cand_emitted += sub;
      }
      return;
    }
    const int out_side = side ^ 1;
    const int wb = P.out_w64 ? 8 : 4;
    e.ensure(e.bind[out_side][0], total * wb);
    if (cb) e.ensure(e.bind[out_side][kMaxSlots + 1], total * cb);
    P.out_words = e.bind[out_side][0].p;
    P.out_tags = e.bind[out_side][kMaxSlots + 1].p;
    P.out_base = 0;
    const u64 ntiles = (total + kEmitTile - 1) / kEmitTile;
    e.ensure(e.part, (ntiles + 1) * 8);
    P.total = total;
    P.j_begin = 0;
    pjoin_partition(P, ntiles, e.part.as<u64>(), e.stream);
    pjoin_emit(sem, P, e.part.as<u64>(), e.stream);
    e.after_launch("join emit");
    e.launches += 2;
    side = out_side;
    in_words = e.bind[side][0].p;
    in_tags = e.bind[side][kMaxSlots + 1].p;
    n_in = total;
  }
}

// sort + unique + difference/merge of one head relation's candidates
static void dedup_sorted(lob_engine& e, RelSt& H, u32 k);
static void merge_unique(lob_engine& e, RelSt& H, u32 k, const void* ukeys, const void* utags, u64 nu);
static u64 bitmap_bits(const RelSt& H) { return 1ull << H.views[0].lay.bits; }

// The primary view's keys, read out of a membership bitmap (sorted).
static void materialize_keys(lob_engine& e, RelSt& H, const u32* bits) {
  ViewSt& V = H.views[0];
  const int kb = V.lay.key64 ? 8 : 4;
  scratch_at_least(e, bits_scratch_bytes(bitmap_bits(H)));
  e.launches += bits_count(bits, nullptr, bitmap_bits(H), e.scratch.p, e.counts.as<u64>() + 1, e.stream);
  e.after_launch("bitmap count");
  const u64 n = e.read_u64(e.counts.as<u64>() + 1);
  if (n != V.n) throw LobError(LOB_E_CUDA, "internal error: membership bitmap and relation size disagree");
  e.ensure(V.keys, n * kb);
  bits_extract(bits, nullptr, bitmap_bits(H), V.lay.key64, V.keys.p, n, e.scratch.p, e.stream);
  e.after_launch("bitmap extract");
  e.launches++;
  H.keys_stale = false;
  for (auto& kv : V.index) kv.second.valid = false;
}

// A relation that no arm probes after iteration 1 (arms whose delta is an
// input relation run in iteration 1 only, before the first dedup).
static bool probed_after_first(const RelSt& H) {
  for (const ViewSt& W : H.views)
    if (W.probed_late) return true;
  return false;
}

// Bitmap delta mode: this iteration's new facts are the bits set in the
// membership bitmap but not in its start-of-iteration copy, read out in key
// order; candidates written by other kernels (projections, general joins) only
// add their bits first.  The full relation's keys are merged only when some arm
// probes it later; otherwise they stay in the bitmap until the fixpoint.
static void dedup_bitmap_delta(lob_engine& e, RelSt& H, u32 k) {
  ViewSt& V = H.views[0];
  const Layout& L = V.lay;
  const int kb = L.key64 ? 8 : 4;
  const u64 n = H.n_cand;
  H.unfiltered = false;
  H.flushed = false;
  if (n) bitmap_set_keys(H.ckeys.p, L.key64, n, H.bitmap.as<u32>(), e.stream);
  e.launches += n ? 1 : 0;
  H.n_cand = 0;
  if (!n && !H.touched) {
    H.last_new = 0;
    return;
  }
  scratch_at_least(e, bits_scratch_bytes(bitmap_bits(H)));
  e.launches += bits_count(H.bitmap.as<u32>(), H.prev_bitmap.as<u32>(), bitmap_bits(H), e.scratch.p,
                           e.counts.as<u64>() + 1, e.stream);
  e.after_launch("bitmap count");
  const u64 nr = e.read_u64(e.counts.as<u64>() + 1);
  H.last_new = nr;
  if (!nr) return;
  e.ensure(H.nkeys, nr * kb);
  bits_extract(H.bitmap.as<u32>(), H.prev_bitmap.as<u32>(), bitmap_bits(H), L.key64, H.nkeys.p, nr, e.scratch.p,
               e.stream);
  e.after_launch("bitmap extract");
  e.launches++;
  H.n_next = nr;
  if (probed_after_first(H)) {
    e.ensure(V.keys2, (V.n + nr) * kb);
    scratch_at_least(e, merge_nodup_scratch_bytes(V.n, nr));
    merge_nodup(L.key64, V.keys.p, V.n, H.nkeys.p, nr, V.keys2.p, e.scratch.p, e.stream);
    e.after_launch("merge");
    e.launches++;
    std::swap(V.keys, V.keys2);
  } else {
    H.keys_stale = true;
  }
  V.n += nr;
  for (auto& kv : V.index) kv.second.valid = false;
  update_secondary_views(e, H, k, nr);
}

// Dense accumulation: the iteration's unique candidates, already (+)-reduced,
// are the touched slots read out in key order; then the usual difference+merge.
static void dedup_dense(lob_engine& e, RelSt& H, u32 k) {
  if (H.n_cand) flush_candidates(e, H);
  H.unfiltered = false;
  H.flushed = false;
  if (!H.touched) {
    H.last_new = 0;
    return;
  }
  H.touched = false;
  const int ks = sem_kernel(e.semiring);
  const Layout& L = H.views[0].lay;
  const int kb = L.key64 ? 8 : 4, cb = cand_bytes(e.semiring);
  const u64 nbits = 1ull << L.bits;
  scratch_at_least(e, bits_scratch_bytes(nbits));
  e.launches += bits_count(H.dtouched.as<u32>(), nullptr, nbits, e.scratch.p, e.counts.as<u64>() + 1, e.stream);
  e.after_launch("dense count");
  const u64 nu = e.read_u64(e.counts.as<u64>() + 1);
  note_loop_cap(e, "u" + std::to_string(&H - &e.rels[0]), nu);
  if (!nu) {
    H.last_new = 0;
    return;
  }
  e.ensure(H.akeys, nu * kb);
  e.ensure(H.atags, nu * cb);
  dense_extract(ks, L.key64, H.dtouched.as<u32>(), H.dacc.p, nbits, H.akeys.p, H.atags.p, nu, e.scratch.p, e.stream);
  e.after_launch("dense extract");
  e.launches++;
  merge_unique(e, H, k, H.akeys.p, H.atags.p, nu);
}

static void dedup_relation(lob_engine& e, RelSt& H, u32 k) {
  H.n_next = 0;
  H.last_cand = H.cand_iter;
  H.cand_iter = 0;
  if (H.dense) {
    dedup_dense(e, H, k);
    return;
  }
  if (H.extract) {
    dedup_bitmap_delta(e, H, k);
    return;
  }
  // sorted-candidate path: the keys must be materialised, and the start-of-
  // iteration bitmap copy (when kept) follows the bitmap at the end
  if (H.keys_stale) materialize_keys(e, H, H.prev_bitmap.as<u32>());
  dedup_sorted(e, H, k);
  if (H.prev_bitmap.p && H.n_next) {
    bitmap_set_keys(H.nkeys.p, H.views[0].lay.key64, H.n_next, H.prev_bitmap.as<u32>(), e.stream);
    e.after_launch("bitmap");
    e.launches++;
  }
}

static void dedup_sorted(lob_engine& e, RelSt& H, u32 k) {
  const u64 n = H.n_cand;
  if (!n && !H.flushed) {
    H.last_new = 0;
    H.unfiltered = false;
    return;
  }
  const int sem = e.semiring;
  const int ks = sem_kernel(sem);
  ViewSt& V = H.views[0];
  const Layout& L = V.lay;
  const int kb = L.key64 ? 8 : 4, cb = cand_bytes(sem), sb = stored_bytes(sem);
  const bool stamps = sem_stamps(sem);
  const bool fast = H.filter_on && !H.flushed && !H.unfiltered;
  H.unfiltered = false;
  if (fast) {
    // every candidate is distinct and absent from F (membership filter at
    // emission): sort them, merge into F, and they are the next recent set
    e.ensure(H.ckeys2, n * kb);
    void* keys = H.ckeys.p;
    void* none = nullptr;
    engine_sort(e, L.key64, 0, &keys, &none, H.ckeys2.p, nullptr, n, L.bits);
    e.after_launch("candidate sort");
      e.ensure(V.keys2, (V.n + n) * kb);
    scratch_at_least(e, merge_nodup_scratch_bytes(V.n, n));
    merge_nodup(L.key64, V.keys.p, V.n, keys, n, V.keys2.p, e.scratch.p, e.stream);
    e.after_launch("merge");
    e.launches += 2;
    V.n += n;
    std::swap(V.keys, V.keys2);
    for (auto& kv : V.index) kv.second.valid = false;
    if (keys == H.ckeys.p) std::swap(H.nkeys, H.ckeys);
    else std::swap(H.nkeys, H.ckeys2);
    H.n_next = n;
    H.last_new = n;
    update_secondary_views(e, H, k, n);
    return;
  }
  void* ukeys;
  void* utags;
  u64 nu;
  if (H.flushed) {  // earlier chunks of this iteration were accumulated: add the rest
    flush_candidates(e, H);
    ukeys = H.akeys.p;
    utags = H.atags.p;
    nu = H.n_acc;
    H.n_acc = 0;
    H.flushed = false;
  } else {
    if (n > e.opt_max_cand || n >= (1ull << 32)) throw LobError(LOB_E_CUDA, "internal error: candidate set too large");
    e.ensure(H.ckeys2, n * kb);
    if (cb) e.ensure(H.ctags2, n * cb);
    void* keys = H.ckeys.p;
    void* tags = H.ctags.p;
    engine_sort(e, L.key64, cb, &keys, &tags, H.ckeys2.p, H.ctags2.p, n, L.bits);
    e.after_launch("candidate sort");
      ukeys = keys == H.ckeys.p ? H.ckeys2.p : H.ckeys.p;
    utags = tags == H.ctags.p ? H.ctags2.p : H.ctags.p;
    scratch_at_least(e, unique_scratch_bytes(n));
    unique_run(ks, L.key64, keys, tags, n, ukeys, utags, e.counts.as<u64>() + 1, e.scratch.p, e.stream);
    e.after_launch("unique");
    e.launches += 2 + scan_launches((n + 4095) / 4096);
    nu = e.read_u64(e.counts.as<u64>() + 1);
  }
  merge_unique(e, H, k, ukeys, utags, nu);
}

// Difference of the iteration's unique candidates U (sorted keys, candidate
// tags) against F, fused with their merge into F; the new (or improved) facts
// become the next recent set and reach the secondary views.
static void merge_unique(lob_engine& e, RelSt& H, u32 k, const void* ukeys, const void* utags, u64 nu) {
  if (!nu) return;
  const int sem = e.semiring;
  const int ks = sem_kernel(sem);
  ViewSt& V = H.views[0];
  const Layout& L = V.lay;
  const int kb = L.key64 ? 8 : 4, sb = stored_bytes(sem);
  const bool stamps = sem_stamps(sem);
  // difference against F fused with the merge into F
  e.ensure(V.keys2, (V.n + nu) * kb);
  if (sb) e.ensure(V.tags2, (V.n + nu) * sb);
  if (stamps) e.ensure(V.stamps2, (V.n + nu) * 4);
  e.ensure(H.nkeys, nu * kb);
  if (sb) e.ensure(H.ntags, nu * sb);
  MergeArgs M{};
  M.sem = ks;
  M.key64 = L.key64;
  M.fkeys = V.keys.p; M.ftags = V.tags.p; M.fstamp = stamps ? V.stamps.as<u32>() : nullptr; M.nf = V.n;
  M.ukeys = ukeys; M.utags = utags; M.nu = nu; M.u_stored = 0;
  M.okeys = V.keys2.p; M.otags = V.tags2.p; M.ostamp = stamps ? V.stamps2.as<u32>() : nullptr;
  M.rkeys = H.nkeys.p; M.rtags = H.ntags.p;
  M.stamp = k;
  M.counts_dev = e.counts.as<u64>() + 2;
  scratch_at_least(e, merge_scratch_bytes(V.n, nu));
  diff_merge(M, e.scratch.p, e.stream);
  e.after_launch("difference+merge");
  const u64 mt = (V.n + nu + 2047) / 2048;
  e.launches += 3 + 2 * scan_launches(mt);
  e.check(cudaMemcpyAsync(e.pinned, e.counts.as<u64>() + 2, 24, cudaMemcpyDeviceToHost, e.stream), "counts");
  e.sync();
  if (e.pinned[2]) throw LobError(LOB_E_CUDA, "internal error: unsorted input to the difference/merge");
  const u64 dups = e.pinned[0], nr = e.pinned[1];
  V.n = V.n + nu - dups;
  if (H.dense) {
    note_loop_cap(e, "full" + std::to_string(&H - &e.rels[0]), V.n);
    note_loop_cap(e, "r" + std::to_string(&H - &e.rels[0]), nr);
  }
  std::swap(V.keys, V.keys2);
  std::swap(V.tags, V.tags2);
  std::swap(V.stamps, V.stamps2);
  for (auto& kv : V.index) kv.second.valid = false;
  H.n_next = nr;
  H.last_new = nr;
  if (H.filter_on && nr) {  // keep the membership bitmap equal to F
    bitmap_set_keys(H.nkeys.p, L.key64, nr, H.bitmap.as<u32>(), e.stream);
    e.after_launch("bitmap");
    e.launches++;
  }
  update_secondary_views(e, H, k, nr);
}

// Unit semiring: keep a membership bitmap of the relation and drop known facts
// and repeated candidates at emission -- from the first iteration when the key
// has at most 32 bits (bitmap <= 512 MB), and for keys of up to 34 bits (2 GB)
// once most of the previous iteration's candidates were duplicates.
static void maybe_enable_filter(lob_engine& e, RelSt& r) {
  if (r.filter_on || e.semiring != SR_UNIT || !e.opt_emit_filter || !r.idb) return;
  const Layout& L = r.views[0].lay;
  if (L.bits > 34) return;
  if (e.opt_emit_filter == 1 && L.bits > 32 && (r.last_cand < (1ull << 20) || r.last_new * 2 > r.last_cand)) return;
  const u64 words = ((1ull << L.bits) + 31) / 32;
  e.ensure(r.bitmap, words * 4);
  e.check(cudaMemsetAsync(r.bitmap.p, 0, words * 4, e.stream), "bitmap");
  bitmap_set_keys(r.views[0].keys.p, L.key64, r.views[0].n, r.bitmap.as<u32>(), e.stream);
  e.after_launch("bitmap");
  e.launches++;
  r.filter_on = true;
  if (e.opt_bitmap_delta) {
    e.ensure(r.prev_bitmap, words * 4);
    e.check(cudaMemcpyAsync(r.prev_bitmap.p, r.bitmap.p, words * 4, cudaMemcpyDeviceToDevice, e.stream), "bitmap copy");
  }
}

// Bitmap delta mode for this iteration when its predicted traffic is lower.
// Bitmap delta: both bitmaps read twice and the copy written (about 2.5 bitmap
// sizes).  Sorted candidates: about 64 bytes of sort work per new fact (the
// last iteration's count as the prediction), plus reading the keys out of the
// bitmap first when they are not materialised.  Both merge the new facts into
// the full relation's keys (a read and a write of them) when a later arm probes
// it; only the sorted path merges them otherwise.
static void choose_dedup_mode(lob_engine& e, RelSt& r) {
  r.touched = false;
  r.extract = false;
  if (!r.filter_on || !r.prev_bitmap.p) return;
  if (e.opt_bitmap_delta != 1) {
    r.extract = e.opt_bitmap_delta == 2;
    return;
  }
  const double bitmap_bytes = (double)(bitmap_bits(r) / 8);
  const double kb = r.views[0].lay.key64 ? 8.0 : 4.0;
  const double merge = 2.0 * kb * (double)r.views[0].n;
  const double delta_cost = 2.5 * bitmap_bytes + (probed_after_first(r) ? merge : 0.0);
  const double sorted_cost = 64.0 * (double)r.last_new + merge +
                             (r.keys_stale ? bitmap_bytes + kb * (double)r.views[0].n : 0.0);
  r.extract = delta_cost <= sorted_cost;
}

// Dense (+)-accumulation for every derived relation of a tagged run whose key
// space has at most opt_acc_bits bits (accumulator: 2^bits candidate tags).
static void enable_dense(lob_engine& e) {
  if (!e.opt_acc_dense || e.semiring == SR_UNIT || sem_top1(e.semiring)) return;
  const int cb = dense_cand_bytes(sem_kernel(e.semiring));
  for (auto& r : e.rels) {
    const Layout& L = r.views[0].lay;
    if (!r.idb || L.bits > e.opt_acc_bits) continue;
    const u64 slots = 1ull << L.bits;
    const u64 bm_bytes = std::max<u64>(16, slots / 8);
    e.ensure(r.dacc, slots * cb);
    e.ensure(r.dtouched, bm_bytes);
    e.check(cudaMemsetAsync(r.dacc.p, 0, slots * cb, e.stream), "dense accumulator");
    e.check(cudaMemsetAsync(r.dtouched.p, 0, bm_bytes, e.stream), "dense bitmap");
    r.dense = true;
    r.touched = false;
  }
}

// Start of a stratum after the first: the recent set of every relation is the
// whole relation (its primary view's keys and tags).
static void all_recent(lob_engine& e) {
  const int sb = stored_bytes(e.semiring);
  for (auto& r : e.rels) {
    ViewSt& V = r.views[0];
    if (r.keys_stale) throw LobError(LOB_E_STATE, "internal error: stratum start without materialised keys");
    r.n_recent = V.n;
    if (!V.n) continue;
    const int kb = V.lay.key64 ? 8 : 4;
    e.ensure(r.rkeys, V.n * kb);
    e.check(cudaMemcpyAsync(r.rkeys.p, V.keys.p, V.n * kb, cudaMemcpyDeviceToDevice, e.stream), "recent keys");
    if (sb) {
      e.ensure(r.rtags, V.n * sb);
      e.check(cudaMemcpyAsync(r.rtags.p, V.tags.p, V.n * sb, cudaMemcpyDeviceToDevice, e.stream), "recent tags");
    }
  }
}

static int run_fixpoint(lob_engine& e, int sem, u32 max_iters, lob_stats* st) {
  if (e.state != 0) throw LobError(LOB_E_STATE, "run_to_fixpoint was already called; call lob_reset first");
  if (sem < 0 || sem > 6) throw LobError(LOB_E_ARG, "unknown semiring id");
  e.peak_bytes = e.live_bytes;
  e.launches = 0;
  const u64 syncs0 = e.host_syncs;
  struct RunEvents {  // destroyed on every exit, the error paths included
    cudaEvent_t a = nullptr, b = nullptr;
    ~RunEvents() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  e.check(cudaEventCreate(&ev.a), "event");
  e.check(cudaEventCreate(&ev.b), "event");
  cudaEvent_t ev0 = ev.a, ev1 = ev.b;
  e.check(cudaEventRecord(ev0, e.stream), "event");
  prepare(e, sem);
  load_facts(e);
  enable_dense(e);
  lob_stats s{};
  s.semiring = (u32)sem;
  int rc = LOB_OK;
  u32 k = 0;
  e.iter_counts.clear();
  e.cand_emitted = 0;
  e.check(cudaMemsetAsync(sort_err(e), 0, sizeof(u32), e.stream), "sort error word");
  e.check(cudaMemsetAsync(e.counts.as<u64>() + 13, 0, sizeof(u64), e.stream), "emitted counter");
  e.stratum_begin.clear();
  int stratum = 0;  // the stratum being run (assign_strata)
  for (;;) {
    if (k >= max_iters) { rc = LOB_E_MAXITER; break; }
    k++;
    e.iter_counts.emplace_back();
    for (auto& r : e.rels) e.iter_counts.back().emplace_back(r.views[0].n, r.n_recent);
    for (auto& r : e.rels) maybe_enable_filter(e, r);
    for (auto& r : e.rels) choose_dedup_mode(e, r);
    for (auto& r : e.rels) r.n_cand = 0;
    for (auto& p : e.plans) {
      if (p.stratum != stratum) continue;
      for (auto& A : p.arms) {
        if (!e.rels[p.ast.body[A.delta].rel].n_recent) continue;
        bool skip = false;  // an atom before the delta atom has no old facts
        for (u32 b : A.before_rels) {
          const RelSt& br = e.rels[b];
          if (br.views[0].n == br.n_recent) { skip = true; break; }
        }
        if (skip) continue;
        if (A.packed.ok) run_arm_packed(e, p, A, k);
        else run_arm(e, p, A, k);
      }
    }
    u64 total_new = 0;
    for (auto& r : e.rels) {
      dedup_relation(e, r, k);
      total_new += r.n_next;
    }
    for (auto& r : e.rels) {
      std::swap(r.rkeys, r.nkeys);
      std::swap(r.rtags, r.ntags);
      r.n_recent = r.n_next;
      r.n_next = 0;
    }
    s.new_facts += total_new;
    if (!total_new) {
      if (stratum + 1 >= e.n_strata) break;
      // the next stratum starts as Algorithm 1 starts one: every fact of the
      // database is recent, so its first iteration joins over all of them
      stratum++;
      all_recent(e);
      e.stratum_begin.push_back(k + 1);
      continue;
    }
    if (k == 1 && e.n_strata == 1) {  // the rest of the run as a device-driven graph, when it qualifies
      bool taken = false;
      const int r2 = run_device_loop(e, k, max_iters, s, &taken);
      if (taken) {
        rc = r2;
        break;
      }
    }
  }
  for (auto& r : e.rels)
    if (r.keys_stale) materialize_keys(e, r, r.bitmap.as<u32>());
  e.cand_emitted += e.read_u64(e.counts.as<u64>() + 13);  // outputs of bitmap-only warp steps
  e.check(cudaEventRecord(ev1, e.stream), "event");
  e.sync();
  e.prof.flush();
  if (e.read_u64(e.counts.as<u64>() + 15) & 0xFFFFFFFFull)
    throw LobError(LOB_E_TIMEOUT, "a bounded device wait of the sort gave up; the run's results are invalid");
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  s.iterations = k;
  s.ms = ms;
  s.candidates = e.cand_emitted;
  for (auto& r : e.rels)
    if (r.idb) s.derived += r.views[0].n;
  s.peak_bytes = e.peak_bytes;
  s.kernel_launches = e.launches;
  s.host_syncs = e.host_syncs - syncs0;
  s.proof_words = e.arena_tail;
  s.strata = (u32)e.n_strata;
  e.stats = s;
  e.last_iter = k;
  e.state = 1;
  e.ran_diff = sem == SR_DIFF_MAX_MIN || sem == SR_DIFF_ADD_MULT || sem == SR_DIFF_TOP1;
  if (st) *st = s;
  return rc;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
template <class F>
static int guarded(lob_engine* e, F&& f) {
  if (!e) return LOB_E_ARG;
  struct ProfOn {
    explicit ProfOn(lob_engine* e) { g_prof = e->opt_profile ? &e->prof : nullptr; }
    ~ProfOn() { g_prof = nullptr; }
  } on(e);
  try {
    e->err.clear();
    cudaSetDevice(e->device);
    return f();
  } catch (const LobError& x) {
    e->err = x.what();
    return x.code;
  } catch (const std::exception& x) {
    e->err = x.what();
    return LOB_E_ARG;
  }
}

extern "C" {

int lob_create(lob_engine** out, const lob_alloc* alloc, void* cuda_stream) {
  g_create_err.clear();
  if (!out) return LOB_E_ARG;
  *out = nullptr;
  lob_engine* e = new lob_engine();
  if (cudaGetDevice(&e->device) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "no CUDA device";
    delete e;
    return LOB_E_CUDA;
  }
  e->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (alloc) {
    if (!alloc->alloc || !alloc->release) {
      g_create_err = "allocator needs both alloc and release";
      delete e;
      return LOB_E_ARG;
    }
    e->alloc = *alloc;
    e->custom_alloc = true;
  }
  if (!e->custom_alloc) {
    // Sec. 4.1 (buffer reuse): an engine-owned pool whose release threshold
    // keeps freed blocks reserved, so repeated runs do not map memory again.
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = e->device;
    uint64_t keep = ~0ull;
    if (cudaMemPoolCreate(&e->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(e->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      g_create_err = "cudaMemPoolCreate failed";
      if (e->pool) cudaMemPoolDestroy(e->pool);
      delete e;
      return LOB_E_CUDA;
    }
  }
  if (cudaMallocHost(&e->pinned, 64 * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "pinned host allocation failed";
    if (e->pool) cudaMemPoolDestroy(e->pool);
    delete e;
    return LOB_E_CUDA;
  }
  int rc = guarded(e, [&] {
    // status and count words: every flag a kernel may set starts cleared, so a
    // flag read back reports the call that set it, never an allocator's leftovers
    e->ensure(e->counts, 64 * sizeof(u64) + 256);
    e->check(cudaMemsetAsync(e->counts.p, 0, e->counts.cap, e->stream), "clear status words");
    e->sync();
    return LOB_OK;
  });
  if (rc != LOB_OK) {
    g_create_err = e->err;
    cudaFreeHost(e->pinned);
    if (e->pool) cudaMemPoolDestroy(e->pool);
    delete e;
    return rc;
  }
  *out = e;
  return LOB_OK;
}

void lob_destroy(lob_engine* e) {
  if (!e) return;
  try {
    cudaSetDevice(e->device);
    e->release_all();
    e->release(e->counts);
    cudaStreamSynchronize(e->stream);
  } catch (...) {
  }
  if (e->pool) cudaMemPoolDestroy(e->pool);
  if (e->capture_stream) cudaStreamDestroy(e->capture_stream);
  if (e->capture_stream2) cudaStreamDestroy(e->capture_stream2);
  cudaFreeHost(e->pinned);
  delete e;
}

const char* lob_last_error(const lob_engine* e) { return e ? e->err.c_str() : g_create_err.c_str(); }

int lob_declare_relation(lob_engine* e, const char* name, uint32_t arity, uint32_t* rel_id) {
  return guarded(e, [&] {
    if (!valid_ident(name)) throw LobError(LOB_E_ARG, "invalid relation name");
    if (arity < 1 || arity > (u32)kMaxArity) throw LobError(LOB_E_ARG, "arity must be 1..8");
    if (e->rel_ids.count(name)) throw LobError(LOB_E_ARG, std::string("relation '") + name + "' already declared");
    if (e->state != 0) throw LobError(LOB_E_STATE, "declare before running");
    RelSt r;
    r.name = name;
    r.arity = arity;
    const u32 id = (u32)e->rels.size();
    e->rels.push_back(std::move(r));
    e->rel_ids[name] = id;
    if (rel_id) *rel_id = id;
    return LOB_OK;
  });
}

int lob_relation_id(const lob_engine* ce, const char* name, uint32_t* rel_id) {
  lob_engine* e = const_cast<lob_engine*>(ce);
  return guarded(e, [&] {
    if (!name || !rel_id) throw LobError(LOB_E_ARG, "null argument");
    auto it = e->rel_ids.find(name);
    if (it == e->rel_ids.end()) throw LobError(LOB_E_UNKNOWN_REL, std::string("unknown relation '") + name + "'");
    *rel_id = it->second;
    return LOB_OK;
  });
}

int lob_load_relation(lob_engine* e, uint32_t rel, const uint32_t* cols, const float* tags, const uint32_t* sample_ids,
                      uint64_t n, int mem) {
  return guarded(e, [&] {
    if (rel >= e->rels.size()) throw LobError(LOB_E_UNKNOWN_REL, "unknown relation id");
    if (e->state != 0) throw LobError(LOB_E_STATE, "load before running (or after lob_reset)");
    if (mem != LOB_MEM_HOST && mem != LOB_MEM_DEVICE) throw LobError(LOB_E_ARG, "mem must be LOB_MEM_HOST or LOB_MEM_DEVICE");
    if (!n) return LOB_OK;
    if (!cols) throw LobError(LOB_E_ARG, "null cols");
    RelSt& r = e->rels[rel];
    const cudaMemcpyKind kind = mem == LOB_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const u64 need = r.n_in + n;
    if (r.in_cols.empty()) r.in_cols.resize(1);
    if (need > r.in_cap) {  // re-layout the column-major buffer with a larger stride
      u64 cap = std::max<u64>(need, r.in_cap + r.in_cap / 2);
      DevBuf nb;
      nb.cap = 0;
      e->ensure(nb, cap * r.arity * 4);
      for (u32 c = 0; c < r.arity && r.n_in; c++)
        e->check(cudaMemcpyAsync(nb.as<u32>() + (u64)c * cap, r.in_cols[0].as<u32>() + (u64)c * r.in_cap, r.n_in * 4,
                                 cudaMemcpyDeviceToDevice, e->stream), "grow input");
      e->release(r.in_cols[0]);
      r.in_cols[0] = nb;
      if (r.in_has_tags) e->ensure(r.in_tags, cap * 4, true);
      if (r.in_has_samples) e->ensure(r.in_samples, cap * 4, true);
      r.in_cap = cap;
    }
    for (u32 c = 0; c < r.arity; c++)
      e->check(cudaMemcpyAsync(r.in_cols[0].as<u32>() + (u64)c * r.in_cap + r.n_in, cols + (u64)c * n, n * 4, kind,
                               e->stream), "load columns");
    if (tags && !r.in_has_tags) {
      e->ensure(r.in_tags, r.in_cap * 4);
      if (r.n_in) {  // earlier rows had tag 1
        std::vector<float> ones(r.n_in, 1.0f);
        e->check(cudaMemcpyAsync(r.in_tags.p, ones.data(), r.n_in * 4, cudaMemcpyHostToDevice, e->stream), "tags");
        e->sync();
      }
      r.in_has_tags = true;
    }
    if (r.in_has_tags) {
      if (tags) {
        e->check(cudaMemcpyAsync(r.in_tags.as<float>() + r.n_in, tags, n * 4, kind, e->stream), "load tags");
      } else {
        std::vector<float> ones(n, 1.0f);
        e->check(cudaMemcpyAsync(r.in_tags.as<float>() + r.n_in, ones.data(), n * 4, cudaMemcpyHostToDevice, e->stream),
                 "tags");
        e->sync();
      }
    }
    if (sample_ids && !r.in_has_samples) {
      e->ensure(r.in_samples, r.in_cap * 4);
      if (r.n_in) e->check(cudaMemsetAsync(r.in_samples.p, 0, r.n_in * 4, e->stream), "samples");
      r.in_has_samples = true;
    }
    if (r.in_has_samples) {
      if (sample_ids)
        e->check(cudaMemcpyAsync(r.in_samples.as<u32>() + r.n_in, sample_ids, n * 4, kind, e->stream), "load samples");
      else
        e->check(cudaMemsetAsync(r.in_samples.as<u32>() + r.n_in, 0, n * 4, e->stream), "samples");
    }
    if (mem == LOB_MEM_HOST) e->sync();  // the caller may reuse its host buffers on return
    // values must leave the all-ones code free
    u32* dmax = e->counts.as<u32>() + 32;
    for (u32 c = 0; c < r.arity; c++) {
      reduce_max_u32(r.in_cols[0].as<u32>() + (u64)c * r.in_cap + r.n_in, n, dmax, e->stream);
      e->after_launch("column max");
      if ((u32)(e->read_u64(reinterpret_cast<u64*>(dmax)) & 0xFFFFFFFFull) == 0xFFFFFFFFu)
        throw LobError(LOB_E_ARG, "column value 0xFFFFFFFF is reserved");
    }
    r.n_in += n;
    return LOB_OK;
  });
}

int lob_add_rule(lob_engine* e, const char* text) {
  return guarded(e, [&] {
    if (!text) throw LobError(LOB_E_ARG, "null rule text");
    if (e->state != 0) throw LobError(LOB_E_STATE, "add rules before running (or after lob_reset)");
    e->rules.push_back(parse_rule(*e, text));
    return LOB_OK;
  });
}

int lob_run_to_fixpoint(lob_engine* e, int semiring, uint32_t max_iters, lob_stats* stats) {
  return guarded(e, [&] { return run_fixpoint(*e, semiring, max_iters, stats); });
}

// ---------------------------------------------------------------------------
// autotuner: coordinate descent over strategy options, timed fixpoint runs
// ---------------------------------------------------------------------------
namespace {
struct TuneKnob {
  int* field;
  std::vector<int> values;
  std::function<bool()> active;  // null: always searched
};
}  // namespace

static int autotune(lob_engine& e, int sem, u32 max_iters, u32 repeats, lob_tune_report* rep) {
  if (e.state != 0) throw LobError(LOB_E_STATE, "autotune a loaded engine before lob_run_to_fixpoint");
  if (sem < 0 || sem > 6) throw LobError(LOB_E_ARG, "unknown semiring id");
  if (!repeats) repeats = 1;
  // the hash table's size (Sec. 5.1's load factor) is searched only when the
  // hash index has been kept
  std::vector<TuneKnob> knobs = {{&e.opt_packed_join, {1, 0}, nullptr},
                                 {&e.opt_join_index, {0, 1, 2, 3}, nullptr},
                                 {&e.opt_hash_slots, {2, 4}, [&e] { return e.opt_join_index == 3; }},
                                 {&e.opt_radix_bits, {8, 6}, nullptr}};
  if (sem == SR_UNIT) {
    knobs.push_back({&e.opt_warp_join, {1, 2, 0}});
    knobs.push_back({&e.opt_bitmap_delta, {1, 2, 0}});
    knobs.push_back({&e.opt_emit_filter, {1, 2, 0}});
    knobs.push_back({&e.opt_cross_join, {1, 0}});
  } else {
    knobs.push_back({&e.opt_acc_dense, {1, 0}});
  }
  std::vector<int> saved;
  for (auto& k : knobs) saved.push_back(*k.field);
  u32 trials = 0;
  auto one_run = [&]() -> double {
    lob_stats st{};
    int rc;
    try {
      rc = run_fixpoint(e, sem, max_iters, &st);
    } catch (...) {
      release_derived(e);
      e.state = 0;
      throw;
    }
    release_derived(e);
    e.state = 0;
    e.ran_diff = false;
    if (rc != LOB_OK) throw LobError(rc, "autotune: a trial run did not reach the fixpoint");
    return st.ms;
  };
  auto score = [&]() -> double {
    std::vector<double> ms;
    for (u32 r = 0; r < repeats; r++) {
      ms.push_back(one_run());
      trials++;
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
  };
  try {
    one_run();  // warm-up: first-touch allocations and kernel attributes
    const double first = score();
    double best = first;
    for (auto& k : knobs) {
      if (k.active && !k.active()) continue;
      const int cur = *k.field;
      int keep = cur;
      for (int v : k.values) {
        if (v == cur) continue;
        *k.field = v;
        const double t = score();
        if (t < best * 0.98) {
          best = t;
          keep = v;
        }
      }
      *k.field = keep;
    }
    if (rep) {
      rep->packed_join = e.opt_packed_join;
      rep->warp_join = e.opt_warp_join;
      rep->bitmap_delta = e.opt_bitmap_delta;
      rep->join_index = e.opt_join_index;
      rep->radix_bits = e.opt_radix_bits;
      rep->emit_filter = e.opt_emit_filter;
      rep->acc_dense = e.opt_acc_dense;
      rep->cross_join = e.opt_cross_join;
      rep->hash_slots = e.opt_hash_slots;
      rep->trials = trials;
      rep->first_ms = first;
      rep->best_ms = best;
    }
  } catch (...) {
    for (size_t i = 0; i < knobs.size(); i++) *knobs[i].field = saved[i];
    throw;
  }
  return LOB_OK;
}

int lob_autotune(lob_engine* e, int semiring, uint32_t max_iters, uint32_t repeats, lob_tune_report* report) {
  return guarded(e, [&] { return autotune(*e, semiring, max_iters, repeats, report); });
}

int lob_relation_size(lob_engine* e, uint32_t rel, uint64_t* n) {
  return guarded(e, [&] {
    if (rel >= e->rels.size()) throw LobError(LOB_E_UNKNOWN_REL, "unknown relation id");
    if (!n) throw LobError(LOB_E_ARG, "null n");
    RelSt& r = e->rels[rel];
    *n = e->state == 1 && !r.views.empty() ? r.views[0].n : r.n_in;
    return LOB_OK;
  });
}

// The device address of host range [p, p + bytes) when the whole range is
// page-locked memory mapped into the device's address space (checked at both
// ends, so that it lies in one mapping); nullptr otherwise.
static void* mapped_range(void* p, u64 bytes) {
  if (!p || !bytes) return nullptr;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  char* last = static_cast<char*>(p) + (bytes - 1);
  if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
    return nullptr;
  if (static_cast<char*>(b.devicePointer) - static_cast<char*>(a.devicePointer) != (ptrdiff_t)(bytes - 1)) return nullptr;
  return a.devicePointer;
}

int lob_read_relation(lob_engine* e, uint32_t rel, uint32_t* cols, float* tags, uint32_t* sample_ids, uint64_t capacity,
                      uint64_t* n_out, int mem) {
  return guarded(e, [&] {
    if (rel >= e->rels.size()) throw LobError(LOB_E_UNKNOWN_REL, "unknown relation id");
    if (e->state != 1) throw LobError(LOB_E_STATE, "read after lob_run_to_fixpoint");
    if (mem != LOB_MEM_HOST && mem != LOB_MEM_DEVICE) throw LobError(LOB_E_ARG, "bad mem");
    RelSt& r = e->rels[rel];
    ViewSt& V = r.views[0];
    const u64 n = V.n;
    if (n_out) *n_out = n;
    if (n > capacity) throw LobError(LOB_E_CAPACITY, "capacity " + std::to_string(capacity) + " < " + std::to_string(n));
    if (!n) return LOB_OK;
    if (!cols) throw LobError(LOB_E_ARG, "null cols");
    const int ks = sem_kernel(e->semiring);
    if (mem == LOB_MEM_DEVICE) {
      read_rows(ks, V.lay, V.perm, V.keys.p, V.tags.p, n, cols, capacity, tags, sample_ids, e->stream);
      e->after_launch("read");
      e->sync();
      return LOB_OK;
    }
    // page-locked, mapped host buffers (cudaHostAlloc, cudaHostRegister): the
    // read-out kernel writes them directly over the host link, with no device
    // staging copy
    u32* dc = static_cast<u32*>(mapped_range(cols, (u64)r.arity * capacity * 4));
    float* dt = tags ? static_cast<float*>(mapped_range(tags, n * 4)) : nullptr;
    u32* ds = sample_ids ? static_cast<u32*>(mapped_range(sample_ids, n * 4)) : nullptr;
    if (dc && (!tags || dt) && (!sample_ids || ds)) {
      read_rows(ks, V.lay, V.perm, V.keys.p, V.tags.p, n, dc, capacity, dt, ds, e->stream);
      e->after_launch("read (mapped host)");
      e->sync();
      return LOB_OK;
    }
    DevBuf c, t, s;
    e->ensure(c, n * r.arity * 4);
    if (tags) e->ensure(t, n * 4);
    if (sample_ids) e->ensure(s, n * 4);
    read_rows(ks, V.lay, V.perm, V.keys.p, V.tags.p, n, c.as<u32>(), n, tags ? t.as<float>() : nullptr,
              sample_ids ? s.as<u32>() : nullptr, e->stream);
    e->after_launch("read");
    for (u32 q = 0; q < r.arity; q++)
      e->check(cudaMemcpyAsync(cols + (u64)q * capacity, c.as<u32>() + (u64)q * n, n * 4, cudaMemcpyDeviceToHost, e->stream),
               "read cols");
    if (tags) e->check(cudaMemcpyAsync(tags, t.p, n * 4, cudaMemcpyDeviceToHost, e->stream), "read tags");
    if (sample_ids) e->check(cudaMemcpyAsync(sample_ids, s.p, n * 4, cudaMemcpyDeviceToHost, e->stream), "read samples");
    e->sync();
    e->release(c);
    e->release(t);
    e->release(s);
    return LOB_OK;
  });
}

int lob_read_proofs(lob_engine* e, uint32_t rel, uint32_t* lens, uint32_t* ids, uint64_t id_capacity, uint64_t* n_ids,
                    int mem) {
  return guarded(e, [&] {
    if (rel >= e->rels.size()) throw LobError(LOB_E_UNKNOWN_REL, "unknown relation id");
    if (e->state != 1) throw LobError(LOB_E_STATE, "read after lob_run_to_fixpoint");
    if (!sem_top1(e->semiring)) throw LobError(LOB_E_STATE, "proofs exist after a top-1-proofs run only");
    if (mem != LOB_MEM_HOST && mem != LOB_MEM_DEVICE) throw LobError(LOB_E_ARG, "bad mem");
    ViewSt& V = e->rels[rel].views[0];
    const u64 n = V.n;
    if (n_ids) *n_ids = 0;
    if (!n) return LOB_OK;
    DevBuf l, off, out;
    e->ensure(l, n * 4);
    e->ensure(off, (n + 1) * 8);
    const u64* tags = V.tags.as<u64>();
    top1_proof_lengths(tags, n, e->arena.as<u32>(), l.as<u32>(), e->stream);
    e->after_launch("proof lengths");
    scratch_at_least(*e, scan_scratch_elems(n) * 8 + 64);
    exclusive_scan<u32, u64>(l.as<u32>(), off.as<u64>(), n, e->counts.as<u64>(), e->scratch.as<u64>(), e->stream);
    e->after_launch("proof offsets");
    const u64 total = e->read_u64(e->counts.as<u64>());
    if (n_ids) *n_ids = total;
    if (lens) {
      e->check(cudaMemcpyAsync(lens, l.p, n * 4, mem == LOB_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                               e->stream), "proof lengths out");
    }
    if (ids && total > id_capacity) {
      e->sync();
      e->release(l);
      e->release(off);
      throw LobError(LOB_E_CAPACITY, "id capacity " + std::to_string(id_capacity) + " < " + std::to_string(total));
    }
    if (ids && total) {
      u32* dst = ids;
      if (mem == LOB_MEM_HOST) {
        e->ensure(out, total * 4);
        dst = out.as<u32>();
      }
      top1_copy_proofs(tags, n, e->arena.as<u32>(), off.as<u64>(), dst, e->stream);
      e->after_launch("proof ids");
      if (mem == LOB_MEM_HOST)
        e->check(cudaMemcpyAsync(ids, out.p, total * 4, cudaMemcpyDeviceToHost, e->stream), "proof ids out");
    }
    e->sync();
    e->release(l);
    e->release(off);
    e->release(out);
    return LOB_OK;
  });
}

int lob_backward(lob_engine* e, uint32_t out_rel, const float* grad_tags, float* const* grad_inputs, int mem) {
  return guarded(e, [&] { return backward_impl(e, out_rel, grad_tags, grad_inputs, mem); });
}

int lob_profile_count(lob_engine* e, uint32_t* n) {
  return guarded(e, [&] {
    if (!n) throw LobError(LOB_E_ARG, "null n");
    e->sync();
    e->prof.flush();
    *n = (uint32_t)e->prof.agg.size();
    return LOB_OK;
  });
}

int lob_profile_entry(lob_engine* e, uint32_t i, char* name, size_t name_cap, uint64_t* launches, double* ms,
                      double* bytes) {
  return guarded(e, [&] {
    if (i >= e->prof.agg.size()) throw LobError(LOB_E_ARG, "profile index out of range");
    auto it = e->prof.agg.begin();
    std::advance(it, i);
    if (name && name_cap) {
      std::strncpy(name, it->first.c_str(), name_cap - 1);
      name[name_cap - 1] = 0;
    }
    if (launches) *launches = it->second.launches;
    if (ms) *ms = it->second.ms;
    if (bytes) *bytes = it->second.bytes;
    return LOB_OK;
  });
}

int lob_profile_reset(lob_engine* e) {
  return guarded(e, [&] {
    e->sync();
    e->prof.flush();
    e->prof.agg.clear();
    return LOB_OK;
  });
}

int lob_prim_sort(lob_engine* e, void* keys, void* payload, uint64_t n, uint32_t key_bits, uint32_t key_bytes,
                  uint32_t payload_bytes) {
  return guarded(e, [&] {
    if ((key_bytes != 4 && key_bytes != 8) || (payload_bytes != 0 && payload_bytes != 4 && payload_bytes != 8) ||
        key_bits > key_bytes * 8 || (n && !keys) || (n && payload_bytes && !payload))
      throw LobError(LOB_E_ARG, "bad sort arguments");
    if (n > 0xFFFFFFFFull) throw LobError(LOB_E_ARG, "sort supports fewer than 2^32 keys");
    if (n < 2) return LOB_OK;
    e->ensure(e->tmp_keys, n * key_bytes);
    if (payload_bytes) e->ensure(e->tmp_tags, n * payload_bytes);
    void* k = keys;
    void* p = payload;
    e->check(cudaMemsetAsync(sort_err(*e), 0, sizeof(u32), e->stream), "sort error word");
    engine_sort(*e, key_bytes == 8, payload_bytes, &k, &p, e->tmp_keys.p, e->tmp_tags.p, n, (int)key_bits);
    e->after_launch("sort");
    if (k != keys) e->check(cudaMemcpyAsync(keys, k, n * key_bytes, cudaMemcpyDeviceToDevice, e->stream), "copy back");
    if (payload_bytes && p != payload)
      e->check(cudaMemcpyAsync(payload, p, n * payload_bytes, cudaMemcpyDeviceToDevice, e->stream), "copy back");
    e->sync();
    if (e->read_u64(e->counts.as<u64>() + 15) & 0xFFFFFFFFull) throw LobError(LOB_E_TIMEOUT, "sort look-back wait gave up");
    return LOB_OK;
  });
}

int lob_prim_exclusive_scan(lob_engine* e, const uint32_t* in, uint64_t* out, uint64_t n, uint64_t* total) {
  return guarded(e, [&] {
    if ((n && (!in || !out)) || !total) throw LobError(LOB_E_ARG, "bad scan arguments");
    scratch_at_least(*e, scan_scratch_elems(n) * 8 + 64);
    exclusive_scan<u32, u64>(in, reinterpret_cast<u64*>(out), n, e->counts.as<u64>(), e->scratch.as<u64>(), e->stream);
    e->after_launch("scan");
    *total = e->read_u64(e->counts.as<u64>());
    return LOB_OK;
  });
}

int lob_prim_unique(lob_engine* e, int semiring, const void* keys, const void* tags, uint64_t n, uint32_t key_bytes,
                    void* out_keys, void* out_tags, uint64_t* n_out) {
  return guarded(e, [&] {
    if (semiring < 0 || semiring > 4 || (key_bytes != 4 && key_bytes != 8) || !n_out || (n && (!keys || !out_keys)) ||
        (n && semiring != LOB_UNIT && (!tags || !out_tags)))
      throw LobError(LOB_E_ARG, "bad unique arguments");
    scratch_at_least(*e, unique_scratch_bytes(n));
    unique_run(sem_kernel(semiring), key_bytes == 8, keys, tags, n, out_keys, out_tags, e->counts.as<u64>() + 1,
               e->scratch.p, e->stream);
    e->after_launch("unique");
    *n_out = e->read_u64(e->counts.as<u64>() + 1);
    return LOB_OK;
  });
}

int lob_prim_diff_merge(lob_engine* e, int semiring, const void* f_keys, const void* f_tags, uint64_t nf,
                        const void* u_keys, const void* u_tags, uint64_t nu, uint32_t key_bytes, void* out_keys,
                        void* out_tags, void* r_keys, void* r_tags, uint64_t* n_out, uint64_t* n_r) {
  return guarded(e, [&] {
    if (semiring < 0 || semiring > 4 || (key_bytes != 4 && key_bytes != 8) || !n_out || !n_r)
      throw LobError(LOB_E_ARG, "bad merge arguments");
    if (!nu) {
      *n_out = nf;
      *n_r = 0;
      if (nf) {
        e->check(cudaMemcpyAsync(out_keys, f_keys, nf * key_bytes, cudaMemcpyDeviceToDevice, e->stream), "copy");
        const int sb = stored_bytes(semiring);
        if (sb) e->check(cudaMemcpyAsync(out_tags, f_tags, nf * sb, cudaMemcpyDeviceToDevice, e->stream), "copy");
      }
      e->sync();
      return LOB_OK;
    }
    MergeArgs M{};
    M.sem = sem_kernel(semiring);
    M.key64 = key_bytes == 8;
    M.fkeys = f_keys; M.ftags = f_tags; M.fstamp = nullptr; M.nf = nf;
    M.ukeys = u_keys; M.utags = u_tags; M.nu = nu; M.u_stored = 0;
    M.okeys = out_keys; M.otags = out_tags; M.ostamp = nullptr;
    M.rkeys = r_keys; M.rtags = r_tags;
    M.stamp = 1;
    M.counts_dev = e->counts.as<u64>() + 2;
    scratch_at_least(*e, merge_scratch_bytes(nf, nu));
    diff_merge(M, e->scratch.p, e->stream);
    e->after_launch("merge");
    e->check(cudaMemcpyAsync(e->pinned, e->counts.as<u64>() + 2, 24, cudaMemcpyDeviceToHost, e->stream), "counts");
    e->sync();
    if (e->pinned[2]) throw LobError(LOB_E_ARG, "inputs are not sorted distinct keys");
    *n_out = nf + nu - e->pinned[0];
    *n_r = e->pinned[1];
    return LOB_OK;
  });
}

int lob_reset(lob_engine* e) {
  return guarded(e, [&] {
    e->sync();
    release_derived(*e);
    for (auto& r : e->rels) {
      for (auto& b : r.in_cols) e->release(b);
      r.in_cols.clear();
      e->release(r.in_tags);
      e->release(r.in_samples);
      r.n_in = r.in_cap = 0;
      r.in_has_tags = r.in_has_samples = false;
    }
    e->state = 0;
    e->ran_diff = false;
    return LOB_OK;
  });
}

int lob_set_option(lob_engine* e, const char* key, int64_t value) {
  return guarded(e, [&] {
    if (!key) throw LobError(LOB_E_ARG, "null key");
    std::string k = key;
    if (k == "join_index" && value >= 0 && value <= 3) e->opt_join_index = (int)value;
    else if (k == "hash_slots" && (value == 2 || value == 4 || value == 8)) e->opt_hash_slots = (int)value;
    else if (k == "dense_bits" && value >= 1 && value <= 30) e->opt_dense_bits = (int)value;
    else if (k == "radix_bits" && value >= 4 && value <= 11) e->opt_radix_bits = sort_supported_radix_bits((int)value);
    else if (k == "sync_check" && (value == 0 || value == 1)) e->opt_sync_check = (int)value;
    else if (k == "profile" && (value == 0 || value == 1)) e->opt_profile = (int)value;
    else if (k == "max_candidates" && value >= 4096 && value <= (int64_t)1 << 31) e->opt_max_cand = (u64)value;
    else if (k == "emit_filter" && value >= 0 && value <= 2) e->opt_emit_filter = (int)value;
    else if (k == "sort_algo" && (value == 0 || value == 1)) e->opt_sort_algo = (int)value;
    else if (k == "packed_join" && (value == 0 || value == 1)) e->opt_packed_join = (int)value;
    else if (k == "bitmap_delta" && value >= 0 && value <= 2) e->opt_bitmap_delta = (int)value;
    else if (k == "warp_join" && value >= 0 && value <= 2) e->opt_warp_join = (int)value;
    else if (k == "acc_dense" && (value == 0 || value == 1)) e->opt_acc_dense = (int)value;
    else if (k == "acc_bits" && value >= 1 && value <= 30) e->opt_acc_bits = (int)value;
    else if (k == "driver" && value >= 0 && value <= 2) e->opt_driver = (int)value;
    else if (k == "loop_guards" && (value == 0 || value == 1)) e->opt_loop_guards = (int)value;
    else if (k == "loop_cap_floor" && value >= 256 && value <= (1 << 24)) e->opt_loop_cap_floor = (int)value;
    else if (k == "packed_backward" && (value == 0 || value == 1)) e->opt_packed_backward = (int)value;
    else if (k == "cross_join" && (value == 0 || value == 1)) e->opt_cross_join = (int)value;
    else if (k == "proof_cap" && value >= 1 && value <= (1 << 20)) e->opt_proof_cap = (int)value;
    else if (k == "proof_arena_words" && value >= 16 && value <= (1ll << 31)) e->opt_arena_words = (u64)value;
    else throw LobError(LOB_E_ARG, "unknown option or value out of range: " + k);
    return LOB_OK;
  });
}

}  // extern "C"
