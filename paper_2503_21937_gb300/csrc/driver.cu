// Device-driven iteration loop (Algorithm 1's "repeat until F_T stops
// growing", with every decision taken on the GPU).
//
// After the first iteration (run by the host loop, which fires the rules whose
// delta atom is an input relation), the remaining iterations of a tagged run
// run as one instantiated CUDA graph: a conditional WHILE node whose body is
// one iteration -- begin, index rebuilds, join arms, dense read-out,
// difference+merge, secondary views, end -- and whose condition the body's
// last kernel sets from the device state.
//
// Every size -- rows of a recent set, outputs of a join step, unique
// candidates, |F| -- lives in a device state block; kernels read it there and
// their grids are sized from capacities.  Each relation's views and recent
// set are double-buffered with their own parity: the begin kernel resolves
// this iteration's current and next buffers into a device pointer table that
// the kernels read, the merges of a relation that received no candidates do
// nothing, and the end kernel flips only what was written.  The begin kernel
// also decides which arms run (the host loop's skip rules); the end kernel
// commits the iteration's sizes and decides whether to stop (no new facts,
// max_iters, or a capacity overflow).  A guard kernel after each
// size-producing step records an overflow; the iteration then ends without
// committing, so the last committed state stays intact in its buffers, and
// the host grows the buffers and launches again.  In the steady state the
// host waits once per run, not per iteration.
#include <algorithm>
#include <cstring>

#include "engine.h"
#include "pjoin.h"
#include "scan.cuh"

#include <functional>

namespace {

constexpr int kGMaxRels = 16, kGMaxArms = 32, kGMaxSteps = 8, kGMaxViews = 4, kGMaxBefore = 8;
constexpr int kRelSlots = 8 + 4 * kGMaxViews;
constexpr int kArmSlots = 1 + kGMaxSteps;
// header slots of the state block
enum : int { S_K = 0, S_STOP, S_UNUSED, S_OVERFLOW, S_EMITTED, S_NEW, S_ERR, S_ITERS, S_HDR = 8 };
enum : u64 { STOP_NONE = 0, STOP_FIXPOINT = 1, STOP_MAXITER = 2, STOP_OVERFLOW = 3, STOP_RECORD = 4 };
// relation slots: |F|, |recent|, unique candidates, then the merge's counts
// (duplicates, new or improved, error word), whether an arm with this head
// runs in the iteration; view j >= 1 at 8 + 4 (j - 1):
// rows, duplicates, new, error word
enum : int { R_FULL = 0, R_RECENT, R_NU, R_DUPS, R_NR, R_MERR, R_ACTIVE };


struct GDesc {
  int nrel, narm;
  u32 max_iters, rec_cap;
  int rel_dense[kGMaxRels];
  int rel_nviews[kGMaxRels];
  int arm_delta[kGMaxArms], arm_last[kGMaxArms], arm_nbefore[kGMaxArms], arm_head[kGMaxArms];
  int arm_before[kGMaxArms][kGMaxBefore];
  // double-buffered groups: per dense relation its primary view, its
  // maintained views (in view-slot order) and its recent set
  int ngroups, par_base;  // group g's parity is state slot par_base + g
  int rel_group[kGMaxRels];  // first group of the relation (primary view); views follow, then the recent set
  // capacities the iteration's buffers were planned with, and the state slots
  // that record what an overflowing iteration needed
  u64 cap_full[kGMaxRels], cap_u[kGMaxRels], cap_r[kGMaxRels], cap_view[kGMaxRels][kGMaxViews];
  u64 cap_bind, cap_outputs;
  int need_full[kGMaxRels], need_u[kGMaxRels], need_r[kGMaxRels], need_view[kGMaxRels][kGMaxViews];
  int need_bind, need_tiles;
};
static_assert(sizeof(GDesc) <= 4096, "loop descriptor must fit the kernel parameter space");
// pointer table entries: tab / res [(g * 2 + b) * 3 + field], field 0 keys,
// 1 tags, 2 stamps; tab's b is the buffer, res's b is 0 = current, 1 = next
LOB_HD int ptr_slot(int g, int b) { return (g * 2 + b) * 3; }

LOB_HD int rel_base(int r) { return S_HDR + r * kRelSlots; }
LOB_HD int view_base(int r, int j) { return rel_base(r) + 8 + 4 * (j - 1); }
LOB_HD int arm_base(int nrel, int a) { return S_HDR + nrel * kRelSlots + a * kArmSlots; }

// Which arms run in the coming iteration (a recent delta relation, and old
// facts in every derived atom before the delta atom), and the iteration's
// record of (|F|, |recent|) per relation for the backward pass.
// handles of the IF guards of the iteration's arms and relation sections
// (on = 0: no guards), set by the begin kernel
struct GGuards {
  int on;
  cudaGraphConditionalHandle arm[kGMaxArms], rel[kGMaxRels];
};

__global__ void k_iter_begin(const __grid_constant__ GDesc d, u64* s, u64* rec, void* const* tab, void** res,
                             const __grid_constant__ GGuards gg) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int g = 0; g < d.ngroups; g++) {  // this iteration's current and next buffers of every group
    const int p = (int)(s[d.par_base + g] & 1);
    for (int f = 0; f < 3; f++) {
      res[ptr_slot(g, 0) + f] = tab[ptr_slot(g, p) + f];
      res[ptr_slot(g, 1) + f] = tab[ptr_slot(g, p ^ 1) + f];
    }
  }
  const u64 k = s[S_K] + 1;
  for (int a = 0; a < d.narm; a++) {
    const u64* D = s + rel_base(d.arm_delta[a]);
    bool active = D[R_RECENT] > 0;
    for (int b = 0; b < d.arm_nbefore[a] && active; b++) {
      const u64* B = s + rel_base(d.arm_before[a][b]);
      if (B[R_FULL] == B[R_RECENT]) active = false;
    }
    u64* A = s + arm_base(d.nrel, a);
    A[0] = active ? D[R_RECENT] : 0;
    // an inactive arm may be skipped by its guard: its step totals read 0
    if (!active)
      for (int st = 1; st <= d.arm_last[a]; st++) A[1 + st] = 0;
  }
  // a relation whose head arms all stay idle gets no candidates (its section
  // may be skipped by its guard, leaving R_NU at 0)
  for (int r = 0; r < d.nrel; r++) {
    if (!d.rel_dense[r]) continue;
    u64 any = 0;
    for (int a = 0; a < d.narm; a++)
      if (d.arm_head[a] == r && s[arm_base(d.nrel, a)]) any = 1;
    s[rel_base(r) + R_ACTIVE] = any;
    s[rel_base(r) + R_NU] = 0;
    // the counts an empty difference+merge would report, so that the end
    // kernel's capacity checks do not read the last active iteration's
    if (!any) s[rel_base(r) + R_DUPS] = s[rel_base(r) + R_NR] = 0;
  }
  if (gg.on) {
    for (int a = 0; a < d.narm; a++) cudaGraphSetConditional(gg.arm[a], s[arm_base(d.nrel, a)] != 0 ? 1u : 0u);
    for (int r = 0; r < d.nrel; r++)
      if (d.rel_dense[r]) cudaGraphSetConditional(gg.rel[r], s[rel_base(r) + R_ACTIVE] != 0 ? 1u : 0u);
  }
  if (k <= d.rec_cap)
    for (int r = 0; r < d.nrel; r++) {
      rec[2 * ((k - 1) * d.nrel + r)] = s[rel_base(r) + R_FULL];
      rec[2 * ((k - 1) * d.nrel + r) + 1] = s[rel_base(r) + R_RECENT];
    }
}

LOB_DEV void need_at_most(u64* s, u64 v, u64 cap, int need) {
  if (v > cap) {
    s[S_OVERFLOW] = 1;
    if (v > s[need]) s[need] = v;
  }
}

// Commit the iteration, or stop without committing when a size outgrew its
// buffer (every kernel clamped its writes to the capacities, so the committed
// state in the current buffers is intact).
__global__ void k_iter_end(const __grid_constant__ GDesc d, u64* s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int a = 0; a < d.narm; a++)
    for (int st = 1; st <= d.arm_last[a]; st++) {
      const u64 t = s[arm_base(d.nrel, a) + 1 + st];
      need_at_most(s, t, d.cap_outputs, d.need_tiles);
      if (st < d.arm_last[a]) need_at_most(s, t, d.cap_bind, d.need_bind);
    }
  for (int r = 0; r < d.nrel; r++) {
    if (!d.rel_dense[r]) continue;
    const u64* R = s + rel_base(r);
    need_at_most(s, R[R_NU], d.cap_u[r], d.need_u[r]);
    need_at_most(s, R[R_FULL] + R[R_NU], d.cap_full[r], d.need_full[r]);
    need_at_most(s, R[R_NR], d.cap_r[r], d.need_r[r]);
    for (int j = 1; j <= d.rel_nviews[r]; j++)
      need_at_most(s, s[view_base(r, j)] + R[R_NR], d.cap_view[r][j - 1], d.need_view[r][j - 1]);
  }
  if (s[S_OVERFLOW]) {
    s[S_STOP] = STOP_OVERFLOW;
    return;
  }
  u64 total_new = 0;
  for (int r = 0; r < d.nrel; r++) {
    if (!d.rel_dense[r]) continue;
    u64* R = s + rel_base(r);
    const int g0 = d.rel_group[r], grec = g0 + 1 + d.rel_nviews[r];
    if (R[R_NU] == 0) {  // no candidates: nothing was merged or written
      R[R_RECENT] = 0;
      continue;
    }
    R[R_FULL] = R[R_FULL] + R[R_NU] - R[R_DUPS];
    R[R_RECENT] = R[R_NR];
    total_new += R[R_NR];
    s[d.par_base + g0] ^= 1ull;    // F and the recent set were written to their next buffers
    s[d.par_base + grec] ^= 1ull;
    if (R[R_NR] == 0) continue;    // the secondary views merged nothing
    for (int j = 1; j <= d.rel_nviews[r]; j++) {
      u64* V = s + view_base(r, j);
      V[0] = V[0] + R[R_NR] - V[1];
      s[d.par_base + g0 + j] ^= 1ull;
    }
  }
  for (int a = 0; a < d.narm; a++) s[S_EMITTED] += s[arm_base(d.nrel, a) + 1 + d.arm_last[a]];
  s[S_K] += 1;
  s[S_NEW] += total_new;
  s[S_ITERS] += 1;
  if (total_new == 0) s[S_STOP] = STOP_FIXPOINT;
  else if (s[S_K] >= d.max_iters) s[S_STOP] = STOP_MAXITER;
  else if (s[S_K] >= d.rec_cap) s[S_STOP] = STOP_RECORD;
}

// In-graph phase timing (engine option "profile"): each call adds the time
// since the previous call to phase i's total (ns, from the global timer).
// t[0] holds the previous time stamp, t[1 + i] phase i's total.
LOB_DEV u64 global_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__global__ void k_phase_mark(u64* t, int i) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const u64 now = global_ns();
  if (i >= 0) t[1 + i] += now - t[0];
  t[0] = now;
}

__global__ void k_set_cond(const u64* s, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, s[S_STOP] == STOP_NONE ? 1u : 0u);
}


// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct GView {
  int rel, view, slot;  // slot: state view index (1..)
};
struct GArm {
  const RulePlan* rp;
  const ArmPlan* A;
};
struct GIndex {
  int rel, view, prefix, size_slot;
};

struct GLoop {
  GDesc d{};
  std::vector<GArm> arms;
  std::vector<std::vector<GView>> views;  // per relation: maintained secondary views
  std::vector<GIndex> indexes;            // dense indexes of derived relations, rebuilt every iteration
  std::vector<u64> cap_full, cap_u, cap_r;  // per relation: |F|, unique candidates, recent set
  std::vector<std::vector<u64>> cap_view; // per relation, per maintained view
  u64 cap_bind = 0, cap_tiles = 0, cap_rows = 0;
  int need_base = 0, n_slots = 0;
  // need slot ids
  std::vector<int> need_full, need_u, need_r;
  std::vector<std::vector<int>> need_view;
  int need_bind = 0, need_tiles = 0;
  DevBuf state, rec, tab, res;
  // in-graph phase timing (profiling only): phase names and their totals
  bool timing = false;
  std::vector<std::string> phases;
  DevBuf times;
};

// the phase id of `name`, added on first use (the same names in both halves)
int phase_id(GLoop& G, const std::string& name) {
  for (size_t i = 0; i < G.phases.size(); i++)
    if (G.phases[i] == name) return (int)i;
  G.phases.push_back(name);
  return (int)G.phases.size() - 1;
}

u64 g_cap_floor = 1ull << 16;  // set per run from the engine's option
u64 round_cap(u64 x) { return std::max<u64>(g_cap_floor, (x + 255) & ~255ull); }

int key_bytes(const Layout& L) { return L.key64 ? 8 : 4; }

// The loop can take over: a tagged run whose derived relations all use dense
// accumulation, and whose arms with a derived delta relation are packed join
// pipelines of at least one probe.
bool loop_eligible(const lob_engine& e) {
  // (hash indexes of derived relations are built on the host; the loop
  // rebuilds only dense offset tables)
  if (!e.opt_driver || e.semiring == SR_UNIT || e.opt_sort_algo != 0 || e.opt_join_index == 3) return false;
  if ((int)e.rels.size() > kGMaxRels) return false;
  int narm = 0;
  for (const auto& r : e.rels) {
    if (r.idb && !r.dense) return false;
    int nv = 0;
    for (size_t vi = 1; vi < r.views.size(); vi++) nv += r.views[vi].maintained;
    if (nv > kGMaxViews) return false;
  }
  for (const auto& p : e.plans)
    for (const auto& A : p.arms) {
      if (!e.rels[p.ast.body[A.delta].rel].idb) continue;
      if (!A.packed.ok || A.steps.size() < 2 || A.steps.size() > (size_t)kGMaxSteps) return false;
      if (A.before_rels.size() > (size_t)kGMaxBefore) return false;
      narm++;
    }
  return narm > 0 && narm <= kGMaxArms;
}

void plan_loop(lob_engine& e, GLoop& G, u32 max_iters) {
  const int nrel = (int)e.rels.size();
  G.d.nrel = nrel;
  G.d.max_iters = max_iters;
  G.views.assign(nrel, {});
  for (int r = 0; r < nrel; r++) {
    RelSt& R = e.rels[r];
    G.d.rel_dense[r] = R.idb && R.dense;
    int slot = 0;
    for (size_t vi = 1; vi < R.views.size(); vi++)
      if (R.views[vi].maintained) G.views[r].push_back({r, (int)vi, ++slot});
    G.d.rel_nviews[r] = slot;
  }
  for (const auto& p : e.plans)
    for (const auto& A : p.arms) {
      if (!e.rels[p.ast.body[A.delta].rel].idb) continue;
      const int a = (int)G.arms.size();
      G.arms.push_back({&p, &A});
      G.d.arm_delta[a] = (int)p.ast.body[A.delta].rel;
      G.d.arm_last[a] = (int)A.steps.size() - 1;
      G.d.arm_nbefore[a] = (int)A.before_rels.size();
      G.d.arm_head[a] = (int)p.ast.head.rel;
      for (size_t b = 0; b < A.before_rels.size(); b++) G.d.arm_before[a][b] = (int)A.before_rels[b];
    }
  G.d.narm = (int)G.arms.size();
  // dense indexes over derived relations' views: rebuilt at the start of every iteration
  for (auto& ga : G.arms)
    for (size_t s = 1; s < ga.A->steps.size(); s++) {
      const StepPlan& S = ga.A->steps[s];
      const int rel = (int)ga.rp->ast.body[S.atom].rel;
      RelSt& R = e.rels[rel];
      ViewSt& W = R.views[S.view];
      engine_ensure_index(e, W, S.prefix_len);
      if (!R.idb || W.index[S.prefix_len].mode != INDEX_DENSE) continue;
      int slot = 0;
      for (auto& gv : G.views[rel])
        if (gv.view == S.view) slot = gv.slot;
      const int size_slot = S.view == 0 ? rel_base(rel) + R_FULL : view_base(rel, slot);
      bool dup = false;
      for (auto& gi : G.indexes) dup = dup || (gi.rel == rel && gi.view == S.view && gi.prefix == S.prefix_len);
      if (!dup) G.indexes.push_back({rel, S.view, S.prefix_len, size_slot});
    }
  // need slots
  int n = arm_base(nrel, G.d.narm);
  G.need_base = n;
  G.need_full.resize(nrel);
  G.need_u.resize(nrel);
  G.need_r.resize(nrel);
  G.need_view.assign(nrel, {});
  for (int r = 0; r < nrel; r++) {
    G.need_full[r] = n++;
    G.need_u[r] = n++;
    G.need_r[r] = n++;
    for (size_t j = 0; j < G.views[r].size(); j++) G.need_view[r].push_back(n++);
  }
  G.need_bind = n++;
  G.need_tiles = n++;
  // buffer groups and their parity slots
  int g = 0;
  for (int r = 0; r < nrel; r++) {
    G.d.rel_group[r] = g;
    if (G.d.rel_dense[r]) g += 2 + (int)G.views[r].size();
  }
  G.d.ngroups = g;
  G.d.par_base = n;
  n += g;
  G.n_slots = n;
}

// the current (b = 0) and twin (b = 1) buffers of group g, as the host holds them
void group_buffers(lob_engine& e, const GLoop& G, int g, int b, void** out3) {
  for (int r = 0; r < G.d.nrel; r++) {
    if (!G.d.rel_dense[r]) continue;
    const int g0 = G.d.rel_group[r], nv = (int)G.views[r].size();
    if (g < g0 || g > g0 + 1 + nv) continue;
    RelSt& R = e.rels[r];
    if (g == g0 + 1 + nv) {  // recent set
      out3[0] = (b ? R.nkeys : R.rkeys).p;
      out3[1] = (b ? R.ntags : R.rtags).p;
      out3[2] = nullptr;
      return;
    }
    ViewSt& W = R.views[g == g0 ? 0 : G.views[r][g - g0 - 1].view];
    out3[0] = (b ? W.keys2 : W.keys).p;
    out3[1] = (b ? W.tags2 : W.tags).p;
    out3[2] = (b ? W.stamps2 : W.stamps).p;
    return;
  }
}

// Capacities: what the engine remembers from earlier runs of this program, or
// a few times the sizes after the first iteration; grown on overflow.
void initial_caps(lob_engine& e, GLoop& G) {
  const int nrel = G.d.nrel;
  auto mem = [&](const std::string& k) { auto it = e.loop_caps.find(k); return it == e.loop_caps.end() ? 0ull : it->second; };
  G.cap_full.assign(nrel, 0);
  G.cap_u.assign(nrel, 0);
  G.cap_r.assign(nrel, 0);
  G.cap_view.assign(nrel, {});
  for (int r = 0; r < nrel; r++) {
    const RelSt& R = e.rels[r];
    const std::string id = std::to_string(r);
    G.cap_full[r] = round_cap(std::max<u64>(mem("full" + id), 4 * R.views[0].n));
    G.cap_u[r] = round_cap(std::max<u64>(mem("u" + id), 4 * std::max<u64>(R.n_recent, R.views[0].n)));
    G.cap_r[r] = round_cap(std::max<u64>(mem("r" + id), 4 * R.n_recent));
    for (auto& gv : G.views[r])
      G.cap_view[r].push_back(round_cap(std::max<u64>(mem("v" + id + "." + std::to_string(gv.view)), 4 * R.views[gv.view].n)));
  }
  G.cap_bind = round_cap(std::max<u64>(mem("bind"), 16 * g_cap_floor));
  G.cap_tiles = std::max<u64>(mem("tiles"), std::max<u64>(1, g_cap_floor / 16));
}

void remember_caps(lob_engine& e, const GLoop& G) {
  for (int r = 0; r < G.d.nrel; r++) {
    const std::string id = std::to_string(r);
    e.loop_caps["full" + id] = G.cap_full[r];
    e.loop_caps["u" + id] = G.cap_u[r];
    e.loop_caps["r" + id] = G.cap_r[r];
    for (size_t j = 0; j < G.views[r].size(); j++)
      e.loop_caps["v" + id + "." + std::to_string(G.views[r][j].view)] = G.cap_view[r][j];
  }
  e.loop_caps["bind"] = G.cap_bind;
  e.loop_caps["tiles"] = G.cap_tiles;
}

// Buffers of both parities at the planned capacities (the current parity's
// contents are kept).
void allocate(lob_engine& e, GLoop& G) {
  const int ks = sem_kernel(e.semiring);
  const int sb = stored_bytes(e.semiring), cb = cand_bytes(e.semiring);
  const bool stamps = sem_stamps(e.semiring);
  u64 max_u = 0, max_rows = G.cap_bind, max_merge = 0, max_sort = 0, max_bits = 0;
  int max_kb = 4;
  for (int r = 0; r < G.d.nrel; r++) {
    if (!G.d.rel_dense[r]) continue;
    RelSt& R = e.rels[r];
    ViewSt& V = R.views[0];
    const int kb = key_bytes(V.lay);
    const u64 nf = G.cap_full[r] + G.cap_u[r], nu = G.cap_u[r], nr = G.cap_r[r];
    e.ensure(V.keys, nf * kb, true);
    e.ensure(V.keys2, nf * kb);
    if (sb) { e.ensure(V.tags, nf * sb, true); e.ensure(V.tags2, nf * sb); }
    if (stamps) { e.ensure(V.stamps, nf * 4, true); e.ensure(V.stamps2, nf * 4); }
    e.ensure(R.rkeys, nr * kb, true);
    e.ensure(R.nkeys, nr * kb);
    if (sb) { e.ensure(R.rtags, nr * sb, true); e.ensure(R.ntags, nr * sb); }
    e.ensure(R.akeys, nu * kb);
    e.ensure(R.atags, nu * cb);
    max_u = std::max(max_u, nu);
    max_rows = std::max(max_rows, nr);
    max_merge = std::max<u64>(max_merge, merge_scratch_bytes(G.cap_full[r], nu));
    max_bits = std::max<u64>(max_bits, 1ull << V.lay.bits);
    for (size_t j = 0; j < G.views[r].size(); j++) {
      ViewSt& W = R.views[G.views[r][j].view];
      const int wkb = key_bytes(W.lay);
      const u64 nw = G.cap_view[r][j] + nr;
      e.ensure(W.keys, nw * wkb, true);
      e.ensure(W.keys2, nw * wkb);
      if (sb) { e.ensure(W.tags, nw * sb, true); e.ensure(W.tags2, nw * sb); }
      if (stamps) { e.ensure(W.stamps, nw * 4, true); e.ensure(W.stamps2, nw * 4); }
      max_kb = std::max(max_kb, wkb);
      max_merge = std::max<u64>(max_merge, merge_scratch_bytes(G.cap_view[r][j], nr));
      max_sort = std::max(max_sort, nr);
    }
  }
  (void)ks;
  if (max_sort) {
    e.ensure(e.tmp_keys, max_sort * max_kb);
    e.ensure(e.tmp_keys2, max_sort * max_kb);
    if (sb) { e.ensure(e.tmp_tags, max_sort * sb); e.ensure(e.tmp_tags2, max_sort * sb); }
  }
  for (int side = 0; side < 2; side++) {
    e.ensure(e.bind[side][0], G.cap_bind * 8);
    if (cb) e.ensure(e.bind[side][kMaxSlots + 1], G.cap_bind * cb);
  }
  G.cap_rows = max_rows;
  // an intermediate step's emission covers the binding-table capacity in tiles
  G.cap_tiles = std::max<u64>(G.cap_tiles, (G.cap_bind + kEmitTile - 1) / kEmitTile);
  const u64 nblk = pjoin_loc_blocks(G.cap_rows);
  e.ensure(e.cnt, G.cap_rows * 4);
  e.ensure(e.lo, G.cap_rows * 4);
  e.ensure(e.off, nblk * 16);
  e.ensure(e.part, (G.cap_tiles + 1) * 8);
  size_t scratch = std::max<size_t>(scan_scratch_elems(nblk) * 8 + 64, max_merge);
  scratch = std::max(scratch, bits_scratch_bytes(max_bits));
  if (max_sort) scratch = std::max(scratch, sort_scratch_bytes(max_sort, e.opt_radix_bits));
  e.ensure(e.scratch, scratch);
  e.ensure(G.state, (size_t)G.n_slots * 8);
}

// One iteration, captured into the stream.  Buffers of derived relations are
// reached through the pointer table the begin kernel resolves.  With guards
// (option "loop_guards"), every join arm and every relation's difference+merge
// section sits in a conditional IF node that runs it only when the arm is
// active / an arm with that head ran, so an iteration in which most rules
// have nothing to do launches few kernels; the IF bodies are captured on the
// second stream `st2`, and their graphs are appended to `bodies`.
void capture_iteration(lob_engine& e, GLoop& G, u64* st_dev, u64* rec_dev, cudaStream_t st0, cudaStream_t st2,
                       std::vector<cudaGraph_t>& bodies) {
  const int sem = e.semiring, ks = sem_kernel(sem);
  const int sb = stored_bytes(sem), cb = cand_bytes(sem);
  const bool stamps = sem_stamps(sem);
  auto slot = [st_dev](int i) { return st_dev + i; };
  void** res = G.res.as<void*>();
  // groups: primary view of r, its maintained view slot j, its recent set
  auto gview = [&](int r, int view) -> int {
    if (view == 0) return G.d.rel_group[r];
    for (auto& gv : G.views[r])
      if (gv.view == view) return G.d.rel_group[r] + gv.slot;
    return -1;
  };
  auto grecent = [&](int r) { return G.d.rel_group[r] + 1 + (int)G.views[r].size(); };
  auto cur = [&](int g) { return res + ptr_slot(g, 0); };
  auto nxt = [&](int g) { return res + ptr_slot(g, 1); };
  auto mark_on = [&](const char* name, cudaStream_t s) {  // closes the phase that just ran
    if (!G.timing) return;
    k_phase_mark<<<1, 32, 0, s>>>(G.times.as<u64>(), name ? phase_id(G, name) : -1);
    e.check(cudaGetLastError(), "phase mark");
  };
  // the guards' handles, created on the graph being captured before the begin
  // kernel that sets them
  GGuards gg{};
  gg.on = e.opt_loop_guards;
  if (gg.on) {
    cudaStreamCaptureStatus cstat;
    cudaGraph_t graph = nullptr;
    e.check(cudaStreamGetCaptureInfo(st0, &cstat, nullptr, &graph, nullptr, nullptr, nullptr), "capture info");
    for (int a = 0; a < G.d.narm; a++)
      e.check(cudaGraphConditionalHandleCreate(&gg.arm[a], graph, 0, cudaGraphCondAssignDefault), "guard handle");
    for (int r = 0; r < G.d.nrel; r++)
      if (G.d.rel_dense[r])
        e.check(cudaGraphConditionalHandleCreate(&gg.rel[r], graph, 0, cudaGraphCondAssignDefault), "guard handle");
  }
  // run body(stream) under the IF node of handle h, or inline
  auto guarded = [&](cudaGraphConditionalHandle h, const std::function<void(cudaStream_t)>& body) {
    if (!gg.on) {
      body(st0);
      return;
    }
    cudaStreamCaptureStatus cstat;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    e.check(cudaStreamGetCaptureInfo(st0, &cstat, nullptr, &graph, &deps, &edata, &ndeps), "capture info");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e.check(cudaGraphAddNode(&node, graph, deps, edata, ndeps, &p), "guard node");
    e.check(cudaStreamUpdateCaptureDependencies(st0, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
            "capture dependencies");
    cudaGraph_t ifbody = p.conditional.phGraph_out[0];
    e.check(cudaStreamBeginCaptureToGraph(st2, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture");
    try {
      body(st2);
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(st2, &dummy);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t done = nullptr;
    e.check(cudaStreamEndCapture(st2, &done), "end capture");
    bodies.push_back(ifbody);
  };
  cudaStream_t st = st0;
  auto mark = [&](const char* name) { mark_on(name, st); };
  mark(nullptr);
  k_iter_begin<<<1, 32, 0, st>>>(G.d, st_dev, rec_dev, G.tab.as<void*>(), res, gg);
  e.check(cudaGetLastError(), "iteration begin");
  for (auto& gi : G.indexes) {
    RelSt& R = e.rels[gi.rel];
    ViewSt& W = R.views[gi.view];
    IndexSt& I = W.index[gi.prefix];
    const u64 cap = gi.view == 0 ? G.cap_full[gi.rel] + G.cap_u[gi.rel] : 0;
    u64 capw = cap;
    for (size_t j = 0; j < G.views[gi.rel].size(); j++)
      if (G.views[gi.rel][j].view == gi.view) capw = G.cap_view[gi.rel][j] + G.cap_r[gi.rel];
    // rebuilt only when the relation gained facts in the previous iteration
    build_dense_index(W.lay, gi.prefix, W.keys.p, capw, I.offs.as<u64>(), I.domain, st, slot(gi.size_slot),
                      slot(rel_base(gi.rel) + R_RECENT), cur(gview(gi.rel, gi.view)));
    e.check(cudaGetLastError(), "index");
  }
  mark("loop_begin_index");
  // the join arms: every output (+)-added into its head's dense accumulator
  for (size_t a = 0; a < G.arms.size(); a++) guarded(gg.arm[a], [&](cudaStream_t st) {
    auto mark = [&](const char* name) { mark_on(name, st); };
    const RuleAst& R = G.arms[a].rp->ast;
    const ArmPlan& A = *G.arms[a].A;
    const int drel = (int)R.body[A.delta].rel;
    RelSt& D = e.rels[drel];
    RelSt& H = e.rels[R.head.rel];
    const int ab = arm_base(G.d.nrel, (int)a);
    const void* in_words = D.rkeys.p;
    const void* in_tags = D.rtags.p;
    void* const* in_pp = cur(grecent(drel));
    u64 n_cap = G.cap_r[drel];
    const u64* n_dev = slot(ab);
    int side = 0;
    for (size_t s = 1; s < A.steps.size(); s++) {
      const StepPlan& S = A.steps[s];
      const bool last = s + 1 == A.steps.size();
      const int vrel = (int)R.body[S.atom].rel;
      RelSt& VR = e.rels[vrel];
      ViewSt& W = VR.views[S.view];
      PStep P = A.packed.steps[s - 1];
      P.in_words = in_words;
      P.in_tags = in_tags;
      P.in_pp = in_pp;
      P.n_in = n_cap;
      P.n_in_dev = n_dev;
      const bool derived = VR.idb;
      P.v_keys = W.keys.p;
      P.v_key64 = W.lay.key64;
      P.v_tags = W.tags.p;
      P.v_stamp = W.stamps.as<u32>();
      P.v_pp = derived ? cur(gview(vrel, S.view)) : nullptr;
      P.v_n = W.n;
      P.v_n_dev = nullptr;
      if (derived) {
        u64 capw = G.cap_full[vrel] + G.cap_u[vrel];
        int size_slot = rel_base(vrel) + R_FULL;
        for (size_t j = 0; j < G.views[vrel].size(); j++)
          if (G.views[vrel][j].view == S.view) {
            capw = G.cap_view[vrel][j] + G.cap_r[vrel];
            size_slot = view_base(vrel, G.views[vrel][j].slot);
          }
        P.v_n = capw;
        P.v_n_dev = slot(size_slot);
      }
      // facts older than the previous iteration's recent set: stamp < k - 1,
      // with k = the iteration being run = state k + 1
      P.v_stamp_mode = S.probe_old ? STAMP_LT : STAMP_NONE;
      P.v_stamp_val = 0;
      P.stamp_dev = slot(S_K);
      const IndexSt& I = W.index[S.prefix_len];
      P.index_mode = I.mode;
      P.dense_offs = I.offs.as<u64>();
      P.hash_bits = I.hash_bits;
      const u64 n_blk = pjoin_loc_blocks(n_cap);
      P.loc = e.cnt.as<u32>();
      P.lo32 = e.lo.as<u32>();
      P.blk_cnt = e.off.as<u64>() + n_blk;
      P.blk_off = e.off.as<u64>();
      P.err = reinterpret_cast<u32*>(slot(S_ERR));
      pjoin_count(ks, P, st);
      e.check(cudaGetLastError(), "join count");
      const int tslot = ab + 1 + (int)s;
      exclusive_scan<u64, u64>(P.blk_cnt, e.off.as<u64>(), n_blk, slot(tslot), e.scratch.as<u64>(), st);
      e.check(cudaGetLastError(), "join scan");
      const std::string tag = "loop_arm" + std::to_string(a) + "_step" + std::to_string(s);
      mark((tag + "_count").c_str());
      P.total_dev = slot(tslot);
      P.j_begin = 0;
      if (last) {
        P.out_words = nullptr;
        P.out_tags = nullptr;
        P.out_base = 0;
        P.out_count = nullptr;
        P.bitmap = H.dtouched.as<u32>();
        P.acc = H.dacc.p;
        P.total = G.cap_tiles * (u64)kEmitTile;
      } else {
        const int out_side = side ^ 1;
        P.out_words = e.bind[out_side][0].p;
        P.out_tags = e.bind[out_side][kMaxSlots + 1].p;
        P.out_base = 0;
        P.bitmap = nullptr;
        P.acc = nullptr;
        P.total = G.cap_bind;
        side = out_side;
      }
      const u64 ntiles = std::min<u64>(G.cap_tiles, (P.total + kEmitTile - 1) / kEmitTile);
      pjoin_partition(P, ntiles, e.part.as<u64>(), st);
      pjoin_emit(ks, P, e.part.as<u64>(), st);
      e.check(cudaGetLastError(), "join emit");
      mark((tag + "_emit").c_str());
      in_words = e.bind[side][0].p;
      in_tags = e.bind[side][kMaxSlots + 1].p;
      in_pp = nullptr;
      n_cap = G.cap_bind;
      n_dev = slot(tslot);
    }
  });
  // per derived relation: unique candidates out of the accumulator, then the
  // difference+merge into F and the secondary views
  for (int r = 0; r < G.d.nrel; r++) {
    if (!G.d.rel_dense[r]) continue;
    guarded(gg.rel[r], [&](cudaStream_t st) {
    auto mark = [&](const char* name) { mark_on(name, st); };
    RelSt& H = e.rels[r];
    ViewSt& V = H.views[0];
    const Layout& L = V.lay;
    const int rb = rel_base(r);
    const u64 nbits = 1ull << L.bits;
    bits_count(H.dtouched.as<u32>(), nullptr, nbits, e.scratch.p, slot(rb + R_NU), st);
    e.check(cudaGetLastError(), "dense count");
    dense_extract(ks, L.key64, H.dtouched.as<u32>(), H.dacc.p, nbits, H.akeys.p, H.atags.p, G.cap_u[r], e.scratch.p, st,
                  G.cap_u[r]);
    e.check(cudaGetLastError(), "dense extract");
    const std::string rtag = "loop_rel" + std::to_string(r);
    mark((rtag + "_dense").c_str());
    MergeArgs M{};
    M.sem = ks;
    M.key64 = L.key64;
    M.fkeys = V.keys.p;
    M.ftags = V.tags.p;
    M.fstamp = stamps ? V.stamps.as<u32>() : nullptr;
    M.f_pp = cur(gview(r, 0));
    M.o_pp = nxt(gview(r, 0));
    M.r_pp = nxt(grecent(r));
    M.skip_empty = 1;
    M.nf = G.cap_full[r];
    M.nf_dev = slot(rb + R_FULL);
    M.ukeys = H.akeys.p;
    M.utags = H.atags.p;
    M.nu = G.cap_u[r];
    M.nu_dev = slot(rb + R_NU);
    M.u_stored = 0;
    M.okeys = V.keys2.p;
    M.otags = V.tags2.p;
    M.ostamp = stamps ? V.stamps2.as<u32>() : nullptr;
    M.rkeys = H.nkeys.p;
    M.rtags = H.ntags.p;
    M.stamp = 1;
    M.stamp_dev = slot(S_K);
    M.counts_dev = slot(rb + R_DUPS);
    M.rcap = G.cap_r[r];
    diff_merge(M, e.scratch.p, st);
    e.check(cudaGetLastError(), "difference+merge");
    mark((rtag + "_merge").c_str());
    for (size_t j = 0; j < G.views[r].size(); j++) {
      ViewSt& W = H.views[G.views[r][j].view];
      const int vb = view_base(r, G.views[r][j].slot);
      const u64 nu = G.cap_r[r];
      repack_keys(L, V.perm, W.lay, W.perm, H.nkeys.p, e.tmp_keys.p, nu, st, slot(rb + R_NR), nxt(grecent(r)));
      if (sb) copy_elems(e.tmp_tags.p, H.ntags.p, nu, sb, slot(rb + R_NR), st, nxt(grecent(r)) + 1);
      void* k = e.tmp_keys.p;
      void* t = e.tmp_tags.p;
      sort_pairs(W.lay.key64, sb, &k, &t, e.tmp_keys2.p, e.tmp_tags2.p, nu, W.lay.bits, e.opt_radix_bits, e.scratch.p,
                 st, slot(rb + R_NR));
      e.check(cudaGetLastError(), "view sort");
      mark((rtag + "_view_sort").c_str());
      MergeArgs M2{};
      M2.sem = ks;
      M2.key64 = W.lay.key64;
      M2.fkeys = W.keys.p;
      M2.ftags = W.tags.p;
      M2.fstamp = stamps ? W.stamps.as<u32>() : nullptr;
      M2.f_pp = cur(gview(r, G.views[r][j].view));
      M2.o_pp = nxt(gview(r, G.views[r][j].view));
      M2.skip_empty = 1;
      M2.nf = G.cap_view[r][j];
      M2.nf_dev = slot(vb);
      M2.ukeys = k;
      M2.utags = t;
      M2.nu = nu;
      M2.nu_dev = slot(rb + R_NR);
      M2.u_stored = 1;
      M2.okeys = W.keys2.p;
      M2.otags = W.tags2.p;
      M2.ostamp = stamps ? W.stamps2.as<u32>() : nullptr;
      M2.stamp = 1;
      M2.stamp_dev = slot(S_K);
      M2.counts_dev = slot(vb + 1);
      diff_merge(M2, e.scratch.p, st);
      e.check(cudaGetLastError(), "view merge");
      mark((rtag + "_view_merge").c_str());
    }
    });
  }
  (void)cb;
  k_iter_end<<<1, 32, 0, st>>>(G.d, st_dev);
  e.check(cudaGetLastError(), "iteration end");
  mark("loop_end");
}

u64 count_kernels(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  u64 k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
  }
  return k;
}

struct GraphHolder {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  ~GraphHolder() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
  }
};

}  // namespace

// Run iterations k+1, ... on the device until the fixpoint, max_iters, or a
// capacity overflow (handled here by growing and launching again).  Returns
// LOB_OK or LOB_E_MAXITER and advances k and the statistics; false in
// *taken when the loop cannot take this run (the host loop continues).
int run_device_loop(lob_engine& e, u32& k, u32 max_iters, lob_stats& s, bool* taken) {
  *taken = false;
  if (!loop_eligible(e) || k >= max_iters) return LOB_OK;
  if (e.opt_driver == 1 && !e.loop_caps.count("history")) {
    // this run stays host-driven and records the sizes the loop will plan with
    e.loop_caps["history"] = 1;
    return LOB_OK;
  }
  *taken = true;
  g_cap_floor = (u64)e.opt_loop_cap_floor;
  GLoop G;
  plan_loop(e, G, max_iters);
  initial_caps(e, G);
  u32 rec_cap = std::min<u32>(max_iters, std::max<u32>(k + 256, 1024));
  KernelProfiler* prof = g_prof;
  struct ProfOff {  // events cannot be recorded into a captured graph
    KernelProfiler* saved;
    ~ProfOff() { g_prof = saved; }
  } prof_off{prof};
  g_prof = nullptr;
  G.timing = prof != nullptr;
  constexpr int kMaxPhases = 256;
  if (G.timing) {
    e.ensure(G.times, (kMaxPhases + 1) * 8);
    e.check(cudaMemsetAsync(G.times.p, 0, (kMaxPhases + 1) * 8, e.stream), "phase times");
  }
  int rc = LOB_OK;
  // the graph is captured on a private stream (the engine's stream may be the
  // legacy default stream, which cannot be captured) and launched on the engine's
  if (!e.capture_stream) e.check(cudaStreamCreateWithFlags(&e.capture_stream, cudaStreamNonBlocking), "capture stream");
  cudaStream_t cap = e.capture_stream;
  if (!e.capture_stream2) e.check(cudaStreamCreateWithFlags(&e.capture_stream2, cudaStreamNonBlocking), "capture stream");
  cudaStream_t cap2 = e.capture_stream2;
  for (int round = 0;; round++) {
    if (round > 64) throw LobError(LOB_E_CUDA, "internal error: device loop capacities did not settle");
    G.d.rec_cap = rec_cap;
    allocate(e, G);
    for (int r = 0; r < G.d.nrel; r++) {
      G.d.cap_full[r] = G.cap_full[r];
      G.d.cap_u[r] = G.cap_u[r];
      G.d.cap_r[r] = G.cap_r[r];
      G.d.need_full[r] = G.need_full[r];
      G.d.need_u[r] = G.need_u[r];
      G.d.need_r[r] = G.need_r[r];
      for (size_t j = 0; j < G.views[r].size(); j++) {
        G.d.cap_view[r][j] = G.cap_view[r][j];
        G.d.need_view[r][j] = G.need_view[r][j];
      }
    }
    G.d.cap_bind = G.cap_bind;
    G.d.cap_outputs = G.cap_tiles * (u64)kEmitTile;
    G.d.need_bind = G.need_bind;
    G.d.need_tiles = G.need_tiles;
    e.ensure(G.rec, (size_t)rec_cap * G.d.nrel * 16);
    // state block: sizes as the host holds them after iteration k
    std::vector<u64> h(G.n_slots, 0);
    h[S_K] = k;
    for (int r = 0; r < G.d.nrel; r++) {
      const RelSt& R = e.rels[r];
      h[rel_base(r) + R_FULL] = R.views[0].n;
      h[rel_base(r) + R_RECENT] = R.n_recent;
      for (auto& gv : G.views[r]) h[view_base(r, gv.slot)] = R.views[gv.view].n;
    }
    for (int g = 0; g < G.d.ngroups; g++) h[G.d.par_base + g] = 0;
    e.check(cudaMemcpyAsync(G.state.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, e.stream), "loop state");
    // pointer table: both buffers of every group
    std::vector<void*> tab((size_t)ptr_slot(G.d.ngroups, 0), nullptr);
    for (int g = 0; g < G.d.ngroups; g++)
      for (int b = 0; b < 2; b++) group_buffers(e, G, g, b, &tab[ptr_slot(g, b)]);
    e.ensure(G.tab, std::max<size_t>(tab.size(), 1) * sizeof(void*));
    e.ensure(G.res, std::max<size_t>(tab.size(), 1) * sizeof(void*));
    if (!tab.empty())
      e.check(cudaMemcpyAsync(G.tab.p, tab.data(), tab.size() * sizeof(void*), cudaMemcpyHostToDevice, e.stream),
              "pointer table");
    u64* st_dev = G.state.as<u64>();
    u64* rec_dev = G.rec.as<u64>();
    // WHILE { one iteration }.  The WHILE handle starts at 0 and a kernel ahead
    // of the node sets it from the state block, as the body's last kernel does
    // after every pass: if a value were never set, the loop would not start,
    // rather than not end.
    GraphHolder gh;
    e.check(cudaGraphCreate(&gh.g, 0), "graph");
    cudaGraphConditionalHandle hw;
    e.check(cudaGraphConditionalHandleCreate(&hw, gh.g, 0, cudaGraphCondAssignDefault), "while handle");
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    e.check(cudaStreamBeginCaptureToGraph(cap, gh.g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture");
    {
      cudaGraph_t top = nullptr;
      try {
        k_set_cond<<<1, 32, 0, cap>>>(st_dev, hw);
        e.check(cudaGetLastError(), "condition");
        cudaStreamCaptureStatus cstat;
        const cudaGraphNode_t* deps = nullptr;
        const cudaGraphEdgeData* edata = nullptr;
        size_t ndeps = 0;
        e.check(cudaStreamGetCaptureInfo(cap, &cstat, nullptr, nullptr, &deps, &edata, &ndeps), "capture info");
        e.check(cudaGraphAddNode(&wnode, gh.g, deps, edata, ndeps, &wp), "while node");
        e.check(cudaStreamUpdateCaptureDependencies(cap, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies),
                "capture dependencies");
      } catch (...) {
        cudaStreamEndCapture(cap, &top);
        cudaGetLastError();
        throw;
      }
      e.check(cudaStreamEndCapture(cap, &top), "end capture");
    }
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    std::vector<cudaGraph_t> if_bodies;
    e.check(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture");
    try {
      capture_iteration(e, G, st_dev, rec_dev, cap, cap2, if_bodies);
      k_set_cond<<<1, 32, 0, cap>>>(st_dev, hw);
      e.check(cudaGetLastError(), "condition");
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(cap, &dummy);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t captured = nullptr;
    e.check(cudaStreamEndCapture(cap, &captured), "end capture");
    u64 per_iter = count_kernels(body);  // guarded sections counted as if they all ran
    for (cudaGraph_t b : if_bodies) per_iter += count_kernels(b);
    e.check(cudaGraphInstantiate(&gh.x, gh.g, 0), "instantiate");
    e.check(cudaGraphLaunch(gh.x, e.stream), "graph launch");
    std::vector<u64> out(G.n_slots);
    e.check(cudaMemcpyAsync(out.data(), G.state.p, out.size() * 8, cudaMemcpyDeviceToHost, e.stream), "loop state");
    e.sync();
    s.graph_launches++;
    const u64 ran = out[S_ITERS];
    e.launches += ran * per_iter;
    if (out[S_ERR] & kErrLocOverflow)
      throw LobError(LOB_E_ARG, "join step: 1024 consecutive input rows have 2^32 or more matches");
    // the iterations' records for the backward pass
    const u64 k_end = out[S_K];
    if (k_end > k) {
      std::vector<u64> rec((k_end - k) * G.d.nrel * 2);
      e.check(cudaMemcpyAsync(rec.data(), rec_dev + (u64)k * G.d.nrel * 2, rec.size() * 8, cudaMemcpyDeviceToHost,
                              e.stream), "loop record");
      e.sync();
      for (u64 it = 0; it < k_end - k; it++) {
        e.iter_counts.emplace_back();
        for (int r = 0; r < G.d.nrel; r++)
          e.iter_counts.back().emplace_back(rec[2 * (it * G.d.nrel + r)], rec[2 * (it * G.d.nrel + r) + 1]);
      }
    }
    // each group's committed state is in the buffer its parity names
    for (int r = 0; r < G.d.nrel; r++) {
      if (!G.d.rel_dense[r]) continue;
      RelSt& R = e.rels[r];
      const int g0 = G.d.rel_group[r], nv = (int)G.views[r].size();
      auto flip = [](ViewSt& W) {
        std::swap(W.keys, W.keys2);
        std::swap(W.tags, W.tags2);
        std::swap(W.stamps, W.stamps2);
      };
      if (out[G.d.par_base + g0] & 1) flip(R.views[0]);
      for (int j = 0; j < nv; j++)
        if (out[G.d.par_base + g0 + 1 + j] & 1) flip(R.views[G.views[r][j].view]);
      if (out[G.d.par_base + g0 + 1 + nv] & 1) {
        std::swap(R.rkeys, R.nkeys);
        std::swap(R.rtags, R.ntags);
      }
    }
    for (int r = 0; r < G.d.nrel; r++) {
      RelSt& R = e.rels[r];
      R.views[0].n = out[rel_base(r) + R_FULL];
      R.n_recent = out[rel_base(r) + R_RECENT];
      for (auto& gv : G.views[r]) R.views[gv.view].n = out[view_base(r, gv.slot)];
      for (auto& W : R.views)
        if (R.idb)
          for (auto& kv : W.index) kv.second.valid = false;
    }
    k = (u32)k_end;
    s.new_facts += out[S_NEW];
    e.cand_emitted += out[S_EMITTED];
    s.device_iterations += (u32)ran;
    const u64 stop = out[S_STOP];
    if (stop == STOP_FIXPOINT) break;
    if (stop == STOP_MAXITER) {
      rc = LOB_E_MAXITER;
      break;
    }
    if (stop == STOP_RECORD) {
      rec_cap = std::min<u32>(max_iters, rec_cap * 2);
      continue;
    }
    if (stop != STOP_OVERFLOW) throw LobError(LOB_E_CUDA, "internal error: device loop stopped without a reason");
    // grow what overflowed; the aborted iteration's accumulators are cleared
    auto grow = [&](u64& cap, int need) {
      if (out[need] > cap) cap = round_cap(2 * out[need]);
    };
    for (int r = 0; r < G.d.nrel; r++) {
      grow(G.cap_full[r], G.need_full[r]);
      grow(G.cap_u[r], G.need_u[r]);
      grow(G.cap_r[r], G.need_r[r]);
      for (size_t j = 0; j < G.views[r].size(); j++) grow(G.cap_view[r][j], G.need_view[r][j]);
      RelSt& R = e.rels[r];
      if (R.dense) {
        e.check(cudaMemsetAsync(R.dacc.p, 0, R.dacc.cap, e.stream), "dense accumulator");
        e.check(cudaMemsetAsync(R.dtouched.p, 0, R.dtouched.cap, e.stream), "dense bitmap");
      }
    }
    if (out[G.need_bind] > G.cap_bind) G.cap_bind = round_cap(2 * out[G.need_bind]);
    if (out[G.need_tiles] > G.cap_tiles * (u64)kEmitTile) G.cap_tiles = 2 * ((out[G.need_tiles] + kEmitTile - 1) / kEmitTile);
  }
  remember_caps(e, G);
  if (G.timing && prof) {  // the phases' totals join the kernel profile (ms; no algorithmic bytes)
    if (G.phases.size() > (size_t)kMaxPhases) throw LobError(LOB_E_CUDA, "internal error: too many loop phases");
    std::vector<u64> t(kMaxPhases + 1);
    e.check(cudaMemcpyAsync(t.data(), G.times.p, t.size() * 8, cudaMemcpyDeviceToHost, e.stream), "phase times");
    e.sync();
    auto* ep = static_cast<EngineProfiler*>(prof);
    for (size_t i = 0; i < G.phases.size(); i++) {
      ProfAgg& a = ep->agg[G.phases[i]];
      a.launches += s.device_iterations;
      a.ms += t[1 + i] / 1e6;
    }
    e.release(G.times);
  }
  e.release(G.state);
  e.release(G.rec);
  e.release(G.tab);
  e.release(G.res);
  return rc;
}
