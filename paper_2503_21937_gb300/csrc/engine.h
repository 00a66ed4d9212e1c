// Host-side state of one fixpoint engine (internal).
#pragma once
#include <algorithm>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/lobster.h"
#include "kernels.h"
#include "pjoin.h"

struct LobError : std::runtime_error {
  int code;
  LobError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// ---------------------------------------------------------------------------
// rules
// ---------------------------------------------------------------------------
struct Term {
  bool var = false;
  u32 v = 0;  // slot or constant
};
struct AtomAst {
  u32 rel = 0;
  std::vector<Term> args;
};
struct FilterAst {
  Term a, b;
  bool eq = false;
  int prog = 0;            // k > 0: a comparison compiled to bytecode program k - 1 (a, b unused)
  std::vector<u32> vars;   // the variables a bytecode filter reads
};
struct RuleAst {
  std::string text;
  AtomAst head;            // a computed head argument holds a placeholder constant here
  std::vector<AtomAst> body;
  std::vector<FilterAst> filters;
  std::vector<std::string> var_names;
  // bytecode (Sec. 5.2): computed head arguments and comparison filters
  std::vector<BcIns> code;
  std::vector<std::pair<int, int>> progs;  // (first instruction, length)
  std::vector<int> head_prog;              // per head argument: k > 0 = program k - 1
  std::vector<u32> head_vars;              // variables read by computed head arguments
  bool computes() const { return !progs.empty(); }
};

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct IndexSt {
  int mode = 0;  // INDEX_DENSE / INDEX_BSEARCH / INDEX_HASH
  u64 domain = 0;
  int hash_bits = 0;  // INDEX_HASH: the table (in offs) has 2^hash_bits slots
  bool valid = false;
  DevBuf offs;
};

struct ViewSt {
  int perm[kMaxArity] = {0};
  Layout lay{};
  DevBuf keys, tags, stamps;     // current sorted rows
  DevBuf keys2, tags2, stamps2;  // merge target
  u64 n = 0;
  bool probed = false;
  bool probed_late = false; // probed by an arm that can run after iteration 1
  bool maintained = false;  // merged with new facts every iteration
  bool stale = false;       // behind the primary view; rebuilt before its next probe
  std::map<int, IndexSt> index;  // by prefix length
};

struct RelSt {
  std::string name;
  u32 arity = 0;
  bool idb = false;
  // loaded input rows, columnar, in load order
  std::vector<DevBuf> in_cols;
  DevBuf in_tags, in_samples;
  u64 n_in = 0, in_cap = 0;
  bool in_has_tags = false, in_has_samples = false;
  std::vector<u64> in_chunks_tagged;  // (row_begin, row_end, tagged) triples flattened
  int width[kMaxArity] = {0};
  std::vector<ViewSt> views;  // [0] = primary (identity permutation)
  DevBuf rkeys, rtags;        // recent (primary layout)
  u64 n_recent = 0;
  DevBuf nkeys, ntags;        // next recent
  u64 n_next = 0;
  DevBuf ckeys, ctags, ckeys2, ctags2;  // candidates + sort ping-pong
  u64 n_cand = 0;
  DevBuf akeys, atags, akeys2, atags2;  // unique candidates of the flushed chunks of this iteration
  u64 n_acc = 0;
  bool flushed = false;
  // membership filter at emission (unit semiring): bitmap over the key space
  DevBuf bitmap;
  DevBuf prev_bitmap;       // the bitmap as the iteration started (bitmap delta mode)
  bool extract = false;     // this iteration: new facts only set bits; read out of bitmap & ~prev_bitmap
  bool touched = false;     // this iteration emitted into the bitmap
  bool keys_stale = false;  // primary view keys not materialised (the bitmaps hold the relation)
  bool filter_on = false;
  bool unfiltered = false;  // this iteration appended candidates that bypassed the filter
  // dense (+)-accumulation (tagged semirings, small key spaces): candidates are
  // (+)-added into dacc[key] and marked in dtouched instead of being written,
  // sorted and uniqued; the iteration's unique candidates are read out in key order
  bool dense = false;
  DevBuf dacc, dtouched;
  u64 last_cand = 0, last_new = 0, cand_iter = 0;
  // gradient routing of loaded rows
  DevBuf row_factor, row_keys;
  u32 id_base = 0;
};

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
struct StepPlan {
  int atom = -1;
  int view = 0;
  int prefix_len = 0;
  int8_t prefix_slot[kMaxArity];
  u32 prefix_const[kMaxArity];
  ColAct act[kMaxArity];
  bool probe_old = false;
  std::vector<int> filters;
  std::vector<int> live;  // slots materialised after this step
};
// The same arm compiled for the packed kernels (pjoin.cu): per probe step (or
// the single projection) a PStep template whose pointers are filled per launch.
struct PackedArm {
  bool ok = false;
  std::vector<PStep> steps;
  // two probes where the second is keyed by the delta row alone: the second
  // probe compiled against the delta row (word 0), the first probe's key
  // (word 1) and its own key (word 3), for the fused cross-product step
  bool cross_ok = false;
  PStep cross;
};
struct ArmPlan {
  int delta = 0;
  std::vector<StepPlan> steps;
  std::vector<u32> before_rels;  // relations of body atoms before the delta atom
  PackedArm packed;
};
struct RulePlan {
  RuleAst ast;
  std::vector<ArmPlan> arms;
  int stratum = 0;  // the stratum its head belongs to (0 when the run uses one loop)
};

struct ProfAgg {
  u64 launches = 0;
  u64 cand_emitted = 0;  // candidates emitted by the joins of the current run
  double ms = 0, bytes = 0;
};
struct EngineProfiler : KernelProfiler {
  struct Open {
    const char* name;
    cudaEvent_t a;
  };
  struct Done {
    std::string name;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Open> open;
  std::vector<Done> done;
  std::map<std::string, ProfAgg> agg;
  cudaEvent_t take();
  void begin(const char* name, cudaStream_t st) override;
  void end(const char* name, double bytes, cudaStream_t st) override;
  void add_last_bytes(double bytes) override;
  void flush();
  ~EngineProfiler();
};

struct lob_engine {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;  // engine-owned pool; freed blocks stay reserved for reuse
  lob_alloc alloc{};
  bool custom_alloc = false;
  std::string err;
  size_t live_bytes = 0, peak_bytes = 0;
  std::vector<RelSt> rels;
  std::map<std::string, u32> rel_ids;
  std::vector<RuleAst> rules;
  std::vector<RulePlan> plans;
  // options
  int opt_join_index = 0, opt_dense_bits = 24, opt_radix_bits = 8, opt_sync_check = 0, opt_profile = 0;
  int opt_hash_slots = 2;         // hash index: slots per view row at least (load factor <= 1 / opt_hash_slots)
  u64 opt_max_cand = 1ull << 30;  // candidates sorted at once (bounds every sort below 2^32 keys)
  int opt_emit_filter = 1;        // unit semiring: membership bitmap at emission when duplicates dominate
  int opt_sort_algo = 0;          // 0: reduce-then-scan passes, 1: one kernel per pass with look-back
  int opt_packed_join = 1;        // packed-word join kernels when an arm's bindings fit 64 bits
  int opt_warp_join = 1;          // unit semiring: warp-balanced packed join steps
  int opt_bitmap_delta = 1;       // filtered relations: 0 never, 1 when predicted cheaper, 2 always read new facts from the bitmap
  int opt_acc_dense = 1;          // tagged semirings: dense (+)-accumulation for head relations of at most opt_acc_bits key bits
  int opt_acc_bits = 28;
  int opt_driver = 1;             // iterations after the first as a device-driven graph when the run qualifies:
                                  // 1 once a host-driven run of the program recorded its sizes, 2 always, 0 never
  int opt_loop_cap_floor = 1 << 16;  // smallest buffer capacity (rows) the device loop plans with
  int opt_packed_backward = 1;    // diff-add-mult backward replays packed arms on the packed kernels
  int opt_cross_join = 1;         // unit semiring: fused cross-product step for two probes keyed by the delta row
  int opt_proof_cap = 300;        // top-1-proofs: longest proof (input facts) a union may produce
  u64 opt_arena_words = 1ull << 22;  // top-1-proofs: free words of a fresh proof arena (it grows on demand)
  std::map<std::string, u64> loop_caps;  // buffer capacities the device loop needed, kept across runs
  u64 host_syncs = 0;             // host waits for the GPU (statistics)
  cudaStream_t capture_stream = nullptr;  // private stream the device loop's graph is captured on (created on first use)
  cudaStream_t capture_stream2 = nullptr; // second private stream: the bodies of the loop's IF guards
  int opt_loop_guards = 1;        // device loop: IF nodes skip idle arms and relations
  EngineProfiler prof;
  // run state
  int state = 0;  // 0 loading, 1 ran
  int semiring = 0;
  int swidth = 0;
  bool ran_diff = false;
  u32 last_iter = 0;
  lob_stats stats{};
  // scratch and transient buffers
  DevBuf scratch, cnt, lo, off, part, counts, tmp_keys, tmp_tags, tmp_keys2, tmp_tags2;
  DevBuf bind[2][kMaxSlots + 2];  // binding tables (cols..., sample, tags) ping-pong
  DevBuf bfact[2][2 * kMaxArity];  // backward: per carried body fact, its row and tag
  std::vector<std::vector<std::pair<u64, u64>>> iter_counts;  // per iteration: (|F|, |recent|) per relation
  // strata of the current run (1: one loop over every rule), and the
  // iterations that begin a stratum after the first (every fact recent)
  int n_strata = 1;
  std::vector<u32> stratum_begin;
  u64* pinned = nullptr;           // host readback slots
  // top-1-proofs: the proof arena (u32 words), its tail and error word
  // (top1_state[0], [1]) and the probability of every input-fact id
  DevBuf arena, top1_state, top1_prob;
  u64 arena_tail = 0, arena_cap = 0;  // host copies, current after every join step
  u64 launches = 0;
  u64 cand_emitted = 0;  // candidates emitted by the joins of the current run

  // memory
  void* dalloc(size_t bytes);
  void dfree(void* p, size_t bytes);
  void ensure(DevBuf& b, size_t bytes, bool keep = false);
  void release(DevBuf& b);
  void release_all();
  // helpers
  void check(cudaError_t e, const char* what);
  void after_launch(const char* what);
  u64 read_u64(const u64* dev);
  void sync();
};

void engine_ensure_index(lob_engine& e, ViewSt& v, int prefix);
// copy a rule's bytecode programs into step parameters
void set_rule_code(const RuleAst& R, StepParams& P);
// device-driven iterations after iteration k (driver.cu)
int run_device_loop(lob_engine& e, u32& k, u32 max_iters, lob_stats& s, bool* taken);
// A size a host-driven iteration reached, kept (with a quarter of slack) so
// that later device-driven runs of the program plan their buffers from it.
inline void note_loop_cap(lob_engine& e, const std::string& key, u64 v) {
  u64& c = e.loop_caps[key];
  c = std::max<u64>(c, v + v / 4);
}

// tag widths and update policy per semiring
inline bool sem_top1(int sem) { return sem == SR_TOP1 || sem == SR_DIFF_TOP1; }
inline int cand_bytes(int sem) { return sem == SR_UNIT ? 0 : (sem == SR_MAX_MIN ? 4 : 8); }
inline int stored_bytes(int sem) { return sem == SR_UNIT ? 0 : (sem == SR_DIFF_MAX_MIN || sem_top1(sem) ? 8 : 4); }
inline bool sem_idempotent(int sem) {
  return sem == SR_UNIT || sem == SR_MAX_MIN || sem == SR_DIFF_MAX_MIN || sem_top1(sem);
}
inline bool sem_stamps(int sem) { return sem == SR_ADD_MULT || sem == SR_DIFF_ADD_MULT; }
// Semirings whose result can depend on running the strata one after another:
// add-mult's tags are fixed when a key first appears, and a top-1 proof kept
// by the improvement policy can rest on a body fact's earlier, since replaced
// proof.  Under unit, max-min and diff-max-min ((+) and (x) a distributive
// lattice) one loop over every rule reaches the same least fixpoint.
inline bool sem_strata(int sem) { return sem_stamps(sem) || sem_top1(sem); }
// the stratum that iteration k belongs to
inline int stratum_of_iter(const std::vector<u32>& begin, u32 k) {
  int s = 0;
  for (u32 b : begin) s += b <= k;
  return s;
}
inline bool begins_stratum(const std::vector<u32>& begin, u32 k) {
  for (u32 b : begin)
    if (b == k) return true;
  return false;
}
inline int sem_kernel(int sem) {
  return sem == SR_DIFF_ADD_MULT ? SR_ADD_MULT : (sem == SR_DIFF_TOP1 ? SR_TOP1 : sem);
}
