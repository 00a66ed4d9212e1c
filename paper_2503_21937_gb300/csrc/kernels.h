// Host-callable launch wrappers of the engine's kernels (internal interface
// between the host driver and the kernel translation units).
#pragma once
#include <type_traits>
#include "common.cuh"

// ---------------------------------------------------------------------------
// per-kernel timing (CUDA events on the launching stream), enabled per engine
// ---------------------------------------------------------------------------
struct KernelProfiler {
  virtual void begin(const char* name, cudaStream_t st) = 0;
  // `bytes`: algorithmic bytes of this launch (what the step must read + write)
  virtual void end(const char* name, double bytes, cudaStream_t st) = 0;
  // more algorithmic bytes for the last finished launch (known only after it ran)
  virtual void add_last_bytes(double bytes) = 0;
  virtual ~KernelProfiler() {}
};
extern thread_local KernelProfiler* g_prof;
struct ProfScope {
  const char* name;
  double bytes;
  cudaStream_t st;
  ProfScope(const char* n, double b, cudaStream_t s) : name(n), bytes(b), st(s) {
    if (g_prof) g_prof->begin(name, st);
  }
  ~ProfScope() {
    if (g_prof) g_prof->end(name, bytes, st);
  }
};

// ---------------------------------------------------------------------------
// radix sort (sort.cu)
// ---------------------------------------------------------------------------
int sort_supported_radix_bits(int rb);
size_t sort_scratch_bytes(u64 n, int rb);
// Stable LSD sort of n (key, payload) pairs on the low `bits` key bits.  keys,
// pay point at the input and are updated to whichever buffer holds the result
// (the inputs or ktmp/ptmp).  pay_bytes is 0 (no payload), 4 or 8.
void sort_pairs(int key64, int pay_bytes, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits, int rb,
                void* scratch, cudaStream_t st, const u64* n_dev = nullptr);
int sort_kernel_launches(u64 n, int bits, int rb);
// Same result with one kernel per digit pass (decoupled look-back); *err is set
// (never cleared) if a bounded wait gave up, in which case the output is invalid.
size_t sort_onesweep_scratch_bytes(u64 n, int rb);
void sort_pairs_onesweep(int key64, int pay_bytes, void** keys, void** pay, void* ktmp, void* ptmp, u64 n, int bits,
                         int rb, void* scratch, u32* err, cudaStream_t st);
int sort_onesweep_launches(u64 n, int bits, int rb);

// ---------------------------------------------------------------------------
// unique, difference + merge, load normalisation (dedup.cu)
// ---------------------------------------------------------------------------
size_t unique_scratch_bytes(u64 n);
// Sorted (keys, Cand tags) -> unique keys with (+)-reduced Cand tags; invalid
// keys dropped; *count_dev receives the unique count.
void unique_run(int sem, int key64, const void* keys, const void* tags, u64 n, void* okeys, void* otags, u64* count_dev,
                void* scratch, cudaStream_t st);

struct MergeArgs {
  int sem, key64;
  const void* fkeys; const void* ftags; const u32* fstamp; u64 nf;  // F: sorted, unique, Stored tags
  const void* ukeys; const void* utags; u64 nu; int u_stored;       // U: sorted, unique; Cand tags unless u_stored
  void* okeys; void* otags; u32* ostamp;                            // F' (room for nf + nu)
  void* rkeys; void* rtags;                                         // R: new or improved facts (nullable)
  u32 stamp;                                                        // stamp of new / improved facts
  u64* counts_dev;                                                  // [0] = #dups of U in F, [1] = |R|, [2] = error flag
  // device-resident sizes (a captured iteration): |F| = *nf_dev, |U| = *nu_dev,
  // with nf and nu the capacities the launches are sized for
  const u64* nf_dev; const u64* nu_dev;
  const u64* stamp_dev;  // when set, new / improved facts get the stamp *stamp_dev + stamp
  u64 rcap;              // when non-zero, R entries past it are not written (the caller checks |R| against it)
  // device-resident buffer pointers: when set, f_pp[0..2] replace fkeys / ftags /
  // fstamp, o_pp[0..2] okeys / otags / ostamp and r_pp[0..1] rkeys / rtags
  void* const* f_pp; void* const* o_pp; void* const* r_pp;
  int skip_empty;        // with U empty, F and U are not read and nothing is written but counts_dev (all 0)
};
size_t merge_scratch_bytes(u64 nf, u64 nu);
void diff_merge(const MergeArgs& a, void* scratch, cudaStream_t st);

// Merge two sorted lists of distinct keys with candidate tags into one,
// combining the tags of a key present in both with (+).  count_dev[0] = number
// of keys present in both (result size = na + nb - that), count_dev[1] = error
// flag (non-zero: the inputs were not sorted; the output is not trustworthy).
size_t combine_scratch_bytes(u64 na, u64 nb);
void combine_merge(int sem, int key64, const void* akeys, const void* atags, u64 na, const void* bkeys,
                   const void* btags, u64 nb, void* okeys, void* otags, u64* count_dev, void* scratch, cudaStream_t st);

struct LoadUniqueArgs {
  int sem, key64;
  const void* keys; const u32* rows; u64 n;  // sorted (key, row) pairs
  const float* raw_tags; u32 id_base; int differentiable;
  void* okeys; void* otags; u32* ostamp; float* row_factor;
  u64* count_dev;
};
void load_unique(const LoadUniqueArgs& a, void* scratch, cudaStream_t st);

// ---------------------------------------------------------------------------
// joins and projections (join.cu)
// ---------------------------------------------------------------------------
enum ColOp : int8_t { OP_BIND = 0, OP_CHECK_SLOT = 1, OP_CHECK_CONST = 2 };
struct ColAct {
  int8_t op, slot;
  u32 cnst;
};
struct FilterP {
  int8_t a_slot, b_slot, eq;  // slot -1: use the constant
  u32 a_const, b_const;
  uint8_t prog;               // k > 0: the filter is bytecode program k - 1 (a comparison); 0: a ==/!= b
};

// Bytecode of computed head arguments and filters (Sec. 5.2: a stack machine,
// one thread per row, a small fixed stack in thread-local memory).  Values are
// u32; +, -, * wrap modulo 2^32, / is unsigned and a zero divisor drops the
// row; comparisons push 1 or 0.  The host checks every program's stack depth.
enum BcOp : uint8_t {
  BC_VAR = 0, BC_CONST, BC_ADD, BC_SUB, BC_MUL, BC_DIV, BC_EQ, BC_NE, BC_LT, BC_LE, BC_GT, BC_GE
};
struct BcIns {
  uint8_t op, slot;
  uint16_t pad;
  u32 imm;
};
constexpr int kMaxCode = 64;   // instructions of one rule
constexpr int kMaxProgs = 16;  // programs of one rule (computed head arguments + comparison filters)
constexpr int kBcStack = 8;
enum { STAMP_NONE = 0, STAMP_LT = 1, STAMP_EQ = 2 };
enum { INDEX_DENSE = 1, INDEX_BSEARCH = 2, INDEX_HASH = 3 };

// One step of a join pipeline: rows of an input table (a packed relation
// segment or a materialised binding table) optionally joined with one
// relation view, filtered, and written as a binding table or as packed head
// keys (candidates).
struct StepParams {
  // input rows
  int in_packed;
  const void* in_keys; Layout in_lay; ColAct in_act[kMaxArity];
  const u32* in_stamp; int in_stamp_mode; u32 in_stamp_val;     // packed input: stamp filter
  int n_in_cols; int8_t in_slot[kMaxSlots]; const u32* in_cols[kMaxSlots];
  const u32* in_sample;                                          // binding tables: sample column, 0xFFFFFFFF = dropped row
  const void* in_tags;                                           // Stored (packed) / Cand (binding) tags
  const u64* in_rowids;                                          // binding tables (backward): per-row fact rows
  u64 n_in;
  int n_in_filters; FilterP in_filters[kMaxFilters];
  // probe
  int has_probe;
  const void* v_keys; Layout v_lay; const void* v_tags; const u32* v_stamp; u64 v_n;
  int v_stamp_mode; u32 v_stamp_val;
  int prefix_len; int8_t prefix_slot[kMaxArity]; u32 prefix_const[kMaxArity];
  ColAct v_act[kMaxArity];
  int index_mode; const u64* dense_offs; u64 dense_domain;  // INDEX_HASH: dense_offs holds the HashSlot table of 2^hash_bits slots
  int hash_bits;
  int n_filters; FilterP filters[kMaxFilters];
  // output
  int out_packed;
  void* out_keys; Layout out_lay; int8_t head_slot[kMaxArity]; u32 head_const[kMaxArity];
  int n_out_cols; int8_t out_slot[kMaxSlots]; u32* out_cols[kMaxSlots];
  u32* out_sample;
  void* out_tags;
  u64 out_base;
  // count / scan products; an emission launch covers outputs [j_begin, j_begin + total)
  u32* cnt; u64* lo; const u64* off; u64 total; u64 j_begin;
  // membership filter (unit semiring): bit `key` of `bitmap` is set for every
  // fact of the head relation and every candidate emitted so far; only
  // candidates that set their bit are written, compacted at out_base + *out_count
  u32* bitmap; u64* out_count;
  // top-1-proofs: the proof arena the tag product (a union of proofs) writes to
  Top1Arena top1;
  // bytecode of the rule: head column j is program head_prog[j] - 1 when
  // head_prog[j] > 0; program k is code[prog_off[k] .. + prog_len[k])
  uint8_t head_prog[kMaxArity];
  uint8_t prog_off[kMaxProgs], prog_len[kMaxProgs];
  BcIns code[kMaxCode];
};

void join_count(int sem, const StepParams& P, cudaStream_t st);
constexpr int kEmitTile = 2048;
// part[t] = last input row whose output range starts at or before j_begin + t * kEmitTile;
// part[ntiles] = the row owning output j_begin + total - 1
void lbs_partition(const u64* off, u64 n_in, u64 j_begin, u64 total, u64* part, cudaStream_t st);
void join_emit(int sem, const StepParams& P, const u64* part, cudaStream_t st);
void project_rows(int sem, const StepParams& P, cudaStream_t st);
// set the bit of every key of a sorted view in a membership bitmap
void bitmap_set_keys(const void* keys, int key64, u64 n, u32* bitmap, cudaStream_t st);

// Sorted keys from membership bitmaps of nbits bits (bitset.cu).  bits_count
// counts the bits of a (of a & ~b when b is given) into *total_dev and places
// them per tile in scratch (bits_scratch_bytes); bits_extract, called next with
// the same a, b and scratch, writes those bits' keys in increasing order to out
// (n_out of them) and sets b |= a.  bits_count returns its kernel launches.
size_t bits_scratch_bytes(u64 nbits);
int bits_count(const u32* a, const u32* b, u64 nbits, void* scratch, u64* total_dev, cudaStream_t st);
void bits_extract(const u32* a, u32* b, u64 nbits, int key64, void* out, u64 n_out, void* scratch, cudaStream_t st);
// Dense (+)-accumulation of tagged candidates (bitset.cu).  acc holds one
// candidate tag (dense_cand_bytes) per key of the relation's key space, all 0
// between iterations; `touched` is a bitmap over the same keys.  dense_fold
// (+)-adds candidate (key, tag) pairs into acc and marks their bits (the packed
// join's emission does the same directly).  After bits_count(touched, nullptr,
// ...) has placed the touched keys, dense_extract writes them in increasing
// order with their reduced tags (n_out of them) and resets acc and touched.
int dense_cand_bytes(int sem);
void dense_fold(int sem, int key64, const void* keys, const void* tags, u64 n, void* acc, u32* touched, cudaStream_t st);
// (keys past `cap` are not written, but every touched slot is reset)
void dense_extract(int sem, int key64, u32* touched, void* acc, u64 nbits, void* okeys, void* otags, u64 n_out,
                   void* scratch, cudaStream_t st, u64 cap = ~0ull);
// merge two sorted key lists known to share no key (keys only)
size_t merge_nodup_scratch_bytes(u64 na, u64 nb);
void merge_nodup(int key64, const void* a, u64 na, const void* b, u64 nb, void* out, void* scratch, cudaStream_t st);

// n_dev (optional): the key count in device memory, n its capacity;
// changed_dev (optional): when it holds 0 the view is unchanged and the index is kept
// keys_pp (optional): device slot holding the keys pointer (replaces keys)
// hash index of the view's prefixes of prefix_len columns (and the sample id)
// into a zeroed table of 2^bits HashSlot entries
void build_hash_index(const Layout& L, int prefix_len, const void* keys, u64 n, void* table, int bits, cudaStream_t st);
void build_dense_index(const Layout& L, int prefix_len, const void* keys, u64 n, u64* offs, u64 domain, cudaStream_t st,
                       const u64* n_dev = nullptr, const u64* changed_dev = nullptr, void* const* keys_pp = nullptr);
// copy n elements of elem_bytes (a multiple of 4); n_dev as above; src_pp
// (optional): device slot holding the source pointer
void copy_elems(void* dst, const void* src, u64 n, int elem_bytes, const u64* n_dev, cudaStream_t st,
                void* const* src_pp = nullptr);
// re-encode keys of layout `from` into layout `to`; view column j of `to` is
// relation column perm_to[j], view column j of `from` is relation column perm_from[j]
void repack_keys(const Layout& from, const int* perm_from, const Layout& to, const int* perm_to, const void* in, void* out,
                 u64 n, cudaStream_t st, const u64* n_dev = nullptr, void* const* in_pp = nullptr);
void pack_rows(const Layout& L, const u32* cols, u64 stride, const u32* samples, u64 n, void* keys, u32* rows,
               cudaStream_t st);
void read_rows(int sem, const Layout& L, const int* perm, const void* keys, const void* tags, u64 n, u32* cols,
               u64 stride, float* otags, u32* samples, cudaStream_t st);
void reduce_max_u32(const u32* a, u64 n, u32* out_dev, cudaStream_t st);
void gather_cand_tags(int sem, const void* stored, const u64* idx, u64 n, void* out, cudaStream_t st);

// top-1-proofs (top1.cu).  The arena: word 0 the empty proof, words 1 + 2i and
// 2 + 2i the singleton proof of input-fact id i (top1_init_arena writes both),
// then the proofs joins append.
void top1_init_arena(u32* words, u64 n_ids, cudaStream_t st);
void fill_f32(float* a, u64 n, float v, cudaStream_t st);
void set_u64_dev(unsigned long long* p, u64 v, cudaStream_t st);
// per fact, the length of the proof its tag points to
void top1_proof_lengths(const u64* tags, u64 n, const u32* words, u32* lens, cudaStream_t st);
// per fact, its proof's ids copied to out + off[i]
void top1_copy_proofs(const u64* tags, u64 n, const u32* words, const u64* off, u32* out, cudaStream_t st);
// gradient of every output's proof probability, added to the input rows
constexpr int kTop1GradRels = 64;
struct Top1GradTable {
  int n;
  u32 base[kTop1GradRels];
  u32 count[kTop1GradRels];
  float* grad[kTop1GradRels];
};
void top1_grad_scatter(const u64* tags, const float* g, u64 n, const u32* words, const float* prob,
                       const Top1GradTable& T, cudaStream_t st);
