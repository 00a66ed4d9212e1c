/*
 * lobster.h -- C ABI of the GB300 semiring-Datalog fixpoint engine.
 *
 * The engine evaluates positive Datalog rules over columnar u32 relations whose
 * tuples carry provenance-semiring tags, by semi-naive fixpoint iteration on
 * one GPU (Lobster, Sec. 3 and Algorithm 1).  Every step of the iteration runs
 * in hand-written CUDA kernels; the host only plans and sequences them.
 *
 * Conventions for every function below:
 *   - The return value is a status: LOB_OK (0) or a negative LOB_E_* code.
 *     No function aborts or exits; lob_last_error() gives a one-line message.
 *   - `mem` says where caller buffers live: LOB_MEM_HOST (pageable or pinned
 *     host memory) or LOB_MEM_DEVICE (device memory of the engine's device).
 *   - The engine copies what it is given and owns all its device state; the
 *     caller keeps ownership of every buffer it passes.
 *   - Work is ordered on the CUDA stream given to lob_create; calls that
 *     return data to the caller synchronise that stream before returning.
 *   - An engine is not thread-safe; use one engine per host thread.
 */
#ifndef LOBSTER_H
#define LOBSTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lob_engine lob_engine;

/* status codes */
#define LOB_OK 0
#define LOB_E_ARG (-1)          /* invalid argument (null pointer, bad arity, duplicate name, ...) */
#define LOB_E_PARSE (-2)        /* rule text does not parse */
#define LOB_E_UNKNOWN_REL (-3)  /* relation id or name not declared */
#define LOB_E_UNSAFE_RULE (-4)  /* head or filter variable not bound by a body atom */
#define LOB_E_OOM (-5)          /* device allocation failed; engine state is unchanged */
#define LOB_E_MAXITER (-6)      /* max_iters reached before the fixpoint; state is kept and readable */
#define LOB_E_TIMEOUT (-7)      /* a bounded device wait gave up; results of the run are invalid */
#define LOB_E_CUDA (-8)         /* a CUDA runtime call failed */
#define LOB_E_CAPACITY (-9)     /* output buffer too small; *n_out holds the required row count */
#define LOB_E_STATE (-10)       /* call not valid in the engine's current state */
#define LOB_E_KEY_WIDTH (-11)   /* a relation's packed key (sample id + columns) needs more than 64 bits */

/* provenance semirings (Sec. 3.1 semiring table; Sec. 3.4 lists the probabilistic ones) */
#define LOB_UNIT 0           /* discrete: every tag is 1 (no tags stored) */
#define LOB_MAX_MIN 1        /* max-min-prob: (+) = max, (x) = min on [0,1] */
#define LOB_ADD_MULT 2       /* add-mult-prob: (+) = min(1, a+b), (x) = a*b on [0,1] */
#define LOB_DIFF_MAX_MIN 3   /* differentiable max-min: gradient 1 to the bounding input fact */
#define LOB_DIFF_ADD_MULT 4  /* differentiable add-mult: exact reverse-mode gradient */
/* top-1-proofs (Sec. 5.3 "Limitations"): a tag is one proof, the set of input
 * facts of one derivation (at most option "proof_cap" of them), with the
 * product of their probabilities.  (x) = union of the proofs, (+) = the likelier
 * proof; an input row loaded without a probability has the empty proof.  The
 * product is taken in FP64 in ascending input-fact id order and rounded once to
 * f32; (+) compares those f32 values, and a fact's proof is replaced only by a
 * strictly likelier one.  Which of two equally likely proofs a key keeps is not
 * fixed.  Proofs are read with lob_read_proofs. */
#define LOB_TOP1_PROOFS 5
#define LOB_DIFF_TOP1_PROOFS 6  /* gradient of each proof's product to the input facts in it */

#define LOB_MEM_HOST 0
#define LOB_MEM_DEVICE 1

/* Optional device allocator.  alloc returns NULL on failure (the engine then
 * reports LOB_E_OOM).  Both are called with the engine's stream. */
typedef struct lob_alloc {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*release)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} lob_alloc;

/* Statistics of the last lob_run_to_fixpoint. */
typedef struct lob_stats {
  uint32_t iterations;      /* iterations executed, counting the final one that found nothing new */
  uint32_t semiring;
  uint64_t derived;         /* facts in relations that are the head of some rule, at the end of the run */
  uint64_t candidates;      /* candidate tuples emitted by all joins, summed over iterations */
  uint64_t new_facts;       /* facts added or improved, summed over iterations */
  uint64_t peak_bytes;      /* peak device memory held by the engine during the run */
  double ms;                /* wall time of the run on the engine's stream (CUDA events) */
  uint64_t kernel_launches; /* kernels launched by the run */
  uint64_t host_syncs;      /* times the host waited for the GPU during the run */
  uint32_t device_iterations; /* iterations run by the device-driven loop (option "driver") */
  uint32_t graph_launches;  /* launches of that loop's graph (1 unless a buffer had to grow) */
  uint64_t proof_words;     /* top-1-proofs: u32 words of the proof arena in use at the end */
  uint32_t strata;          /* strata run one after another (1: one loop over every rule) */
  uint32_t reserved;
} lob_stats;

/* Create an engine on the current CUDA device.  `alloc` may be NULL (stream-
 * ordered cudaMallocAsync is used); `cuda_stream` is a cudaStream_t or NULL
 * for the legacy default stream. */
int lob_create(lob_engine** out, const lob_alloc* alloc, void* cuda_stream);

/* Release all device memory of the engine and the engine itself.  NULL is ignored. */
void lob_destroy(lob_engine* e);

/* Message of the last failing call on this engine ("" if none).  With e == NULL,
 * the message of the last failed lob_create. */
const char* lob_last_error(const lob_engine* e);

/* Declare relation `name` (identifier: letter or '_' then letters, digits, '_')
 * with 1 <= arity <= 8 columns.  Relations are the columnar tables of Sec. 3.3.
 * *rel_id receives the relation's id (0, 1, 2, ... in declaration order).
 * LOB_E_ARG for a duplicate name or bad arity. */
int lob_declare_relation(lob_engine* e, const char* name, uint32_t arity, uint32_t* rel_id);

/* Look up a declared relation by name. */
int lob_relation_id(const lob_engine* e, const char* name, uint32_t* rel_id);

/* Append n input facts to relation `rel` (the `load` of Sec. 3.3's table).
 *   cols       arity x n u32, column-major: column c of row r at cols[c*n + r]
 *   tags       n floats in [0,1], or NULL for tag 1; for the diff semirings a
 *              non-NULL tags array makes these rows differentiable inputs
 *   sample_ids n u32 sample ids (batched evaluation, Sec. 4.3), or NULL for sample 0
 * Rows are numbered in load order across calls; that numbering is the
 * alignment of lob_backward's per-relation gradients.  Duplicate rows are
 * merged with the semiring's (+) when the run starts.  Valid before the first
 * lob_run_to_fixpoint or after lob_reset. */
int lob_load_relation(lob_engine* e, uint32_t rel, const uint32_t* cols, const float* tags,
                      const uint32_t* sample_ids, uint64_t n, int mem);

/* Add one rule, e.g. "path(x,z) :- path(x,y), edge(y,z)."  Terms are variables
 * (identifiers) or u32 decimal constants; the body is a list of atoms and
 * filters `a != b` / `a == b`.  Several rules may share a head (union).  Every
 * head and filter variable must occur in a body atom (LOB_E_UNSAFE_RULE).
 * The RAM operators this covers (Fig. 2): projection with permutation and
 * constants, selection by (in)equality, n-way join, union. */
int lob_add_rule(lob_engine* e, const char* text);

/* Evaluate all rules to the least fixpoint with the given semiring (Algorithm 1
 * with the semi-naive arms of the appendix's Join rule).  At most max_iters
 * iterations run; on LOB_E_MAXITER the partial state stays readable.  A second
 * call needs lob_reset first (LOB_E_STATE).  `stats` may be NULL.
 * Strata (Sec. 3.1; Algorithm 1's loop over the strata of a program): derived
 * relations that depend on one another form a component, and a component runs
 * after every component it reads.  Under the add-mult and top-1-proofs
 * semirings the strata run one after another, each to its own fixpoint, and
 * every fact of the database is recent when a stratum starts; under unit,
 * max-min and diff-max-min, whose least fixpoint does not depend on that
 * order, every rule runs in one loop.  stats->strata gives the count.
 * With option "driver" = 1 (default), a tagged run of one stratum whose
 * derived relations all use dense accumulation and whose recursive rules are
 * packed join pipelines runs its iterations after the first as one CUDA
 * graph: a conditional WHILE node around one iteration, per-relation double
 * buffers chosen through a device pointer table, every size and the stop
 * decision held in device memory, and no host wait between iterations;
 * buffers that turn out too small end the graph early, grow, and the graph is
 * launched again from the last committed iteration. */
int lob_run_to_fixpoint(lob_engine* e, int semiring, uint32_t max_iters, lob_stats* stats);

/* Options chosen by lob_autotune and the timings behind them. */
typedef struct lob_tune_report {
  int32_t packed_join, warp_join, bitmap_delta, join_index, radix_bits, emit_filter;
  uint32_t trials;  /* fixpoint runs timed (warm-up excluded) */
  double first_ms;  /* median run time with the options in force when called */
  double best_ms;   /* median run time with the chosen options */
  int32_t acc_dense, cross_join;
  int32_t hash_slots;  /* hash index: slots per view row at least (option "hash_slots") */
} lob_tune_report;

/* Autotuner for the loaded program (not part of the paper's method).  It picks
 * the engine's strategy options for this program and these inputs by running
 * the fixpoint under candidate settings and timing each run on the engine's
 * stream (CUDA events).  The search is coordinate descent over these knobs:
 *   - packed_join: packed-word vs general join steps;
 *   - join_index: dense offset table vs binary search vs hash table (the join
 *     strategy: offset-table / hash probes vs sorted-merge search);
 *   - hash_slots: the hash table's size per view row (2 or 4, the load
 *     factor of Sec. 5.1's index), when the hash index was kept;
 *   - radix_bits: the sort's digit width;
 *   - for the tagged semirings acc_dense (dense (+)-accumulation vs sorted
 *     candidates);
 *   - for the unit semiring also warp_join (warp-balanced vs tile emission),
 *     bitmap_delta (bitmap read-out vs sorted candidates), emit_filter
 *     (membership filter) and cross_join (fused cross-product step).
 * Tile sizes (emission, merge, unique, sort) are compile-time constants of the
 * kernels and are not searched.
 * Each setting runs `repeats` times (0 = 1) and scores its median run time; a
 * change must win by 2 %.  All settings compute the same relations, so only
 * time decides.  The engine must be loaded and not yet run (LOB_E_STATE
 * otherwise).  On return the chosen options are set, the inputs stay loaded and
 * lob_run_to_fixpoint runs next.  A trial that fails (LOB_E_MAXITER, LOB_E_OOM,
 * ...) ends the search with its status, and the options in force at the call
 * are restored.  `report` may be NULL. */
int lob_autotune(lob_engine* e, int semiring, uint32_t max_iters, uint32_t repeats, lob_tune_report* report);

/* Number of facts of `rel` after the run (or after loading, before it). */
int lob_relation_size(lob_engine* e, uint32_t rel, uint64_t* n);

/* Copy relation `rel` out, sorted by (sample id, column 0, column 1, ...).
 *   cols       arity x capacity u32, column-major with stride `capacity`
 *   tags       capacity floats or NULL (all 1 under LOB_UNIT)
 *   sample_ids capacity u32 or NULL
 * If the relation has more than `capacity` facts nothing is written,
 * *n_out receives the size and LOB_E_CAPACITY is returned.  With mem =
 * LOB_MEM_HOST, buffers that are page-locked and mapped into the device's
 * address space (cudaHostAlloc, cudaHostRegister; checked at both ends of each
 * range) are written directly by the read-out kernel over the host link; other
 * host memory is filled through a device staging buffer and cudaMemcpyAsync. */
int lob_read_relation(lob_engine* e, uint32_t rel, uint32_t* cols, float* tags, uint32_t* sample_ids,
                      uint64_t capacity, uint64_t* n_out, int mem);

/* The proofs of a top-1-proofs run (LOB_STATE otherwise): for fact i of `rel`
 * in lob_read_relation order, lens[i] = the number of input facts in its proof
 * and its ids follow those of facts 0..i-1 in `ids`, ascending.  The id of row
 * q of relation k is q plus the rows loaded into relations 0..k-1 (declaration
 * order).  lens holds lob_relation_size entries (or is NULL); ids holds
 * id_capacity entries (or is NULL); *n_ids (may be NULL) receives the total id
 * count.  When the ids exceed id_capacity nothing is written to ids and
 * LOB_E_CAPACITY is returned.  `mem` says where lens and ids live. */
int lob_read_proofs(lob_engine* e, uint32_t rel, uint32_t* lens, uint32_t* ids, uint64_t id_capacity, uint64_t* n_ids,
                    int mem);

/* Reverse-mode gradient after a LOB_DIFF_* run (Sec. 3.4: differentiable
 * versions of the probabilistic semirings).
 *   grad_tags   d loss / d tag for every fact of out_rel, in lob_read_relation order
 *   grad_inputs array indexed by relation id (length = number of declared
 *               relations); entry k is NULL or points to one float per loaded
 *               row of relation k, in load order; gradients are ADDED there.
 * diff-max-min: each output's gradient goes to the input row that bounds its
 * tag.  diff-top-1-proofs: to every input row of its proof, times the product of
 * the proof's other probabilities.  diff-add-mult: adjoints flow back through every recorded derivation
 * (recomputed per iteration), zero through a clamped (+).  May be called once
 * per output relation; LOB_E_STATE without a diff run. */
int lob_backward(lob_engine* e, uint32_t out_rel, const float* grad_tags, float* const* grad_inputs, int mem);

/* Drop all derived state and loaded facts but keep declarations and rules. */
int lob_reset(lob_engine* e);

/* Engine options (key, value):
 *   "join_index"   0 dense offset table up to dense_bits, else binary
 *                  search; 1 dense up to 30 bits; 2 binary search; 3 a hash
 *                  table of the view's distinct join prefixes (open
 *                  addressing, linear probing, each slot holding the
 *                  prefix's first row and row count)               (default 0)
 *   "hash_slots"   hash index size: the smallest power of two of at least
 *                  this many slots per view row, 2, 4 or 8 (load factor at
 *                  most 1/2, 1/4, 1/8; 16 bytes a slot)              (default 2)
 *   "dense_bits"   largest join-prefix width, in bits, indexed densely (default 24)
 *   "radix_bits"   bits per radix-sort pass: 4, 6 or 8 (other values
 *                  in 4..11 select 8)                                (default 8)
 *   "sync_check"   1: check CUDA errors after every kernel (debug)   (default 0)
 *   "profile"      1: time every kernel launch with CUDA events      (default 0)
 *   "max_candidates" candidates sorted at once; larger candidate sets are
 *                  sorted and deduplicated in chunks (4096..2^31, default 2^30)
 *   "emit_filter"  1: under LOB_UNIT, test candidates against a membership
 *                  bitmap of the relation when they are emitted -- from the
 *                  first iteration for keys of <= 32 bits, and for keys of
 *                  <= 34 bits once most candidates are duplicates; 2: from
 *                  the first iteration for keys of <= 34 bits; 0: never (default 1)
 *   "sort_algo"    0: three kernels per radix pass, no inter-block waiting;
 *                  1: one kernel per pass with decoupled look-back (bounded
 *                  waits; LOB_E_TIMEOUT if one gives up)            (default 0)
 *   "packed_join"  1: join kernels on packed words when an arm's bindings
 *                  fit 64 bits; 0: the general kernels               (default 1)
 *   "warp_join"    1: unit-semiring packed join steps expand 32 input rows
 *                  per warp (no per-row offsets); 2: only bitmap-only last
 *                  steps do; 0: count / offsets / tile emission for every
 *                  step                                              (default 1)
 *   "bitmap_delta" relations with a membership filter: 2 = the joins only
 *                  set bits and each iteration's new facts are read, in key
 *                  order, out of the bitmap and its start-of-iteration copy;
 *                  1 = per iteration, whichever a traffic model predicts
 *                  cheaper: reading the two bitmaps, or sorting the
 *                  predicted new facts (the last iteration's count) and
 *                  merging them / reading the relation's keys out first;
 *                  0 = never (candidates are sorted and merged)      (default 1)
 *   "acc_dense"    1: under the tagged semirings, a derived relation whose
 *                  key has at most acc_bits bits keeps a dense array of one
 *                  candidate tag per key plus a bitmap; join outputs are
 *                  (+)-added into their key's slot (atomics) instead of being
 *                  written, sorted and uniqued, and each iteration's unique
 *                  candidates are read out of the bitmap in key order; 0: never
 *                  (default 1; the array takes 2^acc_bits x 4 or 8 bytes)
 *   "acc_bits"     largest key width, in bits, given a dense accumulator
 *                  (1..30, default 28)
 *   "driver"       1: iterations after the first run as a device-driven
 *                  CUDA graph when the run qualifies (see
 *                  lob_run_to_fixpoint) and an earlier host-driven run of
 *                  this engine recorded the sizes the graph's buffers are
 *                  planned from (the first qualifying run records them);
 *                  2: as 1 without waiting for recorded sizes (the buffers
 *                  start from estimates and grow); 0: the host drives
 *                  every iteration                                   (default 1)
 *   "loop_guards"  1: inside the device-driven loop, every join arm and
 *                  every relation's difference+merge section sits under a
 *                  conditional IF node set by the iteration's first kernel,
 *                  so arms without a recent delta and relations without
 *                  candidates launch nothing; 0: every section launches
 *                  each iteration and exits early on empty input  (default 1)
 *   "loop_cap_floor" smallest row capacity the device-driven loop plans its
 *                  buffers with before they grow (256..2^24, default 65536;
 *                  small values exercise the regrowth path)
 *   "proof_cap"    top-1-proofs: the most input facts a proof may hold; a
 *                  union beyond it ends the run with LOB_E_CAPACITY
 *                  (1 .. 2^20)                                       (default 300)
 *   "proof_arena_words" top-1-proofs: free u32 words of the proof arena
 *                  when a run starts; it doubles whenever a join step runs
 *                  out (that step runs again)        (16 .. 2^31, default 2^22)
 *   "cross_join"   1: under LOB_UNIT, an arm with two probes keyed by the
 *                  delta row alone (same generation: children(a) x
 *                  children(b)) whose new facts only set bitmap bits runs
 *                  as one fused cross-product step; 0: two steps    (default 1)
 *   "packed_backward" 1: the diff-add-mult backward pass replays packed join
 *                  pipelines on the packed kernels (binding words plus the
 *                  rows of the facts matched so far); 0: every arm on the
 *                  general kernels                                   (default 1)
 * LOB_E_ARG for an unknown key or a value out of range. */
int lob_set_option(lob_engine* e, const char* key, int64_t value);

/* Per-kernel timing (engine option "profile" = 1).  Every kernel launch is
 * bracketed by CUDA events on the engine's stream; launches, milliseconds and
 * algorithmic bytes (the bytes the step must read and write, from the sizes
 * it processes) accumulate per kernel name until lob_profile_reset.
 * lob_profile_count synchronises the stream and returns the number of names;
 * lob_profile_entry copies entry i (names in sorted order, NUL-terminated,
 * truncated to name_cap). */
int lob_profile_count(lob_engine* e, uint32_t* n);
int lob_profile_entry(lob_engine* e, uint32_t i, char* name, size_t name_cap, uint64_t* launches, double* ms,
                      double* bytes);
int lob_profile_reset(lob_engine* e);

/* Kernel-level primitives on caller device buffers (mem = device), used by the
 * kernel tests and microbenchmarks.  They use the engine's stream and scratch
 * buffers, leave its relations untouched and synchronise before returning.
 *
 * lob_prim_sort: stable LSD radix sort (the APM `sort`, Sec. 3.2) of n keys
 * (key_bytes 4 or 8) on their low key_bits bits, in place, with an optional
 * payload (payload_bytes 0, 4 or 8) moved along; n < 2^32. */
int lob_prim_sort(lob_engine* e, void* keys, void* payload, uint64_t n, uint32_t key_bits, uint32_t key_bytes,
                  uint32_t payload_bytes);
/* lob_prim_exclusive_scan: out[i] = in[0] + ... + in[i-1] (the APM `scan`);
 * *total (host) = sum of all n inputs. */
int lob_prim_exclusive_scan(lob_engine* e, const uint32_t* in, uint64_t* out, uint64_t n, uint64_t* total);
/* lob_prim_unique: collapse runs of equal keys of a sorted array (the APM
 * `unique<(+)>`), reducing the run's tags with the semiring's (+) (tags:
 * none for LOB_UNIT, f32 for max-min, f64 unclamped sums for the add-mult
 * semirings, u64 (value bits << 32 | 0xFFFFFFFF - id) for diff-max-min).  The
 * all-ones key is treated as absent.  *n_out (host) = number of distinct keys. */
int lob_prim_unique(lob_engine* e, int semiring, const void* keys, const void* tags, uint64_t n, uint32_t key_bytes,
                    void* out_keys, void* out_tags, uint64_t* n_out);
/* lob_prim_diff_merge: with F (sorted, distinct keys, stored tags) and U
 * (sorted, distinct keys, candidate tags as for lob_prim_unique), write
 * out = F merged with the keys of U not in F (for the idempotent semirings a
 * key of U in F replaces F's tag when U's is larger) and r = the new or
 * improved facts of U (the delta-vs-full difference).  out needs room for
 * nf + nu rows, r for nu rows; *n_out and *n_r (host) get their sizes. */
int lob_prim_diff_merge(lob_engine* e, int semiring, const void* f_keys, const void* f_tags, uint64_t nf,
                        const void* u_keys, const void* u_tags, uint64_t nu, uint32_t key_bytes, void* out_keys,
                        void* out_tags, void* r_keys, void* r_tags, uint64_t* n_out, uint64_t* n_r);

/* Allocation-free sort + deduplication of a small batch of rows.  The paper
 * has no counterpart to this call; it exists for callers that cannot allocate
 * device memory when they need the step: latency-critical paths where
 * cudaMalloc / cudaFree would synchronise the device, plug-ins inside an
 * application that owns and budgets all device memory, and processes that have
 * split the GPU's memory among tenants ahead of time.
 *   cols      device memory, arity x n u32, column-major (arity 1 or 2)
 *   out_cols  device memory, arity x n u32, column-major with stride n; gets
 *             the distinct rows in lexicographic order
 *   n_out     device memory, one u64; gets the number of distinct rows
 * The call works in one fixed scratch array compiled into the library (about
 * 4.3 MB, held on every GPU that loads the library until the process exits)
 * and allocates nothing.  n > LOB_NOALLOC_MAX_ROWS returns LOB_E_CAPACITY;
 * a bad arity or a null pointer returns LOB_E_ARG (cols and out_cols may be
 * NULL when n is 0; *n_out then gets 0).  The first call on a device
 * looks up the scratch array's device address; make that first call before
 * any stream capture.  All calls on a device share the scratch array, so
 * calls whose work overlaps on the GPU race: order them (one stream, or
 * events).  A row whose every column is 0xFFFFFFFF is dropped (at arity 1
 * and 2 alike).  The work is
 * queued on cuda_stream (NULL: legacy default stream); the call does not wait. */
#define LOB_NOALLOC_MAX_ROWS 262144u
int lob_unique_rows_noalloc(const uint32_t* cols, uint32_t arity, uint64_t n, uint32_t* out_cols, uint64_t* n_out,
                            void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LOBSTER_H */
