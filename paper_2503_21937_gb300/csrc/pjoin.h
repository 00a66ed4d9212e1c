// Packed join steps (pjoin.cu): rule variables as bit fields of packed words.
#pragma once
#include "kernels.h"

struct POperand {
  uint8_t word;   // 0: input word, 1: matched view key, 2: constant
  uint8_t shift;
  uint8_t width;
  uint8_t pad;
  u32 cval;
};
struct PField {   // operand placed at `shift` of a composed word
  POperand op;
  uint8_t shift;
  uint8_t limit_bits;  // probe prefix: the value must fit this many bits (64: no limit)
};
struct PCheck {
  POperand a, b;
  int8_t eq;
};

constexpr int kMaxPChecks = 16;
constexpr int kMaxPFields = kMaxArity + 1;

struct PStep {
  // input rows: packed relation keys (in_packed, tags are stored tags) or
  // packed binding words (tags are candidate tags)
  int in_packed;
  const void* in_words; int in_w64; const void* in_tags;
  const u32* in_stamp; int in_stamp_mode; u32 in_stamp_val;
  u64 n_in;
  int n_in_checks; PCheck in_checks[kMaxPChecks];
  // probe
  const void* v_keys; int v_key64; const void* v_tags; const u32* v_stamp; u64 v_n;
  int v_stamp_mode; u32 v_stamp_val;
  int n_prefix; PField prefix[kMaxPFields];
  int index_mode; const u64* dense_offs; int rest_shift; int whole_view;  // INDEX_HASH: dense_offs = HashSlot table
  int hash_bits;
  int n_checks; PCheck checks[kMaxPChecks];
  // output word: a head key or a binding word
  void* out_words; int out_w64; void* out_tags; u64 out_base;
  int n_out; PField out[kMaxPFields];
  // count / offsets / emission range / membership filter.  Row r's first output
  // is blk_off[r / kLocRows] + loc[r]: loc is local to the row's block of
  // kLocRows rows, blk_off the exclusive scan of the per-block totals.
  u32* loc; u32* lo32; u64* blk_cnt; const u64* blk_off; u32* err;  // view rows < 2^32
  u64 total; u64 j_begin;
  u32* bitmap; u64* out_count;
  // dense (+)-accumulation (tagged semirings): each output's tag is added into
  // acc[output word] and its bit set in `bitmap`; nothing else is written
  void* acc;
  // device-resident sizes (a captured iteration): when set, the row count and
  // the output count are read from device memory; n_in and total are then
  // the capacities the launch grids and buffers were sized for
  const u64* n_in_dev; const u64* total_dev;
  const u64* v_n_dev;     // the probed view's row count (v_n its capacity)
  const u64* stamp_dev;   // when set, the stamp filters compare with *stamp_dev + v_stamp_val
  // device-resident buffer pointers: when set, in_pp[0..1] replace in_words /
  // in_tags and v_pp[0..2] replace v_keys / v_tags / v_stamp (read at kernel start)
  void* const* in_pp; void* const* v_pp;
};

// the input and probed-view pointers of a step, resolved on the device
struct PPtrs {
  const void* in_words; const void* in_tags; const void* v_keys; const void* v_tags; const u32* v_stamp;
};
LOB_DEV PPtrs resolve_ptrs(const PStep& P) {
  PPtrs q{P.in_words, P.in_tags, P.v_keys, P.v_tags, P.v_stamp};
  if (P.in_pp) { q.in_words = P.in_pp[0]; q.in_tags = P.in_pp[1]; }
  if (P.v_pp) { q.v_keys = P.v_pp[0]; q.v_tags = P.v_pp[1]; q.v_stamp = reinterpret_cast<const u32*>(P.v_pp[2]); }
  return q;
}

// size in device memory, capped by the capacity it was launched for
LOB_DEV u64 dev_size(u64 cap, const u64* dev) { return dev ? (*dev < cap ? *dev : cap) : cap; }

constexpr u64 kLocRows = 1024;  // rows per offset block: 256 threads x 4 consecutive rows
constexpr u32 kErrLocOverflow = 1;  // a block's matches reached 2^32

inline u64 pjoin_loc_blocks(u64 n_in) { return (n_in + kLocRows - 1) / kLocRows; }
// count: loc, lo32 and blk_cnt for every input row / block; sets *err on overflow
void pjoin_count(int sem, const PStep& P, cudaStream_t st);
// tile partition of outputs [j_begin, j_begin + total) (needs blk_off): ntiles + 1 row indices
void pjoin_partition(const PStep& P, u64 ntiles, u64* part, cudaStream_t st);
void pjoin_emit(int sem, const PStep& P, const u64* part, cudaStream_t st);
void pjoin_project(int sem, const PStep& P, cudaStream_t st);

// Backward replay of a packed arm (diff-add-mult): the same count / partition
// as the forward steps, then an emission that carries, per binding row, the
// primary-view rows of the body facts matched so far; the last step forms the
// head key, keeps groundings whose head was first derived (unclamped) in the
// replayed iteration, and adds adjoint(head) * (product of the other facts'
// tags) to each body fact's adjoint.
struct PBwd {
  int packed_source;                    // input rows are rows of the delta relation's primary view (fact 0 = row)
  int n_in_facts;                       // facts carried by a binding-row input
  const u32* in_rows[kMaxArity];        // their rows
  u32* out_rows[kMaxArity + 1];         // intermediate step: the rows carried forward (n_in_facts + 1)
  const u32* v_prow;                    // probed view row -> primary row (null: primary view)
  const float* fact_tags[kMaxArity + 1];  // per body fact of the grounding: its relation's tags, by primary row
  double* fact_adj[kMaxArity + 1];      // per body fact: adjoint array (null: no adjoint needed)
  int last;
  const u32* h_new;                     // bitmap of the head keys new (unclamped) in the replayed iteration
  const u32* h_row;                     // dense head key -> primary row (null: binary search of h_keys)
  const void* h_keys; int h_key64; u64 h_n;
  const double* h_adj;
};
void pjoin_backward_emit(const PStep& P, const PBwd& B, const u64* part, cudaStream_t st);
bool pjoin_backward_supported(const PStep& P);  // the emission has a kernel for the step's shape

// Warp-balanced steps (unit semiring).  pjoin_warp_supported: the step has a
// specialised warp kernel.  pjoin_warp_count: outputs per block of 1024 input
// rows (pjoin_warp_blocks(n_in) entries); after an exclusive scan of them into
// blk_off, pjoin_warp_emit writes the step's binding words at [0, total).
// pjoin_warp_bitmap: last step, only sets the bits of P.bitmap and adds the
// step's outputs to *emitted_dev.
bool pjoin_warp_supported(int sem, const PStep& P);
// Fused cross-product last step (see pjoin.cu): A = the first probe's step
// (input rows, probe of view A, its checks on words 0 / 1), B = the second
// probe keyed by the input word alone (its prefix on word 0, its checks and
// the head fields on words 0 / 1 / 3, the bitmap).  Sets membership bits and
// adds the outputs to *emitted_dev.
bool pjoin_cross_supported(const PStep& A, const PStep& B);
void pjoin_warp_cross_bitmap(const PStep& A, const PStep& B, u64* emitted_dev, cudaStream_t st);
u64 pjoin_warp_blocks(u64 n_in);
void pjoin_warp_count(const PStep& P, u64* blk_cnt, cudaStream_t st);
void pjoin_warp_emit(const PStep& P, u64 total, const u64* blk_off, cudaStream_t st);
void pjoin_warp_bitmap(const PStep& P, u64* emitted_dev, cudaStream_t st);
