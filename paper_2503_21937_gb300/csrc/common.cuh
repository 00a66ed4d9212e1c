// Shared device definitions of the fixpoint engine: packed-key layouts, the
// semiring tag arithmetic, and warp/block scan helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

typedef unsigned int u32;
typedef unsigned long long u64;

#define LOB_DEV __device__ __forceinline__
#define LOB_HD __host__ __device__ __forceinline__

constexpr int kMaxArity = 8;
constexpr int kMaxSlots = 16;   // variables of one rule
constexpr int kMaxFilters = 8;

// Every key type's all-ones value is never a valid packed key: each field is
// stored with enough bits that its value is below the field's all-ones value.
// Candidates dropped by a filter carry this key, sort last, and are removed by
// the unique step.
template <class K> LOB_HD K invalid_key() { return ~K(0); }

// Dynamic shared memory above 48 KB is an attribute of one kernel on one
// device.  It is set before every launch that needs it (a cheap host call, no
// stream work), so it holds on every device and from every host thread.  A
// failure is recorded as the runtime's last error, which the launch check that
// follows reports.
template <class T>
inline cudaError_t allow_dynamic_smem(T* kernel, int bytes) {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(kernel), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ---------------------------------------------------------------------------
// packed keys
// ---------------------------------------------------------------------------
// A relation view packs (sample id, c_0, ..., c_{a-1}) into one integer, sample
// in the top field, view column 0 next, the last view column in the low bits,
// so that integer order is the lexicographic order of the columnar table
// (Sec. 3.3: an arity-n relation is n column registers; Sec. 4.3 puts the
// sample register in front).
struct Layout {
  int arity;
  int bits;               // total key bits
  int sshift, swidth;     // sample field (swidth 0: unbatched)
  int shift[kMaxArity];   // view column j
  int width[kMaxArity];
  int key64;              // key stored as u64 (bits > 32) or u32
};

LOB_HD u64 field_of(u64 key, int shift, int width) {
  return (key >> shift) & ((width >= 64) ? ~0ull : ((1ull << width) - 1ull));
}
// number of key bits below the first `p` view columns
LOB_HD int rest_shift(const Layout& L, int p) { return p == 0 ? L.sshift : L.shift[p - 1]; }
LOB_HD u64 shr64(u64 v, int s) { return s >= 64 ? 0ull : (v >> s); }
LOB_HD u64 shl64(u64 v, int s) { return s >= 64 ? 0ull : (v << s); }

LOB_DEV u64 load_key(const void* keys, int key64, u64 i) {
  return key64 ? reinterpret_cast<const u64*>(keys)[i] : (u64)reinterpret_cast<const u32*>(keys)[i];
}
LOB_DEV void store_key(void* keys, int key64, u64 i, u64 v) {
  if (key64) reinterpret_cast<u64*>(keys)[i] = v;
  else reinterpret_cast<u32*>(keys)[i] = (u32)v;
}
LOB_DEV u64 invalid_of(int key64) { return key64 ? ~0ull : 0xFFFFFFFFull; }

// ---------------------------------------------------------------------------
// semirings (Sec. 3.1 table; Sec. 3.4).  `Stored` is the tag kept with a fact;
// `Cand` is the tag carried by candidates and join intermediates.
// ---------------------------------------------------------------------------
enum SemiringId {
  SR_UNIT = 0, SR_MAX_MIN = 1, SR_ADD_MULT = 2, SR_DIFF_MAX_MIN = 3, SR_DIFF_ADD_MULT = 4, SR_TOP1 = 5, SR_DIFF_TOP1 = 6
};

struct SemUnit {
  typedef u32 Stored;
  typedef u32 Cand;
  static constexpr bool kTags = false;
  static constexpr bool kIdempotent = true;
  LOB_DEV static Cand one() { return 1u; }
  LOB_DEV static Cand from_stored(Stored) { return 1u; }
  LOB_DEV static Cand mul(Cand, Cand) { return 1u; }
  LOB_DEV static Cand add(Cand, Cand) { return 1u; }
  LOB_DEV static Stored store(Cand) { return 1u; }
  LOB_DEV static bool better(Stored, Stored) { return false; }
};

// max-min-prob: (+) = max, (x) = min; both exact in f32.
struct SemMaxMin {
  typedef float Stored;
  typedef float Cand;
  static constexpr bool kTags = true;
  static constexpr bool kIdempotent = true;
  LOB_DEV static Cand one() { return 1.0f; }
  LOB_DEV static Cand from_stored(Stored s) { return s; }
  LOB_DEV static Cand mul(Cand a, Cand b) { return fminf(a, b); }
  LOB_DEV static Cand add(Cand a, Cand b) { return fmaxf(a, b); }
  LOB_DEV static Stored store(Cand c) { return c; }
  LOB_DEV static bool better(Stored a, Stored b) { return a > b; }
};

// add-mult-prob: (x) = a*b, (+) = min(1, a+b).  Because every tag is
// non-negative, min(1, .) folded pairwise equals one clamp of the plain sum, so
// candidates carry unclamped FP64 products/sums and the clamp and the single
// rounding to f32 happen when a fact is stored.
struct SemAddMult {
  typedef float Stored;
  typedef double Cand;
  static constexpr bool kTags = true;
  static constexpr bool kIdempotent = false;
  LOB_DEV static Cand one() { return 1.0; }
  LOB_DEV static Cand from_stored(Stored s) { return (double)s; }
  LOB_DEV static Cand mul(Cand a, Cand b) { return a * b; }
  LOB_DEV static Cand add(Cand a, Cand b) { return a + b; }
  LOB_DEV static Stored store(Cand c) { return (float)fmin(1.0, c); }
  LOB_DEV static bool better(Stored, Stored) { return false; }
};

// diff-max-min: a tag is (v, id) ordered by v, ties to the smaller input-fact
// id.  Packed as (bits(v) << 32) | (0xFFFFFFFF - id): v >= 0, so the IEEE bits
// order like the values, and u64 order is the tag order; (+) = max, (x) = min.
struct SemDiffMaxMin {
  typedef u64 Stored;
  typedef u64 Cand;
  static constexpr bool kTags = true;
  static constexpr bool kIdempotent = true;
  LOB_DEV static Cand one() { return ((u64)__float_as_uint(1.0f) << 32) | 0ull; }
  LOB_DEV static Cand from_stored(Stored s) { return s; }
  LOB_DEV static Cand mul(Cand a, Cand b) { return a < b ? a : b; }
  LOB_DEV static Cand add(Cand a, Cand b) { return a > b ? a : b; }
  LOB_DEV static Stored store(Cand c) { return c; }
  LOB_DEV static bool better(Stored a, Stored b) { return a > b; }
};
// top-1-proofs (Sec. 5.3 "Limitations"; Sec. 3.4): a tag is one proof, the
// set of input facts of one derivation, kept in the engine's proof arena as
// [length, ids ascending]; the tag packs (bits(P) << 32) | word offset of the
// proof, where P is the proof's probability.  (+) keeps the likelier proof (u64
// max: equally likely proofs go to the larger offset); a fact is improved only
// when its probability grows.  (x) is the union of two proofs and needs the
// arena, so the join kernels compute it with top1_union (no Sem::mul here).
struct SemTop1 {
  typedef u64 Stored;
  typedef u64 Cand;
  static constexpr bool kTags = true;
  static constexpr bool kIdempotent = true;
  LOB_DEV static Cand one() { return (u64)__float_as_uint(1.0f) << 32; }  // the empty proof, at offset 0
  LOB_DEV static Cand from_stored(Stored s) { return s; }
  LOB_DEV static Cand add(Cand a, Cand b) { return a > b ? a : b; }
  LOB_DEV static Stored store(Cand c) { return c; }
  LOB_DEV static bool better(Stored a, Stored b) { return (a >> 32) > (b >> 32); }
};

// The proof arena of a top-1-proofs run.  Word 0 is the empty proof; proofs
// are appended by bump allocation; a union that does not fit leaves the tail
// past `cap` (the host grows the arena and runs the step again).
struct Top1Arena {
  u32* words;
  unsigned long long* tail;  // next free word
  u64 cap;                   // words allocated (at most 2^32 - 1)
  const float* prob;         // input-fact id -> probability
  u32 proof_cap;             // longest proof allowed
  u32* err;                  // bit 0: a union longer than proof_cap
};

// (x) of two top-1 tags: the union of their proofs, written to the arena, with
// its probability = the FP64 product of its facts' probabilities in ascending
// id order, rounded once to f32.
LOB_DEV u64 top1_union(const Top1Arena& A, u64 a, u64 b) {
  const u32 ra = (u32)a, rb = (u32)b;
  const u32* pa = A.words + ra;
  const u32* pb = A.words + rb;
  const u32 la = pa[0], lb = pb[0];
  if (la == 0 || ra == rb) return b;  // the empty proof is the identity; a proof with itself is itself
  if (lb == 0) return a;
  const u64 need = (u64)la + lb + 1;
  const u64 at = atomicAdd(A.tail, (unsigned long long)need);
  if (at + need > A.cap) return 0;
  u32* out = A.words + at + 1;
  u32 i = 0, j = 0, n = 0;
  double p = 1.0;
  while (i < la || j < lb) {
    u32 x;
    if (j >= lb) x = pa[1 + i++];
    else if (i >= la) x = pb[1 + j++];
    else {
      const u32 xa = pa[1 + i], xb = pb[1 + j];
      x = xa < xb ? xa : xb;
      i += xa <= xb;
      j += xb <= xa;
    }
    out[n++] = x;
    p *= (double)A.prob[x];
  }
  if (n > A.proof_cap) {
    atomicOr(A.err, 1u);
    return 0;
  }
  out[-1] = n;
  return ((u64)__float_as_uint((float)p) << 32) | at;
}

LOB_HD u64 dmm_pack(float v, u32 id) {
#ifdef __CUDA_ARCH__
  u32 b = __float_as_uint(v);
#else
  union { float f; u32 u; } cv; cv.f = v; u32 b = cv.u;
#endif
  return ((u64)b << 32) | (u64)(0xFFFFFFFFu - id);
}
LOB_HD u32 dmm_id(u64 t) { return 0xFFFFFFFFu - (u32)(t & 0xFFFFFFFFull); }
LOB_DEV float dmm_value(u64 t) { return __uint_as_float((u32)(t >> 32)); }

// Dense (+)-accumulation of a candidate tag into slot `key` of a per-key array
// holding candidate tags (every slot starts at 0, the identity of (+) for the
// tagged semirings: tags are non-negative, and 0 is below every packed
// diff-max-min tag).  add-mult: FP64 add; max-min: max of the f32 bit patterns
// (non-negative floats order like their bits); diff-max-min: max of the packed
// u64 tags.  A slot whose tag cannot grow is left alone without an atomic.
template <class Sem>
LOB_DEV void dense_add(void* acc, u64 key, typename Sem::Cand t) {
  if constexpr (std::is_same<Sem, SemAddMult>::value) {
    atomicAdd(reinterpret_cast<double*>(acc) + key, t);
  } else if constexpr (std::is_same<Sem, SemMaxMin>::value) {
    int* a = reinterpret_cast<int*>(acc) + key;
    const int v = __float_as_int(t);
    if (*reinterpret_cast<volatile int*>(a) < v) atomicMax(a, v);
  } else if constexpr (std::is_same<Sem, SemDiffMaxMin>::value) {
    unsigned long long* a = reinterpret_cast<unsigned long long*>(acc) + key;
    if (*reinterpret_cast<volatile unsigned long long*>(a) < t) atomicMax(a, (unsigned long long)t);
  }
}
// mark `key` as touched in this iteration's bitmap (no atomic when already set)
LOB_DEV void touch_bit(u32* bm, u64 key) {
  const u32 bit = 1u << (u32)(key & 31u);
  u32* w = bm + (key >> 5);
  if (!(*reinterpret_cast<volatile u32*>(w) & bit)) atomicOr(w, bit);
}

// ---------------------------------------------------------------------------
// Hash index of a sorted view's join prefixes (Sec. 5.1: a lock-free hash
// table with open addressing and linear probing whose payload is row
// indices).  A slot holds prefix + 1 (0: empty), the first row of the
// prefix's run in the sorted view and the run's length; 2^bits slots.
// ---------------------------------------------------------------------------
struct HashSlot {
  unsigned long long key;
  u32 lo, cnt;
};
LOB_HD u64 hash_home(u64 pv, int bits) { return (pv * 0x9E3779B97F4A7C15ull) >> (64 - bits); }
// the run [lo, hi) of prefix pv (empty when absent); at most 2^bits probes
LOB_DEV void hash_find(const HashSlot* tab, int bits, u64 pv, u64& lo, u64& hi) {
  const u64 mask = (1ull << bits) - 1;
  u64 s = hash_home(pv, bits);
  lo = hi = 0;
  for (u64 n = 0; n <= mask; n++) {
    const u64 k = tab[s].key;
    if (k == pv + 1) {
      lo = tab[s].lo;
      hi = lo + tab[s].cnt;
      return;
    }
    if (k == 0) return;
    s = (s + 1) & mask;
  }
}

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------
template <class T> LOB_DEV T warp_inclusive_sum(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}
template <class T> LOB_DEV T warp_inclusive_max(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v = v > n ? v : n;
  }
  return v;
}

// Block-wide exclusive sum; `smem` needs blockDim.x/32 + 1 elements.  Returns
// the exclusive prefix of `v` and writes the block total to *total.
template <class T> LOB_DEV T block_exclusive_sum(T v, T* smem, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_inclusive_sum(v);
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? smem[lane] : T(0);
    T wi = warp_inclusive_sum(w);
    if (lane < nw) smem[lane] = wi - w;
    if (lane == nw - 1) smem[nw] = wi;
  }
  __syncthreads();
  T r = smem[warp] + inc - v;
  *total = smem[nw];
  __syncthreads();
  return r;
}

template <class T> LOB_DEV T block_inclusive_max(T v, T* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_inclusive_max(v);
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? smem[lane] : T(0);
    T wi = warp_inclusive_max(w);
    // exclusive max of warp totals
    T ex = __shfl_up_sync(0xFFFFFFFFu, wi, 1);
    if (lane < nw) smem[lane] = lane == 0 ? T(0) : ex;
  }
  __syncthreads();
  T p = smem[warp];
  __syncthreads();
  return inc > p ? inc : p;
}

// first index i in [lo, hi) with a[i] > x (a sorted ascending)
template <class T> LOB_DEV u64 upper_bound_dev(const T* a, u64 lo, u64 hi, T x) {
  while (lo < hi) {
    u64 mid = lo + ((hi - lo) >> 1);
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// first index i in [lo, hi) with a[i] >= x
template <class T> LOB_DEV u64 lower_bound_dev(const T* a, u64 lo, u64 hi, T x) {
  while (lo < hi) {
    u64 mid = lo + ((hi - lo) >> 1);
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
