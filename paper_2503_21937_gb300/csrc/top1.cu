// top-1-proofs (Sec. 5.3 "Limitations"; Sec. 3.4 lists the differentiable
// version): the proof arena's set-up, the read-out of proofs and the gradient.
//
// Arena layout (u32 words): word 0 = 0, the empty proof; for every input-fact
// id i, words 1 + 2i and 2 + 2i hold the singleton proof {i}; after them the
// proofs that joins create (top1_union in common.cuh), each [length, ids
// ascending].  A tag's low 32 bits are the word offset of its proof.
#include "kernels.h"

namespace {

__global__ void k_top1_init(u32* __restrict__ words, u64 n_ids) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i <= n_ids; i += stride) {
    if (i == n_ids) {
      words[0] = 0u;
    } else {
      words[1 + 2 * i] = 1u;
      words[2 + 2 * i] = (u32)i;
    }
  }
}

__global__ void k_fill_f32(float* __restrict__ a, u64 n, float v) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = v;
}

__global__ void k_set_u64(unsigned long long* p, u64 v) { *p = v; }

__global__ void k_top1_lengths(const u64* __restrict__ tags, u64 n, const u32* __restrict__ words, u32* __restrict__ lens) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) lens[i] = words[(u32)tags[i]];
}

// one warp per fact: copy its proof's ids to out + off[i]
__global__ void k_top1_copy(const u64* __restrict__ tags, u64 n, const u32* __restrict__ words, const u64* __restrict__ off,
                            u32* __restrict__ out) {
  const u64 warps = ((u64)gridDim.x * blockDim.x) >> 5;
  const u32 lane = threadIdx.x & 31u;
  for (u64 i = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const u32* p = words + (u32)tags[i];
    const u32 len = p[0];
    for (u32 j = lane; j < len; j += 32) out[off[i] + j] = p[1 + j];
  }
}

// d P / d p_i of a proof's probability P = prod_j p_j is the product of the
// other facts' probabilities: P_nz / p_i when no factor is zero, else nonzero
// only for the single zero factor.  One thread per output fact.
__global__ void k_top1_scatter(const u64* __restrict__ tags, const float* __restrict__ g, u64 n,
                               const u32* __restrict__ words, const float* __restrict__ prob, Top1GradTable T) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float gi = g[i];
    if (gi == 0.0f) continue;
    const u32* p = words + (u32)tags[i];
    const u32 len = p[0];
    double nz = 1.0;
    u32 zeros = 0;
    for (u32 j = 0; j < len; j++) {
      const double x = prob[p[1 + j]];
      if (x == 0.0) zeros++;
      else nz *= x;
    }
    for (u32 j = 0; j < len; j++) {
      const u32 id = p[1 + j];
      const double x = prob[id];
      double d;
      if (x != 0.0) d = zeros ? 0.0 : nz / x;
      else d = zeros == 1 ? nz : 0.0;
      for (int k = 0; k < T.n; k++)
        if (id >= T.base[k] && id - T.base[k] < T.count[k]) {
          if (T.grad[k]) atomicAdd(T.grad[k] + (id - T.base[k]), (float)((double)gi * d));
          break;
        }
    }
  }
}

unsigned grid_of(u64 n, int threads = 256) {
  u64 b = (n + threads - 1) / threads;
  if (b > 152ull * 16) b = 152ull * 16;
  return (unsigned)(b ? b : 1);
}

}  // namespace

void top1_init_arena(u32* words, u64 n_ids, cudaStream_t st) {
  ProfScope ps("top1_init", (2.0 * n_ids + 1) * 4.0, st);
  k_top1_init<<<grid_of(n_ids + 1), 256, 0, st>>>(words, n_ids);
}

void fill_f32(float* a, u64 n, float v, cudaStream_t st) {
  if (n) k_fill_f32<<<grid_of(n), 256, 0, st>>>(a, n, v);
}

void set_u64_dev(unsigned long long* p, u64 v, cudaStream_t st) { k_set_u64<<<1, 1, 0, st>>>(p, v); }

void top1_proof_lengths(const u64* tags, u64 n, const u32* words, u32* lens, cudaStream_t st) {
  ProfScope ps("top1_lengths", n * 12.0, st);
  if (n) k_top1_lengths<<<grid_of(n), 256, 0, st>>>(tags, n, words, lens);
}

void top1_copy_proofs(const u64* tags, u64 n, const u32* words, const u64* off, u32* out, cudaStream_t st) {
  ProfScope ps("top1_copy", n * 16.0, st);
  if (n) k_top1_copy<<<grid_of(n * 32), 256, 0, st>>>(tags, n, words, off, out);
}

void top1_grad_scatter(const u64* tags, const float* g, u64 n, const u32* words, const float* prob,
                       const Top1GradTable& T, cudaStream_t st) {
  ProfScope ps("top1_backward", n * 12.0, st);
  if (n) k_top1_scatter<<<grid_of(n), 256, 0, st>>>(tags, g, n, words, prob, T);
}
