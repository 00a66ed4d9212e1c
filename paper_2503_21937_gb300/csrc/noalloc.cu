// lob_unique_rows_noalloc: sort and deduplicate a small batch of rows without
// allocating any device memory.
//
// Some callers cannot allocate device memory at the point where they need this
// step: latency-critical serving paths where cudaMalloc / cudaFree would
// synchronise the device or wait on the driver, plug-ins that run inside a host
// application which owns and budgets all device memory itself, and processes
// that have split the GPU's memory among tenants ahead of time.  For them this
// entry point works entirely in one fixed scratch array that is part of the
// library image: every GPU that loads the library holds it (kScratchBytes,
// about 4.3 MB) until the process exits.
//
// The scratch array is shared by every call on a device and keeps whatever the
// last call left in it.  Everything a call reads from it is written earlier in
// the same call (digit histograms, scan partials, tile counts, the row count),
// so no region needs clearing between calls.  Two calls whose work overlaps on
// the GPU (for example on two streams at once) race on the array; callers must
// order them.
#include <mutex>

#include "../../include/lobster.h"
#include "kernels.h"
#include "scan.cuh"

namespace {

constexpr u64 kMaxRows = LOB_NOALLOC_MAX_ROWS;
constexpr u64 kKeyBytes = kMaxRows * sizeof(u64);
// sort histograms: 256 digits x (kMaxRows / 4096) tiles, plus their scan workspace
constexpr u64 kHistBytes = 64ull * 1024 + 4096;
// unique: one count per 4096-row tile plus scan workspace and the result count
constexpr u64 kUniqueBytes = 4096;
constexpr u64 kScratchBytes = 2 * kKeyBytes + kHistBytes + kUniqueBytes;
static_assert(kScratchBytes <= 4600000, "scratch budget");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// The sort and unique steps size their workspaces at run time; the fixed
// regions above must hold them for the largest accepted batch.
bool scratch_layout_fits() {
  return sort_scratch_bytes(kMaxRows, 8) <= kHistBytes && unique_scratch_bytes(kMaxRows) + 256 <= kUniqueBytes;
}

// Host code must not use g_noalloc_scratch directly: on the host that name is
// only a stand-in for the device symbol.  The device address comes from
// cudaGetSymbolAddress, once per device, with that device current.
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LOB_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return LOB_E_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    if (!scratch_layout_fits()) return LOB_E_CUDA;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LOB_E_CUDA;
    }
    g_scratch_ptr[dev] = reinterpret_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LOB_OK;
}

__global__ void k_pack_rows_u64(const u32* __restrict__ cols, u32 arity, u64 n, u64* __restrict__ keys) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // an all-ones row becomes the all-ones key, which the unique step drops
  // (arity 1: the value 0xFFFFFFFF alone, widened to 64 bits; it still sorts
  // last on the low 32 bits)
  const u32 c0 = cols[i];
  keys[i] = arity == 1 ? (c0 == 0xFFFFFFFFu ? ~0ull : (u64)c0) : ((u64)c0 << 32) | (u64)cols[n + i];
}

__global__ void k_unpack_rows_u64(const u64* __restrict__ keys, const u64* __restrict__ count, u32 arity, u64 stride,
                                  u32* __restrict__ out, u64* __restrict__ n_out) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 n = *count;
  if (i == 0) *n_out = n;
  if (i >= n) return;
  const u64 k = keys[i];
  if (arity == 1) {
    out[i] = (u32)k;
  } else {
    out[i] = (u32)(k >> 32);
    out[stride + i] = (u32)k;
  }
}

}  // namespace

extern "C" int lob_unique_rows_noalloc(const uint32_t* cols, uint32_t arity, uint64_t n, uint32_t* out_cols,
                                       uint64_t* n_out, void* cuda_stream) {
  if (!n_out || (arity != 1 && arity != 2) || (n && (!cols || !out_cols))) return LOB_E_ARG;
  if (n > kMaxRows) return LOB_E_CAPACITY;
  unsigned char* s = nullptr;
  int rc = scratch_for_current_device(&s);
  if (rc != LOB_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  u64* keys_a = reinterpret_cast<u64*>(s);
  u64* keys_b = reinterpret_cast<u64*>(s + kKeyBytes);
  unsigned char* hist = s + 2 * kKeyBytes;
  unsigned char* uniq = hist + kHistBytes;
  u64* count = reinterpret_cast<u64*>(uniq + kUniqueBytes - 256);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (n) k_pack_rows_u64<<<blocks, 256, 0, st>>>(cols, arity, n, keys_a);
  void* k = keys_a;
  void* pay = nullptr;
  sort_pairs(1, 0, &k, &pay, keys_b, nullptr, n, 32 * (int)arity, 8, hist, st);
  void* uk = k == keys_a ? (void*)keys_b : (void*)keys_a;
  unique_run(SR_UNIT, 1, k, nullptr, n, uk, nullptr, count, uniq, st);
  k_unpack_rows_u64<<<blocks ? blocks : 1, 256, 0, st>>>(reinterpret_cast<const u64*>(uk), count, arity, n, out_cols,
                                                         reinterpret_cast<u64*>(n_out));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LOB_OK : LOB_E_CUDA;
}
