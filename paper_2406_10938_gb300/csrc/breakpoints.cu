// Breakpoint selection (Alg. 1 / closed form of Sec. 4.1) on the GPU.
//
// Alg. 1 finds the order statistics of each projected dimension's sample with
// rounds of QuickSelect; here all L*K sample rows are sorted at once by one
// stable radix sort (value bits, then the row as the most significant digit)
// and the ranks floor(n_s/N_r)*z are read off. Any selection method returns
// the same order statistics, so this is the same output.
#include "common.cuh"

namespace detlsh {
namespace {

// Monotone map of finite floats to uint32 (ascending order preserved).
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_make_keys(const float* __restrict__ Ps, int64_t total, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) {
    keys[i] = ordered_bits(Ps[i]);
    vals[i] = (uint32_t)i;
  }
}

__global__ void k_row_keys(const uint32_t* __restrict__ vals, int64_t total, int64_t n_s,
                           uint32_t* __restrict__ rows) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) rows[i] = (uint32_t)(vals[i] / n_s);
}

__global__ void k_gather_edges(const float* __restrict__ Ps, const uint32_t* __restrict__ order,
                               int64_t n_s, int LK, int Nr, float* __restrict__ E) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)LK * (Nr + 1)) return;
  const int r = (int)(i / (Nr + 1)), z = (int)(i % (Nr + 1));
  const int64_t m = n_s / Nr;
  int64_t rank;
  if (z == 0) rank = 0;
  else if (z == Nr) rank = n_s - 1;
  else rank = m * z;
  E[i] = Ps[order[(int64_t)r * n_s + rank]];
}

}  // namespace

int select_breakpoints(const float* Ps, int64_t n_s, int LK, int Nr, float* E, cudaStream_t s) {
  const int64_t total = n_s * LK;
  Scratch k0, v0, k1, v1;
  DL_TRY(k0.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(v0.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(k1.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(v1.alloc(sizeof(uint32_t) * total, s));
  const unsigned nb = ceil_div(total, 256);
  k_make_keys<<<nb, 256, 0, s>>>(Ps, total, k0.as<uint32_t>(), v0.as<uint32_t>());
  DL_LAUNCH();
  DL_TRY(radix_sort_pairs(k0.as<uint32_t>(), v0.as<uint32_t>(), total, 0, 32, k1.as<uint32_t>(),
                          v1.as<uint32_t>(), s));
  k_row_keys<<<nb, 256, 0, s>>>(v1.as<uint32_t>(), total, n_s, k0.as<uint32_t>());
  DL_LAUNCH();
  DL_TRY(radix_sort_pairs(k0.as<uint32_t>(), v1.as<uint32_t>(), total, 0, 8, k1.as<uint32_t>(),
                          v0.as<uint32_t>(), s));
  k_gather_edges<<<ceil_div((int64_t)LK * (Nr + 1), 256), 256, 0, s>>>(Ps, v0.as<uint32_t>(), n_s,
                                                                        LK, Nr, E);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace detlsh

// ---------------------------------------------------------------------------
// The same breakpoint selection with caller-provided temporary storage.
namespace detlsh {

size_t radix_ws_bytes(int64_t n, int bit_lo, int bit_hi);
int radix_sort_pairs_ws(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int bit_lo,
                        int bit_hi, uint32_t* keys_out, uint32_t* vals_out, void* ws, size_t ws_bytes,
                        cudaStream_t s);

namespace {
size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

size_t select_breakpoints_ws_bytes(int64_t n_s, int LK) {
  const int64_t total = n_s * LK;
  return 4 * al256(sizeof(uint32_t) * total) + radix_ws_bytes(total, 0, 32);
}

int select_breakpoints_ws(const float* Ps, int64_t n_s, int LK, int Nr, float* E, void* ws,
                          size_t ws_bytes, cudaStream_t s) {
  const int64_t total = n_s * LK;
  if (ws_bytes < select_breakpoints_ws_bytes(n_s, LK)) {
    set_error("breakpoint workspace too small");
    return DETLSH_EINTERNAL;
  }
  char* p = static_cast<char*>(ws);
  const size_t arr = al256(sizeof(uint32_t) * total);
  uint32_t* k0 = reinterpret_cast<uint32_t*>(p);
  uint32_t* v0 = reinterpret_cast<uint32_t*>(p + arr);
  uint32_t* k1 = reinterpret_cast<uint32_t*>(p + 2 * arr);
  uint32_t* v1 = reinterpret_cast<uint32_t*>(p + 3 * arr);
  void* sort_ws = p + 4 * arr;
  const size_t sort_b = ws_bytes - 4 * arr;
  const unsigned nb = ceil_div(total, 256);
  k_make_keys<<<nb, 256, 0, s>>>(Ps, total, k0, v0);
  DL_LAUNCH();
  DL_TRY(radix_sort_pairs_ws(k0, v0, total, 0, 32, k1, v1, sort_ws, sort_b, s));
  k_row_keys<<<nb, 256, 0, s>>>(v1, total, n_s, k0);
  DL_LAUNCH();
  DL_TRY(radix_sort_pairs_ws(k0, v1, total, 0, 8, k1, v0, sort_ws, sort_b, s));
  k_gather_edges<<<ceil_div((int64_t)LK * (Nr + 1), 256), 256, 0, s>>>(Ps, v0, n_s, LK, Nr, E);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace detlsh
