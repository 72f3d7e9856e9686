// Device-wide exclusive scan and stable LSD radix sort of (key, value) pairs.
//
// Radix pass (8-bit digit): every tile of TILE items counts its digits, one
// exclusive scan over the digit-major [256][tiles] count table gives every
// (digit, tile) its output base, and the scatter kernel ranks each item among
// the equal digits of its tile in input order (warp match + per-warp counts),
// which makes each pass stable.
#include <algorithm>

#include "common.cuh"

namespace detlsh {
namespace {

constexpr int ST = 256;               // threads per block
constexpr int IPT = 8;                // items per thread
constexpr int TILE = ST * IPT;        // items per tile
constexpr int NW = ST / 32;

// ------------------------------------------------------------------ scan
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < NW ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NW) s_warp[lane] = t;
  }
  __syncthreads();
  const uint32_t before = (w > 0 ? s_warp[w - 1] : 0) + x - v;
  if (total) *total = s_warp[NW - 1];
  __syncthreads();
  return before;
}

__global__ void k_block_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t s_warp[NW];
  const int64_t base = (int64_t)blockIdx.x * TILE;
  uint32_t acc = 0;
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const int64_t i = base + (int64_t)threadIdx.x * IPT + r;
    if (i < n) acc += in[i];
  }
  uint32_t total;
  block_exclusive_scan(acc, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_block_scan(const uint32_t* __restrict__ in, int64_t n,
                             const uint32_t* __restrict__ block_base, uint32_t* __restrict__ out,
                             uint32_t* __restrict__ d_total) {
  __shared__ uint32_t s_warp[NW];
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * IPT;
  uint32_t v[IPT];
  uint32_t acc = 0;
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    v[r] = (base + r < n) ? in[base + r] : 0;
    acc += v[r];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(acc, s_warp, &total);
  if (block_base) run += block_base[blockIdx.x];
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    if (base + r < n) out[base + r] = run;
    run += v[r];
  }
  if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == ST - 1) *d_total = run;
}

// ------------------------------------------------------------------ radix pass
__global__ void __launch_bounds__(ST)
k_digit_hist(const uint32_t* __restrict__ keys, int64_t n, int bit, uint32_t* __restrict__ hist,
             int64_t n_tiles) {
  __shared__ uint32_t s_h[256];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * TILE;
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const int64_t i = base + (int64_t)r * ST + threadIdx.x;
    if (i < n) atomicAdd(&s_h[(keys[i] >> bit) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter of one tile: each item's rank among the equal digits of the
// tile (in input order: warp match, per-warp counts, a running count per
// digit) places it in shared memory in digit order, and the tile then leaves
// as runs of equal digits, consecutive threads writing consecutive outputs.
__global__ void __launch_bounds__(ST)
k_digit_scatter(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                int64_t n, int bit, const uint32_t* __restrict__ hist, const uint32_t* __restrict__ offs,
                int64_t n_tiles, uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t s_base[256];     // global output of the tile's first item of each digit
  __shared__ uint32_t s_lstart[256];   // the tile's first local position of each digit
  __shared__ uint32_t s_run[256];      // items of each digit placed so far
  __shared__ uint32_t s_wc[NW][256];
  __shared__ uint32_t s_warp[NW];
  __shared__ uint32_t s_key[TILE], s_val[TILE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int tile_n = n - base < TILE ? (int)(n - base) : TILE;
  s_base[threadIdx.x] = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  const uint32_t h = hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  s_lstart[threadIdx.x] = block_exclusive_scan(h, s_warp, nullptr);
  s_run[threadIdx.x] = 0;
#pragma unroll
  for (int q = 0; q < NW; ++q) s_wc[q][threadIdx.x] = 0;
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (int r = 0; r < IPT; ++r) {
    const int li = r * ST + threadIdx.x;
    const bool valid = li < tile_n;
    uint32_t key = 0, val = 0;
    int digit = 256;
    if (valid) {
      key = keys_in[base + li];
      val = vals_in[base + li];
      digit = (int)((key >> bit) & 255u);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, digit);
    const uint32_t rank_in_warp = __popc(peers & lt);
    if (valid && rank_in_warp == 0) s_wc[w][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = s_lstart[digit] + s_run[digit] + rank_in_warp;
      for (int q = 0; q < w; ++q) pos += s_wc[q][digit];
      s_key[pos] = key;
      s_val[pos] = val;
    }
    __syncthreads();
    uint32_t add = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      add += s_wc[q][threadIdx.x];
      s_wc[q][threadIdx.x] = 0;
    }
    s_run[threadIdx.x] += add;
    __syncthreads();
  }
  for (int j = threadIdx.x; j < tile_n; j += ST) {
    const uint32_t key = s_key[j];
    const uint32_t d = (key >> bit) & 255u;
    const uint32_t pos = s_base[d] + (uint32_t)j - s_lstart[d];
    keys_out[pos] = key;
    vals_out[pos] = s_val[j];
  }
}

}  // namespace

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                       cudaStream_t s) {
  if (n == 0) {
    if (d_total) DL_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
    return DETLSH_OK;
  }
  const int64_t nb = ceil_div(n, TILE);
  if (nb == 1) {
    k_block_scan<<<1, ST, 0, s>>>(in, n, nullptr, out, d_total);
    DL_LAUNCH();
    return DETLSH_OK;
  }
  Scratch sums, sums_scan;
  DL_TRY(sums.alloc(sizeof(uint32_t) * nb, s));
  DL_TRY(sums_scan.alloc(sizeof(uint32_t) * nb, s));
  k_block_sums<<<(unsigned)nb, ST, 0, s>>>(in, n, sums.as<uint32_t>());
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32(sums.as<uint32_t>(), sums_scan.as<uint32_t>(), nb, nullptr, s));
  k_block_scan<<<(unsigned)nb, ST, 0, s>>>(in, n, sums_scan.as<uint32_t>(), out, d_total);
  DL_LAUNCH();
  return DETLSH_OK;
}

int radix_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int bit_lo,
                     int bit_hi, uint32_t* keys_out, uint32_t* vals_out, cudaStream_t s) {
  if (n == 0) return DETLSH_OK;
  const int passes = (bit_hi - bit_lo + 7) / 8;
  const int64_t n_tiles = ceil_div(n, TILE);
  Scratch hist, offs, kb, vb;
  DL_TRY(hist.alloc(sizeof(uint32_t) * 256 * n_tiles, s));
  DL_TRY(offs.alloc(sizeof(uint32_t) * 256 * n_tiles, s));
  if (passes > 1) {
    DL_TRY(kb.alloc(sizeof(uint32_t) * n, s));
    DL_TRY(vb.alloc(sizeof(uint32_t) * n, s));
  }
  // ping-pong so that the last pass lands in keys_out/vals_out
  const uint32_t* ki = keys_in;
  const uint32_t* vi = vals_in;
  for (int p = 0; p < passes; ++p) {
    const bool last = (p == passes - 1);
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* ko = to_out ? keys_out : kb.as<uint32_t>();
    uint32_t* vo = to_out ? vals_out : vb.as<uint32_t>();
    const int bit = bit_lo + 8 * p;
    k_digit_hist<<<(unsigned)n_tiles, ST, 0, s>>>(ki, n, bit, hist.as<uint32_t>(), n_tiles);
    DL_LAUNCH();
    DL_TRY(exclusive_scan_u32(hist.as<uint32_t>(), offs.as<uint32_t>(), 256 * n_tiles, nullptr, s));
    k_digit_scatter<<<(unsigned)n_tiles, ST, 0, s>>>(ki, vi, n, bit, hist.as<uint32_t>(), offs.as<uint32_t>(),
                                                     n_tiles, ko, vo);
    DL_LAUNCH();
    ki = ko;
    vi = vo;
    (void)last;
  }
  return DETLSH_OK;
}

}  // namespace detlsh

// ---------------------------------------------------------------------------
// Variants of the scan and the radix sort that take their temporary storage
// from the caller instead of allocating it (same kernels, same results).
namespace detlsh {
namespace {

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

size_t scan_ws_bytes(int64_t n) {
  size_t total = 0;
  int64_t m = n;
  while (m > TILE) {
    const int64_t nb = ceil_div(m, TILE);
    total += 2 * align256(sizeof(uint32_t) * nb);
    m = nb;
  }
  return total;
}

int exclusive_scan_u32_ws(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total, void* ws,
                          size_t ws_bytes, cudaStream_t s) {
  if (n == 0) {
    if (d_total) DL_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
    return DETLSH_OK;
  }
  const int64_t nb = ceil_div(n, TILE);
  if (nb == 1) {
    k_block_scan<<<1, ST, 0, s>>>(in, n, nullptr, out, d_total);
    DL_LAUNCH();
    return DETLSH_OK;
  }
  const size_t part = align256(sizeof(uint32_t) * nb);
  if (ws_bytes < 2 * part + scan_ws_bytes(nb)) {
    set_error("scan workspace too small");
    return DETLSH_EINTERNAL;
  }
  uint32_t* sums = static_cast<uint32_t*>(ws);
  uint32_t* sums_scan = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + part);
  k_block_sums<<<(unsigned)nb, ST, 0, s>>>(in, n, sums);
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32_ws(sums, sums_scan, nb, nullptr, static_cast<char*>(ws) + 2 * part,
                               ws_bytes - 2 * part, s));
  k_block_scan<<<(unsigned)nb, ST, 0, s>>>(in, n, sums_scan, out, d_total);
  DL_LAUNCH();
  return DETLSH_OK;
}

size_t radix_ws_bytes(int64_t n, int bit_lo, int bit_hi) {
  const int passes = (bit_hi - bit_lo + 7) / 8;
  const int64_t n_tiles = ceil_div(n, TILE);
  size_t b = 2 * align256(sizeof(uint32_t) * 256 * n_tiles) + scan_ws_bytes(256 * n_tiles);
  if (passes > 1) b += 2 * align256(sizeof(uint32_t) * n);
  return b;
}

int radix_sort_pairs_ws(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int bit_lo,
                        int bit_hi, uint32_t* keys_out, uint32_t* vals_out, void* ws, size_t ws_bytes,
                        cudaStream_t s) {
  if (n == 0) return DETLSH_OK;
  if (ws_bytes < radix_ws_bytes(n, bit_lo, bit_hi)) {
    set_error("radix sort workspace too small");
    return DETLSH_EINTERNAL;
  }
  const int passes = (bit_hi - bit_lo + 7) / 8;
  const int64_t n_tiles = ceil_div(n, TILE);
  char* p = static_cast<char*>(ws);
  const size_t tbl = align256(sizeof(uint32_t) * 256 * n_tiles);
  uint32_t* hist = reinterpret_cast<uint32_t*>(p);
  uint32_t* offs = reinterpret_cast<uint32_t*>(p + tbl);
  p += 2 * tbl;
  const size_t scan_b = scan_ws_bytes(256 * n_tiles);
  void* scan_ws = p;
  p += scan_b;
  uint32_t* kb = nullptr;
  uint32_t* vb = nullptr;
  if (passes > 1) {
    kb = reinterpret_cast<uint32_t*>(p);
    vb = reinterpret_cast<uint32_t*>(p + align256(sizeof(uint32_t) * n));
  }
  const uint32_t* ki = keys_in;
  const uint32_t* vi = vals_in;
  for (int pass = 0; pass < passes; ++pass) {
    const bool to_out = ((passes - 1 - pass) % 2) == 0;
    uint32_t* ko = to_out ? keys_out : kb;
    uint32_t* vo = to_out ? vals_out : vb;
    const int bit = bit_lo + 8 * pass;
    k_digit_hist<<<(unsigned)n_tiles, ST, 0, s>>>(ki, n, bit, hist, n_tiles);
    DL_LAUNCH();
    DL_TRY(exclusive_scan_u32_ws(hist, offs, 256 * n_tiles, nullptr, scan_ws, scan_b, s));
    k_digit_scatter<<<(unsigned)n_tiles, ST, 0, s>>>(ki, vi, n, bit, hist, offs, n_tiles, ko, vo);
    DL_LAUNCH();
    ki = ko;
    vi = vo;
  }
  return DETLSH_OK;
}

}  // namespace detlsh
