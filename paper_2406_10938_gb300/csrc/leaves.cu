// DE-Tree construction (Alg. 3 and the split rule of Sec. 4.2), bulk-loaded.
//
// Per tree the points are first stably sorted by the K-bit vector of their
// codes' top bits (dimension 0 most significant): the runs of that order are
// the root's 2^K first-layer nodes. Then, level-synchronously, every node
// (a contiguous segment of the tree's id array) holding more than max_leaf
// points whose codes still have an unresolved bit is split: its tiles count
// the next bit of every splittable dimension, the dimension minimising
// |2*ones - count| (lowest on ties) is chosen, and the segment is stably
// partitioned bit 0 first. Empty children vanish. Because every split is a
// stable in-place partition, the final segments are the leaves in
// depth-first order with ascending ids inside each leaf.
//
// A splittable segment of at most SCAP entries is finished in one pass by one
// block in shared memory (k_small): the same split rule applied depth-first
// (bit-0 child first) down to its leaves, whose records are staged and then
// placed at scanned positions, so the segment list stays in depth-first order
// without a sort. Larger segments take the level passes above until their
// children fit.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace detlsh {
namespace {

constexpr int LT = 256;          // threads per tile block
constexpr int LIPT = 4;          // items per thread
constexpr int LTILE = LT * LIPT; // items per tile
constexpr int SCAP = 2048;       // entries of a segment finished in shared memory
constexpr int ST = 256;          // threads of that block
constexpr int SSTACK = kMaxK * 8 + 2;   // split stack: one entry per level of the path, plus one

__device__ __forceinline__ uint32_t byte_of(const uint4& v, int j) {
  const uint32_t w = (j < 4) ? v.x : (j < 8) ? v.y : (j < 12) ? v.z : v.w;
  return (w >> ((j & 3) * 8)) & 0xffu;
}
__device__ __forceinline__ void set_byte(uint4& v, int j, uint32_t b) {
  const uint32_t sh = (j & 3) * 8, mask = ~(0xffu << sh);
  if (j < 4) v.x = (v.x & mask) | (b << sh);
  else if (j < 8) v.y = (v.y & mask) | (b << sh);
  else if (j < 12) v.z = (v.z & mask) | (b << sh);
  else v.w = (v.w & mask) | (b << sh);
}

__device__ __forceinline__ uint4 load_code(const uint8_t* __restrict__ codes, int64_t row, int K) {
  if (K == 16) return __ldg(reinterpret_cast<const uint4*>(codes + row * 16));
  uint4 v = make_uint4(0, 0, 0, 0);
  for (int j = 0; j < K; ++j) set_byte(v, j, codes[row * K + j]);
  return v;
}

// ---- root level
// Root key of (tree, point) g = t*n + i: the tree above the K top bits of the
// point's codes in that tree (dimension 0 most significant).
__global__ void k_root_keys(const uint8_t* __restrict__ codes, int64_t n, int64_t total, int K, int bits,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int64_t t = g / n;
  const uint4 c = load_code(codes, g, K);
  uint32_t key = (uint32_t)t;
#pragma unroll
  for (int j = 0; j < kMaxK; ++j)
    if (j < K) key = (key << 1) | ((byte_of(c, j) >> (bits - 1)) & 1u);
  keys[g] = key;
  vals[g] = (uint32_t)(g - t * n);
}

__global__ void k_root_flags(const uint32_t* __restrict__ keys, int64_t total, uint32_t* __restrict__ flags) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  flags[g] = (g == 0 || keys[g] != keys[g - 1]) ? 1u : 0u;
}

__global__ void k_root_segments(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                                const uint32_t* __restrict__ keys_all, int64_t total, int64_t n,
                                int K, int bits, uint32_t* __restrict__ seg_start,
                                uint4* __restrict__ seg_plen, uint4* __restrict__ seg_prefix) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total || !flags[g]) return;
  const uint32_t s = pos[g];
  seg_start[s] = (uint32_t)g;
  const uint32_t key = keys_all[g];
  uint4 pl = make_uint4(0, 0, 0, 0), pf = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int j = 0; j < kMaxK; ++j) {
    set_byte(pl, j, j < K ? 1u : (uint32_t)bits);
    set_byte(pf, j, j < K ? (key >> (K - 1 - j)) & 1u : 0u);
  }
  seg_plen[s] = pl;
  seg_prefix[s] = pf;
  (void)n;
}

__global__ void k_seg_counts(const uint32_t* __restrict__ seg_start, uint32_t nseg, int64_t n,
                             int64_t total, uint32_t* __restrict__ seg_count) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const uint32_t a = seg_start[s];
  // a segment never crosses its tree's end
  const int64_t tree_end = ((int64_t)a / n + 1) * n;
  int64_t b = total;
  if (s + 1 < nseg) b = (int64_t)seg_start[s + 1] < tree_end ? (int64_t)seg_start[s + 1] : tree_end;
  seg_count[s] = (uint32_t)(b - a);
}

// ---- split iteration
// Per segment: tiles of the level pass (large segments), or the flag of a
// segment finished in shared memory (small), or neither (a leaf).
__global__ void k_plan(const uint32_t* __restrict__ seg_count, const uint4* __restrict__ seg_plen,
                       uint32_t nseg, int K, int bits, int max_leaf,
                       uint32_t* __restrict__ tiles_needed, uint32_t* __restrict__ small) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const uint32_t cnt = seg_count[s];
  bool splittable = false;
  const uint4 pl = seg_plen[s];
#pragma unroll
  for (int j = 0; j < kMaxK; ++j)
    if (j < K && byte_of(pl, j) < (uint32_t)bits) splittable = true;
  const bool active = cnt > (uint32_t)max_leaf && splittable;
  const bool sm = active && cnt <= (uint32_t)SCAP;
  tiles_needed[s] = (active && !sm) ? (cnt + LTILE - 1) / LTILE : 0u;
  small[s] = sm ? 1u : 0u;
}

__global__ void k_small_list(const uint32_t* __restrict__ small, const uint32_t* __restrict__ small_pos,
                             uint32_t nseg, uint32_t* __restrict__ small_seg) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nseg && small[s]) small_seg[small_pos[s]] = (uint32_t)s;
}

// One small segment per block: its entries (ids and codes, leaf order) in
// two shared buffers, a stack of pending nodes (offset, count, buffer,
// prefix lengths and prefixes). A node that is a leaf (at most max_leaf
// entries, or no unresolved bit) is emitted; another is split as in the level
// passes: ones of every unresolved next bit counted per warp (each warp owns
// a contiguous range, visited lane-strided), the dimension minimising
// |2*ones - count| (lowest on ties) chosen, the node stably partitioned into
// the other buffer by warp ballots, and its non-empty children pushed, the
// bit-1 child first so that the bit-0 child is popped first. The stack depth
// is uniform over the block and kept in registers; only splits synchronise.
// Each leaf's ids go to ids[] and its record (start, count, prefix lengths as
// 16 nibbles) to rec[start + leaf number], inside the segment's own range of
// the level passes' partition buffer; out_n[seg] = number of leaves.
__global__ void __launch_bounds__(ST)
k_small(const uint32_t* __restrict__ small_seg, const uint32_t* __restrict__ seg_start,
        const uint32_t* __restrict__ seg_count, const uint4* __restrict__ seg_plen,
        const uint4* __restrict__ seg_prefix, const uint4* __restrict__ lcodes, int K, int bits, int max_leaf,
        uint32_t* __restrict__ ids, uint32_t* __restrict__ out_n, uint4* __restrict__ rec) {
  extern __shared__ uint4 smem_u4[];
  uint4* sc = smem_u4;                                              // [2][SCAP] codes
  uint32_t* si = reinterpret_cast<uint32_t*>(smem_u4 + 2 * SCAP);   // [2][SCAP] ids
  __shared__ uint4 st_pl[SSTACK], st_pf[SSTACK];
  __shared__ uint16_t st_o[SSTACK], st_m[SSTACK];
  __shared__ uint8_t st_b[SSTACK];
  __shared__ uint32_t s_wcnt[ST / 32][kMaxK];
  __shared__ uint32_t s_best[2];
  constexpr int NW = ST / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;

  const uint32_t seg = small_seg[blockIdx.x];
  const uint32_t start = seg_start[seg], count = seg_count[seg];
  for (uint32_t i = threadIdx.x; i < count; i += ST) {
    sc[i] = lcodes[start + i];
    si[i] = ids[start + i];
  }
  if (threadIdx.x == 0) {
    st_o[0] = 0;
    st_m[0] = (uint16_t)count;
    st_b[0] = 0;
    st_pl[0] = seg_plen[seg];
    st_pf[0] = seg_prefix[seg];
  }
  __syncthreads();
  int sp = 1;
  uint32_t nleaf = 0;
  while (sp > 0) {
    --sp;
    const uint32_t o = st_o[sp], m = st_m[sp], b = st_b[sp];
    const uint4 pl = st_pl[sp], pf = st_pf[sp];
    bool splittable = false;
#pragma unroll
    for (int j = 0; j < kMaxK; ++j)
      if (j < K && byte_of(pl, j) < (uint32_t)bits) splittable = true;
    const uint4* cb = sc + b * SCAP + o;
    const uint32_t* ib = si + b * SCAP + o;
    if (m <= (uint32_t)max_leaf || !splittable) {
      for (uint32_t i = threadIdx.x; i < m; i += ST) ids[start + o + i] = ib[i];
      if (threadIdx.x == 0) {
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          lo |= byte_of(pl, j) << (4 * j);
          hi |= byte_of(pl, j + 8) << (4 * j);
        }
        rec[start + nleaf] = make_uint4(start + o, m, lo, hi);
      }
      ++nleaf;
      continue;
    }
    // warp w owns [w*wc, min(m, (w+1)*wc)), wc a multiple of 32
    const uint32_t wc = ((m + NW * 32 - 1) / (NW * 32)) * 32;
    const uint32_t w0 = min(m, w * wc), w1 = min(m, w0 + wc);
    uint32_t cnt[kMaxK];
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) cnt[j] = 0;
    for (uint32_t i = w0; i < w1; i += 32) {
      const bool valid = i + lane < w1;
      const uint4 c = valid ? cb[i + lane] : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int j = 0; j < kMaxK; ++j) {
        const uint32_t l = byte_of(pl, j);
        if (j < K && l < (uint32_t)bits)
          cnt[j] += __popc(__ballot_sync(0xffffffffu, valid && ((byte_of(c, j) >> (bits - 1 - l)) & 1u)));
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < kMaxK; ++j) s_wcnt[w][j] = cnt[j];
    }
    __syncthreads();
    if (w == 0) {
      // lane j: dimension j's ones and gap; argmin over lanes, lowest j on ties
      uint32_t v = 0, gap = 0xffffffffu;
      if (lane < K && byte_of(pl, lane & 15) < (uint32_t)bits) {
#pragma unroll
        for (int q = 0; q < NW; ++q) v += s_wcnt[q][lane];
        gap = (2u * v > m) ? 2u * v - m : m - 2u * v;
      }
      uint32_t bj = (uint32_t)lane;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const uint32_t g2 = __shfl_xor_sync(0xffffffffu, gap, off);
        const uint32_t j2 = __shfl_xor_sync(0xffffffffu, bj, off);
        const uint32_t v2 = __shfl_xor_sync(0xffffffffu, v, off);
        if (g2 < gap || (g2 == gap && j2 < bj)) {
          gap = g2;
          bj = j2;
          v = v2;
        }
      }
      if (lane == 0) {
        s_best[0] = bj;
        s_best[1] = v;
      }
    }
    __syncthreads();
    const int best = (int)s_best[0];
    const uint32_t ones = s_best[1];
    const uint32_t zeros = m - ones;
    const uint32_t shift = (uint32_t)(bits - 1) - byte_of(pl, best);
    uint32_t ob = 0;   // ones before this warp's range
    for (int q = 0; q < w; ++q) ob += s_wcnt[q][best];
    uint4* cd = sc + (b ^ 1u) * SCAP + o;
    uint32_t* id = si + (b ^ 1u) * SCAP + o;
    for (uint32_t i = w0; i < w1; i += 32) {
      const bool valid = i + lane < w1;
      uint4 c = make_uint4(0, 0, 0, 0);
      uint32_t v = 0;
      if (valid) {
        c = cb[i + lane];
        v = ib[i + lane];
      }
      const bool bit = valid && ((byte_of(c, best) >> shift) & 1u);
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      const uint32_t before = ob + __popc(bal & lt_mask);
      if (valid) {
        const uint32_t dst = bit ? zeros + before : i + lane - before;
        cd[dst] = c;
        id[dst] = v;
      }
      ob += __popc(bal);
    }
    if (threadIdx.x == 0) {
      uint4 cpl = pl;
      set_byte(cpl, best, byte_of(pl, best) + 1);
      const uint32_t p2 = byte_of(pf, best) * 2;
      int t = sp;
      if (ones) {
        uint4 cpf = pf;
        set_byte(cpf, best, p2 + 1);
        st_o[t] = (uint16_t)(o + zeros);
        st_m[t] = (uint16_t)ones;
        st_b[t] = (uint8_t)(b ^ 1u);
        st_pl[t] = cpl;
        st_pf[t] = cpf;
        ++t;
      }
      if (zeros) {
        uint4 cpf = pf;
        set_byte(cpf, best, p2);
        st_o[t] = (uint16_t)o;
        st_m[t] = (uint16_t)zeros;
        st_b[t] = (uint8_t)(b ^ 1u);
        st_pl[t] = cpl;
        st_pf[t] = cpf;
      }
    }
    sp += (ones ? 1 : 0) + (zeros ? 1 : 0);
    __syncthreads();   // the children's entries and stack slots are in place
  }
  if (threadIdx.x == 0) out_n[seg] = nleaf;
}

// The leaf records of the small segments into the next segment list, at
// out_pos[seg] + leaf number; a leaf's prefixes are the top prefix-length
// bits of the codes of any of its points (its first).
__global__ void k_small_expand(const uint32_t* __restrict__ small_seg, uint32_t nsmall,
                               const uint32_t* __restrict__ seg_start, const uint32_t* __restrict__ out_n,
                               const uint32_t* __restrict__ out_pos, const uint4* __restrict__ rec,
                               const uint32_t* __restrict__ ids, const uint8_t* __restrict__ codes, int64_t n, int K,
                               int bits, uint32_t* __restrict__ n_start, uint32_t* __restrict__ n_count,
                               uint4* __restrict__ n_plen, uint4* __restrict__ n_prefix) {
  const uint32_t t = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (t >= nsmall) return;
  const uint32_t seg = small_seg[t];
  const uint32_t start = seg_start[seg], nl = out_n[seg], base = out_pos[seg];
  for (uint32_t q = threadIdx.x & 31; q < nl; q += 32) {
    const uint4 r = rec[start + q];
    const int64_t tree = (int64_t)r.x / n;
    const uint4 c = load_code(codes, tree * n + ids[r.x], K);
    uint4 pl = make_uint4(0, 0, 0, 0), pf = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) {
      const uint32_t l = ((j < 8 ? r.z : r.w) >> (4 * (j & 7))) & 15u;
      set_byte(pl, j, l);
      set_byte(pf, j, byte_of(c, j) >> (bits - l));
    }
    n_start[base + q] = r.x;
    n_count[base + q] = r.y;
    n_plen[base + q] = pl;
    n_prefix[base + q] = pf;
  }
}

__global__ void k_tile_map(const uint32_t* __restrict__ tiles_needed,
                           const uint32_t* __restrict__ tile_base, uint32_t nseg,
                           uint32_t* __restrict__ tile_seg) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const uint32_t t0 = tile_base[s], nt = tiles_needed[s];
  for (uint32_t t = 0; t < nt; ++t) tile_seg[t0 + t] = (uint32_t)s;
}

// The code vector of every (tree, leaf-ordered position), so that the level
// passes read codes as contiguous streams instead of gathering them by id.
__global__ void k_gather_codes(const uint8_t* __restrict__ codes, const uint32_t* __restrict__ ids, int64_t n,
                               int64_t total, int K, uint4* __restrict__ lcodes) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tree_row = (g / n) * n;
    lcodes[g] = load_code(codes, tree_row + ids[g], K);
  }
}

// Per tile: number of points whose next unresolved bit is 1, for every dimension.
__global__ void __launch_bounds__(LT)
k_tile_count(const uint32_t* __restrict__ tile_seg, const uint32_t* __restrict__ tile_base,
             const uint32_t* __restrict__ seg_start, const uint32_t* __restrict__ seg_count,
             const uint4* __restrict__ seg_plen, const uint4* __restrict__ lcodes, int K, int bits,
             uint32_t* __restrict__ tile_cnt) {
  __shared__ uint32_t s_cnt[kMaxK];
  const uint32_t tile = blockIdx.x;
  const uint32_t s = tile_seg[tile];
  const uint32_t chunk = tile - tile_base[s];
  const uint32_t start = seg_start[s], count = seg_count[s];
  const uint4 pl = seg_plen[s];
  if (threadIdx.x < kMaxK) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  uint32_t cnt[kMaxK];
#pragma unroll
  for (int j = 0; j < kMaxK; ++j) cnt[j] = 0;
  for (int r = 0; r < LIPT; ++r) {
    const uint32_t off = chunk * LTILE + r * LT + threadIdx.x;
    if (off < count) {
      const uint4 c = lcodes[start + off];
#pragma unroll
      for (int j = 0; j < kMaxK; ++j) {
        const uint32_t l = byte_of(pl, j);
        if (j < K && l < (uint32_t)bits) cnt[j] += (byte_of(c, j) >> (bits - 1 - l)) & 1u;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxK; ++j) {
    uint32_t v = cnt[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_cnt[j], v);
  }
  __syncthreads();
  if (threadIdx.x < kMaxK) tile_cnt[(int64_t)tile * kMaxK + threadIdx.x] = s_cnt[threadIdx.x];
}

// Per active segment: choose the split dimension and the per-tile bases.
__global__ void k_choose(const uint32_t* __restrict__ tiles_needed,
                         const uint32_t* __restrict__ tile_base,
                         const uint32_t* __restrict__ seg_count, const uint4* __restrict__ seg_plen,
                         uint32_t nseg, int K, int bits, const uint32_t* __restrict__ tile_cnt,
                         const uint32_t* __restrict__ small,
                         uint32_t* __restrict__ seg_dim, uint32_t* __restrict__ seg_ones,
                         uint32_t* __restrict__ tile_ones_before,
                         uint32_t* __restrict__ out_n) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg || small[s]) return;   // (a small segment's out_n comes from k_small)
  const uint32_t nt = tiles_needed[s];
  if (nt == 0) {
    out_n[s] = 1;
    return;
  }
  const uint32_t t0 = tile_base[s], cnt = seg_count[s];
  const uint4 pl = seg_plen[s];
  int best = -1;
  uint32_t best_gap = 0xffffffffu, best_ones = 0;
  for (int j = 0; j < K; ++j) {
    if (byte_of(pl, j) >= (uint32_t)bits) continue;
    uint32_t ones = 0;
    for (uint32_t t = 0; t < nt; ++t) ones += tile_cnt[(int64_t)(t0 + t) * kMaxK + j];
    const uint32_t gap = (2u * ones > cnt) ? 2u * ones - cnt : cnt - 2u * ones;
    if (gap < best_gap) {
      best_gap = gap;
      best = j;
      best_ones = ones;
    }
  }
  seg_dim[s] = (uint32_t)best;
  seg_ones[s] = best_ones;
  uint32_t run = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    tile_ones_before[t0 + t] = run;
    run += tile_cnt[(int64_t)(t0 + t) * kMaxK + best];
  }
  out_n[s] = (best_ones > 0 ? 1u : 0u) + (best_ones < cnt ? 1u : 0u);
}

// Stable partition of each active segment by the chosen bit, into tmp.
__global__ void __launch_bounds__(LT)
k_tile_scatter(const uint32_t* __restrict__ tile_seg, const uint32_t* __restrict__ tile_base,
               const uint32_t* __restrict__ seg_start, const uint32_t* __restrict__ seg_count,
               const uint4* __restrict__ seg_plen, const uint32_t* __restrict__ seg_dim,
               const uint32_t* __restrict__ seg_ones, const uint32_t* __restrict__ tile_ones_before,
               const uint32_t* __restrict__ ids, const uint4* __restrict__ lcodes, int bits,
               uint32_t* __restrict__ tmp, uint4* __restrict__ tmpc) {
  __shared__ uint32_t s_warp[LT / 32];
  const uint32_t tile = blockIdx.x;
  const uint32_t s = tile_seg[tile];
  const uint32_t chunk = tile - tile_base[s];
  const uint32_t start = seg_start[s], count = seg_count[s];
  const int j = (int)seg_dim[s];
  const uint32_t shift = (uint32_t)(bits - 1) - byte_of(seg_plen[s], j);
  const uint32_t zeros_total = count - seg_ones[s];
  // contiguous items per thread keep the in-tile order for the scan
  uint32_t id[LIPT], bit[LIPT];
  uint4 cv[LIPT];
  uint32_t my_ones = 0;
#pragma unroll
  for (int r = 0; r < LIPT; ++r) {
    const uint32_t off = chunk * LTILE + threadIdx.x * LIPT + r;
    bit[r] = 2;
    if (off < count) {
      id[r] = ids[start + off];
      cv[r] = lcodes[start + off];
      bit[r] = (byte_of(cv[r], j) >> shift) & 1u;
      my_ones += bit[r];
    }
  }
  // exclusive scan of ones over threads
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = my_ones;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  uint32_t warp_before = 0;
  for (int q = 0; q < w; ++q) warp_before += s_warp[q];
  uint32_t ones_before = tile_ones_before[tile] + warp_before + x - my_ones;
#pragma unroll
  for (int r = 0; r < LIPT; ++r) {
    if (bit[r] > 1) continue;
    const uint32_t off = chunk * LTILE + threadIdx.x * LIPT + r;
    uint32_t dest;
    if (bit[r]) {
      dest = start + zeros_total + ones_before;
      ++ones_before;
    } else {
      dest = start + (off - ones_before);
    }
    tmp[dest] = id[r];
    tmpc[dest] = cv[r];
  }
}

__global__ void __launch_bounds__(LT)
k_tile_copyback(const uint32_t* __restrict__ tile_seg, const uint32_t* __restrict__ tile_base,
                const uint32_t* __restrict__ seg_start, const uint32_t* __restrict__ seg_count,
                const uint32_t* __restrict__ tmp, uint32_t* __restrict__ ids,
                const uint4* __restrict__ tmpc, uint4* __restrict__ lcodes) {
  const uint32_t tile = blockIdx.x;
  const uint32_t s = tile_seg[tile];
  const uint32_t chunk = tile - tile_base[s];
  const uint32_t start = seg_start[s], count = seg_count[s];
  for (int r = 0; r < LIPT; ++r) {
    const uint32_t off = chunk * LTILE + r * LT + threadIdx.x;
    if (off < count) {
      ids[start + off] = tmp[start + off];
      lcodes[start + off] = tmpc[start + off];
    }
  }
}

__global__ void k_emit(const uint32_t* __restrict__ tiles_needed, const uint32_t* __restrict__ out_pos,
                       const uint32_t* __restrict__ seg_start, const uint32_t* __restrict__ seg_count,
                       const uint4* __restrict__ seg_plen, const uint4* __restrict__ seg_prefix,
                       const uint32_t* __restrict__ seg_dim, const uint32_t* __restrict__ seg_ones,
                       const uint32_t* __restrict__ small,
                       uint32_t nseg, uint32_t* __restrict__ n_start, uint32_t* __restrict__ n_count,
                       uint4* __restrict__ n_plen, uint4* __restrict__ n_prefix) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg || small[s]) return;   // (k_small writes a small segment's leaves)
  uint32_t o = out_pos[s];
  const uint32_t start = seg_start[s], cnt = seg_count[s];
  const uint4 pl = seg_plen[s], pf = seg_prefix[s];
  if (tiles_needed[s] == 0) {
    n_start[o] = start;
    n_count[o] = cnt;
    n_plen[o] = pl;
    n_prefix[o] = pf;
    return;
  }
  const int j = (int)seg_dim[s];
  const uint32_t ones = seg_ones[s], zeros = cnt - ones;
  uint4 cpl = pl;
  set_byte(cpl, j, byte_of(pl, j) + 1);
  const uint32_t p2 = byte_of(pf, j) * 2;
  if (zeros) {
    uint4 cpf = pf;
    set_byte(cpf, j, p2);
    n_start[o] = start;
    n_count[o] = zeros;
    n_plen[o] = cpl;
    n_prefix[o] = cpf;
    ++o;
  }
  if (ones) {
    uint4 cpf = pf;
    set_byte(cpf, j, p2 + 1);
    n_start[o] = start + zeros;
    n_count[o] = ones;
    n_plen[o] = cpl;
    n_prefix[o] = cpf;
  }
}

// ---- dedup positions: pos0[p] = position of point p in tree 0's leaf order,
// then every entry of every tree mapped through it
__global__ void k_pos0(const uint32_t* __restrict__ ids0, int64_t n, uint32_t* __restrict__ pos0) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    pos0[ids0[j]] = (uint32_t)j;
}
__global__ void k_leaf_pos(const uint32_t* __restrict__ ids, int64_t total, const uint32_t* __restrict__ pos0,
                           uint32_t* __restrict__ pos) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x)
    pos[j] = pos0[ids[j]];
}

// ---- leaf table
__global__ void k_finalize(const uint32_t* __restrict__ seg_start, const uint32_t* __restrict__ seg_count,
                           const uint4* __restrict__ seg_plen, const uint4* __restrict__ seg_prefix,
                           uint32_t nseg, int64_t n, int K, int bits,
                           uint32_t* __restrict__ leaf_range, uint8_t* __restrict__ leaf_plen,
                           uint8_t* __restrict__ leaf_prefix, uint8_t* __restrict__ leaf_lo,
                           uint8_t* __restrict__ leaf_hi, uint16_t* __restrict__ leaf_tree,
                           int64_t* __restrict__ leaf_base, unsigned long long* __restrict__ max_count) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const uint32_t start = seg_start[s];
  const int64_t tree = (int64_t)start / n;
  leaf_range[2 * s] = (uint32_t)(start - tree * n);
  leaf_range[2 * s + 1] = seg_count[s];
  leaf_tree[s] = (uint16_t)tree;
  const uint4 pl = seg_plen[s], pf = seg_prefix[s];
  for (int j = 0; j < K; ++j) {
    const uint32_t l = byte_of(pl, j), p = byte_of(pf, j);
    const uint32_t lo = p << (bits - l);
    const uint32_t hi = lo + (1u << (bits - l)) - 1u;
    leaf_plen[s * K + j] = (uint8_t)l;
    leaf_prefix[s * K + j] = (uint8_t)p;
    leaf_lo[s * K + j] = (uint8_t)lo;
    leaf_hi[s * K + j] = (uint8_t)hi;
  }
  if (s == 0 || (int64_t)seg_start[s - 1] / n != tree) leaf_base[tree] = s;
  if (s == nseg - 1) leaf_base[tree + 1] = nseg;
  atomicMax(max_count, (unsigned long long)seg_count[s]);
}

// Segment list: start, count, prefix lengths and prefixes of each segment.
struct SegTable {
  Scratch st, cn, pl, pf;
  int64_t cap = 0;
  int reserve(int64_t n, cudaStream_t s) {
    if (n <= cap) return DETLSH_OK;
    cap = std::max<int64_t>(n, cap + cap / 2);
    st = Scratch();
    cn = Scratch();
    pl = Scratch();
    pf = Scratch();
    DL_TRY(st.alloc(sizeof(uint32_t) * cap, s));
    DL_TRY(cn.alloc(sizeof(uint32_t) * cap, s));
    DL_TRY(pl.alloc(sizeof(uint4) * cap, s));
    DL_TRY(pf.alloc(sizeof(uint4) * cap, s));
    return DETLSH_OK;
  }
  uint32_t* start() { return st.as<uint32_t>(); }
  uint32_t* count() { return cn.as<uint32_t>(); }
  uint4* plen() { return pl.as<uint4>(); }
  uint4* prefix() { return pf.as<uint4>(); }
};
// Per-segment work arrays of one level iteration (contents do not outlive it).
struct SegWork {
  static constexpr int kArrays = 9;
  Scratch a[kArrays];
  int64_t cap = 0;
  int reserve(int64_t n, cudaStream_t s) {
    if (n <= cap) return DETLSH_OK;
    cap = std::max<int64_t>(n, cap + cap / 2);
    for (auto& x : a) {
      x = Scratch();
      DL_TRY(x.alloc(sizeof(uint32_t) * cap, s));
    }
    return DETLSH_OK;
  }
  uint32_t* tiles_needed() { return a[0].as<uint32_t>(); }
  uint32_t* tile_base() { return a[1].as<uint32_t>(); }
  uint32_t* seg_dim() { return a[2].as<uint32_t>(); }
  uint32_t* seg_ones() { return a[3].as<uint32_t>(); }
  uint32_t* out_n() { return a[4].as<uint32_t>(); }
  uint32_t* out_pos() { return a[5].as<uint32_t>(); }
  uint32_t* small() { return a[6].as<uint32_t>(); }
  uint32_t* small_pos() { return a[7].as<uint32_t>(); }
  uint32_t* small_seg() { return a[8].as<uint32_t>(); }
};

int read_u32(const uint32_t* d, uint32_t* h, cudaStream_t s) {
  DL_CUDA(cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

}  // namespace

int build_leaves(detlsh_index* idx, cudaStream_t s) {
  const int64_t n = idx->n, L = idx->L, total = n * L;
  const int K = idx->K, bits = idx->bits;
  // ---- root level: one stable sort of all (tree, point) entries by (tree,
  // top-bit vector); the tree occupies the key bits above the K top bits
  Scratch keys_all, flags, pos, k0, v0, d_tot;
  DL_TRY(keys_all.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(flags.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(pos.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(k0.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(v0.alloc(sizeof(uint32_t) * total, s));
  DL_TRY(d_tot.alloc(sizeof(uint32_t) * 4, s));
  int tbits = 0;
  while ((1ll << tbits) < L) ++tbits;
  PhaseTimer tm(s);
  tm.begin(TR_LEAF_ROOT);
  k_root_keys<<<ceil_div(total, 256), 256, 0, s>>>(idx->codes, n, total, K, bits, k0.as<uint32_t>(),
                                                   v0.as<uint32_t>());
  DL_LAUNCH();
  DL_TRY(radix_sort_pairs(k0.as<uint32_t>(), v0.as<uint32_t>(), total, 0, K + tbits, keys_all.as<uint32_t>(),
                          idx->leaf_ids, s));
  k_root_flags<<<ceil_div(total, 256), 256, 0, s>>>(keys_all.as<uint32_t>(), total, flags.as<uint32_t>());
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32(flags.as<uint32_t>(), pos.as<uint32_t>(), total, d_tot.as<uint32_t>(), s));
  tm.end();
  uint32_t nseg = 0;
  DL_TRY(read_u32(d_tot.as<uint32_t>(), &nseg, s));

  // segment tables (ping-pong), grown to the segment count as it rises
  SegTable ta, tb;
  DL_TRY(ta.reserve(nseg, s));
  k_root_segments<<<ceil_div(total, 256), 256, 0, s>>>(flags.as<uint32_t>(), pos.as<uint32_t>(),
                                                       keys_all.as<uint32_t>(), total, n, K, bits, ta.start(),
                                                       ta.plen(), ta.prefix());
  DL_LAUNCH();
  k_seg_counts<<<ceil_div(nseg, 256), 256, 0, s>>>(ta.start(), nseg, n, total, ta.count());
  DL_LAUNCH();
  keys_all = Scratch();
  flags = Scratch();
  pos = Scratch();
  k0 = Scratch();
  v0 = Scratch();

  // per-segment work arrays (grown with the segment count) and the partition
  // buffers of the level passes
  SegWork wk;
  Scratch tmp;
  DL_TRY(tmp.alloc(sizeof(uint32_t) * total, s));
  int64_t tile_alloc = ceil_div(total, LTILE) + (int64_t)nseg + 1;
  Scratch tile_seg, tile_cnt, tile_ones_before;
  DL_TRY(tile_seg.alloc(sizeof(uint32_t) * tile_alloc, s));
  DL_TRY(tile_cnt.alloc(sizeof(uint32_t) * kMaxK * tile_alloc, s));
  DL_TRY(tile_ones_before.alloc(sizeof(uint32_t) * tile_alloc, s));
  uint32_t h_tot[2] = {0, 0};

  // codes in leaf order (and their partition buffer)
  Scratch lcodes, tmpc;
  DL_TRY(lcodes.alloc(sizeof(uint4) * total, s));
  DL_TRY(tmpc.alloc(sizeof(uint4) * total, s));
  tm.begin(TR_LEAF_GATHER);
  k_gather_codes<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 32), 256, 0, s>>>(
      idx->codes, idx->leaf_ids, n, total, K, lcodes.as<uint4>());
  DL_LAUNCH();
  const size_t small_smem = (size_t)2 * SCAP * (sizeof(uint4) + sizeof(uint32_t));
  DL_CUDA(cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_smem));

  tm.end();
  SegTable* cur = &ta;
  SegTable* nxt = &tb;
  tm.begin(TR_LEAF_LEVELS);
  int iters = 0;
  for (int iter = 0; iter < kMaxK * 8 + 2; ++iter, ++iters) {
    DL_TRY(wk.reserve(nseg, s));
    k_plan<<<ceil_div(nseg, 256), 256, 0, s>>>(cur->count(), cur->plen(), nseg, K, bits, idx->max_leaf,
                                               wk.tiles_needed(), wk.small());
    DL_LAUNCH();
    DL_TRY(exclusive_scan_u32(wk.tiles_needed(), wk.tile_base(), nseg, d_tot.as<uint32_t>(), s));
    DL_TRY(exclusive_scan_u32(wk.small(), wk.small_pos(), nseg, d_tot.as<uint32_t>() + 1, s));
    DL_CUDA(cudaMemcpyAsync(h_tot, d_tot.p, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, s));
    DL_CUDA(cudaStreamSynchronize(s));
    const uint32_t ntiles = h_tot[0], nsmall = h_tot[1];
    if (ntiles == 0 && nsmall == 0) break;
    if ((int64_t)ntiles > tile_alloc) {
      set_error("leaf build: tile table overflow (%u > %lld)", ntiles, (long long)tile_alloc);
      return DETLSH_EINTERNAL;
    }
    if (nsmall) {
      k_small_list<<<ceil_div(nseg, 256), 256, 0, s>>>(wk.small(), wk.small_pos(), nseg, wk.small_seg());
      DL_LAUNCH();
      k_small<<<nsmall, ST, small_smem, s>>>(wk.small_seg(), cur->start(), cur->count(), cur->plen(),
                                             cur->prefix(), lcodes.as<uint4>(), K, bits, idx->max_leaf,
                                             idx->leaf_ids, wk.out_n(), tmpc.as<uint4>());
      DL_LAUNCH();
    }
    if (ntiles) {
      k_tile_map<<<ceil_div(nseg, 256), 256, 0, s>>>(wk.tiles_needed(), wk.tile_base(), nseg,
                                                     tile_seg.as<uint32_t>());
      DL_LAUNCH();
      k_tile_count<<<ntiles, LT, 0, s>>>(tile_seg.as<uint32_t>(), wk.tile_base(), cur->start(), cur->count(),
                                         cur->plen(), lcodes.as<uint4>(), K, bits, tile_cnt.as<uint32_t>());
      DL_LAUNCH();
    }
    k_choose<<<ceil_div(nseg, 256), 256, 0, s>>>(wk.tiles_needed(), wk.tile_base(), cur->count(), cur->plen(), nseg,
                                                 K, bits, tile_cnt.as<uint32_t>(), wk.small(), wk.seg_dim(),
                                                 wk.seg_ones(), tile_ones_before.as<uint32_t>(), wk.out_n());
    DL_LAUNCH();
    if (ntiles) {
      k_tile_scatter<<<ntiles, LT, 0, s>>>(tile_seg.as<uint32_t>(), wk.tile_base(), cur->start(), cur->count(),
                                           cur->plen(), wk.seg_dim(), wk.seg_ones(), tile_ones_before.as<uint32_t>(),
                                           idx->leaf_ids, lcodes.as<uint4>(), bits, tmp.as<uint32_t>(),
                                           tmpc.as<uint4>());
      DL_LAUNCH();
      k_tile_copyback<<<ntiles, LT, 0, s>>>(tile_seg.as<uint32_t>(), wk.tile_base(), cur->start(), cur->count(),
                                            tmp.as<uint32_t>(), idx->leaf_ids, tmpc.as<uint4>(), lcodes.as<uint4>());
      DL_LAUNCH();
    }
    DL_TRY(exclusive_scan_u32(wk.out_n(), wk.out_pos(), nseg, d_tot.as<uint32_t>(), s));
    uint32_t nseg_new = 0;
    DL_TRY(read_u32(d_tot.as<uint32_t>(), &nseg_new, s));
    if ((int64_t)nseg_new > total) {
      set_error("leaf build: segment table overflow");
      return DETLSH_EINTERNAL;
    }
    DL_TRY(nxt->reserve(nseg_new, s));
    k_emit<<<ceil_div(nseg, 256), 256, 0, s>>>(wk.tiles_needed(), wk.out_pos(), cur->start(), cur->count(),
                                               cur->plen(), cur->prefix(), wk.seg_dim(), wk.seg_ones(), wk.small(),
                                               nseg, nxt->start(), nxt->count(), nxt->plen(), nxt->prefix());
    DL_LAUNCH();
    if (nsmall) {
      k_small_expand<<<ceil_div(nsmall, 8), 256, 0, s>>>(wk.small_seg(), nsmall, cur->start(), wk.out_n(),
                                                        wk.out_pos(), tmpc.as<uint4>(), idx->leaf_ids, idx->codes,
                                                        n, K, bits, nxt->start(), nxt->count(), nxt->plen(),
                                                        nxt->prefix());
      DL_LAUNCH();
    }
    std::swap(cur, nxt);
    nseg = nseg_new;
    // the tile tables must cover the next iteration's active segments
    const int64_t need = ceil_div(total, LTILE) + (int64_t)nseg + 1;
    if (need > tile_alloc) {
      tile_alloc = need;
      Scratch a2, b2, c2;
      DL_TRY(a2.alloc(sizeof(uint32_t) * tile_alloc, s));
      DL_TRY(b2.alloc(sizeof(uint32_t) * kMaxK * tile_alloc, s));
      DL_TRY(c2.alloc(sizeof(uint32_t) * tile_alloc, s));
      std::swap(tile_seg.p, a2.p);
      std::swap(tile_cnt.p, b2.p);
      std::swap(tile_ones_before.p, c2.p);
    }
  }
  tm.end();
  DL_TRY(tm.finish());
  if (trace_on()) trace_add(TR_LEAF_ITERS, iters);
  uint32_t* cs = cur->start();
  uint32_t* cc = cur->count();
  uint4* cpl = cur->plen();
  uint4* cpf = cur->prefix();

  // ---- leaf table
  idx->total_leaves = nseg;
  DL_TRY(index_alloc(&idx->leaf_range, sizeof(uint32_t) * 2 * nseg, s));
  DL_TRY(index_alloc(&idx->leaf_plen, (size_t)nseg * K, s));
  DL_TRY(index_alloc(&idx->leaf_prefix, (size_t)nseg * K, s));
  DL_TRY(index_alloc(&idx->leaf_lo, (size_t)nseg * K, s));
  DL_TRY(index_alloc(&idx->leaf_hi, (size_t)nseg * K, s));
  DL_TRY(index_alloc(&idx->leaf_tree, sizeof(uint16_t) * nseg, s));
  DL_TRY(index_alloc(&idx->leaf_base, sizeof(int64_t) * (L + 1), s));
  Scratch d_max;
  DL_TRY(d_max.alloc(sizeof(unsigned long long), s));
  DL_CUDA(cudaMemsetAsync(d_max.p, 0, sizeof(unsigned long long), s));
  k_finalize<<<ceil_div(nseg, 256), 256, 0, s>>>(cs, cc, cpl, cpf, nseg, n, K, bits,
                                                 idx->leaf_range, idx->leaf_plen, idx->leaf_prefix,
                                                 idx->leaf_lo, idx->leaf_hi, idx->leaf_tree,
                                                 idx->leaf_base, d_max.as<unsigned long long>());
  DL_LAUNCH();
  unsigned long long mx = 0;
  DL_CUDA(cudaMemcpyAsync(idx->leaf_base_h, idx->leaf_base, sizeof(int64_t) * (L + 1),
                          cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaMemcpyAsync(&mx, d_max.p, sizeof(mx), cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaStreamSynchronize(s));
  idx->max_leaf_count = (int64_t)mx;
  // When the walk CTAs' dedup bitmaps (n bits each, about three CTAs per SM)
  // do not fit in L2 together, the bitmap is indexed by tree-0 leaf position,
  // so that the points of one query's leaves set neighbouring bits instead of
  // bits spread over the whole id range.
  int dev = 0, nsm = 0, l2 = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  DL_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
  if ((idx->flags & DETLSH_DEDUP_POS) || (n + 7) / 8 * 3 * (int64_t)nsm > (int64_t)l2) {
    Scratch pos0;
    DL_TRY(pos0.alloc(sizeof(uint32_t) * n, s));
    DL_TRY(index_alloc(&idx->leaf_pos, sizeof(uint32_t) * total, s));
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 32);
    k_pos0<<<g, 256, 0, s>>>(idx->leaf_ids, n, pos0.as<uint32_t>());
    DL_LAUNCH();
    k_leaf_pos<<<g, 256, 0, s>>>(idx->leaf_ids, total, pos0.as<uint32_t>(), idx->leaf_pos);
    DL_LAUNCH();
  }
  return DETLSH_OK;
}

}  // namespace detlsh
