// Query phase: Alg. 7 (c^2-k-ANN) with the optimised range query of
// Sec. 6.2.2, for a batch of queries.
//
// k_leaf_lb   -- the squared lower-bound distance (Alg. 5, first step) of every
//               (query, leaf) pair. One thread owns one leaf and keeps its box
//               edges in registers while it loops over a chunk of queries whose
//               projections sit in shared memory, so the leaf table and the
//               breakpoints are read once per chunk of queries. It also folds
//               each query's smallest positive and largest bound into two
//               per-query words (for r_min and the round table).
// k_search    -- one CTA per query (persistent over the batch). Every leaf is
//               assigned the first round t whose projected threshold
//               (eps*r_t)^2 covers its lower bound; leaves are bucketed by
//               (round, tree). Buckets are visited in Alg. 7's order; a bucket
//               that cannot reach |S| >= beta*n+k is added whole (order inside
//               it does not change S), the one that can is cut at the first
//               leaf, in (lower bound, leaf number) order, where |S| reaches
//               the target -- found by a weighted radix select instead of a
//               sort. New points are deduplicated in a bitmap, their exact
//               distances computed warp-cooperatively from HBM (8 rows per warp
//               in flight, one transposed reduction, the 8 rows' bookkeeping in
//               8 lanes at once), counted per round for the ">= k within c*r"
//               test, and kept in a pruned top-k buffer in shared memory.
#include <algorithm>
#include <cfloat>

#include "common.cuh"

namespace detlsh {

namespace {

// ------------------------------------------------------------------ lower bounds
constexpr int LB_THREADS = 256;
constexpr int LB_QCH = 32;

__global__ void __launch_bounds__(LB_THREADS)
k_leaf_lb(const float* __restrict__ qp, int64_t nqb, int LK, const float* __restrict__ E, int Nr,
          int K, const uint8_t* __restrict__ leaf_lo, const uint8_t* __restrict__ leaf_hi,
          const uint16_t* __restrict__ leaf_tree, int64_t total_leaves, float* __restrict__ lb2,
          uint32_t* __restrict__ minpos, uint32_t* __restrict__ maxlb) {
  __shared__ float s_q[LB_QCH][kMaxLK + 1];
  __shared__ uint32_t s_min[LB_QCH], s_max[LB_QCH];
  const int64_t leaf = (int64_t)blockIdx.x * LB_THREADS + threadIdx.x;
  const int64_t qb0 = (int64_t)blockIdx.y * LB_QCH;
  const int nqc = (int)((nqb - qb0) < LB_QCH ? (nqb - qb0) : LB_QCH);
  for (int i = threadIdx.x; i < nqc * LK; i += LB_THREADS) {
    const int q = i / LK, r = i % LK;
    s_q[q][r] = qp[(qb0 + q) * LK + r];
  }
  if (threadIdx.x < LB_QCH) {
    s_min[threadIdx.x] = 0xffffffffu;
    s_max[threadIdx.x] = 0u;
  }
  __syncthreads();
  const bool valid = leaf < total_leaves;
  const int tree = valid ? leaf_tree[leaf] : 0;
  float el[kMaxK], eh[kMaxK];
#pragma unroll
  for (int j = 0; j < kMaxK; ++j) {
    el[j] = -INFINITY;
    eh[j] = INFINITY;
    if (valid && j < K) {
      const int r = tree * K + j;
      const int lo = leaf_lo[leaf * K + j], hi = leaf_hi[leaf * K + j];
      if (lo > 0) el[j] = __ldg(E + (int64_t)r * (Nr + 1) + lo);
      if (hi < Nr - 1) eh[j] = __ldg(E + (int64_t)r * (Nr + 1) + hi + 1);
    }
  }
  const int rbase = tree * K;
  for (int q = 0; q < nqc; ++q) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) {
      if (j < K) {
        const float x = s_q[q][rbase + j];
        const float a = __fsub_rn(el[j], x);
        const float b = __fsub_rn(x, eh[j]);
        const float dl = fmaxf(fmaxf(a, b), 0.f);
        acc = __fadd_rn(acc, __fmul_rn(dl, dl));
      }
    }
    if (valid) lb2[(qb0 + q) * total_leaves + leaf] = acc;
    // non-negative floats order like their bit patterns
    uint32_t mn = (valid && acc > 0.f) ? __float_as_uint(acc) : 0xffffffffu;
    uint32_t mx = valid ? __float_as_uint(acc) : 0u;
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&s_min[q], mn);
      atomicMax(&s_max[q], mx);
    }
  }
  __syncthreads();
  if (threadIdx.x < nqc) {
    atomicMin(&minpos[qb0 + threadIdx.x], s_min[threadIdx.x]);
    atomicMax(&maxlb[qb0 + threadIdx.x], s_max[threadIdx.x]);
  }
}

// ------------------------------------------------------------------ search
constexpr int ST = 512;           // threads per search CTA
constexpr int NW = ST / 32;
constexpr int TK_CAP = 4096;      // top-k buffer entries
constexpr int QCAP = 3072;        // new points per batch (<= TK_CAP - kMaxTopK)
constexpr int BATCH_LEAVES = ST;  // leaves examined per batch step
constexpr int ILP = 8;            // rows per warp in flight (the transposed reduction assumes 8)
static_assert(QCAP + kMaxTopK <= TK_CAP, "top-k buffer too small for a batch");

struct SearchArgs {
  const void* X;
  int dtype;
  int64_t n;
  int d;
  int K, L, Nr;
  const uint32_t* leaf_ids;
  const uint32_t* leaf_range;
  const uint16_t* leaf_tree;
  int64_t total_leaves;
  const void* Q;
  int64_t q0, nqb;
  const float* lb2;
  const uint32_t* minpos;
  const uint32_t* maxlb;
  const int32_t* k;
  const float* c;
  const float* r_min;
  double eps, beta;
  int k_max;
  int64_t* out_ids;
  float* out_dist;
  int32_t* out_stats;
  uint32_t* cand_ids;
  int64_t cand_cap;
  uint32_t* ws_list;
  uint32_t* ws_newcnt;
  uint8_t* ws_round;
  uint32_t* ws_bitmap;
  int64_t bitmap_words;
  int smem_bitmap;
};

struct SmemLayout {
  size_t thrP, thrC, cnt, pts, boff, hist_u, tk, queue, bpref, bleaf, bstart, fmap, sel, misc, bitmap,
      total;
};

__host__ __device__ inline SmemLayout search_layout(int L, int64_t smem_bitmap_words) {
  SmemLayout o{};
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p += (bytes + 15) & ~size_t(15);
    return at;
  };
  const size_t RL = (size_t)kRoundCap * L;
  o.thrP = take(sizeof(float) * kRoundCap);
  o.thrC = take(sizeof(float) * kRoundCap);
  o.cnt = take(sizeof(uint32_t) * RL);
  o.pts = take(sizeof(uint32_t) * RL);
  o.boff = take(sizeof(uint32_t) * (RL + 1));
  o.hist_u = take(sizeof(uint32_t) * (kRoundCap + 1));
  o.tk = take(sizeof(unsigned long long) * TK_CAP);
  o.queue = take(sizeof(uint32_t) * QCAP);
  o.bpref = take(sizeof(uint32_t) * (BATCH_LEAVES + 1));
  o.bleaf = take(sizeof(uint32_t) * BATCH_LEAVES);
  o.bstart = take(sizeof(uint32_t) * BATCH_LEAVES);
  o.fmap = take(sizeof(uint16_t) * QCAP);
  o.sel = take(sizeof(unsigned long long) * 256);
  o.misc = take(sizeof(unsigned long long) * 64);
  o.bitmap = take(sizeof(uint32_t) * (size_t)smem_bitmap_words);
  o.total = p;
  return o;
}

// misc slots (unsigned long long each)
enum {
  M_S = 0, M_T, M_TAU, M_TKN, M_QN, M_STOP, M_TLAST, M_TCAP, M_RU, M_NEED, M_KSTAR, M_ACC,
  M_TOTNEW, M_LEAFA, M_OFFA
};

// index of the first element >= v in a non-decreasing array (n if none)
__device__ __forceinline__ int lower_bound_f(const float* a, int n, float v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Bitonic sort of TK_CAP keys ascending (block-wide).
__device__ void sort_topk(unsigned long long* tk) {
  for (int size = 2; size <= TK_CAP; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < TK_CAP / 2; i += ST) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const unsigned long long a = tk[lo], b = tk[hi];
        if ((a > b) == up) {
          tk[lo] = b;
          tk[hi] = a;
        }
      }
    }
  }
  __syncthreads();
}

// Keep the k smallest keys of the buffer; tau becomes the largest kept key
// once k keys are held.
__device__ void prune_topk(unsigned long long* tk, unsigned long long* misc, int k) {
  __syncthreads();
  const int cnt = (int)min(misc[M_TKN], (unsigned long long)TK_CAP);
  for (int i = cnt + threadIdx.x; i < TK_CAP; i += ST) tk[i] = ~0ull;
  sort_topk(tk);
  if (threadIdx.x == 0) {
    const int keep = min(cnt, k);
    misc[M_TKN] = keep;
    if (keep == k) misc[M_TAU] = tk[k - 1];
  }
  __syncthreads();
}

template <typename TX>
struct Vec4Of;
template <>
struct Vec4Of<float> {
  using T = float4;
  static __device__ __forceinline__ float4 ld(const float* p, int64_t i) {
    return __ldg(reinterpret_cast<const float4*>(p) + i);
  }
  static __device__ __forceinline__ float4 f(const float4& v) { return v; }
};
template <>
struct Vec4Of<uint8_t> {
  using T = uchar4;
  static __device__ __forceinline__ uchar4 ld(const uint8_t* p, int64_t i) {
    return __ldg(reinterpret_cast<const uchar4*>(p) + i);
  }
  static __device__ __forceinline__ float4 f(const uchar4& v) {
    return make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
  }
};

// Partial squared distances of ILP rows (ids[u] == ~0u: no row) to q; each
// lane covers a strided slice of the d coordinates, all rows' loads of a
// slice are issued before their arithmetic.
template <typename TX>
__device__ __forceinline__ void rows_dist2(const TX* __restrict__ X, int d,
                                           const uint32_t* ids, const TX* __restrict__ q,
                                           bool vec4, int lane, float* acc) {
  using V = Vec4Of<TX>;
  if (vec4) {
    const int d4 = d >> 2;
    for (int i = lane; i < d4; i += 32) {
      const typename V::T qv = V::ld(q, i);
      typename V::T xv[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u)
        xv[u] = (ids[u] != 0xffffffffu) ? V::ld(X + (int64_t)ids[u] * d, i) : qv;
      const float4 qf = V::f(qv);
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        const float4 xf = V::f(xv[u]);
        const float d0 = xf.x - qf.x, d1 = xf.y - qf.y, d2 = xf.z - qf.z, d3 = xf.w - qf.w;
        acc[u] = fmaf(d0, d0, acc[u]);
        acc[u] = fmaf(d1, d1, acc[u]);
        acc[u] = fmaf(d2, d2, acc[u]);
        acc[u] = fmaf(d3, d3, acc[u]);
      }
    }
  } else {
    for (int i = lane; i < d; i += 32) {
      const float qf = (float)__ldg(q + i);
      float xv[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u)
        xv[u] = (ids[u] != 0xffffffffu) ? (float)__ldg(X + (int64_t)ids[u] * d + i) : qf;
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        const float t = xv[u] - qf;
        acc[u] = fmaf(t, t, acc[u]);
      }
    }
  }
}

// Sum 8 per-lane partials over the warp so that lane l ends with the total of
// row (l >> 2) & 7: three halving exchanges (16, 8, 4) each keep half of the
// rows, then two plain butterfly steps.
__device__ __forceinline__ float transpose_reduce8(const float* acc, int lane) {
  float a4[4], a2[2];
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b4 ? acc[i] : acc[i + 4];
    const float keep = b4 ? acc[i + 4] : acc[i];
    a4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b3 ? a4[i] : a4[i + 2];
    const float keep = b3 ? a4[i + 2] : a4[i];
    a2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b2 ? a2[0] : a2[1];
  const float keep = b2 ? a2[1] : a2[0];
  float v = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// Add the points of bucket leaves list[0..nl) (only leaves whose select key is
// <= kstar when filtered) to S. Runs in batches of at most QCAP points: the
// batch's points are tested-and-set in the bitmap, the new ones queued, then
// their distances computed by warps.
template <typename TX>
__device__ void add_leaves(const SearchArgs& a, const TX* __restrict__ X, const TX* __restrict__ q,
                           bool vec4, const uint32_t* list, uint32_t nl, bool filtered,
                           unsigned long long kstar, const float* lbrow, int tree, int kq,
                           int Ru, unsigned char* sm, const SmemLayout& ly, uint32_t* bitmap,
                           int64_t qglob) {
  unsigned long long* misc = reinterpret_cast<unsigned long long*>(sm + ly.misc);
  unsigned long long* tk = reinterpret_cast<unsigned long long*>(sm + ly.tk);
  uint32_t* queue = reinterpret_cast<uint32_t*>(sm + ly.queue);
  uint32_t* bpref = reinterpret_cast<uint32_t*>(sm + ly.bpref);
  uint32_t* bstart = reinterpret_cast<uint32_t*>(sm + ly.bstart);
  uint16_t* fmap = reinterpret_cast<uint16_t*>(sm + ly.fmap);
  uint32_t* hist_u = reinterpret_cast<uint32_t*>(sm + ly.hist_u);
  const float* thrC = reinterpret_cast<const float*>(sm + ly.thrC);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t* tree_ids = a.leaf_ids + (int64_t)tree * a.n;
  __shared__ uint32_t s_w[NW];

  if (threadIdx.x == 0) {
    misc[M_LEAFA] = 0;
    misc[M_OFFA] = 0;
  }
  __syncthreads();
  while (true) {
    const uint32_t la = (uint32_t)misc[M_LEAFA];
    const uint32_t offa = (uint32_t)misc[M_OFFA];
    if (la >= nl) break;
    // --- batch: leaves [la, la+nb) with their (filtered) counts, the first one from offa
    const uint32_t nb = min((uint32_t)BATCH_LEAVES, nl - la);
    uint32_t cnt = 0;
    if (threadIdx.x < nb) {
      const uint32_t leaf = list[la + threadIdx.x];
      const uint32_t st = a.leaf_range[2 * (int64_t)leaf];
      cnt = a.leaf_range[2 * (int64_t)leaf + 1];
      if (filtered) {
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(lbrow[leaf]) << 32) | (unsigned long long)leaf;
        if (key > kstar) cnt = 0;
      }
      if (threadIdx.x == 0) cnt = cnt >= offa ? cnt - offa : 0u;
      bstart[threadIdx.x] = st + (threadIdx.x == 0 ? offa : 0u);
    }
    // inclusive scan of cnt over the block (ST == BATCH_LEAVES)
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    uint32_t wb = 0;
    for (int qq = 0; qq < w; ++qq) wb += s_w[qq];
    bpref[threadIdx.x + 1] = wb + x;   // bpref[j] = points before leaf j of the batch
    if (threadIdx.x == 0) bpref[0] = 0;
    __syncthreads();
    // batch extent: whole leaves while they fit in QCAP points, at least one (partially)
    uint32_t take_leaves, take_pts;
    {
      int lo = 0, hi = (int)nb;   // largest j with bpref[j] <= QCAP
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bpref[mid] <= (uint32_t)QCAP) lo = mid;
        else hi = mid - 1;
      }
      take_leaves = (uint32_t)lo;
      take_pts = bpref[lo];
      if (take_leaves == 0) take_pts = min(bpref[1], (uint32_t)QCAP);
    }
    // flat point -> batch leaf map (a warp per leaf)
    const uint32_t map_leaves = take_leaves == 0 ? 1u : take_leaves;
    for (uint32_t j = (uint32_t)w; j < map_leaves; j += NW) {
      const uint32_t e = min(bpref[j + 1], take_pts);
      for (uint32_t f = bpref[j] + lane; f < e; f += 32) fmap[f] = (uint16_t)j;
    }
    // make room in the top-k buffer for up to take_pts insertions
    if (misc[M_TKN] + take_pts > TK_CAP) prune_topk(tk, misc, kq);
    if (threadIdx.x == 0) misc[M_QN] = 0;
    __syncthreads();
    // --- phase A: test-and-set, queue the new points
    for (uint32_t f0 = 0; f0 < take_pts; f0 += ST) {
      const uint32_t f = f0 + threadIdx.x;
      bool fresh = false;
      uint32_t id = 0;
      if (f < take_pts) {
        const uint32_t j = fmap[f];
        id = tree_ids[bstart[j] + (f - bpref[j])];
        const uint32_t bit = 1u << (id & 31);
        const uint32_t old = atomicOr(bitmap + (id >> 5), bit);
        fresh = !(old & bit);
      }
      const uint32_t m = __ballot_sync(0xffffffffu, fresh);
      uint32_t base = 0;
      if (lane == 0 && m) base = (uint32_t)atomicAdd(&misc[M_QN], (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (fresh) queue[base + __popc(m & lt)] = id;
    }
    __syncthreads();
    const uint32_t qn = (uint32_t)misc[M_QN];
    const unsigned long long S_before = misc[M_S];
    const unsigned long long tau = misc[M_TAU];
    // --- phase B: exact distances of the queued points, 8 rows per warp
    for (uint32_t e0 = (uint32_t)w * ILP; e0 < qn; e0 += NW * ILP) {
      float acc[ILP];
      uint32_t ids[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        ids[u] = (e0 + u < qn) ? queue[e0 + u] : 0xffffffffu;
        acc[u] = 0.f;
      }
      rows_dist2<TX>(X, a.d, ids, q, vec4, lane, acc);
      const float d2 = transpose_reduce8(acc, lane);
      const uint32_t r = (uint32_t)(lane >> 2) & 7u;
      if ((lane & 3) == 0 && e0 + r < qn) {
        const uint32_t id = queue[e0 + r];
        const int uu = lower_bound_f(thrC, Ru, d2);
        atomicAdd(&hist_u[min(uu, kRoundCap)], 1u);
        const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | id;
        if (key < tau) {
          const unsigned long long slot = atomicAdd(&misc[M_TKN], 1ull);
          if (slot < TK_CAP) tk[slot] = key;
        }
        if (a.cand_ids) {
          const unsigned long long pos = S_before + e0 + r;
          if ((int64_t)pos < a.cand_cap) a.cand_ids[qglob * a.cand_cap + (int64_t)pos] = id;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      misc[M_S] += qn;
      // advance the batch cursor
      if (take_leaves == 0) {
        const uint32_t first_total = bpref[1] + offa;  // points of leaf la (after filter)
        const uint32_t newoff = offa + take_pts;
        if (newoff >= first_total) {
          misc[M_LEAFA] = la + 1;
          misc[M_OFFA] = 0;
        } else {
          misc[M_OFFA] = newoff;
        }
      } else {
        misc[M_LEAFA] = la + take_leaves;
        misc[M_OFFA] = 0;
      }
    }
    __syncthreads();
  }
}

template <typename TX>
__global__ void __launch_bounds__(ST, 1) k_search(SearchArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int64_t smem_words = a.smem_bitmap ? a.bitmap_words : 0;
  const SmemLayout ly = search_layout(a.L, smem_words);
  float* thrP = reinterpret_cast<float*>(sm + ly.thrP);
  float* thrC = reinterpret_cast<float*>(sm + ly.thrC);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(sm + ly.cnt);
  uint32_t* s_pts = reinterpret_cast<uint32_t*>(sm + ly.pts);
  uint32_t* s_boff = reinterpret_cast<uint32_t*>(sm + ly.boff);
  uint32_t* hist_u = reinterpret_cast<uint32_t*>(sm + ly.hist_u);
  unsigned long long* tk = reinterpret_cast<unsigned long long*>(sm + ly.tk);
  unsigned long long* sel = reinterpret_cast<unsigned long long*>(sm + ly.sel);
  unsigned long long* misc = reinterpret_cast<unsigned long long*>(sm + ly.misc);
  uint32_t* bitmap = a.smem_bitmap ? reinterpret_cast<uint32_t*>(sm + ly.bitmap)
                                   : a.ws_bitmap + (int64_t)blockIdx.x * a.bitmap_words;
  uint32_t* list = a.ws_list + (int64_t)blockIdx.x * a.total_leaves;
  uint32_t* newcnt = a.ws_newcnt + (int64_t)blockIdx.x * a.total_leaves;
  uint8_t* lround = a.ws_round + (int64_t)blockIdx.x * a.total_leaves;
  const TX* X = static_cast<const TX*>(a.X);
  const int L = a.L;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  __shared__ unsigned long long s_red_u[NW];
  const bool vec4 = (a.d % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(a.X) % (sizeof(TX) == 4 ? 16 : 4) == 0) &&
                    (reinterpret_cast<uintptr_t>(a.Q) % (sizeof(TX) == 4 ? 16 : 4) == 0);
  // every lane of a warp runs the same number of leaf iterations (warp-aggregated atomics)
  const int64_t leaf_iters = (a.total_leaves + ST - 1) / ST * ST;

  for (int64_t qb = blockIdx.x; qb < a.nqb; qb += gridDim.x) {
    const int64_t qg = a.q0 + qb;
    const float* lbrow = a.lb2 + qb * a.total_leaves;
    const TX* q = static_cast<const TX*>(a.Q) + qg * a.d;
    const int kq = a.k[qg];
    // ---- reset per-query state
    for (int64_t i = threadIdx.x; i < a.bitmap_words; i += ST) bitmap[i] = 0u;
    for (int i = threadIdx.x; i < kRoundCap * L; i += ST) {
      s_cnt[i] = 0;
      s_pts[i] = 0;
    }
    for (int i = threadIdx.x; i <= kRoundCap; i += ST) hist_u[i] = 0;
    if (threadIdx.x == 0) {
      misc[M_S] = 0;
      misc[M_TKN] = 0;
      misc[M_TAU] = ~0ull;
      misc[M_STOP] = 0;
      misc[M_TLAST] = 0;
      // Alg. 7 thresholds: r_0 = r_min, r_{t+1} = c * r_t (FP64), rounded once to FP32
      const uint32_t mnb = a.minpos[qb];
      const float m2 = __uint_as_float(a.maxlb[qb]);
      double r = (double)a.r_min[qg];
      if (!(r > 0.0)) r = (mnb != 0xffffffffu) ? sqrt((double)__uint_as_float(mnb)) / a.eps : 1.0;
      const double cq = (double)a.c[qg];
      int Ru = kRoundCap;
      for (int t = 0; t < kRoundCap; ++t) {
        if (t == kRoundCap - 1) {
          thrP[t] = INFINITY;
          thrC[t] = INFINITY;
          break;
        }
        const double er = __dmul_rn(a.eps, r), cr = __dmul_rn(cq, r);
        thrP[t] = __double2float_rn(__dmul_rn(er, er));
        thrC[t] = __double2float_rn(__dmul_rn(cr, cr));
        r = __dmul_rn(r, cq);
        if (thrP[t] >= m2) {
          Ru = t + 1;
          break;
        }
      }
      misc[M_RU] = (unsigned long long)Ru;
      misc[M_T] = (unsigned long long)ceil(__dadd_rn(__dmul_rn(a.beta, (double)a.n), (double)kq));
    }
    __syncthreads();
    const int Ru = (int)misc[M_RU];
    const unsigned long long T = misc[M_T];
    // ---- pass A: round of each leaf; histogram per (round, tree), warp-aggregated
    uint32_t tl = 0;
    for (int64_t l = threadIdx.x; l < leaf_iters; l += ST) {
      const bool valid = l < a.total_leaves;
      uint32_t key = 0xffffffffu, pts = 0;
      if (valid) {
        const int t = lower_bound_f(thrP, Ru, lbrow[l]);
        lround[l] = (uint8_t)t;
        key = (uint32_t)(t * L + a.leaf_tree[l]);
        pts = a.leaf_range[2 * l + 1];
        tl = max(tl, (uint32_t)t);
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, key);
      const uint32_t sum = __reduce_add_sync(peers, pts);
      if (valid && (peers & lt) == 0) {
        atomicAdd(&s_cnt[key], (uint32_t)__popc(peers));
        atomicAdd(&s_pts[key], sum);
      }
    }
    tl = __reduce_max_sync(0xffffffffu, tl);
    if (lane == 0) atomicMax(&misc[M_TLAST], (unsigned long long)tl);
    __syncthreads();
    if (threadIdx.x == 0) {
      // rounds past the first one where some tree alone holds T points are never reached
      const int tlast = (int)misc[M_TLAST];
      int tcap = tlast;
      unsigned long long cum[kMaxL];
      for (int i = 0; i < L; ++i) cum[i] = 0;
      for (int t = 0; t <= tlast && tcap == tlast; ++t) {
        for (int i = 0; i < L; ++i) {
          cum[i] += s_pts[t * L + i];
          if (cum[i] >= T) tcap = t;
        }
      }
      misc[M_TCAP] = (unsigned long long)tcap;
      uint32_t run = 0;
      for (int b = 0; b < (tcap + 1) * L; ++b) {
        s_boff[b] = run;
        run += s_cnt[b];
      }
      s_boff[(tcap + 1) * L] = run;
    }
    __syncthreads();
    const int tcap = (int)misc[M_TCAP];
    const int tlast = (int)misc[M_TLAST];
    // s_cnt now keeps each bucket's point total, s_pts becomes the insertion cursor
    for (int i = threadIdx.x; i < (tcap + 1) * L; i += ST) {
      s_cnt[i] = s_pts[i];
      s_pts[i] = s_boff[i];
    }
    __syncthreads();
    // ---- pass B: bucket the leaves of rounds <= tcap
    for (int64_t l = threadIdx.x; l < leaf_iters; l += ST) {
      uint32_t key = 0xffffffffu;
      if (l < a.total_leaves) {
        const int t = lround[l];
        if (t <= tcap) key = (uint32_t)(t * L + a.leaf_tree[l]);
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (key != 0xffffffffu && lane == leader) base = atomicAdd(&s_pts[key], (uint32_t)__popc(peers));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (key != 0xffffffffu) list[base + __popc(peers & lt)] = (uint32_t)l;
    }
    __syncthreads();
    // ---- walk the buckets in Alg. 7 order
    int t_stop = tcap;
    for (int t = 0; t <= tcap; ++t) {
      for (int i = 0; i < L; ++i) {
        const int b = t * L + i;
        const uint32_t nl = s_boff[b + 1] - s_boff[b];
        if (nl == 0) continue;
        const uint32_t* bl = list + s_boff[b];
        // upper bound on the points this bucket can add: all of its points
        const unsigned long long bpts = s_cnt[b];
        const unsigned long long S0 = misc[M_S];
        bool cut = false;
        if (S0 + bpts >= T) {
          // count the new points of every leaf of the bucket (no bitmap update)
          unsigned long long tot = 0;
          for (uint32_t j = (uint32_t)w; j < nl; j += NW) {
            const uint32_t lf = bl[j];
            const uint32_t st = a.leaf_range[2 * (int64_t)lf], ct = a.leaf_range[2 * (int64_t)lf + 1];
            const uint32_t* ids = a.leaf_ids + (int64_t)i * a.n + st;
            uint32_t nw = 0;
            for (uint32_t e = lane; e < ct; e += 32) {
              const uint32_t id = ids[e];
              nw += (bitmap[id >> 5] >> (id & 31)) & 1u ? 0u : 1u;
            }
            nw = __reduce_add_sync(0xffffffffu, nw);
            if (lane == 0) newcnt[j] = nw;
            tot += nw;
          }
          if (lane == 0) s_red_u[w] = tot;
          __syncthreads();
          if (threadIdx.x == 0) {
            unsigned long long sum = 0;
            for (int qq = 0; qq < NW; ++qq) sum += s_red_u[qq];
            misc[M_TOTNEW] = sum;
          }
          __syncthreads();
          cut = (S0 + misc[M_TOTNEW] >= T);
        }
        unsigned long long kstar = ~0ull;
        if (cut) {
          // weighted radix select: the smallest key (lower bound, leaf) whose
          // prefix of new points reaches T - |S|
          if (threadIdx.x == 0) {
            misc[M_NEED] = T - S0;
            misc[M_KSTAR] = 0;
            misc[M_ACC] = 0;
          }
          __syncthreads();
          unsigned long long prefix = 0, pmask = 0;
          for (int p = 7; p >= 0; --p) {
            for (int i2 = threadIdx.x; i2 < 256; i2 += ST) sel[i2] = 0;
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < nl; j += ST) {
              const uint32_t lf = bl[j];
              const unsigned long long key =
                  ((unsigned long long)__float_as_uint(lbrow[lf]) << 32) | (unsigned long long)lf;
              if ((key & pmask) == prefix && newcnt[j])
                atomicAdd(&sel[(key >> (8 * p)) & 255ull], (unsigned long long)newcnt[j]);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
              unsigned long long acc = misc[M_ACC];
              const unsigned long long need = misc[M_NEED];
              int dg = 0;
              for (; dg < 256; ++dg) {
                if (acc + sel[dg] >= need) break;
                acc += sel[dg];
              }
              misc[M_ACC] = acc;
              misc[M_KSTAR] = prefix | ((unsigned long long)dg << (8 * p));
            }
            __syncthreads();
            prefix = misc[M_KSTAR];
            pmask |= 255ull << (8 * p);
          }
          kstar = prefix;
        }
        add_leaves<TX>(a, X, q, vec4, bl, nl, cut, kstar, lbrow, i, kq, Ru, sm, ly, bitmap, qg);
        if (cut) {
          if (threadIdx.x == 0) misc[M_STOP] = 1;
          break;
        }
      }
      __syncthreads();
      if (misc[M_STOP]) {
        t_stop = t;
        break;
      }
      if (threadIdx.x == 0) {
        unsigned long long within = 0;
        for (int u = 0; u <= t; ++u) within += hist_u[u];
        if (within >= (unsigned long long)kq) misc[M_STOP] = 2;
        else if (t == tlast) misc[M_STOP] = 3;
      }
      __syncthreads();
      if (misc[M_STOP]) {
        t_stop = t;
        break;
      }
    }
    // ---- top-k output
    prune_topk(tk, misc, kq);
    const int have = (int)misc[M_TKN];
    for (int r = threadIdx.x; r < a.k_max; r += ST) {
      int64_t id = -1;
      float dist = INFINITY;
      if (r < have && r < kq) {
        const unsigned long long key = tk[r];
        id = (int64_t)(key & 0xffffffffull);
        dist = sqrtf(__uint_as_float((uint32_t)(key >> 32)));
      }
      a.out_ids[qg * a.k_max + r] = id;
      a.out_dist[qg * a.k_max + r] = dist;
    }
    if (threadIdx.x == 0 && a.out_stats) {
      a.out_stats[qg * 4 + 0] = (int32_t)misc[M_S];
      a.out_stats[qg * 4 + 1] = t_stop + 1;
      a.out_stats[qg * 4 + 2] = (int32_t)misc[M_STOP];
      a.out_stats[qg * 4 + 3] = 0;
    }
    __syncthreads();
  }
}

}  // namespace

int run_query(const detlsh_index* idx, const void* Q, int64_t nq, const int32_t* k, const float* c,
              const float* r_min, int k_max, double eps, double beta, int64_t* out_ids,
              float* out_dist, int32_t* out_stats, uint32_t* cand_ids, int64_t cand_cap,
              cudaStream_t s) {
  if (nq == 0) return DETLSH_OK;
  const int LK = idx->K * idx->L;
  int dev = 0, nsm = 0, smem_optin = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  DL_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

  // projected queries
  Scratch qp;
  DL_TRY(qp.alloc(sizeof(float) * nq * LK, s));
  PhaseTimer tm(s);
  tm.begin(TR_QUERY_PROJ);
  DL_TRY(launch_project_t(Q, idx->dtype, nq, idx->d, nullptr, idx->At, LK, qp.as<float>(), LK, 1,
                          s));
  tm.end();

  // search configuration (static shared memory of the kernel: < 1 KiB)
  const int64_t words = (idx->n + 31) / 32;
  const SmemLayout base = search_layout(idx->L, 0);
  const bool smem_bitmap = (int64_t)base.total + words * 4 + 1024 <= (int64_t)smem_optin;
  const SmemLayout ly = search_layout(idx->L, smem_bitmap ? words : 0);
  if ((int64_t)ly.total + 1024 > smem_optin) {
    set_error("search kernel needs %zu bytes of shared memory", ly.total);
    return DETLSH_EINVAL;
  }
  // batch size bounded by the lower-bound buffer (<= ~2 GiB)
  const int64_t per_q = idx->total_leaves * (int64_t)sizeof(float);
  int64_t qb = std::max<int64_t>(1, std::min<int64_t>(nq, ((int64_t)2 << 30) / std::max<int64_t>(per_q, 1)));
  qb = std::min<int64_t>(qb, 8192);
  const int grid = (int)std::min<int64_t>(qb, nsm);
  Scratch lb, mm, ws_list, ws_new, ws_round, ws_bm;
  DL_TRY(lb.alloc(sizeof(float) * qb * idx->total_leaves, s));
  DL_TRY(mm.alloc(sizeof(uint32_t) * 2 * qb, s));
  DL_TRY(ws_list.alloc(sizeof(uint32_t) * grid * idx->total_leaves, s));
  DL_TRY(ws_new.alloc(sizeof(uint32_t) * grid * idx->total_leaves, s));
  DL_TRY(ws_round.alloc((size_t)grid * idx->total_leaves, s));
  if (!smem_bitmap) DL_TRY(ws_bm.alloc(sizeof(uint32_t) * grid * words, s));
  uint32_t* d_min = mm.as<uint32_t>();
  uint32_t* d_max = d_min + qb;

  auto kern = idx->dtype == DETLSH_U8 ? k_search<uint8_t> : k_search<float>;
  DL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ly.total));

  for (int64_t q0 = 0; q0 < nq; q0 += qb) {
    const int64_t nqb = std::min<int64_t>(qb, nq - q0);
    DL_CUDA(cudaMemsetAsync(d_min, 0xff, sizeof(uint32_t) * nqb, s));
    DL_CUDA(cudaMemsetAsync(d_max, 0x00, sizeof(uint32_t) * nqb, s));
    dim3 g1(ceil_div(idx->total_leaves, LB_THREADS), ceil_div(nqb, LB_QCH));
    tm.begin(TR_LB);
    k_leaf_lb<<<g1, LB_THREADS, 0, s>>>(qp.as<float>() + q0 * LK, nqb, LK, idx->E, idx->Nr, idx->K,
                                        idx->leaf_lo, idx->leaf_hi, idx->leaf_tree,
                                        idx->total_leaves, lb.as<float>(), d_min, d_max);
    DL_LAUNCH();
    tm.end();
    trace_add(TR_LB_LAUNCHES, 1.0);
    SearchArgs sa{};
    sa.X = idx->X;
    sa.dtype = idx->dtype;
    sa.n = idx->n;
    sa.d = idx->d;
    sa.K = idx->K;
    sa.L = idx->L;
    sa.Nr = idx->Nr;
    sa.leaf_ids = idx->leaf_ids;
    sa.leaf_range = idx->leaf_range;
    sa.leaf_tree = idx->leaf_tree;
    sa.total_leaves = idx->total_leaves;
    sa.Q = Q;
    sa.q0 = q0;
    sa.nqb = nqb;
    sa.lb2 = lb.as<float>();
    sa.minpos = d_min;
    sa.maxlb = d_max;
    sa.k = k;
    sa.c = c;
    sa.r_min = r_min;
    sa.eps = eps;
    sa.beta = beta;
    sa.k_max = k_max;
    sa.out_ids = out_ids;
    sa.out_dist = out_dist;
    sa.out_stats = out_stats;
    sa.cand_ids = cand_ids;
    sa.cand_cap = cand_cap;
    sa.ws_list = ws_list.as<uint32_t>();
    sa.ws_newcnt = ws_new.as<uint32_t>();
    sa.ws_round = ws_round.as<uint8_t>();
    sa.ws_bitmap = smem_bitmap ? nullptr : ws_bm.as<uint32_t>();
    sa.bitmap_words = words;
    sa.smem_bitmap = smem_bitmap ? 1 : 0;
    const int gq = (int)std::min<int64_t>(nqb, grid);
    tm.begin(TR_SEARCH);
    kern<<<gq, ST, ly.total, s>>>(sa);
    DL_LAUNCH();
    tm.end();
    trace_add(TR_SEARCH_LAUNCHES, 1.0);
  }
  DL_TRY(tm.finish());
  return DETLSH_OK;
}

}  // namespace detlsh
