// Query phase: Alg. 7 (c^2-k-ANN) with the optimised range query of
// Sec. 6.2.2, for a batch of queries.
//
// k_leaf_lb   -- squared lower-bound distance (Alg. 5, first step) of every
//               (query, leaf) pair. One thread owns one leaf and keeps its box
//               edges in registers while it loops over a chunk of queries whose
//               projections sit in shared memory; it also folds each query's
//               smallest positive and largest bound into two per-query words,
//               and records the smallest bound of every block of 32 leaves.
// k_thresh    -- per query, the FP64 round table r_0, c*r_0, ... (Alg. 7).
// k_round_expand
//             -- one CTA per query: each leaf gets the first round t whose
//               projected threshold (eps*r_t)^2 covers its lower bound, and the
//               leaves of the rounds up to the first one in which some tree
//               alone holds beta*n+k points go to (round, tree) bucket lists;
//               leaf blocks are expanded in the order of their smallest bound's
//               round and only until that round is known.
// k_walk      -- one CTA per query: the buckets in Alg. 7's order. A bucket
//               that cannot bring |S| to beta*n+k is taken whole (order inside
//               it does not change S); the one that can is cut at the first
//               leaf, in (lower bound, leaf number) order, where |S| reaches
//               it, found by weighted radix selects over key-ordered chunks.
//               New points (deduplicated in a bitmap) are appended to the
//               query's candidate list with the round boundaries, and the
//               list's distance work is queued in HBM. The walk needs no
//               distances because it only applies the |S| >= beta*n+k rule and
//               the every-leaf-active rule.
// k_dist      -- the exact FP32 squared distance of every listed candidate: a
//               pure row gather from HBM by persistent warps taking work items
//               from the queue, 8 rows per warp in flight.
// k_finalize  -- one CTA per query. Replays the ">= k candidates within c*r"
//               rule of Alg. 7 after each completed round from the distances
//               and insertion rounds; where it fires first, S is the list's
//               prefix up to that round. Then the k nearest of S by
//               (distance, id) through a pruned top-k buffer.
// The result equals the sequential walk: the rule that needs distances can
// only end the walk at a round boundary, and S at a round boundary is a
// prefix of the list.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <cfloat>

#include "common.cuh"

namespace detlsh {

namespace {

// ------------------------------------------------------------------ lower bounds
constexpr int LB_THREADS = 256;
constexpr int LB_QCH = 128;   // queries per lower-bound CTA (their q' rows staged in shared memory)

// Packed FP32 pair arithmetic (two independent IEEE round-to-nearest
// operations per instruction) and a three-input maximum.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float lo2(unsigned long long v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi2(unsigned long long v) { return __uint_as_float((uint32_t)(v >> 32)); }

// Leaf lower bound: sum over j = 0..K-1, in that order, of
// max(e_lo - x, x - e_hi, 0)^2 in FP32 (no contraction). Dimensions are taken
// in pairs with packed FP32x2 subtractions and products; the sum keeps the
// scalar order. KT > 0: K == KT, known at compile time (an even KT makes every
// tree's q' slice 8-byte aligned and drops the per-dimension tests).
template <int KT>
__global__ void __launch_bounds__(LB_THREADS)
k_leaf_lb(const float* __restrict__ qp, const uint32_t* __restrict__ nqd, int LK, const float* __restrict__ E, int Nr,
          int K, const uint8_t* __restrict__ leaf_lo, const uint8_t* __restrict__ leaf_hi,
          const uint16_t* __restrict__ leaf_tree, int64_t total_leaves, float* __restrict__ lb2,
          uint32_t* __restrict__ minpos, uint32_t* __restrict__ maxlb, uint32_t* __restrict__ blkmin,
          int64_t nblk) {
  // q' rows of the CTA's queries, LKP = L*K rounded up to even, + 2 floats
  // apart (every row starts 8-byte aligned)
  extern __shared__ __align__(16) float s_qrows[];
  const int LKP = (LK + 1) / 2 * 2 + 2;
  __shared__ uint32_t s_min[LB_QCH], s_max[LB_QCH];
  if (KT > 0) K = KT;
  const int64_t leaf = (int64_t)blockIdx.x * LB_THREADS + threadIdx.x;
  const int64_t qb0 = (int64_t)blockIdx.y * LB_QCH;
  const int64_t nqb = *nqd;
  if (qb0 >= nqb) return;
  const int nqc = (int)((nqb - qb0) < LB_QCH ? (nqb - qb0) : LB_QCH);
  for (int i = threadIdx.x; i < nqc * LK; i += LB_THREADS) {
    const int q = i / LK, r = i % LK;
    s_qrows[q * LKP + r] = qp[(qb0 + q) * LK + r];
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
      (void)DL_CHECK(lo <= hi && hi < Nr, 60, leaf);
      if (lo > 0) el[j] = __ldg(E + (int64_t)r * (Nr + 1) + lo);
      if (hi < Nr - 1) eh[j] = __ldg(E + (int64_t)r * (Nr + 1) + hi + 1);
    }
  }
  unsigned long long el2[kMaxK / 2], eh2[kMaxK / 2];
#pragma unroll
  for (int j = 0; j < kMaxK / 2; ++j) {
    el2[j] = pack2(el[2 * j], el[2 * j + 1]);
    eh2[j] = pack2(eh[2 * j], eh[2 * j + 1]);
  }
  const int rbase = tree * K;
  // q' rows at an even base are 8-byte aligned
  const bool paired = (KT > 0 && KT % 2 == 0) || (rbase % 2) == 0;
  float* lbp = lb2 + qb0 * total_leaves + leaf;
  uint32_t* bmp = blkmin + qb0 * nblk + (leaf >> 5);
  for (int q = 0; q < nqc; ++q, lbp += total_leaves, bmp += nblk) {
    float acc = 0.f;
    if (paired) {
      const float* xq = s_qrows + q * LKP + rbase;
#pragma unroll
      for (int j = 0; j < kMaxK; j += 2) {
        if (j + 1 < K) {
          const unsigned long long x2 = *reinterpret_cast<const unsigned long long*>(xq + j);
          const unsigned long long a2 = sub2(el2[j / 2], x2), b2 = sub2(x2, eh2[j / 2]);
          const float d0 = max3f(lo2(a2), lo2(b2), 0.f), d1 = max3f(hi2(a2), hi2(b2), 0.f);
          const unsigned long long dd = mul2(pack2(d0, d1), pack2(d0, d1));
          acc = __fadd_rn(acc, lo2(dd));
          acc = __fadd_rn(acc, hi2(dd));
        } else if (j < K) {
          const float x = xq[j];
          const float dl = max3f(__fsub_rn(el[j], x), __fsub_rn(x, eh[j]), 0.f);
          acc = __fadd_rn(acc, __fmul_rn(dl, dl));
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < kMaxK; ++j) {
        if (j < K) {
          const float x = s_qrows[q * LKP + rbase + j];
          const float dl = max3f(__fsub_rn(el[j], x), __fsub_rn(x, eh[j]), 0.f);
          acc = __fadd_rn(acc, __fmul_rn(dl, dl));
        }
      }
    }
    if (valid) *lbp = acc;
    // non-negative floats order like their bit patterns
    // the smallest bound of the warp's 32 leaves (a lower-bound block)
    const uint32_t mb = __reduce_min_sync(0xffffffffu, valid ? __float_as_uint(acc) : 0x7f800000u);
    if ((threadIdx.x & 31) == 0 && (leaf >> 5) < nblk) *bmp = mb;
    // the smallest positive bound: the block's when that is positive and
    // finite (then every valid bound is positive), else a second reduction
    uint32_t mn = mb;
    if (mb == 0u || mb >= 0x7f800000u)
      mn = __reduce_min_sync(0xffffffffu, (valid && acc > 0.f) ? __float_as_uint(acc) : 0xffffffffu);
    const uint32_t mx = __reduce_max_sync(0xffffffffu, valid ? __float_as_uint(acc) : 0u);
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

// dynamic shared memory of k_leaf_lb for L*K projected dimensions
size_t lb_smem_bytes(int LK) { return sizeof(float) * LB_QCH * (size_t)((LK + 1) / 2 * 2 + 2); }

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

// per-query words of the pipeline (uint32)
enum {
  MQ_RU = 0,      // rounds in the threshold table
  MQ_T_LO,        // T = ceil(beta*n + k), low and high words
  MQ_T_HI,
  MQ_TLAST,       // last round in which some leaf activates
  MQ_TCAP,        // last round the walk can reach
  MQ_NS,          // candidates listed by the walk
  MQ_TEND,        // round in which the walk ended
  MQ_STOP,        // 1: |S| >= T, 3: every leaf active
  MQ_OVERFLOW,    // candidate list overflow (never expected)
  MQ_NREC,        // leaf-run records the walk wrote (coarse distances by leaf)
  MQ_WORDS = 16
};

// ------------------------------------------------------------------ round table
// One thread per query: r_0 = r_min (or sqrt(smallest positive lower bound)/eps),
// r_{t+1} = c * r_t in FP64; (eps*r_t)^2 and (c*r_t)^2 rounded once to FP32; the
// table ends at the first round covering every leaf, or at the round cap with
// infinite thresholds.
__global__ void k_thresh(const uint32_t* __restrict__ minpos, const uint32_t* __restrict__ maxlb,
                         int64_t q0, const uint32_t* __restrict__ nqd, const int32_t* __restrict__ k,
                         const float* __restrict__ c, const float* __restrict__ r_min, double eps,
                         double beta, int64_t n, float* __restrict__ thrP, float* __restrict__ thrC,
                         uint32_t* __restrict__ meta) {
  const int64_t qb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qb >= (int64_t)*nqd) return;
  const int64_t qg = q0 + qb;
  float* tp = thrP + qb * kRoundCap;
  float* tc = thrC + qb * kRoundCap;
  const uint32_t mnb = minpos[qb];
  const float m2 = __uint_as_float(maxlb[qb]);
  double r = (double)r_min[qg];
  if (!(r > 0.0)) r = (mnb != 0xffffffffu) ? sqrt((double)__uint_as_float(mnb)) / eps : 1.0;
  const double cq = (double)c[qg];
  int Ru = kRoundCap;
  for (int t = 0; t < kRoundCap; ++t) {
    if (t == kRoundCap - 1) {
      tp[t] = INFINITY;
      tc[t] = INFINITY;
      break;
    }
    const double er = __dmul_rn(eps, r), cr = __dmul_rn(cq, r);
    tp[t] = __double2float_rn(__dmul_rn(er, er));
    tc[t] = __double2float_rn(__dmul_rn(cr, cr));
    r = __dmul_rn(r, cq);
    if (tp[t] >= m2) {
      Ru = t + 1;
      break;
    }
  }
  const unsigned long long T =
      (unsigned long long)ceil(__dadd_rn(__dmul_rn(beta, (double)n), (double)k[qg]));
  uint32_t* m = meta + qb * MQ_WORDS;
  m[MQ_RU] = (uint32_t)Ru;
  m[MQ_T_LO] = (uint32_t)(T & 0xffffffffull);
  m[MQ_T_HI] = (uint32_t)(T >> 32);
  m[MQ_TLAST] = 0;
}

// ------------------------------------------------------------------ rounds and buckets
// Every leaf joins in the first round t whose projected threshold (eps*r_t)^2
// covers its lower bound; the walk needs, per (round, tree), the leaves and
// points of the rounds up to the first one in which some tree alone holds
// T = beta*n + k points (tcap), and the leaves of those rounds in bucket lists.
// Leaves of later rounds are never needed. k_leaf_lb records the smallest
// lower bound of every block of 32 consecutive leaves; a leaf's round is at
// least its block's, so after the blocks of rounds 0..t have been expanded
// (their leaves' rounds computed exactly) the per-(round, tree) counts of
// rounds 0..t are complete. One CTA per query expands the blocks round by
// round and stops at tcap: only the blocks whose smallest bound is covered by
// the tcap threshold are read leaf by leaf.
constexpr int RX = 512;                 // threads of the per-query round kernel
constexpr int kLbBlock = 32;            // leaves per lower-bound block (one warp of k_leaf_lb)

size_t round_smem_bytes(int L) {
  return sizeof(uint32_t) * (3 * (size_t)kRoundCap + 2 + 4 * (size_t)kRoundCap * L + 1);
}

// warp-aggregated shared-memory adds of (1, w) at key (~0: nothing)
__device__ __forceinline__ void add_key(uint32_t* cnt, uint32_t* wsum, uint32_t key, uint32_t w, int lane) {
  const uint32_t peers = __match_any_sync(0xffffffffu, key);
  const uint32_t sum = __reduce_add_sync(peers, w);
  if (key != 0xffffffffu && (peers & ((1u << lane) - 1u)) == 0) {
    atomicAdd(&cnt[key], (uint32_t)__popc(peers));
    if (wsum) atomicAdd(&wsum[key], sum);
  }
}

__global__ void __launch_bounds__(RX)
k_round_expand(const float* __restrict__ lb2, const uint32_t* __restrict__ blkmin, int64_t TL, int64_t nblk,
               const float* __restrict__ thrP, const uint16_t* __restrict__ leaf_tree,
               const uint32_t* __restrict__ leaf_range, int L, const uint32_t* __restrict__ nqd,
               uint8_t* __restrict__ lround, uint32_t* __restrict__ blist, uint32_t* __restrict__ hpts,
               uint32_t* __restrict__ boff, uint32_t* __restrict__ list, uint32_t* __restrict__ meta) {
  extern __shared__ __align__(16) uint32_t smx[];
  const int RL = kRoundCap * L;
  float* s_thr = reinterpret_cast<float*>(smx);   // [kRoundCap]
  uint32_t* s_bcnt = smx + kRoundCap;             // [kRoundCap] blocks per block round
  uint32_t* s_boffb = s_bcnt + kRoundCap;         // [kRoundCap + 1] their offsets, then cursors
  uint32_t* s_cnt = s_boffb + kRoundCap + 2;      // [RL] leaves per (round, tree)
  uint32_t* s_pts = s_cnt + RL;                   // [RL] points per (round, tree)
  uint32_t* s_off = s_pts + RL;                   // [RL + 1] bucket offsets
  uint32_t* s_cur = s_off + RL + 1;               // [RL] bucket cursors
  __shared__ unsigned long long s_cum[kMaxL];
  __shared__ int s_tcap, s_stop;
  const int64_t qb = blockIdx.x;
  if (qb >= (int64_t)*nqd) return;
  const int tid = threadIdx.x, lane = tid & 31;
  uint32_t* m = meta + qb * MQ_WORDS;
  const int Ru = (int)m[MQ_RU];
  const unsigned long long T = ((unsigned long long)m[MQ_T_HI] << 32) | m[MQ_T_LO];
  for (int i = tid; i < Ru; i += RX) s_thr[i] = thrP[qb * kRoundCap + i];
  for (int i = tid; i < kRoundCap; i += RX) s_bcnt[i] = 0;
  for (int i = tid; i < Ru * L; i += RX) {
    s_cnt[i] = 0;
    s_pts[i] = 0;
    s_cur[i] = 0;
  }
  if (tid < kMaxL) s_cum[tid] = 0;
  if (tid == 0) {
    s_tcap = Ru - 1;   // the last round holds every remaining leaf
    s_stop = 0;
  }
  __syncthreads();
  // blocks by the round of their smallest lower bound
  const uint32_t* bm = blkmin + qb * nblk;
  const int64_t nb_iter = (nblk + RX - 1) / RX * RX;
  for (int64_t bk = tid; bk < nb_iter; bk += RX) {
    const uint32_t rb = bk < nblk ? (uint32_t)lower_bound_f(s_thr, Ru, __uint_as_float(bm[bk])) : 0xffffffffu;
    add_key(s_bcnt, nullptr, rb, 0u, lane);
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t run = 0;
    for (int t = 0; t < Ru; ++t) {
      s_boffb[t] = run;
      run += s_bcnt[t];
    }
    s_boffb[Ru] = run;
  }
  __syncthreads();
  uint32_t* bl = blist + qb * nblk;
  for (int64_t bk = tid; bk < nb_iter; bk += RX) {
    const uint32_t rb = bk < nblk ? (uint32_t)lower_bound_f(s_thr, Ru, __uint_as_float(bm[bk])) : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, rb);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (rb != 0xffffffffu && lane == leader) base = atomicAdd(&s_boffb[rb], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    const uint32_t bp = base + __popc(peers & ((1u << lane) - 1u));
    if (rb != 0xffffffffu && DL_CHECK(bp < nblk, 30, bp)) bl[bp] = (uint32_t)bk;
  }
  __syncthreads();
  // s_boffb[t] now holds the end of round t's blocks; its start is the end of t-1
  const float* lbrow = lb2 + qb * TL;
  uint8_t* lr = lround + qb * TL;
  for (int t = 0; t < Ru; ++t) {
    const uint32_t b0 = t > 0 ? s_boffb[t - 1] : 0u, b1 = s_boffb[t];
    const uint32_t items = (b1 - b0) * kLbBlock;
    const uint32_t it_iter = (items + RX - 1) / RX * RX;
    for (uint32_t it = tid; it < it_iter; it += RX) {
      uint32_t key = 0xffffffffu, pts = 0;
      if (it < items) {
        const int64_t leaf = (int64_t)bl[b0 + it / kLbBlock] * kLbBlock + it % kLbBlock;
        if (leaf < TL) {
          const uint32_t r = (uint32_t)lower_bound_f(s_thr, Ru, lbrow[leaf]);
          lr[leaf] = (uint8_t)r;
          key = r * (uint32_t)L + leaf_tree[leaf];
          pts = leaf_range[2 * leaf + 1];
          if (!DL_CHECK(key < (uint32_t)(Ru * L), 31, key)) key = 0xffffffffu;
        }
      }
      add_key(s_cnt, s_pts, key, pts, lane);
    }
    __syncthreads();
    // rounds 0..t are complete: does some tree alone hold T points?
    if (tid == 0) {
      for (int i = 0; i < L; ++i) {
        s_cum[i] += s_pts[t * L + i];
        if (s_cum[i] >= T) s_stop = 1;
      }
      if (s_stop) s_tcap = t;
    }
    __syncthreads();
    if (s_stop) break;
  }
  const int tcap = s_tcap;
  const int nbk = (tcap + 1) * L;
  if (tid == 0) {
    uint32_t run = 0;
    for (int i = 0; i < nbk; ++i) {
      s_off[i] = run;
      run += s_cnt[i];
    }
    s_off[nbk] = run;
    m[MQ_TCAP] = (uint32_t)tcap;
    m[MQ_TLAST] = (uint32_t)(Ru - 1);
  }
  __syncthreads();
  uint32_t* bo = boff + qb * (kRoundCap * L + 1);
  uint32_t* hp = hpts + qb * kRoundCap * L;
  for (int i = tid; i <= nbk; i += RX) bo[i] = s_off[i];
  for (int i = tid; i < nbk; i += RX) hp[i] = s_pts[i];
  // the leaves of rounds up to tcap into their bucket lists (they lie in the
  // blocks of rounds up to tcap, all expanded)
  uint32_t* ql = list + qb * TL;
  const uint32_t items = s_boffb[tcap] * kLbBlock;
  const uint32_t it_iter = (items + RX - 1) / RX * RX;
  for (uint32_t it = tid; it < it_iter; it += RX) {
    uint32_t key = 0xffffffffu;
    int64_t leaf = 0;
    if (it < items) {
      leaf = (int64_t)bl[it / kLbBlock] * kLbBlock + it % kLbBlock;
      if (leaf < TL) {
        const uint32_t r = lr[leaf];
        if ((int)r <= tcap) key = r * (uint32_t)L + leaf_tree[leaf];
      }
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (key != 0xffffffffu && lane == leader) base = s_off[key] + atomicAdd(&s_cur[key], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    const uint32_t lp = base + __popc(peers & ((1u << lane) - 1u));
    if (key != 0xffffffffu && DL_CHECK(lp < TL, 32, lp)) ql[lp] = (uint32_t)leaf;
  }
}

// ------------------------------------------------------------------ query order
// Locality key of a query: the top bit-planes of its region codes in the first
// projected space (bit 7 of every dimension, then bit 6, ...), 32 bits. Queries
// with equal high bits lie in the same DE-Tree root cells, so they share
// candidates. Positions at or past the batch size get the largest key.
__global__ void k_query_keys(const float* __restrict__ qp, int LK, const uint32_t* __restrict__ nqd,
                             const float* __restrict__ E, int Nr, int K, int64_t B,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  vals[i] = (uint32_t)i;
  if (i >= (int64_t)*nqd) {
    keys[i] = 0xffffffffu;
    return;
  }
  uint32_t code[kMaxK];
  for (int j = 0; j < K; ++j) {
    const float p = qp[i * LK + j];
    const float* e = E + (int64_t)j * (Nr + 1);
    int lo = 1, hi = Nr;   // number of interior edges e[1..Nr-1] that are <= p
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (e[mid] <= p) lo = mid + 1;
      else hi = mid;
    }
    code[j] = (uint32_t)(lo - 1);
  }
  uint32_t key = 0;
  int nb = 0;
  for (int plane = 7; plane >= 0 && nb < 32; --plane)
    for (int j = 0; j < K && nb < 32; ++j, ++nb) key = (key << 1) | ((code[j] >> plane) & 1u);
  keys[i] = key << (32 - nb);
}

// ------------------------------------------------------------------ walk
constexpr int WT = 512;            // threads per walk CTA (two per SM)
constexpr int WNW = WT / 32;
constexpr int WBATCH = 2 * WT;     // leaves examined per batch step (two per thread)
constexpr int WCAP = 8192;         // points examined per batch step
constexpr int WILP = 4;            // points per thread in flight

struct WalkArgs {
  int64_t n;
  int L;
  const uint32_t* leaf_ids;
  const uint32_t* leaf_range;
  const uint16_t* leaf_tree;
  int64_t total_leaves;
  const uint32_t* nqd;        // queries in the batch
  const float* lb2;
  const uint32_t* list;       // [nqb][total_leaves] bucket lists
  const uint32_t* boff;       // [nqb][kRoundCap*L+1]
  const uint32_t* hist_pts;   // [nqb][kRoundCap*L]
  uint32_t* meta;             // [nqb][MQ_WORDS]
  uint32_t* cand;             // [nqb][cap]
  int64_t cap;
  uint32_t* round_end;        // [nqb][kRoundCap] |S| after each round
  uint32_t* ws_newcnt;        // [grid][3][max_bucket] new counts, lower-bound bits, leaf sizes
  int64_t max_bucket;         // most leaves a (round, tree) bucket can hold
  uint32_t* ws_bitmap;        // [grid][bitmap_words] when not in shared memory
  uint32_t* ws_pos;           // [grid][cap] bitmap positions of the query's candidates (global bitmap)
  const uint32_t* leaf_pos;   // [L][n] tree-0 leaf position of each entry's point (the bitmap
                              // index), or null: the point id is the index
  int64_t bitmap_words;
  int smem_bitmap;
  uint32_t* work;             // query counter, zero at launch
  const uint32_t* order;      // [nqb] the batch's queries in locality order
  uint4* items;               // distance work queue: (query, first row, end row) per item
  uint32_t* qtail;            // items queued, zero at launch
  int dist_rows;              // candidate rows per item
  uint4* rec;                 // [nqb][cap] leaf-run records, or null (then items are queued)
  int queue_items;            // 0: the distance work is queued after the walk (by point-id range)
};

struct WalkLayout {
  size_t boff, pts, bpref, bstart, newc, fmap, sel, misc, bitmap, total;
};

__host__ __device__ inline WalkLayout walk_layout(int L, int64_t smem_bitmap_words) {
  WalkLayout o{};
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p += (bytes + 15) & ~size_t(15);
    return at;
  };
  const size_t RL = (size_t)kRoundCap * L;
  o.boff = take(sizeof(uint32_t) * (RL + 1));
  o.pts = take(sizeof(uint32_t) * RL);
  o.bpref = take(sizeof(uint32_t) * (WBATCH + 1));
  o.bstart = take(sizeof(uint32_t) * WBATCH);
  o.newc = take(sizeof(uint32_t) * WBATCH);
  o.fmap = take(sizeof(uint16_t) * WCAP);
  o.sel = take(sizeof(unsigned long long) * 256 + sizeof(uint32_t) * 256);
  o.misc = take(sizeof(unsigned long long) * 32);
  o.bitmap = take(sizeof(uint32_t) * (size_t)smem_bitmap_words);
  o.total = p;
  return o;
}

enum { W_S = 0, W_STOP, W_NEED, W_KSTAR, W_ACC, W_TOTNEW, W_QN, W_LEAFA, W_OFFA, W_OVF, W_ONE, W_NREC, W_LASTEX,
       W_LASTNEW };

// Append the new points of bucket leaves list[0..nl) (only leaves whose select
// key lies in (kmin, kstar] when filtered) to the candidate list, in batches of at most
// WCAP examined points: each point is tested-and-set in the bitmap and, if
// new, written at the list's end.
// With count_only the bitmap is only read: newcnt[j] receives the number of
// points of leaf list[j] not yet in S, lbk[j] its lower-bound bits, and
// misc[W_TOTNEW] their total.
// POS: the bitmap is indexed by a.leaf_pos (tree-0 leaf positions) instead of point ids.
// With a.rec, every run of consecutive points of one leaf within a warp's 32
// lanes that holds new points is also recorded for the leaf-major coarse
// distances: (leaf, offset of the run's first point in the leaf, list
// position of its first new point, mask of its new points).
template <bool POS>
__device__ void walk_add(const WalkArgs& a, const uint32_t* list, uint32_t nl, bool filtered,
                         unsigned long long kstar, const float* lbrow, unsigned char* sm,
                         const WalkLayout& ly, uint32_t* bitmap, uint32_t* cand,
                         bool count_only = false, uint32_t* newcnt = nullptr,
                         uint32_t* lbk = nullptr, bool has_kmin = false, unsigned long long kmin = 0,
                         uint4* rec = nullptr) {
  unsigned long long* misc = reinterpret_cast<unsigned long long*>(sm + ly.misc);
  uint32_t* bpref = reinterpret_cast<uint32_t*>(sm + ly.bpref);
  uint32_t* bstart = reinterpret_cast<uint32_t*>(sm + ly.bstart);
  uint16_t* fmap = reinterpret_cast<uint16_t*>(sm + ly.fmap);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  __shared__ uint32_t s_w[WNW];
  uint32_t& s_nrec = *reinterpret_cast<uint32_t*>(&misc[W_NREC]);   // records of the query so far

  uint32_t* s_newc = reinterpret_cast<uint32_t*>(sm + ly.newc);
  if (threadIdx.x == 0) {
    misc[W_LEAFA] = 0;
    misc[W_OFFA] = 0;
    misc[W_TOTNEW] = 0;
    misc[W_LASTEX] = 0;
    misc[W_LASTNEW] = 0;
  }
  if (count_only)
    for (uint32_t j = threadIdx.x; j < nl; j += WT) newcnt[j] = 0;
  __syncthreads();
  while (true) {
    const uint32_t la = (uint32_t)misc[W_LEAFA];
    const uint32_t offa = (uint32_t)misc[W_OFFA];
    if (la >= nl) break;
    // batch: leaves [la, la+nb) with their (filtered) counts, the first one from
    // offa; thread t owns leaves 2t and 2t+1. bstart holds each leaf's first
    // position in the concatenated per-tree id arrays.
    const uint32_t nb = min((uint32_t)WBATCH, nl - la);
    uint32_t c2[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t j = 2 * threadIdx.x + h;
      if (j < nb && DL_CHECK(list[la + j] < a.total_leaves, 1, list[la + j])) {
        const uint32_t leaf = list[la + j];
        const uint32_t st = a.leaf_range[2 * (int64_t)leaf];
        uint32_t cnt = a.leaf_range[2 * (int64_t)leaf + 1];
        if (filtered) {
          const unsigned long long key =
              ((unsigned long long)__float_as_uint(lbrow[leaf]) << 32) | (unsigned long long)leaf;
          if (key > kstar || (has_kmin && key <= kmin)) cnt = 0;
        }
        if (j == 0) cnt = cnt >= offa ? cnt - offa : 0u;
        c2[h] = cnt;
        if (count_only) {
          s_newc[j] = 0;
          if (offa == 0 || j > 0) lbk[la + j] = __float_as_uint(lbrow[leaf]);
        }
        bstart[j] = (uint32_t)((int64_t)a.leaf_tree[leaf] * a.n) + st + (j == 0 ? offa : 0u);
      }
    }
    const uint32_t cnt = c2[0] + c2[1];
    uint32_t x = cnt;   // inclusive scan over the block of the per-thread pair sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    uint32_t wb = 0;
    for (int qq = 0; qq < w; ++qq) wb += s_w[qq];
    const uint32_t before = wb + x - cnt;
    bpref[2 * threadIdx.x + 1] = before + c2[0];   // bpref[j] = points before leaf j of the batch
    bpref[2 * threadIdx.x + 2] = before + cnt;
    if (threadIdx.x == 0) bpref[0] = 0;
    __syncthreads();
    uint32_t take_leaves, take_pts;
    {
      int lo = 0, hi = (int)nb;   // largest j with bpref[j] <= WCAP
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bpref[mid] <= (uint32_t)WCAP) lo = mid;
        else hi = mid - 1;
      }
      take_leaves = (uint32_t)lo;
      take_pts = bpref[lo];
      if (take_leaves == 0) take_pts = min(bpref[1], (uint32_t)WCAP);
    }
    const uint32_t map_leaves = take_leaves == 0 ? 1u : take_leaves;
    for (uint32_t j = (uint32_t)w; j < map_leaves; j += WNW) {
      const uint32_t e = min(bpref[j + 1], take_pts);
      for (uint32_t f = bpref[j] + lane; f < e; f += 32) fmap[f] = (uint16_t)j;
    }
    if (threadIdx.x == 0) misc[W_QN] = 0;
    __syncthreads();
    const unsigned long long S0 = misc[W_S];
    for (uint32_t f0 = 0; f0 < take_pts; f0 += WT * WILP) {
      // ids[u]: the point (appended to the list); bp[u]: its bit in the bitmap
      uint32_t ids[WILP], bp[WILP];
#pragma unroll
      for (int u = 0; u < WILP; ++u) {
        const uint32_t f = f0 + u * WT + threadIdx.x;
        ids[u] = 0xffffffffu;
        bp[u] = 0xffffffffu;
        if (f < take_pts && DL_CHECK(bstart[fmap[f]] + (f - bpref[fmap[f]]) < (int64_t)a.L * a.n, 2,
                                     bstart[fmap[f]] + (f - bpref[fmap[f]]))) {
          const uint32_t j = fmap[f];
          const int64_t e = bstart[j] + (f - bpref[j]);
          if (POS) {
            bp[u] = __ldg(a.leaf_pos + e);
            if (!count_only) ids[u] = __ldg(a.leaf_ids + e);
          } else {
            ids[u] = __ldg(a.leaf_ids + e);
            bp[u] = ids[u];
          }
        }
      }
      if (count_only) {
        uint32_t word[WILP];
#pragma unroll
        for (int u = 0; u < WILP; ++u)
          word[u] = (bp[u] != 0xffffffffu && DL_CHECK((int64_t)(bp[u] >> 5) < a.bitmap_words, 3, bp[u]))
                        ? bitmap[bp[u] >> 5]
                        : 0xffffffffu;
#pragma unroll
        for (int u = 0; u < WILP; ++u) {
          const uint32_t f = f0 + u * WT + threadIdx.x;
          const uint32_t id = bp[u];
          const bool fresh = id != 0xffffffffu && !((word[u] >> (id & 31)) & 1u);
          const uint32_t key = fresh ? (uint32_t)fmap[f] : 0xffffffffu;
          const uint32_t peers = __match_any_sync(0xffffffffu, key);
          if (fresh && (peers & lt) == 0) atomicAdd(&s_newc[key], (uint32_t)__popc(peers));
          const uint32_t m = __ballot_sync(0xffffffffu, fresh);
          if (lane == 0 && m) atomicAdd(&misc[W_TOTNEW], (unsigned long long)__popc(m));
        }
        continue;
      }
      // all test-and-sets of the step are in flight before any result is used
      uint32_t old[WILP];
#pragma unroll
      for (int u = 0; u < WILP; ++u)
        old[u] = (bp[u] != 0xffffffffu && DL_CHECK((int64_t)(bp[u] >> 5) < a.bitmap_words, 3, bp[u]))
                     ? atomicOr(bitmap + (bp[u] >> 5), 1u << (bp[u] & 31))
                     : 0xffffffffu;
      uint32_t fm[WILP], tot = 0;
#pragma unroll
      for (int u = 0; u < WILP; ++u) {
        const bool fresh = bp[u] != 0xffffffffu && !((old[u] >> (bp[u] & 31)) & 1u);
        fm[u] = __ballot_sync(0xffffffffu, fresh);
        tot += __popc(fm[u]);
      }
      uint32_t base = 0;   // one reservation per warp for the step's new points
      if (lane == 0 && tot) base = (uint32_t)atomicAdd(&misc[W_QN], (unsigned long long)tot);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (rec) {
        // runs of each of the WILP point groups: masks first, then one slot
        // reservation per warp for all of them
        uint32_t rmask[WILP], em[WILP], ntot = 0;
#pragma unroll
        for (int u = 0; u < WILP; ++u) {
          // the valid lanes (f < take_pts) are a prefix of the warp
          const uint32_t f = f0 + u * WT + threadIdx.x;
          const bool valid = f < take_pts;
          const uint32_t j = valid ? (uint32_t)fmap[f] : 0xffffffffu;
          const uint32_t jp = __shfl_up_sync(0xffffffffu, j, 1);
          const uint32_t leaders = __ballot_sync(0xffffffffu, valid && (lane == 0 || jp != j));
          const uint32_t nvalid = __popc(__ballot_sync(0xffffffffu, valid));
          const uint32_t after = leaders & ~((2u << lane) - 1u);   // leaders above this lane
          const uint32_t end = after ? (uint32_t)(__ffs(after) - 1) : nvalid;
          rmask[u] = 0;
          if ((leaders >> lane) & 1u) {
            const uint32_t len = end - lane;
            rmask[u] = (fm[u] >> lane) & (len >= 32 ? 0xffffffffu : ((1u << len) - 1u));
          }
          em[u] = __ballot_sync(0xffffffffu, rmask[u] != 0u);
          ntot += __popc(em[u]);
        }
        uint32_t slot = 0;
        if (lane == 0 && ntot) slot = atomicAdd(&s_nrec, ntot);
        slot = __shfl_sync(0xffffffffu, slot, 0);
#pragma unroll
        for (int u = 0, b2 = 0; u < WILP; b2 += __popc(fm[u]), slot += __popc(em[u]), ++u) {
          const uint32_t rs = slot + __popc(em[u] & lt);
          if (rmask[u] && (int64_t)rs < a.cap) {
            const uint32_t f = f0 + u * WT + threadIdx.x;
            const uint32_t j = fmap[f];
            const uint32_t off = f - bpref[j] + (j == 0 ? offa : 0u);
            const unsigned long long pos = S0 + base + b2 + __popc(fm[u] & lt);
            rec[rs] = make_uint4(list[la + j], off, (uint32_t)pos, rmask[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < WILP; ++u) {
        if ((fm[u] >> lane) & 1u) {
          const unsigned long long pos = S0 + base + __popc(fm[u] & lt);
          if ((int64_t)pos < a.cap) {
            cand[pos] = ids[u];
            if (POS && !a.smem_bitmap) a.ws_pos[(int64_t)blockIdx.x * a.cap + pos] = bp[u];
          } else {
            misc[W_OVF] = 1;
          }
        }
        base += __popc(fm[u]);
      }
    }
    __syncthreads();
    if (count_only) {
      const uint32_t map_leaves2 = take_leaves == 0 ? 1u : take_leaves;
      for (uint32_t j = threadIdx.x; j < map_leaves2; j += WT) newcnt[la + j] += s_newc[j];
    }
    if (threadIdx.x == 0) {
      if (!count_only) misc[W_S] += misc[W_QN];
      // points this call examined and found new (the walk's estimate of the
      // new share of the next points it will examine)
      misc[W_LASTEX] += take_pts;
      misc[W_LASTNEW] = count_only ? misc[W_TOTNEW] : misc[W_LASTNEW] + misc[W_QN];
      if (take_leaves == 0) {
        const uint32_t first_total = bpref[1] + offa;  // points of leaf la (after filter)
        const uint32_t newoff = offa + take_pts;
        if (newoff >= first_total) {
          misc[W_LEAFA] = la + 1;
          misc[W_OFFA] = 0;
        } else {
          misc[W_OFFA] = newoff;
        }
      } else {
        misc[W_LEAFA] = la + take_leaves;
        misc[W_OFFA] = 0;
      }
    }
    __syncthreads();
  }
  // every thread has read the exhausted cursor before the next call resets it
  __syncthreads();
}

// Weighted radix select over the leaves j < nl of a bucket with key(j) =
// (lower-bound bits << 32 | leaf) above kmin (when has_kmin): the smallest key
// K such that the weights wt[j] of the keys in (kmin, K] add up to `need`, or
// ~0 when all of them add up to less. Block-wide; ends with a barrier.
__device__ unsigned long long select_key(const uint32_t* bl, const uint32_t* lbk, const uint32_t* wt, uint32_t nl,
                                         bool has_kmin, unsigned long long kmin, unsigned long long need,
                                         unsigned long long* sel, unsigned long long* misc) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t iters_j = (nl + WT - 1) / WT * WT;
  // total weight above kmin
  if (threadIdx.x == 0) misc[W_ACC] = 0;
  __syncthreads();
  {
    unsigned long long part = 0;
    for (uint32_t j = threadIdx.x; j < nl; j += WT) {
      const unsigned long long key = ((unsigned long long)lbk[j] << 32) | (unsigned long long)bl[j];
      if (!has_kmin || key > kmin) part += wt[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0 && part) atomicAdd(&misc[W_ACC], part);
  }
  __syncthreads();
  const bool enough = misc[W_ACC] >= need;
  __syncthreads();
  if (!enough) return ~0ull;
  if (threadIdx.x == 0) {
    misc[W_NEED] = need;
    misc[W_KSTAR] = 0;
    misc[W_ACC] = 0;
  }
  __syncthreads();
  // sel[0..256): weight per digit; the second half counts the leaves of
  // positive weight per digit, so that a digit holding a single such leaf
  // ends the select early (that leaf's key is the answer)
  uint32_t* selc = reinterpret_cast<uint32_t*>(sel + 256);
  unsigned long long prefix = 0, pmask = 0;
  for (int p = 7; p >= 0; --p) {
    for (int i2 = threadIdx.x; i2 < 256; i2 += WT) {
      sel[i2] = 0;
      selc[i2] = 0;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < iters_j; j += WT) {
      uint32_t dg = 0xffffffffu, wgt = 0;
      if (j < nl) {
        const uint32_t c = wt[j];
        const unsigned long long key = ((unsigned long long)lbk[j] << 32) | (unsigned long long)bl[j];
        if (c && (key & pmask) == prefix && (!has_kmin || key > kmin)) {
          dg = (uint32_t)((key >> (8 * p)) & 255ull);
          wgt = c;
        }
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, dg);
      const uint32_t sum = __reduce_add_sync(peers, wgt);
      if (dg != 0xffffffffu && (peers & lt) == 0) {
        atomicAdd(&sel[dg], (unsigned long long)sum);
        atomicAdd(&selc[dg], (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // the first digit whose cumulative weight reaches the need (a warp scan)
      const unsigned long long nd = misc[W_NEED];
      unsigned long long acc0 = misc[W_ACC];
      unsigned long long v[8], run = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        v[e] = sel[lane * 8 + e];
        run += v[e];
      }
      unsigned long long incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned long long before = incl - run;
      const bool reaches = acc0 + incl >= nd;
      const uint32_t bal = __ballot_sync(0xffffffffu, reaches);
      // a lane always reaches: the selected bin's weight covers the need
      const int first = bal ? __ffs(bal) - 1 : 31;
      if (lane == first) {
        unsigned long long acc = acc0 + before;
        int dg = lane * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          if (acc + v[e] >= nd) break;
          acc += v[e];
          ++dg;
        }
        misc[W_ACC] = acc;
        misc[W_KSTAR] = prefix | ((unsigned long long)min(dg, 255) << (8 * p));
        misc[W_ONE] = (selc[min(dg, 255)] == 1u) ? 1ull : 0ull;
      }
    }
    __syncthreads();
    prefix = misc[W_KSTAR];
    pmask |= 255ull << (8 * p);
    if (p > 0 && misc[W_ONE]) {
      // one leaf of positive weight carries this prefix: its key is the answer
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < nl; j += WT) {
        const unsigned long long key = ((unsigned long long)lbk[j] << 32) | (unsigned long long)bl[j];
        if (wt[j] && (key & pmask) == prefix && (!has_kmin || key > kmin)) misc[W_KSTAR] = key;
      }
      __syncthreads();
      prefix = misc[W_KSTAR];
      __syncthreads();
      return prefix;
    }
  }
  return prefix;
}

// One CTA per query (persistent over the batch): the buckets in Alg. 7 order.
template <bool POS>
__global__ void __launch_bounds__(WT, 3) k_walk(WalkArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const WalkLayout ly = walk_layout(a.L, a.smem_bitmap ? a.bitmap_words : 0);
  uint32_t* s_boff = reinterpret_cast<uint32_t*>(sm + ly.boff);
  uint32_t* s_pts = reinterpret_cast<uint32_t*>(sm + ly.pts);
  unsigned long long* sel = reinterpret_cast<unsigned long long*>(sm + ly.sel);
  unsigned long long* misc = reinterpret_cast<unsigned long long*>(sm + ly.misc);
  uint32_t* bitmap = a.smem_bitmap ? reinterpret_cast<uint32_t*>(sm + ly.bitmap)
                                   : a.ws_bitmap + (int64_t)blockIdx.x * a.bitmap_words;
  uint32_t* newcnt = a.ws_newcnt + (int64_t)blockIdx.x * 3 * a.max_bucket;
  uint32_t* lbk = newcnt + a.max_bucket;
  uint32_t* tcnt = lbk + a.max_bucket;
  const int L = a.L;

  __shared__ long long s_qb;
  const int64_t nqb = *a.nqd;
  while (true) {
    // queries are taken from a counter in global memory, so a CTA that drew
    // short queries takes more of them
    // ... in locality order (queries with similar codes in turn, so that
    // their distance work, queued in this order, shares rows in L2)
    if (threadIdx.x == 0) {
      const uint32_t i = atomicAdd(a.work, 1u);
      s_qb = (int64_t)i < nqb ? (long long)a.order[i] : (long long)nqb;
    }
    __syncthreads();
    const int64_t qb = s_qb;
    if (qb >= nqb) break;
    const float* lbrow = a.lb2 + qb * a.total_leaves;
    const uint32_t* list = a.list + qb * a.total_leaves;
    uint32_t* cand = a.cand + qb * a.cap;
    uint4* rec = a.rec ? a.rec + qb * a.cap : nullptr;
    uint32_t* rend = a.round_end + qb * kRoundCap;
    uint32_t* m = a.meta + qb * MQ_WORDS;
    const unsigned long long T = ((unsigned long long)m[MQ_T_HI] << 32) | m[MQ_T_LO];
    const int tcap = (int)m[MQ_TCAP];
    const int tlast = (int)m[MQ_TLAST];
    const int nbk = (tcap + 1) * L;
    if (a.smem_bitmap)
      for (int64_t i = threadIdx.x; i < a.bitmap_words; i += WT) bitmap[i] = 0u;
    for (int i = threadIdx.x; i <= nbk; i += WT) s_boff[i] = a.boff[qb * (kRoundCap * L + 1) + i];
    for (int i = threadIdx.x; i < nbk; i += WT) s_pts[i] = a.hist_pts[qb * kRoundCap * L + i];
    if (threadIdx.x == 0) {
      misc[W_S] = 0;
      misc[W_STOP] = 0;
      misc[W_OVF] = 0;
      misc[W_NREC] = 0;
    }
    __syncthreads();
    int t_end = tcap;
    for (int t = 0; t <= tcap; ++t) {
      // a round whose points cannot bring |S| to T is taken in one step: the
      // order of its trees does not change S
      unsigned long long rpts = 0;
      for (int i = 0; i < L; ++i) rpts += s_pts[t * L + i];
      const bool whole_round = misc[W_S] + rpts < T;
      if (whole_round) {
        const uint32_t nl = s_boff[(t + 1) * L] - s_boff[t * L];
        if (nl) walk_add<POS>(a, list + s_boff[t * L], nl, false, ~0ull, lbrow, sm, ly, bitmap, cand, false, nullptr,
                              nullptr, false, 0, rec);
      }
      for (int i = 0; i < L && !whole_round; ++i) {
        const int b = t * L + i;
        const uint32_t nl = s_boff[b + 1] - s_boff[b];
        if (nl == 0) continue;
        const uint32_t* bl = list + s_boff[b];
        const unsigned long long bpts = s_pts[b];   // all of the bucket's points
        bool cut = false;
        if (misc[W_S] + bpts < T) {
          walk_add<POS>(a, bl, nl, false, ~0ull, lbrow, sm, ly, bitmap, cand, false, nullptr, nullptr, false, 0, rec);
        } else {
          // the bucket may hold the cut: its leaves in key order (lower bound,
          // leaf) are taken in chunks (a select on the leaves' sizes) of the
          // points still needed over the new share of the points examined last
          // (the previous bucket, or the previous chunk), with a quarter more —
          // twice the need when there is no such share; the new points of a
          // chunk are counted (bitmap read only) and the chunk is added whole,
          // or, if it holds the cut, up to the leaf where |S| reaches T (a
          // select on the new counts). Only the chunks up to the cut are
          // examined. A leaf's new count does not depend on the other leaves
          // of its bucket (one tree holds a point once), so the cut leaf and S
          // do not depend on the chunk sizes.
          for (uint32_t j = threadIdx.x; j < nl; j += WT) {
            const uint32_t leaf = bl[j];
            lbk[j] = __float_as_uint(lbrow[leaf]);
            tcnt[j] = a.leaf_range[2 * (int64_t)leaf + 1];
          }
          __syncthreads();
          bool has_kmin = false;
          unsigned long long kmin = 0;
          while (true) {
            const unsigned long long S0 = misc[W_S];
            const unsigned long long need = T - S0;
            const unsigned long long ex = misc[W_LASTEX], nw = misc[W_LASTNEW];
            unsigned long long target = 2 * need;
            if (ex > 0 && nw > 0)
              target = (unsigned long long)((double)need * fmin(8.0, fmax(1.0, 1.25 * (double)ex / (double)nw)));
            __syncthreads();   // every thread has read the last call's counts
            const unsigned long long kc = select_key(bl, lbk, tcnt, nl, has_kmin, kmin, target, sel, misc);
            walk_add<POS>(a, bl, nl, true, kc, lbrow, sm, ly, bitmap, cand, true, newcnt, lbk, has_kmin, kmin);
            if (S0 + misc[W_TOTNEW] >= T) {
              const unsigned long long kstar = select_key(bl, lbk, newcnt, nl, has_kmin, kmin, need, sel, misc);
              walk_add<POS>(a, bl, nl, true, kstar, lbrow, sm, ly, bitmap, cand, false, nullptr, nullptr, has_kmin, kmin,
                            rec);
              cut = true;
              break;
            }
            walk_add<POS>(a, bl, nl, true, kc, lbrow, sm, ly, bitmap, cand, false, nullptr, nullptr, has_kmin, kmin,
                          rec);
            if (kc == ~0ull) break;   // the bucket is exhausted without a cut
            has_kmin = true;
            kmin = kc;
          }
        }
        if (cut) {
          if (threadIdx.x == 0) misc[W_STOP] = 1;
          break;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        rend[t] = (uint32_t)misc[W_S];
        if (!misc[W_STOP] && t == tlast) misc[W_STOP] = 3;
      }
      __syncthreads();
      if (misc[W_STOP]) {
        t_end = t;
        break;
      }
    }
    if (threadIdx.x == 0) {
      m[MQ_NS] = (uint32_t)misc[W_S];
      m[MQ_TEND] = (uint32_t)t_end;
      m[MQ_STOP] = misc[W_STOP] ? (uint32_t)misc[W_STOP] : 3u;
      m[MQ_OVERFLOW] = (uint32_t)misc[W_OVF];
      m[MQ_NREC] = (uint32_t)misc[W_NREC];
    }
    // queue the distance work of the listed candidates (unless the leaf-run
    // records serve the distances)
    if (!a.rec && a.queue_items) {
      __shared__ uint32_t s_ib, s_ni;
      if (threadIdx.x == 0) {
        const int64_t ns = min((int64_t)misc[W_S], a.cap);
        s_ni = (uint32_t)((ns + a.dist_rows - 1) / a.dist_rows);
        s_ib = s_ni ? atomicAdd(a.qtail, s_ni) : 0u;
      }
      __syncthreads();
      const uint32_t ns = (uint32_t)min((int64_t)misc[W_S], a.cap);
      for (uint32_t i = threadIdx.x; i < s_ni; i += WT) {
        const uint32_t r0 = i * (uint32_t)a.dist_rows;
        a.items[s_ib + i] = make_uint4((uint32_t)qb, r0, min(r0 + (uint32_t)a.dist_rows, ns), 0u);
      }
    }
    __syncthreads();
    if (!a.smem_bitmap) {
      // leave the global bitmap zeroed: through the candidate list when it
      // holds every set bit and is much shorter than the bitmap
      const unsigned long long S = misc[W_S];
      if (!misc[W_OVF] && (int64_t)S * 8 < a.bitmap_words) {
        const uint32_t* bpl = POS ? a.ws_pos + (int64_t)blockIdx.x * a.cap : cand;
        for (unsigned long long p = threadIdx.x; p < S; p += WT) bitmap[bpl[p] >> 5] = 0u;
      } else {
        for (int64_t i = threadIdx.x; i < a.bitmap_words; i += WT) bitmap[i] = 0u;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ distances
constexpr int DT = 256;            // threads per distance CTA
constexpr int DNW = DT / 32;
constexpr int ILP = 8;             // rows per warp in flight (the transposed reduction assumes 8)
constexpr int DROWS = DNW * ILP * 4;  // rows per CTA

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
// TWO_SLICES: the distance kernels' path for d <= 256 (at most two slices per
// lane, addresses formed once per row); the top-k's shortlist re-rank keeps
// the plain loop, which needs fewer registers. Both give the same sums.
template <typename TX, bool TWO_SLICES = true>
__device__ __forceinline__ void rows_dist2(const TX* __restrict__ X, int d,
                                           const uint32_t* ids, const TX* __restrict__ q,
                                           bool vec4, int lane, float* acc) {
  using V = Vec4Of<TX>;
  if (TWO_SLICES && vec4 && d <= 256) {
    // at most two 4-coordinate slices per lane (lane and lane + 32): the
    // lane's offset is folded into each row's address once and the second
    // slice is a constant offset from it. A missing row (id ~0) reads row 0
    // and its sum is not used, so the loads need no branch
    const int d4 = d >> 2;
    const TX* xr[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) xr[u] = X + 4 * lane + (int64_t)(ids[u] != 0xffffffffu ? ids[u] : 0u) * d;
    const TX* ql = q + 4 * lane;
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      if (lane + 32 * sl >= d4) break;
      const typename V::T qv = V::ld(ql, 32 * sl);
      typename V::T xv[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u) xv[u] = V::ld(xr[u], 32 * sl);
      const float4 qf = V::f(qv);
      const unsigned long long qxy = pack2(qf.x, qf.y), qzw = pack2(qf.z, qf.w);
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        const float4 xf = V::f(xv[u]);
        const unsigned long long dxy = sub2(pack2(xf.x, xf.y), qxy), dzw = sub2(pack2(xf.z, xf.w), qzw);
        acc[u] = fmaf(lo2(dxy), lo2(dxy), acc[u]);
        acc[u] = fmaf(hi2(dxy), hi2(dxy), acc[u]);
        acc[u] = fmaf(lo2(dzw), lo2(dzw), acc[u]);
        acc[u] = fmaf(hi2(dzw), hi2(dzw), acc[u]);
      }
    }
  } else if (vec4) {
    const int d4 = d >> 2;
    // a missing row (id ~0) reads row 0 and its sum is not used: the loads
    // need no branch
    const TX* xr[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) xr[u] = X + (int64_t)(ids[u] != 0xffffffffu ? ids[u] : 0u) * d;
    for (int i = lane; i < d4; i += 32) {
      const typename V::T qv = V::ld(q, i);
      typename V::T xv[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u) xv[u] = V::ld(xr[u], i);
      const float4 qf = V::f(qv);
      // (x - q) of two coordinates per packed FP32 subtraction (each rounded
      // as a scalar one), then the squares added in coordinate order by fused
      // multiply-adds
      const unsigned long long qxy = pack2(qf.x, qf.y), qzw = pack2(qf.z, qf.w);
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        const float4 xf = V::f(xv[u]);
        const unsigned long long dxy = sub2(pack2(xf.x, xf.y), qxy), dzw = sub2(pack2(xf.z, xf.w), qzw);
        acc[u] = fmaf(lo2(dxy), lo2(dxy), acc[u]);
        acc[u] = fmaf(hi2(dxy), hi2(dxy), acc[u]);
        acc[u] = fmaf(lo2(dzw), lo2(dzw), acc[u]);
        acc[u] = fmaf(hi2(dzw), hi2(dzw), acc[u]);
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

// Persistent over the work queue the walk filled: item (query, r0, r1)
// covers rows [r0, r1) of that query's candidate list. Each warp takes items
// from a counter in global memory (so the warps finish together), asking for
// its next item as soon as it starts one.
__device__ __forceinline__ uint32_t next_item(uint32_t* head, int lane) {
  uint32_t it = 0;
  if (lane == 0) it = atomicAdd(head, 1u);
  return __shfl_sync(0xffffffffu, it, 0);
}

// BK: the items address the query's candidates grouped by point-id range,
// (point id, list position) pairs; the distance goes to the list position.
template <typename TX, bool BK>
__global__ void __launch_bounds__(DT, 4)
k_dist(const TX* __restrict__ X, int d, int64_t n, const TX* __restrict__ Q, int64_t q0,
       const uint32_t* __restrict__ cand, const uint2* __restrict__ pairs, int64_t cap,
       const uint4* __restrict__ items, const uint32_t* __restrict__ qtail, uint32_t* __restrict__ head,
       float* __restrict__ d2out, bool vec4) {
  const uint32_t nit = *qtail;
  const int lane = threadIdx.x & 31;
  uint32_t it = next_item(head, lane);
  while (it < nit) {
    const uint4 item = items[it];
    const uint32_t nx = next_item(head, lane);
    const int64_t qb = item.x;
    const int64_t r0 = item.y, r1 = item.z;
    const TX* q = Q + (q0 + qb) * (int64_t)d;
    const uint32_t* cl = cand + qb * cap;
    const uint2* pl = BK ? pairs + qb * cap : nullptr;
    float* out = d2out + qb * cap;
    if (BK) {
      // lanes 0..7 load the step's eight (point id, list position) pairs and
      // the warp shares them by shuffles
      for (uint32_t e0 = (uint32_t)r0; e0 < (uint32_t)r1; e0 += ILP) {
        const uint32_t e = e0 + (uint32_t)(lane & 7);
        const uint2 P = (lane < 8 && e < (uint32_t)r1) ? __ldg(pl + e) : make_uint2(0xffffffffu, 0xffffffffu);
        uint32_t ids[ILP];
        float acc[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
          ids[u] = __shfl_sync(0xffffffffu, P.x, u);
          if (ids[u] != 0xffffffffu && !DL_CHECK(ids[u] < n, 10, ids[u])) ids[u] = 0xffffffffu;
          acc[u] = 0.f;
        }
        rows_dist2<TX>(X, d, ids, q, vec4, lane, acc);
        const float v = transpose_reduce8(acc, lane);
        const uint32_t pos = __shfl_sync(0xffffffffu, P.y, (lane >> 2) & 7);
        if ((lane & 3) == 0 && pos != 0xffffffffu && DL_CHECK(pos < cap, 11, pos)) out[pos] = v;
      }
    } else {
      for (int64_t e0 = r0; e0 < r1; e0 += ILP) {
        uint32_t ids[ILP];
        float acc[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
          ids[u] = (e0 + u < r1) ? __ldg(cl + e0 + u) : 0xffffffffu;
          if (ids[u] != 0xffffffffu && !DL_CHECK(ids[u] < n, 10, ids[u])) ids[u] = 0xffffffffu;
          acc[u] = 0.f;
        }
        rows_dist2<TX>(X, d, ids, q, vec4, lane, acc);
        const float v = transpose_reduce8(acc, lane);
        const int r = (lane >> 2) & 7;
        if ((lane & 3) == 0 && e0 + r < r1) out[e0 + r] = v;
      }
    }
    it = nx;
  }
}

// FP32 rows with d <= 128, d a multiple of 4 and 16-byte aligned rows: eight
// lanes per row, lane s of a group holding the 4-coordinate slices s, s + 8,
// s + 16, s + 24 (S of them) of the row and, in registers for the whole item,
// of q. A warp step takes eight rows, two per 8-lane group; every lane loads
// its own rows' ids (eight lanes share an address), so the only shuffles left
// are the three of the 8-lane reduction — with 32 lanes per row the id
// broadcasts and the 32-lane reduction took more L1 data-pipe cycles than the
// row loads' own wavefronts. Per lane and row the squares of even and odd
// coordinates are accumulated by packed FP32 fused multiply-adds in
// coordinate order, added, and the eight lanes' partials summed by a
// butterfly (xor 4, 2, 1): the same order for every row, so a row's distance
// does not depend on where in a step or which item it is taken.
struct G8Lane {
  int sub, g;
  bool hi;
};

// the lane's slices of q as packed pairs (zeros past d)
template <int S>
__device__ __forceinline__ void g8_load_q(const float* q, const bool* has, const G8Lane& gl,
                                          unsigned long long (&qv)[S][2]) {
  const float4* ql = reinterpret_cast<const float4*>(q) + gl.sub;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const float4 f = has[s] ? __ldg(ql + 8 * s) : make_float4(0.f, 0.f, 0.f, 0.f);
    qv[s][0] = pack2(f.x, f.y);
    qv[s][1] = pack2(f.z, f.w);
  }
}

// the distances of one query's candidates [r0, r1): list entries cl[e] (BK:
// pairs pl[e] = (point id, list position)), each written to out[position]
template <int S, bool BK>
__device__ __forceinline__ void g8_rows(const float* __restrict__ X, int d, int64_t n,
                                        const uint32_t* __restrict__ cl, const uint2* __restrict__ pl,
                                        uint32_t r0, uint32_t r1, int64_t cap, const bool* has, const G8Lane& gl,
                                        const unsigned long long (&qv)[S][2], float* __restrict__ out) {
  for (uint32_t e0 = r0; e0 < r1; e0 += 8) {
    uint32_t id[2], pos[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t e = e0 + 2 * gl.g + u;
      id[u] = 0xffffffffu;
      pos[u] = 0xffffffffu;
      if (e < r1) {
        if (BK) {
          const uint2 P = __ldg(pl + e);
          id[u] = P.x;
          pos[u] = P.y;
        } else {
          id[u] = __ldg(cl + e);
          pos[u] = e;
        }
      }
      if (id[u] != 0xffffffffu && !DL_CHECK(id[u] < n, 10, id[u])) id[u] = 0xffffffffu;
    }
    // a missing row (id ~0) reads row 0 and its sum is not stored
    const float4* xr[2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
      xr[u] = reinterpret_cast<const float4*>(X + (int64_t)(id[u] != 0xffffffffu ? id[u] : 0u) * d) + gl.sub;
    float4 xv[2][S];
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int u = 0; u < 2; ++u) xv[u][s] = has[s] ? __ldg(xr[u] + 8 * s) : make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      unsigned long long a2 = 0ull;   // (even, odd) coordinate sums, both +0
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const unsigned long long dxy = sub2(pack2(xv[u][s].x, xv[u][s].y), qv[s][0]);
        const unsigned long long dzw = sub2(pack2(xv[u][s].z, xv[u][s].w), qv[s][1]);
        a2 = fma2(dxy, dxy, a2);
        a2 = fma2(dzw, dzw, a2);
      }
      acc[u] = lo2(a2) + hi2(a2);
    }
    // 8-lane butterfly: after the xor-4 exchange a lane keeps row `hi`
    float v = (gl.hi ? acc[1] : acc[0]) + __shfl_xor_sync(0xffffffffu, gl.hi ? acc[0] : acc[1], 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    const uint32_t p = gl.hi ? pos[1] : pos[0];
    if ((gl.sub & 3) == 0 && p != 0xffffffffu && DL_CHECK(p < cap, 11, p)) out[p] = v;
  }
}

// persistent over the work queue, as k_dist
template <int S, bool BK>
__global__ void __launch_bounds__(DT, 4)
k_dist_g8(const float* __restrict__ X, int d, int64_t n, const float* __restrict__ Q, int64_t q0,
          const uint32_t* __restrict__ cand, const uint2* __restrict__ pairs, int64_t cap,
          const uint4* __restrict__ items, const uint32_t* __restrict__ qtail, uint32_t* __restrict__ head,
          float* __restrict__ d2out) {
  const uint32_t nit = *qtail;
  const int lane = threadIdx.x & 31;
  const G8Lane gl{lane & 7, lane >> 3, (lane & 4) != 0};
  bool has[S];
#pragma unroll
  for (int s = 0; s < S; ++s) has[s] = 8 * s + gl.sub < (d >> 2);
  uint32_t it = next_item(head, lane);
  while (it < nit) {
    const uint4 item = items[it];
    const uint32_t nx = next_item(head, lane);
    const int64_t qb = item.x;
    unsigned long long qv[S][2];
    g8_load_q<S>(Q + (q0 + qb) * (int64_t)d, has, gl, qv);
    g8_rows<S, BK>(X, d, n, cand + qb * cap, BK ? pairs + qb * cap : nullptr, item.y, item.z, cap, has, gl, qv,
                   d2out + qb * cap);
    it = nx;
  }
}

// uint8 rows, d a power of two from 16 to 512: d/16 lanes per row, 16 bytes a
// lane, so one load instruction covers 32/(d/16) rows and a warp keeps eight
// of them (32 rows at d = 128) in flight. The squared distance is
// sum x^2 - 2 sum x q + sum q^2 in 32-bit integers (dp4a), exact whatever the
// order of the sums (at most 512 * 255^2 < 2^31), converted to FP32 once.
template <bool BK>
__global__ void __launch_bounds__(DT, 4)
k_dist_u8(const uint8_t* __restrict__ X, int d, int64_t n, const uint8_t* __restrict__ Q, int64_t q0,
          const uint32_t* __restrict__ cand, const uint2* __restrict__ pairs, int64_t cap,
          const uint4* __restrict__ items, const uint32_t* __restrict__ qtail, uint32_t* __restrict__ head,
          float* __restrict__ d2out) {
  const uint32_t nit = *qtail;
  const int lane = threadIdx.x & 31;
  const int gs = d >> 4;       // lanes per row
  const int rpl = 32 / gs;     // rows per load instruction
  const int sub = lane & (gs - 1), grp = lane / gs;
  uint32_t it = next_item(head, lane);
  while (it < nit) {
    const uint4 item = items[it];
    const uint32_t nx = next_item(head, lane);
    const int64_t qb = item.x;
    const int64_t r0 = item.y, r1 = item.z;
    const uint4 qv = __ldg(reinterpret_cast<const uint4*>(Q + (q0 + qb) * (int64_t)d) + sub);
    int qsq = (int)(__dp4a(qv.x, qv.x, 0u) + __dp4a(qv.y, qv.y, 0u) + __dp4a(qv.z, qv.z, 0u) +
                    __dp4a(qv.w, qv.w, 0u));
    for (int off = gs >> 1; off > 0; off >>= 1) qsq += __shfl_xor_sync(0xffffffffu, qsq, off);
    const uint32_t* cl = cand + qb * cap;
    const uint2* pl = BK ? pairs + qb * cap : nullptr;
    float* out = d2out + qb * cap;
    for (int64_t e0 = r0; e0 < r1; e0 += 8 * rpl) {
      uint32_t ids[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t e = e0 + u * rpl + grp;
        ids[u] = e < r1 ? (BK ? __ldg(&pl[e].x) : __ldg(cl + e)) : 0xffffffffu;
        if (ids[u] != 0xffffffffu && !DL_CHECK(ids[u] < n, 12, ids[u])) ids[u] = 0xffffffffu;
      }
      uint4 xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        xv[u] = ids[u] != 0xffffffffu ? __ldg(reinterpret_cast<const uint4*>(X + (int64_t)ids[u] * d) + sub)
                                      : make_uint4(0u, 0u, 0u, 0u);
      int part[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t xx = __dp4a(xv[u].x, xv[u].x, __dp4a(xv[u].y, xv[u].y,
                                   __dp4a(xv[u].z, xv[u].z, __dp4a(xv[u].w, xv[u].w, 0u))));
        const uint32_t xq = __dp4a(xv[u].x, qv.x, __dp4a(xv[u].y, qv.y,
                                   __dp4a(xv[u].z, qv.z, __dp4a(xv[u].w, qv.w, 0u))));
        part[u] = (int)xx - 2 * (int)xq;
      }
      for (int off = gs >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int u = 0; u < 8; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], off);
      }
      if (sub == 0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t e = e0 + u * rpl + grp;
          if (e < r1) out[BK ? (int64_t)__ldg(&pl[e].y) : e] = (float)(part[u] + qsq);
        }
      }
    }
    it = nx;
  }
}

// ------------------------------------------------------------------ gather by point-id range
// The candidates of a batch grouped by point-id range before the gather: a
// point is a candidate of many queries of a batch (about beta of them), so
// when every query's candidates in ids [0, R) are taken first, then those in
// [R, 2R), ..., the rows read at the same time lie in R rows of X, which stay
// in L2 while all queries read them. The distances are the same; each goes
// to its list position.
constexpr int BKT = 256;   // threads of the per-query grouping kernel
constexpr int kMaxIdBuckets = 1024;

// One CTA per query: its candidates' counts per id range (range-major counts
// bcnt[b][qb] and in-query offsets boffq[qb][b]), then the (point id, list
// position) pairs of each range at its offset. Queries at or past the batch
// size count nothing.
__global__ void __launch_bounds__(BKT)
k_cand_buckets(const uint32_t* __restrict__ cand, int64_t cap, const uint32_t* __restrict__ meta,
               const uint32_t* __restrict__ nqd, int bshift, int nbk, int64_t nqg, uint2* __restrict__ pairs,
               uint32_t* __restrict__ bcnt, uint32_t* __restrict__ boffq) {
  __shared__ uint32_t s_cnt[kMaxIdBuckets], s_off[kMaxIdBuckets];
  __shared__ uint32_t s_w[BKT / 32];
  const int64_t qb = blockIdx.x;
  const bool active = qb < (int64_t)*nqd;
  const int64_t ns = active ? min((int64_t)meta[qb * MQ_WORDS + MQ_NS], cap) : 0;
  for (int b = threadIdx.x; b < nbk; b += BKT) s_cnt[b] = 0;
  __syncthreads();
  const uint32_t* cl = cand + qb * cap;
  for (int64_t i = threadIdx.x; i < ns; i += BKT) {
    const uint32_t bk = __ldg(cl + i) >> bshift;
    if (DL_CHECK(bk < (uint32_t)nbk, 20, bk)) atomicAdd(&s_cnt[bk], 1u);
  }
  __syncthreads();
  // exclusive scan of the counts: each thread a contiguous run of ranges
  const int per = (nbk + BKT - 1) / BKT;
  const int b0 = threadIdx.x * per;
  uint32_t run = 0;
  for (int b = b0; b < min(nbk, b0 + per); ++b) run += s_cnt[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  uint32_t before = x - run;
  for (int i = 0; i < w; ++i) before += s_w[i];
  for (int b = b0; b < min(nbk, b0 + per); ++b) {
    s_off[b] = before;
    boffq[qb * nbk + b] = before;
    bcnt[(int64_t)b * nqg + qb] = s_cnt[b];
    before += s_cnt[b];
  }
  __syncthreads();
  uint2* pl = pairs + qb * cap;
  for (int64_t i = threadIdx.x; i < ns; i += BKT) {
    const uint32_t id = __ldg(cl + i);
    if (!DL_CHECK((id >> bshift) < (uint32_t)nbk, 20, id)) continue;
    const uint32_t p = atomicAdd(&s_off[id >> bshift], 1u);
    if (DL_CHECK(p < cap, 21, p)) pl[p] = make_uint2(id, (uint32_t)i);
  }
}

// distance work items per (range, query) cell
__global__ void k_cell_items(const uint32_t* __restrict__ bcnt, int64_t cells, int rows, uint32_t* __restrict__ icnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cells) icnt[c] = (bcnt[c] + rows - 1) / rows;
}

// the items of each cell at its place in range-major order
__global__ void k_cell_fill(const uint32_t* __restrict__ bcnt, const uint32_t* __restrict__ ioff,
                            const uint32_t* __restrict__ boffq, int nbk, int64_t nqg, int rows,
                            uint4* __restrict__ items) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (int64_t)nbk * nqg) return;
  const int64_t b = c / nqg, qb = c - b * nqg;
  const uint32_t cnt = bcnt[c], r0 = boffq[qb * nbk + b];
  for (uint32_t t = 0; t * (uint32_t)rows < cnt; ++t)
    items[ioff[c] + t] = make_uint4((uint32_t)qb, r0 + t * rows, r0 + min(cnt, (t + 1) * (uint32_t)rows), 0u);
}

// k_dist_u8 applies: uint8 rows and queries 16-byte aligned, d in {16, ..., 512}.
bool dist_u8_eligible(const detlsh_index* idx, const void* Q) {
  const int d = idx->d;
  return idx->dtype == DETLSH_U8 && d >= 16 && d <= 512 && (d & (d - 1)) == 0 &&
         reinterpret_cast<uintptr_t>(idx->X) % 16 == 0 && reinterpret_cast<uintptr_t>(Q) % 16 == 0;
}

// Coarse squared distances from the BF16 copy of X (FP32 accumulation): half
// the bytes of the FP32 rows for the same candidates. Each half-warp reads one
// row with 16-byte loads (8 values per lane, d % 8 == 0), so a warp keeps
// 2*ILP rows in flight; hl is the lane within the half-warp.
__device__ __forceinline__ void rows_dist2_bf16(const __nv_bfloat16* __restrict__ Xb, int d,
                                                const uint32_t* ids, const float* __restrict__ q,
                                                int hl, float* acc) {
  const int d8 = d >> 3;
  for (int i = hl; i < d8; i += 16) {
    const float4 qa = __ldg(reinterpret_cast<const float4*>(q) + 2 * i);
    const float4 qb = __ldg(reinterpret_cast<const float4*>(q) + 2 * i + 1);
    uint4 xv[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u)
      xv[u] = (ids[u] != 0xffffffffu)
                  ? __ldg(reinterpret_cast<const uint4*>(Xb + (int64_t)ids[u] * d) + i)
                  : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      if (ids[u] == 0xffffffffu) continue;
      const float2 x0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xv[u].x));
      const float2 x1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xv[u].y));
      const float2 x2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xv[u].z));
      const float2 x3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xv[u].w));
      const float t0 = x0.x - qa.x, t1 = x0.y - qa.y, t2 = x1.x - qa.z, t3 = x1.y - qa.w;
      const float t4 = x2.x - qb.x, t5 = x2.y - qb.y, t6 = x3.x - qb.z, t7 = x3.y - qb.w;
      acc[u] = fmaf(t0, t0, acc[u]);
      acc[u] = fmaf(t1, t1, acc[u]);
      acc[u] = fmaf(t2, t2, acc[u]);
      acc[u] = fmaf(t3, t3, acc[u]);
      acc[u] = fmaf(t4, t4, acc[u]);
      acc[u] = fmaf(t5, t5, acc[u]);
      acc[u] = fmaf(t6, t6, acc[u]);
      acc[u] = fmaf(t7, t7, acc[u]);
    }
  }
}

// Sum 8 per-lane partials over each half-warp so that lane l ends with the
// total of partial (l >> 1) & 7 of its half: three halving exchanges (8, 4, 2)
// each keep half of the partials, then one butterfly step.
__device__ __forceinline__ float transpose_reduce8_half(const float* acc, int lane) {
  float a4[4], a2[2];
  const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b3 ? acc[i] : acc[i + 4];
    const float keep = b3 ? acc[i + 4] : acc[i];
    a4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b2 ? a4[i] : a4[i + 2];
    const float keep = b2 ? a4[i + 2] : a4[i];
    a2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float send = b1 ? a2[0] : a2[1];
  const float keep = b1 ? a2[1] : a2[0];
  float v = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

template <bool BK>
__global__ void __launch_bounds__(DT, 3)
k_dist_bf16(const __nv_bfloat16* __restrict__ Xb, int d, int64_t n, const float* __restrict__ Qf, int64_t q0,
            const uint32_t* __restrict__ cand, const uint2* __restrict__ pairs, int64_t cap,
            const uint4* __restrict__ items, const uint32_t* __restrict__ qtail, uint32_t* __restrict__ head,
            float* __restrict__ d2out) {
  const uint32_t nit = *qtail;
  const int lane = threadIdx.x & 31, h = lane >> 4;
  uint32_t it = next_item(head, lane);
  while (it < nit) {
    const uint4 item = items[it];
    const uint32_t nx = next_item(head, lane);
    const int64_t qb = item.x;
    const int64_t r0 = item.y, r1 = item.z;
    const float* q = Qf + (q0 + qb) * (int64_t)d;
    const uint32_t* cl = cand + qb * cap;
    const uint2* pl = BK ? pairs + qb * cap : nullptr;
    float* out = d2out + qb * cap;
    // warp step: 2*ILP rows, rows e0 + h*ILP + u of half-warp h
    for (int64_t e0 = r0; e0 < r1; e0 += 2 * ILP) {
      uint32_t ids[ILP];
      float acc[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        const int64_t e = e0 + h * ILP + u;
        ids[u] = (e < r1) ? (BK ? __ldg(&pl[e].x) : __ldg(cl + e)) : 0xffffffffu;
        if (ids[u] != 0xffffffffu && !DL_CHECK(ids[u] < n, 13, ids[u])) ids[u] = 0xffffffffu;
        acc[u] = 0.f;
      }
      rows_dist2_bf16(Xb, d, ids, q, lane & 15, acc);
      const float v = transpose_reduce8_half(acc, lane);
      const int64_t e = e0 + (lane >> 1);   // = e0 + h*ILP + ((lane >> 1) & 7)
      if ((lane & 1) == 0 && e < r1) out[BK ? (int64_t)__ldg(&pl[e].y) : e] = v;
    }
    it = nx;
  }
}

__global__ void k_widen_f32(const void* __restrict__ Q, int dtype, int64_t count, float* __restrict__ Qf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    Qf[i] = dtype == DETLSH_U8 ? (float)static_cast<const uint8_t*>(Q)[i] : static_cast<const float*>(Q)[i];
}

// ------------------------------------------------------------------ finalize
constexpr int FT = 256;            // threads per finalize CTA (a query each)
constexpr int FT_WIDE = 512;       // ... for batches of fewer queries than SMs
constexpr int TKC_MAX = 8192;      // top-k / shortlist buffer entries (dynamic shared memory)

// Bitonic sort of tk[0..m) ascending, m a power of two (block-wide, NT threads).
template <int NT>
__device__ void sort_keys(unsigned long long* tk, int m) {
  for (int size = 2; size <= m; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < m / 2; i += NT) {
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

__device__ __forceinline__ int pow2_at_least(int v) {
  int m = 2;
  while (m < v) m <<= 1;
  return m;
}

// Keep the `keep` smallest of the cnt distinct keys tk[0..cnt) (moved, in any
// order, to the front) and return the largest kept key: a radix select of the
// keep-th key over 8-bit digits, then an in-place compaction in which every
// thread first holds its TKC/NT strided keys in registers.
template <int TKC, int NT>
__device__ unsigned long long prune_keys(unsigned long long* tk, int cnt, int keep, uint32_t* hist,
                                         unsigned long long* s_pref, int* s_need, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  unsigned long long prefix = 0, pmask = 0;
  int need = keep;   // rank (1-based) of the wanted key among the keys matching the prefix
  for (int p = 7; p >= 0; --p) {
    for (int i = threadIdx.x; i < 256; i += NT) hist[i] = 0;
    __syncthreads();
    const int it = (cnt + NT - 1) / NT * NT;
    for (int i = threadIdx.x; i < it; i += NT) {
      uint32_t dg = 0xffffffffu;
      if (i < cnt) {
        const unsigned long long k = tk[i];
        if ((k & pmask) == prefix) dg = (uint32_t)((k >> (8 * p)) & 255ull);
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, dg);
      if (dg != 0xffffffffu && (peers & lt) == 0) atomicAdd(&hist[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (w == 0) {
      // first digit whose cumulative count reaches `need` (8 bins per lane, warp scan)
      uint32_t v[8], run = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        v[e] = hist[lane * 8 + e];
        run += v[e];
      }
      uint32_t incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, incl >= (uint32_t)need);
      const int first = bal ? __ffs(bal) - 1 : 31;
      if (lane == first) {
        int acc = (int)(incl - run), dg = lane * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          if (acc + (int)v[e] >= need) break;
          acc += (int)v[e];
          ++dg;
        }
        *s_pref = prefix | ((unsigned long long)min(dg, 255) << (8 * p));
        *s_need = need - acc;
      }
    }
    __syncthreads();
    prefix = *s_pref;
    need = *s_need;
    pmask |= 255ull << (8 * p);
  }
  const unsigned long long kth = prefix;
  constexpr int PER = TKC / NT;
  unsigned long long v[PER];
  uint32_t mask = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = threadIdx.x + j * NT;
    v[j] = i < cnt ? tk[i] : ~0ull;
    if (i < cnt && v[j] <= kth) mask |= 1u << j;
  }
  const uint32_t mine = __popc(mask);
  uint32_t x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();   // also: every key has been read before any is moved
  uint32_t base = x - mine;
  for (int q = 0; q < w; ++q) base += s_warp[q];
#pragma unroll
  for (int j = 0; j < PER; ++j)
    if ((mask >> j) & 1u) tk[base + __popc(mask & ((1u << j) - 1u))] = v[j];
  __syncthreads();
  return kth;
}

struct FinalArgs {
  const uint32_t* cand;
  int64_t cap;
  const float* d2;
  const uint32_t* round_end;
  const float* thrC;
  const uint32_t* meta;
  int64_t q0;
  const uint32_t* nqd;
  const int32_t* k;
  int k_max;
  int64_t* out_ids;
  float* out_dist;
  int32_t* out_stats;
  uint32_t* cand_ids;
  int64_t cand_cap;
  // shortlist re-rank (coarse distances): keep `shortlist` candidates and
  // recompute their distances exactly from X before the top-k
  int shortlist;
  const void* X;
  const void* Q;
  int d;
  bool vec4;
  int64_t wide_below;   // batches of fewer queries take the FT_WIDE-thread kernel
};

// NT threads per query: FT_WIDE for batches of fewer than a.wide_below
// queries (few CTAs, so each query's candidates are spread over more
// threads), else FT. Both widths are launched for such a batch size range (so
// one captured graph serves any batch size); the one that does not apply to
// the batch returns at once.
template <typename TX, int TKC, int NT>
__global__ void __launch_bounds__(NT) k_finalize(FinalArgs a) {
  extern __shared__ __align__(16) unsigned long long tk[];   // [TKC]
  __shared__ uint32_t s_rend[kRoundCap];
  __shared__ float s_thr[kRoundCap];
  __shared__ uint32_t s_hist[kRoundCap + 1];
  __shared__ unsigned long long s_tkn, s_tau;
  __shared__ uint32_t s_nsf, s_stop, s_rounds;
  __shared__ uint32_t s_sel[256], s_warp[NT / 32];
  __shared__ unsigned long long s_pref;
  __shared__ int s_need;
  if (((int64_t)*a.nqd < a.wide_below) != (NT == FT_WIDE)) return;
  if (blockIdx.x >= *a.nqd) return;
  const int64_t qb = blockIdx.x;
  const int64_t qg = a.q0 + qb;
  const uint32_t* m = a.meta + qb * MQ_WORDS;
  // (the list never holds more than cap entries; an overflow is reported in the stats)
  const uint32_t nS0 = m[MQ_NS];
  const uint32_t nS = (uint32_t)min((int64_t)nS0, a.cap);
  (void)DL_CHECK((int64_t)nS0 <= a.cap, 40, nS0);
  const uint32_t t_end = m[MQ_TEND], stopT = m[MQ_STOP];
  const int Ru = (int)m[MQ_RU];
  const int kq = a.k[qg];
  const int keep = a.shortlist > 0 ? max(a.shortlist, kq) : kq;   // entries the buffer keeps
  const int chunk = TKC - keep;
  const uint32_t* cl = a.cand + qb * a.cap;
  const float* dl = a.d2 + qb * a.cap;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int nr = (int)t_end + 1;
  for (int i = threadIdx.x; i < kRoundCap; i += NT) {
    s_rend[i] = i < nr ? a.round_end[qb * kRoundCap + i] : 0u;
    s_thr[i] = i < Ru ? a.thrC[qb * kRoundCap + i] : INFINITY;
  }
  for (int i = threadIdx.x; i <= kRoundCap; i += NT) s_hist[i] = 0;
  __syncthreads();
  // a candidate inserted in round r counts as within c*r_t for every t >= max(r, u),
  // u = first round whose exact threshold (c*r_u)^2 covers its distance
  constexpr int FU = 4;   // candidates per thread in flight
  const uint32_t iters = (nS + NT * FU - 1) / (NT * FU) * (NT * FU);
  // only a distance within the last tested round's threshold counts (most
  // candidates are farther); a thread's positions only grow, so the round
  // of its current position is kept and advanced
  const float thr_last = nr > 0 ? s_thr[nr - 1] : -INFINITY;
  int rcur = 0;
  for (uint32_t p0 = threadIdx.x; p0 < iters; p0 += NT * FU) {
    float dv[FU];
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const uint32_t p = p0 + u * NT;
      dv[u] = p < nS ? dl[p] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < FU; ++u) {
      const uint32_t p = p0 + u * NT;
      uint32_t key = 0xffffffffu;
      if (p < nS && dv[u] <= thr_last) {
        while (rcur < nr && s_rend[rcur] <= p) ++rcur;   // the round p was inserted in
        const int x = rcur + lower_bound_f(s_thr + rcur, nr - rcur, dv[u]);
        if (x < nr) key = (uint32_t)x;
      }
      if (__any_sync(0xffffffffu, key != 0xffffffffu)) {
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        if (key != 0xffffffffu && (peers & lt) == 0) atomicAdd(&s_hist[key], (uint32_t)__popc(peers));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // the ">= k within c*r" test runs after every completed round (not after a
    // round the |S| rule ended early)
    const int last_check = (stopT == 1) ? (int)t_end - 1 : (int)t_end;
    uint32_t stop = stopT, nsf = nS, rounds = t_end + 1;
    unsigned long long within = 0;
    for (int t = 0; t <= last_check; ++t) {
      within += s_hist[t];
      if (within >= (unsigned long long)kq) {
        stop = 2;
        nsf = s_rend[t];
        rounds = (uint32_t)t + 1;
        break;
      }
    }
    s_nsf = nsf;
    s_stop = stop;
    s_rounds = rounds;
    s_tkn = 0;
    s_tau = ~0ull;
  }
  __syncthreads();
  const uint32_t nsf = s_nsf;
  // the `keep` smallest of the first nsf candidates by (distance, id)
  for (uint32_t c0 = 0; c0 < nsf; c0 += chunk) {
    if (s_tkn + chunk > TKC) {
      const int cnt = (int)min(s_tkn, (unsigned long long)TKC);
      __syncthreads();
      if (cnt > keep) {
        const unsigned long long kth = prune_keys<TKC, NT>(tk, cnt, keep, s_sel, &s_pref, &s_need, s_warp);
        if (threadIdx.x == 0) {
          s_tkn = keep;
          s_tau = kth;
        }
      }
      __syncthreads();
    }
    const unsigned long long tau = s_tau;
    const uint32_t c1 = min(nsf, c0 + (uint32_t)chunk);
    const uint32_t tau_hi = (uint32_t)(tau >> 32);
    for (uint32_t p0 = c0 + threadIdx.x; p0 < c1; p0 += NT * FU) {
      uint32_t db[FU];
#pragma unroll
      for (int u = 0; u < FU; ++u) {
        const uint32_t p = p0 + u * NT;
        db[u] = p < c1 ? __float_as_uint(dl[p]) : 0xffffffffu;
      }
      // the id is read only where the distance alone does not decide
      unsigned long long kv[FU];
#pragma unroll
      for (int u = 0; u < FU; ++u) {
        const uint32_t p = p0 + u * NT;
        kv[u] = (p < c1 && db[u] <= tau_hi) ? (((unsigned long long)db[u] << 32) | cl[p]) : ~0ull;
      }
#pragma unroll
      for (int u = 0; u < FU; ++u) {
        if (kv[u] < tau) {
          const unsigned long long slot = atomicAdd(&s_tkn, 1ull);
          if (slot < TKC) tk[slot] = kv[u];
        }
      }
    }
    __syncthreads();
  }
  int have;
  {
    const int cnt = (int)min(s_tkn, (unsigned long long)TKC);
    const int m = pow2_at_least(cnt);
    for (int i = cnt + threadIdx.x; i < m; i += NT) tk[i] = ~0ull;
    sort_keys<NT>(tk, m);
    have = min(cnt, keep);
  }
  if (a.shortlist > 0) {
    // exact FP32 distances of the shortlist, 8 rows per warp, then re-sort
    const TX* X = static_cast<const TX*>(a.X);
    const TX* q = static_cast<const TX*>(a.Q) + qg * (int64_t)a.d;
    for (int e0 = w * ILP; e0 < have; e0 += (NT / 32) * ILP) {
      uint32_t ids[ILP];
      float acc[ILP];
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        ids[u] = (e0 + u < have) ? (uint32_t)(tk[e0 + u] & 0xffffffffull) : 0xffffffffu;
        acc[u] = 0.f;
      }
      rows_dist2<TX, false>(X, a.d, ids, q, a.vec4, lane, acc);
      const float v = transpose_reduce8(acc, lane);
      const int r = (lane >> 2) & 7;
      __syncwarp();
      if ((lane & 3) == 0 && e0 + r < have)
        tk[e0 + r] = ((unsigned long long)__float_as_uint(v) << 32) | (tk[e0 + r] & 0xffffffffull);
    }
    __syncthreads();
    const int m = pow2_at_least(have);
    for (int i = have + threadIdx.x; i < m; i += NT) tk[i] = ~0ull;
    sort_keys<NT>(tk, m);
    have = min(have, kq);
  }
  for (int r = threadIdx.x; r < a.k_max; r += NT) {
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
  if (a.cand_ids) {
    for (uint32_t p = threadIdx.x; p < nsf && (int64_t)p < a.cand_cap; p += NT)
      a.cand_ids[qg * a.cand_cap + p] = cl[p];
  }
  if (threadIdx.x == 0 && a.out_stats) {
    a.out_stats[qg * 4 + 0] = (int32_t)nsf;
    a.out_stats[qg * 4 + 1] = (int32_t)s_rounds;
    a.out_stats[qg * 4 + 2] = (int32_t)s_stop;
    a.out_stats[qg * 4 + 3] = (int32_t)m[MQ_OVERFLOW];
  }
}

}  // namespace

namespace {

__global__ void k_begin_batch(uint32_t* ctr, uint32_t nq) {
  ctr[CT_NQ] = nq;
  ctr[CT_BAD] = 0;
}

__global__ void k_batch_init(uint32_t* __restrict__ ctr, uint32_t* __restrict__ minpos,
                             uint32_t* __restrict__ maxlb, int64_t B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) {
    minpos[i] = 0xffffffffu;
    maxlb[i] = 0u;
  }
  if (i == 0) {
    ctr[CT_WORK] = 0;
    ctr[CT_QTAIL] = 0;
    ctr[CT_HEAD] = 0;
  }
}

// per-query arguments of the batch: 1 <= k <= k_max, finite c > 1, finite r_min
__global__ void k_check_batch(const uint32_t* __restrict__ ctr_nq, const int32_t* __restrict__ k,
                              const float* __restrict__ c, const float* __restrict__ r_min, int k_max,
                              uint32_t* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)*ctr_nq) return;
  const bool ok = k[i] >= 1 && k[i] <= k_max && isfinite(c[i]) && c[i] > 1.0f && isfinite(r_min[i]);
  if (!ok) atomicExch(bad, 1u);
}

// a batch with a bad argument runs as an empty batch
__global__ void k_gate_batch(uint32_t* ctr) {
  if (ctr[CT_BAD]) ctr[CT_NQ] = 0;
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

int tuning_from_params(const detlsh_query_params* qp, QueryTuning* tu) {
  *tu = QueryTuning{};
  if (!qp || !qp->tuning) return DETLSH_OK;
  const detlsh_tuning& t = *qp->tuning;
  DL_REQUIRE(t.batch >= 0, "tuning.batch must be >= 0");
  tu->batch = t.batch;
  tu->walk_ctas_per_sm = t.walk_ctas_per_sm;
  if (t.dist_rows) tu->dist_rows = t.dist_rows;
  tu->dist_ctas_per_sm = t.dist_ctas_per_sm;
  tu->streams = t.streams;
  DL_REQUIRE(t.coarse_gather == 0 || t.coarse_gather == 1, "tuning.coarse_gather must be 0 or 1");
  tu->coarse_gather = t.coarse_gather;
  DL_REQUIRE(t.id_bucket_log2 == 0 || t.id_bucket_log2 == -1 || (t.id_bucket_log2 >= 10 && t.id_bucket_log2 <= 31),
             "tuning.id_bucket_log2 must be 0, -1 or in [10, 31]");
  tu->id_bucket_log2 = t.id_bucket_log2;
  return DETLSH_OK;
}

int query_shape(const detlsh_index* idx, int64_t nq, int k_max, double beta, int shortlist,
                const QueryTuning& tu, QueryShape* out) {
  QueryShape sh{};
  if (shortlist > 0 && (idx->Xb == nullptr || shortlist > TKC_MAX / 2)) {
    set_error("a shortlist needs an index built with the BF16 projection and at most %d entries",
              TKC_MAX / 2);
    return DETLSH_EINVAL;
  }
  if (tu.dist_rows < 64 || tu.dist_rows > 8192 || tu.dist_rows % 64 != 0) {
    set_error("dist_rows must be a multiple of 64 in [64, 8192]");
    return DETLSH_EINVAL;
  }
  if (tu.walk_ctas_per_sm < 0 || tu.walk_ctas_per_sm > 4 || tu.dist_ctas_per_sm < 0 ||
      tu.dist_ctas_per_sm > 4 || tu.batch < 0 || tu.streams < 0 || tu.streams > 2) {
    set_error("walk_ctas_per_sm must be in [0, 4], dist_ctas_per_sm in [0, 4], streams in [0, 2], batch >= 0");
    return DETLSH_EINVAL;
  }
  sh.L = idx->L;
  sh.LK = idx->K * idx->L;
  sh.TL = idx->total_leaves;
  sh.RL = (int64_t)kRoundCap * idx->L;
  sh.k_max = k_max;
  sh.shortlist = shortlist;
  sh.dist_rows = tu.dist_rows;
  // the top-k buffer: 4096 keys while it keeps at most 1024 (k, or a shortlist
  // of up to 1024), else 8192 for a shortlist of up to 4096
  sh.tkc = shortlist > 1024 ? 8192 : 4096;
  int dev = 0, nsm = 0, smem_optin = 0, smem_sm = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  DL_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  DL_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));

  // walk configuration: the dedup bitmap in shared memory when it fits
  sh.words = (idx->n + 31) / 32;
  const WalkLayout with_bm = walk_layout(sh.L, sh.words);
  sh.smem_bitmap = 4 * ((int64_t)with_bm.total + 2048) <= (int64_t)smem_sm;
  const WalkLayout wl = walk_layout(sh.L, sh.smem_bitmap ? sh.words : 0);
  if ((int64_t)wl.total + 1024 > smem_optin) {
    set_error("walk kernel needs %zu bytes of shared memory", wl.total);
    return DETLSH_EINVAL;
  }
  sh.wl_total = wl.total;
  DL_CUDA(cudaFuncSetAttribute(k_leaf_lb<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lb_smem_bytes(sh.LK)));
  DL_CUDA(cudaFuncSetAttribute(k_leaf_lb<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lb_smem_bytes(sh.LK)));
  DL_CUDA(cudaFuncSetAttribute(k_walk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wl.total));
  DL_CUDA(cudaFuncSetAttribute(k_walk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wl.total));
  int walk_per_sm = 0;
  DL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&walk_per_sm, k_walk<false>, WT, wl.total));
  walk_per_sm = std::max(walk_per_sm, 1);
  if (tu.walk_ctas_per_sm > 0) walk_per_sm = std::min(walk_per_sm, tu.walk_ctas_per_sm);
  // the FP32 and uint8 gathers fit four CTAs per SM, the BF16 one three
  sh.dgrid = nsm * (tu.dist_ctas_per_sm ? tu.dist_ctas_per_sm : (shortlist > 0 ? 3 : 4));
  sh.nsm = nsm;
  // split bucketing: per-CTA histograms over (round, tree)
  sh.rq = 1;
  sh.nblk = (sh.TL + kLbBlock - 1) / kLbBlock;
  sh.bk_smem = round_smem_bytes(sh.L);
  if (sh.bk_smem > 48 * 1024)
    DL_CUDA(cudaFuncSetAttribute(k_round_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.bk_smem));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<float, 4096, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<uint8_t, 4096, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<float, 8192, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<uint8_t, 8192, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<float, 4096, FT_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<uint8_t, 4096, FT_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32768));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<float, 8192, FT_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));
  DL_CUDA(cudaFuncSetAttribute(k_finalize<uint8_t, 8192, FT_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536));

  // candidate capacity per query: S stays below beta*n+k until its last leaf
  const double tmax = std::ceil(beta * (double)idx->n + (double)k_max);
  sh.cap = std::max<int64_t>(
      1, std::min<int64_t>(idx->n, (int64_t)std::min(tmax, 9.0e18) - 1 + idx->max_leaf_count));
  // gather by point-id range: ranges of about 32 MB of rows (the gather's row
  // bytes; measured best among 2 to 64 MB on the mid workload), at most
  // kMaxIdBuckets of them, only with more than one
  if (tu.id_bucket_log2 >= 0) {
    const int64_t row_bytes =
        shortlist > 0 ? (int64_t)idx->d * 2 : (int64_t)idx->d * (idx->dtype == DETLSH_U8 ? 1 : 4);
    int bs = tu.id_bucket_log2;
    if (bs == 0) {
      bs = 10;
      while (bs < 31 && ((int64_t)2 << bs) * row_bytes <= ((int64_t)32 << 20)) ++bs;
    }
    while (bs < 31 && ((idx->n - 1) >> bs) + 1 > kMaxIdBuckets) ++bs;
    const int64_t nbk = ((idx->n - 1) >> bs) + 1;
    if (nbk > 1) {
      sh.bshift = bs;
      sh.nbk = nbk;
    }
  }
  sh.items_per_q = (sh.cap + sh.dist_rows - 1) / sh.dist_rows + sh.nbk;
  // shortlist mode: coarse distances by leaf on the tensor cores (each record
  // holds at least one new point, so a query writes at most cap of them)
  sh.lm = shortlist > 0 && idx->chunk_base != nullptr && tu.coarse_gather == 0;
  sh.nk = sh.lm ? idx->n_chunks : 0;
  // batch size: the tuning's, else bounded by the per-query buffers (at most
  // 96 GiB and a third of the free device memory): fewer, larger batches
  // shorten the tails of the per-query kernels, and the rows a batch's
  // queries share are read once per batch (measured at mid with 10,000
  // queries: one batch 73 ms against 77 ms in three; with the leaf-major
  // coarse distances 57 against 76 ms in six)
  const int64_t per_q = sh.TL * 9 + sh.cap * 8 + sh.RL * 16 + kRoundCap * 12 + MQ_WORDS * 4 +
                        sh.LK * 4 + sh.items_per_q * 16 + sh.nblk * 8 +
                        (idx->Xb ? (int64_t)idx->d * 2 : 0) + (shortlist > 0 ? (int64_t)idx->d * 4 : 0) +
                        (sh.lm ? sh.cap * (16 + 16 + 4) + sh.cap / 8 + 4 : 0) +
                        (!sh.lm && sh.nbk ? sh.cap * 8 + sh.nbk * 16 : 0) + 64;
  int64_t B = tu.batch;
  if (B == 0) {
    size_t mem_free = 0, mem_total = 0;
    DL_CUDA(cudaMemGetInfo(&mem_free, &mem_total));
    const int64_t budget = std::min<int64_t>((int64_t)96 << 30, (int64_t)(mem_free / 3));
    B = std::max<int64_t>(1, budget / per_q);
    B = std::min<int64_t>(B, 16384);
  }
  B = std::max<int64_t>(1, std::min<int64_t>(B, std::max<int64_t>(nq, 1)));
  sh.B = B;
  // the grouping pays when a row is a candidate of many queries of a batch
  // (about beta*B of them); with few (small batches, small beta: the serving
  // shapes) its own passes cost more than the reuse saves, so the automatic
  // setting keeps the walk order below beta*B = 16
  if (sh.nbk && tu.id_bucket_log2 == 0 && beta * (double)B < 16.0) {
    sh.nbk = 0;
    sh.bshift = 0;
    sh.items_per_q = (sh.cap + sh.dist_rows - 1) / sh.dist_rows;
  }
  sh.wgrid = (int)std::min<int64_t>(B, (int64_t)nsm * walk_per_sm);
  int64_t max_tree_leaves = 1;
  for (int t = 0; t < sh.L; ++t)
    max_tree_leaves = std::max<int64_t>(max_tree_leaves, idx->leaf_base_h[t + 1] - idx->leaf_base_h[t]);
  sh.max_tree_leaves = max_tree_leaves;

  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p += al256(bytes);
    return at;
  };
  sh.o_ctr = take(sizeof(uint32_t) * CT_WORDS);
  sh.o_qp = take(sizeof(float) * B * sh.LK);
  sh.o_qb16 = take(idx->Xb ? (size_t)B * idx->d * 2 : 0);
  sh.o_qf = take(shortlist > 0 ? sizeof(float) * B * idx->d : 0);
  sh.o_lb = take(sizeof(float) * B * sh.TL);
  sh.o_mm = take(sizeof(uint32_t) * 2 * B);
  sh.o_lround = take((size_t)B * sh.TL);
  sh.o_hist = take(sizeof(uint32_t) * B * sh.RL);
  sh.o_blkmin = take(sizeof(uint32_t) * B * sh.nblk);
  sh.o_blist = take(sizeof(uint32_t) * B * sh.nblk);
  sh.o_boff = take(sizeof(uint32_t) * B * (sh.RL + 1));
  sh.o_list = take(sizeof(uint32_t) * B * sh.TL);
  sh.o_cand = take(sizeof(uint32_t) * B * sh.cap);
  sh.o_d2 = take(sizeof(float) * B * sh.cap);
  sh.o_rend = take(sizeof(uint32_t) * B * kRoundCap);
  sh.o_thr = take(sizeof(float) * 2 * B * kRoundCap);
  sh.o_meta = take(sizeof(uint32_t) * B * MQ_WORDS);
  sh.o_wsnew = take(sizeof(uint32_t) * 3 * sh.wgrid * max_tree_leaves);
  sh.o_wsbm = take(sh.smem_bitmap ? 0 : sizeof(uint32_t) * sh.wgrid * sh.words);
  sh.o_wspos = take(sh.smem_bitmap || !idx->leaf_pos ? 0 : sizeof(uint32_t) * sh.wgrid * sh.cap);
  sh.o_items = take(sizeof(uint4) * B * sh.items_per_q);
  sh.o_qk = take(sizeof(uint32_t) * 4 * B);
  sh.qsort_bytes = radix_ws_bytes(B, 0, 32);
  sh.o_qsort = take(sh.qsort_bytes);
  if (sh.lm) {
    sh.nbk = 0;   // the leaf-major coarse distances take no items
    sh.bshift = 0;
  }
  if (sh.nbk) {
    const int64_t cells = sh.nbk * B;
    sh.o_pairs = take(sizeof(uint2) * B * sh.cap);
    sh.o_bcnt = take(sizeof(uint32_t) * cells);
    sh.o_boffq = take(sizeof(uint32_t) * cells);
    sh.o_icnt = take(sizeof(uint32_t) * cells);
    sh.o_ioff = take(sizeof(uint32_t) * (cells + 1));
    sh.bscan_bytes = scan_ws_bytes(cells);
    sh.o_bscan = take(sh.bscan_bytes);
  }
  if (sh.lm) {
    sh.max_units = sh.nk + (B * sh.cap) / 128 + 1;
    sh.o_rec = take(sizeof(uint4) * B * sh.cap);
    sh.o_srec = take(sizeof(uint4) * B * sh.cap);
    sh.o_sq = take(sizeof(uint32_t) * B * sh.cap);
    sh.o_qn = take(sizeof(float) * B);
    const int64_t nks = lm_sort_keys(sh.nk);
    sh.o_khist = take(sizeof(uint32_t) * nks);
    sh.o_kcur = take(sizeof(uint32_t) * nks);
    sh.o_koff = take(sizeof(uint32_t) * (nks + 1));
    sh.o_ucnt = take(sizeof(uint32_t) * sh.nk);
    sh.o_uoff = take(sizeof(uint32_t) * (sh.nk + 1));
    sh.o_units = take(sizeof(uint4) * sh.max_units);
    sh.scanws_bytes = scan_ws_bytes(nks);
    sh.o_scanws = take(sh.scanws_bytes);
  }
  sh.bytes = p;
  *out = sh;
  return DETLSH_OK;
}

int init_query_scratch(const QueryShape& sh, void* base, cudaStream_t s) {
  char* b = static_cast<char*>(base);
  DL_CUDA(cudaMemsetAsync(b + sh.o_ctr, 0, sizeof(uint32_t) * CT_WORDS, s));
  // the walk leaves each CTA's bitmap zeroed after every query
  if (!sh.smem_bitmap)
    DL_CUDA(cudaMemsetAsync(b + sh.o_wsbm, 0, sizeof(uint32_t) * sh.wgrid * sh.words, s));
  return DETLSH_OK;
}

uint32_t* query_ctr(const QueryShape& sh, void* base) {
  return reinterpret_cast<uint32_t*>(static_cast<char*>(base) + sh.o_ctr);
}

int set_batch_size(const QueryShape& sh, void* base, int64_t nq, cudaStream_t s) {
  k_begin_batch<<<1, 1, 0, s>>>(query_ctr(sh, base), (uint32_t)nq);
  DL_LAUNCH();
  return DETLSH_OK;
}

int check_batch_args(const QueryShape& sh, void* base, const int32_t* k, const float* c,
                     const float* r_min, cudaStream_t s) {
  uint32_t* ctr = query_ctr(sh, base);
  k_check_batch<<<ceil_div(sh.B, 256), 256, 0, s>>>(ctr + CT_NQ, k, c, r_min, sh.k_max, ctr + CT_BAD);
  DL_LAUNCH();
  k_gate_batch<<<1, 1, 0, s>>>(ctr);
  DL_LAUNCH();
  return DETLSH_OK;
}

int enqueue_batch(const detlsh_index* idx, const QueryShape& sh, void* base, const void* Q, int64_t q0,
                  int64_t nqg, const int32_t* k, const float* c, const float* r_min, double eps,
                  double beta, int64_t* out_ids, float* out_dist, int32_t* out_stats,
                  uint32_t* cand_ids, int64_t cand_cap, float* qproj, bool vec4, PhaseTimer* timer,
                  cudaStream_t s) {
  char* b = static_cast<char*>(base);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(b + sh.o_ctr);
  const uint32_t* nqd = ctr + CT_NQ;
  float* qp = reinterpret_cast<float*>(b + sh.o_qp);
  float* lb = reinterpret_cast<float*>(b + sh.o_lb);
  uint32_t* d_min = reinterpret_cast<uint32_t*>(b + sh.o_mm);
  uint32_t* d_max = d_min + sh.B;
  uint8_t* lround = reinterpret_cast<uint8_t*>(b + sh.o_lround);
  uint32_t* h_pts = reinterpret_cast<uint32_t*>(b + sh.o_hist);
  uint32_t* boff = reinterpret_cast<uint32_t*>(b + sh.o_boff);
  uint32_t* list = reinterpret_cast<uint32_t*>(b + sh.o_list);
  uint32_t* candb = reinterpret_cast<uint32_t*>(b + sh.o_cand);
  float* d2b = reinterpret_cast<float*>(b + sh.o_d2);
  uint32_t* rend = reinterpret_cast<uint32_t*>(b + sh.o_rend);
  float* thrP = reinterpret_cast<float*>(b + sh.o_thr);
  float* thrC = thrP + sh.B * kRoundCap;
  uint32_t* meta = reinterpret_cast<uint32_t*>(b + sh.o_meta);
  uint4* items = reinterpret_cast<uint4*>(b + sh.o_items);
  uint32_t* qk = reinterpret_cast<uint32_t*>(b + sh.o_qk);   // keys, ids, sorted keys, order
  const int LK = sh.LK, L = sh.L;
  const int64_t TL = sh.TL;
  const size_t srow = (size_t)idx->d * (idx->dtype == DETLSH_U8 ? 1 : 4);
  const void* Qb = static_cast<const char*>(Q) + (size_t)q0 * srow;

  PhaseTimer off(s, false);
  PhaseTimer& tm = timer ? *timer : off;
  const bool timed = timer != nullptr;
  k_batch_init<<<ceil_div(sh.B, 256), 256, 0, s>>>(ctr, d_min, d_max, sh.B);
  DL_LAUNCH();
  // projected queries of the batch
  tm.begin(TR_QUERY_PROJ);
  if (idx->proj_mode == DETLSH_PROJ_BF16) {
    void* qb16 = b + sh.o_qb16;
    DL_TRY(to_bf16(Qb, idx->dtype, nqg * idx->d, qb16, s));
    DL_TRY(launch_project_tc(qb16, nqg, idx->d, idx->Ab, LK, idx->K, nullptr, nullptr, nullptr, nullptr, idx->Nr,
                             nullptr, qp, LK,
                             1, idx->d_err, s));
  } else {
    DL_TRY(launch_project_t(Qb, idx->dtype, nqg, idx->d, nullptr, idx->At, LK, qp, LK, 1, s));
  }
  // optional copy of the projected queries (what every later kernel reads)
  if (qproj)
    DL_CUDA(cudaMemcpyAsync(qproj + q0 * LK, qp, sizeof(float) * nqg * LK, cudaMemcpyDeviceToDevice, s));
  // the walk's query order: by locality key
  k_query_keys<<<ceil_div(nqg, 256), 256, 0, s>>>(qp, LK, nqd, idx->E, idx->Nr, idx->K, nqg, qk, qk + sh.B);
  DL_LAUNCH();
  DL_TRY(radix_sort_pairs_ws(qk, qk + sh.B, nqg, 0, 32, qk + 2 * sh.B, qk + 3 * sh.B, b + sh.o_qsort,
                             sh.qsort_bytes, s));
  tm.end();
  // FP32 queries of the batch for the coarse distances
  float* qf = reinterpret_cast<float*>(b + sh.o_qf);
  if (sh.shortlist > 0) {
    k_widen_f32<<<(unsigned)std::min<int64_t>(ceil_div(nqg * idx->d, 256), 152 * 16), 256, 0, s>>>(
        Qb, idx->dtype, nqg * idx->d, qf);
    DL_LAUNCH();
  }

  dim3 g1(ceil_div(TL, LB_THREADS), ceil_div(nqg, LB_QCH));
  tm.begin(TR_LB);
  uint32_t* blkmin = reinterpret_cast<uint32_t*>(b + sh.o_blkmin);
  (idx->K == 16 ? k_leaf_lb<16> : k_leaf_lb<0>)<<<g1, LB_THREADS, lb_smem_bytes(LK), s>>>(qp, nqd, LK, idx->E, idx->Nr, idx->K, idx->leaf_lo, idx->leaf_hi,
                                      idx->leaf_tree, TL, lb, d_min, d_max, blkmin, sh.nblk);
  DL_LAUNCH();
  tm.end();
  trace_add(TR_LB_LAUNCHES, timed ? 1.0 : 0.0);

  tm.begin(TR_BUCKET);
  k_thresh<<<ceil_div(nqg, 128), 128, 0, s>>>(d_min, d_max, q0, nqd, k, c, r_min, eps, beta, idx->n,
                                              thrP, thrC, meta);
  DL_LAUNCH();
  k_round_expand<<<(unsigned)nqg, RX, sh.bk_smem, s>>>(lb, blkmin, TL, sh.nblk, thrP, idx->leaf_tree, idx->leaf_range,
                                                      L, nqd, lround, reinterpret_cast<uint32_t*>(b + sh.o_blist),
                                                      h_pts, boff, list, meta);
  DL_LAUNCH();
  tm.end();

  WalkArgs wa{};
  wa.n = idx->n;
  wa.L = L;
  wa.leaf_ids = idx->leaf_ids;
  wa.leaf_range = idx->leaf_range;
  wa.leaf_tree = idx->leaf_tree;
  wa.total_leaves = TL;
  wa.nqd = nqd;
  wa.lb2 = lb;
  wa.list = list;
  wa.boff = boff;
  wa.hist_pts = h_pts;
  wa.meta = meta;
  wa.cand = candb;
  wa.cap = sh.cap;
  wa.round_end = rend;
  wa.ws_newcnt = reinterpret_cast<uint32_t*>(b + sh.o_wsnew);
  wa.max_bucket = sh.max_tree_leaves;
  wa.ws_bitmap = sh.smem_bitmap ? nullptr : reinterpret_cast<uint32_t*>(b + sh.o_wsbm);
  wa.ws_pos = sh.smem_bitmap || !idx->leaf_pos ? nullptr : reinterpret_cast<uint32_t*>(b + sh.o_wspos);
  wa.leaf_pos = idx->leaf_pos;
  wa.bitmap_words = sh.words;
  wa.smem_bitmap = sh.smem_bitmap ? 1 : 0;
  wa.work = ctr + CT_WORK;
  wa.order = qk + 3 * sh.B;
  wa.items = items;
  wa.qtail = ctr + CT_QTAIL;
  wa.dist_rows = sh.dist_rows;
  wa.rec = sh.lm ? reinterpret_cast<uint4*>(b + sh.o_rec) : nullptr;
  wa.queue_items = sh.nbk ? 0 : 1;
  tm.begin(TR_WALK);
  if (idx->leaf_pos)
    k_walk<true><<<(unsigned)std::min<int64_t>(nqg, sh.wgrid), WT, sh.wl_total, s>>>(wa);
  else
    k_walk<false><<<(unsigned)std::min<int64_t>(nqg, sh.wgrid), WT, sh.wl_total, s>>>(wa);
  DL_LAUNCH();
  tm.end();

  tm.begin(TR_GROUP);
  const uint2* pairs = sh.nbk ? reinterpret_cast<const uint2*>(b + sh.o_pairs) : nullptr;
  if (sh.nbk && nqg > 0) {
    // the distance work by point-id range: per query its candidates grouped by
    // range, then the items of every (range, query) cell, range-major
    uint32_t* bcnt = reinterpret_cast<uint32_t*>(b + sh.o_bcnt);
    uint32_t* boffq = reinterpret_cast<uint32_t*>(b + sh.o_boffq);
    uint32_t* icnt = reinterpret_cast<uint32_t*>(b + sh.o_icnt);
    uint32_t* ioff = reinterpret_cast<uint32_t*>(b + sh.o_ioff);
    const int64_t cells = sh.nbk * nqg;
    k_cand_buckets<<<(unsigned)nqg, BKT, 0, s>>>(candb, sh.cap, meta, nqd, sh.bshift, (int)sh.nbk, nqg,
                                                 reinterpret_cast<uint2*>(b + sh.o_pairs), bcnt, boffq);
    DL_LAUNCH();
    k_cell_items<<<ceil_div(cells, 256), 256, 0, s>>>(bcnt, cells, sh.dist_rows, icnt);
    DL_LAUNCH();
    DL_TRY(exclusive_scan_u32_ws(icnt, ioff, cells, ctr + CT_QTAIL, b + sh.o_bscan, sh.bscan_bytes, s));
    k_cell_fill<<<ceil_div(cells, 256), 256, 0, s>>>(bcnt, ioff, boffq, (int)sh.nbk, nqg, sh.dist_rows, items);
    DL_LAUNCH();
  }
  tm.end();
  tm.begin(TR_DIST);
  if (sh.lm) {
    LmBatch lb{};
    lb.qb16 = b + sh.o_qb16;
    lb.nqg = nqg;
    lb.nqd = nqd;
    lb.rec = reinterpret_cast<const uint4*>(b + sh.o_rec);
    lb.cap = sh.cap;
    lb.meta = meta;
    lb.mq_words = MQ_WORDS;
    lb.mq_nrec = MQ_NREC;
    lb.qn = reinterpret_cast<float*>(b + sh.o_qn);
    lb.khist = reinterpret_cast<uint32_t*>(b + sh.o_khist);
    lb.kcur = reinterpret_cast<uint32_t*>(b + sh.o_kcur);
    lb.koff = reinterpret_cast<uint32_t*>(b + sh.o_koff);
    lb.ucnt = reinterpret_cast<uint32_t*>(b + sh.o_ucnt);
    lb.uoff = reinterpret_cast<uint32_t*>(b + sh.o_uoff);
    lb.nunits = ctr + CT_NUNITS;
    lb.srec = reinterpret_cast<uint4*>(b + sh.o_srec);
    lb.sq = reinterpret_cast<uint32_t*>(b + sh.o_sq);
    lb.units = reinterpret_cast<uint4*>(b + sh.o_units);
    lb.scan_ws = b + sh.o_scanws;
    lb.scan_ws_bytes = sh.scanws_bytes;
    lb.d2 = d2b;
    DL_TRY(enqueue_coarse_lm(idx, lb, s));
  } else if (sh.shortlist > 0) {
    (pairs ? k_dist_bf16<true> : k_dist_bf16<false>)<<<sh.dgrid, DT, 0, s>>>(
        static_cast<const __nv_bfloat16*>(idx->Xb), idx->d, idx->n, qf, 0, candb, pairs, sh.cap, items, ctr + CT_QTAIL,
        ctr + CT_HEAD, d2b);
  } else if (dist_u8_eligible(idx, Q)) {
    (pairs ? k_dist_u8<true> : k_dist_u8<false>)<<<sh.dgrid, DT, 0, s>>>(
        static_cast<const uint8_t*>(idx->X), idx->d, idx->n, static_cast<const uint8_t*>(Q), q0, candb, pairs, sh.cap,
        items, ctr + CT_QTAIL, ctr + CT_HEAD, d2b);
  } else if (idx->dtype == DETLSH_U8) {
    (pairs ? k_dist<uint8_t, true> : k_dist<uint8_t, false>)<<<sh.dgrid, DT, 0, s>>>(
        static_cast<const uint8_t*>(idx->X), idx->d, idx->n, static_cast<const uint8_t*>(Q), q0, candb, pairs, sh.cap,
        items, ctr + CT_QTAIL, ctr + CT_HEAD, d2b, vec4);
  } else if (vec4 && idx->d <= 128) {
    auto kern = pairs ? k_dist_g8<4, true> : k_dist_g8<4, false>;
    switch ((idx->d / 4 + 7) / 8) {
      case 1: kern = pairs ? k_dist_g8<1, true> : k_dist_g8<1, false>; break;
      case 2: kern = pairs ? k_dist_g8<2, true> : k_dist_g8<2, false>; break;
      case 3: kern = pairs ? k_dist_g8<3, true> : k_dist_g8<3, false>; break;
      default: break;
    }
    kern<<<sh.dgrid, DT, 0, s>>>(static_cast<const float*>(idx->X), idx->d, idx->n, static_cast<const float*>(Q), q0,
                                 candb, pairs, sh.cap, items, ctr + CT_QTAIL, ctr + CT_HEAD, d2b);
  } else {
    (pairs ? k_dist<float, true> : k_dist<float, false>)<<<sh.dgrid, DT, 0, s>>>(
        static_cast<const float*>(idx->X), idx->d, idx->n, static_cast<const float*>(Q), q0, candb, pairs, sh.cap, items,
        ctr + CT_QTAIL, ctr + CT_HEAD, d2b, vec4);
  }
  DL_LAUNCH();
  tm.end();
  trace_add(TR_DIST_LAUNCHES, timed ? 1.0 : 0.0);

  FinalArgs fa{};
  fa.cand = candb;
  fa.cap = sh.cap;
  fa.d2 = d2b;
  fa.round_end = rend;
  fa.thrC = thrC;
  fa.meta = meta;
  fa.q0 = q0;
  fa.nqd = nqd;
  fa.k = k;
  fa.k_max = sh.k_max;
  fa.out_ids = out_ids;
  fa.out_dist = out_dist;
  fa.out_stats = out_stats;
  fa.cand_ids = cand_ids;
  fa.cand_cap = cand_cap;
  fa.shortlist = sh.shortlist;
  fa.X = idx->X;
  fa.Q = Q;
  fa.d = idx->d;
  fa.vec4 = vec4;
  fa.wide_below = sh.nsm;
  const size_t fin_smem = sizeof(unsigned long long) * sh.tkc;
  tm.begin(TR_FINALIZE);
  if (idx->dtype == DETLSH_U8) {
    (sh.tkc == 4096 ? k_finalize<uint8_t, 4096, FT> : k_finalize<uint8_t, 8192, FT>)<<<(unsigned)nqg, FT, fin_smem, s>>>(fa);
    DL_LAUNCH();
    if (nqg > 0) {
      (sh.tkc == 4096 ? k_finalize<uint8_t, 4096, FT_WIDE>
                      : k_finalize<uint8_t, 8192, FT_WIDE>)<<<(unsigned)std::min<int64_t>(nqg, sh.nsm), FT_WIDE,
                                                             fin_smem, s>>>(fa);
      DL_LAUNCH();
    }
  } else {
    (sh.tkc == 4096 ? k_finalize<float, 4096, FT> : k_finalize<float, 8192, FT>)<<<(unsigned)nqg, FT, fin_smem, s>>>(fa);
    DL_LAUNCH();
    if (nqg > 0) {
      (sh.tkc == 4096 ? k_finalize<float, 4096, FT_WIDE>
                      : k_finalize<float, 8192, FT_WIDE>)<<<(unsigned)std::min<int64_t>(nqg, sh.nsm), FT_WIDE,
                                                           fin_smem, s>>>(fa);
      DL_LAUNCH();
    }
  }
  tm.end();
  return DETLSH_OK;
}

bool query_vec4(const detlsh_index* idx, const void* Q) {
  const uintptr_t al = idx->dtype == DETLSH_U8 ? 4 : 16;
  return (idx->d % 4 == 0) && (reinterpret_cast<uintptr_t>(idx->X) % al == 0) &&
         (reinterpret_cast<uintptr_t>(Q) % al == 0);
}

namespace {

// A second stream per device for pipelined batches (created on first use).
cudaStream_t side_stream() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static cudaStream_t streams[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    streams[dev] = nullptr;
    cudaGetLastError();
  }
  return streams[dev];
}

// s2 starts after the work already on s, and s waits for s2 at the join. The
// destructor joins a fork left open by an early return, so that memory freed
// in stream order on s is never freed under work still queued on s2.
struct StreamFork {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr, s2 = nullptr;
  bool open = false;
  ~StreamFork() {
    if (open) {
      cudaEventRecord(e1, s2);
      cudaStreamWaitEvent(s, e1, 0);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  int begin(cudaStream_t a, cudaStream_t b) {
    s = a;
    s2 = b;
    DL_CUDA(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
    DL_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
    DL_CUDA(cudaEventRecord(e0, s));
    DL_CUDA(cudaStreamWaitEvent(s2, e0, 0));
    open = true;
    return DETLSH_OK;
  }
  int join() {
    open = false;
    DL_CUDA(cudaEventRecord(e1, s2));
    DL_CUDA(cudaStreamWaitEvent(s, e1, 0));
    return DETLSH_OK;
  }
};

// dst row i = src row perm[i] (gather) or dst row perm[i] = src row i
// (scatter), rows of `words` 32-bit words or of `bytes` bytes
template <typename W, bool GATHER>
__global__ void k_permute_rows(const W* __restrict__ src, W* __restrict__ dst, const uint32_t* __restrict__ perm,
                               int64_t rows, int64_t row_len) {
  const int64_t total = rows * row_len;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / row_len, j = e - i * row_len;
    const int64_t pi = perm[i];
    if (GATHER) dst[i * row_len + j] = src[pi * row_len + j];
    else dst[pi * row_len + j] = src[i * row_len + j];
  }
}

template <bool GATHER>
int permute_rows(const void* src, void* dst, const uint32_t* perm, int64_t rows, size_t row_bytes, cudaStream_t s) {
  if (rows == 0 || row_bytes == 0) return DETLSH_OK;
  const bool w4 = row_bytes % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 4 == 0 &&
                  reinterpret_cast<uintptr_t>(dst) % 4 == 0;
  const int64_t len = w4 ? (int64_t)(row_bytes / 4) : (int64_t)row_bytes;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(rows * len, 256), 152 * 16);
  if (w4)
    k_permute_rows<uint32_t, GATHER><<<blocks, 256, 0, s>>>(static_cast<const uint32_t*>(src),
                                                            static_cast<uint32_t*>(dst), perm, rows, len);
  else
    k_permute_rows<uint8_t, GATHER><<<blocks, 256, 0, s>>>(static_cast<const uint8_t*>(src),
                                                           static_cast<uint8_t*>(dst), perm, rows, len);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace

int run_query(const detlsh_index* idx, const void* Q, int64_t nq, const int32_t* k, const float* c,
              const float* r_min, int k_max, double eps, double beta, int64_t* out_ids,
              float* out_dist, int32_t* out_stats, uint32_t* cand_ids, int64_t cand_cap,
              float* qproj, int shortlist, const QueryTuning& tu, cudaStream_t s) {
  if (nq == 0) return DETLSH_OK;
  // with streams = 2 and several batches, batches alternate between two
  // streams (one batch's distance gather may overlap the next one's walk),
  // each with its own scratch of half the memory budget
  QueryTuning t1 = tu;
  QueryShape sh;
  DL_TRY(query_shape(idx, nq, k_max, beta, shortlist, t1, &sh));
  const int nstreams = (tu.streams == 2 && nq > sh.B) ? 2 : 1;
  if (nstreams == 2 && tu.batch == 0) t1.batch = std::max<int64_t>(1, (sh.B + 1) / 2);
  DL_TRY(query_shape(idx, nq, k_max, beta, shortlist, t1, &sh));
  Scratch ws, ws2;
  DL_TRY(ws.alloc(sh.bytes, s));
  DL_TRY(init_query_scratch(sh, ws.p, s));
  cudaStream_t s2 = nullptr;
  if (nstreams == 2) {
    DL_TRY(ws2.alloc(sh.bytes, s));
    DL_TRY(init_query_scratch(sh, ws2.p, s));
    s2 = side_stream();
    if (!s2) {
      set_error("could not create a query stream");
      return DETLSH_ECUDA;
    }
  }
  const size_t srow = (size_t)idx->d * (idx->dtype == DETLSH_U8 ? 1 : 4);
  const void* Qr = Q;
  const int32_t* kr = k;
  const float *cr = c, *rr = r_min;
  int64_t* oi = out_ids;
  float* od = out_dist;
  int32_t* os = out_stats;
  uint32_t* oc = cand_ids;
  float* oq = qproj;
  Scratch ord, inq, outq;
  const uint32_t* perm = nullptr;
  if (nq > sh.B) {
    // several batches: all queries in locality order first, so that each
    // batch holds neighbouring queries (their candidate rows meet in L2);
    // inputs are gathered in that order and results scattered back
    const int LK = sh.LK;
    const size_t keys_b = (sizeof(uint32_t) * 4 * nq + 255) & ~size_t(255);
    const size_t sort_b = radix_ws_bytes(nq, 0, 32);
    DL_TRY(ord.alloc(sizeof(float) * nq * LK + keys_b + sort_b, s));
    float* qpa = ord.as<float>();
    uint32_t* keys = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ord.p) + sizeof(float) * nq * LK);
    DL_TRY(launch_project_t(Q, idx->dtype, nq, idx->d, nullptr, idx->At, LK, qpa, LK, 1, s));
    DL_TRY(set_batch_size(sh, ws.p, nq, s));
    k_query_keys<<<ceil_div(nq, 256), 256, 0, s>>>(qpa, LK, query_ctr(sh, ws.p) + CT_NQ, idx->E, idx->Nr,
                                                  idx->K, nq, keys, keys + nq);
    DL_LAUNCH();
    DL_TRY(radix_sort_pairs_ws(keys, keys + nq, nq, 0, 32, keys + 2 * nq, keys + 3 * nq,
                               reinterpret_cast<char*>(keys) + keys_b, sort_b, s));
    perm = keys + 3 * nq;
    const size_t q_b = (srow * nq + 255) & ~size_t(255), a_b = (sizeof(float) * nq + 255) & ~size_t(255);
    DL_TRY(inq.alloc(q_b + 3 * a_b, s));
    char* ib = static_cast<char*>(inq.p);
    DL_TRY(permute_rows<true>(Q, ib, perm, nq, srow, s));
    DL_TRY(permute_rows<true>(k, ib + q_b, perm, nq, 4, s));
    DL_TRY(permute_rows<true>(c, ib + q_b + a_b, perm, nq, 4, s));
    DL_TRY(permute_rows<true>(r_min, ib + q_b + 2 * a_b, perm, nq, 4, s));
    Qr = ib;
    kr = reinterpret_cast<const int32_t*>(ib + q_b);
    cr = reinterpret_cast<const float*>(ib + q_b + a_b);
    rr = reinterpret_cast<const float*>(ib + q_b + 2 * a_b);
    const size_t ids_b = (sizeof(int64_t) * nq * k_max + 255) & ~size_t(255);
    const size_t dist_b = (sizeof(float) * nq * k_max + 255) & ~size_t(255);
    const size_t st_b = (sizeof(int32_t) * nq * 4 + 255) & ~size_t(255);
    const size_t cand_b = cand_ids ? (sizeof(uint32_t) * nq * cand_cap + 255) & ~size_t(255) : 0;
    const size_t qp_b = qproj ? sizeof(float) * nq * LK : 0;
    DL_TRY(outq.alloc(ids_b + dist_b + st_b + cand_b + qp_b, s));
    char* obuf = static_cast<char*>(outq.p);
    oi = reinterpret_cast<int64_t*>(obuf);
    od = reinterpret_cast<float*>(obuf + ids_b);
    os = out_stats ? reinterpret_cast<int32_t*>(obuf + ids_b + dist_b) : nullptr;
    oc = cand_ids ? reinterpret_cast<uint32_t*>(obuf + ids_b + dist_b + st_b) : nullptr;
    oq = qproj ? reinterpret_cast<float*>(obuf + ids_b + dist_b + st_b + cand_b) : nullptr;
  }
  const bool vec4 = query_vec4(idx, Qr);
  PhaseTimer tm0(s), tm1(s2 ? s2 : s);
  StreamFork fork;
  if (nstreams == 2) DL_TRY(fork.begin(s, s2));
  int64_t bi = 0;
  for (int64_t q0 = 0; q0 < nq; q0 += sh.B, ++bi) {
    const int64_t nqb = std::min<int64_t>(sh.B, nq - q0);
    const bool odd = nstreams == 2 && (bi & 1);
    cudaStream_t sb = odd ? s2 : s;
    void* wb = odd ? ws2.p : ws.p;
    DL_TRY(set_batch_size(sh, wb, nqb, sb));
    DL_TRY(enqueue_batch(idx, sh, wb, Qr, q0, nqb, kr, cr, rr, eps, beta, oi, od, os, oc, cand_cap, oq, vec4,
                         odd ? &tm1 : &tm0, sb));
  }
  if (nstreams == 2) DL_TRY(fork.join());
  DL_TRY(tm0.finish());
  DL_TRY(tm1.finish());
  if (perm) {
    DL_TRY(permute_rows<false>(oi, out_ids, perm, nq, sizeof(int64_t) * k_max, s));
    DL_TRY(permute_rows<false>(od, out_dist, perm, nq, sizeof(float) * k_max, s));
    if (out_stats) DL_TRY(permute_rows<false>(os, out_stats, perm, nq, sizeof(int32_t) * 4, s));
    if (cand_ids) DL_TRY(permute_rows<false>(oc, cand_ids, perm, nq, sizeof(uint32_t) * cand_cap, s));
    if (qproj) DL_TRY(permute_rows<false>(oq, qproj, perm, nq, sizeof(float) * sh.LK, s));
  }
  if (idx->proj_mode == DETLSH_PROJ_BF16) DL_TRY(check_tc_error(idx->d_err, s));
  return DETLSH_OK;
}

}  // namespace detlsh
