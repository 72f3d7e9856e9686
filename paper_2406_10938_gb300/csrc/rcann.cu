// The (r,c)-ANN query of Alg. 6 over the index's DE-Trees, built on the exact
// range query of Alg. 4 and Alg. 5: a leaf whose lower bound exceeds the
// projected radius eps*r is skipped, a leaf whose upper bound does not exceed
// it gives all its points, and any other leaf gives the points whose own
// projection lies within the radius. Trees are range-queried in order, their
// results added to S; once |S| >= beta*n + 1 the point of S closest to q is
// returned, and after the last tree it is returned if it lies within c*r.
//
// One CTA per query; every value is FP64 (the query's and the checked points'
// projections, the bounds, the distances) with round-to-nearest operations in
// a fixed order, so the results equal an FP64 restatement exactly whenever the
// inputs make those sums exact. This is the paper's un-optimised query
// semantics (the c^2-k-ANN path of query.cu is the throughput path).
#include <cmath>

#include "common.cuh"

namespace detlsh {
namespace {

constexpr int RT = 256;   // threads per query

struct RcArgs {
  const void* X;
  int dtype;
  int64_t n;
  int d;
  const float* A;             // [L*K][d]
  const float* E;             // [L*K][Nr+1]
  int K, L, Nr;
  const uint32_t* leaf_ids;   // [L][n]
  const uint32_t* leaf_range; // [leaves][2]: first position within the tree, count
  const uint8_t* leaf_lo;     // [leaves][K]
  const uint8_t* leaf_hi;     // [leaves][K]
  const int64_t* leaf_base;   // [L+1]
  const void* Q;              // [nq][d], the index's dtype
  const float* r;             // [nq]
  const float* c;             // [nq]
  double eps, beta;
  uint32_t* bitmap;           // [nq][words], zero: membership of S
  int64_t words;
  int64_t* out_id;            // [nq]
  double* out_dist;           // [nq]
  int32_t* out_stats;         // [nq][3]: |S|, trees queried, stop rule
};

__device__ __forceinline__ double value_at(const void* p, int dtype, int64_t i) {
  return dtype == DETLSH_U8 ? (double)static_cast<const uint8_t*>(p)[i] : (double)static_cast<const float*>(p)[i];
}

// Eq. 1 in FP64: sum over t of A[h][t] * v[t], t in order.
__device__ double project_fp64(const float* A, int d, int h, const void* v, int dtype, int64_t off) {
  double acc = 0.0;
  for (int t = 0; t < d; ++t) acc = __dadd_rn(acc, __dmul_rn((double)A[(int64_t)h * d + t], value_at(v, dtype, off + t)));
  return acc;
}

__global__ void __launch_bounds__(RT) k_rc_ann(RcArgs a) {
  extern __shared__ double s_qp[];   // [L*K] the query's projections
  __shared__ unsigned long long s_cnt;
  __shared__ double s_bd[RT / 32];
  __shared__ long long s_bi[RT / 32];
  const int64_t b = blockIdx.x;
  const int d = a.d, K = a.K;
  const int64_t qoff = b * d;
  for (int h = threadIdx.x; h < K * a.L; h += RT) s_qp[h] = project_fp64(a.A, d, h, a.Q, a.dtype, qoff);
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const double rr = (double)a.r[b];
  const double rp = __dmul_rn(a.eps, rr);
  const double rp2 = __dmul_rn(rp, rp);
  const double bound = __dadd_rn(__dmul_rn(a.beta, (double)a.n), 1.0);
  uint32_t* bm = a.bitmap + b * a.words;
  double best_d2 = INFINITY;   // this thread's closest point of S so far, by (distance, id)
  long long best_id = -1;
  int trees = 0, stop = 0;
  unsigned long long cnt = 0;
  for (int i = 0; i < a.L; ++i) {
    unsigned long long added = 0;
    for (int64_t leaf = a.leaf_base[i] + threadIdx.x; leaf < a.leaf_base[i + 1]; leaf += RT) {
      // Alg. 4's bounds of the leaf box; the outermost edges are -inf / +inf
      double lb2 = 0.0, ub2 = 0.0;
      for (int j = 0; j < K; ++j) {
        const int h = i * K + j;
        const double x = s_qp[h];
        const int lo = a.leaf_lo[leaf * K + j], hi = a.leaf_hi[leaf * K + j];
        const double el = lo > 0 ? (double)a.E[(int64_t)h * (a.Nr + 1) + lo] : -INFINITY;
        const double eh = hi < a.Nr - 1 ? (double)a.E[(int64_t)h * (a.Nr + 1) + hi + 1] : INFINITY;
        const double delta = fmax(fmax(__dsub_rn(el, x), __dsub_rn(x, eh)), 0.0);
        const double far = fmax(fabs(__dsub_rn(x, el)), fabs(__dsub_rn(x, eh)));
        lb2 = __dadd_rn(lb2, __dmul_rn(delta, delta));
        ub2 = __dadd_rn(ub2, __dmul_rn(far, far));
      }
      if (lb2 > rp2) continue;
      const bool whole = ub2 <= rp2;
      const uint32_t st = a.leaf_range[2 * leaf], count = a.leaf_range[2 * leaf + 1];
      const uint32_t* ids = a.leaf_ids + (int64_t)i * a.n + st;
      for (uint32_t e = 0; e < count; ++e) {
        const uint32_t id = ids[e];
        if (!whole) {
          double d2 = 0.0;
          for (int j = 0; j < K; ++j) {
            const int h = i * K + j;
            const double df = __dsub_rn(project_fp64(a.A, d, h, a.X, a.dtype, (int64_t)id * d), s_qp[h]);
            d2 = __dadd_rn(d2, __dmul_rn(df, df));
          }
          if (!(d2 <= rp2)) continue;
        }
        const uint32_t bit = 1u << (id & 31);
        if (atomicOr(bm + (id >> 5), bit) & bit) continue;   // already in S
        ++added;
        double dd = 0.0;
        for (int t = 0; t < d; ++t) {
          const double df = __dsub_rn(value_at(a.X, a.dtype, (int64_t)id * d + t), value_at(a.Q, a.dtype, qoff + t));
          dd = __dadd_rn(dd, __dmul_rn(df, df));
        }
        if (dd < best_d2 || (dd == best_d2 && (long long)id < best_id)) {
          best_d2 = dd;
          best_id = id;
        }
      }
    }
    if (added) atomicAdd(&s_cnt, added);
    __syncthreads();
    cnt = s_cnt;
    __syncthreads();   // every thread has read the count before the next tree adds to it
    trees = i + 1;
    if ((double)cnt >= bound) {
      stop = 1;
      break;
    }
  }
  // the closest point of S over the block, by (distance, id)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double od = __shfl_xor_sync(0xffffffffu, best_d2, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, best_id, o);
    if (od < best_d2 || (od == best_d2 && oi >= 0 && (best_id < 0 || oi < best_id))) {
      best_d2 = od;
      best_id = oi;
    }
  }
  if (lane == 0) {
    s_bd[w] = best_d2;
    s_bi[w] = best_id;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bd = s_bd[0];
    long long bi = s_bi[0];
    for (int q = 1; q < RT / 32; ++q)
      if (s_bd[q] < bd || (s_bd[q] == bd && s_bi[q] >= 0 && (bi < 0 || s_bi[q] < bi))) {
        bd = s_bd[q];
        bi = s_bi[q];
      }
    double dist = INFINITY;
    long long id = -1;
    if (cnt > 0) {
      const double dd = sqrt(bd);
      if (stop == 1 || dd <= __dmul_rn((double)a.c[b], rr)) {
        dist = dd;
        id = bi;
        if (stop != 1) stop = 2;
      }
    }
    a.out_id[b] = id;
    a.out_dist[b] = dist;
    a.out_stats[3 * b + 0] = (int32_t)cnt;
    a.out_stats[3 * b + 1] = trees;
    a.out_stats[3 * b + 2] = stop;
  }
}

}  // namespace
}  // namespace detlsh

using namespace detlsh;

extern "C" int detlsh_rc_ann(const detlsh_index* idx, const void* Q, int64_t nq, int32_t dtype, const float* r,
                             const float* c, double eps, double beta, int64_t* out_id, double* out_dist,
                             int32_t* out_stats, void* stream) {
  clear_error();
  DL_REQUIRE(idx, "NULL index");
  DL_REQUIRE(nq >= 0, "nq must be >= 0");
  if (nq == 0) return DETLSH_OK;
  DL_REQUIRE(Q && r && c && out_id && out_dist && out_stats, "NULL argument");
  DL_REQUIRE(dtype == idx->dtype, "the queries must have the index's dtype");
  DL_REQUIRE(eps > 0.0 && std::isfinite(eps), "eps must be positive and finite");
  DL_REQUIRE(beta >= 0.0 && std::isfinite(beta), "beta must be >= 0 and finite");
  DL_TRY(require_device_ptr(Q, "Q"));
  DL_TRY(require_device_ptr(r, "r"));
  DL_TRY(require_device_ptr(c, "c"));
  DL_TRY(require_device_ptr(out_id, "out_id"));
  DL_TRY(require_device_ptr(out_dist, "out_dist"));
  DL_TRY(require_device_ptr(out_stats, "out_stats"));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RcArgs a{};
  a.X = idx->X;
  a.dtype = idx->dtype;
  a.n = idx->n;
  a.d = (int)idx->d;
  a.A = idx->A;
  a.E = idx->E;
  a.K = idx->K;
  a.L = idx->L;
  a.Nr = idx->Nr;
  a.leaf_ids = idx->leaf_ids;
  a.leaf_range = idx->leaf_range;
  a.leaf_lo = idx->leaf_lo;
  a.leaf_hi = idx->leaf_hi;
  a.leaf_base = idx->leaf_base;
  a.Q = Q;
  a.r = r;
  a.c = c;
  a.eps = eps;
  a.beta = beta;
  a.words = (idx->n + 31) / 32;
  a.out_id = out_id;
  a.out_dist = out_dist;
  a.out_stats = out_stats;
  Scratch bm;
  DL_TRY(bm.alloc(sizeof(uint32_t) * nq * a.words, s));
  DL_CUDA(cudaMemsetAsync(bm.p, 0, sizeof(uint32_t) * nq * a.words, s));
  a.bitmap = bm.as<uint32_t>();
  const size_t smem = sizeof(double) * (size_t)idx->K * idx->L;
  k_rc_ann<<<(unsigned)nq, RT, smem, s>>>(a);
  DL_LAUNCH();
  return DETLSH_OK;
}
