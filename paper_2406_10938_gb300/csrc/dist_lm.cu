// Coarse candidate distances by leaf on the tensor cores (BF16 operands, FP32
// accumulation in tensor memory), for the shortlist mode of the query.
//
// The walk of Alg. 7 adds whole leaves to a query's candidate set S, so the
// candidates of a batch are, leaf by leaf, the same rows of X for every query
// that activated the leaf. Instead of gathering one row per (query,
// candidate) pair, the walk records each run of new points it adds (leaf,
// offset in the leaf, list position, mask of the new points) and the records
// of the batch are grouped by leaf chunk (224 points: with a run of at most
// 32 points, every run lies inside a 256-point tile starting at its chunk).
// A persistent kernel then takes (chunk, up to 128 records) units:
//   warps 4-7  stage the 128 records' BF16 query rows (A, M = 128) and the
//              chunk's BF16 point rows (B, N <= 256) into shared memory with
//              cp.async, 64 coordinates (128 bytes) of d per stage, in the
//              128-byte swizzled K-major layout, four stages;
//   warp 8     issues tcgen05.mma (kind::f16, BF16) into one of two TMEM
//              accumulators, q . o for every (record, point) pair of the tile;
//   warps 0-3  read the accumulator (one record per TMEM lane) and write
//              ||q||^2 + ||o||^2 - 2 q.o for the record's new points to their
//              list positions.
// Each leaf's rows are read once per 128 queries that share it instead of
// once per query. ||o||^2 (the BF16 row) is kept with the index, ||q||^2 per
// batch. Every mbarrier wait is bounded; a wait that runs out sets the
// index's error word and the roles wind down (copies waited for, MMAs
// completed) before the tensor memory is freed.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace detlsh {
namespace {

constexpr int LM_M = 128;           // records per tile (MMA M)
constexpr int LM_NMAX = 256;        // points per tile (MMA N at most)
constexpr int LM_KB = 64;           // coordinates per stage (128-byte rows)
constexpr int LM_STAGES = 4;
constexpr int LM_EPI_WARPS = 4;     // warps 0-3, one per TMEM lane quadrant
constexpr int LM_PROD_THREADS = 128;  // warps 4-7
constexpr int LM_THREADS = 32 * LM_EPI_WARPS + LM_PROD_THREADS + 32;   // + warp 8: MMA
constexpr uint32_t LM_ABYTES = LM_M * 128;
constexpr uint32_t LM_BBYTES = LM_NMAX * 128;
constexpr unsigned long long LM_DRAIN_NS = 2000000000ull;
constexpr size_t LM_SMEM = 1024 + LM_STAGES * (LM_ABYTES + LM_BBYTES) + (2 * LM_STAGES + 8) * 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false (and *err set) when it runs out or another role failed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (limit_ns == 0 || globaltimer() - t0 > limit_ns || *(volatile int*)err) {
      atomicExch(err, 1);
      return false;
    }
  }
}
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (globaltimer() - t0 <= LM_DRAIN_NS)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// K-major tile of 128-byte rows, 128-byte swizzle (8-row groups 1024 bytes apart)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 16-byte asynchronous copy; src_bytes 0 fills the destination with zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// the thread's completed generic-proxy writes become visible to the tensor cores
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct LmArgs {
  const __nv_bfloat16* Xb;   // [n][d]
  const float* xn2;          // [n] squared norms of the BF16 rows
  const __nv_bfloat16* Qb;   // [B][d] the batch's queries in BF16
  const float* qn;           // [B] their squared norms
  int d;
  int64_t n;
  const uint32_t* leaf_ids;
  const uint32_t* leaf_range;
  const uint16_t* leaf_tree;
  const uint4* units;        // (leaf, first point, first record, records | points << 16)
  const uint32_t* nunits;
  const uint4* srec;         // records by chunk: (leaf, offset, list position, new-point mask)
  const uint32_t* sq;        // their queries
  float* d2;                 // [B][cap] coarse squared distances at list positions
  int64_t cap;
  int* err;
  unsigned long long wait_ns;
};

__global__ void __launch_bounds__(LM_THREADS, 1) k_dist_lm(LmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sA = base;                                   // [STAGES][LM_ABYTES]
  uint8_t* sB = sA + LM_STAGES * LM_ABYTES;             // [STAGES][LM_BBYTES]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + LM_STAGES * LM_BBYTES);
  // full[0..S), empty[S..2S), acc full [2S..2S+2), acc empty [2S+2..2S+4),
  // drain 2S+4, the TMEM address word at 2S+5
  const uint32_t drain_bar = smem_u32(&bars[2 * LM_STAGES + 4]);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * LM_STAGES + 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t nunits = *a.nunits;
  const int nkb = (a.d + LM_KB - 1) / LM_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < LM_STAGES; ++s) {
      mbar_init(smem_u32(&bars[s]), LM_PROD_THREADS);
      mbar_init(smem_u32(&bars[LM_STAGES + s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars[2 * LM_STAGES + b]), 1);
      mbar_init(smem_u32(&bars[2 * LM_STAGES + 2 + b]), LM_EPI_WARPS);
    }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * LM_NMAX));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= LM_EPI_WARPS && warp < 8) {
    // ---- producers: cp.async of the A (queries) and B (points) rows
    const uint32_t pt = threadIdx.x - 32 * LM_EPI_WARPS;
    uint32_t it = 0;
    int prev = -1;
    bool ok = true;
    for (uint32_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const uint4 U = a.units[u];
      const uint32_t rc = U.w & 0xffffu, N = U.w >> 16, Np = (N + 15u) & ~15u;
      const uint32_t* lids = a.leaf_ids + (int64_t)a.leaf_tree[U.x] * a.n + a.leaf_range[2 * (int64_t)U.x] + U.y;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const uint32_t s = it % LM_STAGES, r = it / LM_STAGES;
        if (!mbar_wait(smem_u32(&bars[LM_STAGES + s]), (r & 1) ^ 1, a.err, a.wait_ns)) {
          ok = false;
          break;
        }
        const uint32_t nch = (LM_M + Np) * 8;
        for (uint32_t c = pt; c < nch; c += LM_PROD_THREADS) {
          const uint32_t row = c >> 3, ch = c & 7;
          const int e = kb * LM_KB + (int)ch * 8;
          const __nv_bfloat16* src;
          uint32_t dst;
          bool valid;
          if (row < (uint32_t)LM_M) {
            valid = row < rc && e < a.d;
            const uint32_t q = valid ? a.sq[U.z + row] : 0u;
            src = a.Qb + (int64_t)q * a.d + (valid ? e : 0);
            dst = smem_u32(sA + s * LM_ABYTES + row * 128 + ((ch ^ (row & 7)) << 4));
          } else {
            const uint32_t j = row - LM_M;
            valid = j < N && e < a.d;
            const uint32_t id = valid ? lids[j] : 0u;
            src = a.Xb + (int64_t)id * a.d + (valid ? e : 0);
            dst = smem_u32(sB + s * LM_BBYTES + j * 128 + ((ch ^ (j & 7)) << 4));
          }
          cp_async16(dst, src, valid ? 16u : 0u);
        }
        cp_async_commit();
        if (prev >= 0) {
          // the previous stage's copies have landed: publish it
          cp_async_wait<1>();
          fence_proxy_async();
          mbar_arrive(smem_u32(&bars[prev]));
        }
        prev = (int)s;
      }
    }
    cp_async_wait<0>();
    if (prev >= 0) {
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars[prev]));
    }
  } else if (warp == 8 && lane == 0) {
    // ---- MMA issuer
    uint32_t it = 0, lt = 0;
    bool ok = true;
    for (uint32_t u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++lt) {
      const uint32_t N = a.units[u].w >> 16, Np = (N + 15u) & ~15u;
      const uint32_t idesc = (1u << 4)     // D: FP32
                             | (1u << 7)   // A: BF16
                             | (1u << 10)  // B: BF16
                             | ((Np >> 3) << 17) | ((uint32_t)(LM_M >> 4) << 24);
      const uint32_t ab = lt & 1, use = lt >> 1;
      if (!mbar_wait(smem_u32(&bars[2 * LM_STAGES + 2 + ab]), (use & 1) ^ 1, a.err, a.wait_ns)) break;
      tc_fence_after();
      const uint32_t dt = tmem + ab * LM_NMAX;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const uint32_t s = it % LM_STAGES, r = it / LM_STAGES;
        if (!mbar_wait(smem_u32(&bars[s]), r & 1, a.err, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = smem_desc(smem_u32(sA + s * LM_ABYTES));
        const uint64_t bd = smem_desc(smem_u32(sB + s * LM_BBYTES));
#pragma unroll
        for (int k = 0; k < LM_KB / 16; ++k)   // 16 BF16 = 32 bytes = 2 in descriptor units
          if (kb * LM_KB + k * 16 < a.d) mma_bf16(dt, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
        mma_commit(smem_u32(&bars[LM_STAGES + s]));
      }
      if (!ok) break;
      mma_commit(smem_u32(&bars[2 * LM_STAGES + ab]));
    }
    // every MMA issued has completed before the TMEM is freed
    mma_commit(drain_bar);
    mbar_drain(drain_bar, 0);
  } else if (warp < LM_EPI_WARPS) {
    // ---- epilogue: record (TMEM lane) 32*warp + lane of the tile
    uint32_t lt = 0;
    const uint32_t row = (uint32_t)(warp * 32 + lane);
    for (uint32_t u = blockIdx.x; u < nunits; u += gridDim.x, ++lt) {
      const uint32_t ab = lt & 1, use = lt >> 1;
      const bool got = mbar_wait(smem_u32(&bars[2 * LM_STAGES + ab]), use & 1, a.err, a.wait_ns);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const uint4 U = a.units[u];
      const uint32_t rc = U.w & 0xffffu, N = U.w >> 16, Np = (N + 15u) & ~15u;
      const bool valid = row < rc;
      uint4 R = make_uint4(0u, 0u, 0u, 0u);
      uint32_t qb = 0;
      float qn = 0.f;
      if (valid) {
        R = a.srec[U.z + row];
        qb = a.sq[U.z + row];
        qn = a.qn[qb];
      }
      const int srel = (int)(R.y - U.y);
      const uint32_t* lids = a.leaf_ids + (int64_t)a.leaf_tree[U.x] * a.n + a.leaf_range[2 * (int64_t)U.x] + U.y;
      float* out = a.d2 + (int64_t)qb * a.cap;
      for (uint32_t cc = 0; cc < Np; cc += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + ab * LM_NMAX + cc, v);
        if (valid) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int i = (int)cc + e - srel;
            if (i >= 0 && i < 32 && ((R.w >> i) & 1u)) {
              const uint32_t id = lids[cc + e];
              const float d2 = fmaxf(__fsub_rn(__fadd_rn(qn, a.xn2[id]), __fmul_rn(2.f, v[e])), 0.f);
              const uint64_t p = (uint64_t)R.z + __popc(R.w & ((1u << i) - 1u));
              if ((int64_t)p < a.cap) out[p] = d2;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars[2 * LM_STAGES + 2 + ab]));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * LM_NMAX));
}

// Squared norm of each BF16 row in FP32: lane-strided partial sums, then a
// fixed butterfly (one warp per row).
__global__ void k_rownorm_bf16(const __nv_bfloat16* __restrict__ X, int64_t rows, const uint32_t* __restrict__ nrows,
                               int d, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nr = nrows ? (int64_t)*nrows : rows;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nr;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const __nv_bfloat16* x = X + r * d;
    float acc = 0.f;
    for (int t = lane; t < d; t += 32) {
      const float v = __bfloat162float(x[t]);
      acc = __fadd_rn(acc, __fmul_rn(v, v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) out[r] = acc;
  }
}

__global__ void k_chunk_counts(const uint32_t* __restrict__ leaf_range, int64_t TL, uint32_t* __restrict__ cnt) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l < TL) cnt[l] = (leaf_range[2 * l + 1] + kLmChunk - 1) / kLmChunk;
}

__global__ void k_chunk_leaf(const uint32_t* __restrict__ chunk_base, const uint32_t* __restrict__ cnt, int64_t TL,
                             uint32_t* __restrict__ chunk_leaf) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= TL) return;
  for (uint32_t c = 0; c < cnt[l]; ++c) chunk_leaf[chunk_base[l] + c] = (uint32_t)l;
}

// one CTA per query of the batch: its records' chunk counts
__global__ void k_rec_hist(const uint4* __restrict__ rec, int64_t cap, const uint32_t* __restrict__ meta,
                           int mq_words, int mq_nrec, const uint32_t* __restrict__ nqd,
                           const uint32_t* __restrict__ chunk_base, uint32_t* __restrict__ khist) {
  const int64_t qb = blockIdx.x;
  if (qb >= (int64_t)*nqd) return;
  const int64_t nr = min((int64_t)meta[qb * mq_words + mq_nrec], cap);
  const uint4* r = rec + qb * cap;
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) {
    const uint4 R = r[i];
    atomicAdd(&khist[chunk_base[R.x] + R.y / kLmChunk], 1u);
  }
}

__global__ void k_rec_scatter(const uint4* __restrict__ rec, int64_t cap, const uint32_t* __restrict__ meta,
                              int mq_words, int mq_nrec, const uint32_t* __restrict__ nqd,
                              const uint32_t* __restrict__ chunk_base, const uint32_t* __restrict__ koff,
                              uint32_t* __restrict__ kcur, uint4* __restrict__ srec, uint32_t* __restrict__ sq) {
  const int64_t qb = blockIdx.x;
  if (qb >= (int64_t)*nqd) return;
  const int64_t nr = min((int64_t)meta[qb * mq_words + mq_nrec], cap);
  const uint4* r = rec + qb * cap;
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) {
    const uint4 R = r[i];
    const uint32_t key = chunk_base[R.x] + R.y / kLmChunk;
    const uint32_t p = koff[key] + atomicAdd(&kcur[key], 1u);
    srec[p] = R;
    sq[p] = (uint32_t)qb;
  }
}

__global__ void k_unit_counts(const uint32_t* __restrict__ khist, int64_t NK, uint32_t* __restrict__ ucnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NK) ucnt[k] = (khist[k] + LM_M - 1) / LM_M;
}

__global__ void k_units(const uint32_t* __restrict__ khist, const uint32_t* __restrict__ koff,
                        const uint32_t* __restrict__ uoff, const uint32_t* __restrict__ chunk_base,
                        const uint32_t* __restrict__ chunk_leaf, const uint32_t* __restrict__ leaf_range, int64_t NK,
                        uint4* __restrict__ units) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NK) return;
  const uint32_t R = khist[k];
  if (R == 0) return;
  const uint32_t leaf = chunk_leaf[k];
  const uint32_t c0 = (uint32_t)(k - chunk_base[leaf]) * kLmChunk;
  const uint32_t N = min((uint32_t)LM_NMAX, leaf_range[2 * (int64_t)leaf + 1] - c0);
  for (uint32_t t = 0; t * LM_M < R; ++t)
    units[uoff[k] + t] = make_uint4(leaf, c0, koff[k] + t * LM_M, min((uint32_t)LM_M, R - t * LM_M) | (N << 16));
}

}  // namespace

size_t lm_smem_bytes() { return LM_SMEM; }

int build_lm_tables(detlsh_index* idx, cudaStream_t s) {
  const int64_t TL = idx->total_leaves;
  DL_TRY(index_alloc(&idx->xn2, sizeof(float) * idx->n, s));
  k_rownorm_bf16<<<152 * 8, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(idx->Xb), idx->n, nullptr, idx->d,
                                         idx->xn2);
  DL_LAUNCH();
  Scratch cnt, tot;
  DL_TRY(cnt.alloc(sizeof(uint32_t) * TL, s));
  DL_TRY(tot.alloc(sizeof(uint32_t), s));
  DL_TRY(index_alloc(&idx->chunk_base, sizeof(uint32_t) * (TL + 1), s));
  k_chunk_counts<<<ceil_div(TL, 256), 256, 0, s>>>(idx->leaf_range, TL, cnt.as<uint32_t>());
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32(cnt.as<uint32_t>(), idx->chunk_base, TL, idx->chunk_base + TL, s));
  uint32_t nk = 0;
  DL_CUDA(cudaMemcpyAsync(&nk, idx->chunk_base + TL, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaStreamSynchronize(s));
  idx->n_chunks = nk;
  DL_TRY(index_alloc(&idx->chunk_leaf, sizeof(uint32_t) * std::max<int64_t>(1, nk), s));
  k_chunk_leaf<<<ceil_div(TL, 256), 256, 0, s>>>(idx->chunk_base, cnt.as<uint32_t>(), TL, idx->chunk_leaf);
  DL_LAUNCH();
  return DETLSH_OK;
}

int enqueue_coarse_lm(const detlsh_index* idx, const LmBatch& b, cudaStream_t s) {
  const int64_t NK = idx->n_chunks;
  // the batch's query norms (BF16 rows, as the MMA sees them)
  k_rownorm_bf16<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(b.nqg * 32, 256), 152 * 8)), 256, 0, s>>>(
      static_cast<const __nv_bfloat16*>(b.qb16), b.nqg, b.nqd, idx->d, b.qn);
  DL_LAUNCH();
  // records grouped by chunk (counting sort), then units of up to 128 records
  DL_CUDA(cudaMemsetAsync(b.khist, 0, sizeof(uint32_t) * NK, s));
  DL_CUDA(cudaMemsetAsync(b.kcur, 0, sizeof(uint32_t) * NK, s));
  k_rec_hist<<<(unsigned)b.nqg, 256, 0, s>>>(b.rec, b.cap, b.meta, b.mq_words, b.mq_nrec, b.nqd, idx->chunk_base,
                                             b.khist);
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32_ws(b.khist, b.koff, NK, nullptr, b.scan_ws, b.scan_ws_bytes, s));
  k_rec_scatter<<<(unsigned)b.nqg, 256, 0, s>>>(b.rec, b.cap, b.meta, b.mq_words, b.mq_nrec, b.nqd, idx->chunk_base,
                                                b.koff, b.kcur, b.srec, b.sq);
  DL_LAUNCH();
  k_unit_counts<<<ceil_div(NK, 256), 256, 0, s>>>(b.khist, NK, b.ucnt);
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32_ws(b.ucnt, b.uoff, NK, b.nunits, b.scan_ws, b.scan_ws_bytes, s));
  k_units<<<ceil_div(NK, 256), 256, 0, s>>>(b.khist, b.koff, b.uoff, idx->chunk_base, idx->chunk_leaf,
                                            idx->leaf_range, NK, b.units);
  DL_LAUNCH();
  LmArgs a{};
  a.Xb = static_cast<const __nv_bfloat16*>(idx->Xb);
  a.xn2 = idx->xn2;
  a.Qb = static_cast<const __nv_bfloat16*>(b.qb16);
  a.qn = b.qn;
  a.d = idx->d;
  a.n = idx->n;
  a.leaf_ids = idx->leaf_ids;
  a.leaf_range = idx->leaf_range;
  a.leaf_tree = idx->leaf_tree;
  a.units = b.units;
  a.nunits = b.nunits;
  a.srec = b.srec;
  a.sq = b.sq;
  a.d2 = b.d2;
  a.cap = b.cap;
  a.err = idx->d_err;
  a.wait_ns = tc_wait_limit_ns();
  DL_CUDA(cudaFuncSetAttribute(k_dist_lm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LM_SMEM));
  int dev = 0, nsm = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  k_dist_lm<<<(unsigned)nsm, LM_THREADS, LM_SMEM, s>>>(a);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace detlsh
