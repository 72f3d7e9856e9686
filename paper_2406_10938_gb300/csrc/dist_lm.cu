// Coarse candidate distances by leaf on the tensor cores (BF16 operands, FP32
// accumulation in tensor memory), for the shortlist mode of the query.
//
// The walk of Alg. 7 adds whole leaves to a query's candidate set S, so the
// candidates of a batch are, leaf by leaf, the same rows of X for every query
// that activated the leaf. Instead of gathering one row per (query,
// candidate) pair, the walk records each run of new points it adds (leaf,
// offset in the leaf, list position, mask of the new points) and the records
// of the batch are grouped by leaf chunk (NMAX - 32 points: a run of at most
// 32 points that starts in a chunk lies inside the NMAX-point tile at the
// chunk's start) and, inside a chunk, by the 32-point window the run starts
// in. NMAX is 64 for indexes of small leaves, else 128 (chosen at build).
// A persistent kernel then takes (chunk, up to 128 records) units:
//   last 4     stage each unit's metadata (query rows, point ids, list
//              positions, masks, norms) into a ring of eight slots, four
//              units' loads in flight at once;
//   warps 4.. (one per stage slot) copy the records' BF16 query rows (A,
//              M = 128) and the chunk's BF16 point rows (B, N <= NMAX) into
//              shared memory, eight 16-byte loads per lane in flight, 64
//              coordinates (128 bytes) of d per stage, in the 128-byte
//              swizzled K-major layout, all slots filling at once;
//   next warp  issues tcgen05.mma (kind::f16, BF16) into one of 512/NMAX
//              TMEM accumulators, q . o for every (record, point) pair;
//   warps 0-7  (two groups of four taking alternate units) read the
//              accumulator (one record per TMEM lane; only the columns the
//              warp's records cover), form ||q||^2 + ||o||^2 - 2 q.o for each
//              record's new points, stage them in shared memory and write
//              every record's run to its list positions with one coalesced
//              store.
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
constexpr int LM_KB = 64;           // coordinates per stage (128-byte rows)
constexpr int LM_META = 8;          // units staged ahead (metadata ring)
constexpr int LM_SUB = 8;           // sort keys per chunk: its 32-point windows
constexpr int LM_EPI_WARPS = 4;     // an epilogue group: four warps, one per TMEM lane quadrant
constexpr int LM_EPI_GROUPS = 2;    // warps 0-3 take the even units, warps 4-7 the odd ones
constexpr int LM_PROD_WARP = LM_EPI_WARPS * LM_EPI_GROUPS;   // then one producer warp per stage slot
constexpr int LM_PF_WARPS = 4;      // prefetch warps (after the MMA warp)
constexpr int LM_ILP = 8;           // 16-byte loads per lane in flight
constexpr uint32_t LM_ABYTES = LM_M * 128;
constexpr int LM_TMEM_COLS = 512;
constexpr int LM_STAGE_BUDGET = 144 * 1024;   // shared memory of the stage ring
constexpr int LM_STG = 33;          // staging row of the epilogue (32 values, padded)
constexpr unsigned long long LM_DRAIN_NS = 2000000000ull;

// Shapes of one tile width: stages and TMEM accumulators that fit.
template <int NMAX>
struct LmShape {
  static constexpr uint32_t BBYTES = NMAX * 128;
  static constexpr int STAGES = LM_STAGE_BUDGET / (LM_ABYTES + BBYTES);
  static constexpr int ACC = LM_TMEM_COLS / NMAX;
  static constexpr int MMA_WARP = LM_PROD_WARP + STAGES;   // lane 0 issues; the warp owns the TMEM
  static constexpr int PF_WARP = MMA_WARP + 1;
  static constexpr int THREADS = 32 * (PF_WARP + LM_PF_WARPS);
};

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
// the thread's completed generic-proxy writes become visible to the tensor cores
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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

// Per-unit data staged by the prefetch warps for the producer (query ids,
// point ids) and the epilogue (everything else): one slot of a ring.
template <int NMAX>
struct LmMeta {
  uint32_t n, rc, pad0, pad1;
  uint32_t qb[LM_M];      // query (row of the batch) of each record
  uint32_t pos[LM_M];     // list position of the record's first new point
  uint32_t mask[LM_M];    // its new points
  int32_t srel[LM_M];     // offset of its first point in the tile
  float qn[LM_M];         // ||q||^2
  uint32_t id[NMAX];      // the tile's points
  float on[NMAX];         // ||o||^2
};

template <int NMAX>
constexpr size_t lm_smem() {
  using S = LmShape<NMAX>;
  return 1024 + (size_t)S::STAGES * (LM_ABYTES + S::BBYTES) + LM_META * sizeof(LmMeta<NMAX>) +
         sizeof(float) * LM_PROD_WARP * 32 * LM_STG + (2 * S::STAGES + 2 * S::ACC + 2 * LM_META + 2) * 8;
}

template <int NMAX>
__global__ void __launch_bounds__(LmShape<NMAX>::THREADS, 1) k_dist_lm(LmArgs a) {
  using Sh = LmShape<NMAX>;
  constexpr int S = Sh::STAGES, ACC = Sh::ACC, LM_MMA_WARP = Sh::MMA_WARP, LM_PF_WARP = Sh::PF_WARP;
  constexpr uint32_t BBYTES = Sh::BBYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sA = base;                                   // [S][LM_ABYTES]
  uint8_t* sB = sA + S * LM_ABYTES;                     // [S][BBYTES]
  LmMeta<NMAX>* meta = reinterpret_cast<LmMeta<NMAX>*>(sB + S * BBYTES);   // [LM_META]
  float* stg = reinterpret_cast<float*>(meta + LM_META);                   // [8 warps][32][LM_STG]
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + LM_PROD_WARP * 32 * LM_STG);
  // full[0..S), empty[S..2S), acc full [2S..2S+ACC), acc empty [2S+ACC..2S+2ACC),
  // meta full [..+MR), meta empty [..+MR), drain, TMEM word
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + ACC;
  uint64_t* mfull = acce + ACC;
  uint64_t* mempty = mfull + LM_META;
  const uint32_t drain_bar = smem_u32(mempty + LM_META);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mempty + LM_META + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t nunits = *a.nunits;
  const int nkb = (a.d + LM_KB - 1) / LM_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bars[s]), 32);
      mbar_init(smem_u32(&bars[S + s]), 1);
    }
    for (int b = 0; b < ACC; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), LM_EPI_WARPS);
    }
    for (int m = 0; m < LM_META; ++m) {
      mbar_init(smem_u32(&mfull[m]), 32);
      mbar_init(smem_u32(&mempty[m]), LM_EPI_WARPS);
    }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == LM_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(LM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= LM_PF_WARP) {
    // ---- prefetch: warp p stages units lu = p, p + LM_PF_WARPS, ... into
    // meta slot lu % LM_META (loads of several units in flight at once)
    const uint32_t p = warp - LM_PF_WARP;
    for (uint32_t lu = p, u = blockIdx.x + p * gridDim.x; u < nunits;
         lu += LM_PF_WARPS, u += LM_PF_WARPS * gridDim.x) {
      const uint32_t m = lu % LM_META, r = lu / LM_META;
      const bool got = mbar_wait(smem_u32(&mempty[m]), (r & 1) ^ 1, a.err, a.wait_ns);
      if (!__all_sync(0xffffffffu, got)) break;
      LmMeta<NMAX>& M = meta[m];
      const uint4 U = a.units[u];
      const uint32_t rc = U.w & 0xffffu, N = U.w >> 16;
      const uint32_t* lids = a.leaf_ids + (int64_t)a.leaf_tree[U.x] * a.n + a.leaf_range[2 * (int64_t)U.x] + U.y;
      uint4 R[LM_M / 32];
      uint32_t q[LM_M / 32], id[NMAX / 32];
#pragma unroll
      for (int i = 0; i < LM_M / 32; ++i) {
        const uint32_t row = lane + 32 * i;
        R[i] = row < rc ? a.srec[U.z + row] : make_uint4(0u, U.y, 0u, 0u);
        q[i] = row < rc ? a.sq[U.z + row] : 0u;
      }
#pragma unroll
      for (int i = 0; i < NMAX / 32; ++i) {
        const uint32_t j = lane + 32 * i;
        id[i] = j < N ? lids[j] : 0u;
        if (!DL_CHECK(id[i] < a.n, 50, id[i])) id[i] = 0u;
      }
#pragma unroll
      for (int i = 0; i < LM_M / 32; ++i) {
        const uint32_t row = lane + 32 * i;
        M.qb[row] = q[i];
        M.pos[row] = R[i].z;
        M.mask[row] = R[i].w;
        M.srel[row] = (int32_t)(R[i].y - U.y);
        M.qn[row] = row < rc ? a.qn[q[i]] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < NMAX / 32; ++i) {
        const uint32_t j = lane + 32 * i;
        M.id[j] = id[i];
        M.on[j] = j < N ? a.xn2[id[i]] : 0.f;
      }
      if (lane == 0) {
        M.n = N;
        M.rc = rc;
      }
      __syncwarp();
      mbar_arrive(smem_u32(&mfull[m]));
    }
  } else if (warp >= LM_PROD_WARP && warp < LM_MMA_WARP) {
    // ---- producers: warp w fills the stages it = w, w + S, ... (slot w):
    // the records' BF16 query rows (A) and the tile's BF16 point rows (B),
    // LM_ILP 16-byte loads per lane in flight, stored into the 128-byte
    // swizzled K-major layout; rows past rc and points past N feed outputs
    // nobody reads and are left as they are, coordinates past d are zeros
    const uint32_t w = warp - LM_PROD_WARP;
    const uint32_t sa = smem_u32(sA + w * LM_ABYTES), sb = smem_u32(sB + w * BBYTES);
    for (uint32_t it = w, r = 0;; it += S, ++r) {
      const uint32_t lu = it / nkb, u = blockIdx.x + lu * gridDim.x;
      if (u >= nunits) break;
      const int x = (int)(it % nkb) * LM_KB;
      const uint32_t m = lu % LM_META;
      bool got = mbar_wait(smem_u32(&mfull[m]), (lu / LM_META) & 1, a.err, a.wait_ns);
      got = got && mbar_wait(smem_u32(&bars[S + w]), (r & 1) ^ 1, a.err, a.wait_ns);
      if (!__all_sync(0xffffffffu, got)) break;
      const LmMeta<NMAX>& M = meta[m];
      const uint32_t rc = M.rc, nitems = (rc + M.n) * 8;
      for (uint32_t b0 = 0; b0 < nitems; b0 += 32 * LM_ILP) {
        uint4 v[LM_ILP];
        uint32_t dst[LM_ILP];
#pragma unroll
        for (int k = 0; k < LM_ILP; ++k) {
          const uint32_t item = b0 + k * 32 + lane;
          dst[k] = 0xffffffffu;
          v[k] = make_uint4(0u, 0u, 0u, 0u);
          if (item < nitems) {
            const uint32_t row = item >> 3, ch = item & 7;
            const int e = x + (int)ch * 8;
            const __nv_bfloat16* src;
            if (row < rc) {
              src = a.Qb + (int64_t)M.qb[row] * a.d + e;
              dst[k] = sa + row * 128 + ((ch ^ (row & 7)) << 4);
            } else {
              const uint32_t j = row - rc;
              src = a.Xb + (int64_t)M.id[j] * a.d + e;
              dst[k] = sb + j * 128 + ((ch ^ (j & 7)) << 4);
            }
            if (e < a.d) v[k] = __ldg(reinterpret_cast<const uint4*>(src));
          }
        }
#pragma unroll
        for (int k = 0; k < LM_ILP; ++k)
          if (dst[k] != 0xffffffffu)
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst[k]), "r"(v[k].x), "r"(v[k].y),
                         "r"(v[k].z), "r"(v[k].w)
                         : "memory");
      }
      // the stage's generic-proxy writes become visible to the tensor cores
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars[w]));
    }
  } else if (warp == LM_MMA_WARP && lane == 0) {
    // ---- MMA issuer
    uint32_t it = 0, lt = 0;
    bool ok = true;
    for (uint32_t u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++lt) {
      const uint32_t m = lt % LM_META;
      if (!mbar_wait(smem_u32(&mfull[m]), (lt / LM_META) & 1, a.err, a.wait_ns)) break;
      const uint32_t Np = (meta[m].n + 15u) & ~15u;
      const uint32_t idesc = (1u << 4)     // D: FP32
                             | (1u << 7)   // A: BF16
                             | (1u << 10)  // B: BF16
                             | ((Np >> 3) << 17) | ((uint32_t)(LM_M >> 4) << 24);
      const uint32_t ab = lt % ACC, use = lt / ACC;
      if (!mbar_wait(smem_u32(&acce[ab]), (use & 1) ^ 1, a.err, a.wait_ns)) break;
      tc_fence_after();
      const uint32_t dt = tmem + ab * NMAX;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const uint32_t s = it % S, r = it / S;
        if (!mbar_wait(smem_u32(&bars[s]), r & 1, a.err, a.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = smem_desc(smem_u32(sA + s * LM_ABYTES));
        const uint64_t bd = smem_desc(smem_u32(sB + s * BBYTES));
#pragma unroll
        for (int k = 0; k < LM_KB / 16; ++k)   // 16 BF16 = 32 bytes = 2 in descriptor units
          if (kb * LM_KB + k * 16 < a.d) mma_bf16(dt, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
        mma_commit(smem_u32(&bars[S + s]));
      }
      if (!ok) break;
      mma_commit(smem_u32(&accf[ab]));
    }
    // every MMA issued has completed before the TMEM is freed
    mma_commit(drain_bar);
    mbar_drain(drain_bar, 0);
  } else if (warp < LM_PROD_WARP) {
    // ---- epilogue: group g takes units lt = g, g + 2, ...; record (TMEM
    // lane) 32*q + lane of the tile, q = warp % 4; the warp reads only the
    // accumulator columns its records' runs cover
    const uint32_t g = warp / LM_EPI_WARPS, q = warp % LM_EPI_WARPS;
    const uint32_t row = q * 32 + (uint32_t)lane;
    float* mystg = stg + warp * 32 * LM_STG;
    float* my = mystg + lane * LM_STG;
    uint32_t lt = g;
    for (uint32_t u = blockIdx.x + g * gridDim.x; u < nunits; u += LM_EPI_GROUPS * gridDim.x, lt += LM_EPI_GROUPS) {
      const uint32_t ab = lt % ACC, use = lt / ACC, m = lt % LM_META;
      bool got = mbar_wait(smem_u32(&accf[ab]), use & 1, a.err, a.wait_ns);
      got = got && mbar_wait(smem_u32(&mfull[m]), (lt / LM_META) & 1, a.err, a.wait_ns);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const LmMeta<NMAX>& M = meta[m];
      const bool valid = row < M.rc;
      const uint32_t mask = valid ? M.mask[row] : 0u;
      const int srel = M.srel[row];
      const float qn = M.qn[row];
      // columns [lo, hi) of this warp's new points, in whole 32-column steps
      const int lo = __reduce_min_sync(0xffffffffu, mask ? srel + __ffs(mask) - 1 : 0x7fffffff);
      const int hi = __reduce_max_sync(0xffffffffu, mask ? srel + 32 - __clz(mask) : 0);
      for (int c0 = lo & ~31; c0 < hi; c0 += 32) {
        uint32_t v[32];
        tmem_ld16_issue(tmem + ((q * 32) << 16) + ab * NMAX + c0, v);
        tmem_ld16_issue(tmem + ((q * 32) << 16) + ab * NMAX + c0 + 16, v + 16);
        tmem_ld_wait();
        if (mask) {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int i = c0 + e - srel;
            if (i >= 0 && i < 32 && ((mask >> i) & 1u)) {
              const float dot = __uint_as_float(v[e]);
              my[__popc(mask & ((1u << i) - 1u))] =
                  fmaxf(__fsub_rn(__fadd_rn(qn, M.on[c0 + e]), __fmul_rn(2.f, dot)), 0.f);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      // the accumulator is free; each record's run goes out in one coalesced
      // store (record fields read from the metadata slot by every lane)
      if (lane == 0) mbar_arrive(smem_u32(&acce[ab]));
      const uint32_t nrow = min(32u, M.rc > q * 32 ? M.rc - q * 32 : 0u);
#pragma unroll 4
      for (uint32_t rr = 0; rr < nrow; ++rr) {
        const uint32_t mr = M.mask[q * 32 + rr];
        const uint64_t p = (uint64_t)M.pos[q * 32 + rr] + lane;
        if (lane < __popc(mr) && (int64_t)p < a.cap)
          a.d2[(int64_t)M.qb[q * 32 + rr] * a.cap + p] = mystg[rr * LM_STG + lane];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&mempty[m]));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == LM_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(LM_TMEM_COLS));
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

__global__ void k_chunk_counts(const uint32_t* __restrict__ leaf_range, int64_t TL, uint32_t chunk,
                               uint32_t* __restrict__ cnt) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l < TL) cnt[l] = (leaf_range[2 * l + 1] + chunk - 1) / chunk;
}

__global__ void k_chunk_leaf(const uint32_t* __restrict__ chunk_base, const uint32_t* __restrict__ cnt, int64_t TL,
                             uint32_t* __restrict__ chunk_leaf) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= TL) return;
  for (uint32_t c = 0; c < cnt[l]; ++c) chunk_leaf[chunk_base[l] + c] = (uint32_t)l;
}

// sort key of a record: its chunk, then the 32-point window of the chunk its
// run starts in (so that neighbouring records of a unit cover nearby columns)
__device__ __forceinline__ uint32_t rec_key(const uint32_t* chunk_base, uint4 R, uint32_t chunk) {
  return (chunk_base[R.x] + R.y / chunk) * LM_SUB + (R.y % chunk) / 32u;
}

// one CTA per query of the batch: its records' key counts
__global__ void k_rec_hist(const uint4* __restrict__ rec, int64_t cap, const uint32_t* __restrict__ meta,
                           int mq_words, int mq_nrec, const uint32_t* __restrict__ nqd,
                           const uint32_t* __restrict__ chunk_base, uint32_t chunk, uint32_t* __restrict__ khist) {
  const int64_t qb = blockIdx.x;
  if (qb >= (int64_t)*nqd) return;
  const int64_t nr = min((int64_t)meta[qb * mq_words + mq_nrec], cap);
  const uint4* r = rec + qb * cap;
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) {
    atomicAdd(&khist[rec_key(chunk_base, r[i], chunk)], 1u);
  }
}

__global__ void k_rec_scatter(const uint4* __restrict__ rec, int64_t cap, const uint32_t* __restrict__ meta,
                              int mq_words, int mq_nrec, const uint32_t* __restrict__ nqd,
                              const uint32_t* __restrict__ chunk_base, uint32_t chunk, const uint32_t* __restrict__ koff,
                              uint32_t* __restrict__ kcur, uint4* __restrict__ srec, uint32_t* __restrict__ sq) {
  const int64_t qb = blockIdx.x;
  if (qb >= (int64_t)*nqd) return;
  const int64_t nr = min((int64_t)meta[qb * mq_words + mq_nrec], cap);
  const uint4* r = rec + qb * cap;
  for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) {
    const uint4 R = r[i];
    const uint32_t key = rec_key(chunk_base, R, chunk);
    const uint32_t p = koff[key] + atomicAdd(&kcur[key], 1u);
    srec[p] = R;
    sq[p] = (uint32_t)qb;
  }
}

// records of chunk k: koff[k*LM_SUB] .. koff[(k+1)*LM_SUB] (koff holds the
// total at its end)
__global__ void k_unit_counts(const uint32_t* __restrict__ koff, int64_t NK, uint32_t* __restrict__ ucnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NK) ucnt[k] = (koff[(k + 1) * LM_SUB] - koff[k * LM_SUB] + LM_M - 1) / LM_M;
}

__global__ void k_units(const uint32_t* __restrict__ koff, const uint32_t* __restrict__ uoff,
                        const uint32_t* __restrict__ chunk_base, const uint32_t* __restrict__ chunk_leaf,
                        const uint32_t* __restrict__ leaf_range, int64_t NK, uint32_t chunk, uint32_t nmax,
                        uint4* __restrict__ units) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NK) return;
  const uint32_t R = koff[(k + 1) * LM_SUB] - koff[k * LM_SUB];
  if (R == 0) return;
  const uint32_t leaf = chunk_leaf[k];
  const uint32_t c0 = (uint32_t)(k - chunk_base[leaf]) * chunk;
  const uint32_t N = min(nmax, leaf_range[2 * (int64_t)leaf + 1] - c0);
  for (uint32_t t = 0; t * LM_M < R; ++t)
    units[uoff[k] + t] =
        make_uint4(leaf, c0, koff[k * LM_SUB] + t * LM_M, min((uint32_t)LM_M, R - t * LM_M) | (N << 16));
}

template <int NMAX>
int launch_lm(const LmArgs& a, cudaStream_t s) {
  constexpr size_t smem = lm_smem<NMAX>();
  static_assert(smem <= 227 * 1024, "shared memory of k_dist_lm");
  DL_CUDA(cudaFuncSetAttribute(k_dist_lm<NMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  k_dist_lm<NMAX><<<(unsigned)nsm, LmShape<NMAX>::THREADS, smem, s>>>(a);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace

int64_t lm_sort_keys(int64_t n_chunks) { return n_chunks * LM_SUB; }

int build_lm_tables(detlsh_index* idx, cudaStream_t s) {
  const int64_t TL = idx->total_leaves;
  // 64-point tiles (six stages, eight accumulators) when the leaves are small
  // on average, else 128-point tiles (four stages, four accumulators)
  idx->lm_nmax = (idx->n * idx->L) <= 48 * TL ? 64 : 128;
  const uint32_t chunk = (uint32_t)idx->lm_nmax - 32;
  DL_TRY(index_alloc(&idx->xn2, sizeof(float) * idx->n, s));
  k_rownorm_bf16<<<152 * 8, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(idx->Xb), idx->n, nullptr, idx->d,
                                         idx->xn2);
  DL_LAUNCH();
  Scratch cnt, tot;
  DL_TRY(cnt.alloc(sizeof(uint32_t) * TL, s));
  DL_TRY(tot.alloc(sizeof(uint32_t), s));
  DL_TRY(index_alloc(&idx->chunk_base, sizeof(uint32_t) * (TL + 1), s));
  k_chunk_counts<<<ceil_div(TL, 256), 256, 0, s>>>(idx->leaf_range, TL, chunk, cnt.as<uint32_t>());
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
  const uint32_t nmax = (uint32_t)idx->lm_nmax, chunk = nmax - 32;
  // the batch's query norms (BF16 rows, as the MMA sees them)
  k_rownorm_bf16<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(b.nqg * 32, 256), 152 * 8)), 256, 0, s>>>(
      static_cast<const __nv_bfloat16*>(b.qb16), b.nqg, b.nqd, idx->d, b.qn);
  DL_LAUNCH();
  // records grouped by (chunk, window) (counting sort), then units of up to
  // 128 records of one chunk
  const int64_t NKS = NK * LM_SUB;
  DL_CUDA(cudaMemsetAsync(b.khist, 0, sizeof(uint32_t) * NKS, s));
  DL_CUDA(cudaMemsetAsync(b.kcur, 0, sizeof(uint32_t) * NKS, s));
  k_rec_hist<<<(unsigned)b.nqg, 256, 0, s>>>(b.rec, b.cap, b.meta, b.mq_words, b.mq_nrec, b.nqd, idx->chunk_base,
                                             chunk, b.khist);
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32_ws(b.khist, b.koff, NKS, b.koff + NKS, b.scan_ws, b.scan_ws_bytes, s));
  k_rec_scatter<<<(unsigned)b.nqg, 256, 0, s>>>(b.rec, b.cap, b.meta, b.mq_words, b.mq_nrec, b.nqd, idx->chunk_base,
                                                chunk, b.koff, b.kcur, b.srec, b.sq);
  DL_LAUNCH();
  k_unit_counts<<<ceil_div(NK, 256), 256, 0, s>>>(b.koff, NK, b.ucnt);
  DL_LAUNCH();
  DL_TRY(exclusive_scan_u32_ws(b.ucnt, b.uoff, NK, b.nunits, b.scan_ws, b.scan_ws_bytes, s));
  k_units<<<ceil_div(NK, 256), 256, 0, s>>>(b.koff, b.uoff, idx->chunk_base, idx->chunk_leaf, idx->leaf_range, NK,
                                            chunk, nmax, b.units);
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
  return nmax == 64 ? launch_lm<64>(a, s) : launch_lm<128>(a, s);
}

}  // namespace detlsh
