// Eq. 1 projection on the 5th-generation tensor cores (BF16 inputs, FP32
// accumulation in tensor memory), fused with the Alg. 2 encoding.
//
// P = Xb * Abᵀ for a BF16 copy Xb [rows][d] of the points and the BF16 hash
// matrix Ab [N][d] (N = L*K padded to a multiple of 16, extra rows zero).
// Persistent CTAs, one per SM, 256 threads in four roles:
//   warp 0  TMA producer: 128-row tiles of Xb and the matching chunk of Ab,
//           64 elements (128 B) of d per stage, 128-byte swizzle, a ring of
//           stages guarded by full/empty mbarriers;
//   warp 1  MMA issuer (one thread): tcgen05.mma M=128, N, K=16 into one of
//           two TMEM accumulators, tcgen05.commit frees a stage / publishes
//           an accumulator;
//   warp 2  owns the TMEM allocation;
//   warps 4-7 epilogue: tcgen05.ld of the 128 x N accumulator (one row per
//           thread), then either the breakpoint search of Alg. 2 (shared
//           memory) and 16-byte code stores, or the FP32 projections.
// Every mbarrier wait is bounded by %globaltimer; a wait that runs out sets
// an error word (the host reports DETLSH_ETIMEOUT) and the roles wind down:
// the producer waits (bounded) for the copies it has issued to land and the
// MMA issuer for its MMAs to complete before the TMEM is freed and the CTA
// exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "common.cuh"

namespace detlsh {
namespace {

constexpr int TC_M = 128;          // rows (points) per tile
constexpr int TC_STAGES = 4;
constexpr int TC_EPI_WARPS = 16;     // 4 per TMEM lane quadrant, 16 accumulator columns each
constexpr int TC_THREADS = 128 + 32 * TC_EPI_WARPS;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // 2 s per wait
constexpr unsigned long long TC_DRAIN_NS = 2000000000ull;  // 2 s per wait while winding down

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
// Bounded wait for the phase of the given parity; false (and *err set) when
// it runs out after limit_ns (limit 0: at the first retry) or another role
// has set *err.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err,
                                          unsigned long long limit_ns) {
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
// Bounded wait used while winding down: ignores the error word.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (globaltimer() - t0 <= TC_DRAIN_NS)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major tile of 128-byte rows with the
// 128-byte swizzle (8-row groups 1024 bytes apart), tcgen05 format.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)(16u >> 4) << 16;                   // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                            // descriptor version
  d |= (uint64_t)2 << 61;                            // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
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
struct TcArgs {
  int64_t rows;
  int d, LK, K, Nr;
  const float* E;        // [LK][Nr+1] (encode mode)
  const uint8_t* Rtab;   // [LK][kRegionRow] region search tables (encode mode)
  const float* Rlo;      // [LK]
  const float* Rinv;     // [LK]
  uint8_t* codes;        // [L][rows][K] (encode mode)
  float* P;              // projections (store mode)
  int64_t p_so, p_sr;
  int* err;
  unsigned long long wait_ns;   // limit of each pipeline wait
};

// Pipeline stages: a TF32 or three-part stage holds more tiles than a BF16 one.
template <bool TF32, bool A3>
__host__ __device__ constexpr int tc_stages() {
  return (TF32 || A3) ? 3 : TC_STAGES;
}
// A tiles per stage: 1 (BF16), 2 (TF32: a_big, a_small), 3 (BF16, A in three parts)
template <bool TF32, bool A3>
__host__ __device__ constexpr int tc_aparts() {
  return TF32 ? 2 : (A3 ? 3 : 1);
}
// Shared memory bytes of k_project_tc below the breakpoints and tables.
// (A3 stages also hold the uint8 tile as loaded, TC_M rows of 64 bytes)
template <int N, bool TF32, bool A3>
__host__ __device__ constexpr size_t tc_tile_bytes() {
  return (size_t)tc_stages<TF32, A3>() * ((size_t)TC_M * 128 * (TF32 ? 2 : 1) + (A3 ? (size_t)TC_M * 64 : 0) +
                                          (size_t)N * 128 * tc_aparts<TF32, A3>()) +
         (3 * tc_stages<TF32, A3>() + 8) * 8;
}

// Four uint8 values (one word) to four BF16 values (two words), exactly:
// 2^23 + u is an FP32 value whose low byte is u, less 2^23 it is u itself,
// and an integer below 256 keeps its value in BF16's top 16 bits.
__device__ __forceinline__ void widen4(uint32_t w, uint32_t& lo, uint32_t& hi) {
  const float f0 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440)) - 8388608.f;
  const float f1 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7441)) - 8388608.f;
  const float f2 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7442)) - 8388608.f;
  const float f3 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7443)) - 8388608.f;
  lo = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
  hi = __byte_perm(__float_as_uint(f2), __float_as_uint(f3), 0x7632);
}

// TF32 mode: X is FP32 and each stage also holds x_small = x - x_big, where
// x_big keeps the top 10 mantissa bits (what a TF32 operand holds exactly);
// D = (x_big + x_small)(a_big + a_small) in four MMAs per K step, a_big /
// a_small the same split of A. x_small and a_small are held to 11 of their
// at most 13 significant bits, so each product is within about 2^-21 of
// |a x|; the tensor cores' FP32 accumulation adds its own rounding, which is
// why this path is used for d <= 256 only. Values with at most 11
// significant bits (the exact-arithmetic inputs) have x_small = 0 and give
// exact sums.
// A3 mode: uint8 X against A split into three BF16 parts a1 + a2 + a3 (about
// 24 significant bits, an FP32 value to within 2^-24 of itself): three MMAs
// per K step. The uint8 tile arrives by TMA as loaded (64 bytes of a row per
// stage) and warps 2-3 widen it to BF16 (exact) into the swizzled operand
// layout, so the points are read from HBM once, one byte per coordinate.
template <int N, bool ENCODE, bool TF32, bool A3>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_project_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmA,
             const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmA3, TcArgs a) {
  constexpr int S = tc_stages<TF32, A3>();
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  // (pointer arithmetic on the shared array, so that every access below stays
  // a shared-memory access rather than a generic one)
  uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr uint32_t XBYTES = TC_M * 128;
  constexpr uint32_t ABYTES = N * 128;
  constexpr int KC = TF32 ? 32 : 64;                  // d elements per stage (128-byte rows)
  uint8_t* sx = base;                                  // [STAGES][XBYTES]
  uint8_t* sa = sx + S * XBYTES;               // [STAGES][ABYTES]
  uint8_t* sxs = sa + S * ABYTES;              // [STAGES][XBYTES] x_small (TF32)
  uint8_t* sas = sxs + (TF32 ? S * XBYTES : 0);   // [STAGES][ABYTES] a_small (TF32) or a2 (A3)
  uint8_t* sa3 = sas + ((TF32 || A3) ? S * ABYTES : 0);   // [STAGES][ABYTES] a3 (A3)
  constexpr uint32_t XUBYTES = TC_M * 64;
  uint8_t* sxu = sa3 + (A3 ? S * ABYTES : 0);     // [STAGES][XUBYTES] uint8 tile (A3)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sxu + (A3 ? S * XUBYTES : 0));
  // full[0..S), empty[S..2S), tfull[2S..2S+2), tempty[2S+2..2S+4), split[2S+4..3S+4),
  // the TMEM address word at 3S+4, drain at 3S+5
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 4);
  const uint32_t drain_bar = smem_u32(&bars[3 * S + 5]);
  float* Es = reinterpret_cast<float*>(bars + 3 * S + 8);    // [LK][Nr] (ENCODE), e_z at [h][z]
  float* Slo = Es + a.LK * a.Nr;                                     // [LK]
  float* Sinv = Slo + a.LK;                                          // [LK]
  uint8_t* Ts = reinterpret_cast<uint8_t*>(Sinv + a.LK);             // [LK][kRegionRow]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (a.rows + TC_M - 1) / TC_M;
  const int nk = (a.d + KC - 1) / KC;
  int* err = a.err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[S + s]), 1);
      mbar_init(smem_u32(&bars[2 * S + 4 + s]), 2);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars[2 * S + b]), 1);
      mbar_init(smem_u32(&bars[2 * S + 2 + b]), TC_EPI_WARPS);
    }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (ENCODE) {
    for (int i = threadIdx.x; i < a.LK * a.Nr; i += TC_THREADS) {
      const int h = i / a.Nr, z = i % a.Nr;
      Es[i] = z > 0 ? a.E[(int64_t)h * (a.Nr + 1) + z] : 0.f;
    }
    for (int i = threadIdx.x; i < a.LK * kRegionRow / 4; i += TC_THREADS)
      reinterpret_cast<uint32_t*>(Ts)[i] = reinterpret_cast<const uint32_t*>(a.Rtab)[i];
    for (int h = threadIdx.x; h < a.LK; h += TC_THREADS) {
      Slo[h] = a.Rlo[h];
      Sinv[h] = a.Rinv[h];
    }
  }
  constexpr uint32_t TCOLS = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : 256;
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    uint32_t it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int kc = 0; kc < nk && ok; ++kc, ++it) {
        const uint32_t s = it % S, r = it / S;
        ok = mbar_wait(smem_u32(&bars[S + s]), (r & 1) ^ 1, err, a.wait_ns);
        if (!ok) break;
        const uint32_t full = smem_u32(&bars[s]);
        mbar_expect_tx(full, (A3 ? XUBYTES : XBYTES) + tc_aparts<TF32, A3>() * ABYTES);
        tma_load_2d(smem_u32(A3 ? sxu + s * XUBYTES : sx + s * XBYTES), &tmX, kc * KC, (int)(tile * TC_M), full);
        tma_load_2d(smem_u32(sa + s * ABYTES), &tmA, kc * KC, 0, full);
        if (TF32 || A3) tma_load_2d(smem_u32(sas + s * ABYTES), &tmA2, kc * KC, 0, full);
        if (A3) tma_load_2d(smem_u32(sa3 + s * ABYTES), &tmA3, kc * KC, 0, full);
      }
    }
    // `it` stages were issued; the last one of each stage must have landed
    // before the CTA exits (at once unless a wait ran out)
    for (uint32_t j = it > (uint32_t)S ? it - S : 0; j < it; ++j)
      mbar_drain(smem_u32(&bars[j % S]), (j / S) & 1);
  } else if (TF32 && (warp == 2 || warp == 3)) {
    // ---- split of each staged X tile into x_big (in place) and x_small
    const int t = threadIdx.x - 64;   // 0..63
    uint32_t it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int kc = 0; kc < nk && ok; ++kc, ++it) {
        const uint32_t s = it % S, r = it / S;
        ok = mbar_wait(smem_u32(&bars[s]), r & 1, err, a.wait_ns);
        if (!ok) break;
        float4* xv = reinterpret_cast<float4*>(sx + s * XBYTES);
        float4* xs = reinterpret_cast<float4*>(sxs + s * XBYTES);
#pragma unroll 4
        for (int i = t; i < (int)(XBYTES / 16); i += 64) {
          const float4 x = xv[i];
          const float4 b = make_float4(__uint_as_float(__float_as_uint(x.x) & 0xffffe000u),
                                       __uint_as_float(__float_as_uint(x.y) & 0xffffe000u),
                                       __uint_as_float(__float_as_uint(x.z) & 0xffffe000u),
                                       __uint_as_float(__float_as_uint(x.w) & 0xffffe000u));
          xv[i] = b;
          xs[i] = make_float4(x.x - b.x, x.y - b.y, x.z - b.z, x.w - b.w);
        }
        // generic-proxy writes become visible to the tensor cores' reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S + 4 + s]));
      }
    }
  } else if (A3 && (warp == 2 || warp == 3)) {
    // ---- widening of each staged uint8 tile into the BF16 operand tile:
    // 16 bytes of row r (elements 16j..16j+15 of the stage) become the 16-byte
    // chunks 2j and 2j+1 of the 128-byte row, each stored at chunk ^ (r % 8)
    // (the 128-byte swizzle)
    const int t = threadIdx.x - 64;   // 0..63
    uint32_t it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int kc = 0; kc < nk && ok; ++kc, ++it) {
        const uint32_t s = it % S, r = it / S;
        ok = mbar_wait(smem_u32(&bars[s]), r & 1, err, a.wait_ns);
        if (!ok) break;
        const uint4* src = reinterpret_cast<const uint4*>(sxu + s * XUBYTES);
        uint8_t* dst = sx + s * XBYTES;
#pragma unroll 4
        for (int i = t; i < TC_M * 4; i += 64) {
          const int row = i >> 2, j = i & 3;
          const uint4 u = src[i];
          uint4 lo, hi;
          widen4(u.x, lo.x, lo.y);
          widen4(u.y, lo.z, lo.w);
          widen4(u.z, hi.x, hi.y);
          widen4(u.w, hi.z, hi.w);
          uint8_t* drow = dst + row * 128;
          *reinterpret_cast<uint4*>(drow + (((2 * j) ^ (row & 7)) << 4)) = lo;
          *reinterpret_cast<uint4*>(drow + (((2 * j + 1) ^ (row & 7)) << 4)) = hi;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S + 4 + s]));
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t ab_fmt = TF32 ? 2u : 1u;   // operand format: BF16 (kind::f16) or TF32
    constexpr uint32_t idesc = (1u << 4)            // D: FP32
                               | (ab_fmt << 7)      // A
                               | (ab_fmt << 10)     // B
                               | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    uint32_t it = 0, lt = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
      const uint32_t ab = lt & 1, use = lt >> 1;
      ok = mbar_wait(smem_u32(&bars[2 * S + 2 + ab]), (use & 1) ^ 1, err, a.wait_ns);
      if (!ok) break;
      tc_fence_after();
      const uint32_t dt = tmem + ab * (TCOLS / 2);
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const uint32_t s = it % S, r = it / S;
        ok = mbar_wait(smem_u32(&bars[(TF32 || A3) ? 2 * S + 4 + s : s]), r & 1, err, a.wait_ns);
        if (!ok) break;
        tc_fence_after();
        const uint64_t ad = smem_desc(smem_u32(sx + s * XBYTES));
        const uint64_t bd = smem_desc(smem_u32(sa + s * ABYTES));
        if (TF32) {
          const uint64_t asd = smem_desc(smem_u32(sxs + s * XBYTES));
          const uint64_t bsd = smem_desc(smem_u32(sas + s * ABYTES));
#pragma unroll
          for (int k = 0; k < 4; ++k) {   // 8 TF32 = 32 bytes = 2 in descriptor units
            mma_tf32(dt, ad + 2 * k, bd + 2 * k, idesc, (kc > 0 || k > 0) ? 1u : 0u);
            mma_tf32(dt, ad + 2 * k, bsd + 2 * k, idesc, 1u);
            mma_tf32(dt, asd + 2 * k, bd + 2 * k, idesc, 1u);
            mma_tf32(dt, asd + 2 * k, bsd + 2 * k, idesc, 1u);
          }
        } else if (A3) {
          const uint64_t b2 = smem_desc(smem_u32(sas + s * ABYTES));
          const uint64_t b3 = smem_desc(smem_u32(sa3 + s * ABYTES));
#pragma unroll
          for (int k = 0; k < KC / 16; ++k) {   // 16 BF16 = 32 bytes = 2 in descriptor units
            mma_bf16(dt, ad + 2 * k, bd + 2 * k, idesc, (kc > 0 || k > 0) ? 1u : 0u);
            mma_bf16(dt, ad + 2 * k, b2 + 2 * k, idesc, 1u);
            mma_bf16(dt, ad + 2 * k, b3 + 2 * k, idesc, 1u);
          }
        } else {
#pragma unroll
          for (int k = 0; k < KC / 16; ++k)   // 16 BF16 = 32 bytes = 2 in descriptor units
            mma_bf16(dt, ad + 2 * k, bd + 2 * k, idesc, (kc > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(smem_u32(&bars[S + s]));
      }
      if (!ok) break;
      mma_commit(smem_u32(&bars[2 * S + ab]));
    }
    // every MMA issued has completed before the TMEM is freed
    mma_commit(drain_bar);
    mbar_drain(drain_bar, 0);
  } else if (warp >= 4) {
    // ---- epilogue: warp w reads TMEM lanes 32*(w%4).. (its quadrant's 32
    // points) and accumulator columns [16g, 16g+16), g = (w-4)/4; one point
    // and 16 projections (one DE-Tree when K = 16) per thread
    const int q = warp & 3, g = (warp - 4) >> 2;
    const int row = q * 32 + lane;
    const bool active = g * 16 < N;
    uint32_t lt = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      const uint32_t ab = lt & 1, use = lt >> 1;
      if (!mbar_wait(smem_u32(&bars[2 * S + ab]), use & 1, err, a.wait_ns)) break;
      tc_fence_after();
      float v[16];
      if (active) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + ab * (TCOLS / 2) + g * 16, v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars[2 * S + 2 + ab]));
      const int64_t p = tile * TC_M + row;
      if (!active || p >= a.rows) continue;
      if (ENCODE) {
        if (a.K == 16 && g * 16 + 16 <= a.LK) {
          uint32_t wv[4];
          region_codes16(Es + g * 16 * a.Nr, a.Nr, Ts + g * 16 * kRegionRow, Slo + g * 16, Sinv + g * 16, v, wv);
          *reinterpret_cast<uint4*>(a.codes + ((int64_t)g * a.rows + p) * 16) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int h = g * 16 + c;
            if (h < a.LK) {
              const int tree = h / a.K, j = h % a.K;
              a.codes[((int64_t)tree * a.rows + p) * a.K + j] =
                  (uint8_t)region_fast(Es + h * a.Nr, Ts + h * kRegionRow, Slo[h], Sinv[h], v[c]);
            }
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int h = g * 16 + c;
          if (h < a.LK) a.P[p * a.p_so + (int64_t)h * a.p_sr] = v[c];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

__global__ void k_to_bf16_f32(const float* __restrict__ x, int64_t count, __nv_bfloat16* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}
__global__ void k_to_bf16_u8(const uint8_t* __restrict__ x, int64_t count, __nv_bfloat16* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn((float)x[i]);
}
// rows of a BF16 matrix gathered by id (the sample)
__global__ void k_gather_rows_bf16(const __nv_bfloat16* __restrict__ x, int d, const int64_t* __restrict__ ids,
                                   int64_t m, __nv_bfloat16* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m * d;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / d, c = i % d;
    y[i] = x[ids[r] * d + c];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

enum MapKind { MAP_BF16, MAP_F32, MAP_U8 };
// 2-D map of a row-major [rows][d] matrix: BF16 or FP32 in boxes of box_rows
// rows by 128 bytes with the 128-byte swizzle, or uint8 in boxes of box_rows
// rows by 64 bytes, unswizzled (widened in the kernel)
int make_map(CUtensorMap* tm, const void* ptr, int64_t rows, int d, int box_rows, MapKind kind = MAP_BF16) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return DETLSH_ECUDA;
  }
  const int esz = kind == MAP_F32 ? 4 : kind == MAP_BF16 ? 2 : 1;
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)d * esz};
  cuuint32_t box[2] = {(cuuint32_t)(kind == MAP_U8 ? 64 : 128 / esz), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapDataType dt = kind == MAP_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : kind == MAP_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const CUresult r = fn(tm, dt, 2, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        kind == MAP_U8 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DETLSH_ECUDA;
  }
  return DETLSH_OK;
}

template <int N, bool ENCODE, bool TF32, bool A3>
int launch_tc(const CUtensorMap& tx, const CUtensorMap& ta, const CUtensorMap& ta2, const CUtensorMap& ta3,
              const TcArgs& args, cudaStream_t s) {
  size_t smem = 1024 + tc_tile_bytes<N, TF32, A3>();
  if (ENCODE) smem += sizeof(float) * ((size_t)args.LK * args.Nr + 2 * args.LK) + (size_t)args.LK * kRegionRow;
  auto kern = k_project_tc<N, ENCODE, TF32, A3>;
  DL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0;
  DL_CUDA(cudaGetDevice(&dev));
  DL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntiles = (args.rows + TC_M - 1) / TC_M;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, nsm));
  kern<<<grid, TC_THREADS, smem, s>>>(tx, ta, ta2, ta3, args);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace

int to_bf16(const void* X, int dtype, int64_t count, void* Y, cudaStream_t s) {
  if (count == 0) return DETLSH_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(count, 256), 152 * 32);
  if (dtype == DETLSH_U8)
    k_to_bf16_u8<<<blocks, 256, 0, s>>>(static_cast<const uint8_t*>(X), count,
                                        static_cast<__nv_bfloat16*>(Y));
  else
    k_to_bf16_f32<<<blocks, 256, 0, s>>>(static_cast<const float*>(X), count,
                                         static_cast<__nv_bfloat16*>(Y));
  DL_LAUNCH();
  return DETLSH_OK;
}

int gather_rows_bf16(const void* Xb, int d, const int64_t* ids, int64_t m, void* Y, cudaStream_t s) {
  if (m == 0) return DETLSH_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(m * d, 256), 152 * 32);
  k_gather_rows_bf16<<<blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(Xb), d, ids, m,
                                            static_cast<__nv_bfloat16*>(Y));
  DL_LAUNCH();
  return DETLSH_OK;
}

std::atomic<unsigned long long> g_tc_wait_ns{TC_WAIT_NS};

unsigned long long tc_wait_limit_ns() { return g_tc_wait_ns.load(); }

int check_tc_error(int* d_err, cudaStream_t s) {
  int h = 0;
  DL_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaStreamSynchronize(s));
  if (h) {
    // reported once: the word is cleared for the index's next call
    DL_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    DL_CUDA(cudaStreamSynchronize(s));
    set_error("a bounded wait of a tensor-core kernel ran out");
    return DETLSH_ETIMEOUT;
  }
  return DETLSH_OK;
}

// P = Xb * Abᵀ on the tensor cores; with E/codes: encoded, else FP32 into P.
int launch_project_tc(const void* Xb, int64_t rows, int d, const void* Ab, int LK, int K,
                      const float* E, const uint8_t* Rtab, const float* Rlo, const float* Rinv, int Nr,
                      uint8_t* codes, float* P, int64_t p_so, int64_t p_sr, int* d_err, cudaStream_t s) {
  if (rows == 0) return DETLSH_OK;
  const int N = (LK + 15) / 16 * 16;
  if (N > 64 || d % 8 != 0) {
    set_error("tensor-core projection needs L*K <= 64 and d a multiple of 8");
    return DETLSH_EINVAL;
  }
  CUtensorMap tx, ta;
  DL_TRY(make_map(&tx, Xb, rows, d, TC_M));
  DL_TRY(make_map(&ta, Ab, N, d, N));
  TcArgs args{};
  args.rows = rows;
  args.d = d;
  args.LK = LK;
  args.K = K;
  args.Nr = Nr;
  args.E = E;
  args.Rtab = Rtab;
  args.Rlo = Rlo;
  args.Rinv = Rinv;
  args.codes = codes;
  args.P = P;
  args.p_so = p_so;
  args.p_sr = p_sr;
  args.err = d_err;
  args.wait_ns = g_tc_wait_ns.load();
  const bool enc = codes != nullptr;
#define DL_TC_CASE(NN)                                                        \
  case NN:                                                                    \
    return enc ? launch_tc<NN, true, false, false>(tx, ta, ta, ta, args, s)          \
               : launch_tc<NN, false, false, false>(tx, ta, ta, ta, args, s);
  switch (N) {
    DL_TC_CASE(16)
    DL_TC_CASE(32)
    DL_TC_CASE(48)
    DL_TC_CASE(64)
    default:
      break;
  }
#undef DL_TC_CASE
  set_error("unsupported projection width %d", N);
  return DETLSH_EINVAL;
}

namespace {
__global__ void k_split_tf32(const float* __restrict__ A, int LK, int N, int d, float* __restrict__ big,
                             float* __restrict__ small) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)N * d) return;
  const int r = (int)(i / d);
  const float x = r < LK ? A[i] : 0.f;
  const float b = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
  big[i] = b;
  small[i] = x - b;
}
}  // namespace

namespace {
__global__ void k_gather_rows_f32(const float* __restrict__ x, int d, const int64_t* __restrict__ ids, int64_t m,
                                  float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m * d;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / d, c = i % d;
    y[i] = x[ids[r] * d + c];
  }
}
}  // namespace

namespace {
// rows of a uint8 matrix gathered by id, 16 bytes at a time (d % 16 == 0)
__global__ void k_gather_rows_u8(const uint4* __restrict__ x, int dv, const int64_t* __restrict__ ids, int64_t m,
                                 uint4* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m * dv;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / dv, c = i % dv;
    y[i] = x[ids[r] * dv + c];
  }
}
}  // namespace

int gather_rows_u8(const uint8_t* X, int d, const int64_t* ids, int64_t m, uint8_t* Y, cudaStream_t s) {
  if (m == 0) return DETLSH_OK;
  if (d % 16 != 0) {
    set_error("gather_rows_u8 needs d a multiple of 16");
    return DETLSH_EINVAL;
  }
  const int dv = d / 16;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(m * dv, 256), 152 * 32);
  k_gather_rows_u8<<<blocks, 256, 0, s>>>(reinterpret_cast<const uint4*>(X), dv, ids, m,
                                          reinterpret_cast<uint4*>(Y));
  DL_LAUNCH();
  return DETLSH_OK;
}

int gather_rows_f32(const float* X, int d, const int64_t* ids, int64_t m, float* Y, cudaStream_t s) {
  if (m == 0) return DETLSH_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(m * d, 256), 152 * 32);
  k_gather_rows_f32<<<blocks, 256, 0, s>>>(X, d, ids, m, Y);
  DL_LAUNCH();
  return DETLSH_OK;
}

int split_tf32(const float* A, int LK, int d, float* Asplit, cudaStream_t s) {
  const int N = (LK + 15) / 16 * 16;
  k_split_tf32<<<ceil_div((int64_t)N * d, 256), 256, 0, s>>>(A, LK, N, d, Asplit, Asplit + (int64_t)N * d);
  DL_LAUNCH();
  return DETLSH_OK;
}

namespace {
__global__ void k_split_bf16x3(const float* __restrict__ A, int LK, int N, int d, __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nd = (int64_t)N * d;
  if (i >= nd) return;
  const int r = (int)(i / d);
  const float x = r < LK ? A[i] : 0.f;
  const __nv_bfloat16 a1 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a1);
  const __nv_bfloat16 a2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(a2);
  out[i] = a1;
  out[nd + i] = a2;
  out[2 * nd + i] = __float2bfloat16_rn(r2);
}
}  // namespace

int split_bf16x3(const float* A, int LK, int d, void* Ab3, cudaStream_t s) {
  const int N = (LK + 15) / 16 * 16;
  k_split_bf16x3<<<ceil_div((int64_t)N * d, 256), 256, 0, s>>>(A, LK, N, d, static_cast<__nv_bfloat16*>(Ab3));
  DL_LAUNCH();
  return DETLSH_OK;
}

bool bf16x3_eligible(int dtype, int d, int LK) {
  return dtype == DETLSH_U8 && d % 16 == 0 && d <= 256 && LK <= 64;
}

int launch_project_bf16x3(const uint8_t* X, int64_t rows, int d, const void* Ab3, int LK, int K, const float* E,
                          const uint8_t* Rtab, const float* Rlo, const float* Rinv, int Nr, uint8_t* codes,
                          float* P, int64_t p_so, int64_t p_sr, int* d_err, cudaStream_t s) {
  if (rows == 0) return DETLSH_OK;
  const int N = (LK + 15) / 16 * 16;
  if (!bf16x3_eligible(DETLSH_U8, d, LK)) {
    set_error("the uint8 tensor-core projection needs L*K <= 64 and d <= 256 a multiple of 16");
    return DETLSH_EINVAL;
  }
  const int64_t nd = (int64_t)N * d;
  CUtensorMap tx, ta, ta2, ta3;
  DL_TRY(make_map(&tx, X, rows, d, TC_M, MAP_U8));
  DL_TRY(make_map(&ta, Ab3, N, d, N));
  DL_TRY(make_map(&ta2, static_cast<const __nv_bfloat16*>(Ab3) + nd, N, d, N));
  DL_TRY(make_map(&ta3, static_cast<const __nv_bfloat16*>(Ab3) + 2 * nd, N, d, N));
  TcArgs args{};
  args.rows = rows;
  args.d = d;
  args.LK = LK;
  args.K = K;
  args.Nr = Nr;
  args.E = E;
  args.Rtab = Rtab;
  args.Rlo = Rlo;
  args.Rinv = Rinv;
  args.codes = codes;
  args.P = P;
  args.p_so = p_so;
  args.p_sr = p_sr;
  args.err = d_err;
  args.wait_ns = g_tc_wait_ns.load();
  const bool enc = codes != nullptr;
#define DL_TC_CASE(NN)                                                        \
  case NN:                                                                    \
    return enc ? launch_tc<NN, true, false, true>(tx, ta, ta2, ta3, args, s)  \
               : launch_tc<NN, false, false, true>(tx, ta, ta2, ta3, args, s);
  switch (N) {
    DL_TC_CASE(16)
    DL_TC_CASE(32)
    DL_TC_CASE(48)
    DL_TC_CASE(64)
    default:
      break;
  }
#undef DL_TC_CASE
  set_error("unsupported projection width %d", N);
  return DETLSH_EINVAL;
}

bool tf32_eligible(int dtype, int d, int LK) {
  return dtype == DETLSH_F32 && d % 4 == 0 && d <= 256 && LK <= 64;
}

int launch_project_tf32(const float* X, int64_t rows, int d, const float* Asplit, int LK, int K, const float* E,
                        const uint8_t* Rtab, const float* Rlo, const float* Rinv, int Nr, uint8_t* codes,
                        float* P, int64_t p_so, int64_t p_sr, int* d_err, cudaStream_t s) {
  if (rows == 0) return DETLSH_OK;
  const int N = (LK + 15) / 16 * 16;
  if (!tf32_eligible(DETLSH_F32, d, LK)) {
    set_error("the TF32 tensor-core projection needs L*K <= 64 and d <= 256 a multiple of 4");
    return DETLSH_EINVAL;
  }
  CUtensorMap tx, ta, ta2;
  DL_TRY(make_map(&tx, X, rows, d, TC_M, MAP_F32));
  DL_TRY(make_map(&ta, Asplit, N, d, N, MAP_F32));
  DL_TRY(make_map(&ta2, Asplit + (int64_t)N * d, N, d, N, MAP_F32));
  TcArgs args{};
  args.rows = rows;
  args.d = d;
  args.LK = LK;
  args.K = K;
  args.Nr = Nr;
  args.E = E;
  args.Rtab = Rtab;
  args.Rlo = Rlo;
  args.Rinv = Rinv;
  args.codes = codes;
  args.P = P;
  args.p_so = p_so;
  args.p_sr = p_sr;
  args.err = d_err;
  args.wait_ns = g_tc_wait_ns.load();
  const bool enc = codes != nullptr;
#define DL_TC_CASE(NN)                                                        \
  case NN:                                                                    \
    return enc ? launch_tc<NN, true, true, false>(tx, ta, ta2, ta2, args, s)          \
               : launch_tc<NN, false, true, false>(tx, ta, ta2, ta2, args, s);
  switch (N) {
    DL_TC_CASE(16)
    DL_TC_CASE(32)
    DL_TC_CASE(48)
    DL_TC_CASE(64)
    default:
      break;
  }
#undef DL_TC_CASE
  set_error("unsupported projection width %d", N);
  return DETLSH_EINVAL;
}

}  // namespace detlsh

extern "C" uint64_t detlsh_test_set_wait_limit_ns(uint64_t ns) {
  return detlsh::g_tc_wait_ns.exchange(ns);
}
