// Eq. 1 projection of points onto the L*K hash vectors, and Alg. 2 region
// encoding of the projected coordinates against the breakpoints.
//
// One thread owns one point and accumulates its 64 projections of one hash
// tile in registers. The hash matrix is read transposed (At [d][LK]) so each
// d-chunk of it is one coalesced block, staged in shared memory and read by
// every thread as broadcast float4 loads; the points' d-chunks are staged
// row-wise with a 4-float pad so the per-thread float4 reads are free of bank
// conflicts. With ENCODE the region search tables of the tile's hashes sit in
// shared memory (the one or two breakpoints a search then reads come through
// L1) and each projection is turned into its region code right away, so the
// projections never reach HBM.
#include "common.cuh"

namespace detlsh {
namespace {

constexpr int PT = 128;  // points per block, one per thread
constexpr int HT = 64;   // hash vectors per block
constexpr int DC = 32;   // d-chunk staged per iteration
constexpr int XS = DC + 4;

// Number of interior breakpoints e_z (z = 1..Nr-1, e[z]) with e_z <= p, for
// sorted e: branchless binary search for the largest such z (0 if none).
__device__ __forceinline__ int region_of(const float* e, int Nr, float p) {
  int pos = 0;
  for (int step = Nr >> 1; step > 0; step >>= 1) {
    pos += (e[pos + step] <= p) ? step : 0;
  }
  return pos;
}

template <typename TX>
__device__ __forceinline__ float4 load4(const TX* p);
template <>
__device__ __forceinline__ float4 load4<float>(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
template <>
__device__ __forceinline__ float4 load4<uint8_t>(const uint8_t* p) {
  uchar4 u = __ldg(reinterpret_cast<const uchar4*>(p));
  return make_float4((float)u.x, (float)u.y, (float)u.z, (float)u.w);
}
template <typename TX>
__device__ __forceinline__ float load1(const TX* p) { return (float)__ldg(p); }

template <typename TX>
__device__ __forceinline__ void stage_x(const TX* __restrict__ X, int64_t n, int d,
                                        const int64_t* __restrict__ rows, int64_t p0, int t0,
                                        bool vec4, float* Xs) {
  if (vec4) {
    // DC/4 float4 per row; consecutive threads read consecutive float4 of a row
    for (int i = threadIdx.x; i < PT * (DC / 4); i += PT) {
      const int pl = i / (DC / 4), c4 = (i % (DC / 4)) * 4;
      const int64_t p = p0 + pl;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (p < n && t0 + c4 < d) {
        const int64_t row = rows ? rows[p] : p;
        v = load4<TX>(X + row * (int64_t)d + t0 + c4);
      }
      *reinterpret_cast<float4*>(Xs + pl * XS + c4) = v;
    }
  } else {
    for (int i = threadIdx.x; i < PT * DC; i += PT) {
      const int pl = i / DC, c = i % DC;
      const int64_t p = p0 + pl;
      float v = 0.f;
      if (p < n && t0 + c < d) {
        const int64_t row = rows ? rows[p] : p;
        v = load1<TX>(X + row * (int64_t)d + t0 + c);
      }
      Xs[pl * XS + c] = v;
    }
  }
}

template <typename TX, bool ENCODE>
__global__ void __launch_bounds__(PT)
k_project(const TX* __restrict__ X, int64_t n, int d, const int64_t* __restrict__ rows,
          const float* __restrict__ At, int LK, float* __restrict__ P, int64_t p_so,
          int64_t p_sr, const float* __restrict__ E, const uint8_t* __restrict__ Rtab,
          const float* __restrict__ Rlo, const float* __restrict__ Rinv, int Nr, int K,
          uint8_t* __restrict__ codes, bool vec4) {
  extern __shared__ __align__(16) float smem[];
  float* As = smem;               // [DC][HT]
  float* Xs = As + DC * HT;       // [PT][XS]
  float* Slo = Xs + PT * XS;      // [HT] (ENCODE)
  float* Sinv = Slo + HT;         // [HT]
  uint8_t* Ts = reinterpret_cast<uint8_t*>(Sinv + HT);   // [HT][kRegionRow]
  const int tid = threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.x * PT;
  const int r0 = blockIdx.y * HT;
  const int nh = min(HT, LK - r0);

  if (ENCODE) {
    for (int i = tid; i < HT * kRegionRow / 4; i += PT) {
      const int h = (4 * i) / kRegionRow;
      reinterpret_cast<uint32_t*>(Ts)[i] =
          h < nh ? reinterpret_cast<const uint32_t*>(Rtab + (int64_t)r0 * kRegionRow)[i] : 0u;
    }
    for (int h = tid; h < HT; h += PT) {
      Slo[h] = h < nh ? Rlo[r0 + h] : 0.f;
      Sinv[h] = h < nh ? Rinv[r0 + h] : 0.f;
    }
  }

  float acc[HT];
#pragma unroll
  for (int h = 0; h < HT; ++h) acc[h] = 0.f;

  for (int t0 = 0; t0 < d; t0 += DC) {
    __syncthreads();
    for (int i = tid; i < DC * HT; i += PT) {
      const int t = i / HT, h = i % HT;
      As[i] = (t0 + t < d && h < nh) ? __ldg(At + (int64_t)(t0 + t) * LK + r0 + h) : 0.f;
    }
    stage_x<TX>(X, n, d, rows, p0, t0, vec4, Xs);
    __syncthreads();
    const float* xr = Xs + tid * XS;
#pragma unroll
    for (int t = 0; t < DC; t += 4) {
      const float4 xv = *reinterpret_cast<const float4*>(xr + t);
      const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4* a4 = reinterpret_cast<const float4*>(As + (t + u) * HT);
#pragma unroll
        for (int h4 = 0; h4 < HT / 4; ++h4) {
          const float4 a = a4[h4];
          acc[4 * h4 + 0] = fmaf(a.x, xs[u], acc[4 * h4 + 0]);
          acc[4 * h4 + 1] = fmaf(a.y, xs[u], acc[4 * h4 + 1]);
          acc[4 * h4 + 2] = fmaf(a.z, xs[u], acc[4 * h4 + 2]);
          acc[4 * h4 + 3] = fmaf(a.w, xs[u], acc[4 * h4 + 3]);
        }
      }
    }
  }

  const int64_t p = p0 + tid;
  if (p >= n) return;
  if (!ENCODE) {
#pragma unroll
    for (int h = 0; h < HT; ++h)
      if (h < nh) P[p * p_so + (int64_t)(r0 + h) * p_sr] = acc[h];
    return;
  }
  if (K == 16 && nh % 16 == 0) {
    // one 16-byte code vector per (tree, point)
#pragma unroll
    for (int g = 0; g < HT / 16; ++g) {
      if (g * 16 >= nh) break;
      uint32_t w[4];
      region_codes16(E + (int64_t)(r0 + g * 16) * (Nr + 1), Nr + 1, Ts + g * 16 * kRegionRow, Slo + g * 16,
                     Sinv + g * 16, acc + g * 16, w);
      const int tree = (r0 + g * 16) / 16;
      *reinterpret_cast<uint4*>(codes + ((int64_t)tree * n + p) * 16) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
#pragma unroll
    for (int h = 0; h < HT; ++h) {
      if (h < nh) {
        const int r = r0 + h, tree = r / K, j = r % K;
        codes[((int64_t)tree * n + p) * K + j] =
            (uint8_t)region_fast(E + (int64_t)(r0 + h) * (Nr + 1), Ts + h * kRegionRow, Slo[h], Sinv[h], acc[h]);
      }
    }
  }
}

__global__ void k_transpose(const float* __restrict__ A, int LK, int d, float* __restrict__ At) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (int64_t)LK * d) {
    const int r = (int)(i / d), t = (int)(i % d);
    At[(int64_t)t * LK + r] = A[i];
  }
}

__global__ void k_encode_values(const float* __restrict__ P, int64_t n, int LK,
                                const float* __restrict__ E, int Nr, uint8_t* __restrict__ codes) {
  const int64_t total = n * LK;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % LK);
    codes[i] = (uint8_t)region_of(E + (int64_t)r * (Nr + 1), Nr, P[i]);
  }
}

size_t project_smem(bool encode, int Nr) {
  return sizeof(float) * ((size_t)DC * HT + (size_t)PT * XS + (encode ? 2 * (size_t)HT : 0)) +
         (encode ? (size_t)HT * kRegionRow : 0);
}

template <typename TX, bool ENCODE>
int launch(const void* X, int64_t n, int d, const int64_t* rows, const float* At, int LK,
           float* P, int64_t p_so, int64_t p_sr, const float* E, const uint8_t* Rtab, const float* Rlo,
           const float* Rinv, int Nr, int K, uint8_t* codes, cudaStream_t s) {
  if (n == 0) return DETLSH_OK;
  const size_t sm = project_smem(ENCODE, Nr);
  auto kern = k_project<TX, ENCODE>;
  DL_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const bool vec4 = (d % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(X) % (sizeof(TX) == 4 ? 16 : 4) == 0);
  dim3 grid(ceil_div(n, PT), ceil_div(LK, HT));
  kern<<<grid, PT, sm, s>>>(static_cast<const TX*>(X), n, d, rows, At, LK, P, p_so, p_sr, E, Rtab, Rlo,
                            Rinv, Nr, K, codes, vec4);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace

int transpose_hashes(const float* A, int LK, int d, float* At, cudaStream_t s) {
  const int64_t tot = (int64_t)LK * d;
  k_transpose<<<ceil_div(tot, 256), 256, 0, s>>>(A, LK, d, At);
  DL_LAUNCH();
  return DETLSH_OK;
}

int launch_project_t(const void* X, int dtype, int64_t n, int d, const int64_t* rows,
                     const float* At, int LK, float* P, int64_t p_so, int64_t p_sr,
                     cudaStream_t s) {
  if (dtype == DETLSH_U8)
    return launch<uint8_t, false>(X, n, d, rows, At, LK, P, p_so, p_sr, nullptr, nullptr, nullptr, nullptr, 2,
                                  1, nullptr, s);
  return launch<float, false>(X, n, d, rows, At, LK, P, p_so, p_sr, nullptr, nullptr, nullptr, nullptr, 2, 1,
                              nullptr, s);
}

int launch_project_encode_t(const void* X, int dtype, int64_t n, int d, const float* At,
                            int K, int L, const float* E, const uint8_t* Rtab, const float* Rlo,
                            const float* Rinv, int Nr, uint8_t* codes, cudaStream_t s) {
  if (dtype == DETLSH_U8)
    return launch<uint8_t, true>(X, n, d, nullptr, At, K * L, nullptr, 0, 0, E, Rtab, Rlo, Rinv, Nr, K, codes,
                                 s);
  return launch<float, true>(X, n, d, nullptr, At, K * L, nullptr, 0, 0, E, Rtab, Rlo, Rinv, Nr, K, codes, s);
}

// ---- region search tables
namespace {

__global__ void k_region_tables(const float* __restrict__ E, int Nr, uint8_t* __restrict__ tab,
                                float* __restrict__ lo_out, float* __restrict__ inv_out) {
  const int h = blockIdx.x;
  const float* e = E + (int64_t)h * (Nr + 1);
  const float lo = e[1], hi = e[Nr - 1];
  float inv = (float)kRegionCells / (hi - lo);
  if (!(inv > 0.f) || !isfinite(inv)) inv = 0.f;
  // tab[c] = #{z >= 1 : cell(e_z) < c}; cell is non-decreasing in z
  for (int c = threadIdx.x; c < kRegionRow; c += blockDim.x) {
    int v = 0;
    if (c > kRegionCells) v = Nr - 1;
    else
      for (int z = 1; z < Nr; ++z) v += region_cell(lo, inv, e[z]) < c ? 1 : 0;
    tab[(int64_t)h * kRegionRow + c] = (uint8_t)v;
  }
  if (threadIdx.x == 0) {
    lo_out[h] = lo;
    inv_out[h] = inv;
  }
}

}  // namespace

int build_region_tables(const float* E, int LK, int Nr, uint8_t* tab, float* lo, float* inv, cudaStream_t s) {
  k_region_tables<<<LK, 256, 0, s>>>(E, Nr, tab, lo, inv);
  DL_LAUNCH();
  return DETLSH_OK;
}

int launch_encode_values(const float* P, int64_t n, int LK, const float* E, int Nr,
                         uint8_t* codes, cudaStream_t s) {
  if (n == 0) return DETLSH_OK;
  const int64_t total = n * LK;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16);
  k_encode_values<<<blocks, 256, 0, s>>>(P, n, LK, E, Nr, codes);
  DL_LAUNCH();
  return DETLSH_OK;
}

}  // namespace detlsh
