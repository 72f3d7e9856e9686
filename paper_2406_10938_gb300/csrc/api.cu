// C ABI of libdetlsh: argument checks, host/device staging and index lifetime.
#include <mutex>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace detlsh {

static thread_local char g_err[512] = "";
static thread_local bool g_trace_on = false;
static thread_local double g_trace[TR_COUNT] = {0};
static unsigned long long g_launches = 0;

void count_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }
bool trace_on() { return g_trace_on; }
void trace_reset(int first, int last) {
  for (int i = first; i <= last; ++i) g_trace[i] = 0.0;
}
void trace_add(int phase, double v) { g_trace[phase] += v; }

PhaseTimer::PhaseTimer(cudaStream_t s, bool allow) : s_(s), on_(g_trace_on && allow) {}
PhaseTimer::~PhaseTimer() {
  for (int i = 0; i < n_; ++i) {
    cudaEventDestroy(a_[i]);
    cudaEventDestroy(b_[i]);
  }
}
void PhaseTimer::begin(int phase) {
  if (!on_ || n_ >= kMax) return;
  cudaEventCreate(&a_[n_]);
  cudaEventCreate(&b_[n_]);
  phase_[n_] = phase;
  cudaEventRecord(a_[n_], s_);
  open_ = n_++;
}
void PhaseTimer::end() {
  if (!on_ || open_ < 0) return;
  cudaEventRecord(b_[open_], s_);
  open_ = -1;
}
int PhaseTimer::finish() {
  if (!on_) return DETLSH_OK;
  DL_CUDA(cudaStreamSynchronize(s_));
  for (int i = 0; i < n_; ++i) {
    float ms = 0.f;
    DL_CUDA(cudaEventElapsedTime(&ms, a_[i], b_[i]));
    g_trace[phase_[i]] += ms;
  }
  return DETLSH_OK;
}

cudaMemPool_t scratch_pool() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDev] = {};
  static bool tried[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!tried[dev]) {
    tried[dev] = true;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
      // freed memory up to a quarter of the device (at least 16 GiB) stays
      // mapped, so repeated builds and queries do not remap it (a build of
      // 1e8 points allocates about 16 GB of index and sort scratch)
      size_t fr = 0, total = 0;
      cudaMemGetInfo(&fr, &total);
      uint64_t keep = std::max<uint64_t>((uint64_t)16 << 30, (uint64_t)total / 4);
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      pools[dev] = pool;
    } else {
      cudaGetLastError();
    }
  }
  return pools[dev];
}

void clear_error() { g_err[0] = 0; }

int require_device_ptr(const void* p, const char* name) {
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: cudaPointerGetAttributes failed: %s", name, cudaGetErrorString(e));
    return e == cudaErrorInvalidValue ? DETLSH_EINVAL : DETLSH_ECUDA;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
    set_error("%s must be a device (or managed) address", name);
    return DETLSH_EINVAL;
  }
  return DETLSH_OK;
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int index_alloc_raw(void** p, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool = scratch_pool();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error("cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return DETLSH_ENOMEM;
  }
  return DETLSH_OK;
}

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int log2i(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return b;
}
size_t dtype_size(int dtype) { return dtype == DETLSH_U8 ? 1 : 4; }

// A device view of a caller buffer: the pointer itself for device memory,
// otherwise a stream-ordered device copy.
struct In {
  const void* d = nullptr;
  Scratch own;
  int stage(const void* p, size_t bytes, int mem, cudaStream_t s) {
    if (mem == DETLSH_MEM_DEVICE || p == nullptr || bytes == 0) {
      d = p;
      return DETLSH_OK;
    }
    DL_TRY(own.alloc(bytes, s));
    DL_CUDA(cudaMemcpyAsync(own.p, p, bytes, cudaMemcpyHostToDevice, s));
    d = own.p;
    return DETLSH_OK;
  }
};

// A device destination for a caller buffer, copied back for host memory.
struct Out {
  void* d = nullptr;
  void* h = nullptr;
  size_t bytes = 0;
  Scratch own;
  int stage(void* p, size_t b, int mem, cudaStream_t s) {
    bytes = b;
    if (mem == DETLSH_MEM_DEVICE || p == nullptr || b == 0) {
      d = p;
      return DETLSH_OK;
    }
    h = p;
    DL_TRY(own.alloc(b, s));
    d = own.p;
    return DETLSH_OK;
  }
  int finish(cudaStream_t s) {
    if (h) DL_CUDA(cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s));
    return DETLSH_OK;
  }
};

__global__ void k_check_ids(const int64_t* ids, int64_t m, int64_t n, int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m && (ids[i] < 0 || ids[i] >= n)) atomicExch(bad, 1);
}

__global__ void k_check_query_args(const int32_t* k, const float* c, const float* r_min, int64_t nq,
                                   int k_max, int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const bool ok = k[i] >= 1 && k[i] <= k_max && isfinite(c[i]) && c[i] > 1.0f &&
                  !isnan(r_min[i]) && isfinite(r_min[i]);
  if (!ok) atomicExch(bad, 1);
}

int check_flag(int* d_bad, cudaStream_t s, const char* what) {
  int h = 0;
  DL_CUDA(cudaMemcpyAsync(&h, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("%s", what);
    return DETLSH_EINVAL;
  }
  return DETLSH_OK;
}

void free_index(detlsh_index* idx) {
  if (!idx) return;
  // no kernel of any stream may still use the arrays
  cudaDeviceSynchronize();
  if (idx->owns_x && idx->X) cudaFreeAsync(const_cast<void*>(idx->X), 0);
  void* arrays[] = {idx->A, idx->At, idx->E, idx->Ps, idx->sample, idx->codes, idx->leaf_ids, idx->leaf_pos, idx->leaf_base,
                    idx->leaf_range, idx->leaf_plen, idx->leaf_prefix, idx->leaf_lo, idx->leaf_hi,
                    idx->leaf_tree, idx->Xb, idx->Ab, idx->d_err, idx->Rtab, idx->Rlo, idx->Rinv, idx->Atf, idx->Ab3,
                    idx->xn2, idx->chunk_base, idx->chunk_leaf};
  for (void* p : arrays)
    if (p) cudaFreeAsync(p, 0);
  cudaStreamSynchronize(0);
  delete idx;
}

int build_impl(const void* X, int64_t n, int32_t d, int32_t dtype, const float* A, int32_t mem_a,
               const int64_t* sample_ids, int32_t mem_ids, int64_t n_s, const detlsh_params* prm,
               int32_t mem, cudaStream_t s, detlsh_index* idx) {
  const int K = prm->K, L = prm->L, Nr = prm->n_regions;
  const int LK = K * L;
  idx->n = n;
  idx->d = d;
  idx->dtype = dtype;
  idx->K = K;
  idx->L = L;
  idx->Nr = Nr;
  idx->bits = log2i(Nr);
  idx->max_leaf = prm->max_leaf;
  idx->n_s = n_s;
  idx->proj_mode = prm->proj_mode;
  idx->flags = prm->flags;
  DL_CUDA(cudaGetDevice(&idx->device));

  const size_t xbytes = (size_t)n * d * dtype_size(dtype);
  if (mem == DETLSH_MEM_DEVICE && (prm->flags & DETLSH_BORROW_X)) {
    idx->X = X;
    idx->owns_x = false;
  } else {
    void* xd = nullptr;
    DL_TRY(index_alloc(&xd, xbytes, s));
    idx->X = xd;
    DL_CUDA(cudaMemcpyAsync(xd, X, xbytes,
                            mem == DETLSH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s));
  }
  DL_TRY(index_alloc(&idx->A, sizeof(float) * LK * d, s));
  DL_CUDA(cudaMemcpyAsync(idx->A, A, sizeof(float) * LK * d,
                          mem_a == DETLSH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  DL_TRY(index_alloc(&idx->At, sizeof(float) * LK * d, s));
  DL_TRY(transpose_hashes(idx->A, LK, d, idx->At, s));

  DL_TRY(index_alloc(&idx->sample, sizeof(int64_t) * n_s, s));
  DL_CUDA(cudaMemcpyAsync(idx->sample, sample_ids, sizeof(int64_t) * n_s,
                          mem_ids == DETLSH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  const int64_t* sid = idx->sample;
  {
    Scratch bad;
    DL_TRY(bad.alloc(sizeof(int), s));
    DL_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_check_ids<<<ceil_div(n_s, 256), 256, 0, s>>>(sid, n_s, n,
                                                       bad.as<int>());
    DL_LAUNCH();
    DL_TRY(check_flag(bad.as<int>(), s, "sample_ids must lie in [0, n)"));
  }
  PhaseTimer tm(s);
  // Alg. 1: projections of the sample, [LK][n_s]
  DL_TRY(index_alloc(&idx->Ps, sizeof(float) * LK * n_s, s));
  DL_TRY(index_alloc(&idx->E, sizeof(float) * LK * (Nr + 1), s));
  DL_TRY(index_alloc(&idx->codes, (size_t)n * LK, s));
  DL_TRY(index_alloc(&idx->leaf_ids, sizeof(uint32_t) * n * L, s));
  DL_TRY(index_alloc(&idx->Rtab, (size_t)LK * kRegionRow, s));
  DL_TRY(index_alloc(&idx->Rlo, sizeof(float) * LK, s));
  DL_TRY(index_alloc(&idx->Rinv, sizeof(float) * LK, s));
  if (prm->proj_mode == DETLSH_PROJ_BF16) {
    // BF16 copies of X and A; projections on the tensor cores
    const int N = (LK + 15) / 16 * 16;
    DL_TRY(index_alloc(&idx->Xb, (size_t)n * d * 2, s));
    DL_TRY(index_alloc(&idx->Ab, (size_t)N * d * 2, s));
    DL_TRY(index_alloc(&idx->d_err, sizeof(int), s));
    DL_CUDA(cudaMemsetAsync(idx->Ab, 0, (size_t)N * d * 2, s));
    DL_CUDA(cudaMemsetAsync(idx->d_err, 0, sizeof(int), s));
    tm.begin(TR_SAMPLE_PROJ);
    DL_TRY(to_bf16(idx->X, dtype, n * d, idx->Xb, s));
    DL_TRY(to_bf16(idx->A, DETLSH_F32, (int64_t)LK * d, idx->Ab, s));
    Scratch xs;
    DL_TRY(xs.alloc((size_t)n_s * d * 2, s));
    DL_TRY(gather_rows_bf16(idx->Xb, d, sid, n_s, xs.p, s));
    DL_TRY(launch_project_tc(xs.p, n_s, d, idx->Ab, LK, K, nullptr, nullptr, nullptr, nullptr, Nr, nullptr,
                             idx->Ps, 1, n_s, idx->d_err, s));
    tm.end();
    tm.begin(TR_BREAKPOINTS);
    DL_TRY(select_breakpoints(idx->Ps, n_s, LK, Nr, idx->E, s));
    DL_TRY(build_region_tables(idx->E, LK, Nr, idx->Rtab, idx->Rlo, idx->Rinv, s));
    tm.end();
    tm.begin(TR_ENCODE);
    DL_TRY(launch_project_tc(idx->Xb, n, d, idx->Ab, LK, K, idx->E, idx->Rtab, idx->Rlo, idx->Rinv, Nr,
                             idx->codes, nullptr, 0, 0, idx->d_err, s));
    tm.end();
    DL_TRY(check_tc_error(idx->d_err, s));
  } else {
    // FP32 inputs: on the tensor cores through the TF32 split where the shapes
    // allow it. The sample is projected by the same kernel as the points, so
    // the points that define breakpoints fall on them exactly when encoded.
    // uint8 points likewise, widened to BF16 (exact) in the kernel against A in
    // three BF16 parts
    // (the tensor-core kernels read X by TMA, which needs a 16-byte aligned base)
    const bool x16 = reinterpret_cast<uintptr_t>(idx->X) % 16 == 0;
    const bool tf32 = x16 && tf32_eligible(dtype, d, LK);
    const bool b3 = x16 && bf16x3_eligible(dtype, d, LK);
    const int Nh = (LK + 15) / 16 * 16;
    if (tf32 || b3) {
      DL_TRY(index_alloc(&idx->d_err, sizeof(int), s));
      DL_CUDA(cudaMemsetAsync(idx->d_err, 0, sizeof(int), s));
    }
    if (tf32) {
      DL_TRY(index_alloc(&idx->Atf, sizeof(float) * 2 * Nh * d, s));
      DL_TRY(split_tf32(idx->A, LK, d, idx->Atf, s));
    }
    if (b3) {
      DL_TRY(index_alloc(&idx->Ab3, (size_t)3 * Nh * d * 2, s));
      DL_TRY(split_bf16x3(idx->A, LK, d, idx->Ab3, s));
    }
    tm.begin(TR_SAMPLE_PROJ);
    if (b3) {
      Scratch xs;
      DL_TRY(xs.alloc((size_t)n_s * d, s));
      DL_TRY(gather_rows_u8(static_cast<const uint8_t*>(idx->X), d, sid, n_s,
                            xs.as<uint8_t>(), s));
      DL_TRY(launch_project_bf16x3(xs.as<uint8_t>(), n_s, d, idx->Ab3, LK, K, nullptr, nullptr, nullptr, nullptr, Nr,
                                   nullptr, idx->Ps, 1, n_s, idx->d_err, s));
    } else if (tf32) {
      Scratch xs;
      DL_TRY(xs.alloc(sizeof(float) * n_s * d, s));
      DL_TRY(gather_rows_f32(static_cast<const float*>(idx->X), d, sid, n_s,
                             xs.as<float>(), s));
      DL_TRY(launch_project_tf32(xs.as<float>(), n_s, d, idx->Atf, LK, K, nullptr, nullptr, nullptr, nullptr,
                                 Nr, nullptr, idx->Ps, 1, n_s, idx->d_err, s));
    } else {
      DL_TRY(launch_project_t(idx->X, dtype, n_s, d, sid, idx->At, LK,
                              idx->Ps, 1, n_s, s));
    }
    tm.end();
    tm.begin(TR_BREAKPOINTS);
    DL_TRY(select_breakpoints(idx->Ps, n_s, LK, Nr, idx->E, s));
    DL_TRY(build_region_tables(idx->E, LK, Nr, idx->Rtab, idx->Rlo, idx->Rinv, s));
    tm.end();
    // Alg. 2: codes of every point, fused with the projection
    tm.begin(TR_ENCODE);
    if (b3) {
      DL_TRY(launch_project_bf16x3(static_cast<const uint8_t*>(idx->X), n, d, idx->Ab3, LK, K, idx->E, idx->Rtab, idx->Rlo, idx->Rinv, Nr,
                                   idx->codes, nullptr, 0, 0, idx->d_err, s));
    } else if (tf32) {
      DL_TRY(launch_project_tf32(static_cast<const float*>(idx->X), n, d, idx->Atf, LK, K, idx->E, idx->Rtab,
                                 idx->Rlo, idx->Rinv, Nr, idx->codes, nullptr, 0, 0, idx->d_err, s));
    } else {
      DL_TRY(launch_project_encode_t(idx->X, dtype, n, d, idx->At, K, L, idx->E, idx->Rtab, idx->Rlo,
                                     idx->Rinv, Nr, idx->codes, s));
    }
    tm.end();
    if (idx->Atf || idx->Ab3) DL_TRY(check_tc_error(idx->d_err, s));
  }
  // Alg. 3: leaves
  tm.begin(TR_LEAVES);
  DL_TRY(build_leaves(idx, s));
  tm.end();
  // BF16 indexes: what the leaf-major coarse distances of the shortlist mode read
  if (idx->Xb) DL_TRY(build_lm_tables(idx, s));
  DL_TRY(tm.finish());
  DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

}  // namespace
}  // namespace detlsh

using namespace detlsh;

namespace detlsh {
namespace {

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

struct TuneCtx {
  const detlsh_index* idx;
  const void* Q;
  int64_t nq;
  const int32_t* k;
  const float* c;
  const float* r;
  int k_max;
  double eps, beta;
  int64_t* ids;
  float* dist;
  cudaStream_t s;
};

int run_tuned(const TuneCtx& x, int shortlist, const QueryTuning& tu) {
  return run_query(x.idx, x.Q, x.nq, x.k, x.c, x.r, x.k_max, x.eps, x.beta, x.ids, x.dist, nullptr,
                   nullptr, 0, nullptr, shortlist, tu, x.s);
}

// device milliseconds of the query (the faster of two runs after one warm-up)
int time_tuned(const TuneCtx& x, int shortlist, const QueryTuning& tu, float* ms) {
  EventPair ev;
  DL_CUDA(cudaEventCreate(&ev.a));
  DL_CUDA(cudaEventCreate(&ev.b));
  DL_TRY(run_tuned(x, shortlist, tu));
  float best = INFINITY;
  for (int rep = 0; rep < 2; ++rep) {
    DL_CUDA(cudaEventRecord(ev.a, x.s));
    DL_TRY(run_tuned(x, shortlist, tu));
    DL_CUDA(cudaEventRecord(ev.b, x.s));
    DL_CUDA(cudaEventSynchronize(ev.b));
    float t = 0.f;
    DL_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
    best = std::min(best, t);
  }
  *ms = best;
  return DETLSH_OK;
}

}  // namespace

}  // namespace detlsh

#ifdef DETLSH_CHECKED
namespace detlsh {
namespace {
constexpr int kMaxCheckReaders = 32;
int (*g_check_readers[kMaxCheckReaders])(unsigned int*) = {};
int g_n_check_readers = 0;
}  // namespace
// called during the library's static initialisation, one reader per
// translation unit
int register_check_reader(int (*read)(unsigned int* words)) {
  if (g_n_check_readers < kMaxCheckReaders) g_check_readers[g_n_check_readers++] = read;
  return g_n_check_readers;
}
}  // namespace detlsh
#endif

extern "C" {

const char* detlsh_strerror(int status) {
  switch (status) {
    case DETLSH_PENDING: return "pending";
    case DETLSH_OK: return "success";
    case DETLSH_EINVAL: return "invalid argument";
    case DETLSH_ENOMEM: return "out of memory";
    case DETLSH_ECUDA: return "CUDA error";
    case DETLSH_ETIMEOUT: return "device wait timed out";
    case DETLSH_EADMIT: return "request not admitted";
    case DETLSH_EINTERNAL: return "internal error";
    default: return "unknown status";
  }
}

const char* detlsh_last_error(void) { return g_err; }

int detlsh_trace_enable(int32_t on) {
  const int prev = g_trace_on ? 1 : 0;
  g_trace_on = on != 0;
  return prev;
}

int detlsh_trace_get(double* out, int32_t len) {
  if (!out || len < 0) return DETLSH_EINVAL;
  const int m = std::min<int>(len, TR_COUNT);
  for (int i = 0; i < m; ++i) out[i] = g_trace[i];
  return m;
}

int detlsh_memory_stats(int32_t reset_peak, int64_t* out, int32_t len) {
  clear_error();
  DL_REQUIRE(out != nullptr && len >= 0, "out must be non-NULL and len >= 0");
  int dev = 0;
  DL_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pools[2] = {scratch_pool(), nullptr};
  DL_CUDA(cudaDeviceGetDefaultMemPool(&pools[1], dev));
  int64_t v[4] = {0, 0, 0, 0};
  for (int i = 0; i < 2; ++i) {
    if (!pools[i]) continue;
    uint64_t cur = 0, peak = 0;
    DL_CUDA(cudaMemPoolGetAttribute(pools[i], cudaMemPoolAttrUsedMemCurrent, &cur));
    DL_CUDA(cudaMemPoolGetAttribute(pools[i], cudaMemPoolAttrUsedMemHigh, &peak));
    v[2 * i] = (int64_t)cur;
    v[2 * i + 1] = (int64_t)peak;
    if (reset_peak) {
      uint64_t zero = 0;   // resets the high-water mark to the current use
      DL_CUDA(cudaMemPoolSetAttribute(pools[i], cudaMemPoolAttrUsedMemHigh, &zero));
    }
  }
  const int m = std::min<int>(len, 4);
  for (int i = 0; i < m; ++i) out[i] = v[i];
  return m;
}

int64_t detlsh_launch_count(void) {
  return (int64_t)__atomic_load_n(&g_launches, __ATOMIC_RELAXED);
}


int detlsh_check_status(uint32_t* out, int32_t len) {
#ifdef DETLSH_CHECKED
  if (cudaDeviceSynchronize() != cudaSuccess) return DETLSH_ECUDA;
  uint32_t tot[4] = {0u, 0u, 0u, 0u};
  for (int i = 0; i < g_n_check_readers; ++i) {
    unsigned int w[4];
    if (g_check_readers[i](w) != 0) return DETLSH_ECUDA;
    if (w[0] && !tot[0]) {
      tot[1] = w[1];
      tot[2] = w[2];
      tot[3] = w[3];
    }
    tot[0] += w[0];
  }
  for (int i = 0; i < std::min<int>(len, 4); ++i) out[i] = tot[i];
  return 1;
#else
  (void)out;
  (void)len;
  return 0;
#endif
}

double detlsh_eps_lemma3(int32_t K, int32_t L) {
  if (K < 1 || L < 1) return -1.0;
  return std::sqrt(chi2_upper_quantile(std::exp(-1.0 / L), K));
}

int detlsh_build(const void* X, int64_t n, int32_t d, int32_t dtype, const float* A,
                 const int64_t* sample_ids, const detlsh_params* params, int32_t mem, void* stream,
                 detlsh_index** out) {
  g_err[0] = 0;
  DL_REQUIRE(out != nullptr && params != nullptr, "out and params must be non-NULL");
  *out = nullptr;
  DL_REQUIRE(X != nullptr, "X must be non-NULL");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(dtype == DETLSH_F32 || dtype == DETLSH_U8, "bad dtype");
  const detlsh_params& p = *params;
  DL_REQUIRE(p.K >= 1 && p.K <= kMaxK, "K must be in [1, %d]", kMaxK);
  DL_REQUIRE(p.L >= 1 && p.L <= kMaxL, "L must be in [1, %d]", kMaxL);
  DL_REQUIRE(is_pow2(p.n_regions) && p.n_regions >= 2 && p.n_regions <= 256,
             "n_regions must be a power of two in [2, 256]");
  DL_REQUIRE(p.max_leaf >= 1, "max_leaf must be >= 1");
  DL_REQUIRE(d >= 1 && d <= 65536, "d must be in [1, 65536]");
  DL_REQUIRE(n >= 1 && n * (int64_t)p.L < ((int64_t)1 << 32), "need 1 <= n and n*L < 2^32");
  DL_REQUIRE(p.sample_size >= 0, "sample_size must be >= 0");
  DL_REQUIRE(sample_ids == nullptr || p.sample_size > 0, "sample_size must give the length of sample_ids");
  // Sec. 6.1: n_s = 0.1 n unless given
  const int64_t n_s = p.sample_size > 0 ? p.sample_size : (n + 9) / 10;
  DL_REQUIRE(n_s >= p.n_regions && n_s <= n, "need n_regions <= n_s <= n (n_s = %lld)", (long long)n_s);
  DL_REQUIRE(p.proj_mode == DETLSH_PROJ_FP32 || p.proj_mode == DETLSH_PROJ_BF16, "unsupported proj_mode");
  DL_REQUIRE((p.flags & ~(DETLSH_BORROW_X | DETLSH_DEDUP_POS)) == 0, "unknown flags");
  DL_REQUIRE(p.proj_mode != DETLSH_PROJ_BF16 || (d % 8 == 0 && p.K * p.L <= 64),
             "the BF16 projection needs d %% 8 == 0 and L*K <= 64");
  DL_REQUIRE(n_s * (int64_t)p.K * p.L < ((int64_t)1 << 32), "n_s*L*K must be < 2^32");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  trace_reset(TR_SAMPLE_PROJ, TR_LEAVES);
  trace_reset(TR_BUILD_TOTAL, TR_BUILD_TOTAL);
  trace_reset(TR_LEAF_ROOT, TR_LEAF_ITERS);
  PhaseTimer total(s);
  total.begin(TR_BUILD_TOTAL);
  detlsh_index* idx = new (std::nothrow) detlsh_index();
  if (!idx) {
    set_error("host allocation failed");
    return DETLSH_ENOMEM;
  }
  // the random draws of the method, when the caller leaves them to the library
  std::vector<float> A_h;
  std::vector<int64_t> ids_h;
  int32_t mem_a = mem, mem_ids = mem;
  if (A == nullptr) {
    A_h.resize((size_t)p.K * p.L * d);
    draw_hashes(p.seed, (int64_t)A_h.size(), A_h.data());
    A = A_h.data();
    mem_a = DETLSH_MEM_HOST;
  }
  if (sample_ids == nullptr) {
    ids_h.resize((size_t)n_s);
    draw_sample(p.seed, n, n_s, ids_h.data());
    sample_ids = ids_h.data();
    mem_ids = DETLSH_MEM_HOST;
  }
  const int st = build_impl(X, n, d, dtype, A, mem_a, sample_ids, mem_ids, n_s, params, mem, s, idx);
  if (st != DETLSH_OK) {
    cudaStreamSynchronize(s);
    free_index(idx);
    return st;
  }
  total.end();
  const int ts = total.finish();
  if (ts != DETLSH_OK) {
    free_index(idx);
    return ts;
  }
  *out = idx;
  return DETLSH_OK;
}

int detlsh_query(const detlsh_index* idx, const void* Q, int64_t nq, int32_t dtype, const int32_t* k,
                 const float* c, const float* r_min, int32_t k_max, const detlsh_query_params* qp,
                 int64_t* out_ids, float* out_dist, int32_t* out_stats, int32_t mem, void* stream) {
  g_err[0] = 0;
  DL_REQUIRE(idx != nullptr, "index is NULL");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(dtype == idx->dtype, "query dtype differs from the index's");
  DL_REQUIRE(nq >= 0, "nq must be >= 0");
  DL_REQUIRE(k_max >= 1 && k_max <= kMaxTopK, "k_max must be in [1, %d]", kMaxTopK);
  if (nq == 0) return DETLSH_OK;
  DL_REQUIRE(Q && k && c && r_min && out_ids && out_dist, "NULL query argument");
  double eps = qp ? qp->eps : 0.0;
  const double beta = qp ? qp->beta : 0.1;
  DL_REQUIRE(beta >= 0.0 && std::isfinite(beta), "beta must be finite and >= 0");
  if (!(eps > 0.0)) eps = detlsh_eps_lemma3(idx->K, idx->L);
  DL_REQUIRE(std::isfinite(eps) && eps > 0.0, "eps must be finite and > 0");
  uint32_t* cand = qp ? qp->cand_ids : nullptr;
  const int64_t cand_cap = qp ? qp->cand_cap : 0;
  const int32_t shortlist = qp ? qp->shortlist : 0;
  DL_REQUIRE(shortlist >= 0, "shortlist must be >= 0");
  DL_REQUIRE(cand == nullptr || cand_cap >= 1, "cand_cap must be >= 1 with cand_ids");
  if (mem == DETLSH_MEM_HOST) {
    for (int64_t i = 0; i < nq; ++i) {
      DL_REQUIRE(k[i] >= 1 && k[i] <= k_max, "k[%lld] must be in [1, k_max]", (long long)i);
      DL_REQUIRE(std::isfinite(c[i]) && c[i] > 1.0f, "c[%lld] must be finite and > 1", (long long)i);
      DL_REQUIRE(std::isfinite(r_min[i]), "r_min[%lld] must be finite", (long long)i);
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  In dQ, dk, dc, dr;
  DL_TRY(dQ.stage(Q, (size_t)nq * idx->d * dtype_size(dtype), mem, s));
  DL_TRY(dk.stage(k, sizeof(int32_t) * nq, mem, s));
  DL_TRY(dc.stage(c, sizeof(float) * nq, mem, s));
  DL_TRY(dr.stage(r_min, sizeof(float) * nq, mem, s));
  if (mem == DETLSH_MEM_DEVICE) {
    Scratch bad;
    DL_TRY(bad.alloc(sizeof(int), s));
    DL_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_check_query_args<<<ceil_div(nq, 256), 256, 0, s>>>(static_cast<const int32_t*>(dk.d),
                                                        static_cast<const float*>(dc.d),
                                                        static_cast<const float*>(dr.d), nq, k_max,
                                                        bad.as<int>());
    DL_LAUNCH();
    DL_TRY(check_flag(bad.as<int>(), s, "each query needs 1 <= k <= k_max, finite c > 1, finite r_min"));
  }
  trace_reset(TR_QUERY_PROJ, TR_LB_LAUNCHES);
  trace_reset(TR_QUERY_TOTAL, TR_BUCKET);
  trace_reset(TR_GROUP, TR_GROUP);
  PhaseTimer total(s);
  total.begin(TR_QUERY_TOTAL);
  Out oi, od, os, oc, oq;
  DL_TRY(oi.stage(out_ids, sizeof(int64_t) * nq * k_max, mem, s));
  DL_TRY(od.stage(out_dist, sizeof(float) * nq * k_max, mem, s));
  DL_TRY(os.stage(out_stats, sizeof(int32_t) * nq * 4, mem, s));
  DL_TRY(oc.stage(cand, cand ? sizeof(uint32_t) * nq * cand_cap : 0, mem, s));
  float* qproj = qp ? qp->qproj : nullptr;
  DL_TRY(oq.stage(qproj, qproj ? sizeof(float) * nq * idx->K * idx->L : 0, mem, s));
  QueryTuning tu;
  DL_TRY(tuning_from_params(qp, &tu));
  DL_TRY(run_query(idx, dQ.d, nq, static_cast<const int32_t*>(dk.d), static_cast<const float*>(dc.d),
                   static_cast<const float*>(dr.d), k_max, eps, beta, static_cast<int64_t*>(oi.d),
                   static_cast<float*>(od.d), static_cast<int32_t*>(os.d), static_cast<uint32_t*>(oc.d),
                   cand_cap, static_cast<float*>(oq.d), shortlist, tu, s));
  DL_TRY(oi.finish(s));
  DL_TRY(od.finish(s));
  DL_TRY(os.finish(s));
  DL_TRY(oc.finish(s));
  DL_TRY(oq.finish(s));
  total.end();
  DL_TRY(total.finish());
  if (mem == DETLSH_MEM_HOST) DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

int detlsh_autotune(const detlsh_index* idx, const void* Q, int64_t nq, int32_t dtype, const int32_t* k,
                    const float* c, const float* r_min, int32_t k_max, const detlsh_query_params* qp,
                    double min_agreement, int32_t mem, void* stream, detlsh_tuning* out) {
  g_err[0] = 0;
  DL_REQUIRE(idx != nullptr && out != nullptr, "NULL argument");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(dtype == idx->dtype, "query dtype differs from the index's");
  DL_REQUIRE(nq >= 1, "autotuning needs at least one query");
  DL_REQUIRE(k_max >= 1 && k_max <= kMaxTopK, "k_max must be in [1, %d]", kMaxTopK);
  DL_REQUIRE(Q && k && c && r_min, "NULL query argument");
  DL_REQUIRE(std::isfinite(min_agreement) && min_agreement <= 1.0, "min_agreement must be <= 1");
  DL_REQUIRE(!qp || (!qp->cand_ids && !qp->qproj), "autotuning does not export candidate lists or projections");
  double eps = qp ? qp->eps : 0.0;
  const double beta = qp ? qp->beta : 0.1;
  DL_REQUIRE(beta >= 0.0 && std::isfinite(beta), "beta must be finite and >= 0");
  if (!(eps > 0.0)) eps = detlsh_eps_lemma3(idx->K, idx->L);
  const int32_t shortlist0 = qp ? qp->shortlist : 0;
  DL_REQUIRE(shortlist0 >= 0, "shortlist must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int32_t> hk(nq);
  if (mem == DETLSH_MEM_HOST) {
    std::memcpy(hk.data(), k, sizeof(int32_t) * nq);
  } else {
    DL_CUDA(cudaMemcpyAsync(hk.data(), k, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, s));
    DL_CUDA(cudaStreamSynchronize(s));
  }
  for (int64_t i = 0; i < nq; ++i)
    DL_REQUIRE(hk[i] >= 1 && hk[i] <= k_max, "k[%lld] must be in [1, k_max]", (long long)i);
  In dQ, dk, dc, dr;
  DL_TRY(dQ.stage(Q, (size_t)nq * idx->d * dtype_size(dtype), mem, s));
  DL_TRY(dk.stage(k, sizeof(int32_t) * nq, mem, s));
  DL_TRY(dc.stage(c, sizeof(float) * nq, mem, s));
  DL_TRY(dr.stage(r_min, sizeof(float) * nq, mem, s));
  Scratch ids, dist;
  DL_TRY(ids.alloc(sizeof(int64_t) * nq * k_max, s));
  DL_TRY(dist.alloc(sizeof(float) * nq * k_max, s));
  const TuneCtx x{idx, dQ.d, nq, static_cast<const int32_t*>(dk.d), static_cast<const float*>(dc.d),
                  static_cast<const float*>(dr.d), k_max, eps, beta, ids.as<int64_t>(),
                  dist.as<float>(), s};
  const bool trace = g_trace_on;
  g_trace_on = false;
  QueryTuning best;
  int st = tuning_from_params(qp, &best);
  float tbest = INFINITY;
  if (st == DETLSH_OK) st = time_tuned(x, shortlist0, best, &tbest);
  // coordinate descent over the launch shapes; a shape that does not fit
  // (shared memory, device memory) is skipped
  auto attempt = [&](const QueryTuning& t) {
    if (st != DETLSH_OK) return;
    float ms = 0.f;
    const int r = time_tuned(x, shortlist0, t, &ms);
    if (r == DETLSH_OK && ms < tbest) {
      tbest = ms;
      best = t;
    } else if (r == DETLSH_ECUDA) {
      st = r;
    }
  };
  for (int w : {1, 2, 3, 4}) {
    QueryTuning t = best;
    t.walk_ctas_per_sm = w;
    attempt(t);
  }
  for (int rows : {128, 256, 512, 1024}) {
    QueryTuning t = best;
    t.dist_rows = rows;
    attempt(t);
  }
  for (int dc3 : {1, 2, 3, 4}) {
    QueryTuning t = best;
    t.dist_ctas_per_sm = dc3;
    attempt(t);
  }
  for (int st : {1, 2}) {
    QueryTuning t = best;
    t.streams = st;
    attempt(t);
  }
  for (int64_t b : {(int64_t)1024, (int64_t)2048, (int64_t)4096, (int64_t)8192, (int64_t)16384}) {
    if (b >= nq) break;
    QueryTuning t = best;
    t.batch = b;
    attempt(t);
  }
  int32_t pick = 0;
  if (st == DETLSH_OK && idx->Xb != nullptr && min_agreement > 0.0) {
    // the exact FP32 top-k of the sample, then the smallest agreeing shortlist
    float t_exact = 0.f;
    st = time_tuned(x, 0, best, &t_exact);
    std::vector<int64_t> ref((size_t)nq * k_max), got((size_t)nq * k_max);
    if (st == DETLSH_OK) {
      cudaMemcpyAsync(ref.data(), x.ids, sizeof(int64_t) * ref.size(), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) st = DETLSH_ECUDA;
    }
    for (int32_t sl = 64; st == DETLSH_OK && sl <= 4096; sl *= 2) {
      if (sl < k_max) continue;
      st = run_tuned(x, sl, best);
      if (st != DETLSH_OK) break;
      cudaMemcpyAsync(got.data(), x.ids, sizeof(int64_t) * got.size(), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        st = DETLSH_ECUDA;
        break;
      }
      double agree = 0.0;
      for (int64_t q = 0; q < nq; ++q) {
        const int64_t* a = &ref[(size_t)q * k_max];
        const int64_t* g = &got[(size_t)q * k_max];
        int64_t have = 0, hit = 0;
        for (int j = 0; j < hk[q]; ++j) {
          if (a[j] < 0) continue;
          ++have;
          for (int i = 0; i < hk[q]; ++i)
            if (g[i] == a[j]) {
              ++hit;
              break;
            }
        }
        agree += have ? (double)hit / (double)have : 1.0;
      }
      agree /= (double)nq;
      if (agree >= min_agreement) {
        // the coarse distances by leaf on the tensor cores or by candidate
        // gather, whichever is faster on this index and sample
        float t_sl = 0.f, t_alt = 0.f;
        st = time_tuned(x, sl, best, &t_sl);
        QueryTuning alt = best;
        alt.coarse_gather = 1 - best.coarse_gather;
        if (st == DETLSH_OK) st = time_tuned(x, sl, alt, &t_alt);
        if (st == DETLSH_OK && t_alt < t_sl) {
          best = alt;
          t_sl = t_alt;
        }
        if (st == DETLSH_OK && t_sl < t_exact) pick = sl;
        break;
      }
    }
  }
  g_trace_on = trace;
  if (st != DETLSH_OK) return st;
  std::memset(out, 0, sizeof(*out));
  out->batch = best.batch;
  out->walk_ctas_per_sm = best.walk_ctas_per_sm;
  out->dist_rows = best.dist_rows;
  out->dist_ctas_per_sm = best.dist_ctas_per_sm;
  out->streams = best.streams;
  out->coarse_gather = best.coarse_gather;
  out->shortlist = pick;
  return DETLSH_OK;
}

void detlsh_free(detlsh_index* idx) {
  if (!idx) return;
  cudaDeviceSynchronize();
  free_index(idx);
}

int detlsh_insert(detlsh_index* idx, const void* X, int64_t m, int32_t dtype, int32_t mem, void* stream) {
  g_err[0] = 0;
  DL_REQUIRE(idx, "NULL index");
  DL_REQUIRE(m >= 0, "m must be >= 0");
  if (m == 0) return DETLSH_OK;
  DL_REQUIRE(X, "NULL points");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(dtype == idx->dtype, "the points must have the index's dtype");
  DL_REQUIRE(idx->proj_mode == DETLSH_PROJ_FP32, "insertion needs an index built with the FP32 projection");
  const int64_t n = idx->n, n2 = n + m;
  DL_REQUIRE(n2 * (int64_t)idx->L < ((int64_t)1 << 32), "need (n+m)*L < 2^32");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = idx->K, L = idx->L, LK = K * L, d = (int)idx->d, Nr = idx->Nr;
  const size_t row = (size_t)d * dtype_size(dtype);
  // the points: one array of n+m rows, owned by the index from now on
  void* Xn = nullptr;
  DL_TRY(index_alloc(&Xn, row * n2, s));
  DL_CUDA(cudaMemcpyAsync(Xn, idx->X, row * n, cudaMemcpyDeviceToDevice, s));
  DL_CUDA(cudaMemcpyAsync(static_cast<char*>(Xn) + row * n, X, row * m,
                          mem == DETLSH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (idx->owns_x) cudaFreeAsync(const_cast<void*>(idx->X), s);
  idx->X = Xn;
  idx->owns_x = true;
  // Alg. 2 codes of the new points against the index's breakpoints, by the
  // projection kernel the build used (the new rows start 16-byte aligned
  // whenever the tensor-core paths apply: d*4 % 16 == 0 resp. d % 16 == 0)
  const void* Xm = static_cast<const char*>(Xn) + row * n;
  Scratch cnew;
  DL_TRY(cnew.alloc((size_t)m * LK, s));
  if (idx->Atf) {
    DL_TRY(launch_project_tf32(static_cast<const float*>(Xm), m, d, idx->Atf, LK, K, idx->E, idx->Rtab, idx->Rlo,
                               idx->Rinv, Nr, cnew.as<uint8_t>(), nullptr, 0, 0, idx->d_err, s));
  } else if (idx->Ab3) {
    DL_TRY(launch_project_bf16x3(static_cast<const uint8_t*>(Xm), m, d, idx->Ab3, LK, K, idx->E, idx->Rtab,
                                 idx->Rlo, idx->Rinv, Nr, cnew.as<uint8_t>(), nullptr, 0, 0, idx->d_err, s));
  } else {
    DL_TRY(launch_project_encode_t(Xm, dtype, m, d, idx->At, K, L, idx->E, idx->Rtab, idx->Rlo, idx->Rinv, Nr,
                                   cnew.as<uint8_t>(), s));
  }
  if (idx->Atf || idx->Ab3) DL_TRY(check_tc_error(idx->d_err, s));
  // codes [L][n+m][K]: per tree the old rows, then the new ones
  uint8_t* codes2 = nullptr;
  DL_TRY(index_alloc(&codes2, (size_t)n2 * LK, s));
  for (int t = 0; t < L; ++t) {
    DL_CUDA(cudaMemcpyAsync(codes2 + (size_t)t * n2 * K, idx->codes + (size_t)t * n * K, (size_t)n * K,
                            cudaMemcpyDeviceToDevice, s));
    DL_CUDA(cudaMemcpyAsync(codes2 + ((size_t)t * n2 + n) * K, cnew.as<uint8_t>() + (size_t)t * m * K,
                            (size_t)m * K, cudaMemcpyDeviceToDevice, s));
  }
  cudaFreeAsync(idx->codes, s);
  idx->codes = codes2;
  // Alg. 3 over all points (reading R3): the leaf tables are rebuilt
  void* old[] = {idx->leaf_ids, idx->leaf_pos, idx->leaf_base, idx->leaf_range, idx->leaf_plen,
                 idx->leaf_prefix, idx->leaf_lo, idx->leaf_hi, idx->leaf_tree};
  for (void* p : old)
    if (p) cudaFreeAsync(p, s);
  idx->leaf_ids = nullptr;
  idx->leaf_pos = nullptr;
  idx->leaf_base = nullptr;
  idx->leaf_range = nullptr;
  idx->leaf_plen = nullptr;
  idx->leaf_prefix = nullptr;
  idx->leaf_lo = nullptr;
  idx->leaf_hi = nullptr;
  idx->leaf_tree = nullptr;
  idx->n = n2;
  DL_TRY(index_alloc(&idx->leaf_ids, sizeof(uint32_t) * n2 * L, s));
  DL_TRY(build_leaves(idx, s));
  DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

int64_t detlsh_export_size(const detlsh_index* idx, int32_t what) {
  if (!idx) return DETLSH_EINVAL;
  const int64_t LK = (int64_t)idx->K * idx->L;
  switch (what) {
    case DETLSH_EXPORT_A: return sizeof(float) * LK * idx->d;
    case DETLSH_EXPORT_EDGES: return sizeof(float) * LK * (idx->Nr + 1);
    case DETLSH_EXPORT_CODES: return idx->n * LK;
    case DETLSH_EXPORT_LEAF_IDS: return sizeof(uint32_t) * idx->n * idx->L;
    case DETLSH_EXPORT_LEAF_BASE: return sizeof(int64_t) * (idx->L + 1);
    case DETLSH_EXPORT_LEAF_RANGE: return sizeof(uint32_t) * 2 * idx->total_leaves;
    case DETLSH_EXPORT_LEAF_PLEN:
    case DETLSH_EXPORT_LEAF_PREFIX: return idx->total_leaves * idx->K;
    case DETLSH_EXPORT_SAMPLE_PROJ: return sizeof(float) * LK * idx->n_s;
    case DETLSH_EXPORT_SAMPLE_IDS: return sizeof(int64_t) * idx->n_s;
    default: set_error("unknown export item %d", what); return DETLSH_EINVAL;
  }
}

int detlsh_export(const detlsh_index* idx, int32_t what, void* dst, int64_t bytes, int32_t mem,
                  void* stream) {
  g_err[0] = 0;
  DL_REQUIRE(idx && dst, "NULL argument");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  const int64_t need = detlsh_export_size(idx, what);
  if (need < 0) return (int)need;
  DL_REQUIRE(bytes >= need, "destination holds %lld bytes, %lld needed", (long long)bytes,
             (long long)need);
  const void* src = nullptr;
  switch (what) {
    case DETLSH_EXPORT_A: src = idx->A; break;
    case DETLSH_EXPORT_EDGES: src = idx->E; break;
    case DETLSH_EXPORT_CODES: src = idx->codes; break;
    case DETLSH_EXPORT_LEAF_IDS: src = idx->leaf_ids; break;
    case DETLSH_EXPORT_LEAF_BASE: src = idx->leaf_base; break;
    case DETLSH_EXPORT_LEAF_RANGE: src = idx->leaf_range; break;
    case DETLSH_EXPORT_LEAF_PLEN: src = idx->leaf_plen; break;
    case DETLSH_EXPORT_LEAF_PREFIX: src = idx->leaf_prefix; break;
    case DETLSH_EXPORT_SAMPLE_PROJ: src = idx->Ps; break;
    case DETLSH_EXPORT_SAMPLE_IDS: src = idx->sample; break;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DL_CUDA(cudaMemcpyAsync(dst, src, need,
                          mem == DETLSH_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

int detlsh_info(const detlsh_index* idx, int64_t* out, int32_t len) {
  if (!idx || !out) return DETLSH_EINVAL;
  const int64_t v[10] = {idx->n, idx->d, idx->dtype, idx->K, idx->L, idx->Nr, idx->max_leaf,
                         idx->n_s, idx->total_leaves, idx->max_leaf_count};
  const int m = std::min(len, 10);
  for (int i = 0; i < m; ++i) out[i] = v[i];
  return m;
}

int detlsh_project(const void* X, int64_t n, int32_t d, int32_t dtype, const float* A, int32_t LK,
                   float* P, int32_t mem, void* stream) {
  g_err[0] = 0;
  DL_REQUIRE(X && A && P, "NULL argument");
  DL_REQUIRE(dtype == DETLSH_F32 || dtype == DETLSH_U8, "bad dtype");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(n >= 0 && d >= 1 && d <= 65536 && LK >= 1 && LK <= kMaxLK, "bad sizes");
  if (n == 0) return DETLSH_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  In dX, dA;
  DL_TRY(dX.stage(X, (size_t)n * d * dtype_size(dtype), mem, s));
  DL_TRY(dA.stage(A, sizeof(float) * LK * d, mem, s));
  Scratch At;
  DL_TRY(At.alloc(sizeof(float) * LK * d, s));
  DL_TRY(transpose_hashes(static_cast<const float*>(dA.d), LK, d, At.as<float>(), s));
  Out dP;
  DL_TRY(dP.stage(P, sizeof(float) * n * LK, mem, s));
  DL_TRY(launch_project_t(dX.d, dtype, n, d, nullptr, At.as<float>(), LK, static_cast<float*>(dP.d), LK,
                          1, s));
  DL_TRY(dP.finish(s));
  DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

int detlsh_encode_values(const float* P, int64_t n, int32_t LK, const float* E, int32_t n_regions,
                         uint8_t* codes, int32_t mem, void* stream) {
  g_err[0] = 0;
  DL_REQUIRE(P && E && codes, "NULL argument");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(n >= 0 && LK >= 1 && LK <= kMaxLK, "bad sizes");
  DL_REQUIRE(is_pow2(n_regions) && n_regions >= 2 && n_regions <= 256, "bad n_regions");
  if (n == 0) return DETLSH_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  In dP, dE;
  DL_TRY(dP.stage(P, sizeof(float) * n * LK, mem, s));
  DL_TRY(dE.stage(E, sizeof(float) * LK * (n_regions + 1), mem, s));
  Out dc;
  DL_TRY(dc.stage(codes, (size_t)n * LK, mem, s));
  DL_TRY(launch_encode_values(static_cast<const float*>(dP.d), n, LK, static_cast<const float*>(dE.d),
                              n_regions, static_cast<uint8_t*>(dc.d), s));
  DL_TRY(dc.finish(s));
  DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

int detlsh_select_breakpoints(const float* Ps, int64_t n_s, int32_t LK, int32_t n_regions, float* E,
                              int32_t mem, void* stream) {
  g_err[0] = 0;
  DL_REQUIRE(Ps && E, "NULL argument");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(LK >= 1 && LK <= kMaxLK, "LK must be in [1, %d]", kMaxLK);
  DL_REQUIRE(is_pow2(n_regions) && n_regions >= 2 && n_regions <= 256, "bad n_regions");
  DL_REQUIRE(n_s >= n_regions && n_s * (int64_t)LK < ((int64_t)1 << 32), "bad n_s");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  In dP;
  DL_TRY(dP.stage(Ps, sizeof(float) * n_s * LK, mem, s));
  Out dE;
  DL_TRY(dE.stage(E, sizeof(float) * LK * (n_regions + 1), mem, s));
  DL_TRY(select_breakpoints(static_cast<const float*>(dP.d), n_s, LK, n_regions, static_cast<float*>(dE.d),
                            s));
  DL_TRY(dE.finish(s));
  DL_CUDA(cudaStreamSynchronize(s));
  return DETLSH_OK;
}

}  // extern "C"
