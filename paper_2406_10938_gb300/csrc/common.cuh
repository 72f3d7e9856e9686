// Internal declarations shared by the translation units of libdetlsh.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "../../include/detlsh.h"

namespace detlsh {

constexpr int kMaxK = 16;
constexpr int kMaxL = 16;
constexpr int kMaxLK = 256;
constexpr int kRoundCap = 256;   // rounds of Alg. 7; the last one has infinite radius
constexpr int kMaxTopK = 1024;

// ---- the checked build (compiled with DETLSH_CHECKED): data-dependent indices
// of the query kernels are checked on the device; a failed check skips the
// access and records (failures, first site, first index) in a status word of
// its translation unit, which detlsh_check_status collects. In the normal
// build DL_CHECK is true and the checks vanish.
#ifdef DETLSH_CHECKED
static __device__ unsigned int g_dl_check[4];
__device__ __forceinline__ bool dl_check(bool ok, unsigned site, unsigned long long index) {
  if (!ok && atomicAdd(&g_dl_check[0], 1u) == 0u) {
    g_dl_check[1] = site;
    g_dl_check[2] = (unsigned)index;
    g_dl_check[3] = (unsigned)(index >> 32);
  }
  return ok;
}
int register_check_reader(int (*read)(unsigned int* words));
// this translation unit's status word: copied out, then cleared
static int read_check_words(unsigned int* w) {
  if (cudaMemcpyFromSymbol(w, g_dl_check, sizeof(unsigned int) * 4) != cudaSuccess) return -1;
  const unsigned int zero[4] = {0u, 0u, 0u, 0u};
  if (cudaMemcpyToSymbol(g_dl_check, zero, sizeof(zero)) != cudaSuccess) return -1;
  return 0;
}
static const int g_dl_check_registered = register_check_reader(&read_check_words);
#define DL_CHECK(cond, site, index) (::detlsh::dl_check((cond), (site), (unsigned long long)(index)))
#else
#define DL_CHECK(cond, site, index) true
#endif

void set_error(const char* fmt, ...);
void clear_error();
void count_launch();
// DETLSH_EINVAL (with the message) unless p is a device or managed address
int require_device_ptr(const void* p, const char* name);

// Per-phase device times of the last build/query on this thread (tracing).
enum TracePhase {
  TR_SAMPLE_PROJ = 0, TR_BREAKPOINTS, TR_ENCODE, TR_LEAVES, TR_QUERY_PROJ, TR_LB, TR_DIST,
  TR_DIST_LAUNCHES, TR_LB_LAUNCHES, TR_BUILD_TOTAL, TR_QUERY_TOTAL, TR_WALK, TR_FINALIZE, TR_BUCKET,
  TR_LEAF_ROOT, TR_LEAF_GATHER, TR_LEAF_LEVELS, TR_LEAF_ITERS, TR_GROUP, TR_COUNT
};
bool trace_on();
void trace_reset(int first, int last);
void trace_add(int phase, double v);

// Records CUDA events around phases on one stream when tracing is on.
class PhaseTimer {
 public:
  // records only while tracing is on and `allow` (false inside a graph capture)
  explicit PhaseTimer(cudaStream_t s, bool allow = true);
  ~PhaseTimer();
  void begin(int phase);
  void end();
  int finish();  // synchronizes and adds the elapsed times to the trace
 private:
  static constexpr int kMax = 256;
  cudaStream_t s_;
  bool on_;
  int n_ = 0, open_ = -1;
  int phase_[kMax];
  cudaEvent_t a_[kMax], b_[kMax];
};

#define DL_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::detlsh::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                          __FILE__, __LINE__);                                     \
      return e_ == cudaErrorMemoryAllocation ? DETLSH_ENOMEM : DETLSH_ECUDA;       \
    }                                                                              \
  } while (0)

#define DL_LAUNCH()                                                                \
  do {                                                                             \
    ::detlsh::count_launch();                                                      \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) {                                                       \
      ::detlsh::set_error("kernel launch failed: %s (%s:%d)",                      \
                          cudaGetErrorString(e_), __FILE__, __LINE__);             \
      return DETLSH_ECUDA;                                                         \
    }                                                                              \
  } while (0)

#define DL_REQUIRE(cond, ...)                                                      \
  do {                                                                             \
    if (!(cond)) {                                                                 \
      ::detlsh::set_error(__VA_ARGS__);                                            \
      return DETLSH_EINVAL;                                                        \
    }                                                                              \
  } while (0)

#define DL_TRY(expr)                                                               \
  do {                                                                             \
    int s_ = (expr);                                                               \
    if (s_ != DETLSH_OK) return s_;                                                \
  } while (0)

// Stream-ordered scratch allocation that frees itself on scope exit.
// The library's stream-ordered pool on the current device (created on first
// use; it keeps up to 16 GiB of freed scratch mapped between calls), or null
// when a pool cannot be created (then the device's default pool serves).
cudaMemPool_t scratch_pool();

struct Scratch {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  Scratch(Scratch&& o) noexcept : p(o.p), s(o.s) { o.p = nullptr; }
  Scratch& operator=(Scratch&& o) noexcept {
    if (this != &o) {
      if (p) cudaFreeAsync(p, s);
      p = o.p;
      s = o.s;
      o.p = nullptr;
    }
    return *this;
  }
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
  int alloc(size_t bytes, cudaStream_t stream) {
    s = stream;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = scratch_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, stream) : cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
      return DETLSH_ENOMEM;
    }
    return DETLSH_OK;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Index arrays come from the same stream-ordered pool (fast once the pool
// holds memory, e.g. from an earlier build); free_index synchronises the
// device and returns them to it.
int index_alloc_raw(void** p, size_t bytes, cudaStream_t s);
template <class T>
int index_alloc(T** p, size_t bytes, cudaStream_t s) {
  void* v = nullptr;
  const int r = index_alloc_raw(&v, bytes, s);
  *p = static_cast<T*>(v);
  return r;
}

}  // namespace detlsh

// The index. Device arrays unless marked _h.
struct detlsh_index {
  int64_t n = 0;
  int32_t d = 0, dtype = 0, K = 0, L = 0, Nr = 0, bits = 0, max_leaf = 0;
  int64_t n_s = 0;
  int32_t device = 0;
  int32_t proj_mode = 0;
  int32_t flags = 0;                // detlsh_params.flags of the build
  void* Xb = nullptr;               // [n][d] BF16 copy of X (BF16 projection mode)
  void* Ab = nullptr;               // [N][d] BF16 hash vectors, N = L*K rounded up to 16
  float* Atf = nullptr;             // [2][N][d] TF32 split of A (FP32 mode on the tensor cores)
  void* Ab3 = nullptr;              // [3][N][d] BF16 three-part split of A (uint8 points on the tensor cores)
  int* d_err = nullptr;             // error word of the tensor-core kernel
  bool owns_x = true;
  const void* X = nullptr;          // [n][d] f32 or u8
  float* A = nullptr;               // [LK][d]
  float* At = nullptr;              // [d][LK] (transposed A)
  float* E = nullptr;               // [LK][Nr+1]
  uint8_t* Rtab = nullptr;          // [LK][kRegionRow] region search tables of E
  float* Rlo = nullptr;             // [LK]
  float* Rinv = nullptr;            // [LK]
  float* Ps = nullptr;              // [LK][n_s]
  int64_t* sample = nullptr;        // [n_s] sampled point ids (Alg. 1)
  uint8_t* codes = nullptr;         // [L][n][K]
  uint32_t* leaf_ids = nullptr;     // [L][n]
  uint32_t* leaf_pos = nullptr;     // [L][n] each entry's point as its position in tree 0's leaf order
                                    // (built for large n only: the walk's dedup bitmap index)
  int64_t* leaf_base = nullptr;     // [L+1]
  uint32_t* leaf_range = nullptr;   // [total][2] (start within tree, count)
  uint8_t* leaf_plen = nullptr;     // [total][K]
  uint8_t* leaf_prefix = nullptr;   // [total][K]
  uint8_t* leaf_lo = nullptr;       // [total][K] lowest code of the leaf box
  uint8_t* leaf_hi = nullptr;       // [total][K] highest code of the leaf box
  uint16_t* leaf_tree = nullptr;    // [total] tree of each leaf
  float* xn2 = nullptr;             // [n] squared norms of the BF16 rows (BF16 mode)
  uint32_t* chunk_base = nullptr;   // [total+1] first chunk of each leaf (BF16 mode)
  uint32_t* chunk_leaf = nullptr;   // [n_chunks] leaf of each chunk
  int64_t n_chunks = 0;             // leaf chunks of lm_nmax - 32 points
  int32_t lm_nmax = 0;              // points per tile of the leaf-major coarse distances (64 or 128)
  int64_t total_leaves = 0;
  int64_t max_leaf_count = 0;
  int64_t leaf_base_h[detlsh::kMaxL + 1] = {0};
};

namespace detlsh {

// ---- the method's random draws from a seed (rng.cpp, host code)
void draw_hashes(uint64_t seed, int64_t count, float* A);
void draw_sample(uint64_t seed, int64_t n, int64_t n_s, int64_t* ids);

// ---- region search tables (Alg. 2 encoding, project.cu)
// For projected dimension h with interior breakpoints e_1 <= ... <= e_{Nr-1}:
// cell(x) = round(clamp((x - lo) * inv, 0, kRegionCells-1)) with lo = e_1 and
// inv = kRegionCells / (e_{Nr-1} - e_1) (0 when that is not finite and
// positive), every step rounded to nearest in FP32 and never contracted (the
// final rounding to an integer by adding 1.5 * 2^23). Each step is monotone
// (a NaN clamps to 0), so cell is monotone non-decreasing in x:
// for p in cell c every e_z of a lower cell is < p and every e_z of a higher
// cell is > p. With tab[c] = #{z >= 1 : cell(e_z) < c} (c = 0..kRegionCells,
// padded with Nr-1), the code of Alg. 2 is
//   #{z : e_z <= p} = tab[c] + #{z : cell(e_z) = c, e_z <= p},
// a search among the breakpoints of p's own cell only, whatever the rounding.
constexpr int kRegionCells = 256;
constexpr int kRegionRow = kRegionCells + 4;

__device__ __forceinline__ int region_cell(float lo, float inv, float p) {
  const float f = fminf(fmaxf(__fmul_rn(__fsub_rn(p, lo), inv), 0.f), (float)(kRegionCells - 1));
  return __float_as_int(__fadd_rn(f, 12582912.f)) & 0x1ff;
}

// The common case, at most three breakpoints in p's cell: three independent
// compares against e[min(a+j, b)], a = tab[c], b = tab[c+1] (e sorted, so the
// true compares form a prefix and the last true index is the code; e[a] < p
// when a >= 1, so a clamped index never overcounts). slow is set when the
// cell holds more than three breakpoints; region_slow then gives the code.
__device__ __forceinline__ int region_fast_part(const float* e, const uint8_t* t, float lo, float inv, float p,
                                                bool& slow) {
  const int c = region_cell(lo, inv, p);
  const int a = t[c], b = t[c + 1];
  const int i1 = min(a + 1, b), i2 = min(a + 2, b), i3 = min(a + 3, b);
  const float x1 = e[i1], x2 = e[i2], x3 = e[i3];
  int r = a;
  r = x1 <= p ? i1 : r;
  r = x2 <= p ? i2 : r;
  r = x3 <= p ? i3 : r;
  slow = b - a > 3;
  return r;
}
// Binary search for the code among the breakpoints of p's cell.
__device__ __forceinline__ int region_slow(const float* e, const uint8_t* t, float lo, float inv, float p) {
  const int c = region_cell(lo, inv, p);
  int a = t[c], b = t[c + 1];
  while (a < b) {
    const int m = (a + b + 1) >> 1;
    if (e[m] <= p) a = m;
    else b = m - 1;
  }
  return a;
}
// code = #{z in 1..Nr-1 : e[z] <= p} for the sorted row e[0..Nr-1] (e[0]
// only read when no breakpoint lies below p's cell) and its table row t.
__device__ __forceinline__ int region_fast(const float* e, const uint8_t* t, float lo, float inv, float p) {
  bool slow;
  const int r = region_fast_part(e, t, lo, inv, p, slow);
  return slow ? region_slow(e, t, lo, inv, p) : r;
}
// Sixteen codes (dimensions h0..h0+15, rows es floats apart from e0) packed
// four per word: the fast parts of all sixteen first, so that their loads
// overlap, then the rare crowded cells.
__device__ __forceinline__ void region_codes16(const float* e0, int es, const uint8_t* t0, const float* lo,
                                               const float* inv, const float* v, uint32_t* w) {
  int r[16];
  uint32_t slow = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    bool sl;
    r[i] = region_fast_part(e0 + i * es, t0 + i * kRegionRow, lo[i], inv[i], v[i], sl);
    slow |= (uint32_t)sl << i;
  }
  if (slow) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if ((slow >> i) & 1u) r[i] = region_slow(e0 + i * es, t0 + i * kRegionRow, lo[i], inv[i], v[i]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    w[q] = (uint32_t)r[4 * q] | ((uint32_t)r[4 * q + 1] << 8) | ((uint32_t)r[4 * q + 2] << 16) |
           ((uint32_t)r[4 * q + 3] << 24);
}

// tab [LK][kRegionRow], lo [LK], inv [LK] from E [LK][Nr+1].
int build_region_tables(const float* E, int LK, int Nr, uint8_t* tab, float* lo, float* inv, cudaStream_t s);

// ---- projection / encoding (project.cu)
// At [d][LK] = transpose of A [LK][d].
int transpose_hashes(const float* A, int LK, int d, float* At, cudaStream_t s);
// P[o*p_so + r*p_sr] = sum_t A[r][t] * X[rows ? rows[o] : o][t], FP32 (At transposed).
int launch_project_t(const void* X, int dtype, int64_t n, int d, const int64_t* rows,
                     const float* At, int LK, float* P, int64_t p_so, int64_t p_sr,
                     cudaStream_t s);
// Same projection, then Alg. 2 against E [LK][Nr+1] (with its region tables);
// writes codes [L][n][K].
int launch_project_encode_t(const void* X, int dtype, int64_t n, int d, const float* At,
                            int K, int L, const float* E, const uint8_t* Rtab, const float* Rlo,
                            const float* Rinv, int Nr, uint8_t* codes,
                            cudaStream_t s);
int launch_encode_values(const float* P, int64_t n, int LK, const float* E, int Nr,
                         uint8_t* codes, cudaStream_t s);

// ---- tensor-core projection (project_tc.cu)
int to_bf16(const void* X, int dtype, int64_t count, void* Y, cudaStream_t s);
int gather_rows_bf16(const void* Xb, int d, const int64_t* ids, int64_t m, void* Y, cudaStream_t s);
int launch_project_tc(const void* Xb, int64_t rows, int d, const void* Ab, int LK, int K,
                      const float* E, const uint8_t* Rtab, const float* Rlo, const float* Rinv, int Nr,
                      uint8_t* codes, float* P, int64_t p_so, int64_t p_sr, int* d_err, cudaStream_t s);
int check_tc_error(int* d_err, cudaStream_t s);
// limit of each bounded wait of the tensor-core kernels (ns)
unsigned long long tc_wait_limit_ns();

// ---- leaf-major coarse distances on the tensor cores (dist_lm.cu)
// BF16 indexes: squared norms of the BF16 rows, leaf chunk tables
int build_lm_tables(detlsh_index* idx, cudaStream_t s);
// sort keys of the records (per leaf chunk, its 32-point windows)
int64_t lm_sort_keys(int64_t n_chunks);
// one batch's buffers: the walk's records [B][cap], their chunk sort, units
struct LmBatch {
  const void* qb16;         // [B][d] BF16 queries
  int64_t nqg;              // grid bound on the batch size
  const uint32_t* nqd;      // batch size (device)
  const uint4* rec;         // [B][cap] records
  int64_t cap;
  const uint32_t* meta;
  int mq_words, mq_nrec;
  float* qn;                // [B]
  uint32_t *khist, *kcur, *koff;   // [lm_sort_keys(n_chunks)] (+1 for koff)
  uint32_t *ucnt, *uoff;           // [n_chunks] (+1 for uoff)
  uint32_t* nunits;         // device word
  uint4* srec;              // records by chunk
  uint32_t* sq;             // their queries
  uint4* units;
  void* scan_ws;
  size_t scan_ws_bytes;
  float* d2;                // [B][cap]
};
int enqueue_coarse_lm(const detlsh_index* idx, const LmBatch& b, cudaStream_t s);
// FP32 inputs on the tensor cores (TF32 split, FP32-faithful): Asplit holds
// a_big [N][d] then a_small [N][d] (N = L*K rounded up to 16), from split_tf32.
bool tf32_eligible(int dtype, int d, int LK);
int split_tf32(const float* A, int LK, int d, float* Asplit, cudaStream_t s);
int gather_rows_f32(const float* X, int d, const int64_t* ids, int64_t m, float* Y, cudaStream_t s);
// uint8 inputs on the tensor cores: the points widened to BF16 (exact) in the
// kernel against A split into three BF16 parts (Ab3 [3][N][d], from
// split_bf16x3), FP32-faithful.
bool bf16x3_eligible(int dtype, int d, int LK);
int split_bf16x3(const float* A, int LK, int d, void* Ab3, cudaStream_t s);
int gather_rows_u8(const uint8_t* X, int d, const int64_t* ids, int64_t m, uint8_t* Y, cudaStream_t s);
int launch_project_bf16x3(const uint8_t* X, int64_t rows, int d, const void* Ab3, int LK, int K, const float* E,
                          const uint8_t* Rtab, const float* Rlo, const float* Rinv, int Nr, uint8_t* codes,
                          float* P, int64_t p_so, int64_t p_sr, int* d_err, cudaStream_t s);
int launch_project_tf32(const float* X, int64_t rows, int d, const float* Asplit, int LK, int K, const float* E,
                        const uint8_t* Rtab, const float* Rlo, const float* Rinv, int Nr, uint8_t* codes,
                        float* P, int64_t p_so, int64_t p_sr, int* d_err, cudaStream_t s);

// ---- sorting / scans (sort.cu)
// Stable LSD radix sort of (key, value) pairs on key bits [bit_lo, bit_hi).
int radix_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n,
                     int bit_lo, int bit_hi, uint32_t* keys_out, uint32_t* vals_out,
                     cudaStream_t s);
// Exclusive prefix sum of n uint32 values into uint32 (sum must fit) ; total to *d_total.
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                       cudaStream_t s);

// ---- breakpoints (breakpoints.cu)
// Ps [LK][n_s] -> E [LK][Nr+1].
int select_breakpoints(const float* Ps, int64_t n_s, int LK, int Nr, float* E,
                       cudaStream_t s);

// ---- leaves (leaves.cu)
int build_leaves(detlsh_index* idx, cudaStream_t s);

// ---- scans and sorts with caller storage (sort.cu)
size_t scan_ws_bytes(int64_t n);
int exclusive_scan_u32_ws(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total, void* ws,
                          size_t ws_bytes, cudaStream_t s);
size_t radix_ws_bytes(int64_t n, int bit_lo, int bit_hi);
int radix_sort_pairs_ws(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n, int bit_lo,
                        int bit_hi, uint32_t* keys_out, uint32_t* vals_out, void* ws, size_t ws_bytes,
                        cudaStream_t s);

// ---- query (query.cu)
// Launch shapes of the query pipeline (results do not depend on them).
struct QueryTuning {
  int64_t batch = 0;         // queries per batch; 0: sized from free device memory
  int walk_ctas_per_sm = 0;  // walk CTAs per SM, 1..4; 0: as many as fit
  int dist_rows = 1024;      // candidate rows per distance work item (multiple of 64)
  int dist_ctas_per_sm = 0;  // persistent distance CTAs per SM, 1..4; 0: 4 (3 for the BF16 gather)
  int streams = 0;           // 2: batches alternate between two streams; 0 or 1: one stream
  int coarse_gather = 0;     // shortlist mode: 1 gathers each candidate's row (no leaf-major tensor cores)
  int id_bucket_log2 = 0;    // gather by point-id range of 2^x rows; 0: automatic; -1: in walk order
};

// Sizes and scratch layout (byte offsets into one device block) of a batch.
struct QueryShape {
  int64_t B, cap, TL, RL, words, max_tree_leaves, items_per_q, nblk;
  int64_t nsm = 0;   // SMs of the device
  int LK, L, wgrid, dgrid, dist_rows, tkc, k_max, shortlist, rq;
  bool smem_bitmap;
  bool lm = false;           // coarse distances by leaf on the tensor cores
  int64_t nk = 0, max_units = 0;
  // gather by point-id range: log2 rows per range (0: walk order), ranges
  int bshift = 0;
  int64_t nbk = 0;
  size_t o_pairs = 0, o_bcnt = 0, o_boffq = 0, o_icnt = 0, o_ioff = 0, o_bscan = 0, bscan_bytes = 0;
  size_t o_rec = 0, o_srec = 0, o_sq = 0, o_qn = 0, o_khist = 0, o_kcur = 0, o_koff = 0, o_ucnt = 0, o_uoff = 0,
         o_units = 0, o_scanws = 0, scanws_bytes = 0;
  size_t wl_total, bk_smem, bytes;
  size_t o_ctr, o_qp, o_qb16, o_qf, o_lb, o_mm, o_lround, o_hist, o_boff, o_list, o_cand, o_d2,
      o_rend, o_thr, o_meta, o_wsnew, o_wsbm, o_wspos, o_items, o_qk, o_qsort, qsort_bytes, o_blkmin, o_blist;
};

// control words of a batch (uint32, at QueryShape::o_ctr): queries in the
// batch, walk query counter, distance items queued, argument error flag,
// distance items taken
enum { CT_NQ = 0, CT_WORK, CT_QTAIL, CT_BAD, CT_HEAD, CT_NUNITS, CT_WORDS = 64 };

// the launch shapes of detlsh_query_params::tuning (defaults for zero fields)
int tuning_from_params(const detlsh_query_params* qp, QueryTuning* tu);
int query_shape(const detlsh_index* idx, int64_t nq, int k_max, double beta, int shortlist,
                const QueryTuning& tu, QueryShape* out);
int init_query_scratch(const QueryShape& sh, void* base, cudaStream_t s);
uint32_t* query_ctr(const QueryShape& sh, void* base);
// the batch size lives in device memory (one captured graph serves any size
// up to the shape's B); set it before the batch's kernels
int set_batch_size(const QueryShape& sh, void* base, int64_t nq, cudaStream_t s);
// device-side argument check; a batch with a bad argument runs empty and
// leaves its error word set
int check_batch_args(const QueryShape& sh, void* base, const int32_t* k, const float* c,
                     const float* r_min, cudaStream_t s);
// the query pipeline of one batch: queries q0.. of Q, k, c, r_min and the
// outputs; nqg bounds the grids (the batch size word may be smaller)
int enqueue_batch(const detlsh_index* idx, const QueryShape& sh, void* base, const void* Q, int64_t q0,
                  int64_t nqg, const int32_t* k, const float* c, const float* r_min, double eps,
                  double beta, int64_t* out_ids, float* out_dist, int32_t* out_stats,
                  uint32_t* cand_ids, int64_t cand_cap, float* qproj, bool vec4, PhaseTimer* timer,
                  cudaStream_t s);
bool query_vec4(const detlsh_index* idx, const void* Q);

// ---- plans (plan.cu), for the server
int64_t plan_capacity(const detlsh_plan* p);
size_t plan_bytes(const detlsh_plan* p);
// a plan batch from caller buffers with the given copy kinds (cudaMemcpyDefault
// for pinned host memory), fully asynchronous on s; no host argument checks
int plan_enqueue(detlsh_plan* p, const void* Q, int64_t nq, const int32_t* k, const float* c,
                 const float* r_min, int64_t* out_ids, float* out_dist, int32_t* out_stats,
                 cudaMemcpyKind in, cudaMemcpyKind outk, cudaStream_t s);
int run_query(const detlsh_index* idx, const void* Q, int64_t nq, const int32_t* k,
              const float* c, const float* r_min, int k_max, double eps, double beta,
              int64_t* out_ids, float* out_dist, int32_t* out_stats, uint32_t* cand_ids,
              int64_t cand_cap, float* qproj, int shortlist, const QueryTuning& tu, cudaStream_t s);

// ---- host math (chi2.cpp)
double chi2_upper_quantile(double alpha, int K);

}  // namespace detlsh
