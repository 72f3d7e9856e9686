// Query plans: the query pipeline of Alg. 7 with every buffer allocated once,
// optionally captured in a CUDA graph that one launch replays per batch.
//
// A plan owns the scratch of one batch of up to B queries plus input and
// output staging for it. detlsh_plan_query copies a chunk of at most B queries
// into the staging buffers, writes the chunk's size into a device word and
// runs the batch: with DETLSH_PLAN_GRAPH by one cudaGraphLaunch of the graph
// captured when the plan was made (every kernel reads the batch size from the
// device word, so the graph serves any size up to B), else by the same
// launches issued directly. Results do not depend on the route.
#include <algorithm>
#include <cmath>
#include <new>

#include "common.cuh"

struct detlsh_plan {
  const detlsh_index* idx = nullptr;
  detlsh::QueryShape sh{};
  double eps = 0.0, beta = 0.0;
  int k_max = 0;
  int flags = 0;
  void* scratch = nullptr;   // sh.bytes
  void* q_in = nullptr;      // [B][d] queries
  int32_t* k_in = nullptr;   // [B]
  float* c_in = nullptr;     // [B]
  float* r_in = nullptr;     // [B]
  int64_t* ids = nullptr;    // [B][k_max]
  float* dist = nullptr;     // [B][k_max]
  int32_t* stats = nullptr;  // [B][4]
  uint32_t* sticky = nullptr;  // argument error seen since the last status call
  bool vec4 = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_launches = 0, batches = 0, graph_kernels = 0;
};

namespace detlsh {
namespace {

__global__ void k_stick(const uint32_t* __restrict__ ctr_bad, uint32_t* sticky) {
  if (*ctr_bad) *sticky = 1u;
}

void release(detlsh_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  void* bufs[] = {p->scratch, p->q_in, p->k_in, p->c_in, p->r_in, p->ids, p->dist, p->stats, p->sticky};
  for (void* b : bufs)
    if (b) cudaFree(b);
}

// the batch's device-side pipeline, all on plan buffers (what the graph holds)
int enqueue_plan_batch(detlsh_plan* p, int64_t nqg, bool timed, cudaStream_t s) {
  PhaseTimer tm(s, timed);
  DL_TRY(check_batch_args(p->sh, p->scratch, p->k_in, p->c_in, p->r_in, s));
  k_stick<<<1, 1, 0, s>>>(query_ctr(p->sh, p->scratch) + CT_BAD, p->sticky);
  DL_LAUNCH();
  DL_TRY(enqueue_batch(p->idx, p->sh, p->scratch, p->q_in, 0, nqg, p->k_in, p->c_in, p->r_in, p->eps, p->beta,
                       p->ids, p->dist, p->stats, nullptr, 0, nullptr, p->vec4, timed ? &tm : nullptr, s));
  return tm.finish();
}

int capture(detlsh_plan* p) {
  cudaStream_t cs = nullptr;
  DL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int st = DETLSH_OK;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const int64_t l0 = detlsh_launch_count();
    st = enqueue_plan_batch(p, p->sh.B, false, cs);
    p->graph_kernels = detlsh_launch_count() - l0;
    e = cudaStreamEndCapture(cs, &g);
    if (st == DETLSH_OK && e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
  }
  cudaStreamDestroy(cs);
  if (st != DETLSH_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_error("graph capture failed: %s", cudaGetErrorString(e));
    return DETLSH_ECUDA;
  }
  p->graph = g;
  return DETLSH_OK;
}

}  // namespace
}  // namespace detlsh

using namespace detlsh;

extern "C" {

int detlsh_plan_create(const detlsh_index* idx, int64_t nq_max, int32_t k_max,
                       const detlsh_query_params* qp, int32_t flags, void* stream, detlsh_plan** out) {
  DL_REQUIRE(idx && out, "NULL argument");
  *out = nullptr;
  DL_REQUIRE(nq_max >= 1, "nq_max must be >= 1");
  DL_REQUIRE(k_max >= 1 && k_max <= kMaxTopK, "k_max must be in [1, %d]", kMaxTopK);
  DL_REQUIRE((flags & ~DETLSH_PLAN_GRAPH) == 0, "unknown plan flags");
  DL_REQUIRE(!qp || (!qp->cand_ids && !qp->qproj), "a plan does not export candidate lists or projections");
  double eps = qp ? qp->eps : 0.0;
  const double beta = qp ? qp->beta : 0.1;
  DL_REQUIRE(beta >= 0.0 && std::isfinite(beta), "beta must be finite and >= 0");
  if (!(eps > 0.0)) eps = detlsh_eps_lemma3(idx->K, idx->L);
  DL_REQUIRE(std::isfinite(eps) && eps > 0.0, "eps must be finite and > 0");
  const int32_t shortlist = qp ? qp->shortlist : 0;
  DL_REQUIRE(shortlist >= 0, "shortlist must be >= 0");
  QueryTuning tu;
  DL_TRY(tuning_from_params(qp, &tu));
  if (tu.batch == 0 || tu.batch > nq_max) tu.batch = nq_max;
  detlsh_plan* p = new (std::nothrow) detlsh_plan();
  if (!p) {
    set_error("host allocation failed");
    return DETLSH_ENOMEM;
  }
  p->idx = idx;
  p->eps = eps;
  p->beta = beta;
  p->k_max = k_max;
  p->flags = flags;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = query_shape(idx, nq_max, k_max, beta, shortlist, tu, &p->sh);
  const int64_t B = p->sh.B;
  const size_t qrow = (size_t)idx->d * (idx->dtype == DETLSH_U8 ? 1 : 4);
  auto grab = [&](void** ptr, size_t bytes) {
    if (st != DETLSH_OK) return;
    const cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      *ptr = nullptr;
      cudaGetLastError();
      set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
      st = DETLSH_ENOMEM;
    }
  };
  grab(&p->scratch, p->sh.bytes);
  grab(&p->q_in, qrow * B);
  grab(reinterpret_cast<void**>(&p->k_in), sizeof(int32_t) * B);
  grab(reinterpret_cast<void**>(&p->c_in), sizeof(float) * B);
  grab(reinterpret_cast<void**>(&p->r_in), sizeof(float) * B);
  grab(reinterpret_cast<void**>(&p->ids), sizeof(int64_t) * B * k_max);
  grab(reinterpret_cast<void**>(&p->dist), sizeof(float) * B * k_max);
  grab(reinterpret_cast<void**>(&p->stats), sizeof(int32_t) * B * 4);
  grab(reinterpret_cast<void**>(&p->sticky), sizeof(uint32_t));
  if (st == DETLSH_OK) {
    p->vec4 = query_vec4(idx, p->q_in);
    st = init_query_scratch(p->sh, p->scratch, s);
  }
  if (st == DETLSH_OK) {
    // staged rows past a batch's end are projected too (the graph's grids
    // are fixed); keep them defined
    if (cudaMemsetAsync(p->q_in, 0, qrow * B, s) != cudaSuccess ||
        cudaMemsetAsync(p->sticky, 0, sizeof(uint32_t), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("plan initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
      st = DETLSH_ECUDA;
    }
  }
  if (st == DETLSH_OK && (flags & DETLSH_PLAN_GRAPH)) st = capture(p);
  if (st != DETLSH_OK) {
    cudaStreamSynchronize(s);
    release(p);
    delete p;
    return st;
  }
  *out = p;
  return DETLSH_OK;
}

}  // extern "C"

namespace detlsh {

int64_t plan_capacity(const detlsh_plan* p) { return p->sh.B; }
size_t plan_bytes(const detlsh_plan* p) { return p->sh.bytes; }

int plan_enqueue(detlsh_plan* p, const void* Q, int64_t nq, const int32_t* k, const float* c,
                 const float* r_min, int64_t* out_ids, float* out_dist, int32_t* out_stats,
                 cudaMemcpyKind in, cudaMemcpyKind outk, cudaStream_t s) {
  const size_t qrow = (size_t)p->idx->d * (p->idx->dtype == DETLSH_U8 ? 1 : 4);
  const int64_t B = p->sh.B;
  const int km = p->k_max;
  for (int64_t q0 = 0; q0 < nq; q0 += B) {
    const int64_t m = std::min<int64_t>(B, nq - q0);
    DL_CUDA(cudaMemcpyAsync(p->q_in, static_cast<const char*>(Q) + q0 * qrow, m * qrow, in, s));
    DL_CUDA(cudaMemcpyAsync(p->k_in, k + q0, sizeof(int32_t) * m, in, s));
    DL_CUDA(cudaMemcpyAsync(p->c_in, c + q0, sizeof(float) * m, in, s));
    DL_CUDA(cudaMemcpyAsync(p->r_in, r_min + q0, sizeof(float) * m, in, s));
    DL_TRY(set_batch_size(p->sh, p->scratch, m, s));
    if (p->exec) {
      DL_CUDA(cudaGraphLaunch(p->exec, s));
      ++p->graph_launches;
    } else {
      DL_TRY(enqueue_plan_batch(p, m, true, s));
    }
    ++p->batches;
    DL_CUDA(cudaMemcpyAsync(out_ids + q0 * km, p->ids, sizeof(int64_t) * m * km, outk, s));
    DL_CUDA(cudaMemcpyAsync(out_dist + q0 * km, p->dist, sizeof(float) * m * km, outk, s));
    if (out_stats)
      DL_CUDA(cudaMemcpyAsync(out_stats + q0 * 4, p->stats, sizeof(int32_t) * m * 4, outk, s));
  }
  return DETLSH_OK;
}

}  // namespace detlsh

extern "C" {

int detlsh_plan_query(detlsh_plan* p, const void* Q, int64_t nq, const int32_t* k, const float* c,
                      const float* r_min, int64_t* out_ids, float* out_dist, int32_t* out_stats,
                      int32_t mem, void* stream) {
  DL_REQUIRE(p != nullptr, "plan is NULL");
  DL_REQUIRE(mem == DETLSH_MEM_HOST || mem == DETLSH_MEM_DEVICE, "bad mem flag");
  DL_REQUIRE(nq >= 0, "nq must be >= 0");
  if (nq == 0) return DETLSH_OK;
  DL_REQUIRE(Q && k && c && r_min && out_ids && out_dist, "NULL query argument");
  if (mem == DETLSH_MEM_HOST) {
    for (int64_t i = 0; i < nq; ++i) {
      DL_REQUIRE(k[i] >= 1 && k[i] <= p->k_max, "k[%lld] must be in [1, k_max]", (long long)i);
      DL_REQUIRE(std::isfinite(c[i]) && c[i] > 1.0f, "c[%lld] must be finite and > 1", (long long)i);
      DL_REQUIRE(std::isfinite(r_min[i]), "r_min[%lld] must be finite", (long long)i);
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind in = mem == DETLSH_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind outk = mem == DETLSH_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  DL_TRY(plan_enqueue(p, Q, nq, k, c, r_min, out_ids, out_dist, out_stats, in, outk, s));
  if (mem == DETLSH_MEM_HOST) return detlsh_plan_status(p, stream);
  return DETLSH_OK;
}

int detlsh_plan_status(detlsh_plan* p, void* stream) {
  DL_REQUIRE(p != nullptr, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t h = 0;
  DL_CUDA(cudaMemcpyAsync(&h, p->sticky, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DL_CUDA(cudaStreamSynchronize(s));
  if (h) {
    DL_CUDA(cudaMemsetAsync(p->sticky, 0, sizeof(uint32_t), s));
    DL_CUDA(cudaStreamSynchronize(s));
    set_error("a batch had a query without 1 <= k <= k_max, finite c > 1, finite r_min; it ran empty");
    return DETLSH_EINVAL;
  }
  if (p->idx->proj_mode == DETLSH_PROJ_BF16) return check_tc_error(p->idx->d_err, s);
  return DETLSH_OK;
}

int detlsh_plan_info(const detlsh_plan* p, int64_t* out5) {
  DL_REQUIRE(p && out5, "NULL argument");
  out5[0] = p->sh.B;
  out5[1] = (int64_t)p->sh.bytes;
  out5[2] = p->graph_launches;
  out5[3] = p->batches;
  out5[4] = p->graph_kernels;
  return DETLSH_OK;
}

void detlsh_plan_destroy(detlsh_plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  release(p);
  delete p;
}

}  // extern "C"
