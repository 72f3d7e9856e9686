// Breakpoint selection that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: a serving
// process that must keep a fixed device-memory footprint (an allocation can
// fail under memory pressure in the middle of a request, and cudaFree
// synchronizes the device), or a host application whose own allocator owns all
// device memory. detlsh_select_breakpoints_noalloc gives them the Alg. 1
// breakpoint selection with its temporary storage taken from one fixed array
// compiled into this library instead of from the allocator.
//
// The array below is a file-scope __device__ variable: every GPU that loads
// the library holds it (kNoallocScratchBytes) until the process exits. Host
// code cannot use its name as a device address, so every call looks the
// address up with cudaGetSymbolAddress on the current device (cheap, and it
// allocates nothing). The first lookup on a device may load the library's
// device code there, so the first call on each device should come before any
// stream capture. Looking the address up per call also keeps it valid after a
// cudaDeviceReset, which destroys the context the array lived in. All calls
// share the array and it keeps the last call's contents; nothing in it needs
// to start at zero (every kernel writes the entries it later reads). Calls
// whose GPU work overlaps (for example on two streams) race on it and must be
// serialized by the caller.
#include "common.cuh"

namespace detlsh {

size_t select_breakpoints_ws_bytes(int64_t n_s, int LK);
int select_breakpoints_ws(const float* Ps, int64_t n_s, int LK, int Nr, float* E, void* ws,
                          size_t ws_bytes, cudaStream_t s);

namespace {

constexpr size_t kNoallocScratchBytes = 7u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// device address of the array on the current device
int scratch_address(void** out) {
  void* p = nullptr;
  DL_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = p;
  return DETLSH_OK;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace detlsh

using namespace detlsh;

extern "C" int detlsh_select_breakpoints_noalloc(const float* Ps, int64_t n_s, int32_t LK,
                                                 int32_t n_regions, float* E, void* stream) {
  clear_error();
  DL_REQUIRE(Ps && E, "NULL argument");
  DL_REQUIRE(LK >= 1 && LK <= kMaxLK, "LK must be in [1, %d]", kMaxLK);
  DL_REQUIRE(is_pow2(n_regions) && n_regions >= 2 && n_regions <= 256, "bad n_regions");
  DL_REQUIRE(n_s >= n_regions, "need n_s >= n_regions");
  DL_REQUIRE(n_s * (int64_t)LK <= DETLSH_NOALLOC_MAX_ITEMS,
             "n_s*LK = %lld exceeds the fixed scratch limit of %d values",
             (long long)(n_s * (int64_t)LK), DETLSH_NOALLOC_MAX_ITEMS);
  DL_TRY(require_device_ptr(Ps, "Ps"));
  DL_TRY(require_device_ptr(E, "E"));
  const size_t need = select_breakpoints_ws_bytes(n_s, LK);
  if (need > kNoallocScratchBytes) {
    set_error("scratch need %zu exceeds %zu bytes", need, kNoallocScratchBytes);
    return DETLSH_EINTERNAL;
  }
  void* ws = nullptr;
  DL_TRY(scratch_address(&ws));
  return select_breakpoints_ws(Ps, n_s, LK, n_regions, E, ws, kNoallocScratchBytes,
                               static_cast<cudaStream_t>(stream));
}
