// mg_static.cu -- mg_chiral_truncate_static: the chiral truncation for
// callers that cannot allocate device memory.
//
// Who needs it: a host application that embeds this library but owns all of
// the device memory through its own pool allocator (a lattice-QCD framework's
// memory manager, say) cannot hand out a separate workspace, and a solver
// loop that must never stall the device cannot call cudaMalloc/cudaFree
// (both may synchronise the whole device).  This entry point takes only the
// inputs and outputs; its scratch is a fixed array compiled into the library.
//
// The array is a file-scope __device__ variable of kStaticScratchBytes
// (64 MiB): every GPU that loads the library reserves it until the process
// exits.  Host code only holds a host-side stand-in for the array's name, so
// its device address is looked up with cudaGetSymbolAddress once per device
// (with that device current) on the first call made on that device.
//
// Every call shares the one array, and each call leaves its contents behind.
// No word of it has to start at zero: every scratch value a call reads was
// written earlier in the same call.  Calls that overlap on the GPU (on
// different streams, or from different host threads) race on the array and
// give undefined results; order them on one stream or synchronise.
#include <cstdio>
#include <mutex>

#include "mg_common.cuh"

namespace mg {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

mg_status static_fail(mg_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

// Device address of the scratch array on the current device (looked up once
// per device).
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace mg

extern "C" mg_status mg_chiral_truncate_static(const mg_problem* prob, const void* psi,
                                               void* Uk, double* sigma, void* coarse_tv,
                                               int32_t* blk_flags, void* stream) {
  using namespace mg;
  // the scratch need is the one mg_workspace_size reports for the truncation
  const size_t need = mg_workspace_size(prob, MG_CALL_TRUNCATE);
  if (need == 0) return MG_ERR_INVALID;  // mg_last_error() already says why
  if (need > kStaticScratchBytes) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "mg_chiral_truncate_static: problem needs %zu bytes of scratch, more than the "
                  "built-in %zu (use mg_chiral_truncate with a caller workspace)",
                  need, kStaticScratchBytes);
    return static_fail(MG_ERR_INVALID, msg);
  }
  void* ws = nullptr;
  const cudaError_t e = static_scratch(&ws);
  if (e != cudaSuccess) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "mg_chiral_truncate_static: cudaGetSymbolAddress: %s",
                  cudaGetErrorString(e));
    return static_fail(MG_ERR_CUDA, msg);
  }
  return mg_chiral_truncate(prob, psi, Uk, sigma, coarse_tv, blk_flags, ws, need, stream);
}
