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
// (with that device current) on the first call made on that device.  The
// address belongs to the device's current CUDA context: the cache also keeps
// that context's id (cuCtxGetId, reached through the runtime's driver entry
// point, so the library needs no link against the driver library), and a
// call from another context -- after cudaDeviceReset, say -- looks the
// address up again instead of using a stale one.
//
// Every call shares the one array, and each call leaves its contents behind.
// No word of it has to start at zero: every scratch value a call reads was
// written earlier in the same call.  Calls that overlap on the GPU (on
// different streams, or from different host threads) race on the array and
// give undefined results; order them on one stream or synchronise.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "mg_common.cuh"

namespace mg {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
struct CachedAddress {
  unsigned long long ctx_id;  // context the address belongs to (0: none yet)
  void* ptr;
};
CachedAddress g_static_ptr[kMaxDevices] = {};

mg_status static_fail(mg_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

// Id of the calling thread's current CUDA context (0 if it cannot be read).
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device, looked up once
// per device and context (a context id that cannot be read forces a lookup).
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> g(g_static_mu);
  CachedAddress& c = g_static_ptr[dev];
  if (ctx == 0 || c.ctx_id != ctx || !c.ptr) {
    void* p = nullptr;
    // (makes the device's primary context current if the thread had none)
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    c.ptr = p;
    c.ctx_id = current_context_id();
  }
  *out = c.ptr;
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
