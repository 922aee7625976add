// mg_common.cuh -- internal definitions shared by the CUDA translation units
// of the chiral rank-k multigrid setup (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/mg.h"

namespace mg {

// ---------------------------------------------------------------------------
// problem geometry, validated on the host
// ---------------------------------------------------------------------------
struct Geom {
  int L[4];       // fine extents
  int b[4];       // block extents
  int Lc[4];      // coarse extents
  long V;         // fine volume
  int nb;         // sites per block
  long nblk;      // number of blocks = coarse volume
  int m;          // test vectors m'
  int k;          // kept per chirality
  int niter;      // smoother iterations
  double m0, xi;  // mass, anisotropy
  float hw[4];    // hop weights -1/2 w_mu
  float diag;     // m0 + sum_mu w_mu
  int prec;       // mg_precision
  int rps = 6;    // rows per site and chirality of the level's vectors (6 = 2 spins x 3
                  // colours at the fine level, k1 at the second level)
  int cps = 12;   // complex components per site (2 rps)
};

constexpr int kMaxM = 64;  // largest m' this build supports
constexpr int kMaxK = 32;  // largest k this build supports

// ---------------------------------------------------------------------------
// workspace layout (byte offsets, 256-aligned), see mg_abi.cu
// ---------------------------------------------------------------------------
struct SmoothWs {
  size_t ra, wa, ps, part, alpha, scale, bytes;
  size_t rb, alpha_b;  // second r buffer and a array (the deferred psi update)
};
struct TruncWs {
  size_t gram, r1, z1, w2, hm, flags, q1, qmax, bytes;  // q1, qmax: 0 unless tensor cores
};

// operator of a level l >= 1: a nearest-neighbour stencil (X, Y) with n = 2 nc
// components per site on the periodic lattice L (mg_level2.cu)
struct StencilGeom {
  int L[4];
  long V;
  int n;
};
struct StencilSmoothWs {
  size_t r, w, part, alpha, scale, bytes;
};

SmoothWs smooth_ws_layout(const Geom& g);
StencilSmoothWs stencil_smooth_ws_layout(const StencilGeom& sg, int m);
TruncWs trunc_ws_layout(const Geom& g);

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Sets the message mg_last_error() returns on the calling thread.
void set_last_error(const char* msg);

// Runs a set-up step (cudaFuncSetAttribute, which applies to the current
// device only) once per device, from any number of host threads.
constexpr int kMaxDevices = 64;
class PerDeviceOnce {
 public:
  template <typename F>
  void run(F f) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
      f();  // unusual device index: set up on every call (cheap)
      return;
    }
    std::lock_guard<std::mutex> g(mu_);
    if (!done_[dev]) {
      f();
      done_[dev] = true;
    }
  }

 private:
  std::mutex mu_;
  bool done_[kMaxDevices] = {};
};

// Tuned slab width of the smoother passes for g's shape (0: not tuned), and
// whether the calling thread is capturing a batch graph (no timing events).
int tuned_pairs(const Geom& g);
void set_tuned_pairs(const Geom& g, int pairs);
bool timing_suspended();

// Validates a problem and fills the derived geometry (mg_abi.cu).
mg_status make_geom(const mg_problem* p, Geom* g);

// ---------------------------------------------------------------------------
// optional per-kernel timing (mg_timing_enable): a scope records a CUDA event
// pair around the launches it encloses on stream s
// ---------------------------------------------------------------------------
int timing_begin(const char* name, cudaStream_t s);
void timing_end(int token, cudaStream_t s);
struct TimedScope {
  int tok;
  cudaStream_t s;
  TimedScope(const char* name, cudaStream_t st) : tok(timing_begin(name, st)), s(st) {}
  ~TimedScope() { timing_end(tok, s); }
};

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files); each returns cudaGetLastError()
// ---------------------------------------------------------------------------
cudaError_t launch_clover(const Geom& g, double csw, const float2* U, float2* C,
                          cudaStream_t s);

cudaError_t launch_dirac(const Geom& g, const float2* U, const float2* C, const float2* in,
                         float2* out, char* ws, cudaStream_t s);

cudaError_t launch_smoother(const Geom& g, const float2* U, const float2* C,
                            const float2* psi0, float2* psi, char* ws, cudaStream_t s);

// Synchronises s, then reads and clears the device status word (bit 0: a
// smoother pass gave up waiting for its staged input; bit 1: a tensor-core
// contraction gave up waiting for its MMAs).
cudaError_t read_device_status(int* out, cudaStream_t s);
// Device address of that word (nullptr on a CUDA error).
int* device_status_word();
// mg_selftest_timeout's kernel.
cudaError_t launch_selftest_timeout(int polls, cudaStream_t s);

// Tensor-core (tcgen05) contractions of the truncation (mg_tc.cu), per
// block-chirality bc: G[bc] = A^dag A (BF16 operands, or FP16 hi/lo split with
// three products), and C[bc] = A B[bc] (FP16 hi/lo split).  A's rows are
// gathered from psi by the block geometry (gather) or contiguous [bc][K][m'].
bool tc_supported(const Geom& g);
cudaError_t launch_tc_gram(const Geom& g, const float2* A, bool gather, bool fp16x3,
                           const float* bound, double2* G, int* status, cudaStream_t s,
                           const char* name);
// Galerkin coarsening on the tensor cores (FP16 hi/lo operands, FP32 accumulation).
bool tc_coarsen_supported(const Geom& g);
cudaError_t launch_tc_coarsen(const Geom& g, const float2* U, const float2* C, const float2* P,
                              float2* X, float2* Y, int* status, cudaStream_t s);
cudaError_t launch_tc_gemm(const Geom& g, const float2* A, bool gather, const double2* gdiag,
                           const float* abound, const float2* B, int n, float2* C, float* cmax,
                           int* status, cudaStream_t s, const char* name);

// psi0 [V][4][3][m] and links U [V][4][3][3] = exp(i eps H) from the
// counter-based generator of seed (mg_starts.cu).
cudaError_t launch_random_starts(const Geom& g, uint64_t seed, float2* psi0, cudaStream_t s);
cudaError_t launch_random_links(const Geom& g, uint64_t seed, double eps, float2* U,
                                cudaStream_t s);

cudaError_t launch_truncate(const Geom& g, const float2* psi, float2* Uk, double* sigma,
                            float2* coarse_tv, int32_t* flags, char* ws, cudaStream_t s);

cudaError_t launch_prolongator(const Geom& g, const float2* Uk, float2* P, cudaStream_t s);

cudaError_t launch_coarsen(const Geom& g, const float2* U, const float2* C, const float2* P,
                           float2* X, float2* Y, cudaStream_t s);

cudaError_t launch_coarse_apply(const Geom& g, const float2* X, const float2* Y,
                                const float2* vin, float2* vout, int nrhs, cudaStream_t s);

// levels l >= 1 (mg_level2.cu): out = D_l v for nrhs <= 64 right-hand sides; the
// smoother on D_l psi = 0; the Galerkin product D_{l+1} = P^dag D_l P with g
// describing the aggregation of the level-l lattice (g.rps = nc)
cudaError_t launch_stencil_apply(const StencilGeom& sg, const float2* X, const float2* Y,
                                 const float2* vin, float2* vout, int nrhs, cudaStream_t s);
cudaError_t launch_stencil_smoother(const StencilGeom& sg, int m, int niter, const float2* X,
                                    const float2* Y, const float2* psi0, float2* psi, char* ws,
                                    cudaStream_t s);
cudaError_t launch_stencil_galerkin(const Geom& g, const float2* X, const float2* Y,
                                    const float2* P, float2* X2, float2* Y2, cudaStream_t s);

// ---------------------------------------------------------------------------
// small complex helpers (float2 / double2 as complex numbers)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
  return make_float2(a.x * s, a.y * s);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

__host__ __device__ __forceinline__ double2 zadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 zsub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 zmulc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 zscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}
__host__ __device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }

}  // namespace mg
