// mg_starts.cu -- random starting vectors psi0 drawn on the device (the
// smoother's "m random initial guesses", paper Sec. 2, Eq. 1), for callers
// that do not bring their own, e.g. a setup server.
//
// The numbers are the ones of the counter-based generator the tests and the
// FP64 reference use (mg_inputs): SplitMix64 (Steele, Lea, Flood, OOPSLA 2014)
// of a counter plus the key of (seed, stream 2), the top 53 bits as a uniform
// double in (0, 1), and Box-Muller's cosine branch (Box & Muller 1958):
//   normal n = sqrt(-2 ln u_{2n}) cos(2 pi u_{2n+1}),
//   psi0 element e (flat index over [V][4][3][m]) = normal 2e + i normal 2e+1.
// The uniforms are bit-identical to the host generator's; the logarithm,
// square root and cosine are taken in FP32 (the result is stored in complex64
// anyway), so the starts agree with the host's to a few 1e-6.
#include <cstdint>

#include "mg_common.cuh"

namespace mg {
namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kM2 = 0x94D049BB133111EBull;
constexpr uint64_t kStreamPsi0 = 2;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + kGolden;
  z = (z ^ (z >> 30)) * kM1;
  z = (z ^ (z >> 27)) * kM2;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform(uint64_t key, uint64_t ctr) {
  return ((double)(splitmix64(ctr + key) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ float normal(uint64_t key, uint64_t n) {
  const float u0 = (float)uniform(key, 2 * n), u1 = (float)uniform(key, 2 * n + 1);
  return sqrtf(-2.f * logf(u0)) * cosf(6.28318530717958647692f * u1);
}

__global__ void starts_kernel(float2* __restrict__ psi0, uint64_t n, uint64_t key) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n;
       e += (uint64_t)gridDim.x * blockDim.x)
    psi0[e] = make_float2(normal(key, 2 * e), normal(key, 2 * e + 1));
}

}  // namespace

cudaError_t launch_random_starts(const Geom& g, uint64_t seed, float2* psi0, cudaStream_t s) {
  const uint64_t key = splitmix64(seed ^ splitmix64(kStreamPsi0));
  const uint64_t n = (uint64_t)g.V * 12 * g.m;
  TimedScope ts("random_starts", s);
  starts_kernel<<<4 * 152 * 8, 256, 0, s>>>(psi0, n, key);
  return cudaGetLastError();
}

}  // namespace mg
