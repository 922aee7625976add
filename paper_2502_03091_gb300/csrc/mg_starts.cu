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
//
// Random gauge links U_mu(x) = exp(i eps H), H = sum_a h_a lambda_a / 2 with
// h_a the normals 8j .. 8j+7 of stream 1 for link j = 4x + mu and lambda_a the
// Gell-Mann matrices, are drawn the same way (normals in FP64); the
// exponential is its Taylor series in FP32, the precision the links are stored
// in (|eps H| stays below ~2 here, where 22 terms leave a remainder below
// 1e-16).
#include <cstdint>

#include "mg_common.cuh"

namespace mg {
namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kM2 = 0x94D049BB133111EBull;
constexpr uint64_t kStreamGauge = 1;
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

__device__ __forceinline__ double normal64(uint64_t key, uint64_t n) {
  const double u0 = uniform(key, 2 * n), u1 = uniform(key, 2 * n + 1);
  return sqrt(-2.0 * log(u0)) * cos(6.283185307179586 * u1);
}

// one link per thread: H from 8 normals (FP64), exp(i eps H) by 22 Taylor terms (FP32)
__global__ void links_kernel(float2* __restrict__ U, uint64_t nlinks, uint64_t key, double eps) {
  const double s3 = 0.57735026918962576451;  // 1 / sqrt(3)
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nlinks;
       j += (uint64_t)gridDim.x * blockDim.x) {
    double h[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) h[a] = normal64(key, 8 * j + a);
    // X = i eps H with H = sum_a h_a lambda_a / 2 (Gell-Mann basis)
    double2 H[3][3];
    H[0][0] = make_double2(0.5 * (h[2] + s3 * h[7]), 0.0);
    H[1][1] = make_double2(0.5 * (-h[2] + s3 * h[7]), 0.0);
    H[2][2] = make_double2(-s3 * h[7], 0.0);
    H[0][1] = make_double2(0.5 * h[0], -0.5 * h[1]);
    H[0][2] = make_double2(0.5 * h[3], -0.5 * h[4]);
    H[1][2] = make_double2(0.5 * h[5], -0.5 * h[6]);
    H[1][0] = zconj(H[0][1]);
    H[2][0] = zconj(H[0][2]);
    H[2][1] = zconj(H[1][2]);
    float2 X[3][3], T[3][3], S[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        X[r][c] = make_float2((float)(-eps * H[r][c].y), (float)(eps * H[r][c].x));  // i eps H
        T[r][c] = S[r][c] = make_float2(r == c ? 1.f : 0.f, 0.f);
      }
    for (int n = 1; n <= 22; ++n) {
      float2 N[3][3];
      const float inv = 1.f / (float)n;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int l = 0; l < 3; ++l) cfma(acc, T[r][l], X[l][c]);
          N[r][c] = cscale(acc, inv);
        }
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T[r][c] = N[r][c];
          S[r][c] = cadd(S[r][c], N[r][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) U[j * 9 + r * 3 + c] = S[r][c];
  }
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

cudaError_t launch_random_links(const Geom& g, uint64_t seed, double eps, float2* U,
                                cudaStream_t s) {
  const uint64_t key = splitmix64(seed ^ splitmix64(kStreamGauge));
  TimedScope ts("random_links", s);
  links_kernel<<<4 * 152 * 4, 128, 0, s>>>(U, (uint64_t)g.V * 4, key, eps);
  return cudaGetLastError();
}

}  // namespace mg
