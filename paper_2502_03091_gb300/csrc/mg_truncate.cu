// mg_truncate.cu -- chiral split and rank-k truncation (paper Sec. 2 Eq. 2,
// Sec. 3 Eq. 4).  For every block Lambda_j and chirality alpha the
// K x m' matrix A = Psi^(alpha)(Lambda_j), K = 6 |Lambda_j| (rows: site,
// spin in chirality, colour), is factored as
//   G1 = A^dag A                  (FP32 products, FP64 across row chunks)
//   R1 = chol(G1)                 (FP64)
//   Q1 = A R1^{-1}, G2 = Q1^dag Q1 (FP32, Q1 never stored)
//   R2 = chol(G2), R = R2 R1      (FP64)          -- CholeskyQR2: A = Q R
//   R R^dag = U~ S^2 U~^dag       (FP64 Householder tridiagonalisation,
//                                  bisection, inverse iteration; top k only)
//   U_k = Q1 (R2^{-1} U~_k), Sigma_k = S_k
// so U_k are the k leading left singular vectors of A (A = Q R, R = U~ S V~^dag),
// the best rank-k basis of Eq. (4).  The chiral split itself is only the
// choice of rows: chirality 0 is spins {0,1}, chirality 1 spins {2,3}.
#include "mg_common.cuh"

namespace mg {
namespace {

constexpr int kThreads = 256;
constexpr int kChunkSites = 8;            // sites staged per chunk
constexpr int kChunkRows = 6 * kChunkSites;  // rows per chunk

// global site of local site `loc` of block `j`
__device__ __forceinline__ int block_site(int j, int loc, const int L[4], const int b[4],
                                          const int Lc[4]) {
  int jc[4], lc[4];
  int t = j;
  jc[0] = t % Lc[0]; t /= Lc[0];
  jc[1] = t % Lc[1]; t /= Lc[1];
  jc[2] = t % Lc[2]; jc[3] = t / Lc[2];
  t = loc;
  lc[0] = t % b[0]; t /= b[0];
  lc[1] = t % b[1]; t /= b[1];
  lc[2] = t % b[2]; lc[3] = t / b[2];
  const int x0 = jc[0] * b[0] + lc[0], x1 = jc[1] * b[1] + lc[1];
  const int x2 = jc[2] * b[2] + lc[2], x3 = jc[3] * b[3] + lc[3];
  return x0 + L[0] * (x1 + L[1] * (x2 + L[2] * x3));
}

struct BlockGeom {
  int L[4], b[4], Lc[4];
  int nb;  // sites per block
  int m, k;
};

// Stage the rows of chunk `ch` (kChunkSites sites) of block-chirality bc
// into As[row][m] (row = local_site_in_chunk*6 + spin_in_chirality*3 + colour).
// Rows past the block end are zero.
__device__ void load_chunk(const float2* __restrict__ psi, const BlockGeom& g, int bc, int ch,
                           float2* As) {
  const int j = bc >> 1, al = bc & 1;
  const int m = g.m;
  const int per_site4 = 6 * m / 2;  // float4 per site (6 rows of m complex)
  for (int idx = threadIdx.x; idx < kChunkSites * per_site4; idx += blockDim.x) {
    const int ls = idx / per_site4, o = idx % per_site4;
    const int loc = ch * kChunkSites + ls;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (loc < g.nb) {
      const int x = block_site(j, loc, g.L, g.b, g.Lc);
      const float4* src = reinterpret_cast<const float4*>(psi + ((long)x * 12 + 6 * al) * m);
      v = __ldg(src + o);
    }
    reinterpret_cast<float4*>(As + ls * 6 * m)[o] = v;
  }
}

// Qs[r][c] = sum_{l <= c} As[r][l] Zs[l][c]   (Zs upper triangular, m x m)
__device__ void right_mul_upper(const float2* As, const float2* Zs, float2* Qs, int rows, int m) {
  for (int idx = threadIdx.x; idx < rows * m; idx += blockDim.x) {
    const int r = idx / m, c = idx % m;
    float2 s = make_float2(0.f, 0.f);
    for (int l = 0; l <= c; ++l) cfma(s, As[r * m + l], Zs[l * m + c]);
    Qs[idx] = s;
  }
}

// ---------------------------------------------------------------------------
// Gram of the (optionally transformed) block: G[bc] = B^dag B, B = A or A Z.
// One CTA per block-chirality; each active thread owns a 4x4 tile of the
// upper triangle of tiles; FP32 within a chunk, FP64 across chunks.
// ---------------------------------------------------------------------------
template <bool TRANSFORM>
__global__ void __launch_bounds__(kThreads) gram_kernel(const float2* __restrict__ psi,
                                                        const float2* __restrict__ Z,
                                                        double2* __restrict__ G, BlockGeom g) {
  extern __shared__ float4 smem4[];
  float2* As = reinterpret_cast<float2*>(smem4);
  float2* Qs = As + kChunkRows * g.m;
  float2* Zs = Qs + kChunkRows * g.m;
  const int bc = blockIdx.x, m = g.m, TT = m / 4;
  if (TRANSFORM) {
    const float2* Zb = Z + (long)bc * m * m;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) Zs[i] = Zb[i];
  }
  // tile (ti, tj), ti <= tj, enumerated row by row
  int ti = -1, tj = -1;
  {
    int t = threadIdx.x;
    for (int r = 0; r < TT; ++r) {
      if (t < TT - r) {
        ti = r;
        tj = r + t;
        break;
      }
      t -= TT - r;
    }
  }
  double2 dacc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) dacc[a][c] = make_double2(0.0, 0.0);
  const int nch = (g.nb + kChunkSites - 1) / kChunkSites;
  for (int ch = 0; ch < nch; ++ch) {
    __syncthreads();
    load_chunk(psi, g, bc, ch, As);
    __syncthreads();
    const float2* Bs = As;
    if (TRANSFORM) {
      right_mul_upper(As, Zs, Qs, kChunkRows, m);
      __syncthreads();
      Bs = Qs;
    }
    if (ti >= 0) {
      float2 acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
      for (int r = 0; r < kChunkRows; ++r) {
        const float4* row = reinterpret_cast<const float4*>(Bs + r * m);
        const float4 a01 = row[2 * ti], a23 = row[2 * ti + 1];
        const float4 b01 = row[2 * tj], b23 = row[2 * tj + 1];
        const float2 av[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                              make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
        const float2 bv[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                              make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) cfmac(acc[a][c], av[a], bv[c]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          dacc[a][c].x += (double)acc[a][c].x;
          dacc[a][c].y += (double)acc[a][c].y;
        }
    }
  }
  if (ti >= 0) {
    double2* Gb = G + (long)bc * m * m;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = 4 * ti + a, jj = 4 * tj + c;
        Gb[i * m + jj] = dacc[a][c];
        Gb[jj * m + i] = zconj(dacc[a][c]);
      }
  }
}

// ---------------------------------------------------------------------------
// FP64 dense helpers on shared memory (one CTA, m <= 64)
// ---------------------------------------------------------------------------

// In-place upper Cholesky G = R^dag R on the upper triangle of Gs (m x m),
// with `shift` added to the diagonal.  Returns false on a pivot <= tol.
__device__ bool chol_upper(double2* Gs, int m, double tol, int* s_fail) {
  if (threadIdx.x == 0) *s_fail = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      const double d = Gs[j * m + j].x;
      if (!(d > tol)) *s_fail = 1;
      Gs[j * m + j] = make_double2(d > tol ? sqrt(d) : 1.0, 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / Gs[j * m + j].x;
    for (int l = j + 1 + threadIdx.x; l < m; l += blockDim.x)
      Gs[j * m + l] = zscale(Gs[j * m + l], inv);
    __syncthreads();
    const int n = m - j - 1;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int a = j + 1 + idx / n, b = j + 1 + idx % n;
      if (b >= a) Gs[a * m + b] = zsub(Gs[a * m + b], zmulc(Gs[j * m + a], Gs[j * m + b]));
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x)
    if (idx / m > idx % m) Gs[idx] = make_double2(0.0, 0.0);
  __syncthreads();
  return *s_fail == 0;
}

// Zs = Rs^{-1} for upper-triangular Rs (column c solved by thread c).
__device__ void tri_inverse_upper(const double2* Rs, double2* Zs, int m) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) Zs[idx] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    for (int i = c; i >= 0; --i) {
      double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int l = i + 1; l <= c; ++l) s = zsub(s, zmul(Rs[i * m + l], Zs[l * m + c]));
      Zs[i * m + c] = zscale(s, 1.0 / Rs[i * m + i].x);
    }
  }
  __syncthreads();
}

// Stage 1: R1 = chol(G1) (with a diagonal shift if a pivot fails), store R1
// (FP64) and Z1 = R1^{-1} (FP32).
__global__ void __launch_bounds__(kThreads) chol_stage1(const double2* __restrict__ G,
                                                        double2* __restrict__ R1,
                                                        float2* __restrict__ Z1,
                                                        int32_t* __restrict__ flags, int m) {
  extern __shared__ double2 dsm[];
  double2* Gs = dsm;
  double2* Zs = dsm + m * m;
  __shared__ int s_fail;
  __shared__ double s_maxd;
  const int bc = blockIdx.x;
  const double2* Gb = G + (long)bc * m * m;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Gs[i] = Gb[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0;
    for (int i = 0; i < m; ++i) mx = fmax(mx, Gs[i * m + i].x);
    s_maxd = mx;
  }
  __syncthreads();
  const double maxd = s_maxd;
  int32_t flag = 0;
  if (!chol_upper(Gs, m, 1e-13 * maxd, &s_fail)) {
    flag |= 1;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
      Gs[i] = Gb[i];
      if (i / m == i % m) Gs[i].x += 1e-5 * maxd;
    }
    __syncthreads();
    if (!chol_upper(Gs, m, 1e-13 * maxd, &s_fail)) flag |= 2;
  }
  tri_inverse_upper(Gs, Zs, m);
  double2* Rb = R1 + (long)bc * m * m;
  float2* Zb = Z1 + (long)bc * m * m;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    Rb[i] = Gs[i];
    Zb[i] = make_float2((float)Zs[i].x, (float)Zs[i].y);
  }
  if (threadIdx.x == 0) flags[bc] = flag;
}

// ---------------------------------------------------------------------------
// FP64 top-k eigenpairs of a Hermitian m x m matrix in shared memory:
// Householder tridiagonalisation, Sturm bisection, inverse iteration.
// ---------------------------------------------------------------------------

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Hs: Hermitian (full). On exit: d[0..m), e[0..m-1) complex subdiagonal
// T[j+1][j], reflector j stored in column j of Hs rows j+1.. (u_j), tau[j].
// H = Q T Q^dag with Q = H_0 H_1 ... H_{m-3}, H_j = I - tau_j u_j u_j^dag.
__device__ void tridiagonalise(double2* Hs, int m, double* d, double2* e, double* tau,
                               double2* p, double* red) {
  for (int j = 0; j + 2 < m; ++j) {
    const int n = m - j - 1;  // length of x = H[j+1.., j]
    double tail = 0;
    for (int i = j + 2 + threadIdx.x; i < m; i += blockDim.x) tail += zabs2(Hs[i * m + j]);
    tail = block_sum(tail, red);
    const double2 x0 = Hs[(j + 1) * m + j];
    double t = 0.0;
    double2 beta = x0;
    if (tail > 0.0) {
      const double ax0 = sqrt(zabs2(x0));
      const double nx = sqrt(zabs2(x0) + tail);
      const double2 ph = ax0 > 0 ? zscale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
      beta = zscale(ph, -nx);
      const double2 u0 = zsub(x0, beta);
      t = 2.0 / (zabs2(u0) + tail);
      __syncthreads();
      if (threadIdx.x == 0) Hs[(j + 1) * m + j] = u0;
      __syncthreads();
      // p = t A u over the trailing block A = H[j+1.., j+1..]
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int a = w; a < n; a += nw) {
        double2 s = make_double2(0.0, 0.0);
        for (int b = lane; b < n; b += 32)
          s = zadd(s, zmul(Hs[(j + 1 + a) * m + j + 1 + b], Hs[(j + 1 + b) * m + j]));
        for (int o = 16; o > 0; o >>= 1) {
          s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
          s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) p[a] = zscale(s, t);
      }
      __syncthreads();
      // K = t/2 u^dag p (real); w = p - K u (stored over p)
      double kr = 0;
      for (int a = threadIdx.x; a < n; a += blockDim.x) kr += zmulc(Hs[(j + 1 + a) * m + j], p[a]).x;
      kr = 0.5 * t * block_sum(kr, red);
      __syncthreads();
      for (int a = threadIdx.x; a < n; a += blockDim.x)
        p[a] = zsub(p[a], zscale(Hs[(j + 1 + a) * m + j], kr));
      __syncthreads();
      // A -= u w^dag + w u^dag
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int a = idx / n, b = idx % n;
        const double2 ua = Hs[(j + 1 + a) * m + j], ub = Hs[(j + 1 + b) * m + j];
        double2 v = Hs[(j + 1 + a) * m + j + 1 + b];
        v = zsub(v, zmul(ua, zconj(p[b])));
        v = zsub(v, zmul(p[a], zconj(ub)));
        Hs[(j + 1 + a) * m + j + 1 + b] = v;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      e[j] = beta;
      tau[j] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (m >= 2) {
      e[m - 2] = Hs[(m - 1) * m + m - 2];
      tau[m - 2] = 0.0;
    }
    for (int i = 0; i < m; ++i) d[i] = Hs[i * m + i].x;
  }
  __syncthreads();
}

// number of eigenvalues of the real symmetric tridiagonal (d, f) below x
__device__ int sturm_count(const double* d, const double* f2, int n, double x, double tiny) {
  double q = d[0] - x;
  int c = q < 0;
  for (int i = 1; i < n; ++i) {
    if (fabs(q) < tiny) q = q < 0 ? -tiny : tiny;
    q = d[i] - x - f2[i - 1] / q;
    c += q < 0;
  }
  return c;
}

// one step of inverse iteration: z <- (T - lam)^{-1} z, LU with partial pivoting
__device__ void tri_solve(const double* d, const double* f, int n, double lam, double tiny,
                          double* z) {
  double a[kMaxM], c[kMaxM], c2[kMaxM], l[kMaxM];
  bool piv[kMaxM];
  for (int i = 0; i < n; ++i) {
    a[i] = d[i] - lam;
    c[i] = i + 1 < n ? f[i] : 0.0;
    c2[i] = 0.0;
  }
  for (int i = 0; i + 1 < n; ++i) {
    const double bsub = f[i];
    if (fabs(a[i]) >= fabs(bsub)) {
      piv[i] = false;
      if (a[i] == 0.0) a[i] = tiny;
      l[i] = bsub / a[i];
      a[i + 1] -= l[i] * c[i];
    } else {
      piv[i] = true;
      l[i] = a[i] / bsub;
      a[i] = bsub;
      const double tmp = a[i + 1];
      a[i + 1] = c[i] - l[i] * tmp;
      if (i + 2 < n) {
        c2[i] = c[i + 1];
        c[i + 1] = -l[i] * c2[i];
      }
      c[i] = tmp;
    }
  }
  for (int i = 0; i + 1 < n; ++i) {
    if (piv[i]) {
      const double t = z[i];
      z[i] = z[i + 1];
      z[i + 1] = t - l[i] * z[i + 1];
    } else {
      z[i + 1] -= l[i] * z[i];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = z[i];
    if (i + 1 < n) s -= c[i] * z[i + 1];
    if (i + 2 < n) s -= c2[i] * z[i + 2];
    const double p = fabs(a[i]) < tiny ? (a[i] < 0 ? -tiny : tiny) : a[i];
    z[i] = s / p;
  }
}

// Stage 2: R2 = chol(G2), R = R2 R1, H = R R^dag, top-k eigenpairs of H,
// sigma = sqrt(lambda), W2 = R2^{-1} U~_k (FP32), optional Sigma_k V_k^dag = U~_k^dag R.
__global__ void __launch_bounds__(kThreads) svd_stage2(
    const double2* __restrict__ G2, const double2* __restrict__ R1, float2* __restrict__ W2,
    double* __restrict__ sigma, float2* __restrict__ ctv, int32_t* __restrict__ flags, int m,
    int k) {
  extern __shared__ double2 dsm[];
  double2* As = dsm;              // R2
  double2* Bs = As + m * m;       // R, later U~_k (m x k) and tridiagonal eigvecs
  double2* Hs = Bs + m * m;       // H, then reflectors
  __shared__ double d[kMaxM], tau[kMaxM], fo[kMaxM], f2[kMaxM], lam[kMaxK];
  __shared__ double2 e[kMaxM], delta[kMaxM], pv[kMaxM];
  __shared__ double red[32];
  __shared__ int s_fail;
  __shared__ int leader[kMaxK];
  const int bc = blockIdx.x;
  // R2
  const double2* Gb = G2 + (long)bc * m * m;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) As[i] = Gb[i];
  __syncthreads();
  double maxd = 0;
  for (int i = 0; i < m; ++i) maxd = fmax(maxd, As[i * m + i].x);
  int32_t flag = 0;
  if (!chol_upper(As, m, 1e-13 * maxd, &s_fail)) flag |= 4;
  // R = R2 R1 (upper)
  const double2* R1b = R1 + (long)bc * m * m;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, c = idx % m;
    double2 s = make_double2(0.0, 0.0);
    for (int l = i; l <= c; ++l) s = zadd(s, zmul(As[i * m + l], R1b[l * m + c]));
    Bs[idx] = s;
  }
  __syncthreads();
  // H = R R^dag
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, c = idx % m;
    const int l0 = i > c ? i : c;
    double2 s = make_double2(0.0, 0.0);
    for (int l = l0; l < m; ++l) s = zadd(s, zmul(Bs[i * m + l], zconj(Bs[c * m + l])));
    Hs[idx] = s;
  }
  __syncthreads();
  // coarse test vectors need R; they are formed after U~_k, so keep R in
  // global scratch only when requested: recompute from As and R1 below.
  tridiagonalise(Hs, m, d, e, tau, pv, red);
  if (threadIdx.x == 0) {
    delta[0] = make_double2(1.0, 0.0);
    for (int j = 0; j + 1 < m; ++j) {
      const double ae = sqrt(zabs2(e[j]));
      fo[j] = ae;
      f2[j] = ae * ae;
      delta[j + 1] = ae > 0 ? zmul(delta[j], zscale(e[j], 1.0 / ae)) : delta[j];
    }
  }
  __syncthreads();
  double tnorm = 0;
  for (int i = 0; i < m; ++i) {
    const double r = fabs(d[i]) + (i > 0 ? fo[i - 1] : 0.0) + (i + 1 < m ? fo[i] : 0.0);
    tnorm = fmax(tnorm, r);
  }
  const double tiny = 1e-300 + 1e-15 * tnorm;
  // eigenvalue i (i-th largest) by bisection, one thread each
  if (threadIdx.x < k) {
    const int target = m - 1 - threadIdx.x;  // index among ascending eigenvalues
    double lo = -tnorm, hi = tnorm;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(d, f2, m, mid, 1e-300) > target) hi = mid;
      else lo = mid;
    }
    lam[threadIdx.x] = 0.5 * (lo + hi);
  }
  __syncthreads();
  // clusters (eigenvalues closer than 1e-10 |T|) are handled by their first member
  if (threadIdx.x < k) {
    const int i = threadIdx.x;
    leader[i] = (i == 0 || fabs(lam[i - 1] - lam[i]) > 1e-10 * tnorm) ? 1 : 0;
  }
  __syncthreads();
  // inverse iteration; the real eigenvector z_i of T' goes to Bs column i (.x)
  double2* Uk = Bs;  // m x k, row-major
  if (threadIdx.x < k && leader[threadIdx.x]) {
    int i = threadIdx.x;
    do {
      double z[kMaxM];
      for (int r = 0; r < m; ++r) z[r] = 1.0 + 0.01 * r + 0.001 * i;
      for (int it = 0; it < 4; ++it) {
        tri_solve(d, fo, m, lam[i], tiny, z);
        for (int pj = threadIdx.x; pj < i; ++pj) {  // previous members of this cluster
          double dot = 0;
          for (int r = 0; r < m; ++r) dot += Uk[r * k + pj].x * z[r];
          for (int r = 0; r < m; ++r) z[r] -= dot * Uk[r * k + pj].x;
        }
        double nrm = 0;
        for (int r = 0; r < m; ++r) nrm += z[r] * z[r];
        nrm = 1.0 / sqrt(nrm);
        for (int r = 0; r < m; ++r) z[r] *= nrm;
      }
      for (int r = 0; r < m; ++r) Uk[r * k + i] = make_double2(z[r], 0.0);
      ++i;
    } while (i < k && !leader[i]);
  }
  __syncthreads();
  // back-transform: y = Q (delta .* z), one warp per vector
  {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < k; i += nw) {
      for (int r = lane; r < m; r += 32) Uk[r * k + i] = zscale(delta[r], Uk[r * k + i].x);
      __syncwarp();
      for (int j = m - 3; j >= 0; --j) {
        if (tau[j] == 0.0) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int r = j + 1 + lane; r < m; r += 32) s = zadd(s, zmulc(Hs[r * m + j], Uk[r * k + i]));
        for (int o = 16; o > 0; o >>= 1) {
          s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
          s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        s = zscale(s, tau[j]);
        for (int r = j + 1 + lane; r < m; r += 32)
          Uk[r * k + i] = zsub(Uk[r * k + i], zmul(s, Hs[r * m + j]));
        __syncwarp();
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < k) sigma[(long)bc * k + threadIdx.x] = sqrt(fmax(lam[threadIdx.x], 0.0));
  // W2 = R2^{-1} U~_k, column i by thread i (back substitution, R2 upper)
  float2* Wb = W2 + (long)bc * m * k;
  if (threadIdx.x < k) {
    const int i = threadIdx.x;
    double2 y[kMaxM];
    for (int r = m - 1; r >= 0; --r) {
      double2 s = Uk[r * k + i];
      for (int l = r + 1; l < m; ++l) s = zsub(s, zmul(As[r * m + l], y[l]));
      y[r] = zscale(s, 1.0 / As[r * m + r].x);
    }
    for (int r = 0; r < m; ++r) Wb[r * k + i] = make_float2((float)y[r].x, (float)y[r].y);
  }
  if (ctv) {
    // Sigma_k V_k^dag = U~_k^dag R,  R = R2 R1 recomputed entry by entry
    float2* cb = ctv + (long)bc * k * m;
    for (int idx = threadIdx.x; idx < k * m; idx += blockDim.x) {
      const int i = idx / m, c = idx % m;
      double2 s = make_double2(0.0, 0.0);
      for (int l = 0; l <= c; ++l) {
        double2 rl = make_double2(0.0, 0.0);
        for (int q = l; q <= c; ++q) rl = zadd(rl, zmul(As[l * m + q], R1b[q * m + c]));
        s = zadd(s, zmulc(Uk[l * k + i], rl));
      }
      cb[idx] = make_float2((float)s.x, (float)s.y);
    }
  }
  if (threadIdx.x == 0) flags[bc] |= flag;
}

// U_k rows = (A Z1) W2 for every row of the block, written in the block-major
// layout Uk[bc][row][k].
__global__ void __launch_bounds__(kThreads) form_uk(const float2* __restrict__ psi,
                                                    const float2* __restrict__ Z1,
                                                    const float2* __restrict__ W2,
                                                    float2* __restrict__ Uk, BlockGeom g) {
  extern __shared__ float4 smem4[];
  const int m = g.m, k = g.k;
  float2* As = reinterpret_cast<float2*>(smem4);
  float2* Qs = As + kChunkRows * m;
  float2* Zs = Qs + kChunkRows * m;
  float2* Ws = Zs + m * m;
  const int bc = blockIdx.x;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Zs[i] = Z1[(long)bc * m * m + i];
  for (int i = threadIdx.x; i < m * k; i += blockDim.x) Ws[i] = W2[(long)bc * m * k + i];
  const int nch = (g.nb + kChunkSites - 1) / kChunkSites;
  float2* out = Uk + (long)bc * 6 * g.nb * k;
  for (int ch = 0; ch < nch; ++ch) {
    __syncthreads();
    load_chunk(psi, g, bc, ch, As);
    __syncthreads();
    right_mul_upper(As, Zs, Qs, kChunkRows, m);
    __syncthreads();
    const int rows = min(kChunkRows, 6 * (g.nb - ch * kChunkSites));
    for (int idx = threadIdx.x; idx < rows * k; idx += blockDim.x) {
      const int r = idx / k, c = idx % k;
      float2 s = make_float2(0.f, 0.f);
      for (int l = 0; l < m; ++l) cfma(s, Qs[r * m + l], Ws[l * k + c]);
      out[(long)(ch * kChunkRows + r) * k + c] = s;
    }
  }
}

}  // namespace

cudaError_t launch_truncate(const Geom& g, const float2* psi, float2* Uk, double* sigma,
                            float2* coarse_tv, int32_t* flags, char* ws, cudaStream_t s) {
  const TruncWs lay = trunc_ws_layout(g);
  double2* G = reinterpret_cast<double2*>(ws + lay.gram);
  double2* R1 = reinterpret_cast<double2*>(ws + lay.r1);
  float2* Z1 = reinterpret_cast<float2*>(ws + lay.z1);
  float2* W2 = reinterpret_cast<float2*>(ws + lay.w2);
  BlockGeom bg;
  for (int i = 0; i < 4; ++i) {
    bg.L[i] = g.L[i];
    bg.b[i] = g.b[i];
    bg.Lc[i] = g.Lc[i];
  }
  bg.nb = g.nb;
  bg.m = g.m;
  bg.k = g.k;
  const int nbc = (int)(2 * g.nblk);
  const int m = g.m, k = g.k;
  const size_t sm_gram0 = sizeof(float2) * (size_t)(2 * kChunkRows * m);
  const size_t sm_gram1 = sm_gram0 + sizeof(float2) * (size_t)m * m;
  const size_t sm_chol = sizeof(double2) * (size_t)2 * m * m;
  const size_t sm_svd = sizeof(double2) * (size_t)3 * m * m;
  const size_t sm_uk = sm_gram1 + sizeof(float2) * (size_t)m * k;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(gram_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(gram_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(chol_stage1, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(svd_stage2, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(form_uk, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    attr_done = true;
  }
  {
    TimedScope ts("trunc_gram", s);
    gram_kernel<false><<<nbc, kThreads, sm_gram0, s>>>(psi, nullptr, G, bg);
  }
  {
    TimedScope ts("trunc_chol64", s);
    chol_stage1<<<nbc, kThreads, sm_chol, s>>>(G, R1, Z1, flags, m);
  }
  {
    TimedScope ts("trunc_gram_q1", s);
    gram_kernel<true><<<nbc, kThreads, sm_gram1, s>>>(psi, Z1, G, bg);
  }
  {
    TimedScope ts("trunc_chol_eig64", s);
    svd_stage2<<<nbc, kThreads, sm_svd, s>>>(G, R1, W2, sigma, coarse_tv, flags, m, k);
  }
  {
    TimedScope ts("trunc_form_uk", s);
    form_uk<<<nbc, kThreads, sm_uk, s>>>(psi, Z1, W2, Uk, bg);
  }
  return cudaGetLastError();
}

}  // namespace mg
