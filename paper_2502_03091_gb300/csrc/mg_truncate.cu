// mg_truncate.cu -- chiral split and rank-k truncation (paper Sec. 2 Eq. 2,
// Sec. 3 Eq. 4).  For every block Lambda_j and chirality alpha the
// K x m' matrix A = Psi^(alpha)(Lambda_j), K = 6 |Lambda_j| (rows: site,
// spin in chirality, colour), is factored as
//   G1 = A^dag A                  (FP32 products, FP64 across row chunks)
//   R1 = chol(G1)                 (FP64)
//   Q1 = A R1^{-1}, G2 = Q1^dag Q1 (FP32, Q1 never stored)
//   R2 = chol(G2), R = R2 R1      (FP32 on the deviations from 1; R in FP64)
//                                                 -- CholeskyQR2: A = Q R
//   R R^dag = U~ S^2 U~^dag       (double-float Householder tridiagonalisation,
//                                  FP32 multisection, FP64 inverse iteration and
//                                  Rayleigh quotients; top k only)
//   U_k = A (Z1 R2^{-1} U~_k), Sigma_k = S_k     (Z1 = R1^{-1})
// so U_k are the k leading left singular vectors of A (A = Q R, R = U~ S V~^dag),
// the best rank-k basis of Eq. (4).  The chiral split itself is only the
// choice of rows: chirality 0 is spins {0,1}, chirality 1 spins {2,3}.
// In the mixed-precision paths G1, Q1 (then stored), G2 and U_k = Q1 (R2^-1 U~_k)
// are tensor-core contractions (mg_tc.cu); the small FP64 stages are shared.
#include "mg_common.cuh"

namespace mg {
namespace {

constexpr int kThreads = 256;
constexpr int kChunkRows = 48;  // rows staged per chunk (8 fine sites x 6 rows)

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
  int nb;      // sites per block
  int m, k;
  int rps;     // rows per site and chirality (6 at the fine level: 2 spins x 3 colours)
  int cps;     // complex components per site (2 rps)
  int csites;  // sites per chunk: kChunkRows / rps, so a chunk has csites * rps <= 48 rows
};

// Stage the rows of chunk `ch` (csites sites) of block-chirality bc into
// As[row][m] (row = local_site_in_chunk * rps + row of the site's chirality
// block; at the fine level spin_in_chirality * 3 + colour).  Rows past the
// block end, and rows csites * rps .. kChunkRows - 1, are zero.
__device__ void load_chunk(const float2* __restrict__ psi, const BlockGeom& g, int bc, int ch,
                           float2* As) {
  const int j = bc >> 1, al = bc & 1;
  const int m = g.m;
  const int per_site4 = g.rps * m / 2;  // float4 per site (rps rows of m complex)
  for (int idx = threadIdx.x; idx < kChunkRows * m / 2; idx += blockDim.x) {
    const int ls = idx / per_site4, o = idx % per_site4;
    const int loc = ch * g.csites + ls;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ls < g.csites && loc < g.nb) {
      const int x = block_site(j, loc, g.L, g.b, g.Lc);
      const float4* src =
          reinterpret_cast<const float4*>(psi + ((long)x * g.cps + g.rps * al) * m);
      v = __ldg(src + o);
    }
    reinterpret_cast<float4*>(As)[idx] = v;
  }
}

// C[r][c] = sum_l A[r][l] B[l][c] for r < rows (a multiple of TR), c < n,
// l < kd (UPPER: B upper triangular, only l <= c is read).  Each thread
// computes a TR x TC register tile (TR + TC shared-memory loads per TR * TC
// complex multiply-adds).  A is rows x lda, B is kd x ldb, C is rows x ldc.
template <int TR, int TC, bool UPPER>
__device__ void tile_gemm(const float2* A, int lda, const float2* B, int ldb, float2* C, int ldc,
                          int rows, int n, int kd) {
  // thread t: rows r0 .. r0+TR-1, columns c0, c0 + cg, ..., c0 + (TC-1) cg, so
  // that neighbouring threads read neighbouring B entries (no bank conflicts)
  const int rg = rows / TR, cg = (n + TC - 1) / TC;
  for (int t = threadIdx.x; t < rg * cg; t += blockDim.x) {
    const int r0 = (t / cg) * TR, c0 = t % cg;
    float2 acc[TR][TC];
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) acc[i][j] = make_float2(0.f, 0.f);
    const int lmax = UPPER ? min(kd, min(n, c0 + (TC - 1) * cg + 1)) : kd;
    for (int l = 0; l < lmax; ++l) {
      float2 a[TR], b[TC];
#pragma unroll
      for (int i = 0; i < TR; ++i) a[i] = A[(r0 + i) * lda + l];
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        const int c = c0 + j * cg;
        b[j] = (c < n && (!UPPER || l <= c)) ? B[l * ldb + c] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TC; ++j) cfma(acc[i][j], a[i], b[j]);
    }
#pragma unroll
    for (int i = 0; i < TR; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j)
        if (c0 + j * cg < n) C[(r0 + i) * ldc + c0 + j * cg] = acc[i][j];
  }
}

// Qs[r][c] = sum_{l <= c} As[r][l] Zs[l][c]   (Zs upper triangular, m x m)
__device__ __forceinline__ void right_mul_upper(const float2* As, const float2* Zs, float2* Qs,
                                                int rows, int m) {
  tile_gemm<3, 4, true>(As, m, Zs, m, Qs, m, rows, m, m);
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
  const int nch = (g.nb + g.csites - 1) / g.csites;
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
// FP64 dense helpers on shared memory (one CTA, m <= 64).  Matrices use the
// leading dimension ld = m + 1: the padding keeps column accesses free of
// bank conflicts.
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

// In-place upper Cholesky G = R^dag R on the upper triangle of Gs (m x m,
// leading dimension ld).  Returns false if a pivot is <= tol; the lower
// triangle is zeroed on exit.
__device__ bool chol_upper(double2* Gs, int m, int ld, double tol, int* s_fail) {
  if (threadIdx.x == 0) *s_fail = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      const double d = Gs[j * ld + j].x;
      if (!(d > tol)) *s_fail = 1;
      Gs[j * ld + j] = make_double2(d > tol ? sqrt(d) : 1.0, 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / Gs[j * ld + j].x;
    for (int l = j + 1 + threadIdx.x; l < m; l += blockDim.x)
      Gs[j * ld + l] = zscale(Gs[j * ld + l], inv);
    __syncthreads();
    const int n = m - j - 1;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = j + 1 + idx / n, c = j + 1 + idx % n;
      if (c >= r) Gs[r * ld + c] = zsub(Gs[r * ld + c], zmulc(Gs[j * ld + r], Gs[j * ld + c]));
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x)
    if (idx / m > idx % m) Gs[(idx / m) * ld + idx % m] = make_double2(0.0, 0.0);
  __syncthreads();
  return *s_fail == 0;
}

// Cholesky of a Hermitian matrix close to the identity, G = 1 + E, in
// deviations: R = 1 + F with F upper triangular.  Every update acts on the
// small quantities only (the diagonal is kept as delta_jj = a_jj - 1 and
// r_jj - 1 = delta_jj / (1 + sqrt(1 + delta_jj)) has no cancellation), so FP32
// gives F to FP32 relative accuracy, i.e. R to ~1e-7 |E| absolute.  Gs (FP64,
// leading dimension ld) holds G on entry and R (upper, 1 + F) on exit; the
// FP32 deviations live in the first 8 bytes of each 16-byte entry meanwhile.
// Returns false if a pivot 1 + delta_jj is not positive (it is then set to 1).
__device__ bool chol_upper_near1(double2* Gs, int m, int ld, int* s_fail) {
  float2* Ef = reinterpret_cast<float2*>(Gs);  // entry e at Ef[2 e]
  if (threadIdx.x == 0) *s_fail = 0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, c = idx % m;
    const double2 v = Gs[i * ld + c];
    Ef[2 * (i * ld + c)] = make_float2((float)(v.x - (i == c ? 1.0 : 0.0)), (float)v.y);
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      float dj = Ef[2 * (j * ld + j)].x;
      if (!(1.0f + dj > 1e-6f)) {
        *s_fail = 1;
        dj = 0.f;
      }
      Ef[2 * (j * ld + j)] = make_float2(dj / (1.0f + sqrtf(1.0f + dj)), 0.f);
    }
    __syncthreads();
    const float inv = 1.0f / (1.0f + Ef[2 * (j * ld + j)].x);
    for (int l = j + 1 + threadIdx.x; l < m; l += blockDim.x) {
      float2& r = Ef[2 * (j * ld + l)];
      r = make_float2(r.x * inv, r.y * inv);
    }
    __syncthreads();
    const int n = m - j - 1;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = j + 1 + idx / n, c = j + 1 + idx % n;
      if (c >= r) {
        const float2 a = Ef[2 * (j * ld + r)], b = Ef[2 * (j * ld + c)];
        float2& e = Ef[2 * (r * ld + c)];
        // e -= conj(a) b
        e = make_float2(e.x - (a.x * b.x + a.y * b.y), e.y - (a.x * b.y - a.y * b.x));
      }
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, c = idx % m;
    const float2 f = Ef[2 * (i * ld + c)];
    Gs[i * ld + c] = c < i ? make_double2(0.0, 0.0)
                           : make_double2((i == c ? 1.0 : 0.0) + (double)f.x, (double)f.y);
  }
  __syncthreads();
  return *s_fail == 0;
}

// Stage 1: R1 = chol(G1) (with a diagonal shift if a pivot fails), store R1
// (FP64) and Z1 = R1^{-1} (FP32).  The inverse is formed row by row from the
// bottom: z_ic = (delta_ic - sum_{i<l<=c} R_il z_lc) / R_ii, four threads per
// column sharing the sum.
__global__ void __launch_bounds__(kThreads, 2) chol_stage1(const double2* __restrict__ G,
                                                           double2* __restrict__ R1,
                                                           float2* __restrict__ Z1,
                                                           int32_t* __restrict__ flags, int m) {
  extern __shared__ double2 dsm[];
  const int ld = m + 1;
  double2* Gs = dsm;                                    // [m][ld] FP64
  float2* Zs = reinterpret_cast<float2*>(Gs + m * ld);  // [m][m] FP32
  __shared__ int s_fail;
  __shared__ double red[32];
  const int bc = blockIdx.x;
  const double2* Gb = G + (long)bc * m * m;
  double mx = 0;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    const double2 v = Gb[i];
    Gs[(i / m) * ld + i % m] = v;
    if (i / m == i % m) mx = fmax(mx, v.x);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  double maxd = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) maxd = fmax(maxd, red[i]);
  int32_t flag = 0;
  if (!chol_upper(Gs, m, ld, 1e-13 * maxd, &s_fail)) {
    flag |= 1;
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
      double2 v = Gb[i];
      if (i / m == i % m) v.x += 1e-5 * maxd;
      Gs[(i / m) * ld + i % m] = v;
    }
    __syncthreads();
    if (!chol_upper(Gs, m, ld, 1e-13 * maxd, &s_fail)) flag |= 2;
  }
  double2* Rb = R1 + (long)bc * m * m;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    Rb[i] = Gs[(i / m) * ld + i % m];
    Zs[i] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  // Z1 is an FP32 output and R1 is well conditioned: the substitution runs in
  // FP32 arithmetic on the FP64 factor rounded to FP32
  const int c = threadIdx.x >> 2, part = threadIdx.x & 3;
  for (int i = m - 1; i >= 0; --i) {
    float2 acc = make_float2(0.f, 0.f);
    if (c < m && c >= i)
      for (int l = i + 1 + part; l <= c; l += 4) {
        const double2 r = Gs[i * ld + l];
        cfma(acc, make_float2((float)r.x, (float)r.y), Zs[l * m + c]);
      }
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
    if (c < m && c >= i && part == 0) {
      const float inv = (float)(1.0 / Gs[i * ld + i].x);
      Zs[i * m + c] = make_float2(((i == c ? 1.f : 0.f) - acc.x) * inv, -acc.y * inv);
    }
    __syncthreads();
  }
  float2* Zb = Z1 + (long)bc * m * m;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Zb[i] = Zs[i];
  if (threadIdx.x == 0) flags[bc] = flag;
}

// ---------------------------------------------------------------------------
// Double-float numbers: value = hi + lo, two FP32 with |lo| <= ulp(hi) / 2.
// Sums by Knuth's TwoSum and products by the FMA form of Dekker's TwoProduct
// (error-free transformations; cf. Hida, Li, Bailey, "Algorithms for quad-double
// precision", 2001) give about 2^-44 relative accuracy on the FP32 pipe, which
// on this GPU issues 64 times the FP64 rate.  The _rn intrinsics keep the
// compiler from fusing the operations the transformations rely on.
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};
struct dz {  // complex double-float
  df re, im;
};

__device__ __forceinline__ df df_from(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}

__device__ __forceinline__ dz dz_from(double2 v) { return dz{df_from(v.x), df_from(v.y)}; }
__device__ __forceinline__ double2 dz_to(dz a) { return make_double2(df_to(a.re), df_to(a.im)); }
__device__ __forceinline__ dz dz_zero() { return dz{df{0.f, 0.f}, df{0.f, 0.f}}; }
__device__ __forceinline__ dz dz_add(dz a, dz b) { return dz{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dz dz_sub(dz a, dz b) { return dz{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dz dz_mul(dz a, dz b) {  // a b
  return dz{df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)),
            df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dz dz_mulc(dz a, dz b) {  // conj(a) b
  return dz{df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)),
            df_sub(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dz dz_conj(dz a) { return dz{a.re, df_neg(a.im)}; }
__device__ __forceinline__ dz dz_scale(dz a, df s) { return dz{df_mul(a.re, s), df_mul(a.im, s)}; }
__device__ __forceinline__ df df_shfl_xor(df a, int o) {
  return df{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ dz dz_warp_sum(dz a) {
  for (int o = 16; o > 0; o >>= 1) {
    a.re = df_add(a.re, df_shfl_xor(a.re, o));
    a.im = df_add(a.im, df_shfl_xor(a.im, o));
  }
  return a;
}

// ---------------------------------------------------------------------------
// Top-k eigenpairs of a Hermitian m x m matrix in shared memory: Householder
// tridiagonalisation (double-float), Sturm multisection (FP32), inverse
// iteration and Rayleigh quotients (FP64).
// ---------------------------------------------------------------------------

// Hs: Hermitian (full, leading dimension ld), double-float.  On exit:
// d[0..m), e[0..m-1) complex subdiagonal T[j+1][j], reflector j stored in
// column j of Hs rows j+1.. (u_j), tau[j].  H = Q T Q^dag with
// Q = H_0 H_1 ... H_{m-3}, H_j = I - tau_j u_j u_j^dag.  The scalars of each
// reflector (norms, tau, beta) are formed in FP64.
__device__ void tridiagonalise(dz* Hs, int m, int ld, double* d, double2* e, double* tau,
                               dz* uv, dz* pv, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j + 2 < m; ++j) {
    const int n = m - j - 1;  // length of x = H[j+1.., j]
    double tail = 0;
    for (int i = j + 2 + threadIdx.x; i < m; i += blockDim.x) tail += zabs2(dz_to(Hs[i * ld + j]));
    tail = block_sum(tail, red);
    const double2 x0 = dz_to(Hs[(j + 1) * ld + j]);
    double t = 0.0;
    double2 beta = x0;
    if (tail > 0.0) {
      const double ax0 = sqrt(zabs2(x0));
      const double nx = sqrt(zabs2(x0) + tail);
      const double2 ph = ax0 > 0 ? zscale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
      beta = zscale(ph, -nx);
      const double2 u0 = zsub(x0, beta);
      t = 2.0 / (zabs2(u0) + tail);
      const df tdf = df_from(t);
      // u (contiguous copy) and its column copy for the back-transform
      for (int a = threadIdx.x; a < n; a += blockDim.x)
        uv[a] = a == 0 ? dz_from(u0) : Hs[(j + 1 + a) * ld + j];
      __syncthreads();
      if (threadIdx.x == 0) Hs[(j + 1) * ld + j] = dz_from(u0);
      // p = t A u over the trailing block A = H[j+1.., j+1..], one warp per row
      for (int a = w; a < n; a += nw) {
        dz sacc = dz_zero();
        const dz* row = Hs + (j + 1 + a) * ld + j + 1;
        for (int b = lane; b < n; b += 32) sacc = dz_add(sacc, dz_mul(row[b], uv[b]));
        sacc = dz_warp_sum(sacc);
        if (lane == 0) pv[a] = dz_scale(sacc, tdf);
      }
      __syncthreads();
      // K = t/2 u^dag p (real); w = p - K u (stored over p)
      double kr = 0;
      for (int a = threadIdx.x; a < n; a += blockDim.x) kr += zmulc(dz_to(uv[a]), dz_to(pv[a])).x;
      kr = 0.5 * t * block_sum(kr, red);
      const df krdf = df_from(kr);
      for (int a = threadIdx.x; a < n; a += blockDim.x)
        pv[a] = dz_sub(pv[a], dz_scale(uv[a], krdf));
      __syncthreads();
      // A -= u w^dag + w u^dag
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int ra = idx / n, cb = idx % n;
        dz v = Hs[(j + 1 + ra) * ld + j + 1 + cb];
        v = dz_sub(v, dz_mul(uv[ra], dz_conj(pv[cb])));
        v = dz_sub(v, dz_mul(pv[ra], dz_conj(uv[cb])));
        Hs[(j + 1 + ra) * ld + j + 1 + cb] = v;
      }
    }
    if (threadIdx.x == 0) {
      e[j] = beta;
      tau[j] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (m >= 2) {
      e[m - 2] = dz_to(Hs[(m - 1) * ld + m - 2]);
      tau[m - 2] = 0.0;
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) d[i] = df_to(Hs[i * ld + i].re);
  __syncthreads();
}

// number of eigenvalues of the real symmetric tridiagonal (d, f) below x, in
// FP32 (locates eigenvalues to ~1e-7 |T|; they are refined in FP64 later)
__device__ int sturm_count32(const float* d, const float* f2, int n, float x, float tiny) {
  float q = d[0] - x;
  int c = q < 0.f;
  for (int i = 1; i < n; ++i) {
    if (fabsf(q) < tiny) q = q < 0.f ? -tiny : tiny;
    q = d[i] - x - __fdividef(f2[i - 1], q);
    c += q < 0.f;
  }
  return c;
}

// LU factorisation with partial pivoting of the tridiagonal T - lam (diagonal
// d, off-diagonal f): U has diagonals a, c, c2; L has multipliers l and the
// row swaps in the bit mask piv
struct TriLU {
  double a[kMaxM], c[kMaxM], c2[kMaxM], l[kMaxM];
  unsigned long long piv;
};

__device__ void tri_factor(const double* d, const double* f, int n, double lam, double tiny,
                           TriLU& F) {
  F.piv = 0ull;
  for (int i = 0; i < n; ++i) {
    F.a[i] = d[i] - lam;
    F.c[i] = i + 1 < n ? f[i] : 0.0;
    F.c2[i] = 0.0;
  }
  for (int i = 0; i + 1 < n; ++i) {
    const double bsub = f[i];
    if (fabs(F.a[i]) >= fabs(bsub)) {
      if (F.a[i] == 0.0) F.a[i] = tiny;
      F.l[i] = bsub / F.a[i];
      F.a[i + 1] -= F.l[i] * F.c[i];
    } else {
      F.piv |= 1ull << i;
      F.l[i] = F.a[i] / bsub;
      F.a[i] = bsub;
      const double tmp = F.a[i + 1];
      F.a[i + 1] = F.c[i] - F.l[i] * tmp;
      if (i + 2 < n) {
        F.c2[i] = F.c[i + 1];
        F.c[i + 1] = -F.l[i] * F.c2[i];
      }
      F.c[i] = tmp;
    }
  }
  for (int i = 0; i < n; ++i)
    if (fabs(F.a[i]) < tiny) F.a[i] = F.a[i] < 0 ? -tiny : tiny;
}

// one step of inverse iteration: z <- (T - lam)^{-1} z with the factors F
__device__ void tri_solve(const TriLU& F, int n, double* z) {
  for (int i = 0; i + 1 < n; ++i) {
    if ((F.piv >> i) & 1ull) {
      const double t = z[i];
      z[i] = z[i + 1];
      z[i + 1] = t - F.l[i] * z[i + 1];
    } else {
      z[i + 1] -= F.l[i] * z[i];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double sacc = z[i];
    if (i + 1 < n) sacc -= F.c[i] * z[i + 1];
    if (i + 2 < n) sacc -= F.c2[i] * z[i + 2];
    z[i] = sacc / F.a[i];
  }
}

// Stage 2: R2 = chol(G2), R = R2 R1, H = R R^dag, top-k eigenpairs of H,
// sigma = sqrt(lambda), W2 = R2^{-1} U~_k (FP32), optional Sigma_k V_k^dag = U~_k^dag R.
// Global scratch per block-chirality: G (in: G2, out: R2), R1 (in: R1,
// out: R), Hg (H).
constexpr int kBisect = 10;  // points per multisection step

__global__ void __launch_bounds__(kThreads, 2) svd_stage2(
    double2* __restrict__ G2, double2* __restrict__ R1, double2* __restrict__ Hg,
    float2* __restrict__ W2, double* __restrict__ sigma, float2* __restrict__ ctv,
    int32_t* __restrict__ flags, int m, int k) {
  extern __shared__ double2 dsm[];
  const int ld = m + 1;
  double2* M = dsm;            // [m][ld]
  double2* Uk = M + m * ld;    // [m][k]
  __shared__ double d[kMaxM], tau[kMaxM], fo[kMaxM];
  __shared__ float d32[kMaxM], f232[kMaxM];
  __shared__ double s_dmax;
  __shared__ double2 e[kMaxM], delta[kMaxM], uv[kMaxM], pv[kMaxM], rowbuf[kMaxM];
  __shared__ double red[32];
  __shared__ double lo[kMaxK], hi[kMaxK], lam[kMaxK];
  __shared__ int cnt[kMaxK][kBisect];
  __shared__ int s_fail;
  __shared__ int leader[kMaxK];
  const int bc = blockIdx.x;
  double2* Gb = G2 + (long)bc * m * m;
  double2* Rg = R1 + (long)bc * m * m;
  double2* Hb = Hg + (long)bc * m * m;
  // R2 = chol(G2), kept in global for W2
  double mx = 0;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    const double2 v = Gb[i];
    M[(i / m) * ld + i % m] = v;
    if (i / m == i % m) mx = fmax(mx, v.x);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  double maxd = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) maxd = fmax(maxd, red[i]);
  int32_t flag = 0;
  // G2 = Q1^dag Q1 is the identity up to the rounding of Q1: the Cholesky of
  // its deviation in FP32 keeps R2 - 1 to FP32 relative accuracy
  (void)maxd;
  if (!chol_upper_near1(M, m, ld, &s_fail)) flag |= 4;
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Gb[i] = M[(i / m) * ld + i % m];
  __syncthreads();
  // R = R2 R1 = R1 + (R2 - 1) R1.  After CholeskyQR2's first pass R2 = 1 + D
  // with D small, so the correction D R1 is formed in FP32 and added to R1 in
  // FP64: its error u_fp32 |D| |R1| is below the FP32 rounding of the input
  // vectors by the factor |D| < 1e-3.  A larger D takes the FP64 product.
  // Column c of R1 is read in chunks of 16 rows; each thread keeps 16 rows of
  // one column.  R -> Hb.
  {
    double dm = 0;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int i = idx / m, c = idx % m;
      const double2 v = M[i * ld + c];
      dm = fmax(dm, fabs(v.x - (i == c ? 1.0 : 0.0)) + fabs(v.y));
    }
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
      s_dmax = t;
    }
    __syncthreads();
    const bool small = s_dmax < 1e-3;
    const int c = threadIdx.x % 64, r0 = threadIdx.x / 64;  // rows r0, r0+4, ...
    if (c < m) {
      if (small) {
        float2 acc[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) acc[r] = make_float2(0.f, 0.f);
        for (int l0 = 0; l0 < m; l0 += 16) {
          float2 col[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int l = l0 + q;
            const double2 v = l < m ? Rg[l * m + c] : make_double2(0.0, 0.0);
            col[q] = make_float2((float)v.x, (float)v.y);
          }
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int i = r0 + 4 * r;
            if (i >= m) continue;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int l = l0 + q;
              if (l < m && l >= i) {
                const double2 dv = M[i * ld + l];
                cfma(acc[r], make_float2((float)(dv.x - (l == i ? 1.0 : 0.0)), (float)dv.y), col[q]);
              }
            }
          }
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int i = r0 + 4 * r;
          if (i < m) {
            const double2 base = c >= i ? Rg[i * m + c] : make_double2(0.0, 0.0);
            Hb[i * m + c] = c >= i ? make_double2(base.x + acc[r].x, base.y + acc[r].y)
                                   : make_double2(0.0, 0.0);
          }
        }
      } else {
        for (int i = r0; i < m; i += 4) {
          double2 acc = make_double2(0.0, 0.0);
          for (int l = i; l <= c; ++l) acc = zadd(acc, zmul(M[i * ld + l], Rg[l * m + c]));
          Hb[i * m + c] = acc;
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
      const double2 v = Hb[i];
      M[(i / m) * ld + i % m] = v;
      Rg[i] = v;
    }
    __syncthreads();
  }
  // R in double-float, in place (a dz occupies the 16 bytes of its double2)
  dz* Mz = reinterpret_cast<dz*>(M);
  for (int i = threadIdx.x; i < m * ld; i += blockDim.x) Mz[i] = dz_from(M[i]);
  __syncthreads();
  // H = R R^dag (upper triangle computed, mirrored) -> global, then back into M
  dz* Hz = reinterpret_cast<dz*>(Hb);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, jj = idx % m;
    if (jj < i) continue;
    dz acc = dz_zero();
    for (int l = jj; l < m; ++l) acc = dz_add(acc, dz_mul(Mz[i * ld + l], dz_conj(Mz[jj * ld + l])));
    Hz[i * m + jj] = acc;
    Hz[jj * m + i] = dz_conj(acc);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Mz[(i / m) * ld + i % m] = Hz[i];
  __syncthreads();
  dz* uvz = reinterpret_cast<dz*>(uv);
  tridiagonalise(Mz, m, ld, d, e, tau, uvz, reinterpret_cast<dz*>(pv), red);
  if (threadIdx.x == 0) {
    delta[0] = make_double2(1.0, 0.0);
    for (int j = 0; j + 1 < m; ++j) {
      const double ae = sqrt(zabs2(e[j]));
      fo[j] = ae;
      f232[j] = (float)(ae * ae);
      delta[j + 1] = ae > 0 ? zmul(delta[j], zscale(e[j], 1.0 / ae)) : delta[j];
    }
    for (int j = 0; j < m; ++j) d32[j] = (float)d[j];
  }
  __syncthreads();
  double tnorm = 0;
  for (int i = 0; i < m; ++i) {
    const double r = fabs(d[i]) + (i > 0 ? fo[i - 1] : 0.0) + (i + 1 < m ? fo[i] : 0.0);
    tnorm = fmax(tnorm, r);
  }
  const double tiny = 1e-300 + 1e-15 * tnorm;
  // multisection: kBisect points per eigenvalue (the ei-th largest); the
  // k * kBisect (eigenvalue, point) pairs are spread over the block's threads
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    lo[i] = -tnorm;
    hi[i] = tnorm;
  }
  __syncthreads();
  {
    const float tiny32 = 1e-30f + 1e-20f * (float)tnorm;
    for (int it = 0; it < 9; ++it) {
      for (int w = threadIdx.x; w < k * kBisect; w += blockDim.x) {
        const int ei = w / kBisect, sp = w % kBisect;
        const double l0 = lo[ei], h0 = hi[ei];
        const double x = l0 + (h0 - l0) * (double)(sp + 1) / (double)(kBisect + 1);
        cnt[ei][sp] = sturm_count32(d32, f232, m, (float)x, tiny32);
      }
      __syncthreads();
      for (int ei = threadIdx.x; ei < k; ei += blockDim.x) {
        const int target = m - 1 - ei;  // index among ascending eigenvalues
        const double l0 = lo[ei], h0 = hi[ei];
        double nl = l0, nh = h0;
        for (int q = 0; q < kBisect; ++q) {
          const double x = l0 + (h0 - l0) * (double)(q + 1) / (double)(kBisect + 1);
          if (cnt[ei][q] > target) {
            nh = x;
            break;
          }
          nl = x;
        }
        lo[ei] = nl;
        hi[ei] = nh;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x < k) lam[threadIdx.x] = 0.5 * (lo[threadIdx.x] + hi[threadIdx.x]);
  __syncthreads();
  // clusters (eigenvalues closer than 1e-6 |T|, above the FP32 resolution of
  // the multisection) are handled by their first member
  if (threadIdx.x < k) {
    const int i = threadIdx.x;
    leader[i] = (i == 0 || fabs(lam[i - 1] - lam[i]) > 1e-6 * tnorm) ? 1 : 0;
  }
  __syncthreads();
  // inverse iteration; the real eigenvector z_i of T' goes to Uk column i (.x)
  if (threadIdx.x < k && leader[threadIdx.x]) {
    int i = threadIdx.x;
    do {
      double z[kMaxM];
      TriLU F;
      tri_factor(d, fo, m, lam[i], tiny, F);
      for (int r = 0; r < m; ++r) z[r] = 1.0 + 0.01 * r + 0.001 * i;
      for (int it = 0; it < 3; ++it) {
        tri_solve(F, m, z);
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
      // FP64 Rayleigh quotient z^T T z refines the FP32 multisection value
      double rq = 0;
      for (int r = 0; r < m; ++r) rq += d[r] * z[r] * z[r];
      for (int r = 0; r + 1 < m; ++r) rq += 2.0 * fo[r] * z[r] * z[r + 1];
      lam[i] = rq;
      for (int r = 0; r < m; ++r) Uk[r * k + i] = make_double2(z[r], 0.0);
      ++i;
    } while (i < k && !leader[i]);
  }
  __syncthreads();
  // back-transform (double-float): y = Q (delta .* z); reflector j copied to uv first
  dz* Ukz = reinterpret_cast<dz*>(Uk);
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x)
    Ukz[idx] = dz_from(zscale(delta[idx / k], Uk[idx].x));
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = m - 3; j >= 0; --j) {
      if (tau[j] == 0.0) continue;
      const int n = m - j - 1;
      const df tj = df_from(tau[j]);
      for (int a = threadIdx.x; a < n; a += blockDim.x) uvz[a] = Mz[(j + 1 + a) * ld + j];
      __syncthreads();
      for (int i = w; i < k; i += nw) {
        dz sacc = dz_zero();
        for (int a = lane; a < n; a += 32)
          sacc = dz_add(sacc, dz_mulc(uvz[a], Ukz[(j + 1 + a) * k + i]));
        sacc = dz_scale(dz_warp_sum(sacc), tj);
        for (int a = lane; a < n; a += 32)
          Ukz[(j + 1 + a) * k + i] = dz_sub(Ukz[(j + 1 + a) * k + i], dz_mul(sacc, uvz[a]));
      }
      __syncthreads();
    }
  }
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) Uk[idx] = dz_to(Ukz[idx]);
  __syncthreads();
  if (threadIdx.x < k) sigma[(long)bc * k + threadIdx.x] = sqrt(fmax(lam[threadIdx.x], 0.0));
  if (ctv) {
    // Sigma_k V_k^dag = U~_k^dag R  (R from global)
    float2* cb = ctv + (long)bc * k * m;
    for (int idx = threadIdx.x; idx < k * m; idx += blockDim.x) {
      const int i = idx / m, c = idx % m;
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l <= c; ++l) acc = zadd(acc, zmulc(Uk[l * k + i], Rg[l * m + c]));
      cb[idx] = make_float2((float)acc.x, (float)acc.y);
    }
    __syncthreads();
  }
  // W2 = R2^{-1} U~_k (an FP32 output; R2 is close to 1): FP32 substitution
  // from the bottom, eight threads per column, R2 staged into M
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) M[(i / m) * ld + i % m] = Gb[i];
  __syncthreads();
  {
    const int c = threadIdx.x >> 3, part = threadIdx.x & 7;
    for (int i = m - 1; i >= 0; --i) {
      float2 acc = make_float2(0.f, 0.f);
      if (c < k)
        for (int l = i + 1 + part; l < m; l += 8) {
          const double2 r = M[i * ld + l], u = Uk[l * k + c];
          cfma(acc, make_float2((float)r.x, (float)r.y), make_float2((float)u.x, (float)u.y));
        }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (c < k && part == 0) {
        const float inv = (float)(1.0 / M[i * ld + i].x);
        const double2 u = Uk[i * k + c];
        Uk[i * k + c] = make_double2(((float)u.x - acc.x) * inv, ((float)u.y - acc.y) * inv);
      }
      __syncthreads();
    }
  }
  float2* Wb = W2 + (long)bc * m * k;
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x)
    Wb[idx] = make_float2((float)Uk[idx].x, (float)Uk[idx].y);
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
  __syncthreads();
  // U_k = (A Z1) W2 = A M with M = Z1 W2 (m x k, Z1 upper triangular), formed
  // once per block-chirality in the Q area
  float2* Ms = Qs;
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) {
    const int i = idx / k, c = idx % k;
    float2 sacc = make_float2(0.f, 0.f);
    for (int l = i; l < m; ++l) cfma(sacc, Zs[i * m + l], Ws[l * k + c]);
    Ms[idx] = sacc;
  }
  const int nch = (g.nb + g.csites - 1) / g.csites;
  float2* out = Uk + (long)bc * g.rps * g.nb * k;
  float2* Us = Ws + m * k;  // chunk of U_k (kChunkRows x k)
  for (int ch = 0; ch < nch; ++ch) {
    __syncthreads();
    load_chunk(psi, g, bc, ch, As);
    __syncthreads();
    tile_gemm<3, 2, false>(As, m, Ms, k, Us, k, kChunkRows, k, m);
    __syncthreads();
    const int rows = g.rps * min(g.csites, g.nb - ch * g.csites);
    for (int idx = threadIdx.x; idx < rows * k; idx += blockDim.x)
      out[(long)(ch * g.csites * g.rps) * k + idx] = Us[idx];
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
  double2* Hm = reinterpret_cast<double2*>(ws + lay.hm);
  BlockGeom bg;
  for (int i = 0; i < 4; ++i) {
    bg.L[i] = g.L[i];
    bg.b[i] = g.b[i];
    bg.Lc[i] = g.Lc[i];
  }
  bg.nb = g.nb;
  bg.m = g.m;
  bg.k = g.k;
  bg.rps = g.rps;
  bg.cps = g.cps;
  bg.csites = kChunkRows / g.rps;
  const int nbc = (int)(2 * g.nblk);
  const int m = g.m, k = g.k;
  const size_t sm_gram0 = sizeof(float2) * (size_t)(2 * kChunkRows * m);
  const size_t sm_gram1 = sm_gram0 + sizeof(float2) * (size_t)m * m;
  const size_t sm_chol = sizeof(double2) * (size_t)m * (m + 1) + sizeof(float2) * (size_t)m * m;
  const size_t sm_svd = sizeof(double2) * ((size_t)m * (m + 1) + (size_t)m * k);
  const size_t sm_uk = sm_gram1 + sizeof(float2) * ((size_t)m * k + (size_t)kChunkRows * k);
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(gram_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(gram_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(chol_stage1, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(svd_stage2, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    cudaFuncSetAttribute(form_uk, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
  });
  if (g.prec != MG_PREC_FP32 && tc_supported(g) && lay.q1) {
    // mixed precision: the dense contractions on the tensor cores
    //   G1 = A^dag A (BF16: it only preconditions the second pass)
    //   R1 = chol(G1), Z1 = R1^-1 (FP64 / FP32, CUDA cores)
    //   Q1 = A Z1 (FP16 hi/lo), stored, and its largest entry
    //   G2 = Q1^dag Q1 (FP16 hi/lo)
    //   R2 = chol(G2), R = R2 R1, eigen-decomposition of R R^dag (as FP32 path)
    //   U_k = Q1 W2 with W2 = R2^-1 U~_k (FP16 hi/lo), straight into Uk
    int* st = device_status_word();
    if (!st) return cudaErrorInvalidSymbol;
    float2* Q1 = reinterpret_cast<float2*>(ws + lay.q1);
    float* qmax = reinterpret_cast<float*>(ws + lay.qmax);
    cudaError_t e = launch_tc_gram(g, psi, true, false, nullptr, G, st, s, "trunc_gram_tc");
    if (e != cudaSuccess) return e;
    {
      TimedScope ts("trunc_chol64", s);
      chol_stage1<<<nbc, kThreads, sm_chol, s>>>(G, R1, Z1, flags, m);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_tc_gemm(g, psi, true, G, nullptr, Z1, m, Q1, qmax, st, s, "trunc_q1_tc");
    if (e != cudaSuccess) return e;
    e = launch_tc_gram(g, Q1, false, true, qmax, G, st, s, "trunc_gram2_tc");
    if (e != cudaSuccess) return e;
    {
      TimedScope ts("trunc_chol_eig64", s);
      svd_stage2<<<nbc, kThreads, sm_svd, s>>>(G, R1, Hm, W2, sigma, coarse_tv, flags, m, k);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_tc_gemm(g, Q1, false, nullptr, qmax, W2, k, Uk, nullptr, st, s, "trunc_uk_tc");
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
    svd_stage2<<<nbc, kThreads, sm_svd, s>>>(G, R1, Hm, W2, sigma, coarse_tv, flags, m, k);
  }
  {
    TimedScope ts("trunc_form_uk", s);
    form_uk<<<nbc, kThreads, sm_uk, s>>>(psi, Z1, W2, Uk, bg);
  }
  return cudaGetLastError();
}

}  // namespace mg
