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
#include <algorithm>

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
// Double-float numbers: value = hi + lo, two FP32 with |lo| <= ulp(hi) / 2.
// Sums by Knuth's TwoSum and products by the FMA form of Dekker's TwoProduct
// (error-free transformations; cf. Hida, Li, Bailey, "Algorithms for quad-double
// precision", 2001) give about 2^-44 relative accuracy on the FP32 pipe, which
// on this GPU issues 64 times the FP64 rate.  The _rn intrinsics keep the
// compiler from fusing the operations the transformations rely on.  The
// small dense stages below run on these numbers; FP64 is left to O(m) scalar
// work per block-chirality (the tridiagonal eigenvectors).
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
__device__ __forceinline__ df df_mulf(df a, float b) {  // a b, b an FP32 number
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_half(df a) { return df{0.5f * a.hi, 0.5f * a.lo}; }
// 1 / a: the FP32 reciprocal q and one Newton step q + q (1 - a q); the
// residual 1 - a q is exact in double-float, so the result has ~2^-46 error
__device__ __forceinline__ df df_recip(df a) {
  const float q = __frcp_rn(a.hi);
  const df r = df_sub(df{1.f, 0.f}, df_mulf(a, q));
  return df_add(df{q, 0.f}, df_mulf(r, q));
}
// sqrt(a) for a > 0: y = sqrt(a.hi) and one Newton step y + (a - y^2) / (2 y)
__device__ __forceinline__ df df_sqrt(df a) {
  const float y = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(y, y);
  const df r = df_sub(a, df{p, __fmaf_rn(y, y, -p)});
  return quick_two_sum(y, __fdiv_rn(r.hi, 2.f * y));
}

__device__ __forceinline__ dz dz_from(double2 v) { return dz{df_from(v.x), df_from(v.y)}; }
__device__ __forceinline__ double2 dz_to(dz a) { return make_double2(df_to(a.re), df_to(a.im)); }
__device__ __forceinline__ float2 dz_to_f(dz a) {
  return make_float2(__fadd_rn(a.re.hi, a.re.lo), __fadd_rn(a.im.hi, a.im.lo));
}
__device__ __forceinline__ dz dz_zero() { return dz{df{0.f, 0.f}, df{0.f, 0.f}}; }
__device__ __forceinline__ dz dz_sub(dz a, dz b) { return dz{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dz dz_scale(dz a, df s) { return dz{df_mul(a.re, s), df_mul(a.im, s)}; }
__device__ __forceinline__ df dz_abs2(dz a) { return df_add(df_mul(a.re, a.re), df_mul(a.im, a.im)); }
__device__ __forceinline__ dz dz_shfl(dz a, int src) {
  return dz{df{__shfl_sync(0xffffffffu, a.re.hi, src), __shfl_sync(0xffffffffu, a.re.lo, src)},
            df{__shfl_sync(0xffffffffu, a.im.hi, src), __shfl_sync(0xffffffffu, a.im.lo, src)}};
}

// Accumulator for sums of double-float products in the manner of Ogita, Rump
// and Oishi's Dot2 ("Accurate sum and dot product", SIAM J. Sci. Comput. 26,
// 2005): the running FP32 sum s, with the rounding error of every addition
// (TwoSum) and of every product (FMA form of TwoProduct, plus the cross terms
// of the low parts) collected in the FP32 term e.  s + e carries double-float
// accuracy (the dropped lo * lo terms are 2^-48 of a product) for about half
// the operations of double-float products and sums.
struct dacc {
  float s, e;
};
struct zacc {
  dacc re, im;
};
__device__ __forceinline__ dacc acc_from(df a) { return dacc{a.hi, a.lo}; }
// a += x y
__device__ __forceinline__ void acc_prod(dacc& a, df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float q = __fmaf_rn(x.hi, y.hi, -p);
  q = __fmaf_rn(x.hi, y.lo, q);
  q = __fmaf_rn(x.lo, y.hi, q);
  const float s = __fadd_rn(a.s, p);
  const float bb = __fsub_rn(s, a.s);
  const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  a.s = s;
  a.e = __fadd_rn(a.e, __fadd_rn(t, q));
}
__device__ __forceinline__ dacc acc_merge(dacc a, dacc b) {
  const df t = two_sum(a.s, b.s);
  return dacc{t.hi, __fadd_rn(__fadd_rn(a.e, b.e), t.lo)};
}
__device__ __forceinline__ df acc_get(dacc a) { return two_sum(a.s, a.e); }
__device__ __forceinline__ dz zacc_get(zacc a) { return dz{acc_get(a.re), acc_get(a.im)}; }
__device__ __forceinline__ zacc zacc_from(dz a) { return zacc{acc_from(a.re), acc_from(a.im)}; }
__device__ __forceinline__ zacc zacc_zero() { return zacc{dacc{0.f, 0.f}, dacc{0.f, 0.f}}; }
// a += x y
__device__ __forceinline__ void zacc_mul(zacc& a, dz x, dz y) {
  acc_prod(a.re, x.re, y.re);
  acc_prod(a.re, df_neg(x.im), y.im);
  acc_prod(a.im, x.re, y.im);
  acc_prod(a.im, x.im, y.re);
}
// a += conj(x) y
__device__ __forceinline__ void zacc_mulc(zacc& a, dz x, dz y) {
  acc_prod(a.re, x.re, y.re);
  acc_prod(a.re, x.im, y.im);
  acc_prod(a.im, x.re, y.im);
  acc_prod(a.im, df_neg(x.im), y.re);
}
// a += x conj(y)
__device__ __forceinline__ void zacc_mul_conj(zacc& a, dz x, dz y) {
  acc_prod(a.re, x.re, y.re);
  acc_prod(a.re, x.im, y.im);
  acc_prod(a.im, x.im, y.re);
  acc_prod(a.im, df_neg(x.re), y.im);
}
// a -= x conj(y)
__device__ __forceinline__ void zacc_sub_mul_conj(zacc& a, dz x, dz y) {
  acc_prod(a.re, df_neg(x.re), y.re);
  acc_prod(a.re, df_neg(x.im), y.im);
  acc_prod(a.im, df_neg(x.im), y.re);
  acc_prod(a.im, x.re, y.im);
}
__device__ __forceinline__ dacc acc_shfl_xor(dacc a, int o) {
  return dacc{__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.e, o)};
}
__device__ __forceinline__ zacc zacc_merge_xor(zacc a, int o) {
  return zacc{acc_merge(a.re, acc_shfl_xor(a.re, o)), acc_merge(a.im, acc_shfl_xor(a.im, o))};
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
    // the Gram is stored in double-float (a pair of FP32 per real number in
    // each 16-byte entry), the form its readers compute in
    dz* Gb = reinterpret_cast<dz*>(G) + (long)bc * m * m;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = 4 * ti + a, jj = 4 * tj + c;
        Gb[i * m + jj] = dz_from(dacc[a][c]);
        Gb[jj * m + i] = dz_from(zconj(dacc[a][c]));
      }
  }
}

// (r, c) of entry idx of a lower triangle stored row by row (idx = r (r+1)/2 + c,
// c <= r); the FP32 square root is within one of the row, fixed up exactly
__device__ __forceinline__ void tri_index(int idx, int& r, int& c) {
  int a = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
  if ((a + 1) * (a + 2) / 2 <= idx) ++a;
  if (a * (a + 1) / 2 > idx) --a;
  r = a;
  c = idx - a * (a + 1) / 2;
}

__device__ __forceinline__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = fmaxf(s, red[i]);
  return s;
}

// ---------------------------------------------------------------------------
// Stage 1: R1 = chol(G1), with a diagonal shift if a pivot fails; R1 is stored
// in FP64 and Z1 = R1^{-1} in FP32.  The elimination runs in double-float as
// G1 = L D L^dag (no square roots inside it), R1 = D^(1/2) L^dag at the end:
// each step reads the pivot d_j, and the trailing upper triangle takes
// g_rc -= conj(g_jr) g_jc / d_j, one barrier per step.  R1 only preconditions
// the second pass of CholeskyQR2, for which ~2^-44 relative accuracy is ample.
// Matrices in shared memory use the leading dimension m + 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) chol_stage1(const double2* __restrict__ G,
                                                           double2* __restrict__ R1,
                                                           float2* __restrict__ Z1,
                                                           int32_t* __restrict__ flags, int m) {
  extern __shared__ double2 dsm[];
  const int ld = m + 1, ldz = m + 4, tid = threadIdx.x;
  constexpr int nt = kThreads;
  dz* Gz = reinterpret_cast<dz*>(dsm);          // [m][ld] during the elimination
  float2* Rf = reinterpret_cast<float2*>(dsm);  // [m][ld] R1 (FP32) afterwards
  float2* Zt = Rf + m * ld;                     // [m][ldz]: column c of Z1 in row c
  __shared__ df piv[kMaxM], rs[kMaxM], rd[kMaxM];
  __shared__ float rinv[kMaxM], redf[kThreads / 32];
  __shared__ int s_fail;
  const int bc = blockIdx.x;
  const dz* Gb = reinterpret_cast<const dz*>(G) + (long)bc * m * m;
  float mx = 0.f;
  for (int i = tid; i < m; i += nt) mx = fmaxf(mx, Gb[i * m + i].re.hi);
  const float maxd = block_max(mx, redf);
  const float tol = 1e-13f * maxd;
  int32_t flag = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const df shift = df{attempt ? 1e-5f * maxd : 0.f, 0.f};
    for (int i = tid; i < m * m; i += nt) {
      const int r = i / m, c = i % m;
      if (c >= r) {
        dz v = Gb[i];
        if (r == c) v.re = df_add(v.re, shift);
        Gz[r * ld + c] = v;
      }
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      df dj = Gz[j * ld + j].re;
      const bool bad = !(dj.hi > tol);
      if (bad) dj = df{1.f, 0.f};
      if (tid == 0) {
        piv[j] = dj;
        if (bad) s_fail = 1;
      }
      const df inv = df_recip(dj);
      const int n = m - j - 1;
      for (int idx = tid; idx < n * (n + 1) / 2; idx += nt) {
        int a, b;
        tri_index(idx, a, b);
        const int r = j + 1 + b, c = j + 1 + a;  // r <= c
        // g_rc -= conj(g_jr) (g_jc / d_j)
        const dz x = Gz[j * ld + r], y = dz_scale(Gz[j * ld + c], inv);
        zacc acc = zacc_from(Gz[r * ld + c]);
        zacc_sub_mul_conj(acc, y, x);
        Gz[r * ld + c] = zacc_get(acc);
      }
      __syncthreads();
    }
    const bool failed = s_fail != 0;
    __syncthreads();  // s_fail is read by all before the next attempt resets it
    if (!failed) break;
    flag |= attempt ? 2 : 1;
  }
  // R1 = D^(1/2) L^dag
  for (int i = tid; i < m; i += nt) {
    rd[i] = df_sqrt(piv[i]);
    rs[i] = df_recip(rd[i]);
  }
  __syncthreads();
  // R1 is stored in double-float (a dz in each 16-byte entry): its only reader,
  // the second stage, works in double-float too
  dz* Rb = reinterpret_cast<dz*>(R1) + (long)bc * m * m;
  constexpr int kSlots = kMaxM * kMaxM / kThreads;
  float2 rf[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int i = tid + s * nt;
    float2 v = make_float2(0.f, 0.f);
    if (i < m * m) {
      const int r = i / m, c = i % m;
      dz o = dz_zero();
      if (c > r)
        o = dz_scale(Gz[r * ld + c], rs[r]);
      else if (c == r)
        o.re = rd[r];
      Rb[i] = o;
      v = dz_to_f(o);
    }
    rf[s] = v;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int i = tid + s * nt;
    if (i < m * m) Rf[(i / m) * ld + i % m] = rf[s];
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) rinv[i] = 1.f / Rf[i * ld + i].x;
  __syncthreads();
  // Z1 = R1^{-1} (an FP32 output; R1 is well conditioned after the shift
  // check): z_ic = (delta_ic - sum_{i<l<=c} R_il z_lc) / R_ii from the bottom,
  // column c by four lanes of one warp, so a warp barrier per row suffices
  {
    const int c = tid >> 2, part = tid & 3;
    for (int i = m - 1; i >= 0; --i) {
      float2 acc = make_float2(0.f, 0.f);
      if (c < m && i <= c)
        for (int l = i + 1 + part; l <= c; l += 4) cfma(acc, Rf[i * ld + l], Zt[c * ldz + l]);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      if (c < m && i <= c && part == 0)
        Zt[c * ldz + i] = make_float2(((i == c ? 1.f : 0.f) - acc.x) * rinv[i], -acc.y * rinv[i]);
      __syncwarp();
    }
  }
  __syncthreads();
  float2* Zb = Z1 + (long)bc * m * m;
  for (int i = tid; i < m * m; i += nt) {
    const int r = i / m, c = i % m;
    Zb[i] = c >= r ? Zt[c * ldz + r] : make_float2(0.f, 0.f);
  }
  if (tid == 0) flags[bc] = flag;
}

// ---------------------------------------------------------------------------
// Top-k eigenpairs of the real symmetric tridiagonal (d, f): Sturm
// multisection (FP32), then inverse iteration and Rayleigh quotients (FP64).
// ---------------------------------------------------------------------------

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
// d, off-diagonal f), in double-float: U has diagonals a (stored as
// reciprocals), c, c2; L has multipliers l and the row swaps in the bit mask
// piv.  The recurrences carry the running entries in registers, so the loads
// and stores of the factor arrays stay off the dependency chain.
struct TriLU {
  df a[kMaxM], c[kMaxM], c2[kMaxM], l[kMaxM];
  unsigned long long piv;
};

__device__ __forceinline__ df df_sel(bool c, df a, df b) { return df{c ? a.hi : b.hi, c ? a.lo : b.lo}; }

// The pivot choice is a select, not a branch: the lanes of the warp (one per
// eigenvalue) stay converged.
__device__ void tri_factor(const df* d, const df* f, int n, df lam, float tiny, TriLU& F) {
  const df zero = df{0.f, 0.f};
  unsigned long long piv = 0ull;
  df ai = df_sub(d[0], lam);         // current diagonal entry a_i
  df ci = n > 1 ? f[0] : zero;       // current super-diagonal entry c_i
#pragma unroll 2
  for (int i = 0; i + 1 < n; ++i) {
    const df bsub = f[i];
    const df dn = df_sub(d[i + 1], lam);  // a_{i+1} before step i
    const df cn = i + 2 < n ? f[i + 1] : zero;
    const bool sw = fabsf(ai.hi) < fabsf(bsub.hi);  // rows i and i+1 swap
    if (!sw && ai.hi == 0.f) ai = df{tiny, 0.f};
    const df num = df_sel(sw, ai, bsub), den = df_sel(sw, bsub, ai);
    const df l = df_mul(num, df_recip(den));
    piv |= (unsigned long long)sw << i;
    F.a[i] = den;
    F.c[i] = df_sel(sw, dn, ci);
    F.c2[i] = df_sel(sw, cn, zero);
    F.l[i] = l;
    const df an = df_sub(df_sel(sw, ci, dn), df_mul(l, df_sel(sw, dn, ci)));
    const df lc = df_mul(l, cn);
    ci = df_sel(sw, df_neg(lc), cn);
    ai = an;
  }
  F.a[n - 1] = ai;
  F.c[n - 1] = zero;
  F.c2[n - 1] = zero;
  F.piv = piv;
#pragma unroll 4
  for (int i = 0; i < n; ++i) {
    df v = F.a[i];
    if (fabsf(v.hi) < tiny) v = df{v.hi < 0.f ? -tiny : tiny, 0.f};
    F.a[i] = df_recip(v);
  }
}

// one step of inverse iteration: z <- (T - lam)^{-1} z with the factors F
__device__ void tri_solve(const TriLU& F, int n, df* z) {
  df zi = z[0];
#pragma unroll 4
  for (int i = 0; i + 1 < n; ++i) {
    const df zn = z[i + 1], l = F.l[i];
    const bool sw = (F.piv >> i) & 1ull;
    const df b = df_sel(sw, zn, zi);
    z[i] = b;
    zi = df_sub(df_sel(sw, zi, zn), df_mul(l, b));
  }
  z[n - 1] = zi;
  df z1 = df{0.f, 0.f}, z2 = df{0.f, 0.f};  // z_{i+1}, z_{i+2}
#pragma unroll 4
  for (int i = n - 1; i >= 0; --i) {
    const df v = df_mul(df_sub(df_sub(z[i], df_mul(F.c[i], z1)), df_mul(F.c2[i], z2)), F.a[i]);
    z[i] = v;
    z2 = z1;
    z1 = v;
  }
}

// ---------------------------------------------------------------------------
// Stage 2, one CTA per block-chirality:
//   1. R2 = chol(G2) = 1 + F in FP32 deviations (G2 = Q1^dag Q1 is 1 up to
//      rounding, so F carries FP32 relative accuracy);
//   2. R = R2 R1 = R1 + F R1 (the small correction in FP32, the sum in
//      double-float; FP64 through global scratch if F is not small);
//   3. H = R R^dag (lower triangle, double-float);
//   4. Householder tridiagonalisation of H (double-float), T = Q^dag H Q;
//   5. top-k eigenpairs of T (multisection FP32, inverse iteration FP64);
//   6. back-transform U~_k = Q Delta Z (double-float, in registers);
//   7. sigma = sqrt(lambda), W2 = R2^{-1} U~_k (FP32) and optionally
//      Sigma_k V_k^dag = U~_k^dag R (FP64).
// Global scratch per block-chirality: G2 (in; F as FP32 out), R1 (in; R out
// when the coarse test vectors are wanted), Hg (R in FP64 if F is not small).
// ---------------------------------------------------------------------------
constexpr int kBisect = 10;  // points per multisection step
constexpr int kHSlots = (kMaxM * (kMaxM + 1) / 2 + kThreads - 1) / kThreads;

__global__ void __launch_bounds__(kThreads, 2) svd_stage2(
    double2* __restrict__ G2, double2* __restrict__ R1, double2* __restrict__ Hg,
    float2* __restrict__ W2, double* __restrict__ sigma, float2* __restrict__ ctv,
    int32_t* __restrict__ flags, int m, int k) {
  extern __shared__ double2 dsm[];
  const int ld = m + 1, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  constexpr int nt = kThreads, nw = kThreads / 32;
  float2* E = reinterpret_cast<float2*>(dsm);            // [m][ld] F = R2 - 1 (steps 1-2, 7)
  float2* R1f = E + m * ld;                              // [m][m] R1 in FP32 (step 2)
  dz* Mz = reinterpret_cast<dz*>(dsm);                   // [m][ld] R, H, reflectors (2-6)
  df* Zt = reinterpret_cast<df*>(dsm + m * ld);          // [k][m] eigenvectors of T_r
  double2* Ut = dsm + m * ld;                            // [m][k] U~_k for the test vectors
  __shared__ dz uvb[2][kMaxM], pvz[kMaxM], wvw[kThreads / 32][kMaxM];
  __shared__ df taud[kMaxM], kred[nw];
  __shared__ double d[kMaxM], fo[kMaxM], lam[kMaxK];
  __shared__ df dd[kMaxM], fd[kMaxM];
  __shared__ double2 e[kMaxM], delta[kMaxM];
  __shared__ double lo[kMaxK], hi[kMaxK];
  __shared__ float d32[kMaxM], f232[kMaxM], rinv[kMaxM], redf[nw];
  __shared__ int cnt[kMaxK][kBisect];
  __shared__ int leader[kMaxK];
  __shared__ int s_fail;
  __shared__ float s_tn;
  const int bc = blockIdx.x;
  double2* Gb = G2 + (long)bc * m * m;
  float2* Fg = reinterpret_cast<float2*>(Gb);
  double2* Rg = R1 + (long)bc * m * m;
  double2* Hb = Hg + (long)bc * m * m;

  // ---- 1. R2 = 1 + F.  Every update acts on small quantities (the pivot as
  // f_jj = e_jj / (1 + sqrt(1 + e_jj)), free of cancellation).  Row j is
  // scaled by 1 / r_jj one step late, when nothing reads it any more, so each
  // step takes one barrier.
  for (int i = tid; i < m * m; i += nt) {
    const int r = i / m, c = i % m;
    if (c >= r) {
      const dz v = reinterpret_cast<const dz*>(Gb)[i];
      const df er = r == c ? df_sub(v.re, df{1.f, 0.f}) : v.re;
      E[r * ld + c] = make_float2(__fadd_rn(er.hi, er.lo), __fadd_rn(v.im.hi, v.im.lo));
    }
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  {
    float inv_prev = 1.f, f_prev = 0.f;
    for (int j = 0; j <= m; ++j) {
      float inv = 1.f, fjj = 0.f;
      if (j < m) {
        float dj = E[j * ld + j].x;
        const bool bad = !(1.f + dj > 1e-6f);
        if (bad) dj = 0.f;
        if (bad && tid == 0) s_fail = 1;
        fjj = dj / (1.f + sqrtf(1.f + dj));
        inv = 1.f / (1.f + fjj);
      }
      if (j > 0)
        for (int l = j - 1 + tid; l < m; l += nt) {
          float2& x = E[(j - 1) * ld + l];
          x = l == j - 1 ? make_float2(f_prev, 0.f) : make_float2(x.x * inv_prev, x.y * inv_prev);
        }
      if (j < m) {
        const float inv2 = inv * inv;
        // column c = tid % 64, rows j+1 + tid/64 + 4s
        const int c = tid & 63;
        if (c > j && c < m) {
          const float2 y = E[j * ld + c];
          for (int r = j + 1 + (tid >> 6); r <= c; r += 4) {
            const float2 x = E[j * ld + r];
            float2& v = E[r * ld + c];
            v = make_float2(v.x - (x.x * y.x + x.y * y.y) * inv2, v.y - (x.x * y.y - x.y * y.x) * inv2);
          }
        }
      }
      inv_prev = inv;
      f_prev = fjj;
      __syncthreads();
    }
  }

  // ---- 2. R = R1 + F R1 (R1 arrives in double-float).  With |F| < 1e-3 the
  // FP32 product F R1 errs below the FP32 rounding of the input vectors by that
  // factor; a larger F (a first Gram far from A's, e.g. the BF16 one of a
  // nearly square block) takes the product in double-float.
  {
    const dz* Rz = reinterpret_cast<const dz*>(Rg);
    dz* Hz = reinterpret_cast<dz*>(Hb);
    float dm = 0.f;
    for (int i = tid; i < m * m; i += nt) {
      const int r = i / m, c = i % m;
      float2 f = make_float2(0.f, 0.f);
      if (c >= r) {
        f = E[r * ld + c];
        dm = fmaxf(dm, fabsf(f.x) + fabsf(f.y));
      }
      Fg[i] = f;
      const dz v = Rz[i];
      R1f[i] = make_float2(v.re.hi, v.im.hi);
    }
    const bool small = block_max(dm, redf) < 1e-3f;
    const int c = tid & 63, r0 = tid >> 6;  // rows r0, r0 + 4, ...
    float2 acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = make_float2(0.f, 0.f);
    if (small) {
      if (c < m) {
        // row i of F times column c of R1: l from i to c (both triangular)
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int i = r0 + 4 * r;
          float2 s2 = make_float2(0.f, 0.f);
          for (int l = i; l <= c; ++l) cfma(s2, E[i * ld + l], R1f[l * m + c]);
          acc[r] = s2;
        }
      }
    } else if (c < m) {
      // R = (1 + F) R1 in double-float, through global scratch
      for (int i = r0; i < m; i += 4) {
        zacc sa = zacc_zero();
        for (int l = i; l <= c; ++l) {
          const float2 f = E[i * ld + l];
          dz fz;
          fz.re = l == i ? two_sum(1.f, f.x) : df{f.x, 0.f};
          fz.im = df{f.y, 0.f};
          zacc_mul(sa, fz, Rz[l * m + c]);
        }
        Hz[i * m + c] = c >= i ? zacc_get(sa) : dz_zero();
      }
    }
    __syncthreads();  // E and R1f are consumed; R (double-float) overwrites them
    if (c < m) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int i = r0 + 4 * r;
        if (i >= m) continue;
        dz rv = dz_zero();
        if (!small) {
          rv = Hz[i * m + c];
        } else if (c >= i) {
          const dz b = Rz[i * m + c];
          rv = dz{df_add(b.re, df{acc[r].x, 0.f}), df_add(b.im, df{acc[r].y, 0.f})};
        }
        Mz[i * ld + c] = rv;
        if (ctv) Rg[i * m + c] = dz_to(rv);  // R in FP64 for the test vectors
      }
    }
    __syncthreads();
  }

  // ---- 3. H = R R^dag, lower triangle: h_ij = sum_{l>=i} r_il conj(r_jl),
  // j <= i.  The results wait in registers until every thread has read R.
  {
    const int T = m * (m + 1) / 2;
    dz h[kHSlots];
#pragma unroll
    for (int s = 0; s < kHSlots; ++s) {
      const int idx = tid + s * nt;
      zacc a = zacc_zero();
      if (idx < T) {
        int i, jj;
        tri_index(idx, i, jj);
        for (int l = i; l < m; ++l) zacc_mul_conj(a, Mz[i * ld + l], Mz[jj * ld + l]);
      }
      h[s] = zacc_get(a);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kHSlots; ++s) {
      const int idx = tid + s * nt;
      if (idx < T) {
        int i, jj;
        tri_index(idx, i, jj);
        Mz[i * ld + jj] = h[s];
      }
    }
    __syncthreads();
  }

  // ---- 4. Householder tridiagonalisation on the lower triangle.  Step j
  // (reflector 1 - t u u^dag on rows j+1..): warp 0 forms u and t from column
  // j, which it holds in registers (u0 = x0 + x0 |x| / |x0|, beta = -x0 |x| /
  // |x0|, t = 1 / (|x| (|x| + |x0|)), all in double-float); then p = t A u
  // over the trailing block A (four lanes per row), w = p - (t/2)(u^dag p) u,
  // and A -= u w^dag + w u^dag, warp 0 taking A's first column, which is the
  // next step's column.  u stays in column j (rows j+1..) for step 6.  Two
  // barriers per step.
  {
    dz cv0 = dz_zero(), cv1 = dz_zero();  // warp 0: rows j + lane, j + 32 + lane of column j
    if (w == 0) {
      if (lane < m) cv0 = Mz[lane * ld];
      if (lane + 32 < m) cv1 = Mz[(lane + 32) * ld];
    }
    for (int j = 0; j + 2 < m; ++j) {
      const int n = m - j - 1, len = m - j;
      dz* uv = uvb[j & 1];
      if (w == 0) {
        dacc ta = dacc{0.f, 0.f};
        if (lane >= 2 && lane < len) {
          acc_prod(ta, cv0.re, cv0.re);
          acc_prod(ta, cv0.im, cv0.im);
        }
        if (lane + 32 < len) {
          acc_prod(ta, cv1.re, cv1.re);
          acc_prod(ta, cv1.im, cv1.im);
        }
        for (int o = 16; o > 0; o >>= 1) ta = acc_merge(ta, acc_shfl_xor(ta, o));
        const df tail = acc_get(ta);
        const dz x0 = dz_shfl(cv0, 1);
        df t = df{0.f, 0.f};
        dz beta = x0, u0 = x0;
        if (tail.hi > 0.f) {
          const df ax2 = dz_abs2(x0);
          const df nx = df_sqrt(df_add(ax2, tail));
          df ax = df{0.f, 0.f};
          if (ax2.hi > 0.f) {
            ax = df_sqrt(ax2);
            beta = dz_scale(x0, df_neg(df_mul(nx, df_recip(ax))));
            u0 = dz_sub(x0, beta);
          } else {
            beta = dz{df_neg(nx), df{0.f, 0.f}};
            u0 = dz{nx, df{0.f, 0.f}};
          }
          t = df_recip(df_mul(nx, df_add(nx, ax)));
        }
        if (lane >= 1 && lane < len) uv[lane - 1] = lane == 1 ? u0 : cv0;
        if (lane + 32 < len) uv[lane + 31] = cv1;
        if (lane == 1) Mz[(j + 1) * ld + j] = u0;
        if (lane == 0) {
          taud[j] = t;
          e[j] = dz_to(beta);
        }
      }
      __syncthreads();
      const df t = taud[j];
      if (t.hi != 0.f) {
        {
          const int a = tid >> 2, part = tid & 3;
          zacc sa = zacc_zero();
          if (a < n)
            for (int b = part; b < n; b += 4) {
              const int rr = a > b ? a : b, cc = a > b ? b : a;
              dz v = Mz[(j + 1 + rr) * ld + j + 1 + cc];
              if (b > a) v.im = df_neg(v.im);
              zacc_mul(sa, v, uv[b]);
            }
          sa = zacc_merge_xor(sa, 1);
          sa = zacc_merge_xor(sa, 2);
          const dz p = dz_scale(zacc_get(sa), t);
          dacc kc = dacc{0.f, 0.f};
          if (a < n && part == 0) {
            pvz[a] = p;
            const dz ua = uv[a];
            acc_prod(kc, ua.re, p.re);
            acc_prod(kc, ua.im, p.im);
          }
          for (int o = 16; o > 0; o >>= 1) kc = acc_merge(kc, acc_shfl_xor(kc, o));
          if (lane == 0) kred[w] = acc_get(kc);
        }
        __syncthreads();
        // w = p - K u, K = (t/2) u^dag p: every warp forms its own copy, so no
        // block barrier separates it from the update
        dz* wvz = wvw[w];
        {
          dacc ka = acc_from(kred[0]);
          for (int i = 1; i < nw; ++i) ka = acc_merge(ka, acc_from(kred[i]));
          const df K = df_half(df_mul(acc_get(ka), t));
          for (int a = lane; a < n; a += 32) wvz[a] = dz_sub(pvz[a], dz_scale(uv[a], K));
          __syncwarp();
        }
        if (w == 0) {
          const dz u0 = uv[0], w0 = wvz[0];
          dz nv[2];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int a = lane + 32 * h2;
            nv[h2] = dz_zero();
            if (a < n) {
              dz* pp = Mz + (j + 1 + a) * ld + j + 1;
              zacc acc = zacc_from(*pp);
              zacc_sub_mul_conj(acc, uv[a], w0);
              zacc_sub_mul_conj(acc, wvz[a], u0);
              const dz v = zacc_get(acc);
              *pp = v;
              nv[h2] = v;
            }
          }
          cv0 = nv[0];
          cv1 = nv[1];
        } else {
          const int T1 = n * (n - 1) / 2;
          for (int idx = tid - 32; idx < T1; idx += nt - 32) {
            int a, b;
            tri_index(idx, a, b);
            ++a;
            ++b;
            dz* pp = Mz + (j + 1 + a) * ld + j + 1 + b;
            zacc acc = zacc_from(*pp);
            zacc_sub_mul_conj(acc, uv[a], wvz[b]);
            zacc_sub_mul_conj(acc, wvz[a], uv[b]);
            *pp = zacc_get(acc);
          }
        }
      } else if (w == 0) {
        cv0 = lane < n ? Mz[(j + 1 + lane) * ld + j + 1] : dz_zero();
        cv1 = lane + 32 < n ? Mz[(j + 33 + lane) * ld + j + 1] : dz_zero();
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    dd[i] = Mz[i * ld + i].re;
    d[i] = df_to(dd[i]);
  }
  if (tid == 0 && m >= 2) e[m - 2] = dz_to(Mz[(m - 1) * ld + m - 2]);
  __syncthreads();

  // ---- 5. T = Delta T_r Delta^dag with T_r real (off-diagonal |e_j|) and the
  // phases delta_{j+1} = delta_j e_j / |e_j|; top-k eigenpairs of T_r
  for (int j = tid; j + 1 < m; j += nt) {
    const double ae = sqrt(zabs2(e[j]));
    fo[j] = ae;
    fd[j] = df_from(ae);
    f232[j] = (float)(ae * ae);
    delta[j + 1] = ae > 0 ? zscale(e[j], 1.0 / ae) : make_double2(1.0, 0.0);
  }
  for (int j = tid; j < m; j += nt) d32[j] = (float)d[j];
  __syncthreads();
  if (tid == 0) {
    delta[0] = make_double2(1.0, 0.0);
    for (int j = 1; j < m; ++j) delta[j] = zmul(delta[j - 1], delta[j]);
  } else if (w == 1) {
    float tn = 0.f;
    for (int i = lane; i < m; i += 32)
      tn = fmaxf(tn, fabsf(d32[i]) + (i > 0 ? (float)fo[i - 1] : 0.f) +
                         (i + 1 < m ? (float)fo[i] : 0.f));
    for (int o = 16; o > 0; o >>= 1) tn = fmaxf(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    if (lane == 0) s_tn = tn;
  }
  __syncthreads();
  // Gershgorin bound (widened past its FP32 rounding)
  const float tn = s_tn * 1.00001f + 1e-30f;
  const double tnorm = (double)tn;
  const float tiny = 1e-30f + 1e-15f * tn;
  if (tid < k) {
    lo[tid] = -tnorm;
    hi[tid] = tnorm;
  }
  __syncthreads();
  {
    // multisection: kBisect points per eigenvalue (the ei-th largest); the
    // k * kBisect (eigenvalue, point) pairs are spread over the block's threads.
    // The Sturm counts are FP32; the interval ends stay FP64, so that equal
    // eigenvalues end in equal intervals within FP32 rounding of their value.
    const float tiny32 = 1e-30f + 1e-20f * tn;
    constexpr double kStep = 1.0 / (kBisect + 1);
    for (int it = 0; it < 9; ++it) {
      for (int q = tid; q < k * kBisect; q += nt) {
        const int ei = q / kBisect, sp = q % kBisect;
        const double l0 = lo[ei], h0 = hi[ei];
        const double x = l0 + (h0 - l0) * ((double)(sp + 1) * kStep);
        cnt[ei][sp] = sturm_count32(d32, f232, m, (float)x, tiny32);
      }
      __syncthreads();
      if (tid < k) {
        const int target = m - 1 - tid;  // index among ascending eigenvalues
        const double l0 = lo[tid], h0 = hi[tid];
        double nl = l0, nh = h0;
        for (int q = 0; q < kBisect; ++q) {
          const double x = l0 + (h0 - l0) * ((double)(q + 1) * kStep);
          if (cnt[tid][q] > target) {
            nh = x;
            break;
          }
          nl = x;
        }
        lo[tid] = nl;
        hi[tid] = nh;
      }
      __syncthreads();
    }
  }
  if (tid < k) lam[tid] = 0.5 * (lo[tid] + hi[tid]);
  __syncthreads();
  // clusters (eigenvalues closer than 1e-6 |T|, above the FP32 resolution of
  // the multisection) are handled by their first member
  if (tid < k) leader[tid] = (tid == 0 || fabs(lam[tid - 1] - lam[tid]) > 1e-6 * tnorm) ? 1 : 0;
  __syncthreads();
  // inverse iteration in double-float (one lane per eigenvalue, all in warp 0:
  // the recurrences are serial, and on the FP32 pipe they issue at 64 times
  // the FP64 rate); the real eigenvector z_i of T_r goes to Zt row i
  if (tid < k && leader[tid]) {
    int i = tid;
    do {
      df z[kMaxM];
      TriLU F;
      tri_factor(dd, fd, m, df_from(lam[i]), tiny, F);
      // start vector: hashed entries in [0.5, 1.5), different for every
      // member of a cluster, so that the members' starts span the cluster's
      // eigenspace (starts differing by a multiple of one vector span two
      // dimensions of it, and the orthogonalisation leaves only rounding)
      for (int r = 0; r < m; ++r) {
        uint32_t h = (uint32_t)r * 0x9E3779B1u + (uint32_t)(i + 1) * 0x85EBCA77u;
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        z[r] = df{0.5f + (float)(h & 0xFFFFu) * (1.f / 65536.f), 0.f};
      }
      for (int it = 0; it < 3; ++it) {
        tri_solve(F, m, z);
        for (int pj = tid; pj < i; ++pj) {  // previous members of this cluster
          dacc dot = dacc{0.f, 0.f};
          for (int r = 0; r < m; ++r) acc_prod(dot, Zt[pj * m + r], z[r]);
          const df nd = df_neg(acc_get(dot));
          for (int r = 0; r < m; ++r) {
            dacc v = acc_from(z[r]);
            acc_prod(v, nd, Zt[pj * m + r]);
            z[r] = acc_get(v);
          }
        }
        dacc nrm = dacc{0.f, 0.f};
        for (int r = 0; r < m; ++r) acc_prod(nrm, z[r], z[r]);
        const df rs = df_recip(df_sqrt(acc_get(nrm)));
        for (int r = 0; r < m; ++r) z[r] = df_mul(z[r], rs);
      }
      // Rayleigh quotient z^T T z (double-float) refines the FP32 multisection value
      dacc rq = dacc{0.f, 0.f};
      for (int r = 0; r < m; ++r) acc_prod(rq, dd[r], df_mul(z[r], z[r]));
      for (int r = 0; r + 1 < m; ++r) acc_prod(rq, df{2.f * fd[r].hi, 2.f * fd[r].lo}, df_mul(z[r], z[r + 1]));
      lam[i] = df_to(acc_get(rq));
      for (int r = 0; r < m; ++r) Zt[i * m + r] = z[r];
      ++i;
    } while (i < k && !leader[i]);
  }
  __syncthreads();
  if (tid < k) sigma[(long)bc * k + tid] = sqrt(fmax(lam[tid], 0.0));

  // ---- 6. back-transform y = Q (Delta z), Q = H_0 H_1 ... H_{m-3}: eight
  // lanes per eigenvector, each keeping rows part + 8q in registers, so the
  // reflectors need no block barrier
  const int ci = tid >> 3, part = tid & 7;
  const bool warp_live = 4 * w < k;  // the warp holds at least one eigenvector
  dz y[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int r = part + 8 * q;
    y[q] = (ci < k && r < m) ? dz_scale(dz_from(delta[r]), Zt[ci * m + r]) : dz_zero();
  }
  if (warp_live)
    for (int j = m - 3; j >= 0; --j) {
      const df tj = taud[j];
      if (tj.hi == 0.f) continue;
      // slots whose eight rows all lie at or above row j are skipped (a
      // warp-uniform test)
      zacc sa = zacc_zero();
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (8 * q + 7 > j) {
          const int r = part + 8 * q;
          if (r > j && r < m) zacc_mulc(sa, Mz[r * ld + j], y[q]);
        }
      sa = zacc_merge_xor(sa, 1);
      sa = zacc_merge_xor(sa, 2);
      sa = zacc_merge_xor(sa, 4);
      const dz s = dz_scale(zacc_get(sa), df_neg(tj));
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (8 * q + 7 > j) {
          const int r = part + 8 * q;
          if (r > j && r < m) {
            zacc acc = zacc_from(y[q]);
            zacc_mul(acc, s, Mz[r * ld + j]);
            y[q] = zacc_get(acc);
          }
        }
    }
  __syncthreads();  // every warp is done with the reflectors

  // ---- 7. W2 = R2^{-1} U~_k (FP32; R2 = 1 + F is close to 1): substitution
  // from the bottom within each eigenvector's eight lanes
  for (int i = tid; i < m * m; i += nt) E[(i / m) * ld + i % m] = Fg[i];
  __syncthreads();
  for (int i = tid; i < m; i += nt) rinv[i] = 1.f / (1.f + E[i * ld + i].x);
  __syncthreads();
  float2 yf[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) yf[q] = dz_to_f(y[q]);
  if (warp_live)
    for (int r = m - 1; r >= 0; --r) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int l = part + 8 * q;
        if (l > r && l < m) cfma(acc, E[r * ld + l], yf[q]);
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (part == (r & 7)) {
        const float ri = rinv[r];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q == (r >> 3)) yf[q] = make_float2((yf[q].x - acc.x) * ri, (yf[q].y - acc.y) * ri);
      }
    }
  float2* Wb = W2 + (long)bc * m * k;
  if (ci < k)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = part + 8 * q;
      if (r < m) Wb[r * k + ci] = yf[q];
    }
  if (ctv) {
    // Sigma_k V_k^dag = U~_k^dag R  (R from global, FP64)
    if (ci < k)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = part + 8 * q;
        if (r < m) Ut[r * k + ci] = dz_to(y[q]);
      }
    __syncthreads();
    float2* cb = ctv + (long)bc * k * m;
    for (int idx = tid; idx < k * m; idx += nt) {
      const int i = idx / m, c = idx % m;
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l <= c; ++l) acc = zadd(acc, zmulc(Ut[l * k + i], Rg[l * m + c]));
      cb[idx] = make_float2((float)acc.x, (float)acc.y);
    }
  }
  if (tid == 0 && s_fail) flags[bc] |= 4;
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
  const size_t sm_chol = std::max(sizeof(double2) * (size_t)m * (m + 1),
                                  sizeof(float2) * ((size_t)m * (m + 1) + (size_t)m * (m + 4)));
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
