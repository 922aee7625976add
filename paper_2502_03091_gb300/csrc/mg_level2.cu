// mg_level2.cu -- the setup one level further down.  The paper builds the
// hierarchy recursively (Sec. 2): D_{l+1} = R D_l P, and at every level l > 0
// the chiral split uses sigma_3 in place of gamma_5.
//
// The operator D_l of a level l >= 1 is a coarse nearest-neighbour stencil
// (X, Y) on a periodic lattice of extents L with n = 2 nc complex components
// per site; chirality alpha is the block of components alpha*nc .. alpha*nc +
// nc - 1.  This file holds
//   * the many-right-hand-side stencil apply out = s D_l v, optionally with
//     the per-site partial inner products the smoother needs; the operands of
//     each of the nine stencil terms are staged by bulk copies (TMA engine)
//     into a two-slot ring, so the copy of term d+1 overlaps the product of
//     term d;
//   * the smoother on D_l psi = 0 (Eq. 1 with D -> D_l): the MR recurrence of
//     the fine level, one step length per vector, as apply + reduction +
//     update kernels, then every vector to unit norm;
//   * the Galerkin product D_{l+1} = P^dag D_l P (Eq. 3), term by term.
// The truncation and the prolongator of such a level are the fine-level
// kernels run with nc rows per site and chirality (mg_truncate.cu and
// mg_coarsen.cu).
//
// Layouts (complex64): X [V][n][n], Y [V][8][n][n] (d = 0..3 hop to x + mu_d,
// d = 4..7 to x - mu_{d-4}), vectors [V][n][m] (right-hand sides fastest),
// P [V][2][nc][k], X2 [V2][2k][2k], Y2 [V2][8][2k][2k].
#include <cstdint>

#include "mg_bulk.cuh"
#include "mg_common.cuh"

namespace mg {
namespace {

constexpr int kThreads = 256;  // 16 x 16 thread tile in every kernel of this file

__device__ __forceinline__ int shift_site(int x, const int L[4], int mu, int step) {
  int c[4];
  int t = x;
  c[0] = t % L[0]; t /= L[0];
  c[1] = t % L[1]; t /= L[1];
  c[2] = t % L[2]; c[3] = t / L[2];
  c[mu] = (c[mu] + step + L[mu]) % L[mu];
  return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
}

// ---------------------------------------------------------------------------
// out(x) = s [ X(x) v(x) + sum_{d<8} Y_d(x) v(x +- mu_d) ]
// One CTA per site.  Thread (ti, tj) owns rows p*16 + ti (p < NR) and
// right-hand sides q*16 + tj (q < NQ) of the site's n x m output.  Stage d of
// the ring holds the n x n matrix of term d and the n x m source block, both
// contiguous, each brought in by one bulk copy completing on the slot's
// mbarrier.  With part != nullptr the CTA also writes, per right-hand side,
// (Re <w, v(x)>, Im <w, v(x)>, |w|^2) of its site (w = the output) in
// part[x][i].xyz (.w is left alone).
// ---------------------------------------------------------------------------
struct ApplyArgs {
  const float2* X;
  const float2* Y;
  const float2* vin;
  float2* vout;
  float4* part;
  int* status;
  int L[4];
  int n, m;
  float scale;
};

template <int NR, int NQ>
__global__ void __launch_bounds__(kThreads, 2) stencil_apply_kernel(ApplyArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ int s_abort;
  const int n = a.n, m = a.m;
  float2* Ms = reinterpret_cast<float2*>(smraw);  // [2][n*n]
  float2* Vs = Ms + 2 * n * n;                     // [2][n*m]
  const int x = blockIdx.x;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  const uint32_t mbytes = (uint32_t)(n * n) * 8u, vbytes = (uint32_t)(n * m) * 8u;

  auto issue = [&](int d) {
    const int slot = d & 1;
    const float2* M = d == 0 ? a.X + (long)x * n * n : a.Y + ((long)x * 8 + d - 1) * n * n;
    const int src = d == 0 ? x : shift_site(x, a.L, (d - 1) & 3, d <= 4 ? 1 : -1);
    mbar_expect_tx(&bar[slot], mbytes + vbytes);
    bulk_g2s(Ms + slot * n * n, M, mbytes, &bar[slot]);
    bulk_g2s(Vs + slot * n * m, a.vin + (long)src * n * m, vbytes, &bar[slot]);
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  if (tid == 0) {
    issue(0);
    issue(1);
  }

  int rows[NR], cols[NQ];
#pragma unroll
  for (int p = 0; p < NR; ++p) rows[p] = min(p * 16 + ti, n - 1);
#pragma unroll
  for (int q = 0; q < NQ; ++q) cols[q] = min(q * 16 + tj, m - 1);
  float2 acc[NR][NQ];
#pragma unroll
  for (int p = 0; p < NR; ++p)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[p][q] = make_float2(0.f, 0.f);

  int dstop = 9;
  for (int d = 0; d < 9; ++d) {
    const int slot = d & 1;
    if (!mbar_wait(&bar[slot], (uint32_t)((d >> 1) & 1))) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      dstop = d;
      break;
    }
    const float2* Mb = Ms + slot * n * n;
    const float2* Vb = Vs + slot * n * m;
    // each term in its own accumulator, then added to the sum: the rounding
    // error grows with n + 9 instead of 9 n
    float2 part[NR][NQ];
#pragma unroll
    for (int p = 0; p < NR; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) part[p][q] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int e = 0; e < n; ++e) {
      float2 av[NR], bv[NQ];
#pragma unroll
      for (int p = 0; p < NR; ++p) av[p] = Mb[rows[p] * n + e];
#pragma unroll
      for (int q = 0; q < NQ; ++q) bv[q] = Vb[e * m + cols[q]];
#pragma unroll
      for (int p = 0; p < NR; ++p)
#pragma unroll
        for (int q = 0; q < NQ; ++q) cfma(part[p][q], av[p], bv[q]);
    }
#pragma unroll
    for (int p = 0; p < NR; ++p)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[p][q] = cadd(acc[p][q], part[p][q]);
    __syncthreads();  // slot free again
    if (tid == 0 && d + 2 < 9) issue(d + 2);
  }
  if (dstop < 9) {
    // give up: report, and let the copies still in flight land before the
    // CTA's shared memory is released
    if (tid == 0) {
      atomicOr(a.status, 1);
      for (int s = dstop; s < min(dstop + 2, 9); ++s)
        (void)mbar_wait(&bar[s & 1], (uint32_t)((s >> 1) & 1));
    }
    return;
  }

  const long base = (long)x * n * m;
  float2 wr[NQ];
  float ww[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    wr[q] = make_float2(0.f, 0.f);
    ww[q] = 0.f;
  }
#pragma unroll
  for (int p = 0; p < NR; ++p) {
    const int row = p * 16 + ti;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int col = q * 16 + tj;
      if (row < n && col < m) {
        const float2 w = cscale(acc[p][q], a.scale);
        a.vout[base + (long)row * m + col] = w;
        if (a.part) {
          const float2 r = __ldg(a.vin + base + (long)row * m + col);
          cfmac(wr[q], w, r);
          ww[q] = fmaf(w.x, w.x, fmaf(w.y, w.y, ww[q]));
        }
      }
    }
  }
  if (a.part) {
    float* red = reinterpret_cast<float*>(smraw);  // [16 ti][64 rhs][3]
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int col = q * 16 + tj;
      if (col < m) {
        float* o = red + (ti * 64 + col) * 3;
        o[0] = wr[q].x;
        o[1] = wr[q].y;
        o[2] = ww[q];
      }
    }
    __syncthreads();
    if (tid < m) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int t = 0; t < 16; ++t) {
        const float* o = red + (t * 64 + tid) * 3;
        s0 += o[0];
        s1 += o[1];
        s2 += o[2];
      }
      float* dst = reinterpret_cast<float*>(a.part + (long)x * m + tid);
      dst[0] = s0;
      dst[1] = s1;
      dst[2] = s2;
    }
  }
}

// The same apply for m <= 4 right-hand sides (the Krylov solves below the
// fine level): thread (row, column) = (tid / 4, tid % 4) owns one output, so
// no thread computes a padded column.  Rows of a warp read the matrix at
// skewed columns e = (t + row) mod n, which puts the 8 rows of a warp on
// different banks (the row stride of 48 or 64 complex numbers is a multiple of
// 32 words).  Operands staged exactly as in stencil_apply_kernel.
__global__ void __launch_bounds__(kThreads) stencil_apply_small_kernel(ApplyArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ int s_abort;
  const int n = a.n, m = a.m;
  float2* Ms = reinterpret_cast<float2*>(smraw);  // [2][n*n]
  float2* Vs = Ms + 2 * n * n;                     // [2][n*m]
  const int x = blockIdx.x;
  const int tid = threadIdx.x, row = tid >> 2, col = tid & 3;
  const bool active = row < n && col < m;
  const uint32_t mbytes = (uint32_t)(n * n) * 8u, vbytes = (uint32_t)(n * m) * 8u;

  auto issue = [&](int d) {
    const int slot = d & 1;
    const float2* M = d == 0 ? a.X + (long)x * n * n : a.Y + ((long)x * 8 + d - 1) * n * n;
    const int src = d == 0 ? x : shift_site(x, a.L, (d - 1) & 3, d <= 4 ? 1 : -1);
    mbar_expect_tx(&bar[slot], mbytes + vbytes);
    bulk_g2s(Ms + slot * n * n, M, mbytes, &bar[slot]);
    bulk_g2s(Vs + slot * n * m, a.vin + (long)src * n * m, vbytes, &bar[slot]);
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  const int r = min(row, n - 1), cq = min(col, m - 1);
  float2 acc = make_float2(0.f, 0.f);
  int dstop = 9;
  for (int d = 0; d < 9; ++d) {
    const int slot = d & 1;
    if (!mbar_wait(&bar[slot], (uint32_t)((d >> 1) & 1))) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      dstop = d;
      break;
    }
    const float2* Mr = Ms + slot * n * n + r * n;
    const float2* Vb = Vs + slot * n * m;
    float2 part = make_float2(0.f, 0.f);
    int e = r % n;
    for (int t = 0; t < n; ++t) {
      cfma(part, Mr[e], Vb[e * m + cq]);
      e = e + 1 == n ? 0 : e + 1;
    }
    acc = cadd(acc, part);
    __syncthreads();  // slot free again
    if (tid == 0 && d + 2 < 9) issue(d + 2);
  }
  if (dstop < 9) {
    if (tid == 0) {
      atomicOr(a.status, 1);
      for (int s = dstop; s < min(dstop + 2, 9); ++s)
        (void)mbar_wait(&bar[s & 1], (uint32_t)((s >> 1) & 1));
    }
    return;
  }
  const long base = (long)x * n * m;
  float2 w = cscale(acc, a.scale);
  float3 pr = make_float3(0.f, 0.f, 0.f);
  if (active) {
    a.vout[base + (long)row * m + col] = w;
    if (a.part) {
      const float2 rv = __ldg(a.vin + base + (long)row * m + col);
      float2 wr = make_float2(0.f, 0.f);
      cfmac(wr, w, rv);
      pr = make_float3(wr.x, wr.y, fmaf(w.x, w.x, w.y * w.y));
    }
  }
  if (a.part) {
    float* red = reinterpret_cast<float*>(smraw);  // [64 rows][4 columns][3]
    red[tid * 3 + 0] = pr.x;
    red[tid * 3 + 1] = pr.y;
    red[tid * 3 + 2] = pr.z;
    __syncthreads();
    if (tid < m) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int rr = 0; rr < n; ++rr) {
        const float* o = red + (rr * 4 + tid) * 3;
        s0 += o[0];
        s1 += o[1];
        s2 += o[2];
      }
      float* dst = reinterpret_cast<float*>(a.part + (long)x * m + tid);
      dst[0] = s0;
      dst[1] = s1;
      dst[2] = s2;
    }
  }
}

// ---------------------------------------------------------------------------
// smoother helpers
// ---------------------------------------------------------------------------
// part[x][i].w = |psi(x)[:, i]|^2; one CTA per site, thread (g, i) sums rows
// g, g + G, ... of right-hand side i (G = 256 / m groups), then a fixed-order
// sum over g
__global__ void __launch_bounds__(kThreads) stencil_norm_kernel(const float2* __restrict__ psi,
                                                                float4* part, int n, int m) {
  __shared__ float red[kThreads];
  const int x = blockIdx.x, tid = threadIdx.x;
  const int G = kThreads / m;
  float s = 0.f;
  if (tid < G * m) {
    const int i = tid % m, g = tid / m;
    const float2* src = psi + (long)x * n * m;
    for (int r = g; r < n; r += G) {
      const float2 v = __ldg(src + (long)r * m + i);
      s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
    }
  }
  red[tid] = s;
  __syncthreads();
  if (tid < m) {
    float t = 0.f;
    for (int g = 0; g < G; ++g) t += red[g * m + tid];
    reinterpret_cast<float*>(part + (long)x * m + tid)[3] = t;
  }
}

// one CTA per right-hand side i: FP64 sums of the per-site partials in a
// fixed order (deterministic), then
//   mode 0: alpha[i] = <w, r> / <w, w> (0 if <w, w> = 0)
//   mode 1: scale[i] = 1 / |psi_i|      (1 if psi_i = 0)
__global__ void __launch_bounds__(kThreads) stencil_reduce_kernel(const float4* __restrict__ part,
                                                                  long V, int m, int mode,
                                                                  float2* alpha, float* scale) {
  __shared__ double red[3][kThreads];
  const int i = blockIdx.x, tid = threadIdx.x;
  double s0 = 0, s1 = 0, s2 = 0;
  for (long x = tid; x < V; x += kThreads) {
    const float4 p = __ldg(part + x * m + i);
    if (mode == 0) {
      s0 += p.x;
      s1 += p.y;
      s2 += p.z;
    } else {
      s2 += p.w;
    }
  }
  red[0][tid] = s0;
  red[1][tid] = s1;
  red[2][tid] = s2;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (tid < h)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + h];
    __syncthreads();
  }
  if (tid == 0) {
    if (mode == 0) {
      const double ww = red[2][0];
      alpha[i] = ww > 0 ? make_float2((float)(red[0][0] / ww), (float)(red[1][0] / ww))
                        : make_float2(0.f, 0.f);
    } else {
      const double nn = red[2][0];
      scale[i] = nn > 0 ? (float)(1.0 / sqrt(nn)) : 1.f;
    }
  }
}

// psi = psi_in + alpha r, r -= alpha w (two right-hand sides per float4)
__global__ void __launch_bounds__(kThreads) stencil_update_kernel(
    const float4* psi_in, float4* psi, float4* r, const float4* __restrict__ w,
    const float2* __restrict__ alpha, long n4, int mh) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % mh) * 2;
    const float2 a0 = __ldg(alpha + c), a1 = __ldg(alpha + c + 1);
    float4 p = psi_in[i], rr = r[i];
    const float4 ww = __ldcs(w + i);
    p.x += a0.x * rr.x - a0.y * rr.y;
    p.y += a0.x * rr.y + a0.y * rr.x;
    p.z += a1.x * rr.z - a1.y * rr.w;
    p.w += a1.x * rr.w + a1.y * rr.z;
    rr.x -= a0.x * ww.x - a0.y * ww.y;
    rr.y -= a0.x * ww.y + a0.y * ww.x;
    rr.z -= a1.x * ww.z - a1.y * ww.w;
    rr.w -= a1.x * ww.w + a1.y * ww.z;
    psi[i] = p;
    r[i] = rr;
  }
}

__global__ void __launch_bounds__(kThreads) stencil_scale_kernel(float4* psi,
                                                                 const float* __restrict__ scale,
                                                                 long n4, int mh) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4;
       i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % mh) * 2;
    const float s0 = __ldg(scale + c), s1 = __ldg(scale + c + 1);
    float4 p = psi[i];
    p.x *= s0;
    p.y *= s0;
    p.z *= s1;
    p.w *= s1;
    psi[i] = p;
  }
}

// ---------------------------------------------------------------------------
// Galerkin product of a level l >= 1, term by term (Eq. 3): for every site x
// of block j, the self term P(x)^dag X(x) P(x) and each hop
// P(x)^dag Y_d(x) P(x +- mu_d) are added to X2(j), except a hop that leaves
// the block (from a site on the block's +mu face in direction +mu, or on its
// -mu face in direction -mu), which is added to Y2_d(j).
// One CTA per block.  A term is two small complex GEMMs with the block
// structure of P (P(x) = diag(P_0(x), P_1(x)), each nc x k):
//   T = M P(y)         (n x 2k;   T[r][b, c] = sum_e M[r][b nc + e] P_b(y)[e][c])
//   acc += P(x)^dag T  (2k x 2k;  acc[a, i][.] += sum_r conj(P_a(x)[r][i]) T[a nc + r][.])
// Columns are padded to 32 per chirality (zero), so thread (ti, tj) owns rows
// p*16 + ti and columns q*16 + tj of the 64 x 64 padded tile, chirality p/2
// and q/2.
// ---------------------------------------------------------------------------
constexpr int kKP = 32;  // padded columns per chirality (k <= 32)

struct GalerkinArgs {
  const float2* X;
  const float2* Y;
  const float2* P;
  float2* X2;
  float2* Y2;
  int L[4], b[4], Lc[4];
  int nb, nc, k;
};

__global__ void __launch_bounds__(kThreads, 1) stencil_galerkin_kernel(GalerkinArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nc = a.nc, n = 2 * nc, k = a.k;
  float2* Ms = reinterpret_cast<float2*>(smraw);  // [n][n]
  float2* Pxs = Ms + n * n;                       // [2][nc][kKP]
  float2* Pys = Pxs + 2 * nc * kKP;               // [2][nc][kKP]
  float2* Ts = Pys + 2 * nc * kKP;                // [n][2 kKP]
  const int j = blockIdx.x;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  int jc[4];
  {
    int t = j;
    jc[0] = t % a.Lc[0]; t /= a.Lc[0];
    jc[1] = t % a.Lc[1]; t /= a.Lc[1];
    jc[2] = t % a.Lc[2]; jc[3] = t / a.Lc[2];
  }
  int ra[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) ra[p] = min(p * 16 + ti, n - 1);

  float2 S[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) S[p][q] = make_float2(0.f, 0.f);

  for (int pass = 0; pass < 9; ++pass) {
    const int d = pass - 1;           // stencil direction of this pass (-1: self term)
    const int mu = d & 3, st = d < 4 ? 1 : -1;
    float2 Yc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) Yc[p][q] = make_float2(0.f, 0.f);
    for (int s = 0; s < a.nb; ++s) {
      int lc[4], xo[4];
      {
        int t = s;
        lc[0] = t % a.b[0]; t /= a.b[0];
        lc[1] = t % a.b[1]; t /= a.b[1];
        lc[2] = t % a.b[2]; lc[3] = t / a.b[2];
      }
      for (int i = 0; i < 4; ++i) xo[i] = jc[i] * a.b[i] + lc[i];
      const int x = xo[0] + a.L[0] * (xo[1] + a.L[1] * (xo[2] + a.L[2] * xo[3]));
      const int y = d < 0 ? x : shift_site(x, a.L, mu, st);
      const bool face = d >= 0 && (st > 0 ? lc[mu] == a.b[mu] - 1 : lc[mu] == 0);
      __syncthreads();  // previous term done with the staged operands
      const float4* msrc = reinterpret_cast<const float4*>(
          d < 0 ? a.X + (long)x * n * n : a.Y + ((long)x * 8 + d) * n * n);
      for (int i = tid; i < n * n / 2; i += kThreads)
        reinterpret_cast<float4*>(Ms)[i] = __ldg(msrc + i);
      for (int i = tid; i < 2 * nc * kKP; i += kThreads) {
        const int al = i / (nc * kKP), rem = i % (nc * kKP);
        const int e = rem / kKP, c = rem % kKP;
        float2 vx = make_float2(0.f, 0.f), vy = vx;
        if (c < k) {
          vx = __ldg(a.P + (((long)x * 2 + al) * nc + e) * k + c);
          vy = __ldg(a.P + (((long)y * 2 + al) * nc + e) * k + c);
        }
        Pxs[i] = vx;
        Pys[i] = vy;
      }
      __syncthreads();
      // T = M P(y)
      float2 t[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) t[p][q] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int e = 0; e < nc; ++e) {
        float2 m0[4], m1[4], pv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          m0[p] = Ms[ra[p] * n + e];
          m1[p] = Ms[ra[p] * n + nc + e];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) pv[q] = Pys[((q >> 1) * nc + e) * kKP + (q & 1) * 16 + tj];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) cfma(t[p][q], (q >> 1) ? m1[p] : m0[p], pv[q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
        if (p * 16 + ti < n)
#pragma unroll
          for (int q = 0; q < 4; ++q) Ts[(p * 16 + ti) * (2 * kKP) + q * 16 + tj] = t[p][q];
      __syncthreads();
      // P(x)^dag T
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) t[p][q] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int r = 0; r < nc; ++r) {
        float2 px[4], t0[4], t1[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) px[p] = Pxs[((p >> 1) * nc + r) * kKP + (p & 1) * 16 + ti];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          t0[q] = Ts[r * (2 * kKP) + q * 16 + tj];
          t1[q] = Ts[(nc + r) * (2 * kKP) + q * 16 + tj];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) cfmac(t[p][q], px[p], (p >> 1) ? t1[q] : t0[q]);
      }
      if (face) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) Yc[p][q] = cadd(Yc[p][q], t[p][q]);
      } else {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) S[p][q] = cadd(S[p][q], t[p][q]);
      }
    }
    if (d >= 0) {
      float2* dst = a.Y2 + ((long)j * 8 + d) * (2 * k) * (2 * k);
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = (p & 1) * 16 + ti, c = (q & 1) * 16 + tj;
          if (i < k && c < k) dst[((p >> 1) * k + i) * (2 * k) + (q >> 1) * k + c] = Yc[p][q];
        }
    }
  }
  float2* dst = a.X2 + (long)j * (2 * k) * (2 * k);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = (p & 1) * 16 + ti, c = (q & 1) * 16 + tj;
      if (i < k && c < k) dst[((p >> 1) * k + i) * (2 * k) + (q >> 1) * k + c] = S[p][q];
    }
}

template <int NR, int NQ>
cudaError_t apply_t(const ApplyArgs& a, long V, cudaStream_t s) {
  const size_t stage = sizeof(float2) * 2 * ((size_t)a.n * a.n + (size_t)a.n * a.m);
  const size_t red = a.part ? sizeof(float) * 16 * 64 * 3 : 0;
  const size_t smem = stage > red ? stage : red;
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(stencil_apply_kernel<NR, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * (64 * 64 + 64 * 64) * (int)sizeof(float2));
  });
  stencil_apply_kernel<NR, NQ><<<(unsigned)V, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NR>
cudaError_t apply_q(const ApplyArgs& a, long V, cudaStream_t s) {
  switch ((a.m + 15) / 16) {
    case 1: return apply_t<NR, 1>(a, V, s);
    case 2: return apply_t<NR, 2>(a, V, s);
    case 3: return apply_t<NR, 3>(a, V, s);
    default: return apply_t<NR, 4>(a, V, s);
  }
}

cudaError_t apply_dispatch(const ApplyArgs& a, long V, cudaStream_t s) {
  if (a.m <= 4) {
    const size_t stage = sizeof(float2) * 2 * ((size_t)a.n * a.n + (size_t)a.n * a.m);
    const size_t red = a.part ? sizeof(float) * kThreads * 3 : 0;
    const size_t smem = stage > red ? stage : red;
    static PerDeviceOnce attr_once;
    attr_once.run([&] {
      cudaFuncSetAttribute(stencil_apply_small_kernel,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           2 * (64 * 64 + 64 * 4) * (int)sizeof(float2));
    });
    stencil_apply_small_kernel<<<(unsigned)V, kThreads, smem, s>>>(a);
    return cudaGetLastError();
  }
  switch ((a.n + 15) / 16) {
    case 1: return apply_q<1>(a, V, s);
    case 2: return apply_q<2>(a, V, s);
    case 3: return apply_q<3>(a, V, s);
    default: return apply_q<4>(a, V, s);
  }
}

int stream_grid(long n4) {
  const long g = (n4 + kThreads - 1) / kThreads;
  return (int)(g < 152L * 8 ? g : 152L * 8);
}

}  // namespace

cudaError_t launch_stencil_apply(const StencilGeom& sg, const float2* X, const float2* Y,
                                 const float2* vin, float2* vout, int nrhs, cudaStream_t s) {
  int* st = device_status_word();
  if (!st) return cudaGetLastError();
  ApplyArgs a{X, Y, vin, vout, nullptr, st, {sg.L[0], sg.L[1], sg.L[2], sg.L[3]}, sg.n, nrhs,
              1.f};
  TimedScope ts("c_apply", s);
  return apply_dispatch(a, sg.V, s);
}

StencilSmoothWs stencil_smooth_ws_layout(const StencilGeom& sg, int m) {
  StencilSmoothWs w{};
  const size_t field = sizeof(float2) * (size_t)sg.V * sg.n * m;
  size_t o = 0;
  w.r = o; o = align256(o + field);
  w.w = o; o = align256(o + field);
  w.part = o; o = align256(o + sizeof(float4) * (size_t)sg.V * m);
  w.alpha = o; o = align256(o + sizeof(float2) * m);
  w.scale = o; o = align256(o + sizeof(float) * m);
  w.bytes = o;
  return w;
}

cudaError_t launch_stencil_smoother(const StencilGeom& sg, int m, int niter, const float2* X,
                                    const float2* Y, const float2* psi0, float2* psi, char* ws,
                                    cudaStream_t s) {
  int* st = device_status_word();
  if (!st) return cudaGetLastError();
  const StencilSmoothWs L = stencil_smooth_ws_layout(sg, m);
  float2* r = reinterpret_cast<float2*>(ws + L.r);
  float2* w = reinterpret_cast<float2*>(ws + L.w);
  float4* part = reinterpret_cast<float4*>(ws + L.part);
  float2* alpha = reinterpret_cast<float2*>(ws + L.alpha);
  float* scale = reinterpret_cast<float*>(ws + L.scale);
  const long n4 = sg.V * sg.n * m / 2;
  const int mh = m / 2;
  const int grid = stream_grid(n4);
  cudaError_t e;
  ApplyArgs a{X, Y, psi0, r, nullptr, st, {sg.L[0], sg.L[1], sg.L[2], sg.L[3]}, sg.n, m, -1.f};
  {
    TimedScope ts("c_mr_apply", s);
    if ((e = apply_dispatch(a, sg.V, s)) != cudaSuccess) return e;  // r = -D psi0
  }
  for (int it = 0; it < niter; ++it) {
    a.vin = r;
    a.vout = w;
    a.part = part;
    a.scale = 1.f;
    {
      TimedScope ts("c_mr_apply", s);
      if ((e = apply_dispatch(a, sg.V, s)) != cudaSuccess) return e;  // w = D r, partials
    }
    {
      TimedScope ts("c_mr_reduce", s);
      stencil_reduce_kernel<<<m, kThreads, 0, s>>>(part, sg.V, m, 0, alpha, scale);
    }
    {
      TimedScope ts("c_mr_update", s);
      stencil_update_kernel<<<grid, kThreads, 0, s>>>(
          reinterpret_cast<const float4*>(it == 0 ? psi0 : psi), reinterpret_cast<float4*>(psi),
          reinterpret_cast<float4*>(r), reinterpret_cast<const float4*>(w), alpha, n4, mh);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    TimedScope ts("c_mr_norm", s);
    stencil_norm_kernel<<<(unsigned)sg.V, kThreads, 0, s>>>(psi, part, sg.n, m);
    stencil_reduce_kernel<<<m, kThreads, 0, s>>>(part, sg.V, m, 1, alpha, scale);
  }
  {
    TimedScope ts("c_mr_scale", s);
    stencil_scale_kernel<<<grid, kThreads, 0, s>>>(reinterpret_cast<float4*>(psi), scale, n4, mh);
  }
  return cudaGetLastError();
}

cudaError_t launch_stencil_galerkin(const Geom& g, const float2* X, const float2* Y,
                                    const float2* P, float2* X2, float2* Y2, cudaStream_t s) {
  GalerkinArgs a;
  a.X = X;
  a.Y = Y;
  a.P = P;
  a.X2 = X2;
  a.Y2 = Y2;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.L[i];
    a.b[i] = g.b[i];
    a.Lc[i] = g.Lc[i];
  }
  a.nb = g.nb;
  a.nc = g.rps;
  a.k = g.k;
  const int n = 2 * a.nc;
  const size_t smem =
      sizeof(float2) * ((size_t)n * n + 4 * (size_t)a.nc * kKP + (size_t)n * 2 * kKP);
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(stencil_galerkin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float2) * (64 * 64 + 4 * 32 * kKP + 64 * 2 * kKP)));
  });
  TimedScope ts("c_galerkin", s);
  stencil_galerkin_kernel<<<(unsigned)g.nblk, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mg
