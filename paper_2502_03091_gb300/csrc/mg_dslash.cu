// mg_dslash.cu -- Wilson(-clover) operator on many right-hand sides and the
// minimal-residual smoother of the setup (paper Sec. 2, Eq. 1: m' random
// starts relaxed on D psi = 0), plus the clover-field preparation.
//
// Layout of every spinor field: float4 f[(site*12 + spin*3 + colour)*(m'/2) + pair],
// i.e. complex64 [V][4][3][m'] read two right-hand sides at a time.
//
// Smoother (per right-hand side, a = step length), the textbook MR order:
//   r_0 = -D psi_0,  w_0 = D r_0,  a_t = <w_t, r_t> / <w_t, w_t>
//   psi_{t+1} = psi_t + a_t r_t,  r_{t+1} = r_t - a_t w_t,  w_{t+1} = D r_{t+1}.
// Each iteration is ONE pass: the pass for t+1 reads r_t and w_t at the site
// and its 8 neighbours, forms r_{t+1} = r_t - a_t w_t on the fly wherever it
// is needed (bitwise the same value at every use), applies D to it, and
// writes r_{t+1}, w_{t+1} and psi_{t+1} together with the partial inner
// products of a_{t+1}.  The last iteration only updates psi; a final pass
// scales each vector to unit norm.
#include "mg_common.cuh"

namespace mg {
namespace {

// ---------------------------------------------------------------------------
// two-right-hand-side complex arithmetic on float4 = (re0, im0, re1, im1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 f4neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 f4i(float4 a) { return make_float4(-a.y, a.x, -a.w, a.z); }
__device__ __forceinline__ float4 f4mi(float4 a) { return make_float4(a.y, -a.x, a.w, -a.z); }
// acc += s * a (real s)
__device__ __forceinline__ void f4axpy(float4& acc, float s, float4 a) {
  acc.x = fmaf(s, a.x, acc.x);
  acc.y = fmaf(s, a.y, acc.y);
  acc.z = fmaf(s, a.z, acc.z);
  acc.w = fmaf(s, a.w, acc.w);
}
// acc += u * a (complex u, same for both right-hand sides)
__device__ __forceinline__ void f4cfma(float4& acc, float2 u, float4 a) {
  acc.x = fmaf(u.x, a.x, fmaf(-u.y, a.y, acc.x));
  acc.y = fmaf(u.x, a.y, fmaf(u.y, a.x, acc.y));
  acc.z = fmaf(u.x, a.z, fmaf(-u.y, a.w, acc.z));
  acc.w = fmaf(u.x, a.w, fmaf(u.y, a.z, acc.w));
}
// acc += conj(u) * a
__device__ __forceinline__ void f4cfmac(float4& acc, float2 u, float4 a) {
  acc.x = fmaf(u.x, a.x, fmaf(u.y, a.y, acc.x));
  acc.y = fmaf(u.x, a.y, fmaf(-u.y, a.x, acc.y));
  acc.z = fmaf(u.x, a.z, fmaf(u.y, a.w, acc.z));
  acc.w = fmaf(u.x, a.w, fmaf(-u.y, a.z, acc.w));
}
// per-right-hand-side complex scale: (a0 * v.xy, a1 * v.zw)
__device__ __forceinline__ float4 f4mul2(float2 a0, float2 a1, float4 v) {
  return make_float4(a0.x * v.x - a0.y * v.y, a0.x * v.y + a0.y * v.x,
                     a1.x * v.z - a1.y * v.w, a1.x * v.w + a1.y * v.z);
}

// ---------------------------------------------------------------------------
// one hop of the Wilson operator, spin-projected:
//   S = +1: acc += hw (1 - gamma_mu) U_mu(x) psi(x + mu)
//   S = -1: acc += hw (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
// With psi = (psi_u, psi_l) in the chiral basis, (1 - S gamma) chi =
// (h, -S B^dag h) with h = chi_u - S B chi_l, so only the half spinor h
// (2 spins x 3 colours) is multiplied by the link.
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.
// ---------------------------------------------------------------------------
// (B_mu chi_l)_sp given the one lower spin component it depends on
template <int MU>
__device__ __forceinline__ float4 b_row(int sp, float4 v) {
  if (MU == 0) return f4mi(v);                     // -i chi_{3-sp}
  if (MU == 1) return sp == 0 ? f4neg(v) : v;      // -chi_3, +chi_2
  if (MU == 2) return sp == 0 ? f4mi(v) : f4i(v);  // -i chi_2, +i chi_3
  return v;                                        // chi_{2+sp}
}
template <int MU>
__device__ __forceinline__ void bdag_apply(float4 g0, float4 g1, float4& o0, float4& o1) {
  // (o0, o1) = B_mu^dag (g0, g1)
  if (MU == 0) { o0 = f4i(g1); o1 = f4i(g0); }
  if (MU == 1) { o0 = g1; o1 = f4neg(g0); }
  if (MU == 2) { o0 = f4i(g0); o1 = f4mi(g1); }
  if (MU == 3) { o0 = g0; o1 = g1; }
}

// Neighbour spinor component e for this thread's two right-hand sides:
// r(y) (COMBINE = false) or r(y) - a w(y) (COMBINE = true).
template <bool COMBINE>
__device__ __forceinline__ float4 nb_load(const float4* __restrict__ r, const float4* __restrict__ w,
                                          long off, float2 a0, float2 a1) {
  const float4 v = __ldg(r + off);
  if (!COMBINE) return v;
  return f4sub(v, f4mul2(a0, a1, __ldg(w + off)));
}

template <int MU, int S, bool COMBINE>
__device__ __forceinline__ void hop(float4 acc[12], const float4* __restrict__ r,
                                    const float4* __restrict__ w, long nb, int np,
                                    const float2* __restrict__ u, float hw, float2 a0, float2 a1) {
  float2 U[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) U[i] = __ldg(u + i);
  // h = chi_u - S B chi_l, built one upper spin at a time:
  // (B chi_l)_sp = coefficient * chi_{2 + lo(sp)}
  float4 h[2][3];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const int lo = (MU == 0 || MU == 1) ? 1 - sp : sp;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 up = nb_load<COMBINE>(r, w, nb + (long)(sp * 3 + c) * np, a0, a1);
      const float4 dn = nb_load<COMBINE>(r, w, nb + (long)((2 + lo) * 3 + c) * np, a0, a1);
      const float4 bl = b_row<MU>(sp, dn);
      h[sp][c] = S > 0 ? f4sub(up, bl) : f4add(up, bl);
    }
  }
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    float4 g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      g[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (S > 0) f4cfma(g[c], U[c * 3 + d], h[sp][d]);
        else f4cfmac(g[c], U[d * 3 + c], h[sp][d]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h[sp][c] = g[c];
      f4axpy(acc[sp * 3 + c], hw, g[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float4 o0, o1;
    bdag_apply<MU>(h[0][c], h[1][c], o0, o1);
    f4axpy(acc[6 + c], -S * hw, o0);
    f4axpy(acc[9 + c], -S * hw, o1);
  }
}

struct SmoothArgs {
  const float4* in;       // dslash input r (neighbours and centre)
  const float4* win;      // w_t for the on-the-fly r_{t+1} = r_t - a_t w_t (fused pass)
  const float4* psi_src;  // centre-only psi_t
  float4* out;            // dslash result: -D psi_0, w_0, or w_{t+1}
  float4* r_out;          // r_{t+1}
  float4* psi_out;        // psi_{t+1}
  const float2* U;
  const float2* C;        // clover or nullptr
  const float2* alpha;    // [m'] step lengths a_t
  double* part;           // [m'][grid][4] partial sums
  int L[4];
  int V;
  int np;                 // m'/2
  float hw[4];
  float diag;
};

enum { MODE_NEG_D = 0, MODE_D_DOT = 1, MODE_FUSED = 2, MODE_LAST = 3 };

// Persistent smoother pass.  The right-hand sides are processed in slices of
// 2*PAIRS (outer loop) and the sites in chunks of 128/PAIRS (grid-stride
// inner loop), so that at any time the whole GPU works on one slice and the
// neighbour reads of that slice stay in L2.
//   MODE_NEG_D: out = -D in
//   MODE_D_DOT: out = D in; partials <out, in>, |out|^2
//   MODE_FUSED: s = in - a win (on the fly), out = D s, r_out = s,
//               psi_out = psi_src + a in; partials <out, s>, |out|^2
//   MODE_LAST:  psi_out = psi_src + a in; partial |psi_out|^2
template <int PAIRS, int MODE>
__global__ void __launch_bounds__(128, 3) smooth_kernel(SmoothArgs a) {
  constexpr int SPC = 128 / PAIRS;  // sites per chunk
  constexpr bool COMBINE = MODE == MODE_FUSED;
  const int p_loc = threadIdx.x % PAIRS;
  const int s_loc = threadIdx.x / PAIRS;
  const int nsl = a.np / PAIRS;
  const long nchunk = ((long)a.V + SPC - 1) / SPC;
  const int S1 = a.L[0], S2 = a.L[0] * a.L[1], S3 = a.L[0] * a.L[1] * a.L[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double red[4][PAIRS][6];

  for (int q = 0; q < nsl; ++q) {
    const int gp = q * PAIRS + p_loc;
    float2 al0 = make_float2(0.f, 0.f), al1 = al0;
    if (MODE == MODE_FUSED || MODE == MODE_LAST) {
      al0 = a.alpha[2 * gp];
      al1 = a.alpha[2 * gp + 1];
    }
    double pr[6] = {0, 0, 0, 0, 0, 0};  // (re<w,r>, im<w,r>, |w|^2) x 2 rhs
    for (long c = blockIdx.x; c < nchunk; c += gridDim.x) {
      const long xl = c * SPC + s_loc;
      if (xl >= a.V) continue;
      const int x = (int)xl;
      const long base = (long)x * 12 * a.np + gp;
      if (MODE == MODE_LAST) {
        float s2a = 0.f, s2b = 0.f;
#pragma unroll
        for (int e = 0; e < 12; ++e) {
          const float4 rc = __ldcs(a.in + base + (long)e * a.np);
          const float4 pc = __ldcs(a.psi_src + base + (long)e * a.np);
          const float4 pn = f4add(pc, f4mul2(al0, al1, rc));
          s2a += pn.x * pn.x + pn.y * pn.y;
          s2b += pn.z * pn.z + pn.w * pn.w;
          __stcs(a.psi_out + base + (long)e * a.np, pn);
        }
        pr[2] += (double)s2a;
        pr[5] += (double)s2b;
        continue;
      }
      int co[4];
      {
        int t = x;
        co[0] = t % a.L[0]; t /= a.L[0];
        co[1] = t % a.L[1]; t /= a.L[1];
        co[2] = t % a.L[2]; co[3] = t / a.L[2];
      }
      const int st[4] = {1, S1, S2, S3};
      int xf[4], xb[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        xf[mu] = co[mu] < a.L[mu] - 1 ? x + st[mu] : x - (a.L[mu] - 1) * st[mu];
        xb[mu] = co[mu] > 0 ? x - st[mu] : x + (a.L[mu] - 1) * st[mu];
      }
      // centre: s = r (or r - a w), z = (m0 + sum w) s + C s
      float4 z[12], cen[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        cen[e] = nb_load<COMBINE>(a.in, a.win, base + (long)e * a.np, al0, al1);
        z[e] = make_float4(a.diag * cen[e].x, a.diag * cen[e].y, a.diag * cen[e].z,
                           a.diag * cen[e].w);
      }
      if (a.C) {
        const float2* cl = a.C + (long)x * 72;
#pragma unroll
        for (int al = 0; al < 2; ++al)
#pragma unroll
          for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < 6; ++j)
              f4cfma(z[6 * al + i], __ldg(cl + al * 36 + i * 6 + j), cen[6 * al + j]);
      }
      const long ps = (long)12 * a.np;
      const float4* R = a.in;
      const float4* W = a.win;
      hop<0, +1, COMBINE>(z, R, W, xf[0] * ps + gp, a.np, a.U + ((long)x * 4 + 0) * 9, a.hw[0], al0, al1);
      hop<0, -1, COMBINE>(z, R, W, xb[0] * ps + gp, a.np, a.U + ((long)xb[0] * 4 + 0) * 9, a.hw[0], al0, al1);
      hop<1, +1, COMBINE>(z, R, W, xf[1] * ps + gp, a.np, a.U + ((long)x * 4 + 1) * 9, a.hw[1], al0, al1);
      hop<1, -1, COMBINE>(z, R, W, xb[1] * ps + gp, a.np, a.U + ((long)xb[1] * 4 + 1) * 9, a.hw[1], al0, al1);
      hop<2, +1, COMBINE>(z, R, W, xf[2] * ps + gp, a.np, a.U + ((long)x * 4 + 2) * 9, a.hw[2], al0, al1);
      hop<2, -1, COMBINE>(z, R, W, xb[2] * ps + gp, a.np, a.U + ((long)xb[2] * 4 + 2) * 9, a.hw[2], al0, al1);
      hop<3, +1, COMBINE>(z, R, W, xf[3] * ps + gp, a.np, a.U + ((long)x * 4 + 3) * 9, a.hw[3], al0, al1);
      hop<3, -1, COMBINE>(z, R, W, xb[3] * ps + gp, a.np, a.U + ((long)xb[3] * 4 + 3) * 9, a.hw[3], al0, al1);
      if (MODE == MODE_NEG_D) {
#pragma unroll
        for (int e = 0; e < 12; ++e) __stcs(a.out + base + (long)e * a.np, f4neg(z[e]));
        continue;
      }
      float s[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        const float4 w = z[e], r = cen[e];
        s[0] += w.x * r.x + w.y * r.y;
        s[1] += w.x * r.y - w.y * r.x;
        s[2] += w.x * w.x + w.y * w.y;
        s[3] += w.z * r.z + w.w * r.w;
        s[4] += w.z * r.w - w.w * r.z;
        s[5] += w.z * w.z + w.w * w.w;
        __stcs(a.out + base + (long)e * a.np, w);
      }
      if (MODE == MODE_FUSED) {
#pragma unroll
        for (int e = 0; e < 12; ++e) {
          const float4 rc = __ldg(a.in + base + (long)e * a.np);
          const float4 pc = __ldcs(a.psi_src + base + (long)e * a.np);
          __stcs(a.r_out + base + (long)e * a.np, cen[e]);
          __stcs(a.psi_out + base + (long)e * a.np, f4add(pc, f4mul2(al0, al1, rc)));
        }
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) pr[i] += (double)s[i];
    }
    if (MODE != MODE_NEG_D) {
      // lanes with the same pair index sit PAIRS apart within the warp
#pragma unroll
      for (int off = 16; off >= PAIRS; off >>= 1)
#pragma unroll
        for (int i = 0; i < 6; ++i) pr[i] += __shfl_xor_sync(0xffffffffu, pr[i], off);
      if (lane < PAIRS)
#pragma unroll
        for (int i = 0; i < 6; ++i) red[warp][lane][i] = pr[i];
      __syncthreads();
      if (threadIdx.x < PAIRS) {
        double t[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = red[0][threadIdx.x][i];
        for (int w = 1; w < 4; ++w)
#pragma unroll
          for (int i = 0; i < 6; ++i) t[i] += red[w][threadIdx.x][i];
        const int rhs0 = 2 * (q * PAIRS + threadIdx.x);
        double* p0 = a.part + ((long)rhs0 * gridDim.x + blockIdx.x) * 4;
        double* p1 = a.part + ((long)(rhs0 + 1) * gridDim.x + blockIdx.x) * 4;
        p0[0] = t[0]; p0[1] = t[1]; p0[2] = t[2];
        p1[0] = t[3]; p1[1] = t[4]; p1[2] = t[5];
      }
      __syncthreads();
    }
  }
}

// Second stage of the inner products, in a fixed order (deterministic):
//   mode 0: a_i = <w,r>_i / <w,w>_i,   mode 1: scale_i = 1 / |psi_i|.
__global__ void finish_reduction(const double* __restrict__ part, int G, int m, int mode,
                                 float2* __restrict__ alpha, float* __restrict__ scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double re = 0, im = 0, nn = 0;
  for (int g = 0; g < G; ++g) {
    const double* p = part + ((long)i * G + g) * 4;
    re += p[0];
    im += p[1];
    nn += p[2];
  }
  if (mode == 0) {
    alpha[i] = nn > 0 ? make_float2((float)(re / nn), (float)(im / nn)) : make_float2(0.f, 0.f);
  } else {
    scale[i] = nn > 0 ? (float)(1.0 / sqrt(nn)) : 1.0f;
  }
}

__global__ void scale_kernel(float4* __restrict__ psi, const float* __restrict__ scale, long n,
                             int np) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const int p = (int)(i % np);
    const float s0 = scale[2 * p], s1 = scale[2 * p + 1];
    float4 v = __ldcs(psi + i);
    v.x *= s0; v.y *= s0; v.z *= s1; v.w *= s1;
    __stcs(psi + i, v);
  }
}

// ---------------------------------------------------------------------------
// clover field C(x) = csw (i/2) sum_{mu<nu} sigma_mu_nu F_mu_nu(x),
// sigma_mu_nu = (i/2)[gamma_mu, gamma_nu] = i gamma_mu gamma_nu (mu != nu),
// F = (Q - Q^dag)/8, Q = sum of the four same-orientation plaquette leaves.
// In the chiral basis gamma_mu gamma_nu = diag(B_mu B_nu^dag, B_mu^dag B_nu),
// so chirality alpha gets C_alpha = -(csw/2) sum_{mu<nu} M_alpha,mu,nu (x) F_mu_nu.
// ---------------------------------------------------------------------------
struct M3 { float2 a[9]; };

__device__ __forceinline__ M3 ld_link(const float2* U, int x, int mu) {
  M3 m;
#pragma unroll
  for (int i = 0; i < 9; ++i) m.a[i] = U[((long)x * 4 + mu) * 9 + i];
  return m;
}
__device__ __forceinline__ M3 mm(const M3& p, const M3& q) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < 3; ++l) cfma(s, p.a[i * 3 + l], q.a[l * 3 + j]);
      r.a[i * 3 + j] = s;
    }
  return r;
}
__device__ __forceinline__ M3 dg(const M3& p) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.a[i * 3 + j] = cconj(p.a[j * 3 + i]);
  return r;
}

__device__ __forceinline__ void bmat(int mu, float2 B[4]) {  // row-major 2x2
  const float2 z = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f);
  const float2 mi = make_float2(0.f, -1.f), pi = make_float2(0.f, 1.f);
  if (mu == 0) { B[0] = z; B[1] = mi; B[2] = mi; B[3] = z; }
  else if (mu == 1) { B[0] = z; B[1] = make_float2(-1.f, 0.f); B[2] = one; B[3] = z; }
  else if (mu == 2) { B[0] = mi; B[1] = z; B[2] = z; B[3] = pi; }
  else { B[0] = one; B[1] = z; B[2] = z; B[3] = one; }
}

__global__ void clover_kernel(int L0, int L1, int L2, int L3, float csw,
                              const float2* __restrict__ U, float2* __restrict__ C) {
  const int V = L0 * L1 * L2 * L3;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= V) return;
  const int L[4] = {L0, L1, L2, L3};
  int co[4];
  {
    int t = x;
    co[0] = t % L0; t /= L0;
    co[1] = t % L1; t /= L1;
    co[2] = t % L2; co[3] = t / L2;
  }
  auto shift = [&](int s, int mu, int d) {
    int c[4];
    int t = s;
    c[0] = t % L0; t /= L0;
    c[1] = t % L1; t /= L1;
    c[2] = t % L2; c[3] = t / L2;
    c[mu] = (c[mu] + d + L[mu]) % L[mu];
    return c[0] + L0 * (c[1] + L1 * (c[2] + L2 * c[3]));
  };
  float2 acc[2][36];
#pragma unroll
  for (int al = 0; al < 2; ++al)
#pragma unroll
    for (int i = 0; i < 36; ++i) acc[al][i] = make_float2(0.f, 0.f);
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu) {
      const int xpm = shift(x, mu, 1), xpn = shift(x, nu, 1);
      const int xmm = shift(x, mu, -1), xmn = shift(x, nu, -1);
      const int xmmpn = shift(xmm, nu, 1), xmmmn = shift(xmm, nu, -1), xmnpm = shift(xmn, mu, 1);
      // four leaves, each a closed loop from x turning +mu -> +nu
      M3 l1 = mm(mm(ld_link(U, x, mu), ld_link(U, xpm, nu)),
                 mm(dg(ld_link(U, xpn, mu)), dg(ld_link(U, x, nu))));
      M3 l2 = mm(mm(ld_link(U, x, nu), dg(ld_link(U, xmmpn, mu))),
                 mm(dg(ld_link(U, xmm, nu)), ld_link(U, xmm, mu)));
      M3 l3 = mm(mm(dg(ld_link(U, xmm, mu)), dg(ld_link(U, xmmmn, nu))),
                 mm(ld_link(U, xmmmn, mu), ld_link(U, xmn, nu)));
      M3 l4 = mm(mm(dg(ld_link(U, xmn, nu)), ld_link(U, xmn, mu)),
                 mm(ld_link(U, xmnpm, nu), dg(ld_link(U, x, mu))));
      float2 F[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float2 qij = cadd(cadd(l1.a[i * 3 + j], l2.a[i * 3 + j]),
                                  cadd(l3.a[i * 3 + j], l4.a[i * 3 + j]));
          const float2 qji = cadd(cadd(l1.a[j * 3 + i], l2.a[j * 3 + i]),
                                  cadd(l3.a[j * 3 + i], l4.a[j * 3 + i]));
          F[i * 3 + j] = cscale(csub(qij, cconj(qji)), 0.125f);
        }
      float2 Bm[4], Bn[4];
      bmat(mu, Bm);
      bmat(nu, Bn);
      for (int al = 0; al < 2; ++al) {
        float2 M[4];  // al = 0: B_mu B_nu^dag ; al = 1: B_mu^dag B_nu
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < 2; ++l) {
              if (al == 0) cfma(v, Bm[s * 2 + l], cconj(Bn[t * 2 + l]));
              else cfma(v, cconj(Bm[l * 2 + s]), Bn[l * 2 + t]);
            }
            M[s * 2 + t] = v;
          }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j)
                cfma(acc[al][(s * 3 + i) * 6 + t * 3 + j], cscale(M[s * 2 + t], -0.5f * csw),
                     F[i * 3 + j]);
      }
    }
  float2* out = C + (long)x * 72;
#pragma unroll
  for (int al = 0; al < 2; ++al)
#pragma unroll
    for (int i = 0; i < 36; ++i) out[al * 36 + i] = acc[al][i];
}

template <int PAIRS, int MODE>
cudaError_t run_pass(const SmoothArgs& a, int grid, cudaStream_t s) {
  static const char* names[4] = {"mr_neg_dslash", "mr_dslash_dot", "mr_fused_iteration",
                                 "mr_last_update"};
  TimedScope ts(names[MODE], s);
  smooth_kernel<PAIRS, MODE><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <int PAIRS>
int persistent_grid() {
  static int cached = 0;
  if (cached) return cached;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, smooth_kernel<PAIRS, MODE_FUSED>, 128, 0);
  int g = sms * (occ > 0 ? occ : 1);
  if (g > kMaxPersistentGrid) g = kMaxPersistentGrid;
  if (g < 1) g = 1;
  cached = g;
  return g;
}

template <int PAIRS>
cudaError_t smoother_impl(const Geom& g, const float2* U, const float2* C, const float2* psi0,
                          float2* psi, char* ws, cudaStream_t s) {
  const SmoothWs lay = smooth_ws_layout(g);
  float4* r[2] = {reinterpret_cast<float4*>(ws + lay.ra), reinterpret_cast<float4*>(ws + lay.rb)};
  float4* w[2] = {reinterpret_cast<float4*>(ws + lay.wa), reinterpret_cast<float4*>(ws + lay.wb)};
  double* part = reinterpret_cast<double*>(ws + lay.part);
  float2* alpha = reinterpret_cast<float2*>(ws + lay.alpha);
  float* scale = reinterpret_cast<float*>(ws + lay.scale);
  const int G = persistent_grid<PAIRS>();

  SmoothArgs a{};
  a.U = U;
  a.C = C;
  a.alpha = alpha;
  a.part = part;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.L[i];
    a.hw[i] = g.hw[i];
  }
  a.V = (int)g.V;
  a.np = g.m / 2;
  a.diag = g.diag;
  const float4* p0 = reinterpret_cast<const float4*>(psi0);
  float4* p = reinterpret_cast<float4*>(psi);
  const int nred = (g.m + 63) / 64;
  cudaError_t e;

  // r_0 = -D psi_0
  a.in = p0;
  a.out = r[0];
  if ((e = run_pass<PAIRS, MODE_NEG_D>(a, G, s)) != cudaSuccess) return e;
  // w_0 = D r_0 -> a_0
  a.in = r[0];
  a.out = w[0];
  if ((e = run_pass<PAIRS, MODE_D_DOT>(a, G, s)) != cudaSuccess) return e;
  {
    TimedScope ts("mr_reduce", s);
    finish_reduction<<<nred, 64, 0, s>>>(part, G, g.m, 0, alpha, scale);
  }
  int cur = 0;
  for (int t = 1; t < g.niter; ++t) {
    // r_t = r_{t-1} - a w_{t-1}, w_t = D r_t, psi_t = psi_{t-1} + a r_{t-1} -> a_t
    a.in = r[cur];
    a.win = w[cur];
    a.psi_src = t == 1 ? p0 : p;
    a.out = w[cur ^ 1];
    a.r_out = r[cur ^ 1];
    a.psi_out = p;
    if ((e = run_pass<PAIRS, MODE_FUSED>(a, G, s)) != cudaSuccess) return e;
    {
    TimedScope ts("mr_reduce", s);
    finish_reduction<<<nred, 64, 0, s>>>(part, G, g.m, 0, alpha, scale);
  }
    cur ^= 1;
  }
  // psi_N = psi_{N-1} + a_{N-1} r_{N-1}, partial |psi_N|^2
  a.in = r[cur];
  a.psi_src = g.niter == 1 ? p0 : p;
  a.psi_out = p;
  if ((e = run_pass<PAIRS, MODE_LAST>(a, G, s)) != cudaSuccess) return e;
  {
    TimedScope ts("mr_reduce", s);
    finish_reduction<<<nred, 64, 0, s>>>(part, G, g.m, 1, alpha, scale);
  }
  const long n4 = g.V * 12L * (g.m / 2);
  {
    TimedScope ts("mr_scale", s);
    scale_kernel<<<1024, 256, 0, s>>>(p, scale, n4, g.m / 2);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_clover(const Geom& g, double csw, const float2* U, float2* C,
                          cudaStream_t s) {
  const int V = (int)g.V;
  TimedScope ts("clover", s);
  clover_kernel<<<(V + 127) / 128, 128, 0, s>>>(g.L[0], g.L[1], g.L[2], g.L[3], (float)csw, U, C);
  return cudaGetLastError();
}

cudaError_t launch_smoother(const Geom& g, const float2* U, const float2* C,
                            const float2* psi0, float2* psi, char* ws, cudaStream_t s) {
  if (g.m % 8 == 0) return smoother_impl<4>(g, U, C, psi0, psi, ws, s);
  return smoother_impl<2>(g, U, C, psi0, psi, ws, s);
}

}  // namespace mg
