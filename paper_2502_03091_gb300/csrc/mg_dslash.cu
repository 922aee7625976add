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

// ---------------------------------------------------------------------------
// t-marching smoother pass.
//
// Internal ("slab") layout of r, w and psi: for right-hand-side slice q of
// 2*PAIRS vectors, float4 f[((q*V + x)*12 + e)*PAIRS + p] -- every site's
// 12 x 2*PAIRS complex numbers of one slice are contiguous.
//
// One CTA owns a patch of kSPC consecutive sites of a timeslice (spatial
// lexicographic index p0 .. p0+kSPC-1) for one slice, and marches t = 0..Lt-1.
// A ring of kRing rows of the dslash input s (s = r, or s = r - a w formed
// when the row is staged) lives in shared memory: hops that stay in the patch
// (x, and y when a patch spans several x-rows) and the two t-hops read the
// ring; only hops that leave the patch go to global memory (L2).  Producer
// warps stage row t+2 while consumer warps apply D to row t; one barrier per
// step.  Ring slot of row r (r = -1 .. Lt+1): (r + 1) & 3.
// ---------------------------------------------------------------------------
constexpr int kSPC = 32;
constexpr int kRing = 4;

struct MarchArgs {
  const float4* in;       // s source r_t (slab) or psi_0 (ABI layout)
  const float4* win;      // w_t (slab), fused pass
  const float4* psi_src;  // psi_t, fused pass (ABI layout for psi_0, else slab)
  float4* out;            // D s (slab)
  float4* r_out;          // r_{t+1} = s (slab), fused pass
  float4* psi_out;        // psi_{t+1} (slab), fused pass
  const float2* U;
  const float2* C;        // clover or nullptr
  const float2* alpha;    // [m'] step lengths
  double* part;           // [m'][npatch][4]
  int L[4];
  int Vs, V, np, npatch;
  int in_abi, psi_abi;    // layouts of `in` and `psi_src`
  float hw[4];
  float diag;
};

enum { MODE_NEG_D = 0, MODE_D_DOT = 1 };

__device__ __forceinline__ long slab_index(int q, int V, int x, int e, int PAIRS, int p) {
  return (((long)q * V + x) * 12 + e) * PAIRS + p;
}

// One hop, split between two partner lanes (hf = 0, 1): lane hf forms the
// half-spinor row h_hf = chi_hf - S (B chi_l)_hf (colour vector), multiplies
// it by U (or U^dag) and accumulates into the two output spins it owns,
// hf (upper) and 2 + hf (lower):
//   upper: acc_u += hw g_hf,   lower: acc_l += -S hw (B^dag g)_hf,
// where (B^dag g)_hf needs the partner's g for mu = x, y (one shuffle).
//
// load_half fetches the lane's inputs (chi_hf and the lower spin entering
// (B chi_l)_hf) from a neighbour whose component e is at src[e * es]; src is
// a generic pointer (shared-memory ring or global memory).
template <int MU>
__device__ __forceinline__ void load_half(const float4* src, int es, int hf, float4 up[3],
                                          float4 dn[3]) {
  const int lo = (MU == 0 || MU == 1) ? 1 - hf : hf;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    up[c] = src[(hf * 3 + c) * es];
    dn[c] = src[((2 + lo) * 3 + c) * es];
  }
}

template <int MU, int S>
__device__ __forceinline__ void apply_half(float4 acc_u[3], float4 acc_l[3], int hf,
                                           const float4 up[3], const float4 dn[3],
                                           const float2* __restrict__ u, float hw) {
  float2 U[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) U[i] = __ldg(u + i);
  float4 h[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // (B chi_l)_hf: mu=x: -i chi_{3-hf}; mu=y: -chi_3 / +chi_2; mu=z: -i chi_2 / +i chi_3; t: chi_{2+hf}
    float4 bl;
    if (MU == 0) bl = f4mi(dn[c]);
    else if (MU == 1) bl = hf == 0 ? f4neg(dn[c]) : dn[c];
    else if (MU == 2) bl = hf == 0 ? f4mi(dn[c]) : f4i(dn[c]);
    else bl = dn[c];
    h[c] = S > 0 ? f4sub(up[c], bl) : f4add(up[c], bl);
  }
  float4 g[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (S > 0) f4cfma(g[c], U[c * 3 + d], h[d]);
      else f4cfmac(g[c], U[d * 3 + c], h[d]);
    }
    f4axpy(acc_u[c], hw, g[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float4 v = g[c];
    if (MU == 0 || MU == 1) {
      v.x = __shfl_xor_sync(0xffffffffu, v.x, 1);
      v.y = __shfl_xor_sync(0xffffffffu, v.y, 1);
      v.z = __shfl_xor_sync(0xffffffffu, v.z, 1);
      v.w = __shfl_xor_sync(0xffffffffu, v.w, 1);
    }
    // (B^dag g)_hf: x: i g_{1-hf}; y: g_1 / -g_0; z: i g_0 / -i g_1; t: g_hf
    float4 b;
    if (MU == 0) b = f4i(v);
    else if (MU == 1) b = hf == 0 ? v : f4neg(v);
    else if (MU == 2) b = hf == 0 ? f4i(v) : f4mi(v);
    else b = v;
    f4axpy(acc_l[c], -S * hw, b);
  }
}

template <int PAIRS>
constexpr int march_threads() {
  return 2 * kSPC * PAIRS;
}

// Dslash pass.  MODE_NEG_D: out = -D in (in = psi_0, ABI layout);
// MODE_D_DOT: out = D in (in = r, slab) with partials <out, in>, |out|^2.
// Each lane (site, pair, spin half hf) also stages its own 6 components of
// ring row t+2: loads are issued before the compute of row t and stored into
// the ring after the step's first barrier.
template <int PAIRS, int MODE>
__global__ void __launch_bounds__(march_threads<PAIRS>(), 2) march_kernel(MarchArgs a) {
  constexpr int NC = 2 * kSPC * PAIRS;  // lanes: (site, pair, spin half)
  constexpr int SS = 12 * PAIRS + 4;    // padded ring site stride (float4)
  constexpr int NW = NC / 32;
  extern __shared__ float4 ring[];      // [kRing][kSPC][SS]
  __shared__ double red[NW][PAIRS][6];
  const int q = blockIdx.x / a.npatch, patch = blockIdx.x % a.npatch;
  const int p0 = patch * kSPC;
  const int Lt = a.L[3];
  const int hf = threadIdx.x & 1;
  const int sp_idx = threadIdx.x >> 1;
  const int s_loc = sp_idx / PAIRS, p = sp_idx % PAIRS;
  const int gp = q * PAIRS + p;
  const int xyz = p0 + s_loc;
  const bool valid = xyz < a.Vs;
  const bool abi = MODE == MODE_NEG_D;  // input layout
  const int ges = abi ? a.np : PAIRS;   // global component stride
  int nf[3] = {0, 0, 0}, nb[3] = {0, 0, 0};
  {
    int c[3];
    int t = xyz;
    c[0] = t % a.L[0]; t /= a.L[0];
    c[1] = t % a.L[1]; c[2] = t / a.L[1];
    const int sst[3] = {1, a.L[0], a.L[0] * a.L[1]};
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      nf[mu] = c[mu] < a.L[mu] - 1 ? xyz + sst[mu] : xyz - (a.L[mu] - 1) * sst[mu];
      nb[mu] = c[mu] > 0 ? xyz - sst[mu] : xyz + (a.L[mu] - 1) * sst[mu];
    }
  }
  // global address of component 0 of site x for this lane's pair
  auto gaddr = [&](int x) -> const float4* {
    return abi ? a.in + (long)x * 12 * a.np + gp : a.in + slab_index(q, a.V, x, 0, PAIRS, p);
  };
  // staging of this lane's 6 components of row r (-1 <= r <= Lt)
  auto stage_load = [&](int r, float4 sv[6]) {
    if (!valid) return;
    const float4* src = gaddr(((r + Lt) % Lt) * a.Vs + xyz);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int e = k < 3 ? hf * 3 + k : (2 + hf) * 3 + k - 3;
      sv[k] = __ldg(src + e * ges);
    }
  };
  auto stage_store = [&](int r, const float4 sv[6]) {
    if (!valid) return;
    float4* dst = ring + ((r + 1) & 3) * kSPC * SS + s_loc * SS + p;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int e = k < 3 ? hf * 3 + k : (2 + hf) * 3 + k - 3;
      dst[e * PAIRS] = sv[k];
    }
  };

  double pr[6] = {0, 0, 0, 0, 0, 0};
  {
    float4 sv[6];
    for (int r = -1; r <= 1; ++r) {
      stage_load(r, sv);
      stage_store(r, sv);
    }
  }
  __syncthreads();
  for (int t = 0; t < Lt; ++t) {
    float4 sv[6];
    const bool do_stage = t + 2 <= Lt;
    if (do_stage) stage_load(t + 2, sv);
    {
      // every lane takes part in the shuffles; lanes of an invalid site
      // compute on site p0 and discard the result
      const int xyzc = valid ? xyz : p0;
      const float4* ring_t = ring + ((t + 1) & 3) * kSPC * SS;
      const float4* ring_f = ring + ((t + 2) & 3) * kSPC * SS;
      const float4* ring_b = ring + (t & 3) * kSPC * SS;
      const int sl = xyzc - p0;
      const int x = t * a.Vs + xyzc;
      const int tb = (t - 1 + Lt) % Lt;
      const float4* cen = ring_t + sl * SS + p;  // component e at cen[e * PAIRS]
      float4 zu[3], zl[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 cu = cen[(hf * 3 + c) * PAIRS], cl4 = cen[((2 + hf) * 3 + c) * PAIRS];
        zu[c] = make_float4(a.diag * cu.x, a.diag * cu.y, a.diag * cu.z, a.diag * cu.w);
        zl[c] = make_float4(a.diag * cl4.x, a.diag * cl4.y, a.diag * cl4.z, a.diag * cl4.w);
      }
      if (a.C) {
        // row (alpha, spin hf, colour c) of the chirality-alpha 6x6 block
        const float2* cl = a.C + (long)x * 72;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            f4cfma(zu[c], __ldg(cl + (hf * 3 + c) * 6 + j), cen[j * PAIRS]);
            f4cfma(zl[c], __ldg(cl + 36 + (hf * 3 + c) * 6 + j), cen[(6 + j) * PAIRS]);
          }
      }
      const float2* Ux = a.U + (long)x * 36;
      const long tV = (long)t * a.Vs;
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) {
        // forward and backward neighbours: ring if inside the patch, else global
        const int f = valid ? nf[mu] : p0, b = valid ? nb[mu] : p0;
        const int lf = f - p0, lb = b - p0;
        const bool rf = lf >= 0 && lf < kSPC && f < a.Vs, rb = lb >= 0 && lb < kSPC && b < a.Vs;
        const float4* pf = rf ? ring_t + lf * SS + p : gaddr(t * a.Vs + f);
        const float4* pb = rb ? ring_t + lb * SS + p : gaddr(t * a.Vs + b);
        const int esf = rf ? PAIRS : ges, esb = rb ? PAIRS : ges;
        float4 uf[3], df[3], ub[3], db[3];
        if (mu == 0) {
          load_half<0>(pf, esf, hf, uf, df);
          load_half<0>(pb, esb, hf, ub, db);
          apply_half<0, +1>(zu, zl, hf, uf, df, Ux + 0, a.hw[0]);
          apply_half<0, -1>(zu, zl, hf, ub, db, a.U + (tV + b) * 36 + 0, a.hw[0]);
        } else if (mu == 1) {
          load_half<1>(pf, esf, hf, uf, df);
          load_half<1>(pb, esb, hf, ub, db);
          apply_half<1, +1>(zu, zl, hf, uf, df, Ux + 9, a.hw[1]);
          apply_half<1, -1>(zu, zl, hf, ub, db, a.U + (tV + b) * 36 + 9, a.hw[1]);
        } else {
          load_half<2>(pf, esf, hf, uf, df);
          load_half<2>(pb, esb, hf, ub, db);
          apply_half<2, +1>(zu, zl, hf, uf, df, Ux + 18, a.hw[2]);
          apply_half<2, -1>(zu, zl, hf, ub, db, a.U + (tV + b) * 36 + 18, a.hw[2]);
        }
      }
      {
        float4 uf[3], df[3], ub[3], db[3];
        load_half<3>(ring_f + sl * SS + p, PAIRS, hf, uf, df);
        load_half<3>(ring_b + sl * SS + p, PAIRS, hf, ub, db);
        apply_half<3, +1>(zu, zl, hf, uf, df, Ux + 27, a.hw[3]);
        apply_half<3, -1>(zu, zl, hf, ub, db, a.U + ((long)tb * a.Vs + xyzc) * 36 + 27, a.hw[3]);
      }
      if (valid) {
        const long so = slab_index(q, a.V, x, 0, PAIRS, p);
        const int eu = hf * 3, el = (2 + hf) * 3;
        if (MODE == MODE_NEG_D) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            __stcs(a.out + so + (eu + c) * PAIRS, f4neg(zu[c]));
            __stcs(a.out + so + (el + c) * PAIRS, f4neg(zl[c]));
          }
        } else {
          float s6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const int e = k < 3 ? eu + k : el + k - 3;
            const float4 w = k < 3 ? zu[k] : zl[k - 3], r = cen[e * PAIRS];
            s6[0] += w.x * r.x + w.y * r.y;
            s6[1] += w.x * r.y - w.y * r.x;
            s6[2] += w.x * w.x + w.y * w.y;
            s6[3] += w.z * r.z + w.w * r.w;
            s6[4] += w.z * r.w - w.w * r.z;
            s6[5] += w.z * w.z + w.w * w.w;
            __stcs(a.out + so + e * PAIRS, w);
          }
#pragma unroll
          for (int i = 0; i < 6; ++i) pr[i] += (double)s6[i];
        }
      }
    }
    // row t+2 goes into the slot of row t-2 (free once every lane is past step t)
    __syncthreads();
    if (do_stage) stage_store(t + 2, sv);
    __syncthreads();
  }
  if (MODE != MODE_NEG_D) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // lane = 2 * (s * PAIRS + p) + hf: sum over hf and s, keep p
#pragma unroll
    for (int i = 0; i < 6; ++i) pr[i] += __shfl_xor_sync(0xffffffffu, pr[i], 1);
#pragma unroll
    for (int off = 16; off >= 2 * PAIRS; off >>= 1)
#pragma unroll
      for (int i = 0; i < 6; ++i) pr[i] += __shfl_xor_sync(0xffffffffu, pr[i], off);
    if (lane < 2 * PAIRS && (lane & 1) == 0)
#pragma unroll
      for (int i = 0; i < 6; ++i) red[warp][lane >> 1][i] = pr[i];
    __syncthreads();
    if (threadIdx.x < PAIRS) {
      double tt[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) tt[i] = red[0][threadIdx.x][i];
      for (int w = 1; w < NW; ++w)
#pragma unroll
        for (int i = 0; i < 6; ++i) tt[i] += red[w][threadIdx.x][i];
      const int rhs0 = 2 * (q * PAIRS + threadIdx.x);
      double* q0 = a.part + ((long)rhs0 * a.npatch + patch) * 4;
      double* q1 = a.part + ((long)(rhs0 + 1) * a.npatch + patch) * 4;
      q0[0] = tt[0]; q0[1] = tt[1]; q0[2] = tt[2];
      q1[0] = tt[3]; q1[1] = tt[4]; q1[2] = tt[5];
    }
  }
}

// MR update between two dslash passes (streaming, slab layout):
//   r <- r - a w  (r_{t+1}),   psi_out <- psi_src + a r_t   (psi_src in the ABI
// layout for psi_0).  One float4 (two right-hand sides) per thread.
template <int PAIRS>
__global__ void mr_update(float4* __restrict__ r, const float4* __restrict__ w,
                          const float4* __restrict__ psi_src, float4* __restrict__ psi_out,
                          const float2* __restrict__ alpha, int V, int np, int psi_abi) {
  const long n = (long)V * 12 * np;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const int p = (int)(i % PAIRS);
    long rr = i / PAIRS;
    const int e = (int)(rr % 12);
    rr /= 12;
    const int x = (int)(rr % V);
    const int q = (int)(rr / V);
    const int gp = q * PAIRS + p;
    const float2 a0 = alpha[2 * gp], a1 = alpha[2 * gp + 1];
    const float4 rv = __ldcs(r + i), wv = __ldcs(w + i);
    const float4 pv = psi_abi ? __ldcs(psi_src + ((long)x * 12 + e) * np + gp) : __ldcs(psi_src + i);
    __stcs(r + i, f4sub(rv, f4mul2(a0, a1, wv)));
    __stcs(psi_out + i, f4add(pv, f4mul2(a0, a1, rv)));
  }
}

// psi_N = psi_{N-1} + a r_{N-1} (slab), partial |psi_N|^2 per right-hand side.
// Grid: one CTA per (slice, patch), looping over t; thread = (site, pair).
template <int PAIRS>
__global__ void __launch_bounds__(kSPC * PAIRS) last_update(MarchArgs a) {
  constexpr int NC = kSPC * PAIRS, NW = NC / 32;
  __shared__ double red[NW][PAIRS][2];
  const int q = blockIdx.x / a.npatch, patch = blockIdx.x % a.npatch;
  const int s_loc = threadIdx.x / PAIRS, p = threadIdx.x % PAIRS;
  const int gp = q * PAIRS + p;
  const int xyz = patch * kSPC + s_loc;
  const float2 al0 = a.alpha[2 * gp], al1 = a.alpha[2 * gp + 1];
  double n0 = 0, n1 = 0;
  if (xyz < a.Vs) {
    for (int t = 0; t < a.L[3]; ++t) {
      const int x = t * a.Vs + xyz;
      const long so = slab_index(q, a.V, x, 0, PAIRS, p);
      const long ao = (long)x * 12 * a.np + gp;
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        const float4 rc = __ldcs(a.in + so + e * PAIRS);
        const float4 pc = a.psi_abi ? __ldcs(a.psi_src + ao + (long)e * a.np)
                                    : __ldcs(a.psi_src + so + e * PAIRS);
        const float4 pn = f4add(pc, f4mul2(al0, al1, rc));
        s0 += pn.x * pn.x + pn.y * pn.y;
        s1 += pn.z * pn.z + pn.w * pn.w;
        __stcs(a.psi_out + so + e * PAIRS, pn);
      }
      n0 += (double)s0;
      n1 += (double)s1;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off >= PAIRS; off >>= 1) {
    n0 += __shfl_xor_sync(0xffffffffu, n0, off);
    n1 += __shfl_xor_sync(0xffffffffu, n1, off);
  }
  if (lane < PAIRS) {
    red[warp][lane][0] = n0;
    red[warp][lane][1] = n1;
  }
  __syncthreads();
  if (threadIdx.x < PAIRS) {
    double t0 = 0, t1 = 0;
    for (int w = 0; w < NW; ++w) {
      t0 += red[w][threadIdx.x][0];
      t1 += red[w][threadIdx.x][1];
    }
    const int rhs0 = 2 * (q * PAIRS + threadIdx.x);
    double* q0 = a.part + ((long)rhs0 * a.npatch + patch) * 4;
    double* q1 = a.part + ((long)(rhs0 + 1) * a.npatch + patch) * 4;
    q0[0] = 0; q0[1] = 0; q0[2] = t0;
    q1[0] = 0; q1[1] = 0; q1[2] = t1;
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
    const double* pp = part + ((long)i * G + g) * 4;
    re += pp[0];
    im += pp[1];
    nn += pp[2];
  }
  if (mode == 0) {
    alpha[i] = nn > 0 ? make_float2((float)(re / nn), (float)(im / nn)) : make_float2(0.f, 0.f);
  } else {
    scale[i] = nn > 0 ? (float)(1.0 / sqrt(nn)) : 1.0f;
  }
}

__global__ void fill_kernel(float* __restrict__ v, int n, float x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = x;
}

// psi (ABI layout) = scale * psi_slab
template <int PAIRS>
__global__ void scale_to_abi(const float4* __restrict__ src, float4* __restrict__ dst,
                             const float* __restrict__ scale, int V, int np) {
  const long n = (long)V * 12 * np;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    // i enumerates the slab: ((q*V + x)*12 + e)*PAIRS + p
    const int p = (int)(i % PAIRS);
    long r = i / PAIRS;
    const int e = (int)(r % 12);
    r /= 12;
    const int x = (int)(r % V);
    const int q = (int)(r / V);
    const int gp = q * PAIRS + p;
    float4 v = __ldcs(src + i);
    const float s0 = scale[2 * gp], s1 = scale[2 * gp + 1];
    v.x *= s0; v.y *= s0; v.z *= s1; v.w *= s1;
    __stcs(dst + ((long)x * 12 + e) * np + gp, v);
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
cudaError_t run_march(const MarchArgs& a, int nsl, cudaStream_t s) {
  static const char* names[2] = {"mr_neg_dslash", "mr_dslash_dot"};
  constexpr int SS = 12 * PAIRS + 4;
  const size_t smem = sizeof(float4) * (size_t)kRing * kSPC * SS;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(march_kernel<PAIRS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  TimedScope ts(names[MODE], s);
  march_kernel<PAIRS, MODE><<<nsl * a.npatch, march_threads<PAIRS>(), smem, s>>>(a);
  return cudaGetLastError();
}

template <int PAIRS>
cudaError_t smoother_impl(const Geom& g, const float2* U, const float2* C, const float2* psi0,
                          float2* psi, char* ws, cudaStream_t s) {
  const SmoothWs lay = smooth_ws_layout(g);
  float4* r = reinterpret_cast<float4*>(ws + lay.ra);
  float4* w = reinterpret_cast<float4*>(ws + lay.wa);
  float4* ps = reinterpret_cast<float4*>(ws + lay.ps);
  double* part = reinterpret_cast<double*>(ws + lay.part);
  float2* alpha = reinterpret_cast<float2*>(ws + lay.alpha);
  float* scale = reinterpret_cast<float*>(ws + lay.scale);

  MarchArgs a{};
  a.U = U;
  a.C = C;
  a.alpha = alpha;
  a.part = part;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.L[i];
    a.hw[i] = g.hw[i];
  }
  a.V = (int)g.V;
  a.Vs = (int)(g.V / g.L[3]);
  a.np = g.m / 2;
  a.npatch = (a.Vs + kSPC - 1) / kSPC;
  a.diag = g.diag;
  const int nsl = a.np / PAIRS;
  const int G = a.npatch;  // partial sums per right-hand side
  const float4* p0 = reinterpret_cast<const float4*>(psi0);
  const int nred = (g.m + 63) / 64;
  cudaError_t e;
  auto reduce = [&](int mode) {
    TimedScope ts("mr_reduce", s);
    finish_reduction<<<nred, 64, 0, s>>>(part, G, g.m, mode, alpha, scale);
  };

  // r_0 = -D psi_0  (psi_0 in the ABI layout)
  a.in = p0;
  a.out = r;
  if ((e = run_march<PAIRS, MODE_NEG_D>(a, nsl, s)) != cudaSuccess) return e;
  // w_0 = D r_0 -> a_0
  a.in = r;
  a.out = w;
  if ((e = run_march<PAIRS, MODE_D_DOT>(a, nsl, s)) != cudaSuccess) return e;
  reduce(0);
  for (int t = 1; t < g.niter; ++t) {
    // r_t = r_{t-1} - a w_{t-1}, psi_t = psi_{t-1} + a r_{t-1}; w_t = D r_t -> a_t
    {
      TimedScope ts("mr_update", s);
      mr_update<PAIRS><<<4096, 256, 0, s>>>(r, w, t == 1 ? p0 : ps, ps, alpha, a.V, a.np,
                                            t == 1 ? 1 : 0);
    }
    if ((e = run_march<PAIRS, MODE_D_DOT>(a, nsl, s)) != cudaSuccess) return e;
    reduce(0);
  }
  // psi_N = psi_{N-1} + a_{N-1} r_{N-1}, partial |psi_N|^2
  a.in = r;
  a.psi_src = g.niter == 1 ? p0 : ps;
  a.psi_abi = g.niter == 1;
  a.psi_out = ps;
  {
    TimedScope ts("mr_last_update", s);
    last_update<PAIRS><<<nsl * a.npatch, kSPC * PAIRS, 0, s>>>(a);
  }
  reduce(1);
  {
    TimedScope ts("mr_scale", s);
    scale_to_abi<PAIRS><<<2048, 256, 0, s>>>(ps, reinterpret_cast<float4*>(psi), scale, a.V, a.np);
  }
  return cudaGetLastError();
}

template <int PAIRS>
cudaError_t dirac_impl(const Geom& g, const float2* U, const float2* C, const float2* in,
                       float2* out, char* ws, cudaStream_t s) {
  const SmoothWs lay = smooth_ws_layout(g);
  float4* tmp = reinterpret_cast<float4*>(ws + lay.ra);
  float* scale = reinterpret_cast<float*>(ws + lay.scale);
  MarchArgs a{};
  a.U = U;
  a.C = C;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.L[i];
    a.hw[i] = g.hw[i];
  }
  a.V = (int)g.V;
  a.Vs = (int)(g.V / g.L[3]);
  a.np = g.m / 2;
  a.npatch = (a.Vs + kSPC - 1) / kSPC;
  a.diag = g.diag;
  a.in = reinterpret_cast<const float4*>(in);
  a.in_abi = 1;
  a.out = tmp;
  cudaError_t e = run_march<PAIRS, MODE_NEG_D>(a, a.np / PAIRS, s);
  if (e != cudaSuccess) return e;
  {
    TimedScope ts("fill", s);
    fill_kernel<<<1, 64, 0, s>>>(scale, g.m, -1.0f);
  }
  TimedScope ts("mr_scale", s);
  scale_to_abi<PAIRS><<<2048, 256, 0, s>>>(tmp, reinterpret_cast<float4*>(out), scale, a.V, a.np);
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

cudaError_t launch_dirac(const Geom& g, const float2* U, const float2* C, const float2* in,
                         float2* out, char* ws, cudaStream_t s) {
  if (g.m % 8 == 0) return dirac_impl<4>(g, U, C, in, out, ws, s);
  return dirac_impl<2>(g, U, C, in, out, ws, s);
}

cudaError_t launch_smoother(const Geom& g, const float2* U, const float2* C,
                            const float2* psi0, float2* psi, char* ws, cudaStream_t s) {
  if (g.m % 8 == 0) return smoother_impl<4>(g, U, C, psi0, psi, ws, s);
  return smoother_impl<2>(g, U, C, psi0, psi, ws, s);
}

}  // namespace mg
