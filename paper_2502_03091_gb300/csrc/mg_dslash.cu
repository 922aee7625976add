// mg_dslash.cu -- Wilson(-clover) operator on many right-hand sides and the
// minimal-residual smoother of the setup (paper Sec. 2, Eq. 1: m' random
// starts relaxed on D psi = 0), plus the clover-field preparation.
//
// Smoother (per right-hand side, a = step length), the textbook MR order:
//   r_0 = -D psi_0,  w_0 = D r_0,  a_t = <w_t, r_t> / <w_t, w_t>
//   psi_{t+1} = psi_t + a_t r_t,  r_{t+1} = r_t - a_t w_t,  w_{t+1} = D r_{t+1},
// and finally psi_i / |psi_i|.  Each iteration is two passes: a streaming
// update of r and psi, then the dslash w = D r with the partial inner
// products of a_{t+1}.
//
// Internal "slab" layout of r, w and psi: the right-hand sides are cut into
// slabs of 2P (P pairs); element f[((q*V + x)*12 + e)*P + p] holds component
// e = spin*3 + colour of site x for the pair (2(qP+p), 2(qP+p)+1) as
// (re_0, re_1, im_0, im_1).  The real parts and the imaginary parts of a
// pair are packed FP32 pairs, the operands of the f32x2 instructions, and the
// 12 x 2P numbers of one site and slab are contiguous.  Elements are float4
// (FP32 storage, 768 bytes per site and slab for P = 4) or four halves in a
// uint2 (FP16 storage of the MG_PREC_MIXED_FP16 path, 384 bytes); arithmetic is
// FP32 in both.
#include <atomic>
#include <cstdint>

#include <cuda_fp16.h>

#include "mg_bulk.cuh"
#include "mg_common.cuh"

namespace mg {
namespace {

// device status word: bit 0 = a smoother pass gave up waiting for its staged
// input; bit 1 = a tensor-core Gram gave up waiting for its MMAs
__device__ int g_status;
// words taken from g_status by read_device_status, one slot per call
constexpr int kStatusSlots = 64;
__device__ int g_status_taken[kStatusSlots];
__global__ void status_take(int* slot) { *slot = atomicExch(&g_status, 0); }

// ---------------------------------------------------------------------------
// packed FP32 pairs: component .x belongs to the first right-hand side of a
// pair, .y to the second (the f32x2 instructions of sm_100 and later; the
// inline-PTX form measured faster here than the compiler's float2 builtins)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long pk(float2 a) {
  unsigned long long u;
  asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(a.x), "f"(a.y));
  return u;
}
__device__ __forceinline__ float2 upk(unsigned long long u) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(u));
  return a;
}
// a * b + c, lane-wise
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return upk(d);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// one complex component of two right-hand sides
struct CP {
  float2 re, im;
};
__device__ __forceinline__ float2 h2_to_f2(unsigned int u) {
  __half2 h;
  *reinterpret_cast<unsigned int*>(&h) = u;
  return __half22float2(h);
}
__device__ __forceinline__ unsigned int f2_to_h2(float2 f) {
  const __half2 h = __float22half2_rn(f);
  return *reinterpret_cast<const unsigned int*>(&h);
}
// storage element <-> two right-hand sides of one component
__device__ __forceinline__ CP cp_unpack(float4 v) {
  return CP{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ CP cp_unpack(uint2 v) { return CP{h2_to_f2(v.x), h2_to_f2(v.y)}; }
template <typename T>
__device__ __forceinline__ T cp_pack(CP a);
template <>
__device__ __forceinline__ float4 cp_pack<float4>(CP a) {
  return make_float4(a.re.x, a.re.y, a.im.x, a.im.y);
}
template <>
__device__ __forceinline__ uint2 cp_pack<uint2>(CP a) {
  return make_uint2(f2_to_h2(a.re), f2_to_h2(a.im));
}
template <typename T>
__device__ __forceinline__ CP cp_ld(const T* p) {
  return cp_unpack(*p);
}

__device__ __forceinline__ CP cp_neg(CP a) {
  return CP{make_float2(-a.re.x, -a.re.y), make_float2(-a.im.x, -a.im.y)};
}

// acc += u h for a link entry u shared by both right-hand sides; nim = -Im h
__device__ __forceinline__ void lmul(CP& acc, float2 u, const CP& h, float2 nim) {
  const float2 ur = dup(u.x), ui = dup(u.y);
  acc.re = pfma(ur, h.re, acc.re);
  acc.re = pfma(ui, nim, acc.re);
  acc.im = pfma(ur, h.im, acc.im);
  acc.im = pfma(ui, h.re, acc.im);
}
// acc += conj(u) h; nre = -Re h
__device__ __forceinline__ void lmulc(CP& acc, float2 u, const CP& h, float2 nre) {
  const float2 ur = dup(u.x), ui = dup(u.y);
  acc.re = pfma(ur, h.re, acc.re);
  acc.re = pfma(ui, h.im, acc.re);
  acc.im = pfma(ur, h.im, acc.im);
  acc.im = pfma(ui, nre, acc.im);
}

__device__ __forceinline__ long slab_index(int q, int V, int x, int e, int PAIRS, int p) {
  return (((long)q * V + x) * 12 + e) * PAIRS + p;
}

// ---------------------------------------------------------------------------
// one hop of the Wilson operator, spin-projected:
//   S = +1: acc += hw (1 - gamma_mu) U_mu(x) chi(x + mu)
//   S = -1: acc += hw (1 + gamma_mu) U_mu(x - mu)^dag chi(x - mu)
// With chi = (chi_u, chi_l) in the chiral basis, (1 - S gamma_mu) chi =
// (h, -S B_mu^dag h) with h = chi_u - S B_mu chi_l, so only the half spinor h
// (2 spins x 3 colours) is multiplied by the link.
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.
//
// The hop is split between two partner lanes (hf = 0, 1): lane hf forms row
// hf of h, multiplies it by the link and accumulates the output spins hf
// (upper: + hw g) and 2 + hf (lower: -S hw (B^dag g)_hf); for mu = x, y the
// lower part needs the partner's g (one shuffle).  src points at component 0
// of the neighbour's pair (component e at src[e * PAIRS], shared ring or
// global slab); u at the 9 entries of the link.
// ---------------------------------------------------------------------------
// the 9 entries of one link at u (u is 8-byte aligned; u16 says whether u
// itself is 16-byte aligned): four 16-byte loads and one 8-byte load.  u
// points into the shared-memory link ring or into global memory.
__device__ __forceinline__ void load_link(const float2* u, bool u16, float2 L[9]) {
  // the 16-byte aligned run of 8 entries starts at u or at u + 1
  const float4* a4 = reinterpret_cast<const float4*>(u16 ? u : u + 1);
  float4 v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = a4[i];
  const float2 last = u16 ? u[8] : u[0];
  if (u16) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      L[2 * i] = make_float2(v[i].x, v[i].y);
      L[2 * i + 1] = make_float2(v[i].z, v[i].w);
    }
    L[8] = last;
  } else {
    L[0] = last;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      L[2 * i + 1] = make_float2(v[i].x, v[i].y);
      L[2 * i + 2] = make_float2(v[i].z, v[i].w);
    }
  }
}

// The six storage elements lane hf reads for one hop: rows (spin hf, colour c)
// and (spin 2 + lo, colour c) of the neighbour, lo = 1 - hf for x, y and hf
// for z, t (B_mu mixes the lower spins that way).
template <int MU, int PAIRS, typename T>
__device__ __forceinline__ void hop_load(const T* src, int hf, T v[6]) {
  const int lo = (MU == 0 || MU == 1) ? 1 - hf : hf;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = src[(hf * 3 + c) * PAIRS];
    v[3 + c] = src[((2 + lo) * 3 + c) * PAIRS];
  }
}

template <int MU, int S, int PAIRS, typename T>
__device__ __forceinline__ void hop_v(CP zu[3], CP zl[3], int hf, const T v[6],
                                      const float2* u, float hw);

template <int MU, int S, int PAIRS, typename T>
__device__ __forceinline__ void hop(CP zu[3], CP zl[3], int hf, const T* src,
                                    const float2* u, float hw) {
  T v[6];
  hop_load<MU, PAIRS, T>(src, hf, v);
  hop_v<MU, S, PAIRS, T>(zu, zl, hf, v, u, hw);
}

template <int MU, int S, int PAIRS, typename T>
__device__ __forceinline__ void hop_v(CP zu[3], CP zl[3], int hf, const T v[6],
                                      const float2* u, float hw) {
  float2 L[9];
  load_link(u, (reinterpret_cast<uintptr_t>(u) & 15) == 0, L);
  CP h[3];
  float2 nh[3];
  {
    // h.re = up.re + cr A, h.im = up.im + ci B with (A, B) = (dn.im, dn.re) for
    // x, z and (dn.re, dn.im) for y, t:
    //   x: B chi_l = -i chi_{3-hf};  y: -chi_3 / +chi_2;  z: -i chi_2 / +i chi_3;  t: chi_{2+hf}
    float cr, ci;
    if (MU == 0) {
      cr = -S;
      ci = S;
    } else if (MU == 1) {
      const float s1 = hf ? 1.f : -1.f;
      cr = ci = -S * s1;
    } else if (MU == 2) {
      const float s2 = hf ? -1.f : 1.f;
      cr = -S * s2;
      ci = S * s2;
    } else {
      cr = ci = -S;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const CP up = cp_unpack(v[c]);
      const CP dn = cp_unpack(v[3 + c]);
      const float2 A = (MU == 0 || MU == 2) ? dn.im : dn.re;
      const float2 B = (MU == 0 || MU == 2) ? dn.re : dn.im;
      h[c].re = pfma(dup(cr), A, up.re);
      h[c].im = pfma(dup(ci), B, up.im);
      nh[c] = pmul(dup(-1.f), S > 0 ? h[c].im : h[c].re);
    }
  }
  // lower-spin coefficients: acc_l.re += kr X, acc_l.im += ki Y
  //   x: i g_{1-hf};  y: g_1 / -g_0;  z: i g_0 / -i g_1;  t: g_hf
  float kr, ki;
  if (MU == 0) {
    kr = S * hw;
    ki = -S * hw;
  } else if (MU == 1) {
    const float t1 = hf ? -1.f : 1.f;
    kr = ki = -S * hw * t1;
  } else if (MU == 2) {
    const float t2 = hf ? -1.f : 1.f;
    kr = S * hw * t2;
    ki = -S * hw * t2;
  } else {
    kr = ki = -S * hw;
  }
  if constexpr (sizeof(T) < 16) {
    // FP16 storage (128 registers): one colour at a time
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      CP g{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (S > 0) lmul(g, L[c * 3 + d], h[d], nh[d]);
        else lmulc(g, L[d * 3 + c], h[d], nh[d]);
      }
      zu[c].re = pfma(dup(hw), g.re, zu[c].re);
      zu[c].im = pfma(dup(hw), g.im, zu[c].im);
      if (MU == 0 || MU == 1) {
        g.re.x = __shfl_xor_sync(0xffffffffu, g.re.x, 1);
        g.re.y = __shfl_xor_sync(0xffffffffu, g.re.y, 1);
        g.im.x = __shfl_xor_sync(0xffffffffu, g.im.x, 1);
        g.im.y = __shfl_xor_sync(0xffffffffu, g.im.y, 1);
      }
      const float2 X = (MU == 0 || MU == 2) ? g.im : g.re;
      const float2 Y = (MU == 0 || MU == 2) ? g.re : g.im;
      zl[c].re = pfma(dup(kr), X, zl[c].re);
      zl[c].im = pfma(dup(ki), Y, zl[c].im);
    }
    return;
  }
  // FP32 storage: the three colours' link products first (six independent FMA
  // chains), then the accumulations and the partner exchange, so no shuffle
  // sits between the chains (1% faster here; it spills at 128 registers)
  CP g[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g[c] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (S > 0) lmul(g[c], L[c * 3 + d], h[d], nh[d]);
      else lmulc(g[c], L[d * 3 + c], h[d], nh[d]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    zu[c].re = pfma(dup(hw), g[c].re, zu[c].re);
    zu[c].im = pfma(dup(hw), g[c].im, zu[c].im);
  }
  if (MU == 0 || MU == 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      g[c].re.x = __shfl_xor_sync(0xffffffffu, g[c].re.x, 1);
      g[c].re.y = __shfl_xor_sync(0xffffffffu, g[c].re.y, 1);
      g[c].im.x = __shfl_xor_sync(0xffffffffu, g[c].im.x, 1);
      g[c].im.y = __shfl_xor_sync(0xffffffffu, g[c].im.y, 1);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 X = (MU == 0 || MU == 2) ? g[c].im : g[c].re;
    const float2 Y = (MU == 0 || MU == 2) ? g[c].re : g[c].im;
    zl[c].re = pfma(dup(kr), X, zl[c].re);
    zl[c].im = pfma(dup(ki), Y, zl[c].im);
  }
}

// acc += c v for a complex number c shared by both right-hand sides
__device__ __forceinline__ void cmul_acc(CP& acc, float2 c, const CP& v) {
  acc.re = pfma(dup(c.x), v.re, acc.re);
  acc.re = pfma(dup(-c.y), v.im, acc.re);
  acc.im = pfma(dup(c.x), v.im, acc.im);
  acc.im = pfma(dup(c.y), v.re, acc.im);
}

// ---------------------------------------------------------------------------
// t-marching dslash pass.
//
// One CTA owns a patch of kSPC consecutive sites of a timeslice (spatial
// lexicographic index p0 .. p0+kSPC-1) for one slab, and marches t = 0..Lt-1.
// A ring of kRing = 3 rows lives in shared memory.  Row r (time r mod Lt) is
// two bulk copies completing on the slot's mbarrier: the patch's contiguous
// slab row of the input (24.6 KB for P = 4 in FP32) and the patch's
// contiguous row of links U[r][p0 .. p0+kSPC-1][4][3][3] (9.2 KB).  Hops that
// stay in the patch (x, and y when a patch spans several x-rows) and both
// t-hops read their neighbour from the ring; every forward link, the
// backward t link (row t-1) and the backward links of in-patch hops come from
// the ring; the remaining neighbours and backward links are read from global
// memory (L2).
// Step t uses rows t-1, t and t+1.  It starts with the -t hop, the only read
// of row t-1; after one barrier thread 0 reuses that slot for row t+2, which
// then has the rest of step t to arrive.  Row r (-1 <= r <= Lt) uses slot
// (r+1) % 3 for the ((r+1)/3)-th time: phase parity ((r+1)/3) & 1.
//
// MODE_NEG_D: out = -D in.  MODE_D_DOT: out = D in, plus per-patch partial
// sums <out, in> and |out|^2 per right-hand side (per lane in FP32 over 8
// steps, reduced over the warp in FP32, accumulated in FP64 in shared memory).
// Lanes: threadIdx = (site * P + pair) * 2 + hf.
// ---------------------------------------------------------------------------
constexpr int kSPC = 32;
constexpr int kRing = 3;
constexpr int kLinkSite = 36;  // float2 per site in a link row

struct MarchArgs {
  const void* in;     // input s (slab, storage type of the pass)
  void* out;          // D s or -D s (slab)
  const float2* U;    // links [V][4][3][3]
  const float2* C;    // clover [V][2][6][6] or nullptr
  double* part;       // [m'][npatch][4]
  int* status;        // device status word
  int L[4];
  int Vs, V, np, npatch;
  float hw[4];
  float diag;
};

enum { MODE_NEG_D = 0, MODE_D_DOT = 1 };

template <int PAIRS>
constexpr int march_threads() {
  return 2 * kSPC * PAIRS;
}

template <int PAIRS, typename T>
constexpr size_t march_smem() {
  return sizeof(T) * (size_t)kRing * kSPC * 12 * PAIRS +
         sizeof(float2) * (size_t)kRing * kSPC * kLinkSite;
}

// FP32 storage: the y/z inputs of a step are loaded at its start (look-ahead,
// measured 18% faster), with one CTA of 256 threads per SM for the registers;
// FP16 storage (half the bytes per hop) measured faster without it, at two CTAs
template <typename T>
__host__ __device__ constexpr bool march_lookahead() {
  return sizeof(T) == 16;
}
template <int PAIRS, typename T>
__host__ __device__ constexpr int march_min_blocks() {
  return (march_lookahead<T>() && PAIRS >= 4) ? 1 : 2;
}

template <int PAIRS, int MODE, typename T>
__global__ void __launch_bounds__(march_threads<PAIRS>(), march_min_blocks<PAIRS, T>())
    march_kernel(MarchArgs a) {
  constexpr bool LA = march_lookahead<T>();
  constexpr int NC = 2 * kSPC * PAIRS;
  constexpr int SS = 12 * PAIRS;  // ring site stride (elements): a row is a copy of the slab row
  constexpr int NW = NC / 32;
  constexpr uint32_t kSiteBytes = 12 * PAIRS * sizeof(T);
  constexpr uint32_t kLinkBytes = kLinkSite * sizeof(float2);
  extern __shared__ __align__(128) unsigned char ring_raw[];
  T* ring = reinterpret_cast<T*>(ring_raw);  // [kRing][kSPC][SS]
  float2* lring = reinterpret_cast<float2*>(ring_raw + sizeof(T) * kRing * kSPC * SS);
  const T* in = static_cast<const T*>(a.in);
  T* out = static_cast<T*>(a.out);
  __shared__ __align__(8) unsigned long long bar[kRing];
  __shared__ double red[MODE == MODE_D_DOT ? NW : 1][PAIRS][6];  // FP64 partial sums per warp
  __shared__ int s_abort;
  const int q = blockIdx.x / a.npatch, patch = blockIdx.x % a.npatch;
  const int p0 = patch * kSPC;
  const int Lt = a.L[3];
  const int nvalid = min(kSPC, a.Vs - p0);
  const int hf = threadIdx.x & 1;
  const int sp_idx = threadIdx.x >> 1;
  const int s_loc = sp_idx / PAIRS, p = sp_idx % PAIRS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int xyz = p0 + s_loc;
  const bool valid = xyz < a.Vs;
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
  if (threadIdx.x == 0) {
    for (int i = 0; i < kRing; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  if (MODE == MODE_D_DOT)
    for (int i = threadIdx.x; i < NW * PAIRS * 6; i += blockDim.x) (&red[0][0][0])[i] = 0.0;
  __syncthreads();
  // thread 0: the two bulk copies of ring row r (the patch's sites are
  // contiguous in the slab and in the link array)
  auto issue = [&](int r) {
    const int slot = (r + 1) % kRing;
    const uint32_t bytes = (uint32_t)nvalid * kSiteBytes, lbytes = (uint32_t)nvalid * kLinkBytes;
    mbar_expect_tx(&bar[slot], bytes + lbytes);
    const int x = ((r + Lt) % Lt) * a.Vs + p0;
    bulk_g2s(ring + slot * kSPC * SS, in + slab_index(q, a.V, x, 0, PAIRS, 0), bytes, &bar[slot]);
    bulk_g2s(lring + slot * kSPC * kLinkSite, a.U + (long)x * kLinkSite, lbytes, &bar[slot]);
  };
  auto wait_row = [&](int r) -> bool {
    return mbar_wait(&bar[(r + 1) % kRing], (uint32_t)(((r + 1) / kRing) & 1));
  };
  auto give_up = [&]() {
    s_abort = 1;
    atomicOr(a.status, 1);
  };
  if (threadIdx.x == 0) {
    issue(-1);
    issue(0);
    issue(1);
  }
  // rows <= waited have all landed; last_issued is the newest row in flight
  int last_issued = 1, waited = -2;
  if (wait_row(-1)) {
    waited = -1;
    if (wait_row(0)) waited = 0;
  }
  if (waited < 0) give_up();

  float2 sre = make_float2(0.f, 0.f), sim = sre, snn = sre;
  // lanes of a site beyond the lattice compute on site p0 and discard it
  const int xyzc = valid ? xyz : p0;
  const int sl = xyzc - p0;
  // y and z neighbours come from global memory (L2).  With the look-ahead a
  // step issues the loads of its four y/z hops first and consumes them after
  // the hops whose inputs are in shared memory (-t, diagonal, x, +t), which
  // hide the L2 round trip.
  const int ny[4] = {valid ? nf[1] : p0, valid ? nb[1] : p0, valid ? nf[2] : p0,
                     valid ? nb[2] : p0};
  auto load_yz = [&](int t, T v[4][6]) {
    const long tV = (long)t * a.Vs;
    hop_load<1, PAIRS, T>(in + slab_index(q, a.V, tV + ny[0], 0, PAIRS, p), hf, v[0]);
    hop_load<1, PAIRS, T>(in + slab_index(q, a.V, tV + ny[1], 0, PAIRS, p), hf, v[1]);
    hop_load<2, PAIRS, T>(in + slab_index(q, a.V, tV + ny[2], 0, PAIRS, p), hf, v[2]);
    hop_load<2, PAIRS, T>(in + slab_index(q, a.V, tV + ny[3], 0, PAIRS, p), hf, v[3]);
  };
  for (int t = 0; t < Lt; ++t) {
    T cur[LA ? 4 : 1][6];
    if constexpr (LA) load_yz(t, cur);
    if (waited == t && wait_row(t + 1)) waited = t + 1;
    else give_up();
    const T* ring_t = ring + ((t + 1) % kRing) * kSPC * SS;
    const T* ring_f = ring + ((t + 2) % kRing) * kSPC * SS;
    const T* ring_b = ring + (t % kRing) * kSPC * SS;
    const float2* lk_t = lring + ((t + 1) % kRing) * kSPC * kLinkSite;  // links of time t
    const float2* lk_b = lring + (t % kRing) * kSPC * kLinkSite;        // links of time t-1
    CP zu[3], zl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) zu[c] = zl[c] = CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    // the -t hop first: the only read of row t-1, whose slot is refilled next
    hop<3, -1, PAIRS, T>(zu, zl, hf, ring_b + sl * SS + p, lk_b + sl * kLinkSite + 27, a.hw[3]);
    __syncthreads();
    if (s_abort) break;
    if (t + 2 <= Lt) {
      if (threadIdx.x == 0) issue(t + 2);
      last_issued = t + 2;
    }
    const int x = t * a.Vs + xyzc;
    const T* cen = ring_t + sl * SS + p;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const CP u = cp_ld(cen + (hf * 3 + c) * PAIRS), l = cp_ld(cen + ((2 + hf) * 3 + c) * PAIRS);
      zu[c].re = pfma(dup(a.diag), u.re, zu[c].re);
      zu[c].im = pfma(dup(a.diag), u.im, zu[c].im);
      zl[c].re = pfma(dup(a.diag), l.re, zl[c].re);
      zl[c].im = pfma(dup(a.diag), l.im, zl[c].im);
    }
    if (a.C) {
      // row (spin hf, colour c) of each chirality's 6x6 block
      const float2* cl = a.C + (long)x * 72;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          cmul_acc(zu[c], __ldg(cl + (hf * 3 + c) * 6 + j), cp_ld(cen + j * PAIRS));
          cmul_acc(zl[c], __ldg(cl + 36 + (hf * 3 + c) * 6 + j), cp_ld(cen + (6 + j) * PAIRS));
        }
    }
    const float2* Ux = lk_t + sl * kLinkSite;
    const long tV = (long)t * a.Vs;
    hop<3, +1, PAIRS, T>(zu, zl, hf, ring_f + sl * SS + p, Ux + 27, a.hw[3]);
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      // x neighbours: ring if inside the patch, else global (same component stride)
      const int b = valid ? nb[mu] : p0;
      const int lb = b - p0;
      const bool rb = lb >= 0 && lb < kSPC && b < a.Vs;
      const float2* ub = rb ? lk_t + lb * kLinkSite + mu * 9 : a.U + (tV + b) * 36 + mu * 9;
      if (mu == 0) {
        const int f = valid ? nf[0] : p0;
        const int lf = f - p0;
        const bool rf = lf >= 0 && lf < kSPC && f < a.Vs;
        const T* pf = rf ? ring_t + lf * SS + p : in + slab_index(q, a.V, tV + f, 0, PAIRS, p);
        const T* pb = rb ? ring_t + lb * SS + p : in + slab_index(q, a.V, tV + b, 0, PAIRS, p);
        hop<0, +1, PAIRS, T>(zu, zl, hf, pf, Ux, a.hw[0]);
        hop<0, -1, PAIRS, T>(zu, zl, hf, pb, ub, a.hw[0]);
      } else if constexpr (LA) {
        if (mu == 1) {
          hop_v<1, +1, PAIRS, T>(zu, zl, hf, cur[0], Ux + 9, a.hw[1]);
          hop_v<1, -1, PAIRS, T>(zu, zl, hf, cur[1], ub, a.hw[1]);
        } else {
          hop_v<2, +1, PAIRS, T>(zu, zl, hf, cur[2], Ux + 18, a.hw[2]);
          hop_v<2, -1, PAIRS, T>(zu, zl, hf, cur[3], ub, a.hw[2]);
        }
      } else {
        // without the look-ahead: ring if inside the patch, else global
        const int f = valid ? nf[mu] : p0;
        const int lf = f - p0;
        const bool rf = lf >= 0 && lf < kSPC && f < a.Vs;
        const T* pf = rf ? ring_t + lf * SS + p : in + slab_index(q, a.V, tV + f, 0, PAIRS, p);
        const T* pb = rb ? ring_t + lb * SS + p : in + slab_index(q, a.V, tV + b, 0, PAIRS, p);
        if (mu == 1) {
          hop<1, +1, PAIRS, T>(zu, zl, hf, pf, Ux + 9, a.hw[1]);
          hop<1, -1, PAIRS, T>(zu, zl, hf, pb, ub, a.hw[1]);
        } else {
          hop<2, +1, PAIRS, T>(zu, zl, hf, pf, Ux + 18, a.hw[2]);
          hop<2, -1, PAIRS, T>(zu, zl, hf, pb, ub, a.hw[2]);
        }
      }
    }
    if (valid) {
      const long so = slab_index(q, a.V, x, 0, PAIRS, p);
      if (MODE == MODE_NEG_D) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int e = k < 3 ? hf * 3 + k : (2 + hf) * 3 + k - 3;
          const CP w = k < 3 ? zu[k] : zl[k - 3];
          __stcs(out + so + e * PAIRS, cp_pack<T>(cp_neg(w)));
        }
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int e = k < 3 ? hf * 3 + k : (2 + hf) * 3 + k - 3;
          const CP w = k < 3 ? zu[k] : zl[k - 3];
          const CP r = cp_ld(cen + e * PAIRS);
          // <w, r> = sum conj(w) r
          sre = pfma(w.re, r.re, sre);
          sre = pfma(w.im, r.im, sre);
          sim = pfma(w.re, r.im, sim);
          sim = pfma(pmul(dup(-1.f), w.im), r.re, sim);
          snn = pfma(w.re, w.re, snn);
          snn = pfma(w.im, w.im, snn);
          __stcs(out + so + e * PAIRS, cp_pack<T>(w));
        }
      }
    }
    if (MODE == MODE_D_DOT && ((t & 7) == 7 || t == Lt - 1)) {
      // lane = 2 * (s * PAIRS + p) + hf: FP32 sum over hf and the warp's sites
      // (at most 8 lanes), per pair, then FP64 across steps and warps (FP64
      // issues at 1/64 of the FP32 rate here; the short FP32 sums cost a few ulp)
      float pr[6] = {sre.x, sim.x, snn.x, sre.y, sim.y, snn.y};
#pragma unroll
      for (int i = 0; i < 6; ++i) pr[i] += __shfl_xor_sync(0xffffffffu, pr[i], 1);
#pragma unroll
      for (int off = 16; off >= 2 * PAIRS; off >>= 1)
#pragma unroll
        for (int i = 0; i < 6; ++i) pr[i] += __shfl_xor_sync(0xffffffffu, pr[i], off);
      if (lane < 2 * PAIRS && (lane & 1) == 0)
#pragma unroll
        for (int i = 0; i < 6; ++i) red[warp][lane >> 1][i] += (double)pr[i];
      sre = sim = snn = make_float2(0.f, 0.f);
    }
  }
  if (s_abort) {
    // let the copies still in flight land before the CTA's shared memory is released
    for (int r = waited + 1; r <= last_issued; ++r) (void)wait_row(r);
    return;
  }
  if (MODE != MODE_NEG_D) {
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

// ---------------------------------------------------------------------------
// streaming kernels over the slab layout
// ---------------------------------------------------------------------------
// decomposes a slab float4 index into (slab q, site x, component e, pair p)
template <int PAIRS>
__device__ __forceinline__ void slab_coords(long i, int V, int& q, int& x, int& e, int& p) {
  p = (int)(i % PAIRS);
  long r = i / PAIRS;
  e = (int)(r % 12);
  r /= 12;
  x = (int)(r % V);
  q = (int)(r / V);
}

// Partial sums of |psi_0|^2 per right-hand side over the ABI layout
// [V][12][m'] (FP16-storage path: psi_0 is scaled to unit RMS per vector
// before it is stored in FP16).  CTA g covers sites [g*cs, (g+1)*cs); the
// block has np * (256 / np) threads, so every thread keeps one pair.
__global__ void __launch_bounds__(256) abi_norm_partials(const float4* __restrict__ src,
                                                         double* __restrict__ part, int V, int np,
                                                         int cs, int nchunk) {
  __shared__ float red[256][2];
  const int g = blockIdx.x;
  const long x0 = (long)g * cs, x1 = min((long)V, x0 + cs);
  const long i0 = x0 * 12 * np, i1 = x1 * 12 * np;
  float s0 = 0.f, s1 = 0.f;
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float4 v = __ldcs(src + i);
    s0 += v.x * v.x + v.y * v.y;
    s1 += v.z * v.z + v.w * v.w;
  }
  red[threadIdx.x][0] = s0;
  red[threadIdx.x][1] = s1;
  __syncthreads();
  // fixed summation order (deterministic): thread p adds threads p, p + np, ...
  if ((int)threadIdx.x < np) {
    double t0 = 0, t1 = 0;
    for (int j = threadIdx.x; j < (int)blockDim.x; j += np) {
      t0 += (double)red[j][0];
      t1 += (double)red[j][1];
    }
    double* q0 = part + ((long)(2 * threadIdx.x) * nchunk + g) * 4;
    double* q1 = part + ((long)(2 * threadIdx.x + 1) * nchunk + g) * 4;
    q0[0] = 0; q0[1] = 0; q0[2] = t0;
    q1[0] = 0; q1[1] = 0; q1[2] = t1;
  }
}

// Layout conversions between the ABI layout [V][12][m'] (complex) and the slab
// layout.  A CTA moves tiles of kTrSites consecutive sites: in the ABI layout
// a tile is one contiguous region, in slab q a contiguous run of
// kTrSites * 12 * PAIRS elements, so both sides are read and written in long
// coalesced runs, with the transpose in shared memory (rows of the tile hold
// the np pairs of one (site, component) at a pitch of np + PAIRS elements, so
// the 16-byte reads of consecutive rows fall on different bank groups).
constexpr int kTrSites = 4;
constexpr int kTrThreads = 256;
constexpr int kTrBlocksPerSm = 8;

inline size_t tr_smem(int np, int pairs) {  // at most 27.6 KB (np <= 32)
  return sizeof(float4) * (size_t)kTrSites * 12 * (np + pairs);
}
// kTrBlocksPerSm CTAs per SM, each walking its tiles
inline int tr_grid() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 152;
  return n * kTrBlocksPerSm;
}

// psi_0 (ABI layout) -> slab layout, each vector times mul * scale[i]
// (scale == nullptr: no scaling)
template <int PAIRS, typename T>
__global__ void __launch_bounds__(kTrThreads) to_slab(const float4* __restrict__ src,
                                                      T* __restrict__ dst,
                                                      const float* __restrict__ scale, float mul,
                                                      int V, int np) {
  extern __shared__ float4 tr_tile[];  // [kTrSites * 12][np + PAIRS]
  const int pitch = np + PAIRS, nsl = np / PAIRS;
  for (int x0 = blockIdx.x * kTrSites; x0 < V; x0 += gridDim.x * kTrSites) {
    const int nrow = min(kTrSites, V - x0) * 12, run = nrow * PAIRS;
    const float4* s0 = src + (long)x0 * 12 * np;
    for (int i = threadIdx.x; i < nrow * np; i += kTrThreads) {
      const int row = i / np;
      tr_tile[row * pitch + (i - row * np)] = __ldcs(s0 + i);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nsl * run; i += kTrThreads) {
      const int q = i / run, k = i - q * run;  // k = (site * 12 + e) * PAIRS + p
      const int row = k / PAIRS, gp = q * PAIRS + (k - row * PAIRS);
      const float4 v = tr_tile[row * pitch + gp];
      const float a0 = scale ? mul * scale[2 * gp] : 1.f, a1 = scale ? mul * scale[2 * gp + 1] : 1.f;
      __stcs(dst + slab_index(q, V, x0, 0, PAIRS, 0) + k,
             cp_pack<T>(CP{make_float2(v.x * a0, v.z * a1), make_float2(v.y * a0, v.w * a1)}));
    }
    __syncthreads();
  }
}

// MR update between two dslash passes, with psi's update deferred by one
// iteration (paper Eq. 1; the terms are the same, the psi field is read and
// written every other iteration):
//   odd t:  r_t = r_{t-1} - a_{t-1} w_{t-1}                  (r_t into the other r buffer)
//   even t: psi += a_{t-2} r_{t-2}, then psi += a_{t-1} r_{t-1}, and r_t as above,
//           written over r_{t-2} after it is read.
// One element (a pair of right-hand sides) per thread.  The two psi terms are
// added in the order and with the operations of one update per iteration.
__device__ __forceinline__ void pair_alpha(const float2* alpha, int gp, float2& ar, float2& ai) {
  const float2 a0 = alpha[2 * gp], a1 = alpha[2 * gp + 1];
  ar = make_float2(a0.x, a1.x);
  ai = make_float2(a0.y, a1.y);
}
// r - a w per right-hand side (ar, ai = Re a, Im a of the pair)
__device__ __forceinline__ CP mr_r_next(const CP& rv, const CP& wv, float2 ar, float2 ai) {
  CP rn;
  rn.re = make_float2(rv.re.x - (ar.x * wv.re.x - ai.x * wv.im.x),
                      rv.re.y - (ar.y * wv.re.y - ai.y * wv.im.y));
  rn.im = make_float2(rv.im.x - (ar.x * wv.im.x + ai.x * wv.re.x),
                      rv.im.y - (ar.y * wv.im.y + ai.y * wv.re.y));
  return rn;
}
// psi + a r per right-hand side
__device__ __forceinline__ CP mr_psi_next(const CP& pv, const CP& rv, float2 ar, float2 ai) {
  CP pn;
  pn.re = make_float2(pv.re.x + (ar.x * rv.re.x - ai.x * rv.im.x),
                      pv.re.y + (ar.y * rv.re.y - ai.y * rv.im.y));
  pn.im = make_float2(pv.im.x + (ar.x * rv.im.x + ai.x * rv.re.x),
                      pv.im.y + (ar.y * rv.im.y + ai.y * rv.re.y));
  return pn;
}

template <int PAIRS, typename T>
__global__ void mr_update_r(const T* __restrict__ r, const T* __restrict__ w, T* __restrict__ rn,
                            const float2* __restrict__ alpha, int V, int np) {
  const long n = (long)V * 12 * np;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    int q, x, e, p;
    slab_coords<PAIRS>(i, V, q, x, e, p);
    float2 ar, ai;
    pair_alpha(alpha, q * PAIRS + p, ar, ai);
    __stcs(rn + i, cp_pack<T>(mr_r_next(cp_unpack(__ldcs(r + i)), cp_unpack(__ldcs(w + i)), ar, ai)));
  }
}

template <int PAIRS, typename T>
__global__ void mr_update_rpsi(const T* __restrict__ r1, const T* __restrict__ w,
                               T* __restrict__ r2, T* __restrict__ psi,
                               const float2* __restrict__ alpha1, const float2* __restrict__ alpha2,
                               int V, int np) {
  const long n = (long)V * 12 * np;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    int q, x, e, p;
    slab_coords<PAIRS>(i, V, q, x, e, p);
    float2 ar1, ai1, ar2, ai2;
    pair_alpha(alpha1, q * PAIRS + p, ar1, ai1);
    pair_alpha(alpha2, q * PAIRS + p, ar2, ai2);
    const CP rv1 = cp_unpack(__ldcs(r1 + i)), rv2 = cp_unpack(__ldcs(r2 + i));
    const CP pv = mr_psi_next(mr_psi_next(cp_unpack(__ldcs(psi + i)), rv2, ar2, ai2), rv1, ar1, ai1);
    __stcs(psi + i, cp_pack<T>(pv));
    __stcs(r2 + i, cp_pack<T>(mr_r_next(rv1, cp_unpack(__ldcs(w + i)), ar1, ai1)));
  }
}

// psi_N = psi_{N-1} + a r_{N-1} in place, partial |psi_N|^2 per right-hand side.
// Streaming: CTA (slab q, chunk g) covers the contiguous sites
// [g*cs, (g+1)*cs) of slab q; thread i handles elements i, i + 256, ... of that
// range, all of one pair (256 is a multiple of P).  Partials go to
// part[(rhs * nchunk + g) * 4 + 2].
template <int PAIRS, typename T>
__global__ void __launch_bounds__(256) last_update(const T* __restrict__ r, T* __restrict__ psi,
                                                   const float2* __restrict__ alpha,
                                                   const T* __restrict__ r_old,
                                                   const float2* __restrict__ alpha_old,
                                                   double* __restrict__ part, int V, int cs,
                                                   int nchunk) {
  constexpr int NW = 256 / 32;
  __shared__ double red[NW][PAIRS][2];
  const int q = blockIdx.x / nchunk, g = blockIdx.x % nchunk;
  const int p = threadIdx.x % PAIRS;
  float2 ar, ai, aro = make_float2(0.f, 0.f), aio = aro;
  pair_alpha(alpha, q * PAIRS + p, ar, ai);
  if (r_old) pair_alpha(alpha_old, q * PAIRS + p, aro, aio);
  const long x0 = (long)g * cs, x1 = min((long)V, x0 + cs);
  const long i0 = slab_index(q, V, (int)x0, 0, PAIRS, 0), i1 = slab_index(q, V, (int)x1, 0, PAIRS, 0);
  float s0 = 0.f, s1 = 0.f;
  for (long i = i0 + threadIdx.x; i < i1; i += 256) {
    CP pn = cp_unpack(__ldcs(psi + i));
    if (r_old) pn = mr_psi_next(pn, cp_unpack(__ldcs(r_old + i)), aro, aio);  // pending term
    pn = mr_psi_next(pn, cp_unpack(__ldcs(r + i)), ar, ai);
    s0 += pn.re.x * pn.re.x + pn.im.x * pn.im.x;
    s1 += pn.re.y * pn.re.y + pn.im.y * pn.im.y;
    __stcs(psi + i, cp_pack<T>(pn));
  }
  double n0 = s0, n1 = s1;
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
    double* q0 = part + ((long)rhs0 * nchunk + g) * 4;
    double* q1 = part + ((long)(rhs0 + 1) * nchunk + g) * 4;
    q0[0] = 0; q0[1] = 0; q0[2] = t0;
    q1[0] = 0; q1[1] = 0; q1[2] = t1;
  }
}

// Second stage of the inner products, in a fixed order (deterministic):
//   mode 0: a_i = <w,r>_i / <w,w>_i,   mode 1: scale_i = 1 / |psi_i|.
// One CTA of kRedThreads per right-hand side: thread j sums partials j,
// j + kRedThreads, ... and a fixed tree combines the threads (deterministic).
constexpr int kRedThreads = 128;
__global__ void __launch_bounds__(kRedThreads) finish_reduction(const double* __restrict__ part,
                                                                int G, int m, int mode,
                                                                float2* __restrict__ alpha,
                                                                float* __restrict__ scale) {
  __shared__ double sred[3][kRedThreads];
  const int i = blockIdx.x;
  double re = 0, im = 0, nn = 0;
  for (int g = threadIdx.x; g < G; g += kRedThreads) {
    const double* pp = part + ((long)i * G + g) * 4;
    re += pp[0];
    im += pp[1];
    nn += pp[2];
  }
  sred[0][threadIdx.x] = re;
  sred[1][threadIdx.x] = im;
  sred[2][threadIdx.x] = nn;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int c = 0; c < 3; ++c) sred[c][threadIdx.x] += sred[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    re = sred[0][0];
    im = sred[1][0];
    nn = sred[2][0];
    if (mode == 0)
      alpha[i] = nn > 0 ? make_float2((float)(re / nn), (float)(im / nn)) : make_float2(0.f, 0.f);
    else
      scale[i] = nn > 0 ? (float)(1.0 / sqrt(nn)) : 1.0f;
  }
}

__global__ void fill_kernel(float* __restrict__ v, int n, float x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = x;
}

// psi (ABI layout) = scale * psi_slab, tile by tile as in to_slab
template <int PAIRS, typename T>
__global__ void __launch_bounds__(kTrThreads) scale_to_abi(const T* __restrict__ src,
                                                           float4* __restrict__ dst,
                                                           const float* __restrict__ scale,
                                                           int V, int np) {
  extern __shared__ float4 tr_tile[];  // [kTrSites * 12][np + PAIRS]
  const int pitch = np + PAIRS, nsl = np / PAIRS;
  for (int x0 = blockIdx.x * kTrSites; x0 < V; x0 += gridDim.x * kTrSites) {
    const int nrow = min(kTrSites, V - x0) * 12, run = nrow * PAIRS;
    for (int i = threadIdx.x; i < nsl * run; i += kTrThreads) {
      const int q = i / run, k = i - q * run;
      const int row = k / PAIRS, gp = q * PAIRS + (k - row * PAIRS);
      const CP v = cp_unpack(__ldcs(src + slab_index(q, V, x0, 0, PAIRS, 0) + k));
      const float a0 = scale[2 * gp], a1 = scale[2 * gp + 1];
      tr_tile[row * pitch + gp] = make_float4(v.re.x * a0, v.im.x * a0, v.re.y * a1, v.im.y * a1);
    }
    __syncthreads();
    float4* d0 = dst + (long)x0 * 12 * np;
    for (int i = threadIdx.x; i < nrow * np; i += kTrThreads) {
      const int row = i / np;
      __stcs(d0 + i, tr_tile[row * pitch + (i - row * np)]);
    }
    __syncthreads();
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

template <int PAIRS, int MODE, typename T>
cudaError_t run_march(const MarchArgs& a, int nsl, cudaStream_t s) {
  static const char* names[2] = {"mr_neg_dslash", "mr_dslash_dot"};
  const size_t smem = march_smem<PAIRS, T>();
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(march_kernel<PAIRS, MODE, T>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  TimedScope ts(names[MODE], s);
  march_kernel<PAIRS, MODE, T><<<nsl * a.npatch, march_threads<PAIRS>(), smem, s>>>(a);
  return cudaGetLastError();
}


// common part of the smoother and the operator apply: the slab copy of the
// input (into ps; in FP16 storage each vector is first scaled to unit RMS,
// which neither the normalised smoother output nor the linear operator
// notices once the scale is undone) and the march arguments
template <int PAIRS, typename T>
cudaError_t march_setup(const Geom& g, const float2* U, const float2* C, const float2* in,
                        char* ws, MarchArgs& a, bool unit_rms, cudaStream_t s) {
  const SmoothWs lay = smooth_ws_layout(g);
  T* ps = reinterpret_cast<T*>(ws + lay.ps);
  a = MarchArgs{};
  a.U = U;
  a.C = C;
  a.part = reinterpret_cast<double*>(ws + lay.part);
  a.status = device_status_word();
  if (!a.status) return cudaErrorInvalidSymbol;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.L[i];
    a.hw[i] = g.hw[i];
  }
  a.V = (int)g.V;
  a.Vs = (int)(g.V / g.L[3]);
  a.np = g.m / 2;
  a.npatch = (a.Vs + kSPC - 1) / kSPC;
  a.diag = g.diag;
  const float* scl = nullptr;
  float mul = 1.f;
  if (unit_rms) {
    float2* alpha = reinterpret_cast<float2*>(ws + lay.alpha);
    float* scale = reinterpret_cast<float*>(ws + lay.scale);
    const int G = a.npatch, cs = (a.V + G - 1) / G;
    TimedScope ts("mr_input_norm", s);
    abi_norm_partials<<<G, a.np * (256 / a.np), 0, s>>>(reinterpret_cast<const float4*>(in),
                                                       a.part, a.V, a.np, cs, G);
    finish_reduction<<<g.m, kRedThreads, 0, s>>>(a.part, G, g.m, 1, alpha, scale);
    scl = scale;
    mul = (float)sqrt(12.0 * (double)g.V);
  }
  {
    TimedScope ts("mr_to_slab", s);
    to_slab<PAIRS, T><<<tr_grid(), kTrThreads, tr_smem(a.np, PAIRS), s>>>(
        reinterpret_cast<const float4*>(in), ps, scl, mul, a.V, a.np);
  }
  return cudaGetLastError();
}

template <int PAIRS, typename T>
cudaError_t smoother_impl(const Geom& g, const float2* U, const float2* C, const float2* psi0,
                          float2* psi, char* ws, cudaStream_t s) {
  const SmoothWs lay = smooth_ws_layout(g);
  T* r = reinterpret_cast<T*>(ws + lay.ra);
  T* w = reinterpret_cast<T*>(ws + lay.wa);
  T* ps = reinterpret_cast<T*>(ws + lay.ps);
  double* part = reinterpret_cast<double*>(ws + lay.part);
  float2* alpha = reinterpret_cast<float2*>(ws + lay.alpha);
  float* scale = reinterpret_cast<float*>(ws + lay.scale);
  MarchArgs a;
  // MR is invariant under a per-vector scale of psi_0 and the output is
  // normalised, so the FP16 path may start from unit-RMS vectors
  cudaError_t e = march_setup<PAIRS, T>(g, U, C, psi0, ws, a, sizeof(T) < sizeof(float4), s);
  if (e != cudaSuccess) return e;
  const int nsl = a.np / PAIRS;
  const int G = a.npatch;  // partial sums per right-hand side
  auto reduce = [&](int mode) {
    TimedScope ts("mr_reduce", s);
    finish_reduction<<<g.m, kRedThreads, 0, s>>>(part, G, g.m, mode, alpha, scale);
  };

  // r_0 = -D psi_0
  a.in = ps;
  a.out = r;
  if ((e = run_march<PAIRS, MODE_NEG_D, T>(a, nsl, s)) != cudaSuccess) return e;
  // w_0 = D r_0 -> a_0
  a.in = r;
  a.out = w;
  if ((e = run_march<PAIRS, MODE_D_DOT, T>(a, nsl, s)) != cudaSuccess) return e;
  reduce(0);
  // r_t alternates between two buffers and a_t between two arrays: psi's update
  // waits one iteration and takes two terms (see mr_update_rpsi)
  T* rbuf[2] = {r, reinterpret_cast<T*>(ws + lay.rb)};
  float2* abuf[2] = {alpha, reinterpret_cast<float2*>(ws + lay.alpha_b)};
  for (int t = 1; t < g.niter; ++t) {
    {
      TimedScope ts("mr_update", s);
      if (t & 1)
        mr_update_r<PAIRS, T><<<4096, 256, 0, s>>>(rbuf[(t - 1) & 1], w, rbuf[t & 1],
                                                   abuf[(t - 1) & 1], a.V, a.np);
      else
        mr_update_rpsi<PAIRS, T><<<4096, 256, 0, s>>>(rbuf[(t - 1) & 1], w, rbuf[t & 1], ps,
                                                      abuf[(t - 1) & 1], abuf[t & 1], a.V, a.np);
    }
    // w_t = D r_t -> a_t
    a.in = rbuf[t & 1];
    if ((e = run_march<PAIRS, MODE_D_DOT, T>(a, nsl, s)) != cudaSuccess) return e;
    {
      TimedScope ts("mr_reduce", s);
      finish_reduction<<<g.m, kRedThreads, 0, s>>>(part, G, g.m, 0, abuf[t & 1], scale);
    }
  }
  // psi_N = psi_{N-1} + a_{N-1} r_{N-1} (and the pending a_{N-2} r_{N-2} when N
  // is even); |psi_N|^2 partials over npatch chunks of the slab (the
  // partial-sum array holds npatch entries per right-hand side)
  {
    const int N = g.niter;
    const int cs = (a.V + G - 1) / G;
    const bool pend = N >= 2 && (N & 1) == 0;
    TimedScope ts("mr_last_update", s);
    last_update<PAIRS, T><<<nsl * G, 256, 0, s>>>(
        rbuf[(N - 1) & 1], ps, abuf[(N - 1) & 1], pend ? rbuf[(N - 2) & 1] : nullptr,
        pend ? abuf[(N - 2) & 1] : nullptr, part, a.V, cs, G);
  }
  reduce(1);
  {
    TimedScope ts("mr_scale", s);
    scale_to_abi<PAIRS, T><<<tr_grid(), kTrThreads, tr_smem(a.np, PAIRS), s>>>(
        ps, reinterpret_cast<float4*>(psi), scale, a.V, a.np);
  }
  return cudaGetLastError();
}

// out = D in: the input is copied to the slab as it is (no scaling, so FP16
// storage needs |in| within the FP16 range)
template <int PAIRS, typename T>
cudaError_t dirac_impl(const Geom& g, const float2* U, const float2* C, const float2* in,
                       float2* out, char* ws, cudaStream_t s) {
  const SmoothWs lay = smooth_ws_layout(g);
  T* r = reinterpret_cast<T*>(ws + lay.ra);
  T* ps = reinterpret_cast<T*>(ws + lay.ps);
  float* scale = reinterpret_cast<float*>(ws + lay.scale);
  MarchArgs a;
  cudaError_t e = march_setup<PAIRS, T>(g, U, C, in, ws, a, false, s);
  if (e != cudaSuccess) return e;
  a.in = ps;
  a.out = r;
  if ((e = run_march<PAIRS, MODE_NEG_D, T>(a, a.np / PAIRS, s)) != cudaSuccess) return e;
  {
    TimedScope ts("fill", s);
    fill_kernel<<<1, 64, 0, s>>>(scale, g.m, -1.0f);
  }
  TimedScope ts("mr_scale", s);
  scale_to_abi<PAIRS, T><<<tr_grid(), kTrThreads, tr_smem(a.np, PAIRS), s>>>(
      r, reinterpret_cast<float4*>(out), scale, a.V, a.np);
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

// slab width: 4 pairs of right-hand sides per CTA when m' allows it, unless a
// batch tuned this shape to 2
static bool wide_slab(const Geom& g) { return g.m % 8 == 0 && tuned_pairs(g) != 2; }

cudaError_t launch_dirac(const Geom& g, const float2* U, const float2* C, const float2* in,
                         float2* out, char* ws, cudaStream_t s) {
  if (g.prec == MG_PREC_MIXED_FP16) {
    if (wide_slab(g)) return dirac_impl<4, uint2>(g, U, C, in, out, ws, s);
    return dirac_impl<2, uint2>(g, U, C, in, out, ws, s);
  }
  if (wide_slab(g)) return dirac_impl<4, float4>(g, U, C, in, out, ws, s);
  return dirac_impl<2, float4>(g, U, C, in, out, ws, s);
}

cudaError_t launch_smoother(const Geom& g, const float2* U, const float2* C,
                            const float2* psi0, float2* psi, char* ws, cudaStream_t s) {
  if (g.prec == MG_PREC_MIXED_FP16) {
    if (wide_slab(g)) return smoother_impl<4, uint2>(g, U, C, psi0, psi, ws, s);
    return smoother_impl<2, uint2>(g, U, C, psi0, psi, ws, s);
  }
  if (wide_slab(g)) return smoother_impl<4, float4>(g, U, C, psi0, psi, ws, s);
  return smoother_impl<2, float4>(g, U, C, psi0, psi, ws, s);
}

// failure-detection self-test: a bounded wait on an mbarrier nothing arrives at
__global__ void selftest_timeout_kernel(int polls, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  bool ok = false;
  for (int i = 0; i < polls && !ok; ++i) ok = mbar_try_wait(&bar, 0);
  if (!ok) atomicOr(status, 1);
}

cudaError_t launch_selftest_timeout(int polls, cudaStream_t s) {
  int* st = device_status_word();
  if (!st) return cudaErrorInvalidSymbol;
  selftest_timeout_kernel<<<1, 32, 0, s>>>(polls, st);
  return cudaGetLastError();
}

int* device_status_word() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
  return static_cast<int*>(p);
}

cudaError_t read_device_status(int* out, cudaStream_t s) {
  // take and clear the word in one atomic step on the stream, into a slot of
  // its own per call, so that a bit set by another stream between the read
  // and the clear is never lost (it stays for the next call)
  static std::atomic<unsigned> next_slot{0};
  int* taken = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&taken), g_status_taken);
  if (e != cudaSuccess) return e;
  int* slot = taken + next_slot.fetch_add(1u) % kStatusSlots;
  status_take<<<1, 1, 0, s>>>(slot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int v = 0;
  if ((e = cudaMemcpyAsync(&v, slot, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *out = v;
  return cudaSuccess;
}

}  // namespace mg
