// mg_coarsen.cu -- prolongator (paper Sec. 3, Eq. 5), Galerkin coarse
// operator D_c = R D P with R = P^dagger (Sec. 2, Eq. 3), and the coarse
// operator apply.
//
// Coarsening uses the spin projection of the Wilson hop: with the chiral
// prolongator P(x) = diag(P_0(x), P_1(x)) (12 x 2k, chirality-sparse),
//   P(x)^dag (1 - gamma_mu) U P(y) = Pi_mu(x)^dag (1_2 x U) Pi_mu(y),
//   Pi_mu = [P_0 , -B_mu P_1]   (6 x 2k: 2 spins x 3 colours),
// so each hop is a depth-6 contraction.  Hops that stay inside a block add to
// X; hops through the +mu face give Y_{+mu}; the backward hops follow from
// gamma_5-hermiticity: X gets S + sigma_3 S^dag sigma_3 and
// Y_{-mu}(xc + mu) = sigma_3 Y_{+mu}(xc)^dag sigma_3.
#include "mg_common.cuh"

namespace mg {
namespace {


// P[x][alpha][e][i] = U_k[j(x)][alpha][loc(x)][e][i], e < rps (rows per site and
// chirality: 6 at the fine level, k1 at the second)
__global__ void prolongator_kernel(const float2* __restrict__ Uk, float2* __restrict__ P, int L0,
                                   int L1, int L2, int L3, int b0, int b1, int b2, int b3,
                                   int k, int rps) {
  // one warp per (site, chirality): its row of rps * k complex numbers is
  // contiguous in both layouts (16-byte copies when the count is even)
  const long V = (long)L0 * L1 * L2 * L3;
  const int nb = b0 * b1 * b2 * b3;
  const int row = rps * k;  // complex per (site, chirality)
  const int nf4 = row / 2;
  const int lane = threadIdx.x & 31;
  const long nw = (long)gridDim.x * (blockDim.x >> 5);
  const int Lc0 = L0 / b0, Lc1 = L1 / b1, Lc2 = L2 / b2;
  for (long wr = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); wr < 2 * V; wr += nw) {
    const long x = wr >> 1;
    const int al = (int)(wr & 1);
    int t = (int)x;
    const int x0 = t % L0; t /= L0;
    const int x1 = t % L1; t /= L1;
    const int x2 = t % L2; const int x3 = t / L2;
    const int j = x0 / b0 + Lc0 * (x1 / b1 + Lc1 * (x2 / b2 + Lc2 * (x3 / b3)));
    const int loc = x0 % b0 + b0 * (x1 % b1 + b1 * (x2 % b2 + b2 * (x3 % b3)));
    const float2* src = Uk + (((long)j * 2 + al) * nb + loc) * row;
    float2* dst = P + wr * row;
    if ((row & 1) == 0) {
      for (int f = lane; f < nf4; f += 32)
        __stcs(reinterpret_cast<float4*>(dst) + f, __ldcs(reinterpret_cast<const float4*>(src) + f));
    } else {
      for (int f = lane; f < row; f += 32) dst[f] = src[f];
    }
  }
}

struct CoarsenArgs {
  const float2* U;
  const float2* C;
  const float2* P;
  float2* X;
  float2* Y;
  int L[4], b[4], Lc[4];
  int nb, k;
  float hw[4];
  float diag;
};

__device__ __forceinline__ int site_of(const CoarsenArgs& a, int j, int loc, int xo[4]) {
  int t = j;
  const int j0 = t % a.Lc[0]; t /= a.Lc[0];
  const int j1 = t % a.Lc[1]; t /= a.Lc[1];
  const int j2 = t % a.Lc[2]; const int j3 = t / a.Lc[2];
  t = loc;
  const int l0 = t % a.b[0]; t /= a.b[0];
  const int l1 = t % a.b[1]; t /= a.b[1];
  const int l2 = t % a.b[2]; const int l3 = t / a.b[2];
  xo[0] = j0 * a.b[0] + l0;
  xo[1] = j1 * a.b[1] + l1;
  xo[2] = j2 * a.b[2] + l2;
  xo[3] = j3 * a.b[3] + l3;
  return xo[0] + a.L[0] * (xo[1] + a.L[1] * (xo[2] + a.L[2] * xo[3]));
}

// Coarsening as register-tiled complex GEMMs.  One CTA (16 x 16 threads) per
// block j.  Thread (ti, tj) owns the T x T output entries
// (a*16 + ti, b*16 + tj), a, b < T, of every 2k x 2k matrix (2k <= 16 T).
// For each pass the block's sites are processed in chunks of kChunk sites; the
// chunk's depth-6 left factor L (6 x 2k per site) and right factor R go to
// shared memory, then every thread accumulates conj(L)^T R into its tile:
//   passes 0, 1 (chirality alpha): L = P_alpha(x), R = 1/2 (m0 + sum w + C_alpha(x)) P_alpha(x)
//     (columns of the other chirality are zero);
//   passes 2..5 (mu = 0..3):       L = Pi_mu(x), R = hw_mu U_mu(x) Pi_mu(x + mu),
//     added to the interior sum S or, for sites on the block's +mu face, to Y_{+mu}.
// At the end X = S + sigma_3 S^dag sigma_3 (the 1/2 on the diagonal term makes
// its two halves add up), and Y_{-mu}(j + mu) = sigma_3 Y_{+mu}(j)^dag sigma_3.
constexpr int kChunk = 16;

// Each row sp of B_mu has a single non-zero B_mu[sp][t]; Pi_mu uses -B_mu, so
// the lower-chirality columns of Pi_mu(z) are g * P_1(z)[t] with g = -B_mu[sp][t].
__device__ __forceinline__ void pi_entry(int mu, int sp, int& t, float2& g) {
  if (mu == 0) { t = 1 - sp; g = make_float2(0.f, 1.f); }                          // -(-i)
  else if (mu == 1) { t = 1 - sp; g = make_float2(sp == 0 ? 1.f : -1.f, 0.f); }    // -(-1), -(+1)
  else if (mu == 2) { t = sp; g = make_float2(0.f, sp == 0 ? 1.f : -1.f); }        // -(-i), -(+i)
  else { t = sp; g = make_float2(-1.f, 0.f); }
}

template <int T>
__global__ void __launch_bounds__(256, 2) coarsen_kernel(CoarsenArgs a) {
  constexpr int NP = 16 * T;  // padded 2k
  extern __shared__ float2 sm[];
  float2* Lf = sm;                        // [kChunk][6][NP]
  float2* Rf = Lf + kChunk * 6 * NP;      // [kChunk][6][NP]
  float2* Tr = Rf + kChunk * 6 * NP;      // [NP][NP + 1] transpose scratch
  __shared__ int s_face[kChunk], s_site[kChunk], s_nbr[kChunk];
  const int k = a.k, n2 = 2 * k;
  const int j = blockIdx.x;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  float2 S[T][T];
#pragma unroll
  for (int p = 0; p < T; ++p)
#pragma unroll
    for (int q = 0; q < T; ++q) S[p][q] = make_float2(0.f, 0.f);

  for (int pass = 0; pass < 6; ++pass) {
    const int mu = pass - 2;
    float2 Yc[T][T];
#pragma unroll
    for (int p = 0; p < T; ++p)
#pragma unroll
      for (int q = 0; q < T; ++q) Yc[p][q] = make_float2(0.f, 0.f);
    for (int s0 = 0; s0 < a.nb; s0 += kChunk) {
      __syncthreads();
      if (tid < kChunk) {
        const int loc = s0 + tid;
        int xo[4];
        const int x = loc < a.nb ? site_of(a, j, loc, xo) : -1;
        s_site[tid] = x;
        s_face[tid] = (x >= 0 && mu >= 0) ? (xo[mu] % a.b[mu]) == a.b[mu] - 1 : 0;
        if (x >= 0 && mu >= 0) {
          xo[mu] = (xo[mu] + 1) % a.L[mu];
          s_nbr[tid] = xo[0] + a.L[0] * (xo[1] + a.L[1] * (xo[2] + a.L[2] * xo[3]));
        } else {
          s_nbr[tid] = x;
        }
      }
      __syncthreads();
      // stage L and R for the chunk
      for (int idx = tid; idx < kChunk * 6 * NP; idx += 256) {
        const int ls = idx / (6 * NP), rem = idx % (6 * NP);
        const int e = rem / NP, col = rem % NP;
        const int x = s_site[ls];
        float2 lv = make_float2(0.f, 0.f), rv = lv;
        if (x >= 0 && col < n2) {
          const int al = col / k, i = col % k;
          const float2* Px = a.P + (long)x * 12 * k;  // [2][6][k]
          if (mu < 0) {
            const int ar = pass;  // chirality of this pass
            if (al == ar) {
              lv = __ldg(Px + (ar * 6 + e) * k + i);
              float2 sacc = cscale(lv, 0.5f * a.diag);
              if (a.C) {
                const float2* cl = a.C + (long)x * 72 + ar * 36 + e * 6;
#pragma unroll
                for (int f = 0; f < 6; ++f)
                  cfma(sacc, cscale(__ldg(cl + f), 0.5f), __ldg(Px + (ar * 6 + f) * k + i));
              }
              rv = sacc;
            }
          } else {
            const int sp = e / 3, c = e % 3;
            int tt;
            float2 gph;
            pi_entry(mu, sp, tt, gph);
            // Pi_mu(z)[sp][d][col]: offset of the P entry and its phase
            const int off = al == 0 ? (sp * 3) * k + i : (6 + tt * 3) * k + i;
            const float2 ph = al == 0 ? make_float2(1.f, 0.f) : gph;
            lv = cmul(ph, __ldg(Px + off + c * k));
            const float2* Py = a.P + (long)s_nbr[ls] * 12 * k + off;
            const float2* u = a.U + ((long)x * 4 + mu) * 9 + c * 3;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < 3; ++d) cfma(acc, __ldg(u + d), __ldg(Py + d * k));
            rv = cscale(cmul(ph, acc), a.hw[mu]);
          }
        }
        Lf[idx] = lv;
        Rf[idx] = rv;
      }
      __syncthreads();
      // accumulate conj(L)^T R into the tile
      for (int ls = 0; ls < kChunk; ++ls) {
        if (s_site[ls] < 0) break;
        const bool face = s_face[ls];
        float2 t[T][T];
#pragma unroll
        for (int p = 0; p < T; ++p)
#pragma unroll
          for (int q = 0; q < T; ++q) t[p][q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          float2 lv[T], rv[T];
#pragma unroll
          for (int p = 0; p < T; ++p) lv[p] = Lf[(ls * 6 + e) * NP + p * 16 + ti];
#pragma unroll
          for (int q = 0; q < T; ++q) rv[q] = Rf[(ls * 6 + e) * NP + q * 16 + tj];
#pragma unroll
          for (int p = 0; p < T; ++p)
#pragma unroll
            for (int q = 0; q < T; ++q) cfmac(t[p][q], lv[p], rv[q]);
        }
#pragma unroll
        for (int p = 0; p < T; ++p)
#pragma unroll
          for (int q = 0; q < T; ++q) {
            if (face) Yc[p][q] = cadd(Yc[p][q], t[p][q]);
            else S[p][q] = cadd(S[p][q], t[p][q]);
          }
      }
    }
    if (mu >= 0) {
      // Y_{+mu}(j) and Y_{-mu}(j + mu) = sigma_3 Y_{+mu}(j)^dag sigma_3
      int jc[4];
      {
        int t = j;
        jc[0] = t % a.Lc[0]; t /= a.Lc[0];
        jc[1] = t % a.Lc[1]; t /= a.Lc[1];
        jc[2] = t % a.Lc[2]; jc[3] = t / a.Lc[2];
      }
      jc[mu] = (jc[mu] + 1) % a.Lc[mu];
      const int jn = jc[0] + a.Lc[0] * (jc[1] + a.Lc[1] * (jc[2] + a.Lc[2] * jc[3]));
      __syncthreads();
#pragma unroll
      for (int p = 0; p < T; ++p)
#pragma unroll
        for (int q = 0; q < T; ++q) {
          const int r = p * 16 + ti, c = q * 16 + tj;
          Tr[r * (NP + 1) + c] = Yc[p][q];
          if (r < n2 && c < n2) a.Y[(((long)j * 8 + mu) * n2 + r) * n2 + c] = Yc[p][q];
        }
      __syncthreads();
      for (int idx = tid; idx < n2 * n2; idx += 256) {
        const int r = idx / n2, c = idx % n2;
        float2 v = cconj(Tr[c * (NP + 1) + r]);
        if ((r < k) != (c < k)) v = make_float2(-v.x, -v.y);
        a.Y[(((long)jn * 8 + 4 + mu) * n2 + r) * n2 + c] = v;
      }
    }
  }
  // X = S + sigma_3 S^dag sigma_3
  __syncthreads();
#pragma unroll
  for (int p = 0; p < T; ++p)
#pragma unroll
    for (int q = 0; q < T; ++q) Tr[(p * 16 + ti) * (NP + 1) + q * 16 + tj] = S[p][q];
  __syncthreads();
  for (int idx = tid; idx < n2 * n2; idx += 256) {
    const int r = idx / n2, c = idx % n2;
    float2 v = cconj(Tr[c * (NP + 1) + r]);
    if ((r < k) != (c < k)) v = make_float2(-v.x, -v.y);
    a.X[((long)j * n2 + r) * n2 + c] = cadd(Tr[r * (NP + 1) + c], v);
  }
}

// out(xc) = X v(xc) + sum_d Y[d] v(xc + mu_d) + Y[4+d] v(xc - mu_d)
// One CTA per coarse site; the nine source vectors are staged in shared
// memory.  A group of kApLanes consecutive lanes owns one output row: lane j
// of the group takes the columns b = j, j + kApLanes, ... of that row of each
// of the nine matrices, so the group reads a matrix row contiguously and every
// matrix entry, loaded once, multiplies kApRhs right-hand sides.  The group's
// partial sums are added by two shuffles in a fixed order (deterministic).
// Each warp covers 32 / kApLanes consecutive rows per trip, with the same trip
// count on all its lanes, so the shuffles always run on the full warp.
constexpr int kApLanes = 4;
constexpr int kApRhs = 8;  // right-hand sides per register pass
__global__ void __launch_bounds__(256) coarse_apply_kernel(const float2* __restrict__ X,
                                                           const float2* __restrict__ Y,
                                                           const float2* __restrict__ vin,
                                                           float2* __restrict__ vout, int Lc0,
                                                           int Lc1, int Lc2, int Lc3, int n2,
                                                           int nrhs) {
  extern __shared__ float2 vs[];  // [9][n2][nrhs]
  const int xc = blockIdx.x;
  int c0, c1, c2, c3;
  {
    int t = xc;
    c0 = t % Lc0; t /= Lc0;
    c1 = t % Lc1; t /= Lc1;
    c2 = t % Lc2; c3 = t / Lc2;
  }
  const int per = n2 * nrhs;
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    // term d: the site itself (d = 0), its +mu (d = 1..4) or -mu (d = 5..8) neighbour
    // (a step of -1 is taken as L - 1 modulo L)
    const int mu = (d + 3) % 4;
    int a0 = c0, a1 = c1, a2 = c2, a3 = c3;
    if (d > 0) {
      if (mu == 0) a0 = (c0 + (d <= 4 ? 1 : Lc0 - 1)) % Lc0;
      if (mu == 1) a1 = (c1 + (d <= 4 ? 1 : Lc1 - 1)) % Lc1;
      if (mu == 2) a2 = (c2 + (d <= 4 ? 1 : Lc2 - 1)) % Lc2;
      if (mu == 3) a3 = (c3 + (d <= 4 ? 1 : Lc3 - 1)) % Lc3;
    }
    const int src = a0 + Lc0 * (a1 + Lc1 * (a2 + Lc2 * a3));
    for (int i = threadIdx.x; i < per; i += blockDim.x) vs[d * per + i] = vin[(long)src * per + i];
  }
  __syncthreads();
  constexpr int kGroupsPerWarp = 32 / kApLanes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = lane % kApLanes, gw = lane / kApLanes;
  const int nwarp = blockDim.x >> 5;
  const long site = (long)xc * n2 * n2;
  for (int row0 = warp * kGroupsPerWarp; row0 < n2; row0 += nwarp * kGroupsPerWarp) {
    const int row = row0 + gw;
    const bool active = row < n2;
    for (int r0 = 0; r0 < nrhs; r0 += kApRhs) {
      float2 s[kApRhs];
#pragma unroll
      for (int r = 0; r < kApRhs; ++r) s[r] = make_float2(0.f, 0.f);
      if (active) {
        for (int d = 0; d < 9; ++d) {
          const float2* M = (d == 0 ? X + site : Y + ((long)xc * 8 + d - 1) * n2 * n2) +
                            (long)row * n2;
          const float2* v = vs + d * per + r0;
#pragma unroll 4
          for (int b = j; b < n2; b += kApLanes) {
            const float2 m = __ldg(M + b);
#pragma unroll
            for (int r = 0; r < kApRhs; ++r)
              if (r0 + r < nrhs) cfma(s[r], m, v[b * nrhs + r]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kApRhs; ++r) {
#pragma unroll
        for (int off = 1; off < kApLanes; off <<= 1) {
          s[r].x += __shfl_xor_sync(0xffffffffu, s[r].x, off);
          s[r].y += __shfl_xor_sync(0xffffffffu, s[r].y, off);
        }
      }
      if (active && j == 0) {
#pragma unroll
        for (int r = 0; r < kApRhs; ++r)
          if (r0 + r < nrhs) vout[((long)xc * n2 + row) * nrhs + r0 + r] = s[r];
      }
    }
  }
}

}  // namespace

cudaError_t launch_prolongator(const Geom& g, const float2* Uk, float2* P, cudaStream_t s) {
  TimedScope ts("prolongator", s);
  prolongator_kernel<<<4 * 152 * 8, 256, 0, s>>>(Uk, P, g.L[0], g.L[1], g.L[2], g.L[3], g.b[0], g.b[1],
                                           g.b[2], g.b[3], g.k, g.rps);
  return cudaGetLastError();
}

template <int T>
cudaError_t coarsen_t(const CoarsenArgs& a, int nblk, cudaStream_t s) {
  constexpr int NP = 16 * T;
  const size_t smem = sizeof(float2) * (size_t)(2 * kChunk * 6 * NP + NP * (NP + 1));
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(coarsen_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  });
  TimedScope ts("coarsen", s);
  coarsen_kernel<T><<<nblk, 256, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_coarsen(const Geom& g, const float2* U, const float2* C, const float2* P,
                           float2* X, float2* Y, cudaStream_t s) {
  if (g.prec != MG_PREC_FP32 && tc_coarsen_supported(g)) {
    // mixed precision: the contractions on the tensor cores (mg_tc.cu)
    int* st = device_status_word();
    if (!st) return cudaErrorInvalidSymbol;
    return launch_tc_coarsen(g, U, C, P, X, Y, st, s);
  }
  CoarsenArgs a;
  a.U = U;
  a.C = C;
  a.P = P;
  a.X = X;
  a.Y = Y;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.L[i];
    a.b[i] = g.b[i];
    a.Lc[i] = g.Lc[i];
    a.hw[i] = g.hw[i];
  }
  a.nb = g.nb;
  a.k = g.k;
  a.diag = g.diag;
  const int n2 = 2 * g.k;
  const int nblk = (int)g.nblk;
  if (n2 <= 16) return coarsen_t<1>(a, nblk, s);
  if (n2 <= 32) return coarsen_t<2>(a, nblk, s);
  if (n2 <= 48) return coarsen_t<3>(a, nblk, s);
  return coarsen_t<4>(a, nblk, s);
}

cudaError_t launch_coarse_apply(const Geom& g, const float2* X, const float2* Y,
                                const float2* vin, float2* vout, int nrhs, cudaStream_t s) {
  const int n2 = 2 * g.k;
  const size_t smem = sizeof(float2) * (size_t)9 * n2 * nrhs;
  static PerDeviceOnce attr_once;
  attr_once.run([&] {
    cudaFuncSetAttribute(coarse_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
  });
  TimedScope ts("coarse_apply", s);
  coarse_apply_kernel<<<(int)g.nblk, 256, smem, s>>>(X, Y, vin, vout, g.Lc[0], g.Lc[1], g.Lc[2],
                                                     g.Lc[3], n2, nrhs);
  return cudaGetLastError();
}

}  // namespace mg
