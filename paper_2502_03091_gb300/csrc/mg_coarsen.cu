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

constexpr int kCoarsenThreads = 256;
constexpr int kSitesPerStage = 4;

__global__ void prolongator_kernel(const float2* __restrict__ Uk, float2* __restrict__ P, int L0,
                                   int L1, int L2, int L3, int b0, int b1, int b2, int b3,
                                   int k) {
  const long V = (long)L0 * L1 * L2 * L3;
  const int nb = b0 * b1 * b2 * b3;
  const int row = 6 * k;  // complex per (site, chirality)
  const long n = V * 2 * row;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const long x = i / (2 * row);
    const int rem = (int)(i % (2 * row));
    const int al = rem / row, e = rem % row;
    int t = (int)x;
    const int x0 = t % L0; t /= L0;
    const int x1 = t % L1; t /= L1;
    const int x2 = t % L2; const int x3 = t / L2;
    const int Lc0 = L0 / b0, Lc1 = L1 / b1, Lc2 = L2 / b2;
    const int j = x0 / b0 + Lc0 * (x1 / b1 + Lc1 * (x2 / b2 + Lc2 * (x3 / b3)));
    const int loc = x0 % b0 + b0 * (x1 % b1 + b1 * (x2 % b2 + b2 * (x3 % b3)));
    P[i] = Uk[(((long)j * 2 + al) * nb + loc) * row + e];
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

// complex value of B_mu[s][t]
__device__ __forceinline__ float2 bent(int mu, int s, int t) {
  if (mu == 0) return s != t ? make_float2(0.f, -1.f) : make_float2(0.f, 0.f);
  if (mu == 1) return s == 0 && t == 1 ? make_float2(-1.f, 0.f)
                    : (s == 1 && t == 0 ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f));
  if (mu == 2) return s != t ? make_float2(0.f, 0.f)
                             : (s == 0 ? make_float2(0.f, -1.f) : make_float2(0.f, 1.f));
  return s == t ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
}

// One CTA per block j.  Each active thread owns a 4x4 tile of the 2k x 2k
// coarse matrices (NP = 2k rounded up to 4).  Per stage, kSitesPerStage sites
// are staged: for every site the depth-6 left factor Pi(x) and right factor
// W(x) = hw U_mu(x) Pi(x+mu) go to shared memory (depth 12 for the
// diagonal/clover term, with W = 1/2 M(x) P(x)).
__global__ void __launch_bounds__(kCoarsenThreads) coarsen_kernel(CoarsenArgs a) {
  extern __shared__ float2 sm[];
  const int k = a.k, n2 = 2 * k, NP = (n2 + 3) & ~3, TT = NP / 4;
  float2* Ls = sm;                          // [kSitesPerStage][12][NP]
  float2* Rs = Ls + kSitesPerStage * 12 * NP;  // [kSitesPerStage][12][NP]
  float2* Ts = Rs + kSitesPerStage * 12 * NP;  // [NP][NP] transpose scratch
  __shared__ int s_face[kSitesPerStage];
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  const bool active = tid < TT * TT;
  const int ti = tid / TT, tj = tid % TT;
  float2 A[4][4];  // X half: 1/2 M-term + interior hops
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) A[p][q] = make_float2(0.f, 0.f);

  // pass -1: diagonal + clover, pass mu = 0..3: hops
  for (int pass = -1; pass < 4; ++pass) {
    const int depth = pass < 0 ? 12 : 6;
    float2 Yacc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) Yacc[p][q] = make_float2(0.f, 0.f);
    for (int s0 = 0; s0 < a.nb; s0 += kSitesPerStage) {
      __syncthreads();
      // build the factors
      for (int idx = tid; idx < kSitesPerStage * depth * NP; idx += blockDim.x) {
        const int ls = idx / (depth * NP), rem = idx % (depth * NP);
        const int e = rem / NP, col = rem % NP;
        const int loc = s0 + ls;
        float2 lv = make_float2(0.f, 0.f), rv = lv;
        if (loc < a.nb && col < n2) {
          int xo[4];
          const int x = site_of(a, j, loc, xo);
          const int al = col / k, i = col % k;
          const float2* Px = a.P + (long)x * 12 * k;  // [2][6][k]
          if (pass < 0) {
            // rows e = (alpha_r, spin, colour) of the 12 x 2k chirality-sparse P(x)
            const int ar = e / 6, er = e % 6;
            lv = ar == al ? Px[(al * 6 + er) * k + i] : make_float2(0.f, 0.f);
            if (ar == al) {
              float2 s = cscale(Px[(al * 6 + er) * k + i], 0.5f * a.diag);
              if (a.C) {
                const float2* cl = a.C + (long)x * 72 + al * 36 + er * 6;
                for (int f = 0; f < 6; ++f) cfma(s, cscale(cl[f], 0.5f), Px[(al * 6 + f) * k + i]);
              }
              rv = s;
            }
            if (idx % (depth * NP) == 0) s_face[ls] = 0;
          } else {
            const int mu = pass;
            const int sp = e / 3, c = e % 3;
            // Pi(x)[sp][c][col]
            if (al == 0) {
              lv = Px[(0 * 6 + sp * 3 + c) * k + i];
            } else {
              float2 s = make_float2(0.f, 0.f);
              for (int t = 0; t < 2; ++t) cfma(s, bent(mu, sp, t), Px[(6 + t * 3 + c) * k + i]);
              lv = make_float2(-s.x, -s.y);
            }
            // W(x) = hw U_mu(x) Pi(x+mu)
            int y[4] = {xo[0], xo[1], xo[2], xo[3]};
            y[mu] = (y[mu] + 1) % a.L[mu];
            const int xy = y[0] + a.L[0] * (y[1] + a.L[1] * (y[2] + a.L[2] * y[3]));
            const float2* Py = a.P + (long)xy * 12 * k;
            const float2* u = a.U + ((long)x * 4 + mu) * 9 + c * 3;
            float2 s = make_float2(0.f, 0.f);
            for (int d = 0; d < 3; ++d) {
              float2 pid;
              if (al == 0) {
                pid = Py[(sp * 3 + d) * k + i];
              } else {
                float2 q = make_float2(0.f, 0.f);
                for (int t = 0; t < 2; ++t) cfma(q, bent(mu, sp, t), Py[(6 + t * 3 + d) * k + i]);
                pid = make_float2(-q.x, -q.y);
              }
              cfma(s, u[d], pid);
            }
            rv = cscale(s, a.hw[mu]);
            if (idx % (depth * NP) == 0) s_face[ls] = (xo[mu] % a.b[mu]) == a.b[mu] - 1;
          }
        }
        Ls[(ls * 12 + e) * NP + col] = lv;
        Rs[(ls * 12 + e) * NP + col] = rv;
      }
      __syncthreads();
      if (active) {
        for (int ls = 0; ls < kSitesPerStage && s0 + ls < a.nb; ++ls) {
          const bool face = pass >= 0 && s_face[ls];
          float2 t[4][4];
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) t[p][q] = make_float2(0.f, 0.f);
          for (int e = 0; e < depth; ++e) {
            const float2* lr = Ls + (ls * 12 + e) * NP;
            const float2* rr = Rs + (ls * 12 + e) * NP;
            float2 lv[4], rv[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              lv[p] = lr[4 * ti + p];
              rv[p] = rr[4 * tj + p];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) cfmac(t[p][q], lv[p], rv[q]);
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (face) Yacc[p][q] = cadd(Yacc[p][q], t[p][q]);
              else A[p][q] = cadd(A[p][q], t[p][q]);
            }
        }
      }
    }
    if (pass >= 0) {
      // Y_{+mu}(j) and Y_{-mu}(j + mu) = sigma_3 Y_{+mu}(j)^dag sigma_3
      const int mu = pass;
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
      if (active) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = 4 * ti + p, c = 4 * tj + q;
            Ts[r * NP + c] = Yacc[p][q];
            if (r < n2 && c < n2) a.Y[(((long)j * 8 + mu) * n2 + r) * n2 + c] = Yacc[p][q];
          }
      }
      __syncthreads();
      for (int idx = tid; idx < n2 * n2; idx += blockDim.x) {
        const int r = idx / n2, c = idx % n2;
        float2 v = cconj(Ts[c * NP + r]);
        if ((r < k) != (c < k)) v = make_float2(-v.x, -v.y);
        a.Y[(((long)jn * 8 + 4 + mu) * n2 + r) * n2 + c] = v;
      }
    }
  }
  // X = A + sigma_3 A^dag sigma_3
  __syncthreads();
  if (active) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) Ts[(4 * ti + p) * NP + 4 * tj + q] = A[p][q];
  }
  __syncthreads();
  for (int idx = tid; idx < n2 * n2; idx += blockDim.x) {
    const int r = idx / n2, c = idx % n2;
    float2 v = cconj(Ts[c * NP + r]);
    if ((r < k) != (c < k)) v = make_float2(-v.x, -v.y);
    a.X[((long)j * n2 + r) * n2 + c] = cadd(Ts[r * NP + c], v);
  }
}

// out(xc) = X v(xc) + sum_d Y[d] v(xc + mu_d) + Y[4+d] v(xc - mu_d)
// One CTA per coarse site; thread (row, rhs); the nine source vectors are
// staged in shared memory.
__global__ void coarse_apply_kernel(const float2* __restrict__ X, const float2* __restrict__ Y,
                                    const float2* __restrict__ vin, float2* __restrict__ vout,
                                    int Lc0, int Lc1, int Lc2, int Lc3, int n2, int nrhs) {
  extern __shared__ float2 vs[];  // [9][n2][nrhs]
  const int xc = blockIdx.x;
  const int Lc[4] = {Lc0, Lc1, Lc2, Lc3};
  int c[4];
  {
    int t = xc;
    c[0] = t % Lc0; t /= Lc0;
    c[1] = t % Lc1; t /= Lc1;
    c[2] = t % Lc2; c[3] = t / Lc2;
  }
  const int per = n2 * nrhs;
  for (int d = 0; d < 9; ++d) {
    int src = xc;
    if (d > 0) {
      const int mu = (d - 1) % 4, st = d <= 4 ? 1 : -1;
      int cc[4] = {c[0], c[1], c[2], c[3]};
      cc[mu] = (cc[mu] + st + Lc[mu]) % Lc[mu];
      src = cc[0] + Lc0 * (cc[1] + Lc1 * (cc[2] + Lc2 * cc[3]));
    }
    for (int i = threadIdx.x; i < per; i += blockDim.x) vs[d * per + i] = vin[(long)src * per + i];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < per; o += blockDim.x) {
    const int row = o / nrhs, r = o % nrhs;
    float2 s = make_float2(0.f, 0.f);
    for (int d = 0; d < 9; ++d) {
      const float2* M = d == 0 ? X + (long)xc * n2 * n2 : Y + ((long)xc * 8 + d - 1) * n2 * n2;
      const float2* v = vs + d * per;
      for (int b = 0; b < n2; ++b) cfma(s, __ldg(M + row * n2 + b), v[b * nrhs + r]);
    }
    vout[(long)xc * per + o] = s;
  }
}

}  // namespace

cudaError_t launch_prolongator(const Geom& g, const float2* Uk, float2* P, cudaStream_t s) {
  TimedScope ts("prolongator", s);
  prolongator_kernel<<<2048, 256, 0, s>>>(Uk, P, g.L[0], g.L[1], g.L[2], g.L[3], g.b[0], g.b[1],
                                           g.b[2], g.b[3], g.k);
  return cudaGetLastError();
}

cudaError_t launch_coarsen(const Geom& g, const float2* U, const float2* C, const float2* P,
                           float2* X, float2* Y, cudaStream_t s) {
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
  const int NP = (2 * g.k + 3) & ~3;
  const size_t smem = sizeof(float2) * (size_t)(2 * kSitesPerStage * 12 * NP + NP * NP);
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(coarsen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100000);
    attr_done = true;
  }
  TimedScope ts("coarsen", s);
  coarsen_kernel<<<(int)g.nblk, kCoarsenThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_coarse_apply(const Geom& g, const float2* X, const float2* Y,
                                const float2* vin, float2* vout, int nrhs, cudaStream_t s) {
  const int n2 = 2 * g.k;
  const size_t smem = sizeof(float2) * (size_t)9 * n2 * nrhs;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(coarse_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000);
    attr_done = true;
  }
  TimedScope ts("coarse_apply", s);
  coarse_apply_kernel<<<(int)g.nblk, 256, smem, s>>>(X, Y, vin, vout, g.Lc[0], g.Lc[1], g.Lc[2],
                                                     g.Lc[3], n2, nrhs);
  return cudaGetLastError();
}

}  // namespace mg
