// mg_solve.cu -- the solve the setup serves (paper Sec. 2: the multigrid
// hierarchy used in a K-cycle as the preconditioner of a flexible outer
// Krylov solver, FGMRES).
//
// Outer solver: restarted FGMRES on the fine operator D.  Preconditioner, the
// K-cycle at level l applied to r:
//   x  = nu_pre MR steps on A_l x = r from x = 0;  s = r - A_l x
//   e  = coarse solve of A_{l+1} e = R_l s: GMRES with coarsest_iters steps on
//        the coarsest level, else kcycle_iters FGMRES steps preconditioned by
//        the K-cycle at level l+1
//   x += P_l e;  x += nu_post MR steps on A_l y = r - A_l x
// Arnoldi uses classical Gram-Schmidt applied twice.
//
// nrhs independent systems are solved together.  Every vector is an R x nrhs
// complex64 array whose column c belongs to system c: at the fine level the
// ABI spinor layout [V][4][3][nrhs] (R = 12 V), below it the coarse vector
// layout [V][n][nrhs] (R = n V).  Inner products, step lengths and Krylov
// coefficients are per column; the Krylov bookkeeping (Hessenberg matrices,
// Givens rotations, least-squares solves) runs on the host in double, the
// vector work in the kernels of this file and the operators' kernels
// (mg_dslash.cu at the fine level, the stencil apply of mg_level2.cu below).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "mg_common.cuh"
#include "mg_krylov.h"

namespace mg {

// mg_abi.cu
mg_status make_cgeom(const mg_coarse_problem* p, StencilGeom* sg, Geom* g, bool full);

namespace {

constexpr int kT = 256;
constexpr int kMaxKrylov = 64;   // longest Krylov cycle on any level
constexpr int kDotGrid = 3 * 152;  // one wave at 3 resident CTAs per SM

using cplx = std::complex<double>;

// ---------------------------------------------------------------------------
// vector kernels on R x nrhs arrays (nrhs divides 256)
// ---------------------------------------------------------------------------
// part[blk][i][c] = sum over the CTA's rows r of conj(A_i[r][c]) B[r][c], i < na.
// Four vectors A_i per sweep over B, four rows per loop trip with all their
// loads issued before the products (so that even one vector pair keeps eight
// loads in flight per thread); FP32 products summed in FP32 over 32 rows, then
// in FP64; fixed order.  Dynamic shared memory: kT / 32 * kDotVec * nrhs double2.
constexpr int kDotVec = 4;
constexpr int kRowUnroll = 4;
__global__ void __launch_bounds__(kT, 3) dots_kernel(const float2* __restrict__ A, long astride,
                                                     int na, const float2* __restrict__ B,
                                                     long R, int nrhs, double2* part) {
  extern __shared__ double2 dred[];  // [warp][vector][column]
  const int G = kT / nrhs, c = threadIdx.x % nrhs, g = threadIdx.x / nrhs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long rstep = (long)gridDim.x * G;
  for (int i0 = 0; i0 < na; i0 += kDotVec) {
    const int nv = min(kDotVec, na - i0);
    double2 acc[kDotVec];
    float2 fac[kDotVec];
#pragma unroll
    for (int u = 0; u < kDotVec; ++u) {
      acc[u] = make_double2(0.0, 0.0);
      fac[u] = make_float2(0.f, 0.f);
    }
    int cnt = 0;
    long r = (long)blockIdx.x * G + g;
    for (; r + (kRowUnroll - 1) * rstep < R; r += kRowUnroll * rstep) {
      float2 bv[kRowUnroll], av[kRowUnroll][kDotVec];
#pragma unroll
      for (int q = 0; q < kRowUnroll; ++q) {
        const long o = (r + q * rstep) * nrhs + c;
        bv[q] = __ldg(B + o);
#pragma unroll
        for (int u = 0; u < kDotVec; ++u)
          av[q][u] = u < nv ? __ldg(A + (i0 + u) * astride + o) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < kRowUnroll; ++q)
#pragma unroll
        for (int u = 0; u < kDotVec; ++u) cfmac(fac[u], av[q][u], bv[q]);
      cnt += kRowUnroll;
      if (cnt >= 32) {
#pragma unroll
        for (int u = 0; u < kDotVec; ++u) {
          acc[u].x += fac[u].x;
          acc[u].y += fac[u].y;
          fac[u] = make_float2(0.f, 0.f);
        }
        cnt = 0;
      }
    }
    for (; r < R; r += rstep) {
      const long o = r * nrhs + c;
      const float2 bv = __ldg(B + o);
#pragma unroll
      for (int u = 0; u < kDotVec; ++u)
        if (u < nv) cfmac(fac[u], __ldg(A + (i0 + u) * astride + o), bv);
    }
    // lanes of a warp with the same column: a fixed shuffle tree, then the
    // warps' sums in warp order
#pragma unroll
    for (int u = 0; u < kDotVec; ++u) {
      double x = acc[u].x + fac[u].x, y = acc[u].y + fac[u].y;
      for (int off = nrhs; off < 32; off <<= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, off);
        y += __shfl_xor_sync(0xffffffffu, y, off);
      }
      if (lane < min(nrhs, 32) && u < nv)
        dred[(warp * kDotVec + u) * nrhs + c] = make_double2(x, y);
    }
    __syncthreads();
    // nrhs <= 32: every warp holds every column; nrhs = 64: warp w holds the
    // columns (w % 2) * 32 .. + 31
    const int wstep = nrhs > 32 ? nrhs / 32 : 1;
    for (int t = threadIdx.x; t < nv * nrhs; t += blockDim.x) {
      const int u = t / nrhs, cc = t % nrhs;
      double2 sum = make_double2(0.0, 0.0);
      for (int w = nrhs > 32 ? cc / 32 : 0; w < kT / 32; w += wstep) {
        sum.x += dred[(w * kDotVec + u) * nrhs + cc].x;
        sum.y += dred[(w * kDotVec + u) * nrhs + cc].y;
      }
      part[((long)blockIdx.x * na + i0 + u) * nrhs + cc] = sum;
    }
    __syncthreads();
  }
}

// out[j] = sum over the CTAs' partials: one CTA of 64 threads per output,
// each thread a strided share, then a fixed-order tree (deterministic)
constexpr int kFinT = 64;
__global__ void __launch_bounds__(kFinT) dots_finish(const double2* __restrict__ part, int nblk,
                                                     int n, double2* out) {
  __shared__ double2 red[kFinT];
  const int j = blockIdx.x;
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += kFinT) {
    const double2 v = part[(long)b * n + j];
    s.x += v.x;
    s.y += v.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kFinT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[threadIdx.x].x += red[threadIdx.x + h].x;
      red[threadIdx.x].y += red[threadIdx.x + h].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}

// w[r][c] += sum_{i < na} coef[i][c] A_i[r][c]
__global__ void __launch_bounds__(kT) combo_kernel(float2* w, const float2* __restrict__ A,
                                                   long astride, int na,
                                                   const float2* __restrict__ coef, long n,
                                                   int nrhs) {
  __shared__ float2 cs[kMaxKrylov * 64];
  for (int i = threadIdx.x; i < na * nrhs; i += blockDim.x) cs[i] = coef[i];
  __syncthreads();
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % nrhs);
    float2 acc = w[idx];
    for (int i = 0; i < na; ++i) cfma(acc, cs[i * nrhs + c], __ldg(A + i * astride + idx));
    w[idx] = acc;
  }
}

// out[r][c] = a[c] x[r][c] + b[c] y[r][c]   (y may be null; out may alias x or y)
__global__ void __launch_bounds__(kT) axpby_kernel(float2* out, const float2* x,
                                                   const float2* __restrict__ a, const float2* y,
                                                   const float2* __restrict__ b, long n,
                                                   int nrhs) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % nrhs);
    float2 v = cmul(__ldg(a + c), x[idx]);
    if (y) cfma(v, __ldg(b + c), y[idx]);
    out[idx] = v;
  }
}

// w[r][c] += sign * sum_{i < na} h[i][c] A_i[r][c], coefficients from FP64 inner products
__global__ void __launch_bounds__(kT) combo_d_kernel(float2* w, const float2* __restrict__ A,
                                                     long astride, int na,
                                                     const double2* __restrict__ h, float sign,
                                                     long n, int nrhs) {
  __shared__ float2 cs[kMaxKrylov * 64];
  for (int i = threadIdx.x; i < na * nrhs; i += blockDim.x)
    cs[i] = make_float2(sign * (float)h[i].x, sign * (float)h[i].y);
  __syncthreads();
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % nrhs);
    float2 acc = w[idx];
    for (int i = 0; i < na; ++i) cfma(acc, cs[i * nrhs + c], __ldg(A + i * astride + idx));
    w[idx] = acc;
  }
}

// out[c] = 1 / sqrt(nn[c].x) (0 if nn[c].x <= 0), as a complex scale
__global__ void inv_norm_kernel(const double2* __restrict__ nn, float2* out, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) out[c] = make_float2(nn[c].x > 0 ? (float)(1.0 / sqrt(nn[c].x)) : 0.f, 0.f);
}

// MR step length a = <w, r> / <w, w> per column (0 if <w, w> = 0); out a and -a
__global__ void mr_coef_kernel(const double2* __restrict__ wr, const double2* __restrict__ ww,
                               float2* a, float2* ma, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double d = ww[c].x;
  const float2 v = d > 0 ? make_float2((float)(wr[c].x / d), (float)(wr[c].y / d))
                         : make_float2(0.f, 0.f);
  a[c] = v;
  ma[c] = make_float2(-v.x, -v.y);
}

// ---------------------------------------------------------------------------
// transfers between level l (lattice L, aggregates b, rps rows per site and
// chirality) and level l+1 (kn columns per chirality of P)
// ---------------------------------------------------------------------------
struct Xfer {
  int L[4], b[4], Lc[4];
  int nb, rps, kn, nrhs;
};

__device__ __forceinline__ int xfer_site(const Xfer& t, int j, int loc) {
  int jc[4], lc[4];
  int u = j;
  jc[0] = u % t.Lc[0]; u /= t.Lc[0];
  jc[1] = u % t.Lc[1]; u /= t.Lc[1];
  jc[2] = u % t.Lc[2]; jc[3] = u / t.Lc[2];
  u = loc;
  lc[0] = u % t.b[0]; u /= t.b[0];
  lc[1] = u % t.b[1]; u /= t.b[1];
  lc[2] = u % t.b[2]; lc[3] = u / t.b[2];
  const int x0 = jc[0] * t.b[0] + lc[0], x1 = jc[1] * t.b[1] + lc[1];
  const int x2 = jc[2] * t.b[2] + lc[2], x3 = jc[3] * t.b[3] + lc[3];
  return x0 + t.L[0] * (x1 + t.L[1] * (x2 + t.L[2] * x3));
}

// out[j][a kn + i][c] = sum_{x in block j} sum_{e < rps} conj(P[x][a][e][i]) v[x][a rps + e][c]
// One CTA per block j.  Thread t: output row a kn + i = t % (2 kn), site group
// t / (2 kn) (G groups share the block's sites); each thread keeps up to 8
// right-hand sides in registers (one P load and two float4 loads of v per
// term), then the groups' sums are added in a fixed order.
__global__ void __launch_bounds__(kT) restrict_kernel(Xfer t, const float2* __restrict__ P,
                                                      const float2* __restrict__ v, float2* out) {
  __shared__ float2 red[kT * 8];
  const int j = blockIdx.x;
  const int nrow = 2 * t.kn;
  const int G = kT / nrow;
  const int ai = threadIdx.x % nrow, grp = threadIdx.x / nrow;
  const bool active = grp < G;
  const int a = ai / t.kn, i = ai % t.kn;
  for (int c0 = 0; c0 < t.nrhs; c0 += 8) {
    const int cw = min(8, t.nrhs - c0);  // 4 or 8
    float2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
    if (active) {
      for (int loc = grp; loc < t.nb; loc += G) {
        const int x = xfer_site(t, j, loc);
        const float2* Px = P + ((long)x * 2 + a) * t.rps * t.kn + i;
        const float2* vx = v + ((long)x * 2 * t.rps + a * t.rps) * t.nrhs + c0;
        for (int e = 0; e < t.rps; ++e) {
          const float2 pv = __ldg(Px + e * t.kn);
          const float4* v4 = reinterpret_cast<const float4*>(vx + (long)e * t.nrhs);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (2 * q < cw) {
              const float4 w = __ldg(v4 + q);
              cfmac(acc[2 * q], pv, make_float2(w.x, w.y));
              cfmac(acc[2 * q + 1], pv, make_float2(w.z, w.w));
            }
        }
      }
    }
    __syncthreads();
    if (active)
#pragma unroll
      for (int q = 0; q < 8; ++q) red[(grp * nrow + ai) * 8 + q] = acc[q];
    __syncthreads();
    if (threadIdx.x < nrow)
      for (int q = 0; q < cw; ++q) {
        float2 s = make_float2(0.f, 0.f);
        for (int g = 0; g < G; ++g) s = cadd(s, red[(g * nrow + threadIdx.x) * 8 + q]);
        out[((long)j * nrow + threadIdx.x) * t.nrhs + c0 + q] = s;
      }
  }
}

// fine[x][a rps + e][c] += sum_i P[x][a][e][i] vc[j(x)][a kn + i][c]
// One thread per (site, row), up to 8 right-hand sides in registers.
__global__ void __launch_bounds__(kT) prolong_kernel(Xfer t, const float2* __restrict__ P,
                                                     const float2* __restrict__ vc, float2* fine,
                                                     long V) {
  const long nxe = V * 2 * t.rps;
  for (long xe = blockIdx.x * (long)blockDim.x + threadIdx.x; xe < nxe;
       xe += (long)gridDim.x * blockDim.x) {
    const int ae = (int)(xe % (2 * t.rps));
    const int x = (int)(xe / (2 * t.rps));
    const int a = ae / t.rps;
    int u = x;
    const int c0_ = u % t.L[0]; u /= t.L[0];
    const int c1 = u % t.L[1]; u /= t.L[1];
    const int c2 = u % t.L[2]; const int c3 = u / t.L[2];
    const int j = c0_ / t.b[0] +
                  t.Lc[0] * (c1 / t.b[1] + t.Lc[1] * (c2 / t.b[2] + t.Lc[2] * (c3 / t.b[3])));
    const float2* Pr = P + xe * t.kn;  // P[x][a][e][:]
    for (int c0 = 0; c0 < t.nrhs; c0 += 8) {
      const int cw = min(8, t.nrhs - c0);
      float4* f4 = reinterpret_cast<float4*>(fine + xe * t.nrhs + c0);
      float2 acc[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (2 * q < cw) w = f4[q];
        acc[2 * q] = make_float2(w.x, w.y);
        acc[2 * q + 1] = make_float2(w.z, w.w);
      }
      const float2* vj = vc + ((long)j * 2 * t.kn + a * t.kn) * t.nrhs + c0;
      for (int i = 0; i < t.kn; ++i) {
        const float2 p = __ldg(Pr + i);
        const float4* v4 = reinterpret_cast<const float4*>(vj + (long)i * t.nrhs);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (2 * q < cw) {
            const float4 w = __ldg(v4 + q);
            cfma(acc[2 * q], p, make_float2(w.x, w.y));
            cfma(acc[2 * q + 1], p, make_float2(w.z, w.w));
          }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (2 * q < cw)
          f4[q] = make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
    }
  }
}

int grid_for(long n) {
  const long g = (n + kT - 1) / kT;
  return (int)std::min<long>(g, 152L * 8);
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
struct Lvl {
  bool fine = false;
  long R = 0;            // rows of a vector
  Geom g{};              // fine operator geometry (fine level only)
  StencilGeom sg{};      // coarse operator geometry
  const float2 *U = nullptr, *C = nullptr, *X = nullptr, *Y = nullptr;
  const float2* P = nullptr;  // to level l+1
  Xfer xf{};
  long Vsites = 0;       // sites of this level's lattice
  int kdim = 0;          // length of the Krylov cycle run on this level
  long vstride = 0;      // float2 between consecutive basis vectors (padded)
  bool flexible = false;
  float2 *ts = nullptr, *tw = nullptr, *tx = nullptr, *mr_r = nullptr, *mr_w = nullptr;
  float2 *rhs = nullptr, *sol = nullptr, *V = nullptr, *Z = nullptr, *kw = nullptr;
  // device results of the Krylov cycle on this level: per step j the two
  // Gram-Schmidt passes' inner products and |w|^2, laid out
  // hdev[j][2 (kdim + 1) + 1][nrhs]; the start norm; the column scales
  double2 *hdev = nullptr, *beta2 = nullptr, *mrres = nullptr;
  float2 *scale = nullptr, *mra = nullptr;
};

struct Plan {
  std::vector<Lvl> lv;
  int nrhs = 0;
  char* dws = nullptr;   // fine operator workspace
  double2* part = nullptr;
  double2* dout = nullptr;
  float2* coef = nullptr;
  float2* ones = nullptr;   // [2][nrhs]: 1, then -1
  size_t bytes = 0;
};

class Solver {
 public:
  Solver(Plan& p, const mg_hierarchy& h, cudaStream_t s) : P_(p), h_(h), s_(s), n_(p.nrhs) {}

  cudaError_t solve(const float2* b, float2* x, double tol, int max_iters, int* iters,
                    double* relres) {
    // constant column scales 1 and -1
    std::vector<float2> ones(2 * n_);
    for (int c = 0; c < n_; ++c) {
      ones[c] = make_float2(1.f, 0.f);
      ones[n_ + c] = make_float2(-1.f, 0.f);
    }
    cudaError_t e = cudaMemcpyAsync(P_.ones, ones.data(), sizeof(float2) * ones.size(),
                                    cudaMemcpyHostToDevice, s_);
    if (e != cudaSuccess) return e;
    int steps = 0;
    if ((e = krylov(0, b, x, P_.lv.size() > 1, tol, max_iters, &steps)) != cudaSuccess) return e;
    *iters = steps;
    // true relative residual per system
    Lvl& L = P_.lv[0];
    if ((e = apply(0, x, L.tw)) != cudaSuccess) return e;
    if ((e = axpby(L.ts, b, one(), L.tw, mone(), L.R)) != cudaSuccess) return e;
    if ((e = dots(L.ts, 0, 1, L.ts, L.R, L.mrres)) != cudaSuccess) return e;
    if ((e = dots(b, 0, 1, b, L.R, L.mrres + n_)) != cudaSuccess) return e;
    std::vector<double2> rb(2 * n_);
    if ((e = fetch(rb, L.mrres)) != cudaSuccess) return e;
    for (int c = 0; c < n_; ++c)
      relres[c] = rb[n_ + c].x > 0 ? std::sqrt(std::max(0.0, rb[c].x) / rb[n_ + c].x) : 0.0;
    return cudaSuccess;
  }

 private:
  Plan& P_;
  const mg_hierarchy& h_;
  cudaStream_t s_;
  int n_;
  std::vector<float2> hcoef_;

  const float2* one() const { return P_.ones; }
  const float2* mone() const { return P_.ones + n_; }

  // device -> host copy of out.size() results, then wait for the stream
  cudaError_t fetch(std::vector<double2>& out, const double2* src) {
    cudaError_t e = cudaMemcpyAsync(out.data(), src, sizeof(double2) * out.size(),
                                    cudaMemcpyDeviceToHost, s_);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s_);
  }

  // out[i * nrhs + c] = <A_i[:, c], B[:, c]> (device, FP64)
  cudaError_t dots(const float2* A, long astride, int na, const float2* B, long R,
                   double2* out) {
    const int G = kT / n_;
    // at least 16 rows per thread
    const int grid = (int)std::max<long>(1, std::min<long>((R + 16 * G - 1) / (16 * G), kDotGrid));
    TimedScope ts("s_dots", s_);
    const size_t smem = sizeof(double2) * (kT / 32) * kDotVec * n_;
    dots_kernel<<<grid, kT, smem, s_>>>(A, astride, na, B, R, n_, P_.part);
    const int n = na * n_;
    dots_finish<<<n, kFinT, 0, s_>>>(P_.part, grid, n, out);
    return cudaGetLastError();
  }

  // w += sign * sum_i h[i][c] A_i  (h: device inner products)
  cudaError_t combo_d(float2* w, const float2* A, long astride, int na, const double2* h,
                      float sign, long R) {
    TimedScope ts("s_combo", s_);
    combo_d_kernel<<<grid_for(R * n_), kT, 0, s_>>>(w, A, astride, na, h, sign, R * n_, n_);
    return cudaGetLastError();
  }

  // w += sum_i coef[i][c] A_i  (coef: host values, uploaded)
  cudaError_t combo_h(float2* w, const float2* A, long astride, int na,
                      const std::vector<cplx>& coef, long R) {
    hcoef_.resize(coef.size());
    for (size_t i = 0; i < coef.size(); ++i)
      hcoef_[i] = make_float2((float)coef[i].real(), (float)coef[i].imag());
    cudaError_t e = cudaMemcpyAsync(P_.coef, hcoef_.data(), sizeof(float2) * coef.size(),
                                    cudaMemcpyHostToDevice, s_);
    if (e != cudaSuccess) return e;
    TimedScope ts("s_combo", s_);
    combo_kernel<<<grid_for(R * n_), kT, 0, s_>>>(w, A, astride, na, P_.coef, R * n_, n_);
    return cudaGetLastError();
  }

  // out = a x + b y  (a, b: device column scales; y may be null)
  cudaError_t axpby(float2* out, const float2* x, const float2* a, const float2* y,
                    const float2* b, long R) {
    TimedScope ts("s_axpby", s_);
    axpby_kernel<<<grid_for(R * n_), kT, 0, s_>>>(out, x, a, y, b, R * n_, n_);
    return cudaGetLastError();
  }

  cudaError_t inv_norm(const double2* nn, float2* out) {
    inv_norm_kernel<<<1, 64, 0, s_>>>(nn, out, n_);
    return cudaGetLastError();
  }

  cudaError_t copy(float2* dst, const float2* src, long R) {
    return cudaMemcpyAsync(dst, src, sizeof(float2) * R * n_, cudaMemcpyDeviceToDevice, s_);
  }
  cudaError_t zero(float2* dst, long R) {
    return cudaMemsetAsync(dst, 0, sizeof(float2) * R * n_, s_);
  }

  cudaError_t apply(int l, const float2* in, float2* out) {
    const Lvl& L = P_.lv[l];
    if (L.fine) return launch_dirac(L.g, L.U, L.C, in, out, P_.dws, s_);
    return launch_stencil_apply(L.sg, L.X, L.Y, in, out, n_, s_);
  }

  // x = nu MR steps on A_l x = r from x = 0 (step lengths computed on the device)
  cudaError_t mr(int l, const float2* r, float2* x, int nu) {
    Lvl& L = P_.lv[l];
    cudaError_t e;
    if ((e = zero(x, L.R)) != cudaSuccess) return e;
    if ((e = copy(L.mr_r, r, L.R)) != cudaSuccess) return e;
    for (int t = 0; t < nu; ++t) {
      if ((e = apply(l, L.mr_r, L.mr_w)) != cudaSuccess) return e;
      if ((e = dots(L.mr_w, 0, 1, L.mr_r, L.R, L.mrres)) != cudaSuccess) return e;
      if ((e = dots(L.mr_w, 0, 1, L.mr_w, L.R, L.mrres + n_)) != cudaSuccess) return e;
      mr_coef_kernel<<<1, 64, 0, s_>>>(L.mrres, L.mrres + n_, L.mra, L.mra + n_, n_);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = axpby(x, x, one(), L.mr_r, L.mra, L.R)) != cudaSuccess) return e;
      if ((e = axpby(L.mr_r, L.mr_r, one(), L.mr_w, L.mra + n_, L.R)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // the K-cycle at level l: x = M_l r
  cudaError_t precond(int l, const float2* r, float2* x) {
    Lvl& L = P_.lv[l];
    Lvl& N = P_.lv[l + 1];
    const bool coarsest = l + 2 == (int)P_.lv.size();
    cudaError_t e;
    const float2* s = r;
    if (h_.nu_pre > 0) {
      if ((e = mr(l, r, x, h_.nu_pre)) != cudaSuccess) return e;
      if ((e = apply(l, x, L.tw)) != cudaSuccess) return e;
      if ((e = axpby(L.ts, r, one(), L.tw, mone(), L.R)) != cudaSuccess) return e;
      s = L.ts;
    } else if ((e = zero(x, L.R)) != cudaSuccess) {
      return e;
    }
    {
      TimedScope ts("s_restrict", s_);
      restrict_kernel<<<(unsigned)N.Vsites, kT, 0, s_>>>(L.xf, L.P, s, N.rhs);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    int steps = 0;
    if ((e = krylov(l + 1, N.rhs, N.sol, !coarsest, -1.0, N.kdim, &steps)) != cudaSuccess)
      return e;
    {
      TimedScope ts("s_prolong", s_);
      prolong_kernel<<<grid_for(L.R), kT, 0, s_>>>(L.xf, L.P, N.sol, x, L.Vsites);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (h_.nu_post > 0) {
      if ((e = apply(l, x, L.tw)) != cudaSuccess) return e;
      if ((e = axpby(L.ts, r, one(), L.tw, mone(), L.R)) != cudaSuccess) return e;
      if ((e = mr(l, L.ts, L.tx, h_.nu_post)) != cudaSuccess) return e;
      if ((e = axpby(x, x, one(), L.tx, one(), L.R)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // (F)GMRES on level l from x = 0.  tol < 0: one cycle of L.kdim steps, the
  // stream synchronised once at its end.  Otherwise cycles of L.kdim steps
  // until every column's least-squares residual is <= tol |b_c| or max_iters
  // steps are done, synchronised once per step for the test.
  cudaError_t krylov(int l, const float2* b, float2* x, bool flexible, double tol, int max_iters,
                     int* steps_out) {
    Lvl& L = P_.lv[l];
    const long R = L.R, vs = L.vstride;
    const int m = L.kdim;
    const size_t hstride = (size_t)(2 * (m + 1) + 1) * n_;  // doubles2 per step in hdev
    cudaError_t e;
    std::vector<double> bn(n_, 0.0);
    if (tol >= 0) {
      std::vector<double2> bb(n_);
      if ((e = dots(b, 0, 1, b, R, L.beta2)) != cudaSuccess) return e;
      if ((e = fetch(bb, L.beta2)) != cudaSuccess) return e;
      for (int c = 0; c < n_; ++c) bn[c] = std::sqrt(std::max(0.0, bb[c].x));
    }
    if ((e = zero(x, R)) != cudaSuccess) return e;
    int total = 0;
    bool first = true;
    KrylovHess hs;
    std::vector<double2> beta2(n_), hbuf;
    for (;;) {
      // V_0 = (b - A x) / |b - A x|
      if (first) {
        if ((e = copy(L.V, b, R)) != cudaSuccess) return e;
      } else {
        if ((e = apply(l, x, L.kw)) != cudaSuccess) return e;
        if ((e = axpby(L.V, b, one(), L.kw, mone(), R)) != cudaSuccess) return e;
      }
      if ((e = dots(L.V, 0, 1, L.V, R, L.beta2)) != cudaSuccess) return e;
      if ((e = inv_norm(L.beta2, L.scale)) != cudaSuccess) return e;
      if ((e = axpby(L.V, L.V, L.scale, nullptr, L.scale, R)) != cudaSuccess) return e;
      if (tol >= 0) {
        if ((e = fetch(beta2, L.beta2)) != cudaSuccess) return e;
        hs.reset(m, n_, reinterpret_cast<const double*>(beta2.data()));
      }
      const int jmax = std::min(m, max_iters - total);
      int steps = 0;
      for (int j = 0; j < jmax; ++j) {
        float2* vj = L.V + j * vs;
        float2* zj = flexible ? L.Z + j * vs : vj;
        double2* hj = L.hdev + (size_t)j * hstride;
        if (flexible && (e = precond(l, vj, zj)) != cudaSuccess) return e;
        if ((e = apply(l, zj, L.kw)) != cudaSuccess) return e;
        for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
          double2* hp = hj + (size_t)pass * (m + 1) * n_;
          if ((e = dots(L.V, vs, j + 1, L.kw, R, hp)) != cudaSuccess) return e;
          if ((e = combo_d(L.kw, L.V, vs, j + 1, hp, -1.f, R)) != cudaSuccess) return e;
        }
        double2* hn2 = hj + (size_t)2 * (m + 1) * n_;
        if ((e = dots(L.kw, 0, 1, L.kw, R, hn2)) != cudaSuccess) return e;
        if ((e = inv_norm(hn2, L.scale)) != cudaSuccess) return e;
        if ((e = axpby(L.V + (j + 1) * vs, L.kw, L.scale, nullptr, L.scale, R)) != cudaSuccess)
          return e;
        steps = j + 1;
        if (tol >= 0) {
          hbuf.resize(hstride);
          if ((e = fetch(hbuf, hj)) != cudaSuccess) return e;
          hs.step(j, reinterpret_cast<const double*>(hbuf.data()));
          if (hs.converged(j, tol, bn)) break;
        }
      }
      if (tol < 0) {
        // one fetch for the whole fixed-length cycle
        hbuf.resize(hstride * steps);
        if ((e = cudaMemcpyAsync(beta2.data(), L.beta2, sizeof(double2) * n_,
                                 cudaMemcpyDeviceToHost, s_)) != cudaSuccess)
          return e;
        if (steps > 0 && (e = fetch(hbuf, L.hdev)) != cudaSuccess) return e;
        if (steps == 0 && (e = cudaStreamSynchronize(s_)) != cudaSuccess) return e;
        hs.reset(m, n_, reinterpret_cast<const double*>(beta2.data()));
        for (int j = 0; j < steps; ++j)
          hs.step(j, reinterpret_cast<const double*>(hbuf.data() + (size_t)j * hstride));
      }
      if (steps > 0 &&
          (e = combo_h(x, flexible ? L.Z : L.V, vs, steps, hs.solve(steps), R)) != cudaSuccess)
        return e;
      total += steps;
      if (tol < 0) break;
      if (hs.converged(steps - 1, tol, bn) || total >= max_iters || steps == 0) break;
      first = false;
    }
    *steps_out = total;
    return cudaSuccess;
  }
};

// ---------------------------------------------------------------------------
// plan: geometry of every level and the workspace layout
// ---------------------------------------------------------------------------
mg_status fail_msg(mg_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

mg_status make_plan(const mg_hierarchy* h, int nrhs, int restart, Plan& p, char* ws) {
  if (!h) return fail_msg(MG_ERR_INVALID, "hierarchy is NULL");
  if (nrhs < 4 || nrhs > 64 || (256 % nrhs) != 0)
    return fail_msg(MG_ERR_UNSUPPORTED, "nrhs must be 4, 8, 16, 32 or 64");
  if (restart < 1 || restart > kMaxKrylov)
    return fail_msg(MG_ERR_INVALID, "restart must be in [1, 64]");
  if (h->n_levels < 1 || h->n_levels > 3)
    return fail_msg(MG_ERR_UNSUPPORTED, "n_levels must be 1, 2 or 3");
  if (h->n_levels > 1 &&
      (h->nu_pre < 0 || h->nu_post < 0 || h->coarsest_iters < 1 ||
       h->coarsest_iters > kMaxKrylov || (h->n_levels == 3 &&
                                          (h->kcycle_iters < 1 || h->kcycle_iters > kMaxKrylov))))
    return fail_msg(MG_ERR_INVALID, "K-cycle parameters out of range");
  mg_problem fp = h->fine;
  const int k1 = fp.k;
  fp.n_vec = nrhs;
  fp.k = 1;
  fp.precision = MG_PREC_FP32;
  Geom g0;
  mg_status st = make_geom(&fp, &g0);
  if (st != MG_OK) return st;
  g0.k = k1;
  if (h->n_levels > 1 && (k1 < 1 || k1 > kMaxK))
    return fail_msg(MG_ERR_SHAPE, "fine.k must be in [1, 32]");
  if (ws && !h->U) return fail_msg(MG_ERR_INVALID, "U is NULL");
  if (ws && h->n_levels > 1 && (!h->P || !h->X || !h->Y))
    return fail_msg(MG_ERR_INVALID, "P, X, Y are required for n_levels > 1");
  p.nrhs = nrhs;
  p.lv.assign(h->n_levels, Lvl{});
  Lvl& L0 = p.lv[0];
  L0.fine = true;
  L0.g = g0;
  L0.U = static_cast<const float2*>(h->U);
  L0.C = static_cast<const float2*>(h->C);
  L0.R = g0.V * 12;
  L0.Vsites = g0.V;
  L0.kdim = restart;
  L0.flexible = h->n_levels > 1;
  if (h->n_levels > 1) {
    L0.P = static_cast<const float2*>(h->P);
    for (int i = 0; i < 4; ++i) {
      L0.xf.L[i] = g0.L[i];
      L0.xf.b[i] = g0.b[i];
      L0.xf.Lc[i] = g0.Lc[i];
    }
    L0.xf.nb = g0.nb;
    L0.xf.rps = 6;
    L0.xf.kn = k1;
    L0.xf.nrhs = nrhs;
    Lvl& L1 = p.lv[1];
    for (int i = 0; i < 4; ++i) L1.sg.L[i] = g0.Lc[i];
    L1.sg.V = g0.nblk;
    L1.sg.n = 2 * k1;
    L1.X = static_cast<const float2*>(h->X);
    L1.Y = static_cast<const float2*>(h->Y);
    L1.R = L1.sg.V * L1.sg.n;
    L1.Vsites = L1.sg.V;
    L1.kdim = h->n_levels == 2 ? h->coarsest_iters : h->kcycle_iters;
    L1.flexible = h->n_levels == 3;
  }
  if (h->n_levels == 3) {
    StencilGeom sgc;
    Geom g1;
    if ((st = make_cgeom(&h->second, &sgc, &g1, true)) != MG_OK) return st;
    for (int i = 0; i < 4; ++i)
      if (h->second.dims[i] != g0.Lc[i])
        return fail_msg(MG_ERR_SHAPE, "second.dims must be the fine problem's coarse lattice");
    if (h->second.nc != k1) return fail_msg(MG_ERR_SHAPE, "second.nc must equal fine.k");
    if (ws && (!h->P2 || !h->X2 || !h->Y2))
      return fail_msg(MG_ERR_INVALID, "P2, X2, Y2 are required for n_levels = 3");
    Lvl& L1 = p.lv[1];
    L1.P = static_cast<const float2*>(h->P2);
    for (int i = 0; i < 4; ++i) {
      L1.xf.L[i] = g1.L[i];
      L1.xf.b[i] = g1.b[i];
      L1.xf.Lc[i] = g1.Lc[i];
    }
    L1.xf.nb = g1.nb;
    L1.xf.rps = k1;
    L1.xf.kn = g1.k;
    L1.xf.nrhs = nrhs;
    Lvl& L2 = p.lv[2];
    for (int i = 0; i < 4; ++i) L2.sg.L[i] = g1.Lc[i];
    L2.sg.V = g1.nblk;
    L2.sg.n = 2 * g1.k;
    L2.X = static_cast<const float2*>(h->X2);
    L2.Y = static_cast<const float2*>(h->Y2);
    L2.R = L2.sg.V * L2.sg.n;
    L2.Vsites = L2.sg.V;
    L2.kdim = h->coarsest_iters;
    L2.flexible = false;
  }
  // workspace layout
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return ws ? ws + at : nullptr;
  };
  p.dws = take(smooth_ws_layout(g0).bytes);
  p.part = reinterpret_cast<double2*>(take(sizeof(double2) * kDotGrid * (kMaxKrylov + 1) * 64));
  p.dout = reinterpret_cast<double2*>(take(sizeof(double2) * (kMaxKrylov + 1) * 64));
  p.coef = reinterpret_cast<float2*>(take(sizeof(float2) * (kMaxKrylov + 1) * 64 * 2));
  p.ones = reinterpret_cast<float2*>(take(sizeof(float2) * 2 * 64));
  for (size_t l = 0; l < p.lv.size(); ++l) {
    Lvl& L = p.lv[l];
    const size_t vb = sizeof(float2) * (size_t)L.R * nrhs;
    // every vector, and every basis vector, starts an odd multiple of 256 B
    // past a whole vector from the previous one, so that a kernel streaming
    // several of them does not address them at one large power-of-two-ish
    // distance (a vector of the 32^3x64 lattice at nrhs = 4 is 3 * 2^28 B)
    const size_t pad = 65 * 256;
    L.vstride = (long)((vb + pad) / sizeof(float2));
    auto vec = [&]() { return reinterpret_cast<float2*>(take(vb + pad)); };
    L.ts = vec();
    L.tw = vec();
    L.tx = vec();
    L.mr_r = vec();
    L.mr_w = vec();
    if (l > 0) {
      L.rhs = vec();
      L.sol = vec();
    }
    L.kw = vec();
    L.hdev = reinterpret_cast<double2*>(
        take(sizeof(double2) * (size_t)L.kdim * (2 * (L.kdim + 1) + 1) * nrhs));
    L.beta2 = reinterpret_cast<double2*>(take(sizeof(double2) * nrhs));
    L.mrres = reinterpret_cast<double2*>(take(sizeof(double2) * 2 * nrhs));
    L.scale = reinterpret_cast<float2*>(take(sizeof(float2) * nrhs));
    L.mra = reinterpret_cast<float2*>(take(sizeof(float2) * 2 * nrhs));
    L.V = reinterpret_cast<float2*>(take((vb + pad) * (L.kdim + 1)));
    if (L.flexible) L.Z = reinterpret_cast<float2*>(take((vb + pad) * L.kdim));
  }
  p.bytes = o;
  return MG_OK;
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" {

size_t mg_solve_workspace_size(const mg_hierarchy* h, int32_t nrhs, int32_t restart) {
  Plan p;
  if (make_plan(h, nrhs, restart, p, nullptr) != MG_OK) return 0;
  return p.bytes;
}

mg_status mg_solve(const mg_hierarchy* h, const void* b, void* x, int32_t nrhs, double tol,
                   int32_t restart, int32_t max_iters, int32_t* iters, double* relres, void* ws,
                   size_t ws_bytes, void* stream) {
  Plan p;
  mg_status st = make_plan(h, nrhs, restart, p, nullptr);
  if (st != MG_OK) return st;
  if (!b || !x || !iters || !relres || !ws) return fail_msg(MG_ERR_INVALID, "mg_solve: NULL argument");
  if (b == x) return fail_msg(MG_ERR_INVALID, "mg_solve: x aliases b");
  if (!(tol > 0) || max_iters < 1) return fail_msg(MG_ERR_INVALID, "mg_solve: tol must be > 0 and max_iters >= 1");
  if (ws_bytes < p.bytes) return fail_msg(MG_ERR_INVALID, "mg_solve: workspace too small");
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0)
    return fail_msg(MG_ERR_INVALID, "mg_solve: workspace must be 256-byte aligned");
  if ((st = make_plan(h, nrhs, restart, p, static_cast<char*>(ws))) != MG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Solver solver(p, *h, s);
  const cudaError_t e = solver.solve(static_cast<const float2*>(b), static_cast<float2*>(x), tol,
                                     max_iters, iters, relres);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  int dev_status = 0;
  const cudaError_t e2 = read_device_status(&dev_status, s);
  if (e2 != cudaSuccess) {
    set_last_error(cudaGetErrorString(e2));
    return MG_ERR_CUDA;
  }
  if (dev_status) {
    set_last_error("mg_solve: an operator pass gave up waiting for its staged input");
    return MG_ERR_TIMEOUT;
  }
  return MG_OK;
}

}  // extern "C"
