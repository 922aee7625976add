// mg_krylov.h -- host-side bookkeeping of one (F)GMRES cycle of mg_solve for
// nrhs independent systems (plain C++, no CUDA types, so that it is unit
// tested on the host).
//
// Per column c: the Hessenberg matrix H_c ((m + 1) x m, column-major), the
// Givens rotations that keep it upper triangular, and the rotated right-hand
// side g_c = Q (beta_c e_1), whose entry j + 1 is the least-squares residual
// after j + 1 steps.  The input of Arnoldi step j is what the device computed:
// the two classical Gram-Schmidt passes' inner products h1[0..j], h2[0..j] and
// |w|^2, as interleaved (re, im) doubles in the layout
//   hj[(i * n + c) * 2]                  pass 1, i <= j
//   hj[((m + 1 + i) * n + c) * 2]        pass 2, i <= j
//   hj[(2 (m + 1) * n + c) * 2]          |w|^2 (real part)
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstddef>
#include <vector>

namespace mg {

struct KrylovHess {
  using cplx = std::complex<double>;
  int m = 0, n = 0;
  std::vector<cplx> H, g, sn;
  std::vector<double> cs;
  std::vector<int> kc;  // -1: growing; else the column's number of valid steps

  // beta2: |r_c|^2 of the cycle's start (real parts of n interleaved pairs)
  void reset(int m_, int n_, const double* beta2) {
    m = m_;
    n = n_;
    H.assign((size_t)n * (m + 1) * m, 0.0);
    g.assign((size_t)n * (m + 1), 0.0);
    sn.assign((size_t)n * m, 0.0);
    cs.assign((size_t)n * m, 0.0);
    kc.assign(n, 0);
    for (int c = 0; c < n; ++c) {
      const double beta = std::sqrt(std::max(0.0, beta2[2 * c]));
      g[(size_t)c * (m + 1)] = beta;
      kc[c] = beta > 0 ? -1 : 0;
    }
  }
  cplx& h(int c, int i, int j) { return H[(size_t)c * (m + 1) * m + i + (size_t)(m + 1) * j]; }
  double res(int c, int j) const { return std::abs(g[(size_t)c * (m + 1) + j]); }

  // Arnoldi step j: fill column j, apply the previous rotations, then a new one
  // that zeroes H[j+1][j]; |w| = 0 is an exact breakdown of that column.
  void step(int j, const double* hj) {
    for (int c = 0; c < n; ++c) {
      if (kc[c] >= 0) continue;
      const double hn = std::sqrt(std::max(0.0, hj[((size_t)2 * (m + 1) * n + c) * 2]));
      for (int i = 0; i <= j; ++i) {
        const double* a1 = hj + ((size_t)i * n + c) * 2;
        const double* a2 = hj + ((size_t)(m + 1 + i) * n + c) * 2;
        h(c, i, j) = cplx(a1[0] + a2[0], a1[1] + a2[1]);
      }
      h(c, j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {
        cplx& a = h(c, i, j);
        cplx& b = h(c, i + 1, j);
        const double ci = cs[(size_t)c * m + i];
        const cplx si = sn[(size_t)c * m + i];
        const cplx t0 = ci * a + si * b;
        const cplx t1 = -std::conj(si) * a + ci * b;
        a = t0;
        b = t1;
      }
      cplx& a = h(c, j, j);
      const double aa = std::abs(a);
      double cj;
      cplx sj;
      if (hn == 0.0) {
        cj = 1.0;
        sj = 0.0;
      } else if (aa == 0.0) {
        cj = 0.0;
        sj = 1.0;
      } else {
        const double t = std::sqrt(aa * aa + hn * hn);
        cj = aa / t;
        sj = (a / aa) * hn / t;
      }
      cs[(size_t)c * m + j] = cj;
      sn[(size_t)c * m + j] = sj;
      a = cj * a + sj * hn;
      h(c, j + 1, j) = 0.0;
      cplx* gc = &g[(size_t)c * (m + 1)];
      gc[j + 1] = -std::conj(sj) * gc[j];
      gc[j] = cj * gc[j];
      if (hn == 0.0) kc[c] = j + 1;  // breakdown: exact in this column
    }
  }

  bool converged(int j, double tol, const std::vector<double>& bn) const {
    for (int c = 0; c < n; ++c)
      if (!(kc[c] >= 0 || res(c, j + 1) <= tol * bn[c])) return false;
    return true;
  }

  // y_c = H_c^-1 g_c over the column's valid steps, as [steps][n]
  std::vector<cplx> solve(int steps) {
    std::vector<cplx> coef((size_t)steps * n, 0.0);
    for (int c = 0; c < n; ++c) {
      const int k = kc[c] < 0 ? steps : std::min(kc[c], steps);
      std::vector<cplx> y(k);
      for (int i = k - 1; i >= 0; --i) {
        cplx acc = g[(size_t)c * (m + 1) + i];
        for (int q = i + 1; q < k; ++q) acc -= h(c, i, q) * y[q];
        const cplx d = h(c, i, i);
        y[i] = std::abs(d) > 0 ? acc / d : 0.0;
      }
      for (int i = 0; i < k; ++i) coef[(size_t)i * n + c] = y[i];
    }
    return coef;
  }
};

}  // namespace mg
