// Test harness (host only): runs mg::KrylovHess, the Arnoldi bookkeeping of
// mg_solve, on inner products supplied by the test and returns the
// least-squares solutions, the residual estimates and the valid step counts.
#include "../paper_2502_03091_gb300/csrc/mg_krylov.h"

extern "C" void kh_run(int m, int n, int steps, const double* beta2, const double* hsteps,
                       double* y, double* res, int* kc) {
  mg::KrylovHess hs;
  hs.reset(m, n, beta2);
  const size_t stride = (size_t)(2 * (m + 1) + 1) * n * 2;
  for (int j = 0; j < steps; ++j) {
    hs.step(j, hsteps + j * stride);
    for (int c = 0; c < n; ++c) res[j * n + c] = hs.res(c, j + 1);
  }
  const auto coef = hs.solve(steps);
  for (size_t i = 0; i < coef.size(); ++i) {
    y[2 * i] = coef[i].real();
    y[2 * i + 1] = coef[i].imag();
  }
  for (int c = 0; c < n; ++c) kc[c] = hs.kc[c];
}
