/*
 * mg_oracle.c -- plain, slow FP64 reference ("oracle") of the chiral rank-k
 * multigrid setup (Whyte, Stathopoulos, Romero, "Chiral rank-k truncations
 * for the multigrid preconditioner of Wilson fermions in lattice QCD",
 * LATTICE2024, arXiv:2502.03091).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  The CUDA path shares no code with
 * it: no headers, no helpers, no tables.
 *
 * Everything is complex128 (interleaved re/im doubles), lexicographic sites
 * s = x + Lx*(y + Ly*(z + Lz*t)).
 *
 * Conventions (the paper leaves them open; these are the readings used):
 *  - chiral gamma basis: gamma_mu = [[0, B_mu], [B_mu^dag, 0]], B_k = -i sigma_k
 *    (k = x, y, z), B_t = 1, so gamma_5 = diag(1, 1, -1, -1).  The chiral split
 *    of Sec. 2 (spins 1,2 vs 3,4) is then plain spin selection.
 *  - Wilson operator, r = 1, hop weights w = (1, 1, 1, 1/xi), periodic:
 *      (D psi)(x) = (m0 + sum_mu w_mu) psi(x) + C(x) psi(x)
 *        - 1/2 sum_mu w_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
 *                          + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]
 *  - clover C(x) = c_sw (i/2) sum_{mu<nu} sigma_mu_nu F_mu_nu(x),
 *    sigma_mu_nu = (i/2)[gamma_mu, gamma_nu], F = (Q - Q^dag)/8, Q the sum of
 *    the four plaquette leaves at x.  (Sign and normalisation are not fixed by
 *    the paper.)
 *  - MR smoother with omega = 1 and one step length per right-hand side, run
 *    on D psi = 0 (Eq. (1)), then each vector scaled to unit 2-norm.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* geometry                                                                  */
/* ------------------------------------------------------------------------ */

static long vol4(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long s, int x[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    x[mu] = (int)(s % L[mu]);
    s /= L[mu];
  }
}

static long lex(const int L[4], const int x[4]) {
  return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

/* neighbour of site s in direction mu, step +1 or -1, periodic */
static long hop(const int L[4], long s, int mu, int step) {
  int x[4];
  coords(L, s, x);
  x[mu] = (x[mu] + step + L[mu]) % L[mu];
  return lex(L, x);
}

/* ------------------------------------------------------------------------ */
/* spin algebra: full 4x4 gamma matrices in the chiral basis                 */
/* ------------------------------------------------------------------------ */

static void gamma_mat(int mu, cplx g[4][4]) {
  cplx B[2][2];
  memset(B, 0, sizeof B);
  switch (mu) {
    case 0: B[0][1] = -I; B[1][0] = -I; break;  /* -i sigma_1 */
    case 1: B[0][1] = -1; B[1][0] = 1; break;   /* -i sigma_2 */
    case 2: B[0][0] = -I; B[1][1] = I; break;   /* -i sigma_3 */
    default: B[0][0] = 1; B[1][1] = 1; break;   /* identity */
  }
  memset(g, 0, sizeof(cplx) * 16);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      g[a][2 + b] = B[a][b];
      g[2 + a][b] = conj(B[b][a]);
    }
}

/* hop weight w_mu */
static double weight(int mu, double xi) { return mu == 3 ? 1.0 / xi : 1.0; }

/* ------------------------------------------------------------------------ */
/* SU(3) helpers                                                            */
/* ------------------------------------------------------------------------ */

static const cplx *link(const double *U, long s, int mu) {
  return (const cplx *)U + ((s * 4 + mu) * 9);
}

static void mat_mul(const cplx *a, const cplx *b, cplx *c) {
  cplx t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += a[i * 3 + k] * b[k * 3 + j];
      t[i * 3 + j] = acc;
    }
  memcpy(c, t, sizeof t);
}

static void mat_dag(const cplx *a, cplx *c) {
  cplx t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t[i * 3 + j] = conj(a[j * 3 + i]);
  memcpy(c, t, sizeof t);
}

/* ------------------------------------------------------------------------ */
/* clover field                                                              */
/* ------------------------------------------------------------------------ */

/* Q_mu_nu(x): sum of the four plaquette leaves in the mu-nu plane at x, all
 * traversed in the same sense (first +mu then +nu). */
static void clover_leaves(const int L[4], const double *U, long x, int mu, int nu,
                          cplx Q[9]) {
  long xpm = hop(L, x, mu, +1), xpn = hop(L, x, nu, +1);
  long xmm = hop(L, x, mu, -1), xmn = hop(L, x, nu, -1);
  long xmm_pn = hop(L, xmm, nu, +1), xmm_mn = hop(L, xmm, nu, -1);
  long xmn_pm = hop(L, xmn, mu, +1);
  cplx a[9], b[9], t[9];
  memset(Q, 0, sizeof(cplx) * 9);
  /* leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x */
  mat_mul(link(U, x, mu), link(U, xpm, nu), t);
  mat_dag(link(U, xpn, mu), a);
  mat_mul(t, a, t);
  mat_dag(link(U, x, nu), a);
  mat_mul(t, a, t);
  for (int i = 0; i < 9; ++i) Q[i] += t[i];
  /* leaf 2: x -> x+nu -> x-mu+nu -> x-mu -> x */
  mat_dag(link(U, xmm_pn, mu), a);
  mat_mul(link(U, x, nu), a, t);
  mat_dag(link(U, xmm, nu), a);
  mat_mul(t, a, t);
  mat_mul(t, link(U, xmm, mu), t);
  for (int i = 0; i < 9; ++i) Q[i] += t[i];
  /* leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x */
  mat_dag(link(U, xmm, mu), a);
  mat_dag(link(U, xmm_mn, nu), b);
  mat_mul(a, b, t);
  mat_mul(t, link(U, xmm_mn, mu), t);
  mat_mul(t, link(U, xmn, nu), t);
  for (int i = 0; i < 9; ++i) Q[i] += t[i];
  /* leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x */
  mat_dag(link(U, xmn, nu), a);
  mat_mul(a, link(U, xmn, mu), t);
  mat_mul(t, link(U, xmn_pm, nu), t);
  mat_dag(link(U, x, mu), a);
  mat_mul(t, a, t);
  for (int i = 0; i < 9; ++i) Q[i] += t[i];
}

/* full 12x12 clover matrix at site x, index (spin*3 + colour) */
static void clover_site(const int L[4], const double *U, double csw, long x,
                        cplx Cf[12][12]) {
  memset(Cf, 0, sizeof(cplx) * 144);
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu) {
      cplx Q[9], F[9], gm[4][4], gn[4][4], sig[4][4];
      clover_leaves(L, U, x, mu, nu, Q);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i * 3 + j] = (Q[i * 3 + j] - conj(Q[j * 3 + i])) / 8.0;
      gamma_mat(mu, gm);
      gamma_mat(nu, gn);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          cplx c = 0;
          for (int e = 0; e < 4; ++e) c += gm[a][e] * gn[e][b] - gn[a][e] * gm[e][b];
          sig[a][b] = 0.5 * I * c;
        }
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              Cf[a * 3 + i][b * 3 + j] += csw * 0.5 * I * sig[a][b] * F[i * 3 + j];
    }
}

/* Clover field, stored per chirality: C[V][2][6][6], index (spin_in_chirality*3 + colour).
 * Also returns (in offblock, if non-NULL) the largest |entry| of the two
 * chirality-mixing 6x6 blocks, which vanish because sigma_mu_nu commutes with gamma_5. */
void or_clover(const int L[4], const double *U, double csw, double *C, double *offblock) {
  long V = vol4(L);
  double off = 0.0;
#pragma omp parallel for schedule(static) reduction(max : off)
  for (long x = 0; x < V; ++x) {
    cplx Cf[12][12];
    clover_site(L, U, csw, x, Cf);
    cplx *c = (cplx *)C + x * 72;
    for (int al = 0; al < 2; ++al)
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) c[al * 36 + i * 6 + j] = Cf[al * 6 + i][al * 6 + j];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double a = cabs(Cf[i][6 + j]), b = cabs(Cf[6 + i][j]);
        if (a > off) off = a;
        if (b > off) off = b;
      }
  }
  if (offblock) *offblock = off;
}

/* ------------------------------------------------------------------------ */
/* Wilson(-clover) operator                                                  */
/* ------------------------------------------------------------------------ */

/* out = D psi for m right-hand sides, psi and out [V][4][3][m].  C may be NULL. */
void or_apply_D(const int L[4], double m0, double xi, const double *U, const double *C,
                int m, const double *psi_in, double *out_) {
  long V = vol4(L);
  const cplx *psi = (const cplx *)psi_in;
  cplx *out = (cplx *)out_;
  double diag = m0;
  for (int mu = 0; mu < 4; ++mu) diag += weight(mu, xi);
  cplx G[4][4][4];
  for (int mu = 0; mu < 4; ++mu) gamma_mat(mu, G[mu]);
#pragma omp parallel for schedule(static)
  for (long x = 0; x < V; ++x) {
    cplx *o = out + x * 12 * m;
    const cplx *px = psi + x * 12 * m;
    for (int i = 0; i < 12 * m; ++i) o[i] = diag * px[i];
    if (C) {
      const cplx *c = (const cplx *)C + x * 72;
      for (int al = 0; al < 2; ++al)
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) {
            cplx cij = c[al * 36 + i * 6 + j];
            for (int r = 0; r < m; ++r) o[(al * 6 + i) * m + r] += cij * px[(al * 6 + j) * m + r];
          }
    }
    for (int mu = 0; mu < 4; ++mu) {
      double hw = -0.5 * weight(mu, xi);
      long xf = hop(L, x, mu, +1), xb = hop(L, x, mu, -1);
      const cplx *uf = link(U, x, mu);
      cplx ub[9];
      mat_dag(link(U, xb, mu), ub);
      const cplx *pf = psi + xf * 12 * m, *pb = psi + xb * 12 * m;
      /* forward: (1 - gamma) U psi(x+mu); backward: (1 + gamma) U^dag psi(x-mu) */
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          cplx sf = (a == b ? 1.0 : 0.0) - G[mu][a][b];
          cplx sb = (a == b ? 1.0 : 0.0) + G[mu][a][b];
          if (sf == 0 && sb == 0) continue;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              cplx cf = hw * sf * uf[i * 3 + j], cb = hw * sb * ub[i * 3 + j];
              for (int r = 0; r < m; ++r)
                o[(a * 3 + i) * m + r] += cf * pf[(b * 3 + j) * m + r] + cb * pb[(b * 3 + j) * m + r];
            }
        }
    }
  }
}

/* Dense matrix of D, (12V) x (12V), row/column index site*12 + spin*3 + colour.
 * Assembled entry by entry (independently of or_apply_D). */
void or_dense_D(const int L[4], double m0, double xi, const double *U, const double *C,
                double *Dm_) {
  long V = vol4(L);
  long n = 12 * V;
  cplx *Dm = (cplx *)Dm_;
  memset(Dm, 0, sizeof(cplx) * n * n);
  double diag = m0;
  for (int mu = 0; mu < 4; ++mu) diag += weight(mu, xi);
  for (long x = 0; x < V; ++x) {
    for (int i = 0; i < 12; ++i) Dm[(x * 12 + i) * n + x * 12 + i] += diag;
    if (C) {
      const cplx *c = (const cplx *)C + x * 72;
      for (int al = 0; al < 2; ++al)
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j)
            Dm[(x * 12 + al * 6 + i) * n + x * 12 + al * 6 + j] += c[al * 36 + i * 6 + j];
    }
    for (int mu = 0; mu < 4; ++mu) {
      cplx g[4][4];
      gamma_mat(mu, g);
      double hw = -0.5 * weight(mu, xi);
      long xf = hop(L, x, mu, +1), xb = hop(L, x, mu, -1);
      const cplx *uf = link(U, x, mu), *ubf = link(U, xb, mu);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              cplx pm = (a == b ? 1.0 : 0.0) - g[a][b];
              cplx pp = (a == b ? 1.0 : 0.0) + g[a][b];
              Dm[(x * 12 + a * 3 + i) * n + xf * 12 + b * 3 + j] += hw * pm * uf[i * 3 + j];
              Dm[(x * 12 + a * 3 + i) * n + xb * 12 + b * 3 + j] += hw * pp * conj(ubf[j * 3 + i]);
            }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* MR smoother on D psi = 0 (Eq. (1))                                        */
/* ------------------------------------------------------------------------ */

/* r = -D psi; for t = 1..niter: w = D r, alpha = <w,r>/<w,w> (per right-hand
 * side, <a,b> = a^dag b), psi += alpha r, r -= alpha w.  Finally psi_i /= |psi_i|.
 * psi0 is not modified.  If resnorm != NULL it receives |r_i| before each
 * iteration and after the last one: [niter+1][m].  If alphas != NULL it
 * receives the step lengths [niter][m] (interleaved complex).  If
 * unnormalised != NULL the vectors before the final scaling are copied there. */
void or_mr(const int L[4], double m0, double xi, const double *U, const double *C, int m,
           int niter, const double *psi0, double *psi_, double *resnorm, double *alphas,
           double *unnormalised) {
  long V = vol4(L);
  long n = 12 * V * (long)m;
  cplx *psi = (cplx *)psi_;
  cplx *r = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n);
  memcpy(psi, psi0, sizeof(cplx) * n);
  or_apply_D(L, m0, xi, U, C, m, (const double *)psi, (double *)r);
  for (long i = 0; i < n; ++i) r[i] = -r[i];
  cplx *wr = malloc(sizeof(cplx) * m);
  double *ww = malloc(sizeof(double) * m), *rr = malloc(sizeof(double) * m);
  for (int t = 0; t <= niter; ++t) {
    if (resnorm) {
      for (int c = 0; c < m; ++c) rr[c] = 0;
      for (long e = 0; e < 12 * V; ++e)
        for (int c = 0; c < m; ++c) {
          cplx v = r[e * m + c];
          rr[c] += creal(v) * creal(v) + cimag(v) * cimag(v);
        }
      for (int c = 0; c < m; ++c) resnorm[t * m + c] = sqrt(rr[c]);
    }
    if (t == niter) break;
    or_apply_D(L, m0, xi, U, C, m, (const double *)r, (double *)w);
    for (int c = 0; c < m; ++c) { wr[c] = 0; ww[c] = 0; }
    for (long e = 0; e < 12 * V; ++e)
      for (int c = 0; c < m; ++c) {
        cplx a = w[e * m + c];
        wr[c] += conj(a) * r[e * m + c];
        ww[c] += creal(a) * creal(a) + cimag(a) * cimag(a);
      }
    for (int c = 0; c < m; ++c) {
      cplx al = ww[c] > 0 ? wr[c] / ww[c] : 0;
      if (alphas) {
        alphas[2 * (t * m + c)] = creal(al);
        alphas[2 * (t * m + c) + 1] = cimag(al);
      }
      wr[c] = al;
    }
#pragma omp parallel for schedule(static)
    for (long e = 0; e < 12 * V; ++e)
      for (int c = 0; c < m; ++c) {
        psi[e * m + c] += wr[c] * r[e * m + c];
        r[e * m + c] -= wr[c] * w[e * m + c];
      }
  }
  if (unnormalised) memcpy(unnormalised, psi, sizeof(cplx) * n);
  for (int c = 0; c < m; ++c) rr[c] = 0;
  for (long e = 0; e < 12 * V; ++e)
    for (int c = 0; c < m; ++c) {
      cplx v = psi[e * m + c];
      rr[c] += creal(v) * creal(v) + cimag(v) * cimag(v);
    }
  for (long e = 0; e < 12 * V; ++e)
    for (int c = 0; c < m; ++c)
      if (rr[c] > 0) psi[e * m + c] /= sqrt(rr[c]);
  free(r);
  free(w);
  free(wr);
  free(ww);
  free(rr);
}

/* ------------------------------------------------------------------------ */
/* dense linear algebra: Householder QR and one-sided Jacobi SVD             */
/* ------------------------------------------------------------------------ */

/* Householder QR of A (K x n, column-major, K >= n), in place: R ends up in
 * the upper triangle; reflector j is H_j = I - tau_j v_j v_j^dag with v_j
 * stored as column j of Vh (K x n, zero above row j). */
static void householder_qr(int K, int n, cplx *A, cplx *Vh, double *tau) {
  for (int j = 0; j < n; ++j) {
    double nx = 0;
    for (int i = j; i < K; ++i) nx += creal(A[j * K + i] * conj(A[j * K + i]));
    nx = sqrt(nx);
    cplx *v = Vh + (long)j * K;
    for (int i = 0; i < K; ++i) v[i] = 0;
    if (nx == 0) {
      tau[j] = 0;
      continue;
    }
    cplx x0 = A[j * K + j];
    cplx ph = cabs(x0) > 0 ? x0 / cabs(x0) : 1.0;
    cplx alpha = -ph * nx; /* reflect x onto alpha e_1 */
    for (int i = j; i < K; ++i) v[i] = A[j * K + i];
    v[j] -= alpha;
    double vv = 0;
    for (int i = j; i < K; ++i) vv += creal(v[i] * conj(v[i]));
    tau[j] = vv > 0 ? 2.0 / vv : 0;
    /* apply H = I - tau v v^dag to columns j..n-1 */
    for (int c = j; c < n; ++c) {
      cplx d = 0;
      for (int i = j; i < K; ++i) d += conj(v[i]) * A[c * K + i];
      d *= tau[j];
      for (int i = j; i < K; ++i) A[c * K + i] -= d * v[i];
    }
  }
}

/* y := Q y for y of length K, Q = H_0 H_1 ... H_{n-1} */
static void apply_q(int K, int n, const cplx *Vh, const double *tau, cplx *y) {
  for (int j = n - 1; j >= 0; --j) {
    if (tau[j] == 0) continue;
    const cplx *v = Vh + (long)j * K;
    cplx d = 0;
    for (int i = j; i < K; ++i) d += conj(v[i]) * y[i];
    d *= tau[j];
    for (int i = j; i < K; ++i) y[i] -= d * v[i];
  }
}

/* One-sided (Hestenes) Jacobi SVD of M (n x n, column-major), in place:
 * on exit the columns of M are sigma_i u_i, and Vm (n x n) holds V with
 * M_in V = U Sigma.  Sweeps until every pair is orthogonal to tol. */
static int hestenes_jacobi(int n, cplx *M, cplx *Vm, double tol, int max_sweeps) {
  for (int i = 0; i < n * n; ++i) Vm[i] = 0;
  for (int i = 0; i < n; ++i) Vm[i * n + i] = 1;
  int sweep;
  for (sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double a = 0, b = 0;
        cplx g = 0;
        for (int i = 0; i < n; ++i) {
          a += creal(M[p * n + i] * conj(M[p * n + i]));
          b += creal(M[q * n + i] * conj(M[q * n + i]));
          g += conj(M[p * n + i]) * M[q * n + i];
        }
        double ag = cabs(g);
        if (ag == 0 || ag <= tol * sqrt(a * b)) continue;
        rotated = 1;
        cplx ph = g / ag; /* phase of the pair's inner product */
        double zeta = (b - a) / (2 * ag);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1 + zeta * zeta));
        double c = 1 / sqrt(1 + t * t), s = c * t;
        for (int i = 0; i < n; ++i) {
          cplx mp = M[p * n + i], mq = M[q * n + i] * conj(ph);
          M[p * n + i] = c * mp - s * mq;
          M[q * n + i] = (s * mp + c * mq) * ph;
          cplx vp = Vm[p * n + i], vq = Vm[q * n + i] * conj(ph);
          Vm[p * n + i] = c * vp - s * vq;
          Vm[q * n + i] = (s * vp + c * vq) * ph;
        }
      }
    if (!rotated) break;
  }
  return sweep;
}

/* Thin SVD of one tall block A (K x n, column-major, K >= n): Householder QR,
 * then one-sided Jacobi on R.  Outputs sigma[n] (descending), Uout (K x n,
 * column-major) left singular vectors, Vout (n x n, column-major) right ones. */
static void block_svd(int K, int n, const cplx *A_in, double *sigma, cplx *Uout, cplx *Vout) {
  cplx *A = malloc(sizeof(cplx) * K * n), *Vh = malloc(sizeof(cplx) * (long)K * n);
  double *tau = malloc(sizeof(double) * n);
  memcpy(A, A_in, sizeof(cplx) * K * n);
  householder_qr(K, n, A, Vh, tau);
  cplx *R = calloc((size_t)n * n, sizeof(cplx)), *Vm = malloc(sizeof(cplx) * n * n);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i <= c; ++i) R[c * n + i] = A[c * K + i];
  hestenes_jacobi(n, R, Vm, 1e-15, 100);
  double *sv = malloc(sizeof(double) * n);
  int *ord = malloc(sizeof(int) * n);
  for (int c = 0; c < n; ++c) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += creal(R[c * n + i] * conj(R[c * n + i]));
    sv[c] = sqrt(s);
    ord[c] = c;
  }
  /* order by descending singular value (insertion sort, stable) */
  for (int i = 1; i < n; ++i) {
    int o = ord[i], j = i - 1;
    while (j >= 0 && sv[ord[j]] < sv[o]) {
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = o;
  }
  cplx *y = malloc(sizeof(cplx) * K);
  for (int c = 0; c < n; ++c) {
    int o = ord[c];
    sigma[c] = sv[o];
    for (int i = 0; i < K; ++i) y[i] = 0;
    if (sv[o] > 0)
      for (int i = 0; i < n; ++i) y[i] = R[o * n + i] / sv[o];
    apply_q(K, n, Vh, tau, y);
    memcpy(Uout + (long)c * K, y, sizeof(cplx) * K);
    memcpy(Vout + (long)c * n, Vm + (long)o * n, sizeof(cplx) * n);
  }
  free(y);
  free(sv);
  free(ord);
  free(R);
  free(Vm);
  free(A);
  free(Vh);
  free(tau);
}

/* Exported for tests: thin SVD of one K x n block given row-major (K x n). */
void or_svd(int K, int n, const double *A_rowmajor, double *sigma, double *U_rowmajor,
            double *V_rowmajor) {
  cplx *A = calloc((size_t)K * n, sizeof(cplx)), *U = malloc(sizeof(cplx) * K * n),
       *Vv = malloc(sizeof(cplx) * n * n);
  const cplx *a = (const cplx *)A_rowmajor;
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < n; ++j) A[j * K + i] = a[(long)i * n + j];
  block_svd(K, n, A, sigma, U, Vv);
  cplx *u = (cplx *)U_rowmajor, *v = (cplx *)V_rowmajor;
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < n; ++j) u[(long)i * n + j] = U[j * K + i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i * n + j] = Vv[j * n + i];
  free(A);
  free(U);
  free(Vv);
}

/* ------------------------------------------------------------------------ */
/* blocking (domain decomposition Lambda_j)                                  */
/* ------------------------------------------------------------------------ */

/* block index j of site x (lexicographic in the coarse coordinate x/b) and
 * local index of x inside its block (lexicographic in x mod b) */
static void block_of(const int L[4], const int b[4], long s, long *j, int *loc) {
  int x[4], xc[4], xl[4], Lc[4];
  coords(L, s, x);
  for (int mu = 0; mu < 4; ++mu) {
    xc[mu] = x[mu] / b[mu];
    xl[mu] = x[mu] % b[mu];
    Lc[mu] = L[mu] / b[mu];
  }
  *j = lex(Lc, xc);
  *loc = (int)lex(b, xl);
}

/* Chiral split + per-block thin SVD + rank-k truncation (Sec. 3, Eq. (4)).
 * For block j and chirality alpha the block A has rows (site in block, spin
 * 2*alpha + s, colour c) and the m test vectors as columns.
 * Outputs:
 *   Uk[nblk][2][|blk|][2][3][k]       the k leading left singular vectors
 *   sigma[nblk][2][m]                 all m singular values, descending
 *   coarse_tv[nblk][2][k][m] (opt.)   Sigma_k V_k^dag
 */
void or_chiral_truncate(const int L[4], const int b[4], int m, int k, const double *psi_,
                        double *Uk_, double *sigma, double *coarse_tv_) {
  long V = vol4(L);
  int nb = b[0] * b[1] * b[2] * b[3];
  long nblk = V / nb;
  int K = 6 * nb;
  const cplx *psi = (const cplx *)psi_;
  cplx *Uk = (cplx *)Uk_, *ctv = (cplx *)coarse_tv_;
  /* site list per block */
  long *sites = malloc(sizeof(long) * V);
  for (long s = 0; s < V; ++s) {
    long j;
    int loc;
    block_of(L, b, s, &j, &loc);
    sites[j * nb + loc] = s;
  }
#pragma omp parallel for schedule(dynamic)
  for (long jb = 0; jb < 2 * nblk; ++jb) {
    long j = jb / 2;
    int al = (int)(jb % 2);
    cplx *A = malloc(sizeof(cplx) * K * m), *U = malloc(sizeof(cplx) * K * m),
         *Vv = malloc(sizeof(cplx) * m * m);
    for (int loc = 0; loc < nb; ++loc)
      for (int s = 0; s < 2; ++s)
        for (int c = 0; c < 3; ++c) {
          int row = (loc * 2 + s) * 3 + c;
          const cplx *src = psi + (sites[j * nb + loc] * 12 + (2 * al + s) * 3 + c) * (long)m;
          for (int i = 0; i < m; ++i) A[(long)i * K + row] = src[i];
        }
    double *sg = sigma + (j * 2 + al) * m;
    block_svd(K, m, A, sg, U, Vv);
    cplx *dst = Uk + (j * 2 + al) * (long)K * k;
    for (int row = 0; row < K; ++row)
      for (int i = 0; i < k; ++i) dst[(long)row * k + i] = U[(long)i * K + row];
    if (ctv) {
      cplx *cd = ctv + (j * 2 + al) * (long)k * m;
      for (int i = 0; i < k; ++i)
        for (int c = 0; c < m; ++c) cd[(long)i * m + c] = sg[i] * conj(Vv[(long)i * m + c]);
    }
    free(A);
    free(U);
    free(Vv);
  }
  free(sites);
}

/* Prolongator (Eq. (5)): P_{alpha i j}(x) = u_i^(alpha)(x) for x in Lambda_j.
 * Stored per site: P[V][2 alpha][2 spin][3 colour][k]; the row (alpha, s, c)
 * is spin 2*alpha + s, the column (alpha, i) is coarse index alpha*k + i. */
void or_prolongator(const int L[4], const int b[4], int k, const double *Uk_, double *P_) {
  long V = vol4(L);
  int nb = b[0] * b[1] * b[2] * b[3];
  const cplx *Uk = (const cplx *)Uk_;
  cplx *P = (cplx *)P_;
  for (long s = 0; s < V; ++s) {
    long j;
    int loc;
    block_of(L, b, s, &j, &loc);
    for (int al = 0; al < 2; ++al)
      for (int e = 0; e < 6; ++e)
        for (int i = 0; i < k; ++i)
          P[((s * 2 + al) * 6 + e) * (long)k + i] =
              Uk[(((j * 2 + al) * nb + loc) * 6 + e) * (long)k + i];
  }
}

/* full 12 x 2k prolongator matrix at site s (rows spin*3+colour) */
static void p_site(int k, const cplx *P, long s, cplx *Pm) {
  for (int i = 0; i < 12 * 2 * k; ++i) Pm[i] = 0;
  for (int al = 0; al < 2; ++al)
    for (int e = 0; e < 6; ++e)
      for (int i = 0; i < k; ++i)
        Pm[(al * 6 + e) * 2 * k + al * k + i] = P[((s * 2 + al) * 6 + e) * (long)k + i];
}

/* acc (2k x 2k) += Pa^dag M Pb with Pa, Pb 12 x 2k, M 12 x 12 */
static void add_pdag_m_p(int k, const cplx *Pa, const cplx M[12][12], const cplx *Pb, cplx *acc) {
  int n = 2 * k;
  cplx *MP = malloc(sizeof(cplx) * 12 * n);
  for (int r = 0; r < 12; ++r)
    for (int c = 0; c < n; ++c) {
      cplx s = 0;
      for (int e = 0; e < 12; ++e) s += M[r][e] * Pb[e * n + c];
      MP[r * n + c] = s;
    }
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) {
      cplx s = 0;
      for (int r = 0; r < 12; ++r) s += conj(Pa[r * n + a]) * MP[r * n + c];
      acc[a * n + c] += s;
    }
  free(MP);
}

/* Galerkin coarse operator D_c = R D P with R = P^dag (Eq. (3)), stored as a
 * nearest-neighbour stencil on the coarse lattice Lc = L / b:
 *   X[nc][2k][2k]     couplings inside one block
 *   Y[nc][8][2k][2k]  Y[xc][d]   couples xc to xc + mu_d     (d = 0..3)
 *                     Y[xc][4+d] couples xc to xc - mu_d
 * (D_c v)(xc) = X v(xc) + sum_d Y[d] v(xc + d) + Y[4+d] v(xc - d).
 * Y[xc][d] holds the hops from the +mu face of block xc; Y[xc][4+d] the hops
 * from its -mu face.  Every term of R D P is computed directly (no symmetry
 * is used). */
void or_coarsen(const int L[4], const int b[4], int k, double m0, double xi, const double *U,
                const double *C, const double *P_, double *X_, double *Y_) {
  long V = vol4(L);
  int n = 2 * k;
  const cplx *P = (const cplx *)P_;
  cplx *X = (cplx *)X_, *Y = (cplx *)Y_;
  int Lc[4];
  for (int mu = 0; mu < 4; ++mu) Lc[mu] = L[mu] / b[mu];
  long nc = vol4(Lc);
  memset(X, 0, sizeof(cplx) * nc * n * n);
  memset(Y, 0, sizeof(cplx) * nc * 8 * n * n);
  double diag = m0;
  for (int mu = 0; mu < 4; ++mu) diag += weight(mu, xi);
  cplx G[4][4][4];
  for (int mu = 0; mu < 4; ++mu) gamma_mat(mu, G[mu]);
  /* serial over sites: the scatter into Y[4+d] of the neighbouring block is
   * not thread-safe and this is a reference, not a fast path */
  cplx *Px = malloc(sizeof(cplx) * 12 * n), *Py = malloc(sizeof(cplx) * 12 * n);
  for (long s = 0; s < V; ++s) {
    long j;
    int loc;
    block_of(L, b, s, &j, &loc);
    int x[4];
    coords(L, s, x);
    p_site(k, P, s, Px);
    cplx M[12][12];
    memset(M, 0, sizeof M);
    for (int e = 0; e < 12; ++e) M[e][e] = diag;
    if (C) {
      const cplx *c = (const cplx *)C + s * 72;
      for (int al = 0; al < 2; ++al)
        for (int i = 0; i < 6; ++i)
          for (int jj = 0; jj < 6; ++jj) M[al * 6 + i][al * 6 + jj] += c[al * 36 + i * 6 + jj];
    }
    add_pdag_m_p(k, Px, M, Px, X + j * n * n);
    for (int mu = 0; mu < 4; ++mu) {
      double hw = -0.5 * weight(mu, xi);
      long y = hop(L, s, mu, +1);
      long jy;
      int locy;
      block_of(L, b, y, &jy, &locy);
      p_site(k, P, y, Py);
      const cplx *u = link(U, s, mu);
      cplx F[12][12], Bk[12][12];
      for (int a = 0; a < 4; ++a)
        for (int bb = 0; bb < 4; ++bb)
          for (int i = 0; i < 3; ++i)
            for (int jj = 0; jj < 3; ++jj) {
              cplx id = (a == bb) ? 1.0 : 0.0;
              /* D(x, x+mu) = hw (1 - gamma) U_mu(x); D(x+mu, x) = hw (1 + gamma) U_mu(x)^dag */
              F[a * 3 + i][bb * 3 + jj] = hw * (id - G[mu][a][bb]) * u[i * 3 + jj];
              Bk[a * 3 + i][bb * 3 + jj] = hw * (id + G[mu][a][bb]) * conj(u[jj * 3 + i]);
            }
      int on_face = (x[mu] % b[mu]) == b[mu] - 1;
      if (!on_face) {
        add_pdag_m_p(k, Px, F, Py, X + j * n * n);  /* x -> x+mu inside the block */
        add_pdag_m_p(k, Py, Bk, Px, X + j * n * n); /* x+mu -> x inside the block */
      } else {
        add_pdag_m_p(k, Px, F, Py, Y + (j * 8 + mu) * n * n);       /* block j -> j+mu */
        add_pdag_m_p(k, Py, Bk, Px, Y + (jy * 8 + 4 + mu) * n * n); /* block j+mu -> j */
      }
    }
  }
  free(Px);
  free(Py);
}

/* Coarse apply: out(xc) = X v(xc) + sum_d Y[d] v(xc + d) + Y[4+d] v(xc - d),
 * v and out [nc][2k][nrhs]. */
void or_coarse_apply(const int Lc[4], int k, const double *X_, const double *Y_, int nrhs,
                     const double *v_, double *out_) {
  long nc = vol4(Lc);
  int n = 2 * k;
  const cplx *X = (const cplx *)X_, *Y = (const cplx *)Y_, *v = (const cplx *)v_;
  cplx *out = (cplx *)out_;
#pragma omp parallel for schedule(static)
  for (long xc = 0; xc < nc; ++xc) {
    cplx *o = out + xc * n * nrhs;
    for (int i = 0; i < n * nrhs; ++i) o[i] = 0;
    for (int d = -1; d < 8; ++d) {
      const cplx *M;
      long src;
      if (d < 0) {
        M = X + xc * n * n;
        src = xc;
      } else {
        M = Y + (xc * 8 + d) * n * n;
        src = hop(Lc, xc, d % 4, d < 4 ? +1 : -1);
      }
      const cplx *vs = v + src * n * nrhs;
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
          cplx mac = M[a * n + c];
          for (int r = 0; r < nrhs; ++r) o[a * nrhs + r] += mac * vs[c * nrhs + r];
        }
    }
  }
}

/* gamma_5-applied copy, for tests: out = gamma_5 psi ([V][4][3][m]) */
void or_gamma5(long V, int m, const double *psi_, double *out_) {
  const cplx *psi = (const cplx *)psi_;
  cplx *out = (cplx *)out_;
  for (long x = 0; x < V; ++x)
    for (int sp = 0; sp < 4; ++sp)
      for (int e = 0; e < 3 * m; ++e) {
        long i = (x * 4 + sp) * 3 * (long)m + e;
        out[i] = sp < 2 ? psi[i] : -psi[i];
      }
}
