/*
 * mg.h -- C ABI of the GB300 (sm_103a) setup path of the chiral rank-k
 * multigrid preconditioner for Wilson fermions (Whyte, Stathopoulos,
 * Romero, arXiv:2502.03091, LATTICE2024).
 *
 * One level of the setup, as the paper states it:
 *   mg_smooth_testvecs    smoother on D psi = 0 from m' random starts   (Sec. 2, Eq. 1)
 *   mg_chiral_truncate    chiral split + per-block SVD, keep rank k    (Sec. 2 Eq. 2; Sec. 3 Eq. 4)
 *   mg_build_prolongator  block-diagonal prolongator P, R = P^dagger   (Sec. 3 Eq. 5; Sec. 2)
 *   mg_coarsen            Galerkin coarse operator D_c = R D P          (Sec. 2 Eq. 3)
 *   mg_coarse_apply       D_c v on the coarse nearest-neighbour stencil (Sec. 2 Eq. 3; Sec. 1)
 * plus the operator preparation mg_clover_field (the clover term of the
 * ensembles of Sec. 4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Memory.  Every array argument is a DEVICE pointer owned by the caller
 *    (the library never allocates or frees device memory).  Scratch space is
 *    passed in as (ws, ws_bytes); mg_workspace_size() gives the size.  A
 *    NULL required pointer, or ws_bytes smaller than required, returns
 *    MG_ERR_INVALID before anything is launched.
 *  Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Calls only enqueue work on that stream and return;
 *    outputs are valid once the stream reaches that point.
 *  Errors.  Argument and shape checks happen synchronously and are returned.
 *    Launch failures return MG_ERR_CUDA.  Numerical trouble found on the
 *    device (non-positive Cholesky pivot) is reported per block in the
 *    blk_flags output of mg_chiral_truncate.  mg_last_error() gives a
 *    human-readable message for the calling thread's last failure.  No call
 *    aborts the process; no exception crosses the ABI.
 *  Numbers.  Complex numbers are interleaved (re, im).  MG_PREC_FP32 stores
 *    every field as complex64 (float2); singular values are double.
 *  Lattice.  Sites are lexicographic, s = x + Lx*(y + Ly*(z + Lz*t)),
 *    periodic in all four directions.  Gamma matrices are in the chiral
 *    basis gamma_mu = [[0, B_mu], [B_mu^dag, 0]], B_{x,y,z} = -i sigma_{1,2,3},
 *    B_t = 1, so gamma_5 = diag(1, 1, -1, -1): chirality alpha = 0 is spins
 *    {0, 1}, alpha = 1 is spins {2, 3}.
 *  Operator.  r = 1 Wilson-clover with hop weights w = (1, 1, 1, 1/xi):
 *    (D psi)(x) = (m0 + sum_mu w_mu) psi(x) + C(x) psi(x)
 *                 - 1/2 sum_mu w_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                   + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ].
 *  Blocks.  Aggregate Lambda_j has extents problem.block; its index j is the
 *    lexicographic index of the coarse coordinate x / block; sites inside
 *    a block are in local lexicographic order.
 *
 * Array layouts (element counts; V = volume, nb = |Lambda|, nblk = V / nb,
 * m = n_vec, k = problem.k, nc = nblk):
 *  U      [V][4 mu][3][3]                       links, U_mu(x) joins x -> x + mu
 *  C      [V][2 alpha][6][6]                    clover, one Hermitian 6x6 per chirality,
 *                                               row/col index = spin_in_chirality*3 + colour
 *  psi    [V][4 spin][3 colour][m]              test vectors, right-hand sides fastest
 *  Uk     [nblk][2 alpha][nb][2 spin][3 col][k] truncated left singular vectors
 *  sigma  [nblk][2 alpha][k]                    retained singular values (double)
 *  P      [V][2 alpha][2 spin][3 col][k]        prolongator per site; row (alpha, s, c) is
 *                                               spin 2*alpha + s, column (alpha, i) is coarse
 *                                               index alpha*k + i
 *  X      [nc][2k][2k]                          coarse self coupling
 *  Y      [nc][8][2k][2k]                       coarse hops, d = 0..3: to xc + mu_d,
 *                                               d = 4..7: to xc - mu_{d-4}
 *  v      [nc][2k][nrhs]                        coarse vectors
 */
#ifndef MG_H_
#define MG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,     /* NULL pointer, bad parameter value, workspace too small */
  MG_ERR_SHAPE = 2,       /* dims not divisible by block, k out of range, ... */
  MG_ERR_NOMEM = 3,       /* reserved: the library itself never allocates */
  MG_ERR_CUDA = 4,        /* a CUDA launch or runtime call failed */
  MG_ERR_NUMERICAL = 5,   /* reserved: numerical trouble of a block is reported per block
                             in blk_flags, not by a call's status */
  MG_ERR_TIMEOUT = 6,     /* a bounded device wait gave up (returned by mg_sync_status
                             and mg_solve); the outputs of the calls it covers are not valid */
  MG_ERR_UNSUPPORTED = 7  /* valid request this build does not implement */
} mg_status;

typedef enum {
  MG_PREC_FP32 = 0,       /* complex64 storage, FP32 arithmetic on the CUDA cores; the
                             small Cholesky / R-factor eigen problems in double-float
                             (pairs of FP32, ~2^-44 relative) */
  MG_PREC_MIXED = 1,      /* the smoother as MG_PREC_FP32; the dense contractions of
                             the truncation and of the Galerkin coarsening on the tensor
                             cores with FP32 accumulation: the first Gram (only the
                             preconditioner of CholeskyQR2's second pass) in BF16; the
                             second Gram, Q1 = A R1^-1, U_k and the coarse-link products
                             with FP16 operands split into hi + lo parts (three products,
                             about FP32 accuracy, a power-of-two scale per block or
                             block-chirality); double-float Cholesky / R-factor eigen
                             problem.
                             Results agree with the FP64 reference as closely as the
                             MG_PREC_FP32 path's do. */
  MG_PREC_MIXED_FP16 = 2  /* as MG_PREC_MIXED, but the smoother's fields are stored
                             in FP16 (FP32 arithmetic): half the smoother's memory
                             traffic, at a test-vector error of about 1e-2 relative
                             (the MR recurrence amplifies the storage rounding) */
} mg_precision;

typedef struct {
  int32_t dims[4];    /* Lx, Ly, Lz, Lt */
  int32_t block[4];   /* aggregate extents, each must divide dims[i] */
  double m0;          /* bare mass */
  double csw;         /* clover coefficient (used only by mg_clover_field) */
  double xi;          /* anisotropy: temporal hop weight 1/xi (xi = 1 isotropic) */
  int32_t n_vec;      /* m' test vectors; 4 <= m' <= 64, m' % 4 == 0, 6*nb >= m' */
  int32_t k;          /* kept per chirality, 1 <= k <= m' */
  int32_t mr_iters;   /* smoother iterations N >= 1 */
  int32_t precision;  /* mg_precision */
  uint64_t seed;      /* read only by mg_random_starts */
} mg_problem;

/* Which call a workspace size is asked for. */
typedef enum {
  MG_CALL_SMOOTH = 0,
  MG_CALL_TRUNCATE = 1,
  MG_CALL_COARSEN = 2
} mg_call;

/* Bytes of scratch the call `which` (mg_call) needs for this problem; 0 for
 * an invalid problem (mg_last_error() says why). */
size_t mg_workspace_size(const mg_problem* prob, int which);

/* Clover field of the ensembles' clover action (Sec. 4 of the paper; the
 * normalisation is this library's reading):
 *   C(x) = csw (i/2) sum_{mu<nu} sigma_mu_nu F_mu_nu(x),
 *   sigma_mu_nu = (i/2)[gamma_mu, gamma_nu], F = (Q - Q^dag)/8,
 * Q the sum of the four plaquette leaves in the mu-nu plane at x.
 * In: U.  Out: C (layout above).  FP32 arithmetic. */
mg_status mg_clover_field(const mg_problem* prob, const void* U, void* C, void* stream);

/* The fine operator D (Sec. 1-2: the Wilson-Dirac operator whose near null
 * space the setup exposes) applied to n_vec right-hand sides:
 * out = D in, layouts [V][4][3][n_vec].  In: U, C (NULL for pure Wilson), in.
 * Out: out (must not alias in).  ws: mg_workspace_size(prob, MG_CALL_SMOOTH)
 * bytes (the same scratch as the smoother). */
mg_status mg_apply_dirac(const mg_problem* prob, const void* U, const void* C, const void* in,
                         void* out, void* ws, size_t ws_bytes, void* stream);

/* Smoother on the homogeneous system D psi_i ~ 0 (Sec. 2, Eq. 1): minimal
 * residual with one step length per vector, mr_iters iterations, starting
 * from psi0, then every vector scaled to unit 2-norm.  In exact arithmetic:
 *   r = -D psi; repeat N times { w = D r; a = <w,r>/<w,w>; psi += a r; r -= a w };
 *   psi_i /= |psi_i|.
 * In: U, C (NULL for pure Wilson), psi0.  Out: psi (may alias psi0).
 * ws: mg_workspace_size(prob, MG_CALL_SMOOTH) bytes. */
mg_status mg_smooth_testvecs(const mg_problem* prob, const void* U, const void* C,
                             const void* psi0, void* psi, void* ws, size_t ws_bytes,
                             void* stream);

/* Chiral split and rank-k truncation (Sec. 2 Eq. 2, Sec. 3 Eq. 4).  For
 * every block Lambda_j and chirality alpha the 6*nb x m' matrix
 * Psi^(alpha)(Lambda_j) (rows: site, spin in chirality, colour) is factored
 * by CholeskyQR2 and the SVD of its m' x m' R factor; the k leading left
 * singular vectors U_k and singular values Sigma_k are kept.
 * In: psi.  Out: Uk, sigma (double), optional coarse_tv (NULL to skip):
 * Sigma_k V_k^dag as [nblk][2][k][m'] complex64, and blk_flags[nblk*2]
 * (int32; 0 = clean, bit 0 = Cholesky of the Gram needed a diagonal shift,
 * bit 1 = the shifted Cholesky failed as well, results of that block are
 * not meaningful).  ws: mg_workspace_size(prob, MG_CALL_TRUNCATE) bytes. */
mg_status mg_chiral_truncate(const mg_problem* prob, const void* psi, void* Uk,
                             double* sigma, void* coarse_tv, int32_t* blk_flags, void* ws,
                             size_t ws_bytes, void* stream);

/* Prolongator (Sec. 3, Eq. 5): P_{alpha i j}(x) = u_i^(alpha)(x) for x in
 * Lambda_j, zero elsewhere; R = P^dagger is never stored.  Re-packs the
 * block-major Uk into the site-major P.  In: Uk.  Out: P. */
mg_status mg_build_prolongator(const mg_problem* prob, const void* Uk, void* P, void* stream);

/* Galerkin coarse operator D_c = R D P, R = P^dagger (Sec. 2, Eq. 3), as the
 * coarse nearest-neighbour stencil X, Y (layouts above).  Y for the -mu
 * directions is obtained from gamma_5-hermiticity, Y_{-mu}(xc + mu) =
 * sigma_3 Y_{+mu}(xc)^dag sigma_3 with sigma_3 = diag(1_k, -1_k).
 * In: U, C (NULL for pure Wilson), P.  Out: X, Y.
 * ws: mg_workspace_size(prob, MG_CALL_COARSEN) bytes (may be 0). */
mg_status mg_coarsen(const mg_problem* prob, const void* U, const void* C, const void* P,
                     void* X, void* Y, void* ws, size_t ws_bytes, void* stream);

/* Coarse operator apply: out(xc) = X v(xc) + sum_{d<4} Y[d] v(xc + mu_d)
 * + Y[4+d] v(xc - mu_d) on the periodic coarse lattice dims/block.
 * In: X, Y, v_in [nc][2k][nrhs].  Out: v_out (must not alias v_in).
 * 1 <= nrhs <= 64, and the nine source vectors of a coarse site,
 * 9 x 2k x nrhs complex64, must fit the 200000 bytes the call stages in
 * shared memory (nrhs <= 57 at k = 24, <= 43 at k = 32); a larger request is
 * rejected with MG_ERR_UNSUPPORTED before anything is launched. */
mg_status mg_coarse_apply(const mg_problem* prob, const void* X, const void* Y,
                          const void* v_in, void* v_out, int32_t nrhs, void* stream);

/* ------------------------------------------------------------------------
 * Levels l >= 1 (Sec. 2: the hierarchy is built recursively, D_{l+1} = R D_l P,
 * and for l > 0 the chiral split uses gamma_5^l = sigma_3).  The operator D_l
 * is a coarse stencil (X, Y) -- the output of mg_coarsen, or of
 * mg_coarse_coarsen one level up -- on the periodic lattice `dims` with
 * 2*nc complex components per site; chirality alpha is the component block
 * alpha*nc .. alpha*nc + nc - 1.  Each call repeats the fine-level call of
 * the same name with D -> D_l and gamma_5 -> sigma_3, and follows the same
 * conventions (caller-owned device memory, stream semantics, errors).
 * Array layouts (complex64 unless noted; V = volume of dims, nb = |block|,
 * nblk = V / nb, m = n_vec, k = problem.k):
 *  X      [V][2nc][2nc]            D_l self coupling
 *  Y      [V][8][2nc][2nc]         D_l hops (d = 0..3 to x + mu_d, 4..7 to x - mu_{d-4})
 *  v, psi [V][2nc][nrhs or m]      vectors, right-hand sides fastest
 *  Uk     [nblk][2][nb][nc][k]     truncated left singular vectors
 *  sigma  [nblk][2][k]             retained singular values (double)
 *  P      [V][2][nc][k]            prolongator; row (alpha, e) is component
 *                                  alpha*nc + e, column (alpha, i) is coarse
 *                                  index alpha*k + i
 *  X2     [nblk][2k][2k]           D_{l+1} self coupling
 *  Y2     [nblk][8][2k][2k]        D_{l+1} hops
 * X, Y, v and psi must be 16-byte aligned (they are staged by bulk copies).
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t dims[4];   /* lattice of D_l (the coarse lattice of level l - 1) */
  int32_t block[4];  /* aggregate extents on that lattice, each divides dims[i] */
  int32_t nc;        /* D_l has 2*nc components per site; 1 <= nc <= 32 */
  int32_t n_vec;     /* m test vectors; 4 <= m <= 64, m % 4 == 0, nc*nb >= m */
  int32_t k;         /* kept per chirality, 1 <= k <= min(m, 32) */
  int32_t mr_iters;  /* smoother iterations N >= 1 */
} mg_coarse_problem;

/* Scratch bytes of mg_coarse_smooth_testvecs (MG_CALL_SMOOTH) or
 * mg_coarse_chiral_truncate (MG_CALL_TRUNCATE); 0 for MG_CALL_COARSEN and
 * for an invalid problem (mg_last_error() then says why). */
size_t mg_coarse_workspace_size(const mg_coarse_problem* prob, int which);

/* out = D_l v for 1 <= nrhs <= 64 right-hand sides (Sec. 2, Eq. 3: the
 * coarse stencil applied as a nearest-neighbour operator):
 *   out(x) = X(x) v(x) + sum_{d<4} Y_d(x) v(x + mu_d) + Y_{4+d}(x) v(x - mu_d).
 * Only prob->dims and prob->nc are read (so the same call applies D_{l+1}
 * with dims = the aggregated lattice and nc = k).  In: X, Y, v_in.  Out:
 * v_out (must not alias v_in).  FP32 arithmetic. */
mg_status mg_coarse_op_apply(const mg_coarse_problem* prob, const void* X, const void* Y,
                             const void* v_in, void* v_out, int32_t nrhs, void* stream);

/* Smoother on D_l psi_i ~ 0 (Sec. 2, Eq. 1 with D -> D_l): the minimal
 * residual recurrence of mg_smooth_testvecs, mr_iters iterations, one step
 * length per vector, then every vector to unit 2-norm.  In: X, Y, psi0.
 * Out: psi (may alias psi0).  ws: mg_coarse_workspace_size(prob,
 * MG_CALL_SMOOTH) bytes.  FP32 arithmetic, FP64 sums of the inner products. */
mg_status mg_coarse_smooth_testvecs(const mg_coarse_problem* prob, const void* X, const void* Y,
                                    const void* psi0, void* psi, void* ws, size_t ws_bytes,
                                    void* stream);

/* Chiral split by sigma_3 and rank-k truncation (Sec. 2 Eq. 2, Sec. 3 Eq. 4)
 * of the nc*nb x m matrices Psi^(alpha)(Lambda_j) (rows: site, component of
 * chirality alpha), by the kernels of mg_chiral_truncate.  In: psi.  Out:
 * Uk, sigma, optional coarse_tv ([nblk][2][k][m], NULL to skip), blk_flags
 * (as mg_chiral_truncate).  ws: mg_coarse_workspace_size(prob,
 * MG_CALL_TRUNCATE) bytes. */
mg_status mg_coarse_chiral_truncate(const mg_coarse_problem* prob, const void* psi, void* Uk,
                                    double* sigma, void* coarse_tv, int32_t* blk_flags, void* ws,
                                    size_t ws_bytes, void* stream);

/* Prolongator of level l (Sec. 3, Eq. 5 with gamma_5 -> sigma_3):
 * P_{alpha i j}(x) = u_i^(alpha)(x) for x in Lambda_j.  In: Uk.  Out: P. */
mg_status mg_coarse_build_prolongator(const mg_coarse_problem* prob, const void* Uk, void* P,
                                      void* stream);

/* D_{l+1} = P^dag D_l P (Sec. 2, Eq. 3), term by term: for every site x of
 * block j, P(x)^dag X(x) P(x) and every hop P(x)^dag Y_d(x) P(x +- mu_d) go to
 * X2(j), except a hop from a site on the block's +mu (-mu) face in direction
 * +mu (-mu), which goes to Y2_d(j).  Every direction is computed (no symmetry
 * is assumed of D_l).  In: X, Y, P.  Out: X2, Y2.  FP32 arithmetic. */
mg_status mg_coarse_coarsen(const mg_coarse_problem* prob, const void* X, const void* Y,
                            const void* P, void* X2, void* Y2, void* stream);

/* ------------------------------------------------------------------------
 * The solve the setup serves (Sec. 2: the multigrid hierarchy used in a
 * K-cycle as the preconditioner of a flexible outer Krylov solver, FGMRES).
 * A hierarchy is the output of the setup calls above: the fine operator
 * (fine, U, C), its prolongator P and coarse operator X, Y (mg_build_prolongator,
 * mg_coarsen), and for three levels the second level's P2, X2, Y2
 * (mg_coarse_build_prolongator, mg_coarse_coarsen with problem `second`).
 * Preconditioner, the K-cycle at level l applied to r:
 *   x = nu_pre MR steps on A_l x = r from 0;  s = r - A_l x;
 *   e = approximate solve of A_{l+1} e = P_l^dag s: coarsest_iters GMRES steps
 *       on the coarsest level, else kcycle_iters FGMRES steps preconditioned by
 *       the K-cycle at level l+1;
 *   x += P_l e;  x += nu_post MR steps on A_l y = r - A_l x.
 * n_levels = 1 is restarted GMRES on D alone (no preconditioner).
 * Arnoldi uses classical Gram-Schmidt twice; all vectors are complex64, the
 * Krylov bookkeeping is FP64 on the host.
 * ------------------------------------------------------------------------ */
typedef struct {
  mg_problem fine;          /* fine operator and first aggregation; k = k1 (n_vec is not read) */
  const void* U;
  const void* C;            /* NULL for pure Wilson */
  const void* P;            /* [V][2][2][3][k1] */
  const void* X;            /* [nc][2k1][2k1] */
  const void* Y;            /* [nc][8][2k1][2k1] */
  int32_t n_levels;         /* 1, 2 or 3 */
  mg_coarse_problem second; /* n_levels = 3: dims = the fine coarse lattice, nc = k1, block, k = k2 */
  const void* P2;           /* [nc][2][k1][k2] */
  const void* X2;           /* [nc2][2k2][2k2] */
  const void* Y2;           /* [nc2][8][2k2][2k2] */
  int32_t nu_pre, nu_post;  /* MR steps before / after the coarse correction, >= 0 */
  int32_t kcycle_iters;     /* FGMRES steps on each intermediate level (1..64) */
  int32_t coarsest_iters;   /* GMRES steps on the coarsest level (1..64) */
} mg_hierarchy;

/* Scratch bytes of mg_solve for nrhs systems and an outer restart length
 * (0 for invalid arguments; mg_last_error() says why). */
size_t mg_solve_workspace_size(const mg_hierarchy* h, int32_t nrhs, int32_t restart);

/* Solves D x_c = b_c for nrhs independent systems (nrhs = 4, 8, 16, 32 or 64),
 * b and x in the spinor layout [V][4][3][nrhs] (x must not alias b), from
 * x = 0, by FGMRES(restart) preconditioned by the K-cycle, until every
 * system's least-squares residual estimate is <= tol |b_c| or max_iters outer
 * steps are done.  Out (host): *iters = outer steps taken; relres[nrhs] = the
 * true |b_c - D x_c| / |b_c| at the end (FP32 residual, FP64 norms).
 * ws: mg_solve_workspace_size(h, nrhs, restart) bytes, 256-byte aligned.
 * Synchronous: the call returns when the solve is done.  It synchronises
 * `stream` once per outer step (the convergence test) and once per coarse
 * Krylov cycle (its least-squares solve); the step lengths and Gram-Schmidt
 * coefficients are computed on the device.  A timeout of an operator's
 * staged input (see mg_sync_status) is returned as MG_ERR_TIMEOUT. */
mg_status mg_solve(const mg_hierarchy* h, const void* b, void* x, int32_t nrhs, double tol,
                   int32_t restart, int32_t max_iters, int32_t* iters, double* relres, void* ws,
                   size_t ws_bytes, void* stream);

/* mg_chiral_truncate for callers that cannot allocate device memory (the
 * paper has no counterpart; this is a service of this library).  A host
 * application whose device memory is owned by its own pool allocator, or a
 * solver loop that must not stall the device with cudaMalloc/cudaFree (both
 * may synchronise the device), passes only inputs and outputs here: the
 * scratch lives in a 64 MiB array compiled into the library, reserved on
 * every GPU that loads it until the process exits.
 * Same inputs, outputs and results as mg_chiral_truncate.  A problem whose
 * scratch need (mg_workspace_size(prob, MG_CALL_TRUNCATE)) exceeds 64 MiB is
 * rejected with MG_ERR_INVALID and a message.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is kept per device together with the id of the CUDA context it
 * belongs to; the first call from a new context on that device (after a
 * cudaDeviceReset, for instance) looks it up again, so make that call
 * outside a capture too.  All calls
 * share the one array and leave their data in it (nothing in it needs to
 * start at zero); calls that overlap on the GPU race on it, so serialise
 * them (one stream, or synchronise between calls).  It allocates nothing. */
mg_status mg_chiral_truncate_static(const mg_problem* prob, const void* psi, void* Uk,
                                    double* sigma, void* coarse_tv, int32_t* blk_flags,
                                    void* stream);

/* Random starting vectors for the smoother (the "m random initial guesses" of
 * Sec. 2, Eq. 1), for callers that do not bring their own (a setup server,
 * say): psi0 [V][4][3][n_vec] complex64 on the device, element e (flat index)
 * = normal 2e + i normal 2e+1 of the counter-based generator of prob->seed
 * (SplitMix64 of counter + key(seed, stream 2), 53-bit uniforms, Box-Muller's
 * cosine branch), the definition the library's tests draw their inputs from;
 * uniforms bit-identical, the transcendental functions in FP32 (within a
 * few 1e-6 of the FP64 definition).  Only dims and n_vec of prob are used besides the seed.  Out:
 * psi0 (caller-owned device memory).  Asynchronous on `stream`. */
mg_status mg_random_starts(const mg_problem* prob, void* psi0, void* stream);

/* Random SU(3) gauge links for synthetic inputs (input synthesis, not part of
 * the method; the ensembles of Sec. 4 are not available): U [V][4][3][3]
 * complex64, U_mu(x) = exp(i eps H), H = sum_a h_a lambda_a / 2, h_a the
 * normals 8j .. 8j+7 (j = 4x + mu) of stream 1 of the counter-based generator
 * of prob->seed, lambda_a the Gell-Mann matrices; the exponential by its
 * Taylor series in FP32 (within a few 1e-7 of the exact exponential).
 * 0 <= eps <= 1, else MG_ERR_INVALID.  Out: U
 * (caller-owned device memory).  Asynchronous on `stream`. */
mg_status mg_random_links(const mg_problem* prob, double eps, void* U, void* stream);

/* Failure-detection self-test (no counterpart in the paper).  Enqueues on
 * `stream` one kernel whose single thread waits on a shared-memory mbarrier
 * that nothing ever arrives at, giving up after `polls` polls
 * (1 <= polls <= 1048576, the limit the library's own waits use), exactly as
 * the smoother's and the tensor-core kernels' bounded waits give up; it then
 * records a timeout in the device status word.  No copy or matrix multiply
 * is in flight when it gives up, so the device and the library stay usable:
 * the next mg_sync_status(stream) returns MG_ERR_TIMEOUT, the one after that
 * MG_OK.  Errors: MG_ERR_INVALID for polls out of range. */
mg_status mg_selftest_timeout(int32_t polls, void* stream);

/* Per-kernel timing (measurement aid; no counterpart in the paper).  While
 * enabled, every kernel the library launches is bracketed by two CUDA events
 * recorded on the launching stream.  mg_timing_read waits for the recorded
 * events, writes up to `max` entries (one per kernel kind: name, number of
 * launches, summed milliseconds) accumulated since the previous read, resets
 * the accumulators and returns the number of entries written (or -1 on a CUDA
 * error).  Events come from a pool owned by the library (CUDA events, not
 * device memory). */
typedef struct {
  char name[48];
  int64_t launches;
  double ms;
} mg_timing_entry;

mg_status mg_timing_enable(int on);
int mg_timing_read(mg_timing_entry* out, int max);

/* ------------------------------------------------------------------------
 * Batched setup (not in the paper: many independent levels, e.g. hierarchies
 * of lattices of uneven volume, built together).  One descriptor per level
 * holds that level's problem and arrays exactly as the single calls take them
 * (ws_smooth / ws_trunc: mg_workspace_size(prob, MG_CALL_SMOOTH / _TRUNCATE)
 * bytes; the arrays of different levels must not overlap).
 * mg_batch_create validates the descriptors, tunes the smoother's slab width
 * once per distinct shape by timing both variants on the level's own buffers
 * (it runs the smoother, so psi and ws_smooth are overwritten), and captures
 * every level's four calls (smoother, truncation, prolongator, coarsening;
 * no coarse test vectors) into one CUDA graph that forks over n_streams
 * streams from the launching stream and joins back; n_streams <= 0 tunes the
 * stream count (1, 2, 4, 8) as well.  It synchronises `stream`.
 * mg_batch_launch enqueues the whole batch on `stream` (one graph launch);
 * the descriptors' arrays must stay valid while the batch exists.
 * mg_batch_destroy releases the graph.  Errors: MG_ERR_INVALID for a bad
 * descriptor (mg_last_error() names the level), MG_ERR_CUDA otherwise.
 * ------------------------------------------------------------------------ */
typedef struct {
  mg_problem prob;
  const void* U;
  const void* C;        /* NULL for pure Wilson */
  const void* psi0;
  void* psi;
  void* Uk;
  double* sigma;
  int32_t* blk_flags;
  void* P;
  void* X;
  void* Y;
  void* ws_smooth;
  size_t ws_smooth_bytes;
  void* ws_trunc;
  size_t ws_trunc_bytes;
} mg_level_desc;

typedef struct mg_batch mg_batch;

mg_status mg_batch_create(const mg_level_desc* levels, int n, int n_streams, void* stream,
                          mg_batch** out);
mg_status mg_batch_launch(mg_batch* batch, void* stream);
/* Number of streams the batch's graph forks over (0 for NULL). */
int mg_batch_streams(const mg_batch* batch);
void mg_batch_destroy(mg_batch* batch);
/* Slab width (pairs of right-hand sides per CTA, 2 or 4) the smoother uses for
 * this problem's shape: the tuned value if a batch tuned it, else the default;
 * -1 for an invalid problem. */
int mg_tuned_pairs(const mg_problem* prob);

/* Device status of the work enqueued so far on `stream` (not in the paper;
 * the failure-detection side of the library).  Waits for the stream, then
 * reads and clears the library's device status word.  Returns MG_OK, or
 * MG_ERR_TIMEOUT if a smoother or operator pass since the previous call gave
 * up waiting (after a bounded number of polls, about a second) for input it
 * had staged into shared memory, or a tensor-core Gram of the mixed-precision
 * truncation gave up waiting for its matrix multiplies: that kernel stopped
 * early and its outputs are not valid.  MG_ERR_CUDA if the stream reports a CUDA error.  The status
 * word is shared by every stream of the process on the current device. */
mg_status mg_sync_status(void* stream);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* mg_last_error(void);

/* Library version string. */
const char* mg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MG_H_ */
