"""Seeded synthetic inputs for the chiral rank-k multigrid setup.

This module is the only code shared by the FP64 oracle side (tests) and the
CUDA side (tests, bench, server).  It draws random numbers and builds the
inputs the method starts from; it holds none of the method's arithmetic
(no Dirac operator, no smoother, no SVD, no coarsening).

Random numbers (counter based, so any element can be drawn independently):
  * SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014) hashes (seed, stream, counter) to 64 bits.
  * The top 53 bits give a uniform double in (0, 1).
  * Box-Muller (Box & Muller, Ann. Math. Stat. 29, 1958) turns the uniform
    pair with counters (2n, 2n+1) into normal number n (cosine branch).

Inputs (the paper's ensembles are not available; these are stand-ins with
the same shapes, see Sec. 4 of the paper for the lattices they mimic):
  * gauge links U_mu(x) = exp(i eps H), H = sum_a h_a lambda_a / 2 with
    h_a ~ N(0,1) i.i.d. and lambda_a the Gell-Mann matrices (traceless
    Hermitian H, so U is in SU(3));
  * complex Gaussian test-vector starts psi0 (the "m random initial guesses"
    of Eq. (1) of the paper);
  * random SU(3) gauge transformations (for covariance tests);
  * random nearest-neighbour stencils with 2 nc components per site and the
    structure of a coarse operator (stand-ins for the operator of a level
    l >= 1), and complex Gaussian coarse vectors.

Layouts (lexicographic site index s = x + Lx*(y + Ly*(z + Lz*t))):
  U    complex128 [V][4 mu][3][3]          (U_mu(x) links x -> x + mu)
  psi  complex128 [V][4 spin][3 colour][m] (right-hand sides fastest)
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids: independent sub-sequences per input kind
STREAM_GAUGE = 1
STREAM_PSI0 = 2
STREAM_GAUGE_TRANSFORM = 3
STREAM_COARSE_VEC = 4
STREAM_MISC = 5
STREAM_STENCIL = 6


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied to x + golden gamma (uint64, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _GOLDEN) & _MASK
        z = ((z ^ (z >> np.uint64(30))) * _M1) & _MASK
        z = ((z ^ (z >> np.uint64(27))) * _M2) & _MASK
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """64-bit key of the (seed, stream) sub-sequence."""
    s = splitmix64(np.array([stream], dtype=np.uint64))[0]
    return splitmix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ s],
                               dtype=np.uint64))[0]


def uniforms(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in (0, 1) for counters start .. start+count-1."""
    key = stream_key(seed, stream)
    ctr = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        bits = splitmix64((ctr + key) & _MASK)
    return ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Standard normal doubles n_start .. n_{start+count-1} (Box-Muller, cosine branch)."""
    u = uniforms(seed, stream, 2 * start, 2 * count).reshape(count, 2)
    return np.sqrt(-2.0 * np.log(u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


def _expi_hermitian(H: np.ndarray, eps) -> np.ndarray:
    """exp(i eps H) for a batch of 3x3 Hermitian H, via the eigendecomposition."""
    w, Q = np.linalg.eigh(H)
    ph = np.exp(1j * np.asarray(eps)[..., None] * w)
    return np.einsum("nij,nj,nkj->nik", Q, ph, Q.conj())


def random_su3(seed: int, stream: int, n: int, eps, start: int = 0,
               chunk: int = 1 << 20) -> np.ndarray:
    """n SU(3) matrices exp(i eps H_j), H_j = sum_a h_{j,a} lambda_a / 2.

    Matrix j uses normals 8*(start+j) .. 8*(start+j)+7 of the stream.  eps is a
    scalar or an array of length n.
    """
    lam = gell_mann() / 2.0
    out = np.empty((n, 3, 3), dtype=np.complex128)
    eps_arr = np.broadcast_to(np.asarray(eps, dtype=np.float64), (n,))
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        h = normals(seed, stream, 8 * (start + lo), 8 * (hi - lo)).reshape(hi - lo, 8)
        H = np.einsum("na,aij->nij", h, lam)
        out[lo:hi] = _expi_hermitian(H, eps_arr[lo:hi])
    return out


def gauge_field(dims, eps: float, seed: int, threads: int = 1) -> np.ndarray:
    """Random SU(3) gauge field U[V][4][3][3] (complex128), U_mu(x) = exp(i eps H).
    threads > 1 draws contiguous chunks of links on host threads (the same
    numbers: link j always uses normals 8j .. 8j+7)."""
    V = volume(dims)
    n = 4 * V
    if threads <= 1 or n < 65536:
        return random_su3(seed, STREAM_GAUGE, n, eps).reshape(V, 4, 3, 3)
    import concurrent.futures as cf
    step = -(-n // threads)
    parts = [(lo, min(n, lo + step)) for lo in range(0, n, step)]
    with cf.ThreadPoolExecutor(threads) as ex:
        out = list(ex.map(lambda r: random_su3(seed, STREAM_GAUGE, r[1] - r[0], eps, start=r[0]),
                          parts))
    return np.concatenate(out).reshape(V, 4, 3, 3)


def unit_gauge_field(dims) -> np.ndarray:
    """Free field: every link is the identity."""
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1.0
    return U


def gauge_transform(dims, seed: int, eps: float = 1.0) -> np.ndarray:
    """Random site-local SU(3) matrices G[V][3][3]."""
    return random_su3(seed, STREAM_GAUGE_TRANSFORM, volume(dims), eps)


def psi0(dims, m: int, seed: int, stream: int = STREAM_PSI0, threads: int = 1) -> np.ndarray:
    """m complex Gaussian vectors, layout [V][4][3][m]; re and im are N(0,1).
    threads > 1 draws site chunks on host threads (the same numbers)."""
    V = volume(dims)
    if threads > 1 and V >= 4096:
        import concurrent.futures as cf
        step = -(-V // threads)
        parts = [(lo, min(V, lo + step)) for lo in range(0, V, step)]
        with cf.ThreadPoolExecutor(threads) as ex:
            out = list(ex.map(lambda r: psi0_sites(dims, m, seed, r[0], r[1], stream), parts))
        return np.concatenate(out)
    n = V * 12 * m
    g = normals(seed, stream, 0, 2 * n)
    return (g[0::2] + 1j * g[1::2]).reshape(V, 4, 3, m)


def psi0_sites(dims, m: int, seed: int, lo: int, hi: int,
               stream: int = STREAM_PSI0) -> np.ndarray:
    """Sites lo .. hi-1 of psi0(dims, m, seed): layout [hi-lo][4][3][m], the
    same numbers (element n of the full array uses normals 2n and 2n+1), for
    lattices whose full start set is too large to draw at once."""
    per = 12 * m
    g = normals(seed, stream, 2 * lo * per, 2 * (hi - lo) * per)
    return (g[0::2] + 1j * g[1::2]).reshape(hi - lo, 4, 3, m)


def psi0_columns(dims, m: int, seed: int, cols, stream: int = STREAM_PSI0) -> np.ndarray:
    """Columns `cols` of psi0(dims, m, seed): layout [V][4][3][len(cols)]."""
    V = volume(dims)
    cols = np.asarray(cols, dtype=np.int64)
    n = (np.arange(V * 12, dtype=np.int64)[:, None] * m + cols[None, :]).ravel()
    key = stream_key(seed, stream)
    ctr = np.stack([4 * n, 4 * n + 1, 4 * n + 2, 4 * n + 3], axis=1).astype(np.uint64)
    with np.errstate(over="ignore"):
        bits = splitmix64((ctr + key) & _MASK)
    u = ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    re = np.sqrt(-2.0 * np.log(u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])
    im = np.sqrt(-2.0 * np.log(u[:, 2])) * np.cos(2.0 * np.pi * u[:, 3])
    return (re + 1j * im).reshape(V, 4, 3, len(cols))


def coarse_vectors(n_coarse: int, two_k: int, nrhs: int, seed: int) -> np.ndarray:
    """Complex Gaussian coarse vectors, layout [nc][2k][nrhs]."""
    n = n_coarse * two_k * nrhs
    g = normals(seed, STREAM_COARSE_VEC, 0, 2 * n)
    return (g[0::2] + 1j * g[1::2]).reshape(n_coarse, two_k, nrhs)


def round_to_c64(a: np.ndarray) -> np.ndarray:
    """Round complex128 values to complex64 and back, so both sides see the same numbers."""
    return np.asarray(a, dtype=np.complex64).astype(np.complex128)


def batch_workload(seed: int = 30, m0_table=None):
    """The 24-hierarchy batch: 8 each of 8^4, 12^3x24 and 16^3x32, with m' drawn
    from {32, 48, 64}, k from {16, 24}, aggregates 2^4 or 4^4 and the gauge
    spread eps uniform in [0.15, 0.35], all from the batch seed (stream MISC,
    four uniforms per hierarchy).  Hierarchy i uses gauge and start seed
    300 + i.  m0 (if a table {eps: m0} is given) is the entry of the nearest
    tabulated eps; 20 smoother iterations.  Returns a list of dicts."""
    vols = [[8, 8, 8, 8]] * 8 + [[12, 12, 12, 24]] * 8 + [[16, 16, 16, 32]] * 8
    u = uniforms(seed, STREAM_MISC, 0, 4 * len(vols)).reshape(len(vols), 4)
    out = []
    for i, d in enumerate(vols):
        m = (32, 48, 64)[min(2, int(u[i, 0] * 3))]
        k = (16, 24)[min(1, int(u[i, 1] * 2))]
        b = 2 if u[i, 2] < 0.5 else 4
        eps = 0.15 + 0.2 * u[i, 3]
        m0 = None
        if m0_table:
            m0 = m0_table[min(m0_table, key=lambda e: abs(e - eps))]
        out.append(dict(dims=list(d), block=[b] * 4, m=m, k=k, eps=float(eps), m0=m0, N=20,
                        gauge_seed=300 + i, psi_seed=300 + i))
    return out


def stencil_operator(cdims, nc: int, seed: int, diag: float = 3.0, hop: float = 0.3,
                     threads: int = 1):
    """A random nearest-neighbour operator on the periodic lattice cdims with
    n = 2 nc components per site, in the coarse-operator layout X [V][n][n],
    Y [V][8][n][n] (d = 0..3 hop to x + mu_d, 4..7 to x - mu_{d-4}).  It has
    the symmetry of a coarse Wilson operator under s3 = diag(1_nc, -1_nc):
      X = S + s3 S^dag s3,  S = Z_0 + diag 1,   Y_mu(x) = hop Z_{1+mu}(x),
      Y_{4+mu}(x + mu) = s3 Y_mu(x)^dag s3,
    with Z_i(x) complex Gaussian n x n matrices drawn from stream STENCIL
    (site by site, so any chunk of sites can be drawn on its own).
    complex128."""
    V = volume(cdims)
    n = 2 * nc
    per = 5 * n * n

    # one complex number per pair of normals: site x takes normals
    # 2 x per .. 2 (x + 1) per - 1, so a chunk of sites is drawn on its own
    def site_block(lo, hi):
        g = normals(seed, STREAM_STENCIL, 2 * lo * per, 2 * (hi - lo) * per)
        return (g[0::2] + 1j * g[1::2]).reshape(hi - lo, 5, n, n)

    step = 256
    chunks = [(lo, min(V, lo + step)) for lo in range(0, V, step)]
    if threads > 1:
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(lambda c: site_block(*c), chunks))
    else:
        parts = [site_block(*c) for c in chunks]
    Z = np.concatenate(parts, axis=0)
    s3 = np.r_[np.ones(nc), -np.ones(nc)]
    S = Z[:, 0] + diag * np.eye(n)
    X = S + s3[:, None] * S.conj().transpose(0, 2, 1) * s3[None, :]
    Y = np.empty((V, 8, n, n), dtype=np.complex128)
    s = np.arange(V)
    c = []
    t = s.copy()
    for L in cdims:
        c.append(t % L)
        t = t // L
    for mu in range(4):
        Y[:, mu] = hop * Z[:, 1 + mu]
        cf_ = [a.copy() for a in c]
        cf_[mu] = (cf_[mu] + 1) % cdims[mu]
        fwd = cf_[0] + cdims[0] * (cf_[1] + cdims[1] * (cf_[2] + cdims[2] * cf_[3]))
        Y[fwd, 4 + mu] = s3[:, None] * Y[:, mu].conj().transpose(0, 2, 1) * s3[None, :]
    return X, Y
