"""FP64 CPU oracle of the second level of the setup (the recursion of Sec. 2).

TEST INFRASTRUCTURE ONLY (the same rule as the rest of ``oracle``): only
``tests/`` and ``bench.py``'s CPU legs may import it.

The level-1 coarse operator D_c (X, Y on the coarse lattice, 2k1 components
per site) takes the place of the fine operator; its chirality is sigma_3, so
chirality alpha is the block of components alpha*k1 .. alpha*k1 + k1 - 1 of a
coarse site.  Each function repeats the corresponding level-1 step with that
substitution, in plain numpy over the level-1 oracle's coarse apply and block
SVD:

  mr(...)               smoother on D_c psi = 0 (Eq. 1 with D -> D_c)
  chiral_truncate(...)  sigma_3 split + per-block SVD, rank-k2 truncation (Eqs. 2, 4)
  prolongator(...)      P2 from the truncated left singular vectors (Eq. 5)
  coarsen(...)          D_cc = P2^dag D_c P2 (Eq. 3), term by term, as X2, Y2

Layouts: vectors [nc][2 k1][m] (the coarse-vector layout of mg_coarse_apply);
U_k [nblk2][2][|Lambda2|][k1][k2]; P2 [nc][2][k1][k2]; X2 [nc2][2 k2][2 k2],
Y2 [nc2][8][2 k2][2 k2] with directions +x, +y, +z, +t, -x, -y, -z, -t.
"""
from __future__ import annotations

import numpy as np

from . import coarse_apply, coarse_dims, svd


def _vol(d):
    return int(d[0]) * int(d[1]) * int(d[2]) * int(d[3])


def _coords(dims, s):
    c = []
    for L in dims:
        c.append(s % L)
        s = s // L
    return c


def _index(dims, c):
    return c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))


def block_sites(dims, block, j):
    """Sites of block j in the block's local lexicographic order."""
    Lc = coarse_dims(dims, block)
    jc = _coords(Lc, j)
    loc = np.arange(_vol(block))
    lc = _coords(block, loc)
    return _index(dims, [jc[i] * block[i] + lc[i] for i in range(4)])


def mr(cdims, X, Y, psi0, niter, return_history: bool = False):
    """Minimal residual on D_c psi = 0, one step length per vector, then every
    vector to unit 2-norm:  r = -D_c psi;  N times { w = D_c r;
    a = <w, r> / <w, w>;  psi += a r;  r -= a w }.
    return_history: also the residual norms |r_t| per vector (t = 0..N) and
    the overlaps |<w_t, r_{t+1}>| / (|w_t| |r_{t+1}|)."""
    A = lambda v: coarse_apply(cdims, X, Y, v)  # noqa: E731
    dot = lambda a, b: np.einsum("xai,xai->i", a.conj(), b)  # noqa: E731
    psi = np.array(psi0, dtype=np.complex128)
    r = -A(psi)
    rn, ov = [np.sqrt(dot(r, r).real)], []
    for _ in range(niter):
        w = A(r)
        ww = dot(w, w).real
        a = np.where(ww > 0, dot(w, r) / np.where(ww > 0, ww, 1.0), 0.0)
        psi = psi + a * r
        r = r - a * w
        rn.append(np.sqrt(dot(r, r).real))
        ov.append(np.abs(dot(w, r)) / np.maximum(np.sqrt(ww) * rn[-1], 1e-300))
    nrm = np.sqrt(dot(psi, psi).real)
    out = psi / np.where(nrm > 0, nrm, 1.0)
    if return_history:
        return out, np.array(rn), np.array(ov)
    return out


def block_matrix(cdims, block, k1, psi, j, alpha):
    """Rows of chirality alpha of block j: A[loc * k1 + r][i] = psi[x(loc)][alpha k1 + r][i]."""
    xs = block_sites(cdims, block, j)
    return psi[xs, alpha * k1:(alpha + 1) * k1, :].reshape(len(xs) * k1, psi.shape[-1])


def chiral_truncate(cdims, block, k1, psi, k2):
    """sigma_3 split + per-block thin SVD (the level-1 oracle's Householder QR +
    one-sided Jacobi), rank-k2 truncation.  Returns Uk[nblk2][2][nb2][k1][k2]
    and sigma[nblk2][2][m] (all m values, descending)."""
    psi = np.asarray(psi, dtype=np.complex128)
    m = psi.shape[-1]
    nb = _vol(block)
    nblk = _vol(coarse_dims(cdims, block))
    if nb * k1 < m:
        raise ValueError("block too small: k1 |Lambda2| < m")
    Uk = np.empty((nblk, 2, nb, k1, k2), dtype=np.complex128)
    sig = np.empty((nblk, 2, m))
    for j in range(nblk):
        for al in range(2):
            s, U, _ = svd(block_matrix(cdims, block, k1, psi, j, al))
            Uk[j, al] = U[:, :k2].reshape(nb, k1, k2)
            sig[j, al] = s
    return Uk, sig


def prolongator(cdims, block, Uk):
    """Site-major P2[nc][2][k1][k2] from block-major Uk (Eq. 5)."""
    nblk, _, nb, k1, k2 = Uk.shape
    P = np.empty((_vol(cdims), 2, k1, k2), dtype=np.complex128)
    for j in range(nblk):
        P[block_sites(cdims, block, j)] = Uk[j].transpose(1, 0, 2, 3)
    return P


def _p_full(P, x):
    """The 2k1 x 2k2 block-diagonal matrix P2(x) (chirality blocks)."""
    _, _, k1, k2 = P.shape
    M = np.zeros((2 * k1, 2 * k2), dtype=np.complex128)
    M[:k1, :k2] = P[x, 0]
    M[k1:, k2:] = P[x, 1]
    return M


def coarsen(cdims, block, X, Y, P):
    """D_cc = P2^dag D_c P2 on the level-2 lattice, term by term: for every
    level-1 site x of block j, the diagonal term P2(x)^dag X(x) P2(x) and every
    hop P2(x)^dag Y_d(x) P2(x +- mu) go to X2(j), except hops from a site on the
    block's +mu (-mu) face in direction +mu (-mu), which go to Y2_d(j)."""
    k2 = P.shape[-1]
    c2 = coarse_dims(cdims, block)
    nc2 = _vol(c2)
    X2 = np.zeros((nc2, 2 * k2, 2 * k2), dtype=np.complex128)
    Y2 = np.zeros((nc2, 8, 2 * k2, 2 * k2), dtype=np.complex128)
    for x in range(_vol(cdims)):
        c = _coords(cdims, x)
        j = _index(c2, [c[i] // block[i] for i in range(4)])
        Px = _p_full(P, x)
        X2[j] += Px.conj().T @ X[x] @ Px
        for d in range(8):
            mu, s = d % 4, (1 if d < 4 else -1)
            cy = list(c)
            cy[mu] = (cy[mu] + s) % cdims[mu]
            y = _index(cdims, cy)
            term = Px.conj().T @ Y[x, d] @ _p_full(P, y)
            lmu = c[mu] % block[mu]
            if (s > 0 and lmu == block[mu] - 1) or (s < 0 and lmu == 0):
                Y2[j, d] += term
            else:
                X2[j] += term
    return X2, Y2


def restrict(cdims, block, P, z):
    """P2^dag z for z[nc][2k1] -> [nc2][2k2]."""
    nc2 = _vol(coarse_dims(cdims, block))
    k1, k2 = P.shape[2], P.shape[3]
    out = np.zeros((nc2, 2 * k2), dtype=np.complex128)
    c2 = coarse_dims(cdims, block)
    for x in range(_vol(cdims)):
        c = _coords(cdims, x)
        j = _index(c2, [c[i] // block[i] for i in range(4)])
        out[j] += _p_full(P, x).conj().T @ z[x]
    return out


def prolong(cdims, block, P, v):
    """P2 v for v[nc2][2k2] -> [nc][2k1]."""
    k1 = P.shape[2]
    c2 = coarse_dims(cdims, block)
    out = np.zeros((_vol(cdims), 2 * k1), dtype=np.complex128)
    for x in range(_vol(cdims)):
        c = _coords(cdims, x)
        j = _index(c2, [c[i] // block[i] for i in range(4)])
        out[x] = _p_full(P, x) @ v[j]
    return out
