"""Pins of the oracle's chiral split and rank-k truncation (Sec. 2 Eq. 2; Sec. 3
Eq. 4 of the paper): the best rank-k approximation (Eckart-Young), orthonormal
left singular vectors, exact reconstruction, a matrix with a prescribed
spectrum, a library SVD on small blocks, and the k = m' case that reduces to
the conventional per-block orthonormalisation of Sec. 2."""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from conftest import coords, lex, vol


def _rand(K, n, seed):
    g = G.normals(seed, G.STREAM_MISC, 0, 2 * K * n)
    return (g[0::2] + 1j * g[1::2]).reshape(K, n)


@pytest.mark.parametrize("K,n", [(96, 8), (300, 24), (48, 48)])
def test_svd_factorisation(K, n):
    A = _rand(K, n, K + n)
    s, U, V = O.svd(A)
    assert np.all(np.diff(s) <= 0)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(U @ np.diag(s) @ V.conj().T, A, atol=1e-12)
    # library cross-check of the spectrum
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12)


def test_prescribed_spectrum():
    """A = Q_1 diag(s) Q_2^dagger with unitary Q_1, Q_2 returns exactly s."""
    K, n = 200, 16
    Q1, _ = np.linalg.qr(_rand(K, n, 1))
    Q2, _ = np.linalg.qr(_rand(n, n, 2))
    s_ref = np.logspace(0, -6, n)
    s, U, _ = O.svd(Q1 @ np.diag(s_ref) @ Q2.conj().T)
    np.testing.assert_allclose(s, s_ref, rtol=1e-9)
    # each left singular vector is the prescribed one up to a phase
    np.testing.assert_allclose(np.abs(np.sum(U.conj() * Q1, axis=0)), 1.0, atol=1e-9)


@pytest.mark.parametrize("k", [1, 5, 12])
def test_eckart_young(k):
    """|A - U_k U_k^dag A|_F^2 = sum_{i>k} sigma_i^2: U_k spans the best rank-k fit."""
    A = _rand(120, 20, 7)
    s, U, _ = O.svd(A)
    Uk = U[:, :k]
    resid = np.linalg.norm(A - Uk @ (Uk.conj().T @ A)) ** 2
    np.testing.assert_allclose(resid, np.sum(s[k:] ** 2), rtol=1e-12)
    # and no random rank-k subspace does better
    Qr, _ = np.linalg.qr(_rand(120, k, 8))
    assert np.linalg.norm(A - Qr @ (Qr.conj().T @ A)) ** 2 >= resid


def test_rank_deficient_block():
    """A block of rank r < n keeps a valid orthonormal basis of its range."""
    A = _rand(60, 4, 9) @ _rand(4, 10, 10)
    s, U, _ = O.svd(A)
    assert s[4] < 1e-12 * s[0]
    Ur = U[:, :4]
    np.testing.assert_allclose(Ur.conj().T @ Ur, np.eye(4), atol=1e-13)
    np.testing.assert_allclose(Ur @ (Ur.conj().T @ A), A, atol=1e-12)


def _gather_block(dims, block, psi, j, al):
    """The 6|Lambda| x m block of Eq. (2) gathered by hand from the site layout."""
    Lc = [dims[i] // block[i] for i in range(4)]
    rows = []
    nb = vol(block)
    for loc in range(nb):
        xl = coords(block, loc)
        xc = coords(Lc, j)
        s = lex(dims, [xc[i] * block[i] + xl[i] for i in range(4)])
        for sp in range(2):
            for c in range(3):
                rows.append(psi[s, 2 * al + sp, c, :])
    return np.array(rows)


def test_chiral_truncate_blocks_and_k_equals_m():
    """Per block and chirality: the retained U_k spans the leading singular space
    of the hand-gathered block (library SVD), the singular values agree, and
    with k = m' the projector U U^dag is the orthogonal projector onto the range
    of the block (the conventional orthonormalisation of Sec. 2)."""
    dims, block, m = [4, 4, 2, 2], [2, 2, 2, 2], 8
    psi = G.psi0(dims, m, 21)
    for k in (3, m):
        Uk, sig = O.chiral_truncate(dims, block, psi, k)
        for j in (0, 3):
            for al in (0, 1):
                A = _gather_block(dims, block, psi, j, al)
                np.testing.assert_allclose(sig[j, al], np.linalg.svd(A, compute_uv=False),
                                           rtol=1e-12)
                U = Uk[j, al].reshape(-1, k)
                Ul, sl, _ = np.linalg.svd(A, full_matrices=False)
                np.testing.assert_allclose(U @ U.conj().T, Ul[:, :k] @ Ul[:, :k].conj().T,
                                           atol=1e-12)
                if k == m:
                    Q, _ = np.linalg.qr(A)
                    np.testing.assert_allclose(U @ U.conj().T, Q @ Q.conj().T, atol=1e-12)


def test_coarse_test_vectors():
    """Sigma_k V_k^dag is the coarse representation: U_k (Sigma_k V_k^dag) is the
    best rank-k approximation of the block (Eq. 4)."""
    dims, block, m, k = [4, 2, 2, 2], [2, 2, 2, 2], 6, 4
    psi = G.psi0(dims, m, 22)
    Uk, sig, ctv = O.chiral_truncate(dims, block, psi, k, want_coarse_tv=True)
    A = _gather_block(dims, block, psi, 1, 1)
    approx = Uk[1, 1].reshape(-1, k) @ ctv[1, 1]
    np.testing.assert_allclose(np.linalg.norm(A - approx) ** 2, np.sum(sig[1, 1, k:] ** 2),
                               rtol=1e-11)
