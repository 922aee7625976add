"""Pins of the second-level oracle (oracle.level2) on a random coarse operator
with the structure of D_c (sigma_3-hermitian: X = S + sigma_3 S^dag sigma_3,
Y_{-mu}(x + mu) = sigma_3 Y_{+mu}(x)^dag sigma_3), independent of the
functions they check:

  * D_cc = P2^dag D_c P2 assembled term by term equals the matrix-free product
    restrict(D_c(prolong(v))) (brute force), and is sigma_3-hermitian;
  * P2^dag P2 = 1 (block-orthonormal), P2 maps chirality to chirality;
  * the smoother's residual never grows, each step length makes the new
    residual orthogonal to D_c r (the minimal-residual condition), and the
    result does not depend on the scale of the starts;
  * the truncation is the best rank-k2 approximation per block (Eckart-Young)
    with orthonormal U_k, and k2 = m'' spans each block's range;
  * at U = 1, with the constant vectors fed to both truncations, D_cc is m0
    times the identity (a closed form through both levels).
"""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from oracle import level2 as L2


def _sigma3(k1):
    return np.r_[np.ones(k1), -np.ones(k1)]


def random_dc(cdims, k1, seed):
    """A random sigma_3-hermitian nearest-neighbour coarse operator."""
    nc = int(np.prod(cdims))
    n = 2 * k1
    g = G.normals(seed, G.STREAM_MISC, 0, 2 * nc * 5 * n * n)
    z = (g[0::2] + 1j * g[1::2]).reshape(nc, 5, n, n)
    s3 = _sigma3(k1)
    S = z[:, 0] + 3.0 * np.eye(n)
    X = S + s3[:, None] * S.conj().transpose(0, 2, 1) * s3[None, :]
    Y = np.zeros((nc, 8, n, n), dtype=np.complex128)
    for x in range(nc):
        c = L2._coords(cdims, x)
        for mu in range(4):
            Y[x, mu] = 0.3 * z[x, 1 + mu]
            cy = list(c)
            cy[mu] = (cy[mu] + 1) % cdims[mu]
            y = L2._index(cdims, cy)
            Y[y, 4 + mu] = s3[:, None] * Y[x, mu].conj().T * s3[None, :]
    return X, Y


CD, K1 = [4, 4, 2, 2], 3
B2 = [2, 2, 1, 2]


@pytest.fixture(scope="module")
def dc():
    return random_dc(CD, K1, 11)


def _starts(m, seed):
    nc = int(np.prod(CD))
    g = G.normals(seed, G.STREAM_MISC, 0, 2 * nc * 2 * K1 * m)
    return (g[0::2] + 1j * g[1::2]).reshape(nc, 2 * K1, m)


def test_dc_fixture_is_sigma3_hermitian(dc):
    X, Y = dc
    n = int(np.prod(CD)) * 2 * K1
    D = O.coarse_apply(CD, X, Y, np.eye(n).reshape(-1, 2 * K1, n)).reshape(n, n)
    s3 = np.tile(_sigma3(K1), int(np.prod(CD)))
    H = s3[:, None] * D
    assert np.abs(H - H.conj().T).max() < 1e-12


def test_mr_minimal_residual_and_scale(dc):
    X, Y = dc
    p0 = _starts(6, 3)
    psi, rn, ov = L2.mr(CD, X, Y, p0, 8, return_history=True)
    assert np.all(np.diff(rn, axis=0) <= 1e-12 * rn[:-1])
    assert ov.max() < 1e-12
    psi2 = L2.mr(CD, X, Y, p0 * np.array([1e3, 1e-3, 2, 3, 4, 5]), 8)
    assert np.abs(psi - psi2).max() < 1e-10
    assert np.allclose(np.linalg.norm(psi.reshape(-1, 6), axis=0), 1.0)


def test_truncation_eckart_young_and_full_rank(dc):
    X, Y = dc
    m, k2 = 8, 5
    psi = L2.mr(CD, X, Y, _starts(m, 4), 3)
    Uk, sig = L2.chiral_truncate(CD, B2, K1, psi, k2)
    for j in range(Uk.shape[0]):
        for al in range(2):
            A = L2.block_matrix(CD, B2, K1, psi, j, al)
            U = Uk[j, al].reshape(-1, k2)
            assert np.abs(U.conj().T @ U - np.eye(k2)).max() < 1e-12
            res = np.linalg.norm(A - U @ (U.conj().T @ A)) ** 2
            assert abs(res - np.sum(sig[j, al, k2:] ** 2)) < 1e-10 * np.sum(sig[j, al] ** 2)
            np.testing.assert_allclose(sig[j, al], np.linalg.svd(A, compute_uv=False),
                                       rtol=1e-12)
    Uf, _ = L2.chiral_truncate(CD, B2, K1, psi, m)
    for j in range(Uf.shape[0]):
        for al in range(2):
            A = L2.block_matrix(CD, B2, K1, psi, j, al)
            Uj = Uf[j, al].reshape(-1, m)
            assert np.abs(Uj @ Uj.conj().T - A @ np.linalg.pinv(A)).max() < 1e-10


def test_prolongator_and_galerkin(dc):
    X, Y = dc
    m, k2 = 8, 4
    psi = L2.mr(CD, X, Y, _starts(m, 5), 3)
    Uk, _ = L2.chiral_truncate(CD, B2, K1, psi, k2)
    P = L2.prolongator(CD, B2, Uk)
    c2 = O.coarse_dims(CD, B2)
    nc2 = int(np.prod(c2))
    rng = np.random.default_rng(2)
    v = rng.standard_normal((nc2, 2 * k2)) + 1j * rng.standard_normal((nc2, 2 * k2))
    assert np.abs(L2.restrict(CD, B2, P, L2.prolong(CD, B2, P, v)) - v).max() < 1e-12
    # chirality: the upper k2 coarse-coarse components feed only the upper k1
    vu = v.copy()
    vu[:, k2:] = 0
    assert np.abs(L2.prolong(CD, B2, P, vu)[:, K1:]).max() == 0
    X2, Y2 = L2.coarsen(CD, B2, X, Y, P)
    for _ in range(3):
        v = rng.standard_normal((nc2, 2 * k2, 1)) + 1j * rng.standard_normal((nc2, 2 * k2, 1))
        lhs = O.coarse_apply(c2, X2, Y2, v)[..., 0]
        z = L2.prolong(CD, B2, P, v[..., 0])[..., None]
        rhs = L2.restrict(CD, B2, P, O.coarse_apply(CD, X, Y, z)[..., 0])
        assert np.abs(lhs - rhs).max() < 1e-11 * np.abs(rhs).max()
    n = nc2 * 2 * k2
    D2 = O.coarse_apply(c2, X2, Y2, np.eye(n).reshape(nc2, 2 * k2, n)).reshape(n, n)
    s3 = np.tile(np.r_[np.ones(k2), -np.ones(k2)], nc2)
    H = s3[:, None] * D2
    assert np.abs(H - H.conj().T).max() < 1e-11 * np.abs(H).max()


def test_free_field_constant_modes_two_levels():
    """At U = 1 the 12 constant spin-colour vectors are eigenvectors of D with
    eigenvalue m0; fed to the first truncation (m' = 12, k1 = 6) their coarse
    images, the 12 constant unit vectors of the coarse lattice, are eigenvectors
    of D_c with eigenvalue m0.  Fed in turn to the second truncation (m = 12,
    k2 = 6, one aggregate holding the whole coarse lattice) they span range(P2),
    so D_cc = P2^dag D_c P2 is m0 times the identity: the recursion of both
    levels against a closed form."""
    from conftest import dense_coarse
    dims, block, m0 = [4, 4, 4, 4], [2, 2, 2, 2], 0.37
    V = int(np.prod(dims))
    psi = np.zeros((V, 4, 3, 12), dtype=np.complex128)
    for sp in range(4):
        for c in range(3):
            psi[:, sp, c, sp * 3 + c] = 1.0
    Uk, _ = O.chiral_truncate(dims, block, psi, 6)
    P = O.prolongator(dims, block, Uk)
    X, Y = O.coarsen(dims, block, m0, 1.0, G.unit_gauge_field(dims), None, P)
    cd = O.coarse_dims(dims, block)
    nc = int(np.prod(cd))
    q = np.zeros((nc, 12, 12), dtype=np.complex128)
    for e in range(12):
        q[:, e, e] = 1.0
    # the constant coarse vectors are eigenvectors of D_c with eigenvalue m0
    assert np.abs(O.coarse_apply(cd, X, Y, q) - m0 * q).max() < 1e-12
    Uk2, sig2 = L2.chiral_truncate(cd, [2, 2, 2, 2], 6, q, 6)
    P2 = L2.prolongator(cd, [2, 2, 2, 2], Uk2)
    X2, Y2 = L2.coarsen(cd, [2, 2, 2, 2], X, Y, P2)
    D2 = dense_coarse(O.coarse_dims(cd, [2, 2, 2, 2]), X2, Y2)
    assert D2.shape == (12, 12)
    assert np.abs(D2 - m0 * np.eye(12)).max() < 1e-12
