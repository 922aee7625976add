"""Pins of the oracle's prolongator (Eq. 5) and Galerkin coarse operator
D_c = R D P (Eq. 3), R = P^dagger, by brute force, the symmetries the paper
states (P^dagger P = I per block, gamma_5 P = P sigma_3) and their
consequences, and an exactly solvable free-field case."""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from conftest import coords, dense_coarse, dense_P, gamma5_diag, lex, vol


def _hierarchy(dims, block, m, k, eps=0.3, csw=1.0, m0=-0.2, xi=1.0, seed=0, iters=6):
    U = G.gauge_field(dims, eps, seed)
    C = O.clover(dims, U, csw) if csw else None
    psi = O.mr(dims, m0, xi, U, C, G.psi0(dims, m, seed + 1), iters)
    Uk, sig = O.chiral_truncate(dims, block, psi, k)
    P = O.prolongator(dims, block, Uk)
    return U, C, psi, P


@pytest.mark.parametrize("dims,block,xi,csw", [([4, 4, 4, 4], [2, 2, 2, 2], 1.0, 1.0),
                                               ([4, 2, 4, 4], [2, 2, 4, 2], 3.5, 0.0)])
def test_galerkin_equals_dense_rdp(dims, block, xi, csw):
    """Link formula X, Y equals the dense product P^dag D P (brute force, 4^4).
    The second case has a coarse extent of 1 (hops wrap into the same block)."""
    m0, k = -0.2, 3
    U, C, psi, P = _hierarchy(dims, block, 8, k, csw=csw, xi=xi)
    X, Y = O.coarsen(dims, block, m0, xi, U, C, P)
    Pd = dense_P(dims, block, P)
    ref = Pd.conj().T @ O.dense_D(dims, m0, xi, U, C) @ Pd
    got = dense_coarse(O.coarse_dims(dims, block), X, Y)
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_prolongator_orthonormal_and_chiral():
    """P_j^dag P_j = 1 per block (Sec. 3: no re-orthonormalisation needed) and
    gamma_5 P = P sigma_3 (Sec. 2)."""
    dims, block, k = [4, 4, 2, 2], [2, 2, 2, 2], 4
    _, _, _, P = _hierarchy(dims, block, 8, k)
    Pd = dense_P(dims, block, P)
    np.testing.assert_allclose(Pd.conj().T @ Pd, np.eye(Pd.shape[1]), atol=1e-13)
    nc = Pd.shape[1] // (2 * k)
    s3 = np.tile(np.r_[np.ones(k), -np.ones(k)], nc)
    g5 = gamma5_diag(vol(dims))
    np.testing.assert_array_equal(g5[:, None] * Pd, Pd * s3[None, :])


def test_sigma3_hermiticity():
    """D_c^dag = sigma_3 D_c sigma_3, inherited from gamma_5-hermiticity of D."""
    dims, block, k = [4, 4, 4, 2], [2, 2, 2, 2], 3
    m0 = -0.2
    U, C, _, P = _hierarchy(dims, block, 6, k)
    X, Y = O.coarsen(dims, block, m0, 1.0, U, C, P)
    cd = O.coarse_dims(dims, block)
    Dc = dense_coarse(cd, X, Y)
    s3 = np.tile(np.r_[np.ones(k), -np.ones(k)], vol(cd))
    np.testing.assert_allclose(s3[:, None] * Dc * s3[None, :], Dc.conj().T, atol=1e-14)
    # the stencil form: Y_{-mu}(xc + mu) = sigma_3 Y_{+mu}(xc)^dag sigma_3
    s = np.r_[np.ones(k), -np.ones(k)]
    for xc in range(vol(cd)):
        c = coords(cd, xc)
        for mu in range(4):
            y = list(c)
            y[mu] = (y[mu] + 1) % cd[mu]
            yc = lex(cd, y)
            np.testing.assert_allclose(Y[yc, 4 + mu], s[:, None] * Y[xc, mu].conj().T * s[None, :],
                                       atol=1e-14)


def test_free_field_constant_modes():
    """At U = 1 the 12 constant spin-colour vectors are eigenvectors of D with
    eigenvalue m0 (p = 0).  Fed straight to the truncation (m' = 12, k = 6) they
    lie in range(P), so m0 is a 12-fold eigenvalue of D_c = R D P."""
    dims, block, m0 = [4, 4, 4, 4], [2, 2, 2, 2], 0.37
    V = vol(dims)
    psi = np.zeros((V, 4, 3, 12), dtype=np.complex128)
    for sp in range(4):
        for c in range(3):
            psi[:, sp, c, sp * 3 + c] = 1.0
    Uk, sig = O.chiral_truncate(dims, block, psi, 6)
    P = O.prolongator(dims, block, Uk)
    U = G.unit_gauge_field(dims)
    X, Y = O.coarsen(dims, block, m0, 1.0, U, None, P)
    ev = np.linalg.eigvals(dense_coarse(O.coarse_dims(dims, block), X, Y))
    assert np.sum(np.abs(ev - m0) < 1e-10) == 12


def test_gauge_invariance_of_coarse_spectrum():
    """Transforming U and psi0 together leaves the spectrum of D_c unchanged (the
    coarse basis only changes by a block-unitary that commutes with sigma_3)."""
    dims, block, k, m0 = [4, 4, 2, 2], [2, 2, 2, 2], 3, -0.15
    U = G.gauge_field(dims, 0.3, 30)
    p0 = G.psi0(dims, 6, 31)
    Gx = G.gauge_transform(dims, 32)
    Ut = np.empty_like(U)
    for s in range(vol(dims)):
        x = coords(dims, s)
        for mu in range(4):
            y = list(x)
            y[mu] = (y[mu] + 1) % dims[mu]
            Ut[s, mu] = Gx[s] @ U[s, mu] @ Gx[lex(dims, y)].conj().T
    spectra = []
    for UU, pp in ((U, p0), (Ut, np.einsum("sab,sibm->siam", Gx, p0))):
        C = O.clover(dims, UU, 1.0)
        psi = O.mr(dims, m0, 1.0, UU, C, pp, 4)
        Uk, _ = O.chiral_truncate(dims, block, psi, k)
        P = O.prolongator(dims, block, Uk)
        X, Y = O.coarsen(dims, block, m0, 1.0, UU, C, P)
        ev = np.linalg.eigvals(dense_coarse(O.coarse_dims(dims, block), X, Y))
        spectra.append(np.sort_complex(np.round(ev, 10)))
    np.testing.assert_allclose(spectra[0], spectra[1], atol=1e-9)


@pytest.mark.parametrize("cdims", [[2, 2, 2, 2], [3, 1, 2, 4]])
def test_coarse_apply_equals_dense(cdims):
    """The stencil apply equals the dense coarse matrix times v, including coarse
    extents 1 and 2 where forward and backward hops reach the same site."""
    nc, k, nrhs = vol(cdims), 3, 5
    n = 2 * k
    g = G.normals(40, G.STREAM_MISC, 0, 2 * nc * 9 * n * n)
    Z = (g[0::2] + 1j * g[1::2]).reshape(nc, 9, n, n)
    X, Y = Z[:, 0].copy(), Z[:, 1:].copy()
    v = G.coarse_vectors(nc, n, nrhs, 41)
    out = O.coarse_apply(cdims, X, Y, v)
    ref = (dense_coarse(cdims, X, Y) @ v.reshape(-1, nrhs)).reshape(out.shape)
    np.testing.assert_allclose(out, ref, atol=1e-12)
