"""Pins of the oracle's inputs and fine operator D against closed forms and
symmetries (nothing here compares the oracle with itself).

Operator: Wilson(-clover) D of the paper's Sec. 1-2 in the chiral basis; the
free-field (unit-link) spectrum, gamma_5-hermiticity and gauge covariance are
properties the operator must have whatever the implementation.
"""
import itertools

import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from conftest import coords, gamma5_diag, lex, vol


def _free_spectrum(dims, m0, w):
    """Closed form: m0 + sum w(1 - cos p) +- i sqrt(sum w^2 sin^2 p), 6-fold each."""
    ev = []
    for n in itertools.product(*[range(L) for L in dims]):
        p = 2 * np.pi * np.array(n) / np.array(dims)
        re = m0 + np.sum(w * (1 - np.cos(p)))
        im = np.sqrt(np.sum(w ** 2 * np.sin(p) ** 2))
        ev += [re + 1j * im] * 6 + [re - 1j * im] * 6
    return np.array(ev)


def _sorted(z):
    o = np.lexsort((np.round(z.imag, 9), np.round(z.real, 9)))
    return z[o]


@pytest.mark.parametrize("dims,m0,xi", [([4, 4, 2, 2], 0.1, 1.0), ([2, 3, 4, 4], -0.3, 3.5),
                                        ([3, 4, 2, 5], 0.05, 1.0)])
def test_free_field_spectrum(dims, m0, xi):
    """At U = 1 the eigenvalues of D are the free Wilson dispersion, 6-fold."""
    U = G.unit_gauge_field(dims)
    ev = np.linalg.eigvals(O.dense_D(dims, m0, xi, U, None))
    ref = _free_spectrum(dims, m0, np.array([1, 1, 1, 1 / xi]))
    np.testing.assert_allclose(_sorted(ev), _sorted(ref), atol=1e-12)


def test_plane_waves_are_eigenvectors():
    """e^{ipx} chi with chi an eigenvector of the 4x4 free symbol is annihilated by D - lambda."""
    dims, m0, xi = [4, 4, 4, 2], 0.2, 2.0
    V = vol(dims)
    w = np.array([1, 1, 1, 1 / xi])
    U = G.unit_gauge_field(dims)
    # chiral-basis gamma matrices written out from their definition
    B = [np.array([[0, -1j], [-1j, 0]]), np.array([[0, -1], [1, 0]]),
         np.array([[-1j, 0], [0, 1j]]), np.eye(2)]
    gam = [np.block([[np.zeros((2, 2)), b], [b.conj().T, np.zeros((2, 2))]]) for b in B]
    for n in [(1, 0, 0, 0), (1, 2, 3, 1), (0, 0, 1, 1)]:
        p = 2 * np.pi * np.array(n) / np.array(dims)
        sym = (m0 + np.sum(w * (1 - np.cos(p)))) * np.eye(4) + \
            1j * sum(w[mu] * np.sin(p[mu]) * gam[mu] for mu in range(4))
        lam, vec = np.linalg.eig(sym)
        psi = np.zeros((V, 4, 3, 4), dtype=np.complex128)
        for s in range(V):
            x = np.array(coords(dims, s))
            ph = np.exp(1j * np.dot(p, x))
            for c in range(4):
                psi[s, :, c % 3, c] = ph * vec[:, c]
        out = O.apply_D(dims, m0, xi, U, None, psi)
        np.testing.assert_allclose(out, psi * lam[None, None, None, :], atol=1e-13)


def test_gauge_links_are_su3():
    U = G.gauge_field([4, 4, 4, 4], 0.3, 0).reshape(-1, 3, 3)
    uu = np.einsum("nji,njk->nik", U.conj(), U)
    np.testing.assert_allclose(uu, np.broadcast_to(np.eye(3), uu.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(U), 1.0, atol=1e-14)


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_gamma5_hermiticity(csw):
    """gamma_5 D gamma_5 = D^dagger (Wilson and Wilson-clover)."""
    dims = [4, 2, 2, 4]
    U = G.gauge_field(dims, 0.4, 3)
    C = O.clover(dims, U, csw) if csw else None
    Dm = O.dense_D(dims, -0.2, 1.7, U, C)
    g5 = gamma5_diag(vol(dims))
    np.testing.assert_allclose(g5[:, None] * Dm * g5[None, :], Dm.conj().T, atol=1e-14)


def test_matrix_free_equals_dense():
    dims = [4, 4, 2, 2]
    U = G.gauge_field(dims, 0.3, 5)
    C = O.clover(dims, U, 1.0)
    psi = G.psi0(dims, 3, 6)
    Dm = O.dense_D(dims, -0.1, 1.3, U, C)
    out = O.apply_D(dims, -0.1, 1.3, U, C, psi)
    ref = (Dm @ psi.reshape(-1, 3)).reshape(out.shape)
    np.testing.assert_allclose(out, ref, atol=1e-13)


def _transform_links(dims, U, Gx):
    """U_mu(x) -> G(x) U_mu(x) G(x+mu)^dagger."""
    V = vol(dims)
    Ut = np.empty_like(U)
    for s in range(V):
        x = coords(dims, s)
        for mu in range(4):
            y = list(x)
            y[mu] = (y[mu] + 1) % dims[mu]
            Ut[s, mu] = Gx[s] @ U[s, mu] @ Gx[lex(dims, y)].conj().T
    return Ut


def test_gauge_covariance_of_D():
    """D[U^G] (G psi) = G (D[U] psi)."""
    dims = [2, 4, 2, 4]
    U = G.gauge_field(dims, 0.3, 7)
    Gx = G.gauge_transform(dims, 8)
    Ut = _transform_links(dims, U, Gx)
    psi = G.psi0(dims, 2, 9)
    gpsi = np.einsum("sab,sibm->siam", Gx, psi)
    for csw in (0.0, 1.0):
        C = O.clover(dims, U, csw) if csw else None
        Ct = O.clover(dims, Ut, csw) if csw else None
        lhs = O.apply_D(dims, 0.1, 1.0, Ut, Ct, gpsi)
        rhs = np.einsum("sab,sibm->siam", Gx, O.apply_D(dims, 0.1, 1.0, U, C, psi))
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_clover_structure():
    """Hermitian, no chirality mixing, zero for the unit and for a pure-gauge field."""
    dims = [4, 4, 2, 2]
    U = G.gauge_field(dims, 0.5, 11)
    C, off = O.clover(dims, U, 1.0, return_offblock=True)
    assert off < 1e-15
    np.testing.assert_allclose(C, np.conj(np.swapaxes(C, -1, -2)), atol=1e-15)
    assert np.abs(C).max() > 1e-2
    assert np.abs(O.clover(dims, G.unit_gauge_field(dims), 1.0)).max() == 0.0
    pure = _transform_links(dims, G.unit_gauge_field(dims), G.gauge_transform(dims, 12))
    assert np.abs(O.clover(dims, pure, 1.0)).max() < 1e-14


def test_clover_gauge_covariance():
    """C(x) -> G(x) C(x) G(x)^dagger on the colour index of each chirality block."""
    dims = [2, 2, 4, 4]
    U = G.gauge_field(dims, 0.3, 13)
    Gx = G.gauge_transform(dims, 14)
    C = O.clover(dims, U, 1.3)
    Ct = O.clover(dims, _transform_links(dims, U, Gx), 1.3)
    C6 = C.reshape(-1, 2, 2, 3, 2, 3)
    ref = np.einsum("xpa,xlsaqb,xrb->xlspqr", Gx, C6, Gx.conj()).reshape(C.shape)
    np.testing.assert_allclose(Ct, ref, atol=1e-14)


def test_clover_uniform_abelian_flux():
    """Uniform flux B in the x-y plane (U_y(x) = e^{iBx} 1): every leaf is e^{iB},
    F_xy = i sin(B) 1, and C = (csw/2) sin(B) diag(sigma_3, sigma_3) x 1_colour,
    since sigma_xy = -diag(sigma_3, sigma_3) in the chiral basis."""
    dims = [4, 3, 2, 2]
    Bf = 2 * np.pi / 4
    U = G.unit_gauge_field(dims)
    for s in range(vol(dims)):
        x = coords(dims, s)
        U[s, 1] = np.exp(1j * Bf * x[0]) * np.eye(3)
    csw = 0.7
    C = O.clover(dims, U, csw)
    s3 = np.diag([1.0, -1.0])
    blk = 0.5 * csw * np.sin(Bf) * np.kron(s3, np.eye(3))
    for al in range(2):
        np.testing.assert_allclose(C[:, al], np.broadcast_to(blk, C[:, al].shape), atol=1e-15)
