"""Pins of the oracle's smoother (Eq. 1 of the paper: m random starts relaxed on
D psi = 0) by properties of minimal-residual steps that hold for any correct
implementation, not by retyping the update."""
import numpy as np

import mg_inputs as G
import oracle as O
from conftest import coords, vol

DIMS = [4, 4, 2, 4]
M0, XI = -0.1, 1.0


def _setup(seed=1, m=4, csw=1.0):
    U = G.gauge_field(DIMS, 0.3, seed)
    C = O.clover(DIMS, U, csw)
    return U, C, G.psi0(DIMS, m, seed + 100)


def _norms(a):
    return np.sqrt(np.sum(np.abs(a) ** 2, axis=(0, 1, 2)))


def test_residual_decreases_and_matches_recomputed():
    """|r_t| is non-increasing per vector, and the final residual equals -D psi."""
    U, C, p0 = _setup()
    psi, res, alpha, raw = O.mr(DIMS, M0, XI, U, C, p0, 8, return_history=True)
    assert np.all(np.diff(res, axis=0) <= 1e-12 * res[:-1])
    r_true = -O.apply_D(DIMS, M0, XI, U, C, raw)
    np.testing.assert_allclose(_norms(r_true), res[-1], rtol=1e-11)


def test_one_step_is_minimal_residual():
    """After one step r_1 is orthogonal to D r_0 (the MR Galerkin condition), so no
    other multiple of D r_0 gives a smaller residual."""
    U, C, p0 = _setup(seed=2)
    _, _, _, raw = O.mr(DIMS, M0, XI, U, C, p0, 1, return_history=True)
    r0 = -O.apply_D(DIMS, M0, XI, U, C, p0)
    w0 = O.apply_D(DIMS, M0, XI, U, C, r0)
    r1 = -O.apply_D(DIMS, M0, XI, U, C, raw)
    ip = np.sum(np.conj(w0) * r1, axis=(0, 1, 2))
    assert np.all(np.abs(ip) <= 1e-12 * _norms(w0) * _norms(r1))
    # perturbing the step along D r0 can only increase |r1|
    for eps in (1e-3, -1e-3, 1e-3j):
        assert np.all(_norms(r1 - eps * w0) >= _norms(r1))


def test_output_normalised():
    U, C, p0 = _setup(seed=3)
    psi = O.mr(DIMS, M0, XI, U, C, p0, 5)
    np.testing.assert_allclose(_norms(psi), 1.0, rtol=1e-14)


def test_scale_invariance():
    """psi0 -> c psi0 scales the unnormalised result by c (each step length is
    scale free), so the normalised output is unchanged."""
    U, C, p0 = _setup(seed=4)
    _, _, _, a = O.mr(DIMS, M0, XI, U, C, p0, 6, return_history=True)
    c = np.array([2.0, -0.5j, 3 + 4j, 1e-3])
    _, _, _, b = O.mr(DIMS, M0, XI, U, C, p0 * c, 6, return_history=True)
    np.testing.assert_allclose(b, a * c, rtol=1e-11, atol=1e-14)


def test_gauge_covariance_of_smoother():
    """Transforming U and psi0 together transforms the smoothed vectors."""
    U, C, p0 = _setup(seed=5, csw=0.0)
    Gx = G.gauge_transform(DIMS, 55)
    Ut = np.empty_like(U)
    for s in range(vol(DIMS)):
        x = coords(DIMS, s)
        for mu in range(4):
            y = list(x)
            y[mu] = (y[mu] + 1) % DIMS[mu]
            t = y[0] + DIMS[0] * (y[1] + DIMS[1] * (y[2] + DIMS[2] * y[3]))
            Ut[s, mu] = Gx[s] @ U[s, mu] @ Gx[t].conj().T
    rot = lambda p: np.einsum("sab,sibm->siam", Gx, p)  # noqa: E731
    a = O.mr(DIMS, M0, XI, U, None, p0, 6)
    b = O.mr(DIMS, M0, XI, Ut, None, rot(p0), 6)
    np.testing.assert_allclose(b, rot(a), atol=1e-12)


def test_eigenvector_start_is_annihilated():
    """A free-field eigenvector start: r_0 = -lambda psi0, D r_0 = lambda r_0, the
    step length is 1/lambda and one step gives psi = 0 and r = 0 exactly."""
    dims = [4, 4, 4, 4]
    U = G.unit_gauge_field(dims)
    m0 = 0.3
    p = 2 * np.pi * np.array([1, 0, 2, 0]) / 4
    w = np.ones(4)
    B = [np.array([[0, -1j], [-1j, 0]]), np.array([[0, -1], [1, 0]]),
         np.array([[-1j, 0], [0, 1j]]), np.eye(2)]
    gam = [np.block([[np.zeros((2, 2)), b], [b.conj().T, np.zeros((2, 2))]]) for b in B]
    sym = (m0 + np.sum(w * (1 - np.cos(p)))) * np.eye(4) + \
        1j * sum(np.sin(p[mu]) * gam[mu] for mu in range(4))
    lam, vec = np.linalg.eig(sym)
    psi0 = np.zeros((vol(dims), 4, 3, 2), dtype=np.complex128)
    for s in range(vol(dims)):
        ph = np.exp(1j * np.dot(p, coords(dims, s)))
        psi0[s, :, 0, 0] = ph * vec[:, 0]
        psi0[s, :, 2, 1] = ph * vec[:, 1]
    _, res, alpha, raw = O.mr(dims, m0, 1.0, U, None, psi0, 1, return_history=True)
    np.testing.assert_allclose(alpha[0], 1.0 / lam[:2], rtol=1e-12)
    assert np.all(res[1] < 1e-12 * res[0])
    assert np.abs(raw).max() < 1e-13
