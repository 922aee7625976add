"""Pins of the solve oracle (oracle.solve), independent of the functions they
check:

  * a GMRES cycle of j steps returns the minimiser of |b - A x| over the Krylov
    space span{b, Ab, ..., A^(j-1) b}, found by brute force (least squares on
    the explicit Krylov matrix); n steps solve an n x n system exactly;
  * FGMRES with the identity as preconditioner is GMRES, with the exact
    inverse it converges in one step, with a fixed linear M it is M times the
    GMRES iterate of A M; restarted FGMRES reaches its tolerance (true
    residual, not the estimate);
  * one MR step is x = a r with a = <Ar, r> / <Ar, Ar>, and MR never increases
    the residual;
  * the multigrid K-cycle solve on the 4^4 workload, with two and with three
    levels, returns numpy.linalg.solve of the dense D; with an exact coarse
    solve and no post-smoothing the
    coarse correction leaves a residual that the restriction annihilates
    (R (r - D x) = 0, because D_c = R D P), and the two-level solve needs fewer
    steps than GMRES on D alone.
"""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from oracle import solve as S


def _dense(n, seed, shift=3.0):
    g = G.normals(seed, G.STREAM_MISC, 0, 2 * n * n + 2 * n)
    z = g[0::2] + 1j * g[1::2]
    A = z[:n * n].reshape(n, n) + shift * np.eye(n)
    return A, z[n * n:]


def test_gmres_is_krylov_least_squares():
    A, b = _dense(10, 1)
    op = lambda v: A @ v  # noqa: E731
    for j in (1, 3, 6):
        x = S.gmres(op, b, j)
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(j)], axis=1)
        y, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
        assert np.linalg.norm(x - K @ y) <= 1e-10 * np.linalg.norm(K @ y)
    x = S.gmres(op, b, 10)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)


def test_fgmres_preconditioners():
    A, b = _dense(10, 2)
    op = lambda v: A @ v  # noqa: E731
    x1 = S.arnoldi_cycle(op, b, None, 4, M=lambda v: v.copy())[0]
    assert np.allclose(x1, S.gmres(op, b, 4), rtol=1e-12, atol=1e-14)
    Ainv = np.linalg.inv(A)
    x2, steps, est = S.arnoldi_cycle(op, b, None, 5, M=lambda v: Ainv @ v, tol_abs=1e-10)
    assert steps == 1 and est < 1e-10
    x3, total = S.fgmres(op, b, None, 1e-9, 3, 200)
    assert np.linalg.norm(b - A @ x3) <= 1e-9 * np.linalg.norm(b) * 1.0001
    assert total > 3  # needed restarts


def test_fgmres_with_linear_preconditioner_is_right_preconditioned_gmres():
    """With a fixed linear M, one FGMRES cycle of j steps returns M y, y the
    j-step GMRES iterate of the operator A M (right preconditioning)."""
    A, b = _dense(10, 4)
    Mm, _ = _dense(10, 5, shift=2.0)
    op = lambda v: A @ v  # noqa: E731
    for j in (2, 5):
        x = S.arnoldi_cycle(op, b, None, j, M=lambda v: Mm @ v)[0]
        y = S.gmres(lambda v: A @ (Mm @ v), b, j)
        assert np.linalg.norm(x - Mm @ y) <= 1e-10 * np.linalg.norm(x)


def test_mr_step_and_monotone_residual():
    A, b = _dense(12, 3, shift=4.0)
    op = lambda v: A @ v  # noqa: E731
    Ab = A @ b
    a = np.vdot(Ab, b) / np.vdot(Ab, Ab)
    assert np.allclose(S.mr(op, b, 1), a * b, rtol=1e-13)
    res = [np.linalg.norm(b - A @ S.mr(op, b, nu)) for nu in range(6)]
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(5))


@pytest.fixture(scope="module")
def h44():
    dims, block, m, k, N = [4, 4, 4, 4], [2, 2, 2, 2], 24, 12, 50
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "m0.json")) as fh:
        m0 = json.load(fh)["workloads"]["4^4 Wilson eps=0.3"]["m0"]
    U = G.gauge_field(dims, 0.3, 0)
    p0 = G.psi0(dims, m, 1)
    psi = O.mr(dims, m0, 1.0, U, None, p0, N)
    Uk, _ = O.chiral_truncate(dims, block, psi, k)
    P = O.prolongator(dims, block, Uk)
    X, Y = O.coarsen(dims, block, m0, 1.0, U, None, P)
    levels = S.fine_levels(dims, block, m0, 1.0, U, None, P, X, Y)
    g = G.normals(2, G.STREAM_MISC, 0, 2 * 256 * 12)
    b = (g[0::2] + 1j * g[1::2]).reshape(256, 4, 3)
    return dict(dims=dims, m0=m0, U=U, levels=levels, b=b, k=k, P=P, XY=(X, Y))


def test_kcycle_solve_equals_dense_solve(h44):
    c = h44
    p = S.KParams(nu_pre=2, nu_post=2, kcycle_iters=2, coarsest_iters=32)
    x, steps = S.solve(c["levels"], c["b"], p, 1e-10, 16, 400)
    D = O.dense_D(c["dims"], c["m0"], 1.0, c["U"], None)
    xs = np.linalg.solve(D, c["b"].reshape(-1)).reshape(c["b"].shape)
    r = c["b"] - c["levels"][0].A(x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(c["b"]) * 1.0001
    # |x - x*| <= |D^-1| |r|
    smin = np.linalg.svd(D, compute_uv=False)[-1]
    assert np.linalg.norm(x - xs) <= np.linalg.norm(r) / smin * 1.01
    _, steps1 = S.solve(c["levels"][:1], c["b"], p, 1e-10, 16, 400)
    assert steps < steps1


def test_exact_coarse_correction_is_galerkin(h44):
    c = h44
    k = c["k"]
    p = S.KParams(nu_pre=1, nu_post=0, coarsest_iters=16 * 2 * k)
    r = c["b"]
    x = S.kcycle(c["levels"], 0, r, p)
    L0 = c["levels"][0]
    s = L0.R(r - L0.A(x))
    assert np.linalg.norm(s) <= 1e-9 * np.linalg.norm(L0.R(r))


def test_three_level_kcycle_solve_equals_dense_solve(h44):
    """The recursion: level 2 built by the level-2 oracle on the 4^4 hierarchy's
    D_c (2^4 coarse sites, one aggregate), K-cycle FGMRES steps on level 1."""
    from oracle import level2 as L2
    c = h44
    dims, block, k = c["dims"], [2, 2, 2, 2], c["k"]
    L0, L1 = c["levels"]
    cd = O.coarse_dims(dims, block)
    X, Y = c["XY"]
    g = G.normals(4, G.STREAM_MISC, 0, 2 * 16 * 2 * k * 16)
    q0 = (g[0::2] + 1j * g[1::2]).reshape(16, 2 * k, 16)
    psi2 = L2.mr(cd, X, Y, q0, 20)
    Uk2, _ = L2.chiral_truncate(cd, [2, 2, 2, 2], k, psi2, 8)
    P2 = L2.prolongator(cd, [2, 2, 2, 2], Uk2)
    X2, Y2 = L2.coarsen(cd, [2, 2, 2, 2], X, Y, P2)
    levels = S.fine_levels(dims, block, c["m0"], 1.0, c["U"], None, c["P"], X, Y,
                           P2, [2, 2, 2, 2], X2, Y2)
    p = S.KParams(nu_pre=2, nu_post=2, kcycle_iters=2, coarsest_iters=16)
    x, steps = S.solve(levels, c["b"], p, 1e-10, 16, 400)
    r = c["b"] - L0.A(x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(c["b"]) * 1.0001
    D = O.dense_D(dims, c["m0"], 1.0, c["U"], None)
    xs = np.linalg.solve(D, c["b"].reshape(-1)).reshape(c["b"].shape)
    smin = np.linalg.svd(D, compute_uv=False)[-1]
    assert np.linalg.norm(x - xs) <= np.linalg.norm(r) / smin * 1.01
