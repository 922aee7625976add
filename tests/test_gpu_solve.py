"""The solve (mg_solve: FGMRES preconditioned by the K-cycle over the
hierarchy, Sec. 2) on the GPU against the FP64 oracle of the same algorithm
(oracle.solve), on a hierarchy the oracle built, rounded to complex64 so that
both sides see the same numbers.

Hierarchy: 8^4 Wilson-clover (eps = 0.25, the near-critical m0 of the
16^3x32 workload), m' = 48 test vectors, k1 = 24, 20 MR iterations, 2^4
aggregates; second level on its D_c with m = 64, k2 = 32, 20 MR iterations,
2^4 aggregates.  K-cycle: 2 + 2 MR steps, 2 FGMRES steps on level 1 when it
is not the coarsest, 32 GMRES steps on the coarsest level; outer FGMRES(16),
tolerance 1e-5, four right-hand sides.

Checks:
  * every system's true residual |b - D x| / |b|, with the FP64 D of the oracle
    applied to the GPU's x, is <= 2e-5 (the FP32 Arnoldi's estimate stops the
    solve at 1e-5; the recomputed residual differs by FP32 rounding of the
    iterates), and the residual the call reports matches it to 1e-6;
  * the number of outer steps equals the oracle's (FP64, the largest over the
    four systems, which the GPU solves in lock step) within 2;
  * with three levels it is no larger than with two, and with one level
    (plain GMRES on D) the reported residual is again the true one.
"""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from gpu_common import M0, to_dev, to_host
from oracle import level2 as L2
from oracle import solve as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg  # noqa: E402

_build.build()

DIMS, B1, M1, K1, N1 = [8, 8, 8, 8], [2, 2, 2, 2], 48, 24, 20
B2, M2, K2, N2 = [2, 2, 2, 2], 64, 32, 20
M0_ = M0["16^3x32 Wilson-clover eps=0.25"]
TOL, RESTART, NRHS = 1e-5, 16, 4
KC = dict(nu_pre=2, nu_post=2, kcycle_iters=2, coarsest_iters=32)


@pytest.fixture(scope="module")
def hier():
    U = G.round_to_c64(G.gauge_field(DIMS, 0.25, 10))
    C = G.round_to_c64(O.clover(DIMS, U, 1.0))
    p0 = G.round_to_c64(G.psi0(DIMS, M1, 11))
    psi = O.mr(DIMS, M0_, 1.0, U, C, p0, N1)
    Uk, _ = O.chiral_truncate(DIMS, B1, psi, K1)
    P = G.round_to_c64(O.prolongator(DIMS, B1, Uk))
    X, Y = O.coarsen(DIMS, B1, M0_, 1.0, U, C, P)
    X, Y = G.round_to_c64(X), G.round_to_c64(Y)
    cd = O.coarse_dims(DIMS, B1)
    q0 = G.round_to_c64(G.coarse_vectors(G.volume(cd), 2 * K1, M2, 5))
    psi2 = L2.mr(cd, X, Y, q0, N2)
    Uk2, _ = L2.chiral_truncate(cd, B2, K1, psi2, K2)
    P2 = G.round_to_c64(L2.prolongator(cd, B2, Uk2))
    X2, Y2 = L2.coarsen(cd, B2, X, Y, P2)
    X2, Y2 = G.round_to_c64(X2), G.round_to_c64(Y2)
    b = G.round_to_c64(G.psi0(DIMS, NRHS, 12))
    prob = mg.Problem(dims=DIMS, block=B1, m0=M0_, n_vec=M1, k=K1, mr_iters=N1, csw=1.0)
    second = mg.CoarseProblem(cd, B2, K1, M2, K2, N2)
    dev = dict(U=to_dev(U), C=to_dev(C.reshape(-1, 2, 6, 6)), P=to_dev(P), X=to_dev(X),
               Y=to_dev(Y), P2=to_dev(P2), X2=to_dev(X2), Y2=to_dev(Y2), b=to_dev(b))
    return dict(U=U, C=C, P=P, X=X, Y=Y, P2=P2, X2=X2, Y2=Y2, b=b, prob=prob, second=second,
                dev=dev, cd=cd)


def _oracle_steps(h, levels):
    lv = S.fine_levels(DIMS, B1, M0_, 1.0, h["U"], h["C"], h["P"], h["X"], h["Y"],
                       *((h["P2"], B2, h["X2"], h["Y2"]) if levels == 3 else ()))
    p = S.KParams(**KC)
    steps = []
    for c in range(NRHS):
        _, n = S.solve(lv, np.ascontiguousarray(h["b"][..., c]), p, TOL, RESTART, 400)
        steps.append(n)
    return max(steps)


def _gpu_solve(h, levels, max_iters=400):
    d = h["dev"]
    x = torch.full(d["b"].shape, float("nan"), dtype=torch.complex64, device="cuda")
    kw = dict(P=d["P"], X=d["X"], Y=d["Y"]) if levels >= 2 else {}
    if levels == 3:
        kw.update(second=h["second"], P2=d["P2"], X2=d["X2"], Y2=d["Y2"])
    steps, rel = mg.mg_solve(h["prob"], d["U"], d["C"], d["b"], x, TOL, RESTART, max_iters,
                             kcycle=mg.KCycle(**KC), **kw)
    return steps, rel, to_host(x)


def _true_residual(h, x):
    r = h["b"] - O.apply_D(DIMS, M0_, 1.0, h["U"], h["C"], x)
    return (np.linalg.norm(r.reshape(-1, NRHS), axis=0)
            / np.linalg.norm(h["b"].reshape(-1, NRHS), axis=0))


_steps = {}


@pytest.mark.parametrize("levels", [2, 3])
def test_kcycle_solve_matches_oracle(hier, levels):
    steps, rel, x = _gpu_solve(hier, levels)
    true = _true_residual(hier, x)
    assert np.all(true <= 2 * TOL), true
    np.testing.assert_allclose(rel, true, atol=1e-6)
    want = _oracle_steps(hier, levels)
    assert abs(steps - want) <= 2, (steps, want)
    _steps[levels] = steps


def test_three_levels_no_more_steps_than_two(hier):
    if 2 not in _steps or 3 not in _steps:
        _steps[2] = _gpu_solve(hier, 2)[0]
        _steps[3] = _gpu_solve(hier, 3)[0]
    assert _steps[3] <= _steps[2]


def test_plain_gmres_reports_true_residual(hier):
    steps, rel, x = _gpu_solve(hier, 1, max_iters=48)
    assert steps == 48
    np.testing.assert_allclose(rel, _true_residual(hier, x), atol=1e-6)
    assert np.all(rel < 1.0)
