"""FP64 CPU oracle of the multigrid solve the setup serves (Sec. 2: the
hierarchy used in a K-cycle as the preconditioner of a flexible outer Krylov
solver, FGMRES).

TEST INFRASTRUCTURE ONLY (the same rule as the rest of ``oracle``): only
``tests/`` and ``bench.py``'s CPU legs may import it.

Textbook algorithms, written out one right-hand side at a time, in the order
and with the choices the GPU solver makes (so that iteration counts compare):

  mr(A, r, nu)             nu minimal-residual steps on A x = r from x = 0
  arnoldi_cycle(...)       one (F)GMRES cycle from x0: Arnoldi with classical
                           Gram-Schmidt applied twice, right preconditioner M
                           (flexible: z_j = M(v_j) is kept), stop after `iters`
                           steps or once the least-squares residual is
                           <= tol_abs; x = x0 + Z y with y the least-squares
                           solution of min |beta e_1 - H y|
  gmres(A, b, iters)       one cycle, x0 = 0, no preconditioner, fixed length
  fgmres(A, b, M, ...)     restarted flexible GMRES until |r| <= tol |b|
  kcycle(levels, l, r, p)  the K-cycle at level l: nu_pre MR steps, coarse
                           correction (GMRES on the coarsest level, else
                           kcycle_iters FGMRES steps preconditioned by the
                           K-cycle one level down), nu_post MR steps
Levels are (A, R, P) triples of callables: A the level's operator, R the
restriction to the next level (P^dagger), P the prolongation from it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import apply_D, coarse_apply, coarse_dims
from . import level2 as _l2


def _dot(a, b):
    return np.vdot(a, b)  # conj(a) . b over all entries


def _norm(a):
    return float(np.sqrt(_dot(a, a).real))


def mr(A, r, nu):
    """x with nu MR steps on A x = r from x = 0: w = A rr, a = <w, rr>/<w, w>,
    x += a rr, rr -= a w."""
    x = np.zeros_like(r)
    rr = r.copy()
    for _ in range(nu):
        w = A(rr)
        ww = _dot(w, w).real
        a = _dot(w, rr) / ww if ww > 0 else 0.0
        x = x + a * rr
        rr = rr - a * w
    return x


def arnoldi_cycle(A, b, x0, iters, M=None, tol_abs=None):
    """One GMRES (M None) or FGMRES cycle; returns (x, steps, residual estimate)."""
    r = b.copy() if x0 is None else b - A(x0)
    beta = _norm(r)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if beta == 0.0:
        return x, 0, 0.0
    V = [r / beta]
    Z = []
    H = np.zeros((iters + 1, iters), dtype=np.complex128)
    steps, est = 0, beta
    for j in range(iters):
        z = M(V[j]) if M is not None else V[j]
        Z.append(z)
        w = A(z)
        for _ in range(2):  # classical Gram-Schmidt, twice
            h = np.array([_dot(V[i], w) for i in range(j + 1)])
            for i in range(j + 1):
                w = w - h[i] * V[i]
            H[:j + 1, j] += h
        hn = _norm(w)
        H[j + 1, j] = hn
        steps = j + 1
        g = np.zeros(steps + 1, dtype=np.complex128)
        g[0] = beta
        y, *_ = np.linalg.lstsq(H[:steps + 1, :steps], g, rcond=None)
        est = float(np.linalg.norm(g - H[:steps + 1, :steps] @ y))
        if hn == 0.0:
            break
        V.append(w / hn)
        if tol_abs is not None and est <= tol_abs:
            break
    g = np.zeros(steps + 1, dtype=np.complex128)
    g[0] = beta
    y, *_ = np.linalg.lstsq(H[:steps + 1, :steps], g, rcond=None)
    for i in range(steps):
        x = x + y[i] * Z[i]
    return x, steps, est


def gmres(A, b, iters):
    """GMRES from x = 0, `iters` Arnoldi steps, no preconditioner."""
    return arnoldi_cycle(A, b, None, iters)[0]


def fgmres(A, b, M, tol, restart, max_iters):
    """Restarted FGMRES from x = 0 until the cycle's least-squares residual is
    <= tol |b| (or max_iters steps); returns (x, steps)."""
    bn = _norm(b)
    x, total = None, 0
    while True:
        n = min(restart, max_iters - total)
        x, steps, est = arnoldi_cycle(A, b, x, n, M, tol * bn)
        total += steps
        if est <= tol * bn or total >= max_iters or steps == 0:
            return x, total


@dataclass
class KParams:
    nu_pre: int = 2
    nu_post: int = 2
    kcycle_iters: int = 2
    coarsest_iters: int = 8


@dataclass
class Level:
    A: object
    R: object = None   # to the next level (P^dagger)
    P: object = None   # from the next level


def kcycle(levels, l, r, p: KParams):
    """The K-cycle preconditioner at level l applied to r."""
    L = levels[l]
    x = mr(L.A, r, p.nu_pre)
    s = r - L.A(x) if p.nu_pre > 0 else r
    rc = L.R(s)
    nxt = l + 1
    if nxt == len(levels) - 1:
        ec = gmres(levels[nxt].A, rc, p.coarsest_iters)
    else:
        ec = arnoldi_cycle(levels[nxt].A, rc, None, p.kcycle_iters,
                           lambda v: kcycle(levels, nxt, v, p))[0]
    x = x + L.P(ec)
    if p.nu_post > 0:
        s = r - L.A(x)
        x = x + mr(L.A, s, p.nu_post)
    return x


def solve(levels, b, p: KParams, tol, restart, max_iters):
    """FGMRES on levels[0] preconditioned by the K-cycle (plain restarted GMRES
    when there is a single level); returns (x, steps)."""
    M = (lambda v: kcycle(levels, 0, v, p)) if len(levels) > 1 else None
    return fgmres(levels[0].A, b, M, tol, restart, max_iters)


# ---------------------------------------------------------------------------
# the levels of a setup hierarchy (vectors: fine [V][4][3], coarse [nc][2k])
# ---------------------------------------------------------------------------
def _block_of_site(dims, block):
    V = int(np.prod(dims))
    s = np.arange(V)
    c = []
    for L in dims:
        c.append(s % L)
        s = s // L
    Lc = coarse_dims(dims, block)
    jc = [c[i] // block[i] for i in range(4)]
    return jc[0] + Lc[0] * (jc[1] + Lc[1] * (jc[2] + Lc[2] * jc[3]))


def fine_levels(dims, block, m0, xi, U, C, P, X, Y, P2=None, block2=None, X2=None, Y2=None):
    """Levels of a two- or three-level hierarchy: D on the fine lattice, D_c
    (X, Y) with fine prolongator P[V][2][2][3][k1], and optionally D_cc (X2, Y2)
    with the level-1 prolongator P2[nc][2][k1][k2]."""
    V = int(np.prod(dims))
    k1 = P.shape[-1]
    jx = _block_of_site(dims, block)
    nc = int(np.prod(coarse_dims(dims, block)))
    cd = coarse_dims(dims, block)
    Pf = P.reshape(V, 2, 6, k1)

    def A0(v):
        return apply_D(dims, m0, xi, U, C, v[..., None])[..., 0]

    def R0(v):
        loc = np.einsum("xaei,xae->xai", Pf.conj(), v.reshape(V, 2, 6)).reshape(V, 2 * k1)
        out = np.zeros((nc, 2 * k1), dtype=np.complex128)
        np.add.at(out, jx, loc)
        return out

    def P0(vc):
        return np.einsum("xaei,xai->xae", Pf, vc[jx].reshape(V, 2, k1)).reshape(V, 4, 3)

    def A1(v):
        return coarse_apply(cd, X, Y, v[..., None])[..., 0]

    levels = [Level(A0, R0, P0), Level(A1)]
    if P2 is not None:
        c2 = coarse_dims(cd, block2)
        levels[1].R = lambda v: _l2.restrict(cd, block2, P2, v)
        levels[1].P = lambda v: _l2.prolong(cd, block2, P2, v)
        levels.append(Level(lambda v: coarse_apply(c2, X2, Y2, v[..., None])[..., 0]))
    return levels
