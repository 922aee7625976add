"""Shared pytest configuration: the ``gpu`` marker and common lattice helpers."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def vol(d):
    return int(np.prod(d))


def coords(dims, s):
    x = []
    for L in dims:
        x.append(s % L)
        s //= L
    return x


def lex(dims, x):
    return x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))


def gamma5_diag(V, m=None):
    """Diagonal of gamma_5 in the [site][spin][colour] order."""
    return np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)


def dense_P(dims, block, P):
    """Dense (12V x 2k*nc) prolongator from the site-major P[V][2][2][3][k]."""
    V = vol(dims)
    k = P.shape[-1]
    Lc = [dims[i] // block[i] for i in range(4)]
    nc = vol(Lc)
    n = 2 * k
    Pd = np.zeros((12 * V, n * nc), dtype=np.complex128)
    for s in range(V):
        x = coords(dims, s)
        j = lex(Lc, [x[i] // block[i] for i in range(4)])
        for al in range(2):
            Pd[s * 12 + al * 6: s * 12 + al * 6 + 6, j * n + al * k: j * n + al * k + k] = \
                P[s, al].reshape(6, k)
    return Pd


def dense_coarse(cdims, X, Y):
    """Dense coarse operator from the X, Y stencil (hops to the same site add)."""
    nc = vol(cdims)
    n = X.shape[-1]
    Dc = np.zeros((nc * n, nc * n), dtype=np.complex128)
    for xc in range(nc):
        c = coords(cdims, xc)
        Dc[xc * n:(xc + 1) * n, xc * n:(xc + 1) * n] += X[xc]
        for d in range(8):
            mu, st = d % 4, (1 if d < 4 else -1)
            cc = list(c)
            cc[mu] = (cc[mu] + st) % cdims[mu]
            yc = lex(cdims, cc)
            Dc[xc * n:(xc + 1) * n, yc * n:(yc + 1) * n] += Y[xc, d]
    return Dc
