"""FP64 CPU oracle of the chiral rank-k multigrid setup (arXiv:2502.03091).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA path never
imports it and shares no code with it.

The arithmetic lives in ``mg_oracle.c`` (plain C99, complex128, OpenMP over
sites and blocks); this module only compiles it and marshals numpy arrays.
Every function follows one passage of the paper:

  clover(U)                  operator input (the clover term of the ensembles, Sec. 4;
                             sign and normalisation are this library's reading: pinned
                             to that convention by a closed form, parity against the
                             paper unpinned)
  apply_D / dense_D          the fine operator D (Sec. 1, 2)
  mr(...)                    smoother on D psi = 0 with m random starts (Eq. 1)
  chiral_truncate(...)       chiral split (Eq. 2) + per-block SVD, rank-k truncation (Eq. 4)
  prolongator(...)           P from the truncated left singular vectors (Eq. 5)
  coarsen(...)               D_c = R D P with R = P^dagger (Eq. 3)
  coarse_apply(...)          D_c v on the coarse stencil
  svd(A)                     thin SVD of one block (Householder QR + one-sided Jacobi)

The second level (the same steps on D_c, chirality sigma_3) is in ``level2``
(numpy over coarse_apply and svd).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I4 = ctypes.POINTER(ctypes.c_int)
        d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
        lib.or_clover.argtypes = [I4, P, d, P, P]
        lib.or_apply_D.argtypes = [I4, d, d, P, P, i, P, P]
        lib.or_dense_D.argtypes = [I4, d, d, P, P, P]
        lib.or_mr.argtypes = [I4, d, d, P, P, i, i, P, P, P, P, P]
        lib.or_svd.argtypes = [i, i, P, P, P, P]
        lib.or_chiral_truncate.argtypes = [I4, I4, i, i, P, P, P, P]
        lib.or_prolongator.argtypes = [I4, I4, i, P, P]
        lib.or_coarsen.argtypes = [I4, I4, i, d, d, P, P, P, P, P]
        lib.or_coarse_apply.argtypes = [I4, i, P, P, i, P, P]
        lib.or_gamma5.argtypes = [l, i, P, P]
        for f in (lib.or_clover, lib.or_apply_D, lib.or_dense_D, lib.or_mr, lib.or_svd,
                  lib.or_chiral_truncate, lib.or_prolongator, lib.or_coarsen,
                  lib.or_coarse_apply, lib.or_gamma5):
            f.restype = None
        _lib = lib
    return _lib


def _dims(d):
    return (ctypes.c_int * 4)(*[int(v) for v in d])


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _vol(d):
    return int(d[0]) * int(d[1]) * int(d[2]) * int(d[3])


def clover(dims, U, csw: float, return_offblock: bool = False):
    """Clover field C[V][2][6][6] (per chirality) from the links U[V][4][3][3]."""
    U = _c128(U)
    C = np.zeros((_vol(dims), 2, 6, 6), dtype=np.complex128)
    off = ctypes.c_double(0.0)
    _load().or_clover(_dims(dims), _ptr(U), csw, _ptr(C), ctypes.byref(off))
    return (C, off.value) if return_offblock else C


def apply_D(dims, m0, xi, U, C, psi):
    """D psi for psi[V][4][3][m] (C may be None for pure Wilson)."""
    U, psi = _c128(U), _c128(psi)
    C = None if C is None else _c128(C)
    m = psi.shape[-1]
    out = np.empty_like(psi)
    _load().or_apply_D(_dims(dims), m0, xi, _ptr(U), _ptr(C), m, _ptr(psi), _ptr(out))
    return out


def dense_D(dims, m0, xi, U, C):
    """Dense (12V x 12V) matrix of D, index site*12 + spin*3 + colour."""
    U = _c128(U)
    C = None if C is None else _c128(C)
    n = 12 * _vol(dims)
    Dm = np.empty((n, n), dtype=np.complex128)
    _load().or_dense_D(_dims(dims), m0, xi, _ptr(U), _ptr(C), _ptr(Dm))
    return Dm


def mr(dims, m0, xi, U, C, psi0, niter, return_history: bool = False):
    """MR smoother (Eq. 1): returns the normalised vectors [V][4][3][m].

    With return_history, also returns (resnorm[niter+1][m], alpha[niter][m],
    unnormalised vectors).
    """
    U, psi0 = _c128(U), _c128(psi0)
    C = None if C is None else _c128(C)
    m = psi0.shape[-1]
    psi = np.empty_like(psi0)
    res = np.zeros((niter + 1, m))
    alph = np.zeros((niter, m), dtype=np.complex128)
    raw = np.empty_like(psi0) if return_history else None
    _load().or_mr(_dims(dims), m0, xi, _ptr(U), _ptr(C), m, niter, _ptr(psi0), _ptr(psi),
                  _ptr(res), _ptr(alph), _ptr(raw))
    if return_history:
        return psi, res, alph, raw
    return psi


def svd(A):
    """Thin SVD of a K x n block (K >= n): sigma (desc), U (K x n), V (n x n); A = U diag(s) V^dag."""
    A = _c128(A)
    K, n = A.shape
    s = np.empty(n)
    Uo = np.empty((K, n), dtype=np.complex128)
    Vo = np.empty((n, n), dtype=np.complex128)
    _load().or_svd(K, n, _ptr(A), _ptr(s), _ptr(Uo), _ptr(Vo))
    return s, Uo, Vo


def n_blocks(dims, block):
    return _vol(dims) // _vol(block)


def chiral_truncate(dims, block, psi, k, want_coarse_tv: bool = False):
    """Chiral split + per-block SVD + rank-k truncation (Eqs. 2, 4).

    Returns Uk[nblk][2][|blk|][2][3][k], sigma[nblk][2][m] (all m values) and,
    optionally, Sigma_k V_k^dag [nblk][2][k][m].
    """
    psi = _c128(psi)
    m = psi.shape[-1]
    nb = _vol(block)
    nblk = n_blocks(dims, block)
    if 6 * nb < m:
        raise ValueError("block too small: 6|Lambda| < m")
    Uk = np.empty((nblk, 2, nb, 2, 3, k), dtype=np.complex128)
    sig = np.empty((nblk, 2, m))
    ctv = np.empty((nblk, 2, k, m), dtype=np.complex128) if want_coarse_tv else None
    _load().or_chiral_truncate(_dims(dims), _dims(block), m, k, _ptr(psi), _ptr(Uk),
                               _ptr(sig), _ptr(ctv))
    if want_coarse_tv:
        return Uk, sig, ctv
    return Uk, sig


def prolongator(dims, block, Uk):
    """Site-major prolongator P[V][2][2][3][k] from block-major Uk (Eq. 5)."""
    Uk = _c128(Uk)
    k = Uk.shape[-1]
    P = np.empty((_vol(dims), 2, 2, 3, k), dtype=np.complex128)
    _load().or_prolongator(_dims(dims), _dims(block), k, _ptr(Uk), _ptr(P))
    return P


def coarse_dims(dims, block):
    return [int(dims[i]) // int(block[i]) for i in range(4)]


def coarsen(dims, block, m0, xi, U, C, P):
    """Galerkin coarse operator (Eq. 3) as X[nc][2k][2k], Y[nc][8][2k][2k]."""
    U, P = _c128(U), _c128(P)
    C = None if C is None else _c128(C)
    k = P.shape[-1]
    nc = _vol(coarse_dims(dims, block))
    X = np.empty((nc, 2 * k, 2 * k), dtype=np.complex128)
    Y = np.empty((nc, 8, 2 * k, 2 * k), dtype=np.complex128)
    _load().or_coarsen(_dims(dims), _dims(block), k, m0, xi, _ptr(U), _ptr(C), _ptr(P),
                       _ptr(X), _ptr(Y))
    return X, Y


def coarse_apply(cdims, X, Y, v):
    """D_c v for v[nc][2k][nrhs] on the periodic coarse lattice cdims."""
    X, Y, v = _c128(X), _c128(Y), _c128(v)
    two_k, nrhs = v.shape[1], v.shape[2]
    out = np.empty_like(v)
    _load().or_coarse_apply(_dims(cdims), two_k // 2, _ptr(X), _ptr(Y), nrhs, _ptr(v),
                            _ptr(out))
    return out


def gamma5(psi):
    """gamma_5 psi in the chiral basis (spins 0,1 -> +, spins 2,3 -> -)."""
    psi = _c128(psi)
    out = np.empty_like(psi)
    _load().or_gamma5(psi.shape[0], psi.shape[-1], _ptr(psi), _ptr(out))
    return out
