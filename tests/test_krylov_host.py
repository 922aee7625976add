"""The host-side Arnoldi bookkeeping of mg_solve (csrc/mg_krylov.h: Hessenberg
columns from the two Gram-Schmidt passes, Givens rotations, residual
estimates, triangular solve), compiled on the host and fed inner products
computed here in FP64, against numpy's least-squares solution of
min |beta e_1 - H y| after every step.  Columns are independent systems; one
has an exact breakdown (|w| = 0 at step 2) and one a zero right-hand side."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def kh(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("kh") / "libkh.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           os.path.join(HERE, "krylov_host.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.kh_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
    return lib


def _arnoldi(A, b, m):
    """CGS2 Arnoldi in FP64: per step the two passes' coefficients and |w|^2."""
    beta = np.linalg.norm(b)
    V = [b / beta]
    steps = []
    for j in range(m):
        w = A @ V[j]
        h1 = np.array([np.vdot(V[i], w) for i in range(j + 1)])
        w = w - sum(h1[i] * V[i] for i in range(j + 1))
        h2 = np.array([np.vdot(V[i], w) for i in range(j + 1)])
        w = w - sum(h2[i] * V[i] for i in range(j + 1))
        hn2 = np.vdot(w, w).real
        steps.append((h1, h2, hn2))
        V.append(w / np.sqrt(hn2))
    return beta, steps


def test_krylov_bookkeeping_matches_least_squares(kh):
    rng = np.random.default_rng(7)
    n, m, K = 4, 6, 12
    A = rng.standard_normal((K, K)) + 1j * rng.standard_normal((K, K)) + 3 * np.eye(K)
    cols = []
    for c in range(n):
        b = rng.standard_normal(K) + 1j * rng.standard_normal(K)
        cols.append(_arnoldi(A, b, m))
    # column 2: exact breakdown at step 2; column 3: zero right-hand side
    beta2, st2 = cols[2]
    st2 = list(st2)
    st2[2] = (st2[2][0], st2[2][1], 0.0)
    cols[2] = (beta2, st2)
    cols[3] = (0.0, cols[3][1])
    stride = (2 * (m + 1) + 1) * n
    hs = np.zeros((m, stride), dtype=np.complex128)
    for c, (_, st) in enumerate(cols):
        for j, (h1, h2, hn2) in enumerate(st):
            hs[j, np.arange(j + 1) * n + c] = h1
            hs[j, (m + 1 + np.arange(j + 1)) * n + c] = h2
            hs[j, 2 * (m + 1) * n + c] = hn2
    beta2 = np.array([cb ** 2 for cb, _ in cols], dtype=np.complex128)
    hsv = np.ascontiguousarray(hs).view(np.float64)
    y = np.zeros((m, n), dtype=np.complex128)
    res = np.zeros((m, n))
    kc = np.zeros(n, dtype=np.int32)
    kh.kh_run(m, n, m, beta2.ctypes.data, hsv.ctypes.data, y.ctypes.data, res.ctypes.data,
              kc.ctypes.data)
    assert list(kc) == [-1, -1, 3, 0]
    for c, (beta, st) in enumerate(cols):
        if beta == 0:
            assert np.all(y[:, c] == 0)
            continue
        H = np.zeros((m + 1, m), dtype=np.complex128)
        for j, (h1, h2, hn2) in enumerate(st):
            H[:j + 1, j] = h1 + h2
            H[j + 1, j] = np.sqrt(hn2)
        k = m if kc[c] < 0 else kc[c]
        for j in range(k):
            g = np.zeros(j + 2, dtype=np.complex128)
            g[0] = beta
            yj, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], g, rcond=None)
            est = np.linalg.norm(g - H[:j + 2, :j + 1] @ yj)
            assert abs(res[j, c] - est) <= 1e-12 * beta, (c, j)
        g = np.zeros(k + 1, dtype=np.complex128)
        g[0] = beta
        yk, *_ = np.linalg.lstsq(H[:k + 1, :k], g, rcond=None)
        np.testing.assert_allclose(y[:k, c], yk, rtol=1e-10, atol=1e-12 * np.abs(yk).max())
        assert np.all(y[k:, c] == 0)
