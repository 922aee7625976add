"""Evidence for the precision reading (why the FP32-accurate mixed path keeps
the smoother's fields in FP32): the minimal-residual smoother (paper Sec. 2,
Eq. 1) is run in FP64 arithmetic with its three fields (psi, r, w) rounded to
a storage precision after every iteration, chosen per iteration, and the 16
smallest |eigenvalues| of sigma_3 D_c of the resulting coarse operator are
compared with the all-FP64 run.  The operator, truncation and coarsening are
the oracle's.  Storage rounding anywhere before the last iteration is
amplified by the rest of the MR trajectory (the per-vector step lengths react
to it): FP16 storage in the first two iterations alone gives the same
coarse-spectrum error as FP16 everywhere, about 1e-3 relative and far above
the FP32 error, while FP16 in the last iteration only stays near the FP32
level.  So no schedule that keeps FP16 in a meaningful part of the smoother
reaches the FP32 path's accuracy.
"""
import json
import os

import numpy as np
import pytest

import mg_inputs as G
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def setting():
    with open(os.path.join(HERE, "golden", "m0.json")) as fh:
        m0 = json.load(fh)["workloads"]["32^3x64 aniso xi=3.5 eps=0.2"]["m0"]
    d, b, k, m, N, xi = [4, 4, 4, 8], [2, 2, 2, 4], 8, 16, 20, 3.5
    U = G.round_to_c64(G.gauge_field(d, 0.2, 20))
    p0 = G.round_to_c64(G.psi0(d, m, 21))
    return dict(d=d, b=b, k=k, m=m, N=N, xi=xi, m0=m0, U=U, p0=p0)


def _round(x, prec):
    if prec == "f64":
        return x
    if prec == "f32":
        return x.astype(np.complex64).astype(np.complex128)
    return x.real.astype(np.float16).astype(np.float64) + \
        1j * x.imag.astype(np.float16).astype(np.float64)


def _mr(s, precs):
    """MR with storage precision precs[t] after iteration t (precs[0]: the start)."""
    D = lambda x: O.apply_D(s["d"], s["m0"], s["xi"], s["U"], None, x)  # noqa: E731
    p0, m = s["p0"], s["m"]
    # per-vector unit-RMS scale first (as an FP16 store needs; MR is scale invariant)
    psi = _round(p0 / np.sqrt(np.sum(np.abs(p0) ** 2, axis=(0, 1, 2)) / (p0.size / m)), precs[0])
    r = _round(-D(psi), precs[0])
    for t in range(s["N"]):
        w = _round(D(r), precs[t])
        a = np.sum(np.conj(w) * r, axis=(0, 1, 2)) / np.sum(np.abs(w) ** 2, axis=(0, 1, 2))
        psi = _round(psi + a * r, precs[t + 1])
        r = _round(r - a * w, precs[t + 1])
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2, axis=(0, 1, 2)))


def _lowest16(s, psi):
    d, b, k = s["d"], s["b"], s["k"]
    Uk, _ = O.chiral_truncate(d, b, psi, k)
    P = O.prolongator(d, b, Uk)
    X, Y = O.coarsen(d, b, s["m0"], s["xi"], s["U"], None, P)
    cd = O.coarse_dims(d, b)
    nc = int(np.prod(cd))
    n = nc * 2 * k
    Dc = O.coarse_apply(cd, X, Y, np.eye(n).reshape(nc, 2 * k, n)).reshape(n, n)
    H = np.tile(np.r_[np.ones(k), -np.ones(k)], nc)[:, None] * Dc
    return np.sort(np.abs(np.linalg.eigvalsh((H + H.conj().T) / 2)))[:16]


def test_fp16_storage_before_the_last_iteration_misses_fp32_accuracy(setting):
    s = setting
    N = s["N"]
    ref = _lowest16(s, O.mr(s["d"], s["m0"], s["xi"], s["U"], None, s["p0"], N))
    err = {}
    for name, precs in {"f32": ["f32"] * (N + 1), "f16": ["f16"] * (N + 1),
                        "f16 first 2": ["f16"] * 3 + ["f32"] * (N - 2),
                        "f16 last 1": ["f32"] * N + ["f16"]}.items():
        lo = _lowest16(s, _mr(s, precs))
        err[name] = np.max(np.abs(lo - ref) / ref)
    assert err["f32"] <= 1e-5, err
    assert err["f16"] >= 1e-3, err
    assert err["f16 first 2"] >= 1e-3, err       # early FP16 rounding is amplified
    assert err["f16 first 2"] >= 0.5 * err["f16"], err
    assert err["f16 last 1"] <= 1e-4, err         # late rounding is not
