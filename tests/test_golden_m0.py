"""The stored bare masses (tests/golden/m0.json) against what they stand for:
each workload's m0 makes the smallest singular value of D about 1e-2 on the
4^4 lattice with that workload's eps, xi, c_sw and gauge seed, on the branch
above the critical mass.

The golden file was written from the smallest |eigenvalue| of the Hermitian
gamma_5 D; here sigma_min is taken by another route, the square root of the
smallest eigenvalue of D^dag D, so the check also pins the identity
sigma_min(D) = min |lambda(gamma_5 D)| (gamma_5 is unitary) that the golden
script relies on.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import mg_inputs as G
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "m0.json")) as fh:
    GOLD = json.load(fh)


@pytest.mark.parametrize("name", sorted(GOLD["workloads"]))
def test_stored_m0_gives_the_target_sigma_min(name):
    w = GOLD["workloads"][name]
    dims = GOLD["lattice"]
    U = G.gauge_field(dims, w["eps"], w["gauge_seed"])
    C = O.clover(dims, U, w["csw"]) if w["csw"] else None
    D = O.dense_D(dims, w["m0"], w["xi"], U, C)
    lam = scipy.linalg.eigh(D.conj().T @ D, eigvals_only=True, subset_by_index=[0, 0])[0]
    smin = float(np.sqrt(lam))
    # m0 is stored to 6 decimals and d sigma_min / d m0 is about 1 there
    assert abs(smin - GOLD["target_sigma_min"]) <= 2e-6, smin
    assert abs(smin - w["sigma_min"]) <= 2e-6
    # the branch above the critical mass (where sigma_min dips to ~0)
    assert w["m0"] > w["m_crit"]
    Dc = O.dense_D(dims, w["m_crit"], w["xi"], U, C)
    lam_c = scipy.linalg.eigh(Dc.conj().T @ Dc, eigvals_only=True, subset_by_index=[0, 0])[0]
    assert np.sqrt(max(lam_c, 0.0)) < smin
