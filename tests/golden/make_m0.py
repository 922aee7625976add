"""Writes tests/golden/m0.json: the bare mass m0 of each workload, chosen (as
the workloads state) so that the smallest singular value of D is about 1e-2.

Uses only the oracle and the seeded input generators.  sigma_min(D) is the
smallest |eigenvalue| of the Hermitian gamma_5 D (gamma_5 is unitary), taken
from a dense eigensolve on a 4^4 lattice with the workload's eps, xi, c_sw
and gauge seed.  sigma_min(m0) dips to ~0 at the critical mass m_c; m0 is
taken on the branch m0 > m_c by golden-section search for m_c followed by
bisection on [m_c, 0.5].

    python tests/golden/make_m0.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import mg_inputs as G  # noqa: E402
import oracle as O  # noqa: E402

TARGET = 1e-2
DIMS = [4, 4, 4, 4]

# name: (eps, csw, xi, gauge seed) -- the workloads' gauge parameters
WORKLOADS = {
    "4^4 Wilson eps=0.3": (0.3, 0.0, 1.0, 0),
    "16^3x32 Wilson-clover eps=0.25": (0.25, 1.0, 1.0, 10),
    "32^3x64 aniso xi=3.5 eps=0.2": (0.2, 0.0, 3.5, 20),
    "Wilson eps=0.15": (0.15, 0.0, 1.0, 50),
    "Wilson eps=0.25": (0.25, 0.0, 1.0, 50),
    "Wilson eps=0.35": (0.35, 0.0, 1.0, 50),
}


def sigma_min(m0, U, C, xi):
    Dm = O.dense_D(DIMS, m0, xi, U, C)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), G.volume(DIMS))
    return float(np.abs(np.linalg.eigvalsh(g5[:, None] * Dm)).min())


def find_m0(eps, csw, xi, seed):
    U = G.gauge_field(DIMS, eps, seed)
    C = O.clover(DIMS, U, csw) if csw else None
    f = lambda m: sigma_min(m, U, C, xi)  # noqa: E731
    a, b = -1.0, 0.3
    gr = (np.sqrt(5) - 1) / 2
    c, d = b - gr * (b - a), a + gr * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(14):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = f(d)
    mc = 0.5 * (a + b)
    if f(mc) >= TARGET:
        return mc, f(mc), mc
    lo, hi = mc, 0.5
    for _ in range(22):
        mid = 0.5 * (lo + hi)
        if f(mid) < TARGET:
            lo = mid
        else:
            hi = mid
    return hi, f(hi), mc


def main():
    out = {"target_sigma_min": TARGET, "lattice": DIMS, "workloads": {}}
    for name, (eps, csw, xi, seed) in WORKLOADS.items():
        m0, smin, mc = find_m0(eps, csw, xi, seed)
        out["workloads"][name] = {"eps": eps, "csw": csw, "xi": xi, "gauge_seed": seed,
                                  "m0": round(m0, 6), "sigma_min": smin, "m_crit": round(mc, 6)}
        print(name, out["workloads"][name], flush=True)
    with open(os.path.join(HERE, "m0.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
