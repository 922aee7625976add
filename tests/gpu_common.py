"""Helpers shared by the GPU tests: workload definitions, host<->device copies
and the basis-invariant comparison quantities."""
import json
import os

import numpy as np

import mg_inputs as G

HERE = os.path.dirname(os.path.abspath(__file__))

with open(os.path.join(HERE, "golden", "m0.json")) as fh:
    M0 = {k: v["m0"] for k, v in json.load(fh)["workloads"].items()}

# FP32 unit roundoff
U32 = 2.0 ** -24


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def to_host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def projector_error(Ua, Ub):
    """|Ua Ua^dag - Ub Ub^dag|_F for K x k bases without forming K x K matrices:
    |Ua^dag Ua|_F^2 + |Ub^dag Ub|_F^2 - 2 |Ua^dag Ub|_F^2 (exact for any Ua, Ub;
    the shortcut 2k - 2|Ua^dag Ub|^2 needs exactly orthonormal bases)."""
    aa = np.linalg.norm(Ua.conj().T @ Ua) ** 2
    bb = np.linalg.norm(Ub.conj().T @ Ub) ** 2
    ab = np.linalg.norm(Ua.conj().T @ Ub) ** 2
    return np.sqrt(max(0.0, aa + bb - 2 * ab))


def dk_bound(sig, k, c=16.0):
    """Davis-Kahan-type bound of the projector change caused by FP32-level
    perturbations: c * 2^-24 * |A|_F / (sigma_k - sigma_{k+1}), per block."""
    frob = np.sqrt(np.sum(sig ** 2, axis=-1))
    gap = sig[..., k - 1] - (sig[..., k] if sig.shape[-1] > k else 0.0)
    return c * U32 * frob / np.maximum(gap, 1e-300)


def c64_inputs(dims, eps, gauge_seed, m, psi_seed, csw, oracle):
    """Gauge field, clover and starts rounded to complex64, so that the FP64
    oracle and the FP32 GPU path see exactly the same numbers."""
    U = G.round_to_c64(G.gauge_field(dims, eps, gauge_seed))
    C = G.round_to_c64(oracle.clover(dims, U, csw)) if csw else None
    p0 = G.round_to_c64(G.psi0(dims, m, psi_seed))
    return U, C, p0


def block_index(dims, block):
    """Block index of every site (lexicographic coarse coordinate)."""
    V = int(np.prod(dims))
    s = np.arange(V)
    x = []
    for L in dims:
        x.append(s % L)
        s = s // L
    Lc = [dims[i] // block[i] for i in range(4)]
    xc = [x[i] // block[i] for i in range(4)]
    return xc[0] + Lc[0] * (xc[1] + Lc[1] * (xc[2] + Lc[2] * xc[3]))


def restrict(dims, block, P, z):
    """R z = P^dag z for z[V][4][3] (one vector) -> [nc][2k]."""
    V, k = P.shape[0], P.shape[-1]
    j = block_index(dims, block)
    nc = V // int(np.prod(block))
    zz = z.reshape(V, 2, 2, 3)
    loc = np.einsum("xasci,xasc->xai", P.conj(), zz).reshape(V, 2 * k)
    out = np.zeros((nc, 2 * k), dtype=np.complex128)
    np.add.at(out, j, loc)
    return out


def prolong(dims, block, P, v):
    """P v for v[nc][2k] -> [V][4][3]."""
    V, k = P.shape[0], P.shape[-1]
    j = block_index(dims, block)
    vv = v[j].reshape(V, 2, k)
    return np.einsum("xasci,xai->xasc", P, vv).reshape(V, 4, 3)
