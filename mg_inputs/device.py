"""The seeded input generator of ``mg_inputs`` on a torch device.

The same counter-based definition (SplitMix64 of (seed, stream, counter),
53-bit uniforms, Box-Muller's cosine branch), written with torch int64
arithmetic so that a server can draw a request's links and starts on the GPU
instead of on the host.  Uniforms are bit-identical to ``mg_inputs.uniforms``;
normals agree to the last few ulps (the device's log/cos/sqrt); links are
exp(i eps H) by a Taylor series of elementwise products in complex128.

Two's-complement int64 multiplication and addition wrap modulo 2^64 exactly
like uint64 arithmetic; right shifts are done arithmetically and masked, which
gives the logical shift of the unsigned value.
"""
from __future__ import annotations

import numpy as np

from . import (STREAM_GAUGE, STREAM_PSI0, gell_mann, stream_key)


def _s64(u: int) -> int:
    """uint64 constant as the int64 with the same bits."""
    u &= 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= (1 << 63) else u


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_M1 = _s64(0xBF58476D1CE4E5B9)
_M2 = _s64(0x94D049BB133111EB)


def _shr(z, n: int):
    """Logical right shift of int64 bits."""
    return (z >> n) & ((1 << (64 - n)) - 1)


def splitmix64_t(x):
    """SplitMix64 finaliser of x + golden gamma on an int64 tensor (wrapping)."""
    z = x + _GOLDEN
    z = (z ^ _shr(z, 30)) * _M1
    z = (z ^ _shr(z, 27)) * _M2
    return z ^ _shr(z, 31)


def uniforms_t(seed: int, stream: int, start: int, count: int, device="cuda"):
    """Uniform doubles in (0, 1) for counters start .. start+count-1 (float64 tensor)."""
    import torch
    key = _s64(int(stream_key(seed, stream)))
    ctr = torch.arange(start, start + count, dtype=torch.int64, device=device)
    bits = splitmix64_t(ctr + key)
    return (_shr(bits, 11).to(torch.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals_t(seed: int, stream: int, start: int, count: int, device="cuda"):
    """Standard normal doubles n_start .. n_{start+count-1} (float64 tensor)."""
    import torch
    u = uniforms_t(seed, stream, 2 * start, 2 * count, device).reshape(count, 2)
    return torch.sqrt(-2.0 * torch.log(u[:, 0])) * torch.cos(2.0 * np.pi * u[:, 1])


def _mm3(a, b):
    """Batched 3 x 3 products as nine elementwise sums (no batched GEMM calls)."""
    import torch
    return torch.stack([torch.stack([a[:, i, 0] * b[:, 0, j] + a[:, i, 1] * b[:, 1, j] +
                                     a[:, i, 2] * b[:, 2, j] for j in range(3)], dim=-1)
                        for i in range(3)], dim=-2)


def _expi(H, eps: float, order: int = 22):
    """exp(i eps H) for a batch of 3 x 3 Hermitian H by its Taylor series.
    |eps H|_2 stays below ~2 for these inputs, where order 22 leaves a remainder
    below 1e-16 (2^23 / 23!), so the result matches the host's eigendecomposition
    to rounding."""
    import torch
    X = 1j * eps * H
    term = torch.eye(3, dtype=H.dtype, device=H.device).expand_as(H).clone()
    U = term.clone()
    for j in range(1, order + 1):
        term = _mm3(term, X) / j
        U = U + term
    return U


def gauge_field_t(dims, eps: float, seed: int, device="cuda", chunk: int = 1 << 20):
    """mg_inputs.gauge_field on the device: U[V][4][3][3] complex128."""
    import torch
    V = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    n = 4 * V
    lam = torch.from_numpy(gell_mann() / 2.0).to(device)
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        h = normals_t(seed, STREAM_GAUGE, 8 * lo, 8 * (hi - lo), device).reshape(hi - lo, 8)
        H = torch.einsum("na,aij->nij", h.to(torch.complex128), lam)
        out[lo:hi] = _expi(H, eps)
    return out.reshape(V, 4, 3, 3)


def psi0_t(dims, m: int, seed: int, device="cuda", dtype=None, chunk: int = 1 << 24):
    """mg_inputs.psi0 on the device: [V][4][3][m], complex128 (or dtype)."""
    import torch
    V = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    n = V * 12 * m
    dtype = dtype or torch.complex128
    out = torch.empty(n, dtype=dtype, device=device)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        g = normals_t(seed, STREAM_PSI0, 2 * lo, 2 * (hi - lo), device)
        out[lo:hi] = torch.complex(g[0::2], g[1::2]).to(dtype)
    return out.reshape(V, 4, 3, m)
