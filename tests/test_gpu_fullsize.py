"""Parity at the full workload sizes, in the launch configuration bench.py times
(Level.run: smoother -> truncation -> prolongator -> coarsening, same problem
parameters), on outputs the FP64 oracle can compute one at a time:

  * smoother: the whole MR run of sampled vectors (the smoother acts on each
    right-hand side independently; Sec. 2, Eq. 1), per-vector relative
    2-norm error <= 2e-5 as in the small-lattice parity tests;
  * truncation: the SVD (FP64) of sampled blocks of the GPU's smoothed
    vectors (stage-isolated; Sec. 3, Eq. 4): retained singular values
    relative <= 1e-5, per-block projector error <= max(1e-5, Davis-Kahan
    bound), every block's flags clear, sigma positive and descending;
  * coarse operator: the Galerkin identity D_c v = P^dag D P v (Sec. 2, Eq. 3)
    for random coarse vectors v, with the oracle's D in FP64 and the GPU's P:
    |D_c v - P^dag D P v| <= 1e-6 |D| |v| (|D| bounded above by
    |m0 + sum w| + max|C| + 2 sum w) and <= 2e-5 |P^dag D P v|.

Workloads: 16^3x32 Wilson-clover (c_sw = 1, eps = 0.25, m' = 48, k = 24,
4^4 aggregates: 512 blocks) and 32^3x64 anisotropic Wilson (xi = 3.5,
eps = 0.2, m' = 64, k = 24, 4^3x8 aggregates: 4096 blocks), each in the FP32
plain path and in the mixed path (tensor-core contractions), which is held to
the same tolerances.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from gpu_common import M0, block_index, dk_bound, projector_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg  # noqa: E402

_build.build()

# name: dims, block, eps, csw, xi, m0, m', k, N, gauge seed, psi seed,
#       sampled vectors, sampled blocks
WORKLOADS = {
    "16^3x32 clover": ([16, 16, 16, 32], [4, 4, 4, 4], 0.25, 1.0, 1.0,
                       M0["16^3x32 Wilson-clover eps=0.25"], 48, 24, 20, 10, 11,
                       [0, 47], [0, 1, 77, 255, 256, 511]),
    "32^3x64 aniso": ([32, 32, 32, 64], [4, 4, 4, 8], 0.2, 0.0, 3.5,
                      M0["32^3x64 aniso xi=3.5 eps=0.2"], 64, 24, 20, 20, 21,
                      [5], [0, 1, 1000, 2047, 4095]),
}

_POOL = 16


def _psi0_device(dims, m, seed):
    """psi0(dims, m, seed) as complex64 on the device, drawn in site chunks."""
    V = G.volume(dims)
    out = torch.empty((V, 4, 3, m), dtype=torch.complex64, device="cuda")
    step = 1 << 15
    chunks = [(lo, min(V, lo + step)) for lo in range(0, V, step)]

    def draw(r):
        return r, G.psi0_sites(dims, m, seed, r[0], r[1]).astype(np.complex64)

    with cf.ThreadPoolExecutor(_POOL) as ex:
        for (lo, hi), a in ex.map(draw, chunks):
            out[lo:hi].copy_(torch.from_numpy(a))
    return out


def _block_sites(dims, block, j):
    """Sites of block j in the block's local lexicographic order."""
    Lc = [dims[i] // block[i] for i in range(4)]
    jc = []
    t = j
    for i in range(4):
        jc.append(t % Lc[i])
        t //= Lc[i]
    loc = np.arange(int(np.prod(block)))
    xs = []
    t = loc.copy()
    for i in range(4):
        xs.append(jc[i] * block[i] + t % block[i])
        t //= block[i]
    return xs[0] + dims[0] * (xs[1] + dims[1] * (xs[2] + dims[2] * xs[3]))


_inputs = {}
_runs = {}
PRECISIONS = {"fp32": mg.MG_PREC_FP32, "mixed": mg.MG_PREC_MIXED}


def _run(name, precision="fp32"):
    key = (name, precision)
    if key in _runs:
        return _runs[key]
    dims, block, eps, csw, xi, m0, m, k, N, gs, ps, cols, blocks = WORKLOADS[name]
    if name not in _inputs:
        U = G.round_to_c64(G.gauge_field(dims, eps, gs, threads=_POOL))
        C = G.round_to_c64(O.clover(dims, U, csw)) if csw else None
        Ud = torch.from_numpy(U.astype(np.complex64)).cuda()
        Cd = torch.from_numpy(C.astype(np.complex64).reshape(-1, 2, 6, 6)).cuda() if csw else None
        _inputs[name] = (U, C, Ud, Cd, _psi0_device(dims, m, ps))
    U, C, Ud, Cd, p0 = _inputs[name]
    prob = mg.Problem(dims=dims, block=block, m0=m0, n_vec=m, k=k, mr_iters=N, csw=csw, xi=xi,
                      precision=PRECISIONS[precision])
    lv = mg.Level.allocate(prob, Ud, Cd, p0)
    lv.run()
    torch.cuda.synchronize()
    mg.mg_sync_status()
    lv.ws_smooth = lv.ws_trunc = None  # the tests read only the level's outputs
    torch.cuda.empty_cache()
    _runs[key] = dict(prob=prob, U=U, C=C, lv=lv, dims=dims, block=block, m0=m0, xi=xi,
                      m=m, k=k, N=N, ps=ps, cols=cols, blocks=blocks, csw=csw)
    return _runs[key]


@pytest.mark.parametrize("precision", list(PRECISIONS))
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fullsize_smoother_sampled_vectors(name, precision):
    r = _run(name, precision)
    cols = r["cols"]
    p0 = G.round_to_c64(G.psi0_columns(r["dims"], r["m"], r["ps"], cols))
    want = O.mr(r["dims"], r["m0"], r["xi"], r["U"], r["C"], p0, r["N"])
    got = r["lv"].psi[..., cols].cpu().numpy().astype(np.complex128)
    for i in range(len(cols)):
        err = np.linalg.norm(got[..., i] - want[..., i]) / np.linalg.norm(want[..., i])
        assert err <= 2e-5, (cols[i], err)


@pytest.mark.parametrize("precision", list(PRECISIONS))
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fullsize_truncation_sampled_blocks(name, precision):
    r = _run(name, precision)
    lv, k = r["lv"], r["k"]
    flags = lv.flags.cpu().numpy()
    assert np.all(flags == 0)
    sig = lv.sigma.cpu().numpy()
    assert np.all(sig > 0) and np.all(np.diff(sig, axis=-1) <= 0)
    for j in r["blocks"]:
        sites = torch.from_numpy(_block_sites(r["dims"], r["block"], j)).cuda()
        blk = lv.psi.index_select(0, sites).cpu().numpy().astype(np.complex128)
        Ukj = lv.Uk[j].cpu().numpy().astype(np.complex128)
        for al in range(2):
            A = blk[:, 2 * al:2 * al + 2].reshape(-1, r["m"])
            so, Uo, _ = O.svd(A)
            np.testing.assert_allclose(sig[j, al], so[:k], rtol=1e-5)
            e = projector_error(Ukj[al].reshape(-1, k), Uo[:, :k])
            assert e <= max(1e-5, float(dk_bound(so, k))), (j, al, e)


@pytest.mark.parametrize("precision", list(PRECISIONS))
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_fullsize_galerkin_identity(name, precision):
    r = _run(name, precision)
    lv, prob, k = r["lv"], r["prob"], r["k"]
    dims, block = r["dims"], r["block"]
    nc = prob.n_blocks
    v = G.round_to_c64(G.coarse_vectors(nc, 2 * k, 2, 9))
    vd = torch.from_numpy(v.astype(np.complex64)).cuda()
    out = torch.empty_like(vd)
    mg.mg_coarse_apply(prob, lv.X, lv.Y, vd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.complex128)
    # P v and P^dag (D P v) in FP64 (torch on the device: data movement and
    # sums only), D by the oracle
    jx = torch.from_numpy(block_index(dims, block)).cuda()  # block of every site
    P = lv.P.to(torch.complex128)  # [V][2][2][3][k]
    V = P.shape[0]
    w = [1.0, 1.0, 1.0, 1.0 / r["xi"]]
    cmax = float(np.abs(r["C"]).max()) * 6 if r["C"] is not None else 0.0
    dnorm = abs(r["m0"] + sum(w)) + cmax + 2 * sum(w)
    for c in range(v.shape[-1]):
        vc = torch.from_numpy(v[..., c]).cuda().reshape(nc, 2, k)[jx]  # [V][2][k]
        z = torch.einsum("xascI,xaI->xasc", P, vc).reshape(V, 4, 3, 1).cpu().numpy()
        Dz = O.apply_D(dims, r["m0"], r["xi"], r["U"], r["C"], z)
        Dzd = torch.from_numpy(Dz.reshape(V, 2, 2, 3)).cuda()
        loc = torch.einsum("xascI,xasc->xaI", P.conj(), Dzd).reshape(V, 2 * k)
        ref = torch.zeros((nc, 2 * k), dtype=torch.complex128, device="cuda")
        ref.index_add_(0, jx, loc)
        ref = ref.cpu().numpy()
        err = np.linalg.norm(got[..., c] - ref)
        assert err <= 1e-6 * dnorm * np.linalg.norm(v[..., c]), (c, err)
        assert err <= 2e-5 * np.linalg.norm(ref), (c, err / np.linalg.norm(ref))
