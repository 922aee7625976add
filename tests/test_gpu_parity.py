"""GPU (sm_103a, through the C ABI) versus the FP64 oracle, stage by stage and
end to end, on identical complex64-representable inputs.

Tolerances (FP32 path):
  * clover, prolongator pack: the clover is FP32 arithmetic on O(1) entries
    (abs 2e-6); the pack is pure data movement (bit exact).
  * smoother: each vector's relative 2-norm error <= 2e-5 (N FP32 dslash
    passes, each ~1e-7 relative, with per-vector step lengths in FP64).
  * truncation: retained singular values relative <= 1e-5; per-block
    projector |U U^dag - U^ U^dag|_F <= max(1e-5, Davis-Kahan bound of an
    FP32-level perturbation, see gpu_common.dk_bound); P_j^dag P_j = 1 to 1e-5.
  * coarse operator: |X - X^|, |Y - Y^| <= 1e-5 * max|X^|.
  * end to end: the 16 smallest |eigenvalues| of sigma_3 D_c relative 1e-5
    (with the degenerate-gap caveat above), and the Galerkin identity
    |P D_c P^dag z - P P^dag D P P^dag z| / |D| |z| <= 1e-6.
"""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from conftest import dense_coarse, dense_P
from gpu_common import (M0, c64_inputs, dk_bound, projector_error, prolong, restrict,
                        to_dev, to_host)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg  # noqa: E402

_build.build()

# (name, dims, block, eps, csw, xi, m0, m, k, N, gauge seed, psi seed)
CASES = {
    "4^4 Wilson m'=8 k=4 (workload 1)": ([4, 4, 4, 4], [2, 2, 2, 2], 0.3, 0.0, 1.0,
                                         M0["4^4 Wilson eps=0.3"], 8, 4, 10, 0, 1),
    "8^4 clover m'=48 k=24": ([8, 8, 8, 8], [4, 4, 4, 4], 0.25, 1.0, 1.0,
                              M0["16^3x32 Wilson-clover eps=0.25"], 48, 24, 20, 10, 11),
    "8^3x16 aniso m'=64 k=24": ([8, 8, 8, 16], [4, 4, 4, 8], 0.2, 0.0, 3.5,
                                M0["32^3x64 aniso xi=3.5 eps=0.2"], 64, 24, 6, 20, 21),
    "ragged 6x4x2x6 m'=12 k=5": ([6, 4, 2, 6], [2, 2, 2, 3], 0.3, 1.0, 1.3, -0.1, 12, 5, 4, 3, 4),
}

_cache = {}


def _case(name):
    """Inputs and the oracle chain of one case (computed once)."""
    if name in _cache:
        return _cache[name]
    dims, block, eps, csw, xi, m0, m, k, N, gs, ps = CASES[name]
    U, C, p0 = c64_inputs(dims, eps, gs, m, ps, csw, O)
    prob = mg.Problem(dims=dims, block=block, m0=m0, n_vec=m, k=k, mr_iters=N, csw=csw, xi=xi)
    psi = O.mr(dims, m0, xi, U, C, p0, N)
    _cache[name] = dict(prob=prob, U=U, C=C, p0=p0, psi=psi, dims=dims, block=block, m0=m0,
                        xi=xi, k=k, m=m, csw=csw)
    return _cache[name]


def _dev(c):
    U = to_dev(c["U"])
    C = to_dev(c["C"].reshape(-1, 2, 6, 6)) if c["C"] is not None else None
    return U, C


@pytest.mark.parametrize("name", list(CASES))
def test_clover_field(name):
    c = _case(name)
    if not c["csw"]:
        pytest.skip("Wilson case")
    U, _ = _dev(c)
    Cg = torch.empty(mg.shape_C(c["prob"]), dtype=torch.complex64, device="cuda")
    mg.mg_clover_field(c["prob"], U, Cg)
    torch.cuda.synchronize()
    np.testing.assert_allclose(to_host(Cg), c["C"], atol=2e-6)


@pytest.mark.parametrize("name", list(CASES))
def test_dirac_apply(name):
    """The multi-right-hand-side Wilson(-clover) operator against the oracle's."""
    c = _case(name)
    p = c["prob"]
    U, C = _dev(c)
    vin = to_dev(c["p0"])
    out = torch.empty_like(vin)
    mg.mg_apply_dirac(p, U, C, vin, out, mg.workspace(p, mg.MG_CALL_SMOOTH))
    torch.cuda.synchronize()
    ref = O.apply_D(c["dims"], c["m0"], c["xi"], c["U"], c["C"], c["p0"])
    got = to_host(out)
    err = np.linalg.norm((got - ref).reshape(-1, c["m"]), axis=0) / \
        np.linalg.norm(ref.reshape(-1, c["m"]), axis=0)
    assert err.max() <= 1e-6, err.max()


@pytest.mark.parametrize("prec", [mg.MG_PREC_FP32, mg.MG_PREC_MIXED_FP16])
def test_odd_volume_layout_tail(prec):
    """A volume that is not a multiple of the 4-site tiles of the interface <->
    slab transposes (3^3 x 5: 135 sites, a last tile of 3) and a timeslice of
    27 sites (one ragged patch): D psi and 3 MR iterations against the oracle,
    for FP32 and FP16 slab storage."""
    dims, m0, xi, m = [3, 3, 3, 5], -0.1, 1.0, 8
    U = G.round_to_c64(G.gauge_field(dims, 0.3, 31))
    p0 = G.round_to_c64(G.psi0(dims, m, 32))
    p = mg.Problem(dims=dims, block=[3, 3, 3, 5], m0=m0, n_vec=m, k=4, mr_iters=3, xi=xi,
                   precision=prec)
    ws = mg.workspace(p, mg.MG_CALL_SMOOTH)
    out = torch.empty(p0.shape, dtype=torch.complex64, device="cuda")
    mg.mg_apply_dirac(p, to_dev(U), None, to_dev(p0), out, ws)
    mg.mg_sync_status()
    ref = O.apply_D(dims, m0, xi, U, None, p0)
    err = np.linalg.norm((to_host(out) - ref).reshape(-1, m), axis=0) / \
        np.linalg.norm(ref.reshape(-1, m), axis=0)
    assert err.max() <= (1e-6 if prec == mg.MG_PREC_FP32 else 4 * U16), err.max()
    if prec == mg.MG_PREC_FP32:
        mg.mg_smooth_testvecs(p, to_dev(U), None, to_dev(p0), out, ws)
        mg.mg_sync_status()
        ref = O.mr(dims, m0, xi, U, None, p0, 3)
        err = np.linalg.norm((to_host(out) - ref).reshape(-1, m), axis=0)
        assert err.max() <= 2e-5, err.max()


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_smoother_iteration_counts(N):
    """psi's update waits one iteration and takes two terms; odd and even N end
    with one or two pending terms (and N = 1 with none of the two-term steps)."""
    c = _case("4^4 Wilson m'=8 k=4 (workload 1)")
    p0 = c["p0"]
    p = mg.Problem(dims=c["dims"], block=c["block"], m0=c["m0"], n_vec=c["m"], k=c["k"],
                   mr_iters=N, csw=c["csw"], xi=c["xi"])
    U, C = _dev(c)
    psi = torch.empty(p0.shape, dtype=torch.complex64, device="cuda")
    mg.mg_smooth_testvecs(p, U, C, to_dev(p0), psi, mg.workspace(p, mg.MG_CALL_SMOOTH))
    mg.mg_sync_status()
    ref = O.mr(c["dims"], c["m0"], c["xi"], c["U"], c["C"], p0, N)
    err = np.linalg.norm((to_host(psi) - ref).reshape(-1, c["m"]), axis=0)
    assert err.max() <= 2e-5, (N, err.max())


@pytest.mark.parametrize("name", list(CASES))
def test_smoother(name):
    c = _case(name)
    p = c["prob"]
    U, C = _dev(c)
    psi0 = to_dev(c["p0"])
    psi = torch.empty_like(psi0)
    ws = mg.workspace(p, mg.MG_CALL_SMOOTH)
    mg.mg_smooth_testvecs(p, U, C, psi0, psi, ws)
    torch.cuda.synchronize()
    got = to_host(psi)
    ref = c["psi"]
    err = np.linalg.norm((got - ref).reshape(-1, c["m"]), axis=0)
    assert np.all(np.isfinite(got))
    assert err.max() <= 2e-5, err.max()
    # the input is not modified
    np.testing.assert_array_equal(to_host(psi0), c["p0"])
    # in place (psi aliasing psi0) gives the same bits
    mg.mg_smooth_testvecs(p, U, C, psi0, psi0, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_host(psi0), got)


def _with_precision(p, precision):
    return mg.Problem(dims=p.dims, block=p.block, m0=p.m0, n_vec=p.n_vec, k=p.k,
                      mr_iters=p.mr_iters, csw=p.csw, xi=p.xi, precision=precision)


def _truncate(c, psi_host, want_ctv=False, precision=None):
    p = c["prob"] if precision is None else _with_precision(c["prob"], precision)
    psi = to_dev(psi_host)
    Uk = torch.empty(mg.shape_Uk(p), dtype=torch.complex64, device="cuda")
    sig = torch.empty(mg.shape_sigma(p), dtype=torch.float64, device="cuda")
    flags = torch.full((p.n_blocks, 2), -1, dtype=torch.int32, device="cuda")
    ctv = torch.empty((p.n_blocks, 2, p.k, p.n_vec), dtype=torch.complex64,
                      device="cuda") if want_ctv else None
    ws = mg.workspace(p, mg.MG_CALL_TRUNCATE)
    mg.mg_chiral_truncate(p, psi, Uk, sig, ctv, flags, ws)
    torch.cuda.synchronize()
    out = (to_host(Uk), sig.cpu().numpy(), flags.cpu().numpy())
    if want_ctv:
        out = out + (to_host(ctv),)
    return out


@pytest.mark.parametrize("precision", [mg.MG_PREC_FP32, mg.MG_PREC_MIXED])
@pytest.mark.parametrize("name", list(CASES))
def test_truncation(name, precision):
    """Stage-isolated: the oracle's smoothed vectors (rounded to complex64) in.
    The mixed path (tensor-core Grams and products with FP16 hi/lo operands)
    is held to the FP32 path's tolerances."""
    c = _case(name)
    k = c["k"]
    psi32 = G.round_to_c64(c["psi"])
    Uk, sig, flags, ctv = _truncate(c, psi32, want_ctv=True, precision=precision)
    assert np.all(flags == 0), flags
    Ur, sr, cr = O.chiral_truncate(c["dims"], c["block"], psi32, k, want_coarse_tv=True)
    np.testing.assert_allclose(sig, sr[..., :k], rtol=1e-5)
    nblk = Uk.shape[0]
    bound = dk_bound(sr, k)
    for j in range(nblk):
        for al in range(2):
            Ug = Uk[j, al].reshape(-1, k)
            Uo = Ur[j, al].reshape(-1, k)
            np.testing.assert_allclose(Ug.conj().T @ Ug, np.eye(k), atol=1e-5)
            e = projector_error(Ug, Uo)
            assert e <= max(1e-5, bound[j, al]), (j, al, e, bound[j, al])
            # Sigma_k V_k^dag: U_k (Sigma_k V_k^dag) is the same rank-k approximation
            A_g = Ug @ ctv[j, al]
            A_o = Uo @ cr[j, al]
            assert np.linalg.norm(A_g - A_o) <= 1e-5 * np.linalg.norm(A_o) + \
                2 * bound[j, al] * np.linalg.norm(A_o)


@pytest.mark.parametrize("precision", [mg.MG_PREC_FP32, mg.MG_PREC_MIXED])
def test_conventional_setup_k_equals_m(precision):
    """k = m': no truncation, the conventional per-block orthonormalisation of
    the chirally split vectors (Sec. 2, the paper's comparison setup).  U U^dag
    must be the orthogonal projector onto each block-chirality's range (the
    oracle's k = m' case, pinned on the CPU against that projector), with all
    m' singular values, and the coarse operator must keep sigma_3-hermiticity.
    The mixed path takes its first Gram in BF16 on the tensor cores; the
    second, FP32 CholeskyQR pass gives the same orthonormal basis."""
    dims, block, m = [8, 8, 8, 8], [4, 4, 4, 4], 32
    p = mg.Problem(dims=dims, block=block, m0=-0.1, n_vec=m, k=m, mr_iters=1,
                   precision=precision)
    psi = G.round_to_c64(G.psi0(dims, m, 17))
    Uk, sig, flags = _truncate({"prob": p}, psi)
    assert np.all(flags == 0)
    Ur, sr = O.chiral_truncate(dims, block, psi, m)
    np.testing.assert_allclose(sig, sr[..., :m], rtol=1e-5)
    for j in range(Uk.shape[0]):
        for al in range(2):
            Ug = Uk[j, al].reshape(-1, m)
            np.testing.assert_allclose(Ug.conj().T @ Ug, np.eye(m), atol=1e-5)
            assert projector_error(Ug, Ur[j, al].reshape(-1, m)) <= 1e-5
    U = G.round_to_c64(G.gauge_field(dims, 0.25, 3))
    P = torch.empty(mg.shape_P(p), dtype=torch.complex64, device="cuda")
    X = torch.empty(mg.shape_X(p), dtype=torch.complex64, device="cuda")
    Y = torch.empty(mg.shape_Y(p), dtype=torch.complex64, device="cuda")
    mg.mg_build_prolongator(p, to_dev(Uk), P)
    mg.mg_coarsen(p, to_dev(U), None, P, X, Y)
    torch.cuda.synchronize()
    Dc = dense_coarse(O.coarse_dims(dims, block), to_host(X), to_host(Y))
    s3 = np.tile(np.r_[np.ones(m), -np.ones(m)], Dc.shape[0] // (2 * m))
    H = s3[:, None] * Dc
    assert np.linalg.norm(H - H.conj().T) <= 1e-5 * np.linalg.norm(H)


@pytest.mark.parametrize("name", list(CASES))
def test_prolongator_pack_exact(name):
    c = _case(name)
    p = c["prob"]
    psi32 = G.round_to_c64(c["psi"])
    Uk, _, _ = _truncate(c, psi32)
    Ukd = to_dev(Uk)
    P = torch.empty(mg.shape_P(p), dtype=torch.complex64, device="cuda")
    mg.mg_build_prolongator(p, Ukd, P)
    torch.cuda.synchronize()
    ref = O.prolongator(c["dims"], c["block"], Uk)
    np.testing.assert_array_equal(to_host(P), ref)
    # gamma_5 P = P sigma_3 and block orthonormality of the GPU prolongator
    Pd = dense_P(c["dims"], c["block"], to_host(P))
    np.testing.assert_allclose(Pd.conj().T @ Pd, np.eye(Pd.shape[1]), atol=1e-5)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [mg.MG_PREC_FP32, mg.MG_PREC_MIXED])
def test_coarsen(name, precision):
    """Stage-isolated: the oracle's prolongator (rounded to complex64) in.
    The mixed path (tensor-core contractions, FP16 hi/lo operands) is held to
    the FP32 path's tolerance."""
    c = _case(name)
    p = _with_precision(c["prob"], precision)
    Uk, _ = O.chiral_truncate(c["dims"], c["block"], c["psi"], c["k"])
    P = G.round_to_c64(O.prolongator(c["dims"], c["block"], Uk))
    Xo, Yo = O.coarsen(c["dims"], c["block"], c["m0"], c["xi"], c["U"], c["C"], P)
    U, C = _dev(c)
    X = torch.empty(mg.shape_X(p), dtype=torch.complex64, device="cuda")
    Y = torch.empty(mg.shape_Y(p), dtype=torch.complex64, device="cuda")
    mg.mg_coarsen(p, U, C, to_dev(P), X, Y)
    torch.cuda.synchronize()
    scale = np.abs(Xo).max()
    np.testing.assert_allclose(to_host(X), Xo, atol=1e-5 * scale)
    np.testing.assert_allclose(to_host(Y), Yo, atol=1e-5 * scale)


@pytest.mark.parametrize("nrhs", [1, 8, 13])
def test_coarse_apply(nrhs):
    cd, k = [2, 3, 1, 4], 5
    nc, n = 24, 10
    g = G.normals(77, G.STREAM_MISC, 0, 2 * nc * 9 * n * n)
    Z = G.round_to_c64((g[0::2] + 1j * g[1::2]).reshape(nc, 9, n, n))
    X, Y = Z[:, 0].copy(), Z[:, 1:].copy()
    v = G.round_to_c64(G.coarse_vectors(nc, n, nrhs, 78))
    ref = O.coarse_apply(cd, X, Y, v)
    p = mg.Problem(dims=[2 * d for d in cd], block=[2, 2, 2, 2], m0=0.0, n_vec=12, k=k,
                   mr_iters=1)
    out = torch.empty((nc, n, nrhs), dtype=torch.complex64, device="cuda")
    mg.mg_coarse_apply(p, to_dev(X), to_dev(Y), to_dev(v), out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(to_host(out), ref, atol=2e-5 * np.abs(ref).max())


def _lowest_sigma3(cdims, X, Y, k, nev=16):
    Dc = dense_coarse(cdims, X, Y)
    s3 = np.tile(np.r_[np.ones(k), -np.ones(k)], Dc.shape[0] // (2 * k))
    ev = np.linalg.eigvalsh(s3[:, None] * Dc)
    return ev[np.argsort(np.abs(ev))[:nev]]


@pytest.mark.parametrize("precision", [mg.MG_PREC_FP32, mg.MG_PREC_MIXED])
@pytest.mark.parametrize("name", ["4^4 Wilson m'=8 k=4 (workload 1)", "8^4 clover m'=48 k=24",
                                  "8^3x16 aniso m'=64 k=24"])
def test_end_to_end(name, precision):
    """Full GPU chain from the same inputs as the oracle chain; the mixed path
    at the FP32 path's tolerances."""
    c = _case(name)
    p = _with_precision(c["prob"], precision)
    k = c["k"]
    U, C = _dev(c)
    lv = mg.Level.allocate(p, U, C, to_dev(c["p0"]))
    lv.run()
    torch.cuda.synchronize()
    assert np.all(lv.flags.cpu().numpy() == 0)
    Ur, sr = O.chiral_truncate(c["dims"], c["block"], c["psi"], k)
    np.testing.assert_allclose(lv.sigma.cpu().numpy(), sr[..., :k], rtol=2e-5)
    Po = O.prolongator(c["dims"], c["block"], Ur)
    Xo, Yo = O.coarsen(c["dims"], c["block"], c["m0"], c["xi"], c["U"], c["C"], Po)
    cd = O.coarse_dims(c["dims"], c["block"])
    Xg, Yg = to_host(lv.X), to_host(lv.Y)
    ev_o = _lowest_sigma3(cd, Xo, Yo, k)
    ev_g = _lowest_sigma3(cd, Xg, Yg, k)
    np.testing.assert_allclose(np.sort(ev_g), np.sort(ev_o), rtol=1e-5,
                               atol=1e-5 * np.abs(ev_o).max())
    # Galerkin identity with the GPU's own P and D_c against the FP64 fine operator
    _galerkin_identity(c, to_host(lv.P), Xg, Yg)


def _galerkin_identity(c, P, X, Y, nprobe=4, tol=1e-6):
    """|P D_c P^dag z - P P^dag D P P^dag z| <= tol |D| |z| (matrix free)."""
    dims, block = c["dims"], c["block"]
    cd = O.coarse_dims(dims, block)
    D = lambda v: O.apply_D(dims, c["m0"], c["xi"], c["U"], c["C"], v[..., None])[..., 0]  # noqa
    V = int(np.prod(dims))
    rng = np.random.default_rng(5)
    b = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    for _ in range(30):  # power iteration on D^dag D for |D|_2
        b = D(b)
        b = O.gamma5(D(O.gamma5(b[..., None])[..., 0])[..., None])[..., 0]  # D^dag = g5 D g5
        nb = np.linalg.norm(b)
        b /= nb
    normD = np.sqrt(nb)
    for _ in range(nprobe):
        z = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
        rz = restrict(dims, block, P, z)
        lhs = prolong(dims, block, P, O.coarse_apply(cd, X, Y, rz[..., None])[..., 0])
        rhs = prolong(dims, block, P, restrict(dims, block, P, D(prolong(dims, block, P, rz))))
        assert np.linalg.norm(lhs - rhs) <= tol * normD * np.linalg.norm(z)


# ---------------------------------------------------------------------------
# FP16-storage path (MG_PREC_MIXED_FP16): the smoother's fields are stored in
# FP16 (unit roundoff u16 = 2^-11 = 4.9e-4) with FP32 arithmetic; truncation
# as MG_PREC_MIXED.  This path trades accuracy for smoother bandwidth: FP16
# rounding anywhere before the last MR iteration is amplified by the rest of
# the trajectory, so it cannot meet the FP32 tolerances.  Its stated bounds:
#   * operator: input and output rounded to FP16 once each: <= 4 u16 = 2e-3
#     relative per vector;
#   * smoother: the MR trajectory amplifies storage rounding (the FP32 path
#     shows the same factor, ~50x its unit roundoff): <= 100 u16 = 5e-2
#     relative per vector;
#   * end to end: retained singular values <= 1e-2 relative, the 16 lowest
#     |eigenvalues| of sigma_3 D_c <= 2e-2 relative, and the quality of the
#     coarse space (their mean) within 1% of the FP64 oracle's.
# ---------------------------------------------------------------------------
U16 = 2.0 ** -11
FP16_STORAGE_CASES = ["8^4 clover m'=48 k=24", "8^3x16 aniso m'=64 k=24"]


def _fp16_storage(c):
    p = c["prob"]
    return mg.Problem(dims=p.dims, block=p.block, m0=p.m0, n_vec=p.n_vec, k=p.k,
                      mr_iters=p.mr_iters, csw=p.csw, xi=p.xi, precision=mg.MG_PREC_MIXED_FP16)


@pytest.mark.parametrize("name", FP16_STORAGE_CASES)
def test_fp16_storage_dirac_apply(name):
    c = _case(name)
    p = _fp16_storage(c)
    U, C = _dev(c)
    vin = to_dev(c["p0"])
    out = torch.empty_like(vin)
    mg.mg_apply_dirac(p, U, C, vin, out, mg.workspace(p, mg.MG_CALL_SMOOTH))
    mg.mg_sync_status()
    ref = O.apply_D(c["dims"], c["m0"], c["xi"], c["U"], c["C"], c["p0"])
    got = to_host(out)
    err = np.linalg.norm((got - ref).reshape(-1, c["m"]), axis=0) / \
        np.linalg.norm(ref.reshape(-1, c["m"]), axis=0)
    assert err.max() <= 4 * U16, err.max()
    # FP16 storage halves the smoother workspace
    assert mg.mg_workspace_size(p, mg.MG_CALL_SMOOTH) < \
        0.6 * mg.mg_workspace_size(c["prob"], mg.MG_CALL_SMOOTH)


@pytest.mark.parametrize("name", FP16_STORAGE_CASES)
def test_fp16_storage_smoother_and_end_to_end(name):
    c = _case(name)
    p = _fp16_storage(c)
    k = c["k"]
    U, C = _dev(c)
    # a per-vector scale of the starts changes nothing (MR is scale invariant
    # and the output is normalised); large scales would overflow unscaled FP16
    p0 = c["p0"] * np.where(np.arange(c["m"]) % 2 == 0, 1.0e5, 1.0e-5)
    lv = mg.Level.allocate(p, U, C, to_dev(p0))
    lv.run()
    mg.mg_sync_status()
    got = to_host(lv.psi)
    assert np.all(np.isfinite(got))
    err = np.linalg.norm((got - c["psi"]).reshape(-1, c["m"]), axis=0)
    assert err.max() <= 100 * U16, err.max()
    assert np.all(lv.flags.cpu().numpy() == 0)
    Ur, sr = O.chiral_truncate(c["dims"], c["block"], c["psi"], k)
    np.testing.assert_allclose(lv.sigma.cpu().numpy(), sr[..., :k], rtol=1e-2)
    Po = O.prolongator(c["dims"], c["block"], Ur)
    Xo, Yo = O.coarsen(c["dims"], c["block"], c["m0"], c["xi"], c["U"], c["C"], Po)
    cd = O.coarse_dims(c["dims"], c["block"])
    lo = np.sort(np.abs(_lowest_sigma3(cd, Xo, Yo, k)))
    lg = np.sort(np.abs(_lowest_sigma3(cd, to_host(lv.X), to_host(lv.Y), k)))
    assert np.max(np.abs(lg - lo) / lo) <= 2e-2
    assert abs(lg.mean() - lo.mean()) <= 1e-2 * lo.mean()
