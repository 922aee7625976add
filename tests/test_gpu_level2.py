"""Levels l >= 1 on the GPU (the mg_coarse_* calls through the C ABI) against
the FP64 oracle of the second level (oracle.level2), stage by stage, on
identical complex64-representable inputs.

Operators D_1 the second level is built on:
  * "chain": the oracle's own first-level setup of an 8^4 Wilson-clover
    lattice (eps = 0.25, m' = 48, k1 = 24, 2^4 aggregates, 10 MR iterations):
    a real coarse operator with 48 components per site on the 4^4 coarse
    lattice.  The second level uses 2^4 aggregates, m = 64, k2 = 32 (the
    paper's k at l = 1, Sec. 4) and 20 MR iterations;
  * "stencil": a random stencil with the symmetry of a coarse operator
    (mg_inputs.stencil_operator) at the size of the first coarse level of the
    32^3x64 hierarchy (8^3x8 sites, 48 components), in the launch
    configuration bench.py times; there the oracle checks sampled
    right-hand sides and blocks.

Tolerances (FP32 arithmetic on complex64 inputs, unit roundoff u = 2^-24):
  * apply and Galerkin product: elementwise |got - want| <= 3 K u (|M| |v|),
    the forward bound of a length-K complex dot product in FP32 (2K real
    products per component, each term bounded by |a| |b|), with |M| |v| the
    same sums of absolute values (K = 9 n for the apply; K = 2 nc + 9 |Lambda|
    for the Galerkin product: two GEMMs of depth nc and up to 9 |Lambda|
    accumulated terms);
  * smoother: each vector's relative 2-norm error <= 2e-5 on the random
    stencil, as at the fine level (N FP32 applies, FP64 sums of the inner
    products), and <= 5e-5 on the chain's D_1: along its MR trajectory the
    cancellation ratio | |D_1| |r| | / |D_1 r| grows to 15 (r turns into
    near-null vectors of D_1), and an FP32 restatement of the same recurrence
    (per-term partial sums, FP64 inner products) lands 2.3e-5 from the FP64
    oracle on it;
  * truncation: retained singular values relative <= 1e-5; per-block projector
    error <= max(1e-5, the Davis-Kahan bound of an FP32-level perturbation);
  * prolongator: bit exact (data movement);
  * whole GPU chain: singular values within Weyl's bound |s_g - s_o| <=
    |A_g - A_o|_F + 1e-5 s_1 of the two chains' block matrices, and the
    Galerkin identity D_2 v = P^dag D_1 P v with the GPU's own P and D_2.
"""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from gpu_common import M0, dk_bound, projector_error, to_dev, to_host
from oracle import level2 as L2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg  # noqa: E402

_build.build()

U32 = 2.0 ** -24


def _abs_apply(cdims, X, Y, v):
    return O.coarse_apply(cdims, np.abs(X), np.abs(Y), np.abs(v)).real


def _check_apply(cdims, X, Y, v, got):
    want = O.coarse_apply(cdims, X, Y, v)
    scale = _abs_apply(cdims, X, Y, v)
    K = 9 * X.shape[-1]
    err = np.abs(got - want)
    assert np.all(err <= 3 * K * U32 * scale + 1e-30), float((err / (scale + 1e-30)).max())


def _starts(nc_sites, n, m, seed):
    return G.round_to_c64(G.coarse_vectors(nc_sites, n, m, seed))


# ---------------------------------------------------------------------------
# stencil apply: ragged sizes, every tile shape
# ---------------------------------------------------------------------------
APPLY_CASES = [([4, 4, 4, 4], 24, 64), ([4, 4, 2, 4], 24, 13), ([2, 2, 2, 2], 32, 1),
               ([3, 2, 1, 5], 5, 7), ([2, 3, 2, 2], 17, 40)]


@pytest.mark.parametrize("cdims,nc,nrhs", APPLY_CASES)
def test_stencil_apply(cdims, nc, nrhs):
    X, Y = G.stencil_operator(cdims, nc, 3)
    X, Y = G.round_to_c64(X), G.round_to_c64(Y)
    V = G.volume(cdims)
    v = _starts(V, 2 * nc, nrhs, 4)
    cp = mg.CoarseProblem(cdims, [1, 1, 1, 1], nc, 4, 1, 1)
    out = torch.full(v.shape, float("nan"), dtype=torch.complex64, device="cuda")
    mg.mg_coarse_op_apply(cp, to_dev(X), to_dev(Y), to_dev(v), out)
    mg.mg_sync_status()
    _check_apply(cdims, X, Y, v, to_host(out))


def test_stencil_apply_rejects_bad_arguments():
    cp = mg.CoarseProblem([2, 2, 2, 2], [1, 1, 1, 1], 4, 4, 1, 1)
    X = torch.zeros(mg.shape_cX(cp), dtype=torch.complex64, device="cuda")
    Y = torch.zeros(mg.shape_cY(cp), dtype=torch.complex64, device="cuda")
    v = torch.zeros(mg.shape_cvec(cp, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(mg.MgError):
        mg.mg_coarse_op_apply(cp, X, Y, v, v)                      # aliasing
    out = torch.zeros_like(v)
    lib = mg.library()
    pc = cp.c()
    # a misaligned X is refused on the host, before anything is launched
    st = lib.mg_coarse_op_apply(mg.ctypes.byref(pc), X.data_ptr() + 8, Y.data_ptr(),
                                v.data_ptr(), out.data_ptr(), 4, None)
    assert st == 1 and b"aligned" in lib.mg_last_error()


# ---------------------------------------------------------------------------
# the chain case: a real D_1 from the oracle's first level
# ---------------------------------------------------------------------------
DIMS, BLOCK1, EPS, CSW, M1, K1, N1 = [8, 8, 8, 8], [2, 2, 2, 2], 0.25, 1.0, 48, 24, 10
BLOCK2, M2, K2, N2 = [2, 2, 2, 2], 64, 32, 20
M0_CHAIN = M0["16^3x32 Wilson-clover eps=0.25"]


@pytest.fixture(scope="module")
def chain():
    U = G.round_to_c64(G.gauge_field(DIMS, EPS, 10))
    C = G.round_to_c64(O.clover(DIMS, U, CSW))
    p0 = G.round_to_c64(G.psi0(DIMS, M1, 11))
    psi = O.mr(DIMS, M0_CHAIN, 1.0, U, C, p0, N1)
    Uk, _ = O.chiral_truncate(DIMS, BLOCK1, psi, K1)
    P = O.prolongator(DIMS, BLOCK1, Uk)
    X, Y = O.coarsen(DIMS, BLOCK1, M0_CHAIN, 1.0, U, C, P)
    cd = O.coarse_dims(DIMS, BLOCK1)
    X, Y = G.round_to_c64(X), G.round_to_c64(Y)
    q0 = _starts(G.volume(cd), 2 * K1, M2, 5)
    psi2 = L2.mr(cd, X, Y, q0, N2)
    psi2r = G.round_to_c64(psi2)
    Uk2, s2 = L2.chiral_truncate(cd, BLOCK2, K1, psi2r, K2)
    Uk2r = G.round_to_c64(Uk2)
    P2r = G.round_to_c64(L2.prolongator(cd, BLOCK2, Uk2r))
    X2, Y2 = L2.coarsen(cd, BLOCK2, X, Y, P2r)
    cp = mg.CoarseProblem(cd, BLOCK2, K1, M2, K2, N2)
    return dict(cd=cd, X=X, Y=Y, q0=q0, psi2=psi2, psi2r=psi2r, Uk2=Uk2, Uk2r=Uk2r, s2=s2,
                P2r=P2r, X2=X2, Y2=Y2, cp=cp)


def test_chain_smoother(chain):
    c = chain
    cp = c["cp"]
    ws = mg.coarse_workspace(cp, mg.MG_CALL_SMOOTH)
    psi = torch.full(mg.shape_cvec(cp, M2), float("nan"), dtype=torch.complex64, device="cuda")
    mg.mg_coarse_smooth_testvecs(cp, to_dev(c["X"]), to_dev(c["Y"]), to_dev(c["q0"]), psi, ws)
    mg.mg_sync_status()
    got = to_host(psi)
    want = c["psi2"]
    err = np.linalg.norm((got - want).reshape(-1, M2), axis=0) / np.linalg.norm(
        want.reshape(-1, M2), axis=0)
    assert err.max() <= 5e-5, err.max()


def test_chain_truncation(chain):
    c = chain
    cp = c["cp"]
    nblk = cp.n_blocks
    Uk = torch.empty(mg.shape_cUk(cp), dtype=torch.complex64, device="cuda")
    sig = torch.empty((nblk, 2, K2), dtype=torch.float64, device="cuda")
    ctv = torch.empty((nblk, 2, K2, M2), dtype=torch.complex64, device="cuda")
    flags = torch.full((nblk, 2), -1, dtype=torch.int32, device="cuda")
    ws = mg.coarse_workspace(cp, mg.MG_CALL_TRUNCATE)
    mg.mg_coarse_chiral_truncate(cp, to_dev(c["psi2r"]), Uk, sig, ctv, flags, ws)
    torch.cuda.synchronize()
    assert np.all(flags.cpu().numpy() == 0)
    sg, Ug, Cg = sig.cpu().numpy(), to_host(Uk), to_host(ctv)
    np.testing.assert_allclose(sg, c["s2"][..., :K2], rtol=1e-5)
    for j in range(nblk):
        for al in range(2):
            A = L2.block_matrix(c["cd"], BLOCK2, K1, c["psi2r"], j, al)
            so, Uo, _ = O.svd(A)
            Ugj = Ug[j, al].reshape(-1, K2)
            tol = max(1e-5, float(dk_bound(so, K2)))
            assert projector_error(Ugj, Uo[:, :K2]) <= tol, (j, al)
            # U_k (Sigma_k V_k^dag) is the best rank-k approximation of A
            best = Uo[:, :K2] @ (Uo[:, :K2].conj().T @ A)
            assert np.linalg.norm(Ugj @ Cg[j, al] - best) <= 2 * tol * np.linalg.norm(A)


def test_chain_prolongator_bit_exact(chain):
    c = chain
    cp = c["cp"]
    P = torch.full(mg.shape_cP(cp), float("nan"), dtype=torch.complex64, device="cuda")
    mg.mg_coarse_build_prolongator(cp, to_dev(c["Uk2r"]), P)
    torch.cuda.synchronize()
    want = L2.prolongator(c["cd"], BLOCK2, c["Uk2r"]).astype(np.complex64)
    assert np.array_equal(P.cpu().numpy(), want)


def _check_galerkin(cd, block, X, Y, P, X2g, Y2g, X2o, Y2o):
    aX, aY = L2.coarsen(cd, block, np.abs(X), np.abs(Y), np.abs(P))
    nc = P.shape[2]
    K = 2 * nc + 9 * int(np.prod(block))
    for got, want, scale in ((X2g, X2o, aX.real), (Y2g, Y2o, aY.real)):
        err = np.abs(got - want)
        assert np.all(err <= 3 * K * U32 * scale + 1e-30), float((err / (scale + 1e-30)).max())


def test_chain_coarsen(chain):
    c = chain
    cp = c["cp"]
    X2 = torch.full(mg.shape_cX2(cp), float("nan"), dtype=torch.complex64, device="cuda")
    Y2 = torch.full(mg.shape_cY2(cp), float("nan"), dtype=torch.complex64, device="cuda")
    mg.mg_coarse_coarsen(cp, to_dev(c["X"]), to_dev(c["Y"]), to_dev(c["P2r"]), X2, Y2)
    torch.cuda.synchronize()
    _check_galerkin(c["cd"], BLOCK2, c["X"], c["Y"], c["P2r"], to_host(X2), to_host(Y2),
                    c["X2"], c["Y2"])


def test_chain_second_coarse_apply(chain):
    """D_2 (2 k2 = 64 components on the 2^4 lattice) through the same call."""
    c = chain
    c2 = O.coarse_dims(c["cd"], BLOCK2)
    X2, Y2 = G.round_to_c64(c["X2"]), G.round_to_c64(c["Y2"])
    cp2 = mg.CoarseProblem(c2, [1, 1, 1, 1], K2, 4, 1, 1)
    v = _starts(G.volume(c2), 2 * K2, 24, 8)
    out = torch.empty(v.shape, dtype=torch.complex64, device="cuda")
    mg.mg_coarse_op_apply(cp2, to_dev(X2), to_dev(Y2), to_dev(v), out)
    torch.cuda.synchronize()
    _check_apply(c2, X2, Y2, v, to_host(out))


def test_chain_whole_gpu_level(chain):
    """The four calls in a row on the GPU (CoarseLevel.run) from the same D_1
    and starts as the oracle chain."""
    c = chain
    cp = c["cp"]
    lv = mg.CoarseLevel.allocate(cp, to_dev(c["X"]), to_dev(c["Y"]), to_dev(c["q0"]))
    lv.run()
    mg.mg_sync_status()
    assert np.all(lv.flags.cpu().numpy() == 0)
    psi_g = to_host(lv.psi)
    sg = lv.sigma.cpu().numpy()
    for j in range(cp.n_blocks):
        for al in range(2):
            Ag = L2.block_matrix(c["cd"], BLOCK2, K1, psi_g, j, al)
            Ao = L2.block_matrix(c["cd"], BLOCK2, K1, c["psi2r"], j, al)
            so = c["s2"][j, al, :K2]
            bound = np.linalg.norm(Ag - Ao) + 1e-5 * so[0]
            assert np.all(np.abs(sg[j, al] - so) <= bound), (j, al)
    # Galerkin identity with the GPU's own P and D_2, D_1 in FP64
    P = to_host(lv.P)
    X2g, Y2g = to_host(lv.X2), to_host(lv.Y2)
    c2 = O.coarse_dims(c["cd"], BLOCK2)
    v = G.coarse_vectors(G.volume(c2), 2 * K2, 3, 12)
    lhs = O.coarse_apply(c2, X2g, Y2g, v)
    aX, aY = L2.coarsen(c["cd"], BLOCK2, np.abs(c["X"]), np.abs(c["Y"]), np.abs(P))
    bound = 3 * (2 * K1 + 9 * int(np.prod(BLOCK2))) * U32 * O.coarse_apply(c2, aX, aY, np.abs(v))
    for i in range(v.shape[-1]):
        Pv = L2.prolong(c["cd"], BLOCK2, P, v[..., i])
        rhs = L2.restrict(c["cd"], BLOCK2, P, O.coarse_apply(c["cd"], c["X"], c["Y"],
                                                             Pv[..., None])[..., 0])
        err = np.linalg.norm(lhs[..., i] - rhs)
        assert err <= np.linalg.norm(bound[..., i]), err / np.linalg.norm(bound[..., i])


# ---------------------------------------------------------------------------
# full size: the first coarse level of the 32^3x64 hierarchy (8^3x8 sites,
# nc = 24), second level m = 64, k = 32, 2^4 aggregates, 20 iterations
# ---------------------------------------------------------------------------
FULL_CD, FULL_NC = [8, 8, 8, 8], 24


@pytest.fixture(scope="module")
def full():
    X, Y = G.stencil_operator(FULL_CD, FULL_NC, 40, threads=16)
    X, Y = G.round_to_c64(X), G.round_to_c64(Y)
    cp = mg.CoarseProblem(FULL_CD, BLOCK2, FULL_NC, M2, K2, N2)
    return dict(X=X, Y=Y, Xd=to_dev(X), Yd=to_dev(Y), cp=cp)


def test_fullsize_apply_sampled(full):
    cp = full["cp"]
    V = cp.volume
    v = _starts(V, 2 * FULL_NC, M2, 41)
    out = torch.empty(v.shape, dtype=torch.complex64, device="cuda")
    mg.mg_coarse_op_apply(cp, full["Xd"], full["Yd"], to_dev(v), out)
    mg.mg_sync_status()
    cols = [0, 37, 63]
    got = to_host(out)[..., cols]
    _check_apply(FULL_CD, full["X"], full["Y"], np.ascontiguousarray(v[..., cols]), got)


def test_fullsize_smoother_sampled(full):
    cp = full["cp"]
    q0 = _starts(cp.volume, 2 * FULL_NC, M2, 42)
    ws = mg.coarse_workspace(cp, mg.MG_CALL_SMOOTH)
    psi = torch.empty(q0.shape, dtype=torch.complex64, device="cuda")
    mg.mg_coarse_smooth_testvecs(cp, full["Xd"], full["Yd"], to_dev(q0), psi, ws)
    mg.mg_sync_status()
    cols = [1, 50]
    want = L2.mr(FULL_CD, full["X"], full["Y"], np.ascontiguousarray(q0[..., cols]), N2)
    got = to_host(psi)[..., cols]
    for i in range(len(cols)):
        err = np.linalg.norm(got[..., i] - want[..., i]) / np.linalg.norm(want[..., i])
        assert err <= 2e-5, (cols[i], err)


def test_fullsize_truncation_sampled(full):
    cp = full["cp"]
    psi = _starts(cp.volume, 2 * FULL_NC, M2, 43)
    nblk = cp.n_blocks
    Uk = torch.empty(mg.shape_cUk(cp), dtype=torch.complex64, device="cuda")
    sig = torch.empty((nblk, 2, K2), dtype=torch.float64, device="cuda")
    flags = torch.full((nblk, 2), -1, dtype=torch.int32, device="cuda")
    ws = mg.coarse_workspace(cp, mg.MG_CALL_TRUNCATE)
    mg.mg_coarse_chiral_truncate(cp, to_dev(psi), Uk, sig, None, flags, ws)
    torch.cuda.synchronize()
    assert np.all(flags.cpu().numpy() == 0)
    sg = sig.cpu().numpy()
    assert np.all(sg > 0) and np.all(np.diff(sg, axis=-1) <= 0)
    Ug = to_host(Uk)
    for j in (0, 1, 100, nblk - 1):
        for al in range(2):
            A = L2.block_matrix(FULL_CD, BLOCK2, FULL_NC, psi, j, al)
            so, Uo, _ = O.svd(A)
            np.testing.assert_allclose(sg[j, al], so[:K2], rtol=1e-5)
            e = projector_error(Ug[j, al].reshape(-1, K2), Uo[:, :K2])
            assert e <= max(1e-5, float(dk_bound(so, K2))), (j, al, e)


def test_fullsize_coarsen(full):
    cp = full["cp"]
    P = G.round_to_c64(G.coarse_vectors(cp.volume, 2 * FULL_NC, K2, 44)).reshape(
        cp.volume, 2, FULL_NC, K2)
    X2 = torch.empty(mg.shape_cX2(cp), dtype=torch.complex64, device="cuda")
    Y2 = torch.empty(mg.shape_cY2(cp), dtype=torch.complex64, device="cuda")
    mg.mg_coarse_coarsen(cp, full["Xd"], full["Yd"], to_dev(P), X2, Y2)
    torch.cuda.synchronize()
    X2o, Y2o = L2.coarsen(FULL_CD, BLOCK2, full["X"], full["Y"], P)
    _check_galerkin(FULL_CD, BLOCK2, full["X"], full["Y"], P, to_host(X2), to_host(Y2), X2o, Y2o)
