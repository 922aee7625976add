"""Edge cases of the method on the GPU, through the C ABI, against the FP64
oracle (both precisions that claim FP32-level results):

* the free-field constant modes (U = 1, the 12 constant spin-colour vectors fed
  straight to the truncation, m' = 12, k = 6): every block-chirality is rank
  deficient (6 of its 12 columns vanish), so the Cholesky of its Gram needs the
  diagonal shift, which blk_flags must report; the retained singular values and
  projectors must still match the oracle, and m0 (the p = 0 eigenvalue of the
  free Wilson operator, whose eigenvectors lie in range(P)) must be a 12-fold
  eigenvalue of the GPU's D_c, as it is of the oracle's (pinned on the CPU in
  test_oracle_coarse.py);
* ill-conditioned blocks: test vectors whose block-chirality matrices have
  singular values spread over four decades (sigma_1 / sigma_m' = 1e4): the
  retained singular values and projectors must match the oracle (the oracle's
  Householder QR + Jacobi SVD is not affected by the conditioning);
* failure detection: a bounded device wait that runs out is reported as
  MG_ERR_TIMEOUT by mg_sync_status, after which the library works as before.
"""
import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from conftest import dense_coarse
from gpu_common import dk_bound, projector_error, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg  # noqa: E402

_build.build()

PRECISIONS = [mg.MG_PREC_FP32, mg.MG_PREC_MIXED]


def _truncate(p, psi):
    Uk = torch.empty(mg.shape_Uk(p), dtype=torch.complex64, device="cuda")
    sig = torch.empty(mg.shape_sigma(p), dtype=torch.float64, device="cuda")
    flags = torch.full((p.n_blocks, 2), -1, dtype=torch.int32, device="cuda")
    mg.mg_chiral_truncate(p, to_dev(psi), Uk, sig, None, flags,
                          mg.workspace(p, mg.MG_CALL_TRUNCATE))
    mg.mg_sync_status()
    return Uk, sig.cpu().numpy(), flags.cpu().numpy()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_free_field_constant_modes(precision):
    dims, block, m0, k = [4, 4, 4, 4], [2, 2, 2, 2], 0.37, 6
    V = int(np.prod(dims))
    psi = np.zeros((V, 4, 3, 12), dtype=np.complex128)
    for sp in range(4):
        for c in range(3):
            psi[:, sp, c, sp * 3 + c] = 1.0
    p = mg.Problem(dims=dims, block=block, m0=m0, n_vec=12, k=k, mr_iters=1,
                   precision=precision)
    Uk, sig, flags = _truncate(p, psi)
    # rank deficient: the Gram's Cholesky needed the shift, and it succeeded
    assert np.all(flags & 1), flags
    assert not np.any(flags & 2), flags
    Ur, sr = O.chiral_truncate(dims, block, psi, k)
    np.testing.assert_allclose(sig, sr[..., :k], rtol=1e-5)
    Ug_all = to_host(Uk)
    for j in range(p.n_blocks):
        for al in range(2):
            assert projector_error(Ug_all[j, al].reshape(-1, k), Ur[j, al].reshape(-1, k)) <= 1e-5
    # m0 is a 12-fold eigenvalue of D_c
    U = to_dev(G.unit_gauge_field(dims))
    P = torch.empty(mg.shape_P(p), dtype=torch.complex64, device="cuda")
    X = torch.empty(mg.shape_X(p), dtype=torch.complex64, device="cuda")
    Y = torch.empty(mg.shape_Y(p), dtype=torch.complex64, device="cuda")
    mg.mg_build_prolongator(p, Uk, P)
    mg.mg_coarsen(p, U, None, P, X, Y)
    mg.mg_sync_status()
    ev = np.linalg.eigvals(dense_coarse(O.coarse_dims(dims, block), to_host(X), to_host(Y)))
    assert np.sum(np.abs(ev - m0) < 1e-5) == 12, np.sort(np.abs(ev - m0))[:14]


def _block_rows(dims, block):
    """Site of every (block j, local site loc) in the ABI's block order."""
    Lc = [dims[i] // block[i] for i in range(4)]
    nblk, nb = int(np.prod(Lc)), int(np.prod(block))
    out = np.empty((nblk, nb), dtype=np.int64)
    for j in range(nblk):
        jc, t = [], j
        for i in range(4):
            jc.append(t % Lc[i])
            t //= Lc[i]
        for loc in range(nb):
            lc, t = [], loc
            for i in range(4):
                lc.append(t % block[i])
                t //= block[i]
            x = [jc[i] * block[i] + lc[i] for i in range(4)]
            out[j, loc] = x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))
    return out


@pytest.mark.parametrize("precision", PRECISIONS)
def test_ill_conditioned_blocks(precision):
    dims, block, m, k = [4, 4, 4, 4], [2, 2, 2, 2], 32, 8
    nb = int(np.prod(block))
    K = 6 * nb
    rng = np.random.default_rng(11)
    sites = _block_rows(dims, block)
    psi = np.zeros((int(np.prod(dims)), 4, 3, m), dtype=np.complex128)
    sigma = 10.0 ** (-4.0 * np.arange(m) / (m - 1))  # sigma_1 / sigma_m' = 1e4
    for j in range(sites.shape[0]):
        for al in range(2):
            W, _ = np.linalg.qr(rng.standard_normal((K, m)) + 1j * rng.standard_normal((K, m)))
            Vh, _ = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
            A = (W * sigma) @ Vh.conj().T
            for r in range(K):
                e = r % 6
                psi[sites[j, r // 6], 2 * al + e // 3, e % 3, :] = A[r]
    psi = G.round_to_c64(psi)
    p = mg.Problem(dims=dims, block=block, m0=-0.1, n_vec=m, k=k, mr_iters=1,
                   precision=precision)
    Uk, sig, flags = _truncate(p, psi)
    assert not np.any(flags & 2), flags
    Ur, sr = O.chiral_truncate(dims, block, psi, k)
    np.testing.assert_allclose(sig, sr[..., :k], rtol=1e-5)
    bound = dk_bound(sr, k)
    Ug_all = to_host(Uk)
    for j in range(p.n_blocks):
        for al in range(2):
            e = projector_error(Ug_all[j, al].reshape(-1, k), Ur[j, al].reshape(-1, k))
            assert e <= max(1e-5, bound[j, al]), (j, al, e)


def test_timeout_is_reported_and_the_library_stays_usable():
    mg.mg_sync_status()  # clear anything left by earlier tests
    mg.mg_selftest_timeout(1000)
    with pytest.raises(mg.MgError) as e:
        mg.mg_sync_status()
    assert e.value.status == mg.MG_ERR_TIMEOUT
    mg.mg_sync_status()  # the word was taken: clean again
    with pytest.raises(mg.MgError):
        mg.mg_selftest_timeout(0)
    # the device still computes: one small level against the oracle
    dims, block, m, k, N, m0 = [4, 4, 4, 4], [2, 2, 2, 2], 8, 4, 10, -0.228492
    U = G.round_to_c64(G.gauge_field(dims, 0.3, 0))
    p0 = G.round_to_c64(G.psi0(dims, m, 1))
    p = mg.Problem(dims=dims, block=block, m0=m0, n_vec=m, k=k, mr_iters=N)
    lv = mg.Level.allocate(p, to_dev(U), None, to_dev(p0))
    lv.run()
    mg.mg_sync_status()
    psi = O.mr(dims, m0, 1.0, U, None, p0, N)
    err = np.linalg.norm((to_host(lv.psi) - psi).reshape(-1, m), axis=0)
    assert err.max() <= 2e-5
