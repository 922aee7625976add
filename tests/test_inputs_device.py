"""The device form of the seeded input generator (mg_inputs.device, used by the
setup server to draw a request's links and starts on the GPU) against the host
generator mg_inputs: uniforms bit for bit, normals, links and starts to within
a few ulps.  Runs on the CPU device here and on cuda:0 with -m gpu."""
import numpy as np
import pytest

import mg_inputs as G

torch = pytest.importorskip("torch")
from mg_inputs import device as D  # noqa: E402


def _devices():
    out = [pytest.param("cpu")]
    out.append(pytest.param("cuda", marks=pytest.mark.gpu))
    return out


@pytest.mark.parametrize("device", _devices())
def test_uniforms_bit_identical(device):
    if device == "cuda" and not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for seed, stream, start in ((0, 1, 0), (400, 2, 12345), (2 ** 40 + 7, 5, 3 * 10 ** 9)):
        u = D.uniforms_t(seed, stream, start, 4096, device).cpu().numpy()
        np.testing.assert_array_equal(u, G.uniforms(seed, stream, start, 4096))


@pytest.mark.parametrize("device", _devices())
def test_normals_links_and_starts_agree(device):
    if device == "cuda" and not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = D.normals_t(401, G.STREAM_PSI0, 77, 5000, device).cpu().numpy()
    ref = G.normals(401, G.STREAM_PSI0, 77, 5000)
    np.testing.assert_allclose(g, ref, rtol=1e-14, atol=1e-14)
    dims = [4, 4, 2, 6]
    U = D.gauge_field_t(dims, 0.25, 402, device).cpu().numpy()
    Uh = G.gauge_field(dims, 0.25, 402)
    assert np.abs(U - Uh).max() <= 1e-13
    p = D.psi0_t(dims, 8, 403, device).cpu().numpy()
    np.testing.assert_allclose(p, G.psi0(dims, 8, 403), rtol=1e-14, atol=1e-14)


@pytest.mark.gpu
def test_library_random_starts_match_host_generator():
    """mg_random_starts draws the same counter-based starts as mg_inputs.psi0
    (uniforms bit for bit; log, sqrt and cos in FP32: the argument of the
    cosine carries the FP32 rounding of u, about 6e-8, times the radius
    sqrt(-2 ln u) <= 9, so within 5e-6)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03091_gb300 import build as _build
    from paper_2502_03091_gb300 import mg
    _build.build()
    for dims, m, seed in (([4, 4, 2, 6], 8, 405), ([6, 4, 4, 4], 12, 2 ** 40 + 3)):
        p = mg.Problem(dims=dims, block=[2, 2, 2, 2], m0=0.0, n_vec=m, k=4, mr_iters=1,
                       seed=seed)
        psi0 = torch.empty(mg.shape_psi(p), dtype=torch.complex64, device="cuda")
        mg.mg_random_starts(p, psi0)
        torch.cuda.synchronize()
        got = psi0.cpu().numpy().astype(np.complex128)
        np.testing.assert_allclose(got, G.psi0(dims, m, seed), rtol=1e-6, atol=5e-6)


@pytest.mark.gpu
def test_library_random_links_match_host_generator():
    """mg_random_links draws mg_inputs.gauge_field's links exp(i eps H) (normals
    in FP64, the exponential's Taylor series in FP32: within 1e-6), and they
    are SU(3) to FP32 rounding."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03091_gb300 import build as _build
    from paper_2502_03091_gb300 import mg
    _build.build()
    for dims, eps, seed in (([4, 4, 2, 6], 0.25, 406), ([4, 2, 2, 4], 0.35, 2 ** 33 + 1)):
        p = mg.Problem(dims=dims, block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=4, mr_iters=1,
                       seed=seed)
        U = torch.empty(mg.shape_U(p), dtype=torch.complex64, device="cuda")
        mg.mg_random_links(p, eps, U)
        torch.cuda.synchronize()
        got = U.cpu().numpy().astype(np.complex128)
        np.testing.assert_allclose(got, G.gauge_field(dims, eps, seed), rtol=0, atol=1e-6)
        g = got.reshape(-1, 3, 3)
        np.testing.assert_allclose(np.einsum("nij,nkj->nik", g, g.conj()),
                                   np.broadcast_to(np.eye(3), g.shape), atol=1e-6)
