"""mg_chiral_truncate_static, the truncation entry point for callers that cannot
allocate device memory (a host application whose device memory belongs to its
own pool allocator, or a loop that must not stall the device with
cudaMalloc/cudaFree).  It must give the results of mg_chiral_truncate (which
takes a caller workspace) on two calls in a row -- the second call finds the
first call's data in the shared built-in scratch array -- and must reject a
problem whose scratch need exceeds the built-in 64 MiB.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

import mg_inputs as G
from gpu_common import projector_error, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg  # noqa: E402

_build.build()


def _outputs(p):
    Uk = torch.empty(mg.shape_Uk(p), dtype=torch.complex64, device="cuda")
    sig = torch.empty(mg.shape_sigma(p), dtype=torch.float64, device="cuda")
    flags = torch.full((p.n_blocks, 2), -1, dtype=torch.int32, device="cuda")
    return Uk, sig, flags


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_static_scratch_matches_workspace_call_twice(precision):
    # the mixed-precision truncation runs its Grams on the tensor cores, which
    # write into the same built-in array and report through the status word
    prec = mg.MG_PREC_MIXED if precision == "mixed" else mg.MG_PREC_FP32
    p = mg.Problem(dims=[8, 8, 8, 8], block=[4, 4, 4, 4], m0=-0.1, n_vec=48, k=24, mr_iters=1,
                   precision=prec)
    assert mg.mg_workspace_size(p, mg.MG_CALL_TRUNCATE) <= 64 << 20
    ws = mg.workspace(p, mg.MG_CALL_TRUNCATE)
    for call, seed in enumerate((5, 6)):  # two calls in a row, different inputs
        psi = to_dev(G.psi0(p.dims, p.n_vec, seed))
        Uk_ref, s_ref, f_ref = _outputs(p)
        mg.mg_chiral_truncate(p, psi, Uk_ref, s_ref, None, f_ref, ws)
        mg.mg_sync_status()  # raises on a device-side timeout
        Uk, s, f = _outputs(p)
        mg.mg_chiral_truncate_static(p, psi, Uk, s, None, f)
        mg.mg_sync_status()
        torch.cuda.synchronize()
        assert np.all(f.cpu().numpy() == 0) and np.all(f_ref.cpu().numpy() == 0)
        np.testing.assert_allclose(s.cpu().numpy(), s_ref.cpu().numpy(), rtol=1e-5)
        a, b = to_host(Uk), to_host(Uk_ref)
        k = p.k
        for j in range(p.n_blocks):
            for al in range(2):
                e = projector_error(a[j, al].reshape(-1, k), b[j, al].reshape(-1, k))
                assert e <= 1e-5, (call, j, al, e)


def test_static_scratch_rejects_oversized_problem():
    p = mg.Problem(dims=[16, 16, 16, 32], block=[4, 4, 4, 4], m0=-0.1, n_vec=64, k=24,
                   mr_iters=1)
    assert mg.mg_workspace_size(p, mg.MG_CALL_TRUNCATE) > 64 << 20
    psi = torch.zeros(mg.shape_psi(p), dtype=torch.complex64, device="cuda")
    Uk, s, f = _outputs(p)
    with pytest.raises(mg.MgError) as e:
        mg.mg_chiral_truncate_static(p, psi, Uk, s, None, f)
    assert "built-in" in str(e.value)
