"""Setup serving (paper_2502_03091_gb300.serve): requests that overlap on the
device give each result exactly as the same request served alone (the kernels
are deterministic and requests share nothing but the device), admission keeps
the HBM ledger within its budget, and every request completes."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg, serve  # noqa: E402

_build.build()

SMALL = ([8, 8, 8, 8], [12, 12, 12, 24], [16, 16, 16, 32])


@pytest.mark.parametrize("precision", [mg.MG_PREC_MIXED, mg.MG_PREC_FP32])
def test_solo_equals_mix(precision):
    reqs = serve.request_stream(10, rate=1000.0, seed=41, m0=-0.15, volumes=SMALL)
    mix = serve.Server(max_slots=4, precision=precision, keep_results=True)
    st = mix.run(reqs, realtime=False)
    assert st["requests"] == len(reqs)
    assert st["hbm_high_water_gb"] * 1e9 <= mix.budget
    for r in reqs:
        alone = serve.Server(max_slots=1, precision=precision, keep_results=True)
        r1 = serve.Request(rid=r.rid, arrival=0.0, dims=r.dims, m=r.m, k=r.k, m0=r.m0,
                           seed=r.seed)
        alone.run([r1], realtime=False)
        for a, b in zip(mix.results[r.rid], alone.results[r.rid]):
            assert torch.equal(a, b), r.rid
