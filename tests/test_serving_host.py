"""Host side of the setup server: the request stream (seeded Poisson arrivals,
volumes and (m', k) drawn uniformly) and the memory ledger's sizes."""
from paper_2502_03091_gb300 import build as _build
from paper_2502_03091_gb300 import mg, serve

_build.build()


def test_request_stream_and_ledger():
    reqs = serve.request_stream(200, rate=20.0, seed=40)
    assert len(reqs) == 200
    arr = [r.arrival for r in reqs]
    assert all(b > a for a, b in zip(arr, arr[1:]))
    assert 5.0 < arr[-1] < 20.0                  # about 200 / 20 s
    assert {tuple(r.dims) for r in reqs} == {tuple(d) for d in serve.VOLUMES}
    p = mg.Problem(dims=[32, 32, 32, 64], block=[4, 4, 4, 4], m0=-0.15, n_vec=64, k=24,
                   mr_iters=20, precision=mg.MG_PREC_MIXED)
    assert serve.resident_bytes(p) < serve.need_bytes(p)
