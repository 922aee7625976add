"""Batched setup (mg_batch_*): the 24-hierarchy batch (8 each of 8^4,
12^3x24 and 16^3x32; m' in {32, 48, 64}, k in {16, 24}, aggregates 2^4 or
4^4, eps in [0.15, 0.35], drawn from batch seed 30) built by one graph launch
must give every level bit for bit what the level gives when it is built
alone with the single calls (the kernels are deterministic and the levels
share nothing), and the smallest levels must match the FP64 oracle; in the
FP32 path and in the mixed path (tensor-core contractions)."""
import json
import os

import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from gpu_common import HERE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_03091_gb300 import build as _build  # noqa: E402
from paper_2502_03091_gb300 import mg  # noqa: E402

_build.build()


def _m0_by_eps():
    with open(os.path.join(HERE, "golden", "m0.json")) as fh:
        w = json.load(fh)["workloads"]
    return {v["eps"]: v["m0"] for k, v in w.items() if k.startswith("Wilson eps=")}


def _levels(precision=mg.MG_PREC_FP32):
    out = []
    for h in G.batch_workload(30, _m0_by_eps()):
        p = mg.Problem(dims=h["dims"], block=h["block"], m0=h["m0"], n_vec=h["m"], k=h["k"],
                       mr_iters=h["N"], precision=precision)
        U = G.round_to_c64(G.gauge_field(h["dims"], h["eps"], h["gauge_seed"], threads=16))
        p0 = G.round_to_c64(G.psi0(h["dims"], h["m"], h["psi_seed"], threads=16))
        lv = mg.Level.allocate(p, torch.from_numpy(U.astype(np.complex64)).cuda(), None,
                               torch.from_numpy(p0.astype(np.complex64)).cuda())
        out.append((h, U, p0, lv))
    return out


def _snapshot(lv):
    torch.cuda.synchronize()
    return [t.clone() for t in (lv.psi, lv.sigma, lv.flags, lv.P, lv.X, lv.Y)]


@pytest.mark.parametrize("precision", [mg.MG_PREC_FP32, mg.MG_PREC_MIXED])
def test_batch_equals_solo_and_oracle(precision):
    levels = _levels(precision)
    batch = mg.Batch([lv for _, _, _, lv in levels], n_streams=0)
    assert batch.n_streams in (1, 2, 4, 8)
    for _, _, _, lv in levels:   # poison the outputs the batch must write
        for t in (lv.psi, lv.P, lv.X, lv.Y):
            t.fill_(float("nan"))
        lv.sigma.fill_(-1.0)
        lv.flags.fill_(-1)
    batch.launch()
    mg.mg_sync_status()
    got = [_snapshot(lv) for _, _, _, lv in levels]
    for (h, U, p0, lv), g in zip(levels, got):
        assert torch.all(g[2] == 0), h
        lv.run()   # the same level alone, same (tuned) kernels
        solo = _snapshot(lv)
        for a, b in zip(g, solo):
            assert torch.equal(a, b), h
    # the two smallest distinct 8^4 levels against the oracle chain
    for h, U, p0, lv in levels[:2]:
        d, b, k = h["dims"], h["block"], h["k"]
        psi = O.mr(d, h["m0"], 1.0, U, None, p0, h["N"])
        _, so = O.chiral_truncate(d, b, psi, k)
        np.testing.assert_allclose(lv.sigma.cpu().numpy(), so[..., :k], rtol=2e-5)
    batch.close()


def test_batch_rejects_bad_descriptor():
    h = G.batch_workload(30, _m0_by_eps())[0]
    p = mg.Problem(dims=h["dims"], block=h["block"], m0=h["m0"], n_vec=h["m"], k=h["k"],
                   mr_iters=2)
    U = torch.zeros((G.volume(h["dims"]), 4, 3, 3), dtype=torch.complex64, device="cuda")
    p0 = torch.zeros(mg.shape_psi(p), dtype=torch.complex64, device="cuda")
    lv = mg.Level.allocate(p, U, None, p0)
    lv.X = None
    with pytest.raises(mg.MgError) as e:
        mg.Batch([lv])
    assert "level 0" in str(e.value)
    lv2 = mg.Level.allocate(p, U, None, p0)
    lv2.prob = mg.Problem(dims=[8, 8, 8, 8], block=[3, 3, 3, 3], m0=0.0, n_vec=8, k=4,
                          mr_iters=2)
    with pytest.raises(mg.MgError):
        mg.Batch([lv2])
