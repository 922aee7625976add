"""Checkpoint / resume of a built level (paper_2502_03091_gb300.checkpoint), on
the host: the arrays of an oracle-built 4^4 level come back bit for bit with
their problem and metadata, and damaged files are refused."""
import os

import numpy as np
import pytest

import mg_inputs as G
import oracle as O
from paper_2502_03091_gb300 import checkpoint as CK
from paper_2502_03091_gb300 import mg


@pytest.fixture(scope="module")
def level44():
    dims, block, m, k, N, m0 = [4, 4, 4, 4], [2, 2, 2, 2], 8, 4, 10, -0.2
    U = G.gauge_field(dims, 0.3, 0)
    psi = O.mr(dims, m0, 1.0, U, None, G.psi0(dims, m, 1), N)
    Uk, sig = O.chiral_truncate(dims, block, psi, k)
    P = O.prolongator(dims, block, Uk)
    X, Y = O.coarsen(dims, block, m0, 1.0, U, None, P)
    prob = mg.Problem(dims=dims, block=block, m0=m0, n_vec=m, k=k, mr_iters=N)
    arrays = {"P": P.astype(np.complex64), "X": X.astype(np.complex64),
              "Y": Y.astype(np.complex64), "sigma": sig[..., :k].copy(),
              "flags": np.zeros((16, 2), dtype=np.int32)}
    return prob, arrays


def test_round_trip_is_bitwise(tmp_path, level44):
    prob, arrays = level44
    path = os.path.join(tmp_path, "h.mgh")
    CK.save(path, prob, arrays, meta={"gauge_seed": 0, "psi_seed": 1})
    p, back, meta = CK.load(path)
    assert p["dims"] == [4, 4, 4, 4] and p["k"] == 4 and p["m0"] == -0.2
    assert meta == {"gauge_seed": 0, "psi_seed": 1}
    for name, a in arrays.items():
        assert back[name].dtype == a.dtype and back[name].shape == a.shape
        assert back[name].tobytes() == a.tobytes()
    # reloaded operator applies exactly as the saved one
    cd = O.coarse_dims(p["dims"], p["block"])
    v = G.coarse_vectors(16, 8, 3, 5)
    np.testing.assert_array_equal(O.coarse_apply(cd, back["X"], back["Y"], v),
                                  O.coarse_apply(cd, arrays["X"], arrays["Y"], v))


def test_torch_tensors_and_coarse_problem(tmp_path):
    torch = pytest.importorskip("torch")
    cp = mg.CoarseProblem([2, 2, 2, 2], [2, 2, 2, 2], 3, 8, 2, 5)
    t = torch.arange(24, dtype=torch.float64).reshape(2, 3, 4)
    path = os.path.join(tmp_path, "c.mgh")
    CK.save(path, cp, {"t": t})
    p, back, _ = CK.load(path, device="cpu")
    assert p["nc"] == 3 and torch.equal(back["t"], t)


def test_damaged_files_are_refused(tmp_path, level44):
    prob, arrays = level44
    path = os.path.join(tmp_path, "h.mgh")
    CK.save(path, prob, arrays)
    data = open(path, "rb").read()
    bad = bytearray(data)
    bad[-5] ^= 0xFF
    for blob, msg in ((bytes(bad), "checksum"), (data[:-7], "payload"),
                      (b"XXXXXXXX" + data[8:], "magic"), (data[:20], "header")):
        p2 = os.path.join(tmp_path, "bad.mgh")
        open(p2, "wb").write(blob)
        with pytest.raises(CK.CheckpointError) as e:
            CK.load(p2)
        assert msg in str(e.value)
