"""The chunked and column-wise draws of the test-vector starts give the same
numbers as the whole-array draw (they stand in for it on lattices whose full
start set is too large to draw at once)."""
import numpy as np

import mg_inputs as G


def test_psi0_sites_and_columns_match_full_draw():
    d, m, seed = [4, 4, 2, 6], 8, 7
    full = G.psi0(d, m, seed)
    assert np.array_equal(G.psi0_sites(d, m, seed, 5, 40), full[5:40])
    assert np.array_equal(G.psi0_sites(d, m, seed, 0, G.volume(d)), full)
    assert np.array_equal(G.psi0_columns(d, m, seed, [1, 6]), full[..., [1, 6]])
    assert np.array_equal(G.psi0_columns(d, m, seed, [3]), full[..., [3]])


def test_random_su3_chunks_match_gauge_field():
    d, eps, seed = [2, 2, 2, 4], 0.3, 5
    U = G.gauge_field(d, eps, seed)
    n = 4 * G.volume(d)
    parts = [G.random_su3(seed, G.STREAM_GAUGE, b - a, eps, start=a)
             for a, b in ((0, 37), (37, 100), (100, n))]
    assert np.allclose(np.concatenate(parts).reshape(U.shape), U, rtol=0, atol=1e-15)


def test_threaded_gauge_field_matches():
    d, eps, seed = [8, 8, 8, 8], 0.25, 3
    assert np.array_equal(G.gauge_field(d, eps, seed, threads=4), G.gauge_field(d, eps, seed))


def test_threaded_psi0_matches():
    d, m, seed = [8, 8, 8, 8], 8, 4
    assert np.array_equal(G.psi0(d, m, seed, threads=3), G.psi0(d, m, seed))


def test_batch_workload_draw():
    w = G.batch_workload(30)
    assert len(w) == 24
    assert [h["dims"] for h in w] == [[8] * 4] * 8 + [[12, 12, 12, 24]] * 8 + [[16, 16, 16, 32]] * 8
    for h in w:
        assert h["m"] in (32, 48, 64) and h["k"] in (16, 24) and h["block"] in ([2] * 4, [4] * 4)
        assert 0.15 <= h["eps"] <= 0.35
        assert 6 * int(np.prod(h["block"])) >= h["m"] and h["k"] <= h["m"]
    assert w == G.batch_workload(30)          # a pure function of the seed
    assert w != G.batch_workload(31)
