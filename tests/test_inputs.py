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


def test_stencil_operator_structure_and_chunking():
    """The random level-l operator has the coarse-operator symmetry
    (sigma_3 D is Hermitian) and does not depend on how it is drawn."""
    cd, nc = [2, 3, 2, 2], 3
    X, Y = G.stencil_operator(cd, nc, 7)
    X4, Y4 = G.stencil_operator(cd, nc, 7, threads=4)
    assert np.array_equal(X, X4) and np.array_equal(Y, Y4)
    V, n = G.volume(cd), 2 * nc
    D = np.zeros((V * n, V * n), dtype=np.complex128)
    s = np.arange(V)
    c = [s % 2, (s // 2) % 3, (s // 6) % 2, s // 12]
    for x in range(V):
        D[x * n:(x + 1) * n, x * n:(x + 1) * n] += X[x]
        for d in range(8):
            mu, st = d % 4, (1 if d < 4 else -1)
            cc = [a[x] for a in c]
            cc[mu] = (cc[mu] + st) % cd[mu]
            y = cc[0] + 2 * (cc[1] + 3 * (cc[2] + 2 * cc[3]))
            D[x * n:(x + 1) * n, y * n:(y + 1) * n] += Y[x, d]
    s3 = np.tile(np.r_[np.ones(nc), -np.ones(nc)], V)
    H = s3[:, None] * D
    assert np.abs(H - H.conj().T).max() < 1e-12


def test_splitmix64_published_sequence():
    """SplitMix64 from state 0 (the state advances by the golden gamma
    0x9E3779B97F4A7C15 per step) gives the generator's published first
    outputs."""
    gamma = 0x9E3779B97F4A7C15
    states = np.array([0, gamma, (2 * gamma) % 2 ** 64], dtype=np.uint64)
    got = [int(v) for v in G.splitmix64(states)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniforms_and_normals_distribution():
    """Uniforms lie strictly inside (0, 1) with mean 1/2 and variance 1/12;
    the Box-Muller normals have mean 0, variance 1 and fourth moment 3
    (bounds: five standard errors of each sample moment)."""
    n = 1 << 20
    u = G.uniforms(7, G.STREAM_MISC, 0, n)
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    z = G.normals(7, G.STREAM_MISC, 0, n)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * np.sqrt(96 / n)
