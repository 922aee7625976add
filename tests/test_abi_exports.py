"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/mg.h declares; host-side argument validation works without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2502_03091_gb300 import build as B
from paper_2502_03091_gb300 import mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mg.library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(mg.EXPORTS)


def test_version_and_validation(lib):
    assert "sm_103a" in mg.version()
    p = mg.Problem(dims=[4, 4, 4, 4], block=[3, 2, 2, 2], m0=0.0, n_vec=8, k=4, mr_iters=2)
    with pytest.raises(mg.MgError) as e:
        mg.mg_workspace_size(p, mg.MG_CALL_SMOOTH)
    assert "does not divide" in str(e.value)
    p = mg.Problem(dims=[4, 4, 4, 4], block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=9, mr_iters=2)
    with pytest.raises(mg.MgError):
        mg.mg_workspace_size(p, mg.MG_CALL_TRUNCATE)
    p = mg.Problem(dims=[4, 4, 4, 4], block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=4, mr_iters=2)
    V = 256
    # four complex64 fields of V x 12 x n_vec (two residual buffers, D r, psi) at least
    assert mg.mg_workspace_size(p, mg.MG_CALL_SMOOTH) >= 4 * V * 12 * 8 * 8
    assert mg.mg_workspace_size(p, mg.MG_CALL_TRUNCATE) > 0
    # NULL arrays are rejected before anything is launched
    pc = p.c()
    st = lib.mg_smooth_testvecs(ctypes.byref(pc), None, None, None, None, None, 0, None)
    assert st == 1 and b"NULL" in lib.mg_last_error()
    st = lib.mg_coarse_apply(ctypes.byref(pc), None, None, None, None, 8, None)
    assert st == 1
    # a coarse apply whose nine staged source vectors (9 x 2k x nrhs complex64)
    # exceed the 200000 bytes of shared memory is refused before any launch
    # (the pointers are never dereferenced: validation fails first)
    fake = [ctypes.c_void_p(256 * (i + 1)) for i in range(4)]
    big = mg.Problem(dims=[8, 8, 8, 16], block=[4, 4, 4, 8], m0=0.0, n_vec=64, k=24,
                     mr_iters=2).c()
    st = lib.mg_coarse_apply(ctypes.byref(big), *fake, 58, None)
    assert st == 7 and b"nrhs <= 57" in lib.mg_last_error()
    big = mg.Problem(dims=[8, 8, 8, 16], block=[4, 4, 4, 8], m0=0.0, n_vec=64, k=32,
                     mr_iters=2).c()
    st = lib.mg_coarse_apply(ctypes.byref(big), *fake, 44, None)
    assert st == 7 and b"nrhs <= 43" in lib.mg_last_error()


def test_coarse_level_validation(lib):
    """Levels l >= 1: problem checks and workspace sizes on the host."""
    cp = mg.CoarseProblem([8, 8, 8, 8], [2, 2, 2, 2], 24, 64, 32, 20)
    V, n, m = 4096, 48, 64
    # residual and D r fields plus one float4 partial per (site, vector)
    assert mg.mg_coarse_workspace_size(cp, mg.MG_CALL_SMOOTH) >= 2 * V * n * m * 8 + V * m * 16
    assert mg.mg_coarse_workspace_size(cp, mg.MG_CALL_TRUNCATE) > 0
    assert mg.mg_coarse_workspace_size(cp, mg.MG_CALL_COARSEN) == 0
    for bad, msg in ((dict(nc=33), "nc"), (dict(nc=0), "nc"), (dict(block=[3, 2, 2, 2]), "divide"),
                     (dict(n_vec=30), "n_vec"), (dict(k=33), "k ="),
                     (dict(nc=1, block=[1, 1, 1, 2], n_vec=8), "rows")):
        kw = dict(dims=[8, 8, 8, 8], block=[2, 2, 2, 2], nc=24, n_vec=64, k=32, mr_iters=20)
        kw.update(bad)
        with pytest.raises(mg.MgError) as e:
            mg.mg_coarse_workspace_size(mg.CoarseProblem(**kw), mg.MG_CALL_SMOOTH)
        assert msg in str(e.value), (bad, str(e.value))
    pc = cp.c()
    st = lib.mg_coarse_smooth_testvecs(ctypes.byref(pc), None, None, None, None, None, 0, None)
    assert st == 1 and b"NULL" in lib.mg_last_error()
    st = lib.mg_coarse_coarsen(ctypes.byref(pc), None, None, None, None, None, None)
    assert st == 1
    st = lib.mg_coarse_op_apply(ctypes.byref(pc), None, None, None, None, 8, None)
    assert st == 1
    cp0 = mg.CoarseProblem([8, 8, 8, 8], [2, 2, 2, 2], 24, 64, 32, 0)
    pc0 = cp0.c()
    st = lib.mg_coarse_smooth_testvecs(ctypes.byref(pc0), None, None, None, None, None, 0, None)
    assert st == 1 and b"mr_iters" in lib.mg_last_error()


def test_solve_validation(lib):
    """mg_solve: argument checks and workspace sizes on the host."""
    p = mg.Problem(dims=[8, 8, 8, 8], block=[2, 2, 2, 2], m0=-0.1, n_vec=48, k=24, mr_iters=10)
    cp = mg.CoarseProblem([4, 4, 4, 4], [2, 2, 2, 2], 24, 64, 32, 20)
    kc = mg.KCycle()

    def size(levels, nrhs=4, restart=16, **kw):
        h = mg._hierarchy(p, None, None, None, None, None, None, None, None, None,
                          mg.KCycle(**kw) if kw else kc)
        h.n_levels = levels
        if levels == 3:
            h.second = cp.c()
        return lib.mg_solve_workspace_size(ctypes.byref(h), nrhs, restart)

    V = 4096
    s1, s2, s3 = size(1), size(2), size(3)
    # one level: 4 + 17 fine vectors of 12 V x 4 complex64 at least
    assert s1 >= 21 * V * 12 * 4 * 8
    assert s2 > s1 and s3 > s1
    assert size(2, nrhs=12) == 0 and b"nrhs" in lib.mg_last_error()
    assert size(2, restart=0) == 0
    assert size(2, coarsest_iters=0) == 0
    assert size(4) == 0
    h = mg._hierarchy(p, None, None, None, None, None, None, None, None, None, kc)
    it = ctypes.c_int32(0)
    rel = (ctypes.c_double * 4)()
    st = lib.mg_solve(ctypes.byref(h), None, None, 4, 1e-5, 16, 10, ctypes.byref(it), rel, None,
                      0, None)
    assert st == 1


@pytest.mark.parametrize("bad, status, msg", [
    (dict(dims=[4, 4, 4, 0]), 2, "must be >= 1"),
    (dict(block=[2, 2, 2, 0]), 2, "must be >= 1"),
    (dict(block=[4, 4, 4, 3]), 2, "does not divide"),
    (dict(n_vec=0), 7, "n_vec"),
    (dict(n_vec=6), 7, "n_vec"),
    (dict(n_vec=68), 7, "n_vec"),
    (dict(k=0), 2, "k ="),
    (dict(k=9), 2, "k ="),
    (dict(xi=0.0), 1, "xi"),
    (dict(xi=float("nan")), 1, "xi"),
    (dict(precision=3), 7, "precision"),
    (dict(block=[1, 1, 1, 1], n_vec=8, k=4), 2, "rows"),
])
def test_problem_preconditions_are_rejected_on_the_host(lib, bad, status, msg):
    """The preconditions include/mg.h states for mg_problem (dims and block
    extents >= 1 with block | dims; 4 <= m' <= 64, m' % 4 == 0, 6|Lambda| >= m';
    1 <= k <= m'; xi > 0; a known precision) are checked before anything is
    launched, with the status and a message; the workspace query answers 0."""
    kw = dict(dims=[4, 4, 4, 4], block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=4, mr_iters=2)
    kw.update(bad)
    pc = mg.Problem(**kw).c()
    assert lib.mg_workspace_size(ctypes.byref(pc), mg.MG_CALL_SMOOTH) == 0
    assert msg in lib.mg_last_error().decode()
    fake = [ctypes.c_void_p(256 * (i + 1)) for i in range(6)]
    st = lib.mg_smooth_testvecs(ctypes.byref(pc), fake[0], None, fake[1], fake[2], fake[3],
                                1 << 30, None)
    assert st == status, (bad, st, lib.mg_last_error())
    st = lib.mg_chiral_truncate(ctypes.byref(pc), fake[0], fake[1], fake[2], None, fake[3],
                                fake[4], 1 << 30, None)
    assert st == status


def test_workspace_too_small_and_aliasing_are_rejected(lib):
    pc = mg.Problem(dims=[4, 4, 4, 4], block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=4,
                    mr_iters=2).c()
    need = lib.mg_workspace_size(ctypes.byref(pc), mg.MG_CALL_SMOOTH)
    fake = [ctypes.c_void_p(256 * (i + 1)) for i in range(6)]
    st = lib.mg_smooth_testvecs(ctypes.byref(pc), fake[0], None, fake[1], fake[2], fake[3],
                                need - 1, None)
    assert st == 1 and b"workspace" in lib.mg_last_error()
    st = lib.mg_apply_dirac(ctypes.byref(pc), fake[0], None, fake[1], fake[1], fake[3], need,
                            None)
    assert st == 1 and b"aliases" in lib.mg_last_error()
    st = lib.mg_coarse_apply(ctypes.byref(pc), fake[0], fake[1], fake[2], fake[2], 8, None)
    assert st == 1 and b"aliases" in lib.mg_last_error()
    for nrhs in (0, 65):
        st = lib.mg_coarse_apply(ctypes.byref(pc), fake[0], fake[1], fake[2], fake[3], nrhs, None)
        assert st == 1 and b"nrhs" in lib.mg_last_error()
    pc0 = mg.Problem(dims=[4, 4, 4, 4], block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=4,
                     mr_iters=0).c()
    st = lib.mg_smooth_testvecs(ctypes.byref(pc0), fake[0], None, fake[1], fake[2], fake[3],
                                1 << 30, None)
    assert st == 1 and b"mr_iters" in lib.mg_last_error()


def test_static_truncation_rejects_oversized_problem_before_any_cuda_call(lib):
    """mg_chiral_truncate_static refuses a problem whose truncation scratch
    exceeds its built-in 64 MiB before it touches the device."""
    pc = mg.Problem(dims=[16, 16, 16, 32], block=[4, 4, 4, 4], m0=0.0, n_vec=64, k=24,
                    mr_iters=2).c()
    assert lib.mg_workspace_size(ctypes.byref(pc), mg.MG_CALL_TRUNCATE) > 64 << 20
    fake = [ctypes.c_void_p(256 * (i + 1)) for i in range(4)]
    st = lib.mg_chiral_truncate_static(ctypes.byref(pc), fake[0], fake[1], fake[2], None,
                                       fake[3], None)
    assert st == 1 and b"built-in" in lib.mg_last_error()


def test_batch_descriptors_are_checked_before_any_cuda_call(lib):
    """mg_batch_create validates its arguments and every level descriptor
    (the problem and every array) before it tunes or captures anything."""
    out = ctypes.c_void_p()
    st = lib.mg_batch_create(None, 0, 0, None, ctypes.byref(out))
    assert st == 1 and b"no levels" in lib.mg_last_error() and not out.value
    good = mg.Problem(dims=[4, 4, 4, 4], block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=4,
                      mr_iters=2)
    descs = (mg._LevelDesc * 2)()
    for i, d in enumerate(descs):
        d.prob = good.c()
        for j, (name, t) in enumerate(mg._LevelDesc._fields_[1:]):
            setattr(d, name, 256 * (16 * i + j + 1))
    st = lib.mg_batch_create(descs, 2, 65, None, ctypes.byref(out))
    assert st == 1 and b"64 streams" in lib.mg_last_error()
    descs[1].psi = None
    st = lib.mg_batch_create(descs, 2, 1, None, ctypes.byref(out))
    assert st == 1 and b"level 1: NULL array" in lib.mg_last_error()
    descs[1].psi = 4096
    descs[0].prob = mg.Problem(dims=[4, 4, 4, 4], block=[3, 2, 2, 2], m0=0.0, n_vec=8, k=4,
                               mr_iters=2).c()
    st = lib.mg_batch_create(descs, 2, 1, None, ctypes.byref(out))
    err = lib.mg_last_error()
    assert st == 1 and b"level 0: " in err and b"does not divide" in err and not out.value


def test_generator_and_selftest_arguments_are_checked(lib):
    pc = mg.Problem(dims=[4, 4, 4, 4], block=[2, 2, 2, 2], m0=0.0, n_vec=8, k=4,
                    mr_iters=2).c()
    fake = ctypes.c_void_p(256)
    for eps in (-0.1, 1.5, float("nan")):
        st = lib.mg_random_links(ctypes.byref(pc), ctypes.c_double(eps), fake, None)
        assert st == 1 and b"eps" in lib.mg_last_error(), eps
    assert lib.mg_random_links(ctypes.byref(pc), ctypes.c_double(0.2), None, None) == 1
    assert lib.mg_random_starts(ctypes.byref(pc), None, None) == 1
    for polls in (0, (1 << 20) + 1):
        assert lib.mg_selftest_timeout(polls, None) == 1
        assert b"polls" in lib.mg_last_error()
