"""ctypes binding of libmg.so (include/mg.h).

Argument marshalling only: every step of the setup runs in the CUDA kernels
behind the C ABI.  Device arrays are torch tensors (complex64 / float64 /
int32, contiguous, on the current CUDA device); the current torch stream is
passed to the library unless a stream is given.  If the library is missing
or a call fails, an exception is raised -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmg.so")

MG_OK = 0
STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID", 2: "MG_ERR_SHAPE", 3: "MG_ERR_NOMEM",
                4: "MG_ERR_CUDA", 5: "MG_ERR_NUMERICAL", 6: "MG_ERR_TIMEOUT",
                7: "MG_ERR_UNSUPPORTED"}
MG_PREC_FP32 = 0
MG_PREC_MIXED = 1
MG_PREC_MIXED_FP16 = 2
MG_ERR_TIMEOUT = 6
MG_CALL_SMOOTH, MG_CALL_TRUNCATE, MG_CALL_COARSEN = 0, 1, 2

# every symbol include/mg.h declares
EXPORTS = ("mg_workspace_size", "mg_clover_field", "mg_apply_dirac", "mg_smooth_testvecs", "mg_chiral_truncate",
           "mg_build_prolongator", "mg_coarsen", "mg_coarse_apply", "mg_chiral_truncate_static",
           "mg_timing_enable",
           "mg_timing_read", "mg_batch_create", "mg_batch_launch", "mg_batch_streams",
           "mg_batch_destroy", "mg_tuned_pairs", "mg_sync_status", "mg_last_error", "mg_version",
           "mg_selftest_timeout", "mg_random_starts", "mg_random_links",
           "mg_coarse_workspace_size", "mg_coarse_op_apply", "mg_coarse_smooth_testvecs",
           "mg_coarse_chiral_truncate", "mg_coarse_build_prolongator", "mg_coarse_coarsen",
           "mg_solve_workspace_size", "mg_solve")


class MgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _TimingEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


class _Problem(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("block", ctypes.c_int32 * 4),
                ("m0", ctypes.c_double), ("csw", ctypes.c_double), ("xi", ctypes.c_double),
                ("n_vec", ctypes.c_int32), ("k", ctypes.c_int32), ("mr_iters", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class _CoarseProblem(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("block", ctypes.c_int32 * 4),
                ("nc", ctypes.c_int32), ("n_vec", ctypes.c_int32), ("k", ctypes.c_int32),
                ("mr_iters", ctypes.c_int32)]


class _Hierarchy(ctypes.Structure):
    _fields_ = [("fine", _Problem), ("U", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("P", ctypes.c_void_p), ("X", ctypes.c_void_p), ("Y", ctypes.c_void_p),
                ("n_levels", ctypes.c_int32), ("second", _CoarseProblem),
                ("P2", ctypes.c_void_p), ("X2", ctypes.c_void_p), ("Y2", ctypes.c_void_p),
                ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32),
                ("kcycle_iters", ctypes.c_int32), ("coarsest_iters", ctypes.c_int32)]


class _LevelDesc(ctypes.Structure):
    _fields_ = [("prob", _Problem), ("U", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("psi0", ctypes.c_void_p), ("psi", ctypes.c_void_p), ("Uk", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("blk_flags", ctypes.c_void_p),
                ("P", ctypes.c_void_p), ("X", ctypes.c_void_p), ("Y", ctypes.c_void_p),
                ("ws_smooth", ctypes.c_void_p), ("ws_smooth_bytes", ctypes.c_size_t),
                ("ws_trunc", ctypes.c_void_p), ("ws_trunc_bytes", ctypes.c_size_t)]


@dataclass
class Problem:
    """Python mirror of mg_problem."""
    dims: Sequence[int]
    block: Sequence[int]
    m0: float
    n_vec: int
    k: int
    mr_iters: int
    csw: float = 0.0
    xi: float = 1.0
    precision: int = MG_PREC_FP32
    seed: int = 0

    def c(self) -> _Problem:
        p = _Problem()
        p.dims[:] = [int(v) for v in self.dims]
        p.block[:] = [int(v) for v in self.block]
        p.m0, p.csw, p.xi = float(self.m0), float(self.csw), float(self.xi)
        p.n_vec, p.k, p.mr_iters = int(self.n_vec), int(self.k), int(self.mr_iters)
        p.precision, p.seed = int(self.precision), int(self.seed)
        return p

    # derived sizes
    @property
    def volume(self) -> int:
        v = 1
        for d in self.dims:
            v *= int(d)
        return v

    @property
    def block_volume(self) -> int:
        v = 1
        for d in self.block:
            v *= int(d)
        return v

    @property
    def coarse_dims(self):
        return [int(self.dims[i]) // int(self.block[i]) for i in range(4)]

    @property
    def n_blocks(self) -> int:
        return self.volume // self.block_volume


@dataclass
class CoarseProblem:
    """Python mirror of mg_coarse_problem: a level l >= 1 whose operator is the
    stencil (X, Y) with 2*nc components per site on the lattice dims."""
    dims: Sequence[int]
    block: Sequence[int]
    nc: int
    n_vec: int
    k: int
    mr_iters: int

    def c(self) -> _CoarseProblem:
        p = _CoarseProblem()
        p.dims[:] = [int(v) for v in self.dims]
        p.block[:] = [int(v) for v in self.block]
        p.nc, p.n_vec, p.k, p.mr_iters = int(self.nc), int(self.n_vec), int(self.k), int(self.mr_iters)
        return p

    volume = Problem.volume
    block_volume = Problem.block_volume
    coarse_dims = Problem.coarse_dims
    n_blocks = Problem.n_blocks

    @classmethod
    def below(cls, prob: "Problem", block, n_vec: int, k: int, mr_iters: int) -> "CoarseProblem":
        """The level under the fine problem prob: its lattice is prob's coarse
        lattice and its operator has 2 prob.k components per site."""
        return cls(prob.coarse_dims, block, prob.k, n_vec, k, mr_iters)


_lib = None


def library(path: str = LIB_PATH):
    """Load libmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_2502_03091_gb300.build`")
    lib = ctypes.CDLL(path)
    P, Pp = ctypes.c_void_p, ctypes.POINTER(_Problem)
    lib.mg_workspace_size.argtypes = [Pp, ctypes.c_int]
    lib.mg_workspace_size.restype = ctypes.c_size_t
    lib.mg_clover_field.argtypes = [Pp, P, P, P]
    lib.mg_apply_dirac.argtypes = [Pp, P, P, P, P, P, ctypes.c_size_t, P]
    lib.mg_smooth_testvecs.argtypes = [Pp, P, P, P, P, P, ctypes.c_size_t, P]
    lib.mg_chiral_truncate.argtypes = [Pp, P, P, P, P, P, P, ctypes.c_size_t, P]
    lib.mg_chiral_truncate_static.argtypes = [Pp, P, P, P, P, P, P]
    lib.mg_build_prolongator.argtypes = [Pp, P, P, P]
    lib.mg_coarsen.argtypes = [Pp, P, P, P, P, P, P, ctypes.c_size_t, P]
    lib.mg_coarse_apply.argtypes = [Pp, P, P, P, P, ctypes.c_int32, P]
    for f in ("mg_clover_field", "mg_apply_dirac", "mg_smooth_testvecs", "mg_chiral_truncate",
              "mg_chiral_truncate_static", "mg_build_prolongator", "mg_coarsen",
              "mg_coarse_apply"):
        getattr(lib, f).restype = ctypes.c_int
    Cp = ctypes.POINTER(_CoarseProblem)
    lib.mg_coarse_workspace_size.argtypes = [Cp, ctypes.c_int]
    lib.mg_coarse_workspace_size.restype = ctypes.c_size_t
    lib.mg_coarse_op_apply.argtypes = [Cp, P, P, P, P, ctypes.c_int32, P]
    lib.mg_coarse_smooth_testvecs.argtypes = [Cp, P, P, P, P, P, ctypes.c_size_t, P]
    lib.mg_coarse_chiral_truncate.argtypes = [Cp, P, P, P, P, P, P, ctypes.c_size_t, P]
    lib.mg_coarse_build_prolongator.argtypes = [Cp, P, P, P]
    lib.mg_coarse_coarsen.argtypes = [Cp, P, P, P, P, P, P]
    for f in ("mg_coarse_op_apply", "mg_coarse_smooth_testvecs", "mg_coarse_chiral_truncate",
              "mg_coarse_build_prolongator", "mg_coarse_coarsen"):
        getattr(lib, f).restype = ctypes.c_int
    Hp = ctypes.POINTER(_Hierarchy)
    lib.mg_solve_workspace_size.argtypes = [Hp, ctypes.c_int32, ctypes.c_int32]
    lib.mg_solve_workspace_size.restype = ctypes.c_size_t
    lib.mg_solve.argtypes = [Hp, P, P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                             ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_double), P, ctypes.c_size_t, P]
    lib.mg_solve.restype = ctypes.c_int
    lib.mg_timing_enable.argtypes = [ctypes.c_int]
    lib.mg_timing_enable.restype = ctypes.c_int
    lib.mg_timing_read.argtypes = [ctypes.POINTER(_TimingEntry), ctypes.c_int]
    lib.mg_timing_read.restype = ctypes.c_int
    lib.mg_batch_create.argtypes = [ctypes.POINTER(_LevelDesc), ctypes.c_int, ctypes.c_int, P,
                                    ctypes.POINTER(ctypes.c_void_p)]
    lib.mg_batch_create.restype = ctypes.c_int
    lib.mg_batch_launch.argtypes = [P, P]
    lib.mg_batch_launch.restype = ctypes.c_int
    lib.mg_batch_streams.argtypes = [P]
    lib.mg_batch_streams.restype = ctypes.c_int
    lib.mg_batch_destroy.argtypes = [P]
    lib.mg_batch_destroy.restype = None
    lib.mg_tuned_pairs.argtypes = [Pp]
    lib.mg_tuned_pairs.restype = ctypes.c_int
    lib.mg_sync_status.argtypes = [P]
    lib.mg_sync_status.restype = ctypes.c_int
    lib.mg_selftest_timeout.argtypes = [ctypes.c_int32, P]
    lib.mg_selftest_timeout.restype = ctypes.c_int
    lib.mg_random_starts.argtypes = [Pp, P, P]
    lib.mg_random_starts.restype = ctypes.c_int
    lib.mg_random_links.argtypes = [Pp, ctypes.c_double, P, P]
    lib.mg_random_links.restype = ctypes.c_int
    lib.mg_last_error.restype = ctypes.c_char_p
    lib.mg_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int):
    if st != MG_OK:
        raise MgError(st, library().mg_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _expect(t, shape, dtype, name):
    if t is None:
        return
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype} != {dtype}")


def version() -> str:
    return library().mg_version().decode()


def mg_timing_enable(on: bool = True):
    _check(library().mg_timing_enable(1 if on else 0))


def mg_timing_read() -> dict:
    """{kernel name: (launches, total ms)} since the previous read (then reset)."""
    buf = (_TimingEntry * 64)()
    n = library().mg_timing_read(buf, 64)
    if n < 0:
        raise MgError(4, library().mg_last_error().decode())
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(n)}


def mg_sync_status(stream=None):
    """Waits for the stream; raises MgError (MG_ERR_TIMEOUT) if a smoother or
    operator pass enqueued since the previous call gave up waiting for its
    staged input."""
    _check(library().mg_sync_status(_stream(stream)))


def mg_random_starts(prob: Problem, psi0, stream=None):
    """psi0 <- the counter-based starting vectors of prob.seed (see include/mg.h)."""
    import torch
    _expect(psi0, shape_psi(prob), torch.complex64, "psi0")
    pc = prob.c()
    _check(library().mg_random_starts(ctypes.byref(pc), _ptr(psi0), _stream(stream)))


def mg_random_links(prob: Problem, eps: float, U, stream=None):
    """U <- exp(i eps H) links of the counter-based generator of prob.seed."""
    import torch
    _expect(U, shape_U(prob), torch.complex64, "U")
    pc = prob.c()
    _check(library().mg_random_links(ctypes.byref(pc), float(eps), _ptr(U), _stream(stream)))


def mg_selftest_timeout(polls: int, stream=None):
    """Enqueues the failure-detection self-test: one bounded device wait that
    runs out after `polls` polls and records a timeout (see include/mg.h)."""
    _check(library().mg_selftest_timeout(int(polls), _stream(stream)))


def mg_workspace_size(prob: Problem, which: int) -> int:
    pc = prob.c()
    n = library().mg_workspace_size(ctypes.byref(pc), which)
    if n == 0 and which != MG_CALL_COARSEN:
        raise MgError(1, library().mg_last_error().decode())
    return int(n)


def workspace(prob: Problem, which: int, device=None):
    """A uint8 CUDA tensor of mg_workspace_size(prob, which) bytes (at least 256)."""
    import torch
    return torch.empty(max(256, mg_workspace_size(prob, which)), dtype=torch.uint8,
                       device=device or "cuda")


# ---------------------------------------------------------------------------
# shapes of the ABI arrays
# ---------------------------------------------------------------------------
def shape_U(p: Problem):
    return (p.volume, 4, 3, 3)


def shape_C(p: Problem):
    return (p.volume, 2, 6, 6)


def shape_psi(p: Problem):
    return (p.volume, 4, 3, p.n_vec)


def shape_Uk(p: Problem):
    return (p.n_blocks, 2, p.block_volume, 2, 3, p.k)


def shape_sigma(p: Problem):
    return (p.n_blocks, 2, p.k)


def shape_P(p: Problem):
    return (p.volume, 2, 2, 3, p.k)


def shape_X(p: Problem):
    return (p.n_blocks, 2 * p.k, 2 * p.k)


def shape_Y(p: Problem):
    return (p.n_blocks, 8, 2 * p.k, 2 * p.k)


# ---------------------------------------------------------------------------
# the ABI calls
# ---------------------------------------------------------------------------
def mg_clover_field(prob: Problem, U, C, stream=None):
    import torch
    _expect(U, shape_U(prob), torch.complex64, "U")
    _expect(C, shape_C(prob), torch.complex64, "C")
    pc = prob.c()
    _check(library().mg_clover_field(ctypes.byref(pc), _ptr(U), _ptr(C), _stream(stream)))


def mg_apply_dirac(prob: Problem, U, C, v_in, v_out, ws, stream=None):
    """out = D in for n_vec right-hand sides ([V][4][3][n_vec] complex64)."""
    import torch
    _expect(U, shape_U(prob), torch.complex64, "U")
    _expect(C, shape_C(prob), torch.complex64, "C")
    _expect(v_in, shape_psi(prob), torch.complex64, "in")
    _expect(v_out, shape_psi(prob), torch.complex64, "out")
    pc = prob.c()
    _check(library().mg_apply_dirac(ctypes.byref(pc), _ptr(U), _ptr(C), _ptr(v_in), _ptr(v_out),
                                    _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def mg_smooth_testvecs(prob: Problem, U, C, psi0, psi, ws, stream=None):
    import torch
    _expect(U, shape_U(prob), torch.complex64, "U")
    _expect(C, shape_C(prob), torch.complex64, "C")
    _expect(psi0, shape_psi(prob), torch.complex64, "psi0")
    _expect(psi, shape_psi(prob), torch.complex64, "psi")
    pc = prob.c()
    _check(library().mg_smooth_testvecs(ctypes.byref(pc), _ptr(U), _ptr(C), _ptr(psi0), _ptr(psi),
                                        _ptr(ws), ws.numel() * ws.element_size(),
                                        _stream(stream)))


def mg_chiral_truncate(prob: Problem, psi, Uk, sigma, coarse_tv, blk_flags, ws, stream=None):
    import torch
    _expect(psi, shape_psi(prob), torch.complex64, "psi")
    _expect(Uk, shape_Uk(prob), torch.complex64, "Uk")
    _expect(sigma, shape_sigma(prob), torch.float64, "sigma")
    _expect(coarse_tv, (prob.n_blocks, 2, prob.k, prob.n_vec), torch.complex64, "coarse_tv")
    _expect(blk_flags, (prob.n_blocks, 2), torch.int32, "blk_flags")
    pc = prob.c()
    _check(library().mg_chiral_truncate(ctypes.byref(pc), _ptr(psi), _ptr(Uk), _ptr(sigma),
                                        _ptr(coarse_tv), _ptr(blk_flags), _ptr(ws),
                                        ws.numel() * ws.element_size(), _stream(stream)))


def mg_chiral_truncate_static(prob: Problem, psi, Uk, sigma, coarse_tv, blk_flags, stream=None):
    """mg_chiral_truncate without a workspace argument: for callers that cannot
    allocate device memory; scratch is a fixed 64 MiB array inside libmg.so."""
    import torch
    _expect(psi, shape_psi(prob), torch.complex64, "psi")
    _expect(Uk, shape_Uk(prob), torch.complex64, "Uk")
    _expect(sigma, shape_sigma(prob), torch.float64, "sigma")
    _expect(coarse_tv, (prob.n_blocks, 2, prob.k, prob.n_vec), torch.complex64, "coarse_tv")
    _expect(blk_flags, (prob.n_blocks, 2), torch.int32, "blk_flags")
    pc = prob.c()
    _check(library().mg_chiral_truncate_static(ctypes.byref(pc), _ptr(psi), _ptr(Uk),
                                               _ptr(sigma), _ptr(coarse_tv), _ptr(blk_flags),
                                               _stream(stream)))


def mg_build_prolongator(prob: Problem, Uk, P, stream=None):
    import torch
    _expect(Uk, shape_Uk(prob), torch.complex64, "Uk")
    _expect(P, shape_P(prob), torch.complex64, "P")
    pc = prob.c()
    _check(library().mg_build_prolongator(ctypes.byref(pc), _ptr(Uk), _ptr(P), _stream(stream)))


def mg_coarsen(prob: Problem, U, C, P, X, Y, ws=None, stream=None):
    import torch
    _expect(U, shape_U(prob), torch.complex64, "U")
    _expect(C, shape_C(prob), torch.complex64, "C")
    _expect(P, shape_P(prob), torch.complex64, "P")
    _expect(X, shape_X(prob), torch.complex64, "X")
    _expect(Y, shape_Y(prob), torch.complex64, "Y")
    pc = prob.c()
    nbytes = 0 if ws is None else ws.numel() * ws.element_size()
    _check(library().mg_coarsen(ctypes.byref(pc), _ptr(U), _ptr(C), _ptr(P), _ptr(X), _ptr(Y),
                                _ptr(ws), nbytes, _stream(stream)))


def mg_coarse_apply(prob: Problem, X, Y, v_in, v_out, stream=None):
    import torch
    nrhs = int(v_in.shape[-1])
    _expect(X, shape_X(prob), torch.complex64, "X")
    _expect(Y, shape_Y(prob), torch.complex64, "Y")
    _expect(v_in, (prob.n_blocks, 2 * prob.k, nrhs), torch.complex64, "v_in")
    _expect(v_out, (prob.n_blocks, 2 * prob.k, nrhs), torch.complex64, "v_out")
    pc = prob.c()
    _check(library().mg_coarse_apply(ctypes.byref(pc), _ptr(X), _ptr(Y), _ptr(v_in), _ptr(v_out),
                                     nrhs, _stream(stream)))


# ---------------------------------------------------------------------------
# levels l >= 1
# ---------------------------------------------------------------------------
def shape_cX(cp: CoarseProblem):
    return (cp.volume, 2 * cp.nc, 2 * cp.nc)


def shape_cY(cp: CoarseProblem):
    return (cp.volume, 8, 2 * cp.nc, 2 * cp.nc)


def shape_cvec(cp: CoarseProblem, nrhs: int):
    return (cp.volume, 2 * cp.nc, nrhs)


def shape_cUk(cp: CoarseProblem):
    return (cp.n_blocks, 2, cp.block_volume, cp.nc, cp.k)


def shape_cP(cp: CoarseProblem):
    return (cp.volume, 2, cp.nc, cp.k)


def shape_cX2(cp: CoarseProblem):
    return (cp.n_blocks, 2 * cp.k, 2 * cp.k)


def shape_cY2(cp: CoarseProblem):
    return (cp.n_blocks, 8, 2 * cp.k, 2 * cp.k)


def mg_coarse_workspace_size(cp: CoarseProblem, which: int) -> int:
    pc = cp.c()
    n = library().mg_coarse_workspace_size(ctypes.byref(pc), which)
    if n == 0 and which != MG_CALL_COARSEN:
        raise MgError(1, library().mg_last_error().decode())
    return int(n)


def coarse_workspace(cp: CoarseProblem, which: int, device=None):
    import torch
    return torch.empty(max(256, mg_coarse_workspace_size(cp, which)), dtype=torch.uint8,
                       device=device or "cuda")


def mg_coarse_op_apply(cp: CoarseProblem, X, Y, v_in, v_out, stream=None):
    """v_out = D_l v_in on cp's lattice (only dims and nc are used)."""
    import torch
    nrhs = int(v_in.shape[-1])
    _expect(X, shape_cX(cp), torch.complex64, "X")
    _expect(Y, shape_cY(cp), torch.complex64, "Y")
    _expect(v_in, shape_cvec(cp, nrhs), torch.complex64, "v_in")
    _expect(v_out, shape_cvec(cp, nrhs), torch.complex64, "v_out")
    pc = cp.c()
    _check(library().mg_coarse_op_apply(ctypes.byref(pc), _ptr(X), _ptr(Y), _ptr(v_in),
                                        _ptr(v_out), nrhs, _stream(stream)))


def mg_coarse_smooth_testvecs(cp: CoarseProblem, X, Y, psi0, psi, ws, stream=None):
    import torch
    _expect(X, shape_cX(cp), torch.complex64, "X")
    _expect(Y, shape_cY(cp), torch.complex64, "Y")
    _expect(psi0, shape_cvec(cp, cp.n_vec), torch.complex64, "psi0")
    _expect(psi, shape_cvec(cp, cp.n_vec), torch.complex64, "psi")
    pc = cp.c()
    _check(library().mg_coarse_smooth_testvecs(ctypes.byref(pc), _ptr(X), _ptr(Y), _ptr(psi0),
                                               _ptr(psi), _ptr(ws),
                                               ws.numel() * ws.element_size(), _stream(stream)))


def mg_coarse_chiral_truncate(cp: CoarseProblem, psi, Uk, sigma, coarse_tv, blk_flags, ws,
                              stream=None):
    import torch
    _expect(psi, shape_cvec(cp, cp.n_vec), torch.complex64, "psi")
    _expect(Uk, shape_cUk(cp), torch.complex64, "Uk")
    _expect(sigma, (cp.n_blocks, 2, cp.k), torch.float64, "sigma")
    _expect(coarse_tv, (cp.n_blocks, 2, cp.k, cp.n_vec), torch.complex64, "coarse_tv")
    _expect(blk_flags, (cp.n_blocks, 2), torch.int32, "blk_flags")
    pc = cp.c()
    _check(library().mg_coarse_chiral_truncate(ctypes.byref(pc), _ptr(psi), _ptr(Uk),
                                               _ptr(sigma), _ptr(coarse_tv), _ptr(blk_flags),
                                               _ptr(ws), ws.numel() * ws.element_size(),
                                               _stream(stream)))


def mg_coarse_build_prolongator(cp: CoarseProblem, Uk, P, stream=None):
    import torch
    _expect(Uk, shape_cUk(cp), torch.complex64, "Uk")
    _expect(P, shape_cP(cp), torch.complex64, "P")
    pc = cp.c()
    _check(library().mg_coarse_build_prolongator(ctypes.byref(pc), _ptr(Uk), _ptr(P),
                                                 _stream(stream)))


def mg_coarse_coarsen(cp: CoarseProblem, X, Y, P, X2, Y2, stream=None):
    import torch
    _expect(X, shape_cX(cp), torch.complex64, "X")
    _expect(Y, shape_cY(cp), torch.complex64, "Y")
    _expect(P, shape_cP(cp), torch.complex64, "P")
    _expect(X2, shape_cX2(cp), torch.complex64, "X2")
    _expect(Y2, shape_cY2(cp), torch.complex64, "Y2")
    pc = cp.c()
    _check(library().mg_coarse_coarsen(ctypes.byref(pc), _ptr(X), _ptr(Y), _ptr(P), _ptr(X2),
                                       _ptr(Y2), _stream(stream)))


@dataclass
class CoarseLevel:
    """Device buffers of one level l >= 1 (its operator X, Y comes from the
    level above)."""
    prob: CoarseProblem
    X: object
    Y: object
    psi0: object
    psi: object = None
    Uk: object = None
    sigma: object = None
    flags: object = None
    P: object = None
    X2: object = None
    Y2: object = None
    ws_smooth: object = None
    ws_trunc: object = None

    @classmethod
    def allocate(cls, cp: CoarseProblem, X, Y, psi0):
        import torch
        dev, c64 = X.device, torch.complex64
        lv = cls(cp, X, Y, psi0)
        lv.psi = torch.empty(shape_cvec(cp, cp.n_vec), dtype=c64, device=dev)
        lv.Uk = torch.empty(shape_cUk(cp), dtype=c64, device=dev)
        lv.sigma = torch.empty((cp.n_blocks, 2, cp.k), dtype=torch.float64, device=dev)
        lv.flags = torch.empty((cp.n_blocks, 2), dtype=torch.int32, device=dev)
        lv.P = torch.empty(shape_cP(cp), dtype=c64, device=dev)
        lv.X2 = torch.empty(shape_cX2(cp), dtype=c64, device=dev)
        lv.Y2 = torch.empty(shape_cY2(cp), dtype=c64, device=dev)
        lv.ws_smooth = coarse_workspace(cp, MG_CALL_SMOOTH, dev)
        lv.ws_trunc = coarse_workspace(cp, MG_CALL_TRUNCATE, dev)
        return lv

    def run(self, stream=None):
        """Smoother -> sigma_3 truncation -> prolongator -> next coarse operator."""
        p = self.prob
        mg_coarse_smooth_testvecs(p, self.X, self.Y, self.psi0, self.psi, self.ws_smooth, stream)
        mg_coarse_chiral_truncate(p, self.psi, self.Uk, self.sigma, None, self.flags,
                                  self.ws_trunc, stream)
        mg_coarse_build_prolongator(p, self.Uk, self.P, stream)
        mg_coarse_coarsen(p, self.X, self.Y, self.P, self.X2, self.Y2, stream)


# ---------------------------------------------------------------------------
# the solve (FGMRES preconditioned by the K-cycle over the hierarchy)
# ---------------------------------------------------------------------------
@dataclass
class KCycle:
    """K-cycle parameters of mg_solve."""
    nu_pre: int = 2
    nu_post: int = 2
    kcycle_iters: int = 2
    coarsest_iters: int = 32


def _hierarchy(prob: Problem, U, C, P, X, Y, second, P2, X2, Y2, kc: KCycle) -> _Hierarchy:
    h = _Hierarchy()
    h.fine = prob.c()
    h.U, h.C, h.P, h.X, h.Y = _ptr(U), _ptr(C), _ptr(P), _ptr(X), _ptr(Y)
    h.n_levels = 1 if P is None else (2 if second is None else 3)
    if second is not None:
        h.second = second.c()
        h.P2, h.X2, h.Y2 = _ptr(P2), _ptr(X2), _ptr(Y2)
    h.nu_pre, h.nu_post = int(kc.nu_pre), int(kc.nu_post)
    h.kcycle_iters, h.coarsest_iters = int(kc.kcycle_iters), int(kc.coarsest_iters)
    return h


def mg_solve(prob: Problem, U, C, b, x, tol: float, restart: int = 16, max_iters: int = 500,
             P=None, X=None, Y=None, second: Optional[CoarseProblem] = None, P2=None, X2=None,
             Y2=None, kcycle: KCycle = KCycle(), ws=None, stream=None):
    """Solve D x = b for the nrhs = b.shape[-1] systems of b ([V][4][3][nrhs]),
    preconditioned by the K-cycle over the levels given (none: plain GMRES;
    P, X, Y: two levels; plus second, P2, X2, Y2: three levels).  Returns
    (outer steps, per-system true relative residuals)."""
    import numpy as np
    import torch
    nrhs = int(b.shape[-1])
    _expect(b, (prob.volume, 4, 3, nrhs), torch.complex64, "b")
    _expect(x, (prob.volume, 4, 3, nrhs), torch.complex64, "x")
    h = _hierarchy(prob, U, C, P, X, Y, second, P2, X2, Y2, kcycle)
    lib = library()
    need = lib.mg_solve_workspace_size(ctypes.byref(h), nrhs, restart)
    if need == 0:
        raise MgError(1, lib.mg_last_error().decode())
    if ws is None or ws.numel() * ws.element_size() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=b.device)
    iters = ctypes.c_int32(0)
    rel = (ctypes.c_double * nrhs)()
    _check(lib.mg_solve(ctypes.byref(h), _ptr(b), _ptr(x), nrhs, float(tol), int(restart),
                        int(max_iters), ctypes.byref(iters), rel, _ptr(ws),
                        ws.numel() * ws.element_size(), _stream(stream)))
    return int(iters.value), np.array(rel[:])


# ---------------------------------------------------------------------------
# one level of the setup, buffers owned by torch
# ---------------------------------------------------------------------------
@dataclass
class Level:
    """Device buffers of one setup level (inputs, outputs and scratch)."""
    prob: Problem
    U: object
    C: object
    psi0: object
    psi: object = None
    Uk: object = None
    sigma: object = None
    flags: object = None
    P: object = None
    X: object = None
    Y: object = None
    ws_smooth: object = None
    ws_trunc: object = None
    coarse_tv: object = None
    extra: dict = field(default_factory=dict)

    @classmethod
    def allocate(cls, prob: Problem, U, C, psi0, want_coarse_tv: bool = False):
        import torch
        dev = U.device
        c64 = torch.complex64
        lv = cls(prob, U, C, psi0)
        lv.psi = torch.empty(shape_psi(prob), dtype=c64, device=dev)
        lv.Uk = torch.empty(shape_Uk(prob), dtype=c64, device=dev)
        lv.sigma = torch.empty(shape_sigma(prob), dtype=torch.float64, device=dev)
        lv.flags = torch.empty((prob.n_blocks, 2), dtype=torch.int32, device=dev)
        lv.P = torch.empty(shape_P(prob), dtype=c64, device=dev)
        lv.X = torch.empty(shape_X(prob), dtype=c64, device=dev)
        lv.Y = torch.empty(shape_Y(prob), dtype=c64, device=dev)
        lv.ws_smooth = workspace(prob, MG_CALL_SMOOTH, dev)
        lv.ws_trunc = workspace(prob, MG_CALL_TRUNCATE, dev)
        if want_coarse_tv:
            lv.coarse_tv = torch.empty((prob.n_blocks, 2, prob.k, prob.n_vec), dtype=c64,
                                       device=dev)
        return lv

    def run(self, stream=None):
        """Smoother -> chiral truncation -> prolongator -> coarse operator."""
        p = self.prob
        mg_smooth_testvecs(p, self.U, self.C, self.psi0, self.psi, self.ws_smooth, stream)
        mg_chiral_truncate(p, self.psi, self.Uk, self.sigma, self.coarse_tv, self.flags,
                           self.ws_trunc, stream)
        mg_build_prolongator(p, self.Uk, self.P, stream)
        mg_coarsen(p, self.U, self.C, self.P, self.X, self.Y, None, stream)


class Batch:
    """mg_batch_create / mg_batch_launch / mg_batch_destroy over a list of
    allocated Levels (every level's arrays must stay alive with the batch)."""

    def __init__(self, levels, n_streams: int = 0, stream=None):
        self.levels = list(levels)
        descs = (_LevelDesc * len(self.levels))()
        for d, lv in zip(descs, self.levels):
            d.prob = lv.prob.c()
            d.U, d.C, d.psi0 = _ptr(lv.U), _ptr(lv.C), _ptr(lv.psi0)
            d.psi, d.Uk, d.sigma = _ptr(lv.psi), _ptr(lv.Uk), _ptr(lv.sigma)
            d.blk_flags, d.P, d.X, d.Y = _ptr(lv.flags), _ptr(lv.P), _ptr(lv.X), _ptr(lv.Y)
            d.ws_smooth, d.ws_smooth_bytes = _ptr(lv.ws_smooth), lv.ws_smooth.numel()
            d.ws_trunc, d.ws_trunc_bytes = _ptr(lv.ws_trunc), lv.ws_trunc.numel()
        self._descs = descs
        h = ctypes.c_void_p()
        _check(library().mg_batch_create(descs, len(self.levels), int(n_streams),
                                          _stream(stream), ctypes.byref(h)))
        self._h = h

    @property
    def n_streams(self) -> int:
        return int(library().mg_batch_streams(self._h))

    def launch(self, stream=None):
        _check(library().mg_batch_launch(self._h, _stream(stream)))

    def close(self):
        if self._h:
            library().mg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def mg_tuned_pairs(prob: Problem) -> int:
    pc = prob.c()
    return int(library().mg_tuned_pairs(ctypes.byref(pc)))
