"""Run one stage of the fine-level setup on its own, for timing and for ncu.

    python -m paper_2502_03091_gb300.profile_case --stage truncate --dims 16 16 16 32 \
        --precision mixed --reps 1

Inputs are drawn on the device by the library's own generators (random links
exp(i eps H), Gaussian test vectors, normalised per vector); the parameters are
the 32^3x64 workload's (4^4 x 8 aggregates, m' = 64, k = 24, 20 MR iterations,
xi = 3.5, m0 = -0.4).  Two untimed calls come first, then --reps calls with the
library's per-kernel CUDA-event timing on; one JSON line per run gives the
per-kernel milliseconds per call.  Stages: smooth (mg_smooth_testvecs),
truncate (mg_chiral_truncate), coarsen (mg_build_prolongator + mg_coarsen),
level (all four).
"""
from __future__ import annotations

import argparse
import json

PRECISIONS = {"fp32": 0, "mixed": 1, "mixed_fp16": 2}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--stage", default="truncate", choices=["smooth", "truncate", "coarsen", "level"])
    ap.add_argument("--dims", type=int, nargs=4, default=[32, 32, 32, 64])
    ap.add_argument("--precision", default="mixed", choices=sorted(PRECISIONS))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=7)
    a = ap.parse_args(argv)

    import torch
    from . import build as _build
    _build.build()
    from . import mg

    p = mg.Problem(dims=a.dims, block=[4, 4, 4, 8], m0=-0.4, n_vec=64, k=24, mr_iters=20, xi=3.5,
                   precision=PRECISIONS[a.precision], seed=a.seed)
    U = torch.empty(mg.shape_U(p), dtype=torch.complex64, device="cuda")
    mg.mg_random_links(p, 0.2, U)
    psi0 = torch.empty(mg.shape_psi(p), dtype=torch.complex64, device="cuda")
    mg.mg_random_starts(p, psi0)
    psi0 /= torch.linalg.vector_norm(psi0.reshape(-1, p.n_vec), dim=0)
    psi = torch.empty_like(psi0)
    Uk = torch.empty(mg.shape_Uk(p), dtype=torch.complex64, device="cuda")
    sig = torch.empty(mg.shape_sigma(p), dtype=torch.float64, device="cuda")
    fl = torch.empty((p.n_blocks, 2), dtype=torch.int32, device="cuda")
    P = torch.empty(mg.shape_P(p), dtype=torch.complex64, device="cuda")
    X = torch.empty(mg.shape_X(p), dtype=torch.complex64, device="cuda")
    Y = torch.empty(mg.shape_Y(p), dtype=torch.complex64, device="cuda")
    ws_s = mg.workspace(p, mg.MG_CALL_SMOOTH) if a.stage in ("smooth", "level") else None
    ws_t = mg.workspace(p, mg.MG_CALL_TRUNCATE) if a.stage in ("truncate", "level") else None
    if a.stage in ("truncate", "coarsen"):
        psi.copy_(psi0)
    if a.stage == "coarsen":
        mg.mg_chiral_truncate(p, psi, Uk, sig, None, fl, mg.workspace(p, mg.MG_CALL_TRUNCATE))

    def run():
        if a.stage in ("smooth", "level"):
            mg.mg_smooth_testvecs(p, U, None, psi0, psi, ws_s)
        if a.stage in ("truncate", "level"):
            mg.mg_chiral_truncate(p, psi, Uk, sig, None, fl, ws_t)
        if a.stage in ("coarsen", "level"):
            mg.mg_build_prolongator(p, Uk, P)
            mg.mg_coarsen(p, U, None, P, X, Y)

    for _ in range(2):
        run()
    torch.cuda.synchronize()
    mg.mg_sync_status()
    mg.mg_timing_enable(True)
    mg.mg_timing_read()
    for _ in range(a.reps):
        run()
    torch.cuda.synchronize()
    mg.mg_sync_status()
    kern = mg.mg_timing_read()
    mg.mg_timing_enable(False)
    out = {"stage": a.stage, "dims": a.dims, "precision": a.precision, "reps": a.reps}
    if a.stage in ("truncate", "level"):
        out["blk_flags_nonzero"] = int((fl != 0).sum())
        out["sigma_block0"] = [round(v, 6) for v in sig[0, 0, :4].tolist()]
    out["kernels_ms_per_call"] = {n: round(t / a.reps, 3) for n, (_, t) in kern.items()}
    out["total_ms"] = round(sum(t for _, t in kern.values()) / a.reps, 2)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
