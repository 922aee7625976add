#!/usr/bin/env python
"""Benchmark of one setup level of the chiral rank-k multigrid (arXiv:2502.03091)
on the 32^3x64 anisotropic workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole setup path through the C ABI on inputs that
are already resident in HBM: MR smoother (20 iterations, m' = 64) -> chiral
split + rank-24 truncation -> prolongator -> Galerkin coarse operator -> one
coarse apply (8 right-hand sides).  The metric is seconds per setup level
(lower is better).  Printed as one JSON line by rank 0.

Multi-GPU: every rank builds its own level (independent replicas, no
data-path collective); value = (max over ranks of the time per step) / N.

--impl reference times the FP64 CPU oracle (the checker of this project) on
the host cores, on a bounded sub-lattice sample of the same workload, scaled
to the full lattice.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MG setup s/level at 32^3x64, mixed vs FP32 plain; dslash HBM GB/s; p50/p99 setup"
UNIT = "s/level"


def _m0_table():
    with open(os.path.join(ROOT, "tests", "golden", "m0.json")) as fh:
        return {k: v["m0"] for k, v in json.load(fh)["workloads"].items()}


def workload(name: str):
    m0 = _m0_table()
    if name == "32^3x64":
        return dict(workload="32^3x64 anisotropic (xi=3.5) Wilson, eps=0.2, m'=64, k=24, "
                             "4^3x8 aggregates, 20 MR iterations",
                    dims=[32, 32, 32, 64], block=[4, 4, 4, 8], eps=0.2, csw=0.0, xi=3.5,
                    m=64, k=24, N=20, m0=m0["32^3x64 aniso xi=3.5 eps=0.2"], gauge_seed=20,
                    psi_seed=21, sample_dims=[8, 8, 8, 16])
    if name == "16^3x32-aniso":
        # the 32^3x64 parameters on 1/16 of the volume: kernel-profiling case
        w = workload("32^3x64")
        w.update(workload="16^3x32 anisotropic (xi=3.5) Wilson, eps=0.2, m'=64, k=24, "
                          "4^3x8 aggregates, 20 MR iterations",
                 dims=[16, 16, 16, 32], sample_dims=[8, 8, 8, 16])
        return w
    if name == "16^3x32":
        return dict(workload="16^3x32 Wilson-clover c_sw=1, eps=0.25, m'=48, k=24, 4^4 "
                             "aggregates, 20 MR iterations",
                    dims=[16, 16, 16, 32], block=[4, 4, 4, 4], eps=0.25, csw=1.0, xi=1.0,
                    m=48, k=24, N=20, m0=m0["16^3x32 Wilson-clover eps=0.25"], gauge_seed=10,
                    psi_seed=11, sample_dims=[8, 8, 8, 8])
    raise SystemExit(f"unknown workload {name}")


def vol(d):
    return int(d[0]) * int(d[1]) * int(d[2]) * int(d[3])


# ---------------------------------------------------------------------------
# algorithmic work per kernel launch (what the method must move or compute)
# ---------------------------------------------------------------------------
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # CUDA-core FP32 FMA peak at max clock
PEAK_SOURCE = {"fp32": "nominal FP32: 152 SMs x 128 FMA lanes x 2 flop x 2.07 GHz"}


def dslash_bytes(w, prec="fp32"):
    """One dslash pass: read 12 + write 12 complex numbers per site and
    right-hand side (192 B in complex64, 96 B in FP16), plus links (288 B) and
    clover (288 B) per site."""
    per_site = (96 if prec == "mixed_fp16" else 192) * w["m"] + 288 + (288 if w["csw"] else 0)
    return vol(w["dims"]) * per_site


def kernel_work(w, prec="fp32"):
    """{kernel: (bound, amount, unit)} -- bytes for HBM-bound kernels, flop for
    arithmetic-bound ones (per launch).  prec "mixed_fp16": the smoother's
    fields are FP16 (half the bytes of complex64).  The tensor-core kernels of
    the mixed paths are counted by the bytes they must move (their arithmetic
    runs far below the tensor pipe's rate)."""
    V, m, k = vol(w["dims"]), w["m"], w["k"]
    nb = vol(w["block"])
    nbc = 2 * V // nb
    K = 6 * nb
    abi = V * 96 * m  # one complex64 field [V][4][3][m] (the interface)
    spinor = abi // 2 if prec == "mixed_fp16" else abi  # one smoother field
    uk = V * 12 * k * 8  # U_k (and P): [V][2][6][k] complex64
    xy = (V // nb) * 9 * (2 * k) ** 2 * 8  # X and Y
    n_upd = max(w["N"] - 1, 1)
    upd_streams = (3 * ((w["N"] - 1 + 1) // 2) + 6 * ((w["N"] - 1) // 2)) / n_upd
    return {
        "mr_input_norm": ("hbm", abi, "B"),
        "mr_to_slab": ("hbm", abi + spinor, "B"),
        "mr_neg_dslash": ("hbm", dslash_bytes(w, prec), "B"),
        "mr_dslash_dot": ("hbm", dslash_bytes(w, prec), "B"),
        # odd iterations read r, w and write r; even ones also read r_{t-2} and
        # read and write psi (its update deferred by one iteration): per launch
        # the mean over the N - 1 updates
        "mr_update": ("hbm", upd_streams * spinor, "B"),
        "mr_last_update": ("hbm", (4 if w["N"] % 2 == 0 and w["N"] >= 2 else 3) * spinor, "B"),
        "mr_scale": ("hbm", spinor + abi, "B"),
        "trunc_gram": ("hbm", abi, "B"),               # read every block once
        "trunc_gram_tc": ("hbm", abi, "B"),            # the same on BF16 tensor cores
        "trunc_q1_tc": ("hbm", 2 * abi, "B"),          # read A, write Q1 = A R1^-1
        "trunc_gram2_tc": ("hbm", abi, "B"),           # read Q1
        "trunc_uk_tc": ("hbm", abi + uk, "B"),         # read Q1, write U_k
        "coarsen_tc": ("hbm", uk + V * 288 + xy, "B"),  # read P and U once, write X, Y
        "trunc_gram_q1": ("fp32", nbc * (8 * K * m * m + 4 * K * m * m), "flop"),
        "trunc_form_uk": ("fp32", nbc * (4 * K * m * m + 8 * K * m * k), "flop"),
        # one CTA per m' x m' problem, a serial chain of factorisation steps
        # (double-float on the FP32 pipe): latency-bound, reported with its
        # achieved rate and no peak
        "trunc_chol64": ("latency", nbc * (8 * m ** 3 / 3 + 8 * m ** 3 / 3), "flop"),
        "trunc_chol_eig64": ("latency", nbc * (8 * m ** 3 / 3 + 8 * m ** 3 / 3 + 8 * m ** 3 / 3
                                               + 16 * m ** 3 / 3 + 8 * m * m * k), "flop"),
        "prolongator": ("hbm", 2 * V * 12 * k * 8, "B"),
        "coarsen": ("fp32", V * (4 * 8 * 6 * (2 * k) ** 2 + 8 * 12 * (2 * k) ** 2), "flop"),
        "coarse_apply": ("hbm", xy, "B"),
    }


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(w):
    """Runs the FP64 oracle's whole setup level on the sample sub-lattice (same
    m', k, N, aggregate shape); returns (seconds, scale to the full lattice,
    threads, description).  Every stage's cost grows linearly with the volume
    (MR: sites x m'; truncation: aggregates; coarsening: sites)."""
    import mg_inputs as G
    import oracle as O
    d = w["sample_dims"]
    U = G.gauge_field(d, w["eps"], w["gauge_seed"])
    C = O.clover(d, U, w["csw"]) if w["csw"] else None
    p0 = G.psi0(d, w["m"], w["psi_seed"])
    t0 = time.perf_counter()
    psi = O.mr(d, w["m0"], w["xi"], U, C, p0, w["N"])
    Uk, sig = O.chiral_truncate(d, w["block"], psi, w["k"])
    P = O.prolongator(d, w["block"], Uk)
    X, Y = O.coarsen(d, w["block"], w["m0"], w["xi"], U, C, P)
    v = G.coarse_vectors(X.shape[0], 2 * w["k"], 8, 1)
    O.coarse_apply(O.coarse_dims(d, w["block"]), X, Y, v)
    dt = time.perf_counter() - t0
    scale = vol(w["dims"]) / vol(d)
    threads = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    desc = (f"oracle setup level on a {'x'.join(map(str, d))} sub-lattice "
            f"(1/{int(scale)} of the volume; same m', k, N, aggregates), time x {int(scale)}")
    return dt, scale, threads, desc


class Replicas:
    """N independent replicas of the setup, one process per GPU (the path is
    not sharded: no data-path collective).  Only the timing needs the group:
    a barrier on both sides of the timed region and the maximum over ranks.
    Reads RANK / WORLD_SIZE / LOCAL_RANK; backend "nccl" on GPUs, "gloo" for
    the CPU tests of this logic."""

    def __init__(self, backend: str = "nccl", device: str = "cuda"):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.cuda = device == "cuda"
        self.device = torch.device("cuda", self.local) if self.cuda else torch.device("cpu")
        if self.cuda:
            torch.cuda.set_device(self.local)
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=self.device)
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def _sync(self):
        if self.cuda:
            import torch
            torch.cuda.synchronize()

    def barrier(self):
        self._sync()
        if self.dist:
            self.dist.barrier()
        self._sync()

    def max(self, x: float) -> float:
        if not self.dist:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def step_stats(per_step_ms) -> dict:
    """Median, p90 (nearest rank), min and max of the per-step times."""
    v = sorted(per_step_ms)
    n = len(v)
    med = v[(n - 1) // 2] if n % 2 else 0.5 * (v[n // 2 - 1] + v[n // 2])
    return {"median": med, "p90": v[max(0, -(-9 * n // 10) - 1)], "min": v[0], "max": v[-1]}


def per_level(ms_max: float, world: int) -> float:
    """Whole-job seconds per level: `world` replicas each built one level in
    (at most) ms_max milliseconds."""
    return ms_max / 1e3 / world


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.build()
    for _ in range(args.warmup):
        oracle_sample(w)
    times = []
    for _ in range(args.steps):
        dt, scale, threads, desc = oracle_sample(w)
        times.append(dt * scale)
    v = sum(times) / len(times)
    cfg = config_of(w, args, "fp32" if getattr(args, "precision", "all") == "fp32" else "mixed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        # every step is one run of the oracle on the sample sub-lattice:
        # ms_per_step is that run's own time; value scales it to the workload
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v / scale * 1e3,
        "sample_scale_to_workload": scale,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


PRECISION_NOTE = {
    "fp32": "FP32 plain: complex64 storage and FP32 arithmetic on the CUDA cores; Cholesky "
            "and small eigenproblem in double-float (pairs of FP32)",
    "mixed": "mixed: smoother as FP32 plain; truncation Grams, Q1 = A R1^-1, U_k and the "
             "Galerkin contractions on tcgen05 tensor cores with FP32 accumulation (first Gram "
             "BF16, the rest FP16 hi/lo split, 3 products); Cholesky and small eigenproblem in double-float",
    "mixed_fp16": "mixed with FP16 storage of the smoother fields (FP32 arithmetic); truncation "
                  "and coarsening as mixed",
}
DTYPE = {"fp32": "f32; double-float (2xf32) eig",
         "mixed": "f32 smoother; fp16x3+bf16 tensor-core contractions (f32 accum); double-float (2xf32) eig",
         "mixed_fp16": "f16-stored smoother (f32 math); fp16x3+bf16 tensor-core contractions; "
                       "double-float (2xf32) eig"}
PREC_ID = {"fp32": 0, "mixed": 1, "mixed_fp16": 2}


def config_of(w, args, prec="fp32"):
    return {"workload": w["workload"], "dims": w["dims"], "aggregate": w["block"],
            "n_vec": w["m"], "k": w["k"], "mr_iters": w["N"], "xi": w["xi"], "eps": w["eps"],
            "c_sw": w["csw"], "m0": w["m0"], "precision": PRECISION_NOTE[prec],
            "global_batch": args.gpus, "parallelism": f"replicas x{args.gpus}",
            "l2": "inputs larger than L2 (psi0 alone is "
                  f"{vol(w['dims']) * 12 * w['m'] * 8 / 1e9:.1f} GB)"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _peaks():
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh:
            peaks = json.load(fh)
    hbm = peaks.get("hbm_gbs")
    return (hbm or 6800.0), ("measured" if hbm else "fallback")


def _roofline_table(w, prec, kern, steps):
    """Per-stage achieved rates, the top kernel's roofline object and the dslash line."""
    hbm, peak_src = _peaks()
    work = kernel_work(w, prec)

    def roof(name, launches, ms_total):
        bound, amount, unit = work[name]
        per = ms_total / max(launches, 1) * 1e-3
        if bound == "hbm":
            ach = amount / per / 1e9
            return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "peak_source": f"{peak_src} hbm_gbs (copy)",
                    "algorithmic_bytes_per_launch": amount}
        ach = amount / per / 1e12
        if bound == "latency":
            return {"kernel": name, "bound": "latency", "achieved": ach, "peak": None,
                    "unit": "TFLOP/s", "frac": None,
                    "peak_source": "none: a serial chain per small problem, not a throughput bound",
                    "algorithmic_flop_per_launch": amount}
        pk_t = FP32_TFLOPS
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": pk_t, "unit": "TFLOP/s",
                "frac": ach / pk_t, "peak_source": PEAK_SOURCE[bound],
                "algorithmic_flop_per_launch": amount}

    stages = {}
    for n, (l, t) in kern.items():
        st = {"launches": l, "ms_per_step": t / steps, "ms_per_launch": t / max(l, 1)}
        if n in work:
            r = roof(n, l, t)
            st.update({"achieved": r["achieved"], "unit": r["unit"], "frac": r["frac"]})
        stages[n] = st
    top = max((kv for kv in kern.items() if kv[0] in work and work[kv[0]][0] != "latency"),
              key=lambda kv: kv[1][1])[0]
    roofline = roof(top, *kern[top])
    traffic = None
    prof = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if os.path.exists(prof):
        with open(prof) as fh:
            pj = json.load(fh)
        ent = pj.get(prec, {}).get(top, {})
        if (ent.get("source_sha1") == _kernel_sha1(top) and ent.get("workload") == w["workload"]
                and ent.get("precision") == prec):
            traffic = ent.get("dram_bytes_per_launch")
    roofline["traffic"] = traffic
    dl, dt = kern["mr_dslash_dot"]
    d = roof("mr_dslash_dot", dl, dt)
    # the same pass against the CUDA-core FP32 peak: 1320 flop per site and
    # right-hand side for the eight hops, plus 48 (Wilson diagonal) or 504 (clover)
    flop = vol(w["dims"]) * w["m"] * (1320 + (504 if w["csw"] else 48))
    tflops = flop / (dt / max(dl, 1) * 1e-3) / 1e12
    dslash = {"kernel": "mr_dslash_dot", "gbs": d["achieved"], "frac": d["frac"],
              "algorithmic_bytes_per_launch": d["algorithmic_bytes_per_launch"],
              "tflops": tflops, "fp32_alu_frac": tflops / FP32_TFLOPS,
              "algorithmic_flop_per_launch": flop}
    return stages, top, roofline, dslash


# the second level, built on the first level's own coarse operator D_c: the
# paper keeps k = 32 at l = 1 (Sec. 4); m = 64 vectors, 2^4 aggregates of the
# coarse lattice, the fine level's 20 MR iterations
LEVEL2 = dict(block=[2, 2, 2, 2], m=64, k=32, N=20, psi_seed=22)


def level2_work(cp):
    """{kernel: (bound, amount, unit)} of the second level (per launch)."""
    V, n, m, k = cp.volume, 2 * cp.nc, cp.n_vec, cp.k
    nb = cp.block_volume
    nbc = 2 * cp.n_blocks
    K = cp.nc * nb
    return {
        # out = D_c v: 9 n x n by n x m complex products per site
        "c_mr_apply": ("fp32", V * 9 * n * n * m * 8, "flop"),
        "c_mr_update": ("hbm", V * n * m * 8 * 5, "B"),
        "c_mr_scale": ("hbm", V * n * m * 8 * 2, "B"),
        "trunc_gram_q1": ("fp32", nbc * (8 * K * m * m + 4 * K * m * m), "flop"),
        "trunc_form_uk": ("fp32", nbc * (4 * K * m * m + 8 * K * m * k), "flop"),
        # per term: T = M P(y) (n x 2k, depth nc) and P(x)^dag T (2k x 2k, depth nc)
        "c_galerkin": ("fp32", V * 9 * (n * 2 * k * cp.nc + 4 * k * k * cp.nc) * 8, "flop"),
    }


def level2_measure(args, prob, lv, stream):
    """Time the second level (smoother, sigma_3 truncation, prolongator,
    Galerkin product) on the level's own D_c, resident in HBM."""
    import torch

    from paper_2502_03091_gb300 import mg

    cp = mg.CoarseProblem.below(prob, LEVEL2["block"], LEVEL2["m"], LEVEL2["k"], LEVEL2["N"])
    gen = torch.Generator(device="cuda").manual_seed(LEVEL2["psi_seed"])
    shape = mg.shape_cvec(cp, cp.n_vec)
    q0 = torch.complex(torch.randn(shape, device="cuda", generator=gen),
                       torch.randn(shape, device="cuda", generator=gen))
    lv2 = mg.CoarseLevel.allocate(cp, lv.X, lv.Y, q0)
    for _ in range(max(1, args.warmup)):
        lv2.run(stream)
    mg.mg_sync_status(stream)
    steps = max(1, args.steps)
    mg.mg_timing_enable(True)
    mg.mg_timing_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        lv2.run(stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kern = mg.mg_timing_read()
    mg.mg_timing_enable(False)
    mg.mg_sync_status(stream)
    work = level2_work(cp)
    hbm_peak, _ = _peaks()
    stages, top = {}, None
    for name, (launches, tot) in kern.items():
        per = tot / launches
        e = {"launches_per_step": launches / steps, "ms_per_step": tot / steps}
        if name in work:
            bound, amount, unit = work[name]
            if unit == "flop":
                ach = amount / (per * 1e-3) / 1e12
                e["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP32_TFLOPS,
                                 "unit": "TFLOP/s", "frac": ach / FP32_TFLOPS}
            else:
                ach = amount / (per * 1e-3) / 1e9
                e["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak,
                                 "unit": "GB/s", "frac": ach / hbm_peak}
        stages[name] = e
        if top is None or tot > kern[top][1]:
            top = name
    sig0 = lv2.sigma[0].cpu().tolist()
    out = {"value": ms / 1e3, "unit": "s/level", "ms_per_step": ms, "steps": steps,
           "workload": (f"second level on the first level's D_c: {'x'.join(map(str, cp.dims))} "
                        f"coarse lattice, {2 * cp.nc} components, m={cp.n_vec}, k={cp.k}, "
                        f"{'x'.join(map(str, cp.block))} aggregates, {cp.mr_iters} MR iterations"),
           "dtype": "f32", "top_kernel": top, "stages": stages,
           "gpu_launches": sum(l for l, _ in kern.values()) / steps,
           "blk_flags_nonzero": int((lv2.flags.cpu().numpy() != 0).sum()),
           "sigma_decay_block0": {f"alpha{a}": sig0[a][-1] / sig0[a][0] for a in range(2)}}
    if not args.no_solve:
        out_solve = solve_measure(args, prob, lv, cp, lv2, stream)
    else:
        out_solve = None
    del lv2, q0
    return out, out_solve


# the solve the hierarchy serves: FGMRES on D preconditioned by the K-cycle
SOLVE = dict(nrhs=4, tol=1e-5, restart=16, max_iters=200, b_seed=23, conventional_m=24)


def _solve_rhs(prob):
    import torch
    shape = (prob.volume, 4, 3, SOLVE["nrhs"])
    gen = torch.Generator(device="cuda").manual_seed(SOLVE["b_seed"])
    b = torch.complex(torch.randn(shape, device="cuda", generator=gen),
                      torch.randn(shape, device="cuda", generator=gen))
    return b, torch.empty_like(b)


def _solve_run(prob, lv, levels, P, X, Y, b, x, tag, stream, cp=None, lv2=None, timed=False):
    """One mg_solve call on the level's fine operator (FP32), wall-clock timed."""
    import time

    import torch

    from paper_2502_03091_gb300 import mg

    fp = mg.Problem(dims=prob.dims, block=prob.block, m0=prob.m0, n_vec=prob.n_vec, k=prob.k,
                    mr_iters=prob.mr_iters, csw=prob.csw, xi=prob.xi)
    kw = dict(P=P, X=X, Y=Y)
    if levels == 3:
        kw.update(second=cp, P2=lv2.P, X2=lv2.X2, Y2=lv2.Y2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, rel = mg.mg_solve(fp, lv.U, lv.C, b, x, SOLVE["tol"], SOLVE["restart"],
                             SOLVE["max_iters"], kcycle=mg.KCycle(), stream=stream, **kw)
    dt = time.perf_counter() - t0
    out = {"setup": tag, "levels": levels, "outer_steps": steps, "s": dt,
           "relres_max": float(rel.max())}
    if timed:
        # the same solve again with per-kernel CUDA-event timing (identical
        # arithmetic; the events add a little host work per launch)
        mg.mg_timing_enable(True)
        mg.mg_timing_read()
        mg.mg_solve(fp, lv.U, lv.C, b, x, SOLVE["tol"], SOLVE["restart"], SOLVE["max_iters"],
                    kcycle=mg.KCycle(), stream=stream, **kw)
        kern = mg.mg_timing_read()
        mg.mg_timing_enable(False)
        out["kernel_ms"] = {n: round(t, 2) for n, (_, t) in
                            sorted(kern.items(), key=lambda kv: -kv[1][1])}
        out["launches"] = sum(n for n, _ in kern.values())
    return out


def solve_measure(args, prob, lv, cp, lv2, stream):
    """Solve D x = b (4 seeded Gaussian right-hand sides, relative tolerance
    1e-5, FGMRES(16)) with the three- and two-level K-cycle over the level's
    own hierarchy, and with the two-level hierarchy of the conventional setup
    (k = m' = 24 test vectors, no truncation) for the paper's comparison of
    iteration counts.  Wall-clock seconds of the whole call (it synchronises
    at every Krylov step)."""
    from paper_2502_03091_gb300 import mg

    kc = mg.KCycle()
    b, x = _solve_rhs(prob)

    def run(levels, P, X, Y, tag, timed=False):
        return _solve_run(prob, lv, levels, P, X, Y, b, x, tag, stream, cp, lv2, timed)

    out = {"nrhs": SOLVE["nrhs"], "tol": SOLVE["tol"], "restart": SOLVE["restart"],
           "kcycle": {"nu_pre": kc.nu_pre, "nu_post": kc.nu_post,
                      "kcycle_iters": kc.kcycle_iters, "coarsest_iters": kc.coarsest_iters},
           "dtype": "f32", "runs": []}
    run(3, lv.P, lv.X, lv.Y, "warm-up")
    out["runs"].append(run(3, lv.P, lv.X, lv.Y, f"chiral rank-k (m'={prob.n_vec}, k={prob.k})"
                           f" + level 2 (m={cp.n_vec}, k={cp.k})"))
    out["runs"].append(run(2, lv.P, lv.X, lv.Y, f"chiral rank-k (m'={prob.n_vec}, k={prob.k})",
                           timed=True))
    # conventional setup: k = m' test vectors, the same smoother, no truncation
    mc = SOLVE["conventional_m"]
    pc = mg.Problem(dims=prob.dims, block=prob.block, m0=prob.m0, n_vec=mc, k=mc,
                    mr_iters=prob.mr_iters, csw=prob.csw, xi=prob.xi,
                    precision=prob.precision)
    lvc = mg.Level.allocate(pc, lv.U, lv.C, lv.psi0[..., :mc].contiguous())
    lvc.run(stream)
    mg.mg_sync_status(stream)
    out["runs"].append(run(2, lvc.P, lvc.X, lvc.Y, f"conventional (k = m' = {mc})"))
    del lvc, b, x
    return out


def _measure(args, w, prec, rep, U_host, psi0, level2=False):
    """One precision: warm-up, the device-resident timed steps (CUDA events on
    the launching stream, per-kernel event timing, clocks sampled meanwhile),
    then the end-to-end steps through the public API with host buffers."""
    import torch

    from paper_2502_03091_gb300 import mg

    prob = mg.Problem(dims=w["dims"], block=w["block"], m0=w["m0"], n_vec=w["m"], k=w["k"],
                      mr_iters=w["N"], csw=w["csw"], xi=w["xi"],
                      precision=PREC_ID[prec])
    U = U_host.cuda()
    C = None
    if w["csw"]:
        C = torch.empty(mg.shape_C(prob), dtype=torch.complex64, device="cuda")
        mg.mg_clover_field(prob, U, C)
    lv = mg.Level.allocate(prob, U, C, psi0)
    v_in = torch.ones((prob.n_blocks, 2 * prob.k, 8), dtype=torch.complex64, device="cuda")
    v_out = torch.empty_like(v_in)
    stream = torch.cuda.current_stream()

    def step():
        lv.run(stream)
        mg.mg_coarse_apply(prob, lv.X, lv.Y, v_in, v_out, stream)

    for _ in range(args.warmup):
        step()
    rep.barrier()
    mg.mg_sync_status(stream)
    flags = lv.flags.cpu().numpy()

    # ---- device-resident timed region ----
    sampler = ClockSampler(rep.local)
    sampler.start()
    mg.mg_timing_enable(True)
    mg.mg_timing_read()
    rep.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0.record(stream)
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    e1.record(stream)
    rep.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    step_ms = step_stats([ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)])
    kern = mg.mg_timing_read()
    mg.mg_timing_enable(False)
    clocks = sampler.stop()
    ms = rep.max(ms)

    # ---- end to end through the public API with host buffers ----
    # Every step copies its inputs (links, starts) up from pinned host memory
    # and its results (X, Y, sigma) back.  The copies run on a second stream
    # into a second set of buffers, so the upload of step i+1 and the download
    # of step i overlap the compute of the steps around them; all of them are
    # inside the timed region.
    psi0_host = torch.empty(psi0.shape, dtype=psi0.dtype, pin_memory=True)
    psi0_host.copy_(psi0)
    X_host = torch.empty(lv.X.shape, dtype=lv.X.dtype, pin_memory=True)
    Y_host = torch.empty(lv.Y.shape, dtype=lv.Y.dtype, pin_memory=True)
    s_host = torch.empty(lv.sigma.shape, dtype=lv.sigma.dtype, pin_memory=True)
    h2d = U_host.numel() * 8 + psi0_host.numel() * 8
    d2h = X_host.numel() * 8 + Y_host.numel() * 8 + s_host.numel() * 8
    e2e_steps = max(1, min(args.steps, 5))
    cs = torch.cuda.Stream()
    ins = [(lv.U, lv.psi0), (torch.empty_like(lv.U), torch.empty_like(lv.psi0))]
    outs = [(lv.X, lv.Y, lv.sigma),
            (torch.empty_like(lv.X), torch.empty_like(lv.Y), torch.empty_like(lv.sigma))]
    ev_in = [torch.cuda.Event() for _ in range(2)]    # the slot's inputs have landed
    ev_done = [torch.cuda.Event() for _ in range(2)]  # the step using the slot is done
    ev_out = [torch.cuda.Event() for _ in range(2)]   # the slot's results are on the host

    def upload(i):
        sl = i % 2
        with torch.cuda.stream(cs):
            if i >= 2:
                cs.wait_event(ev_done[sl])
            ins[sl][0].copy_(U_host, non_blocking=True)
            ins[sl][1].copy_(psi0_host, non_blocking=True)
            ev_in[sl].record(cs)

    def compute(i):
        sl = i % 2
        stream.wait_event(ev_in[sl])
        if i >= 2:
            stream.wait_event(ev_out[sl])
        lv.U, lv.psi0 = ins[sl]
        lv.X, lv.Y, lv.sigma = outs[sl]
        step()
        ev_done[sl].record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_done[sl])
            X_host.copy_(lv.X, non_blocking=True)
            Y_host.copy_(lv.Y, non_blocking=True)
            s_host.copy_(lv.sigma, non_blocking=True)
            ev_out[sl].record(cs)

    rep.barrier()
    e0.record(stream)
    cs.wait_event(e0)
    upload(0)
    for i in range(e2e_steps):
        if i + 1 < e2e_steps:
            upload(i + 1)
        compute(i)
    stream.wait_event(ev_out[(e2e_steps - 1) % 2])
    e1.record(stream)
    rep.barrier()
    mg.mg_sync_status(stream)
    e2e_ms = rep.max(e0.elapsed_time(e1) / e2e_steps)
    # singular-value decay of block 0 (the paper's diagnostic of how much of
    # the m' vectors' span the rank-k truncation keeps)
    sig0 = lv.sigma[0].cpu().tolist()
    decay = {f"alpha{a}": {"sigma_1": sig0[a][0], "sigma_k": sig0[a][-1],
                           "sigma_k_over_sigma_1": sig0[a][-1] / sig0[a][0]} for a in range(2)}
    res = dict(ms=ms, kern=kern, clocks=clocks, flags=int((flags != 0).sum()), e2e_ms=e2e_ms,
               e2e_steps=e2e_steps, h2d=h2d, d2h=d2h, sigma_decay=decay, step_ms=step_ms)
    if level2:
        res["level2"], res["solve"] = level2_measure(args, prob, lv, stream)
    elif not args.no_solve and not args.no_level2:
        # the same two-level solve on this precision's hierarchy: the quality of
        # the coarse space measured by what it is for
        b, x = _solve_rhs(prob)
        res["solve_2level"] = _solve_run(prob, lv, 2, lv.P, lv.X, lv.Y, b, x,
                                         f"chiral rank-k (m'={prob.n_vec}, k={prob.k}), "
                                         f"{prec} setup", stream)
        del b, x
    del lv, psi0_host, X_host, Y_host, s_host, U, C
    torch.cuda.empty_cache()
    return res


def accuracy_check(w):
    """Lowest-16 eigenvalues of sigma_3 D_c of both GPU paths against the FP64
    oracle on the validation lattice (the workload's parameters on 8^3x16 for
    the 32^3x64 workload: a volume the oracle finishes in seconds).  Returns
    per path the largest relative error of the 16 values and their mean |lambda|
    (the quality of the coarse space: smaller is better), and the oracle's."""
    import numpy as np
    import torch

    import mg_inputs as G
    import oracle as O
    from paper_2502_03091_gb300 import mg

    O.build()
    d, b, k, m = w["sample_dims"], w["block"], w["k"], w["m"]
    U = G.round_to_c64(G.gauge_field(d, w["eps"], w["gauge_seed"]))
    C = G.round_to_c64(O.clover(d, U, w["csw"])) if w["csw"] else None
    p0 = G.round_to_c64(G.psi0(d, m, w["psi_seed"]))
    cd = O.coarse_dims(d, b)
    nc = int(np.prod(cd))
    s3 = np.tile(np.r_[np.ones(k), -np.ones(k)], nc)

    def lowest16(X, Y):
        n = nc * 2 * k
        Dc = O.coarse_apply(cd, X, Y, np.eye(n).reshape(nc, 2 * k, n)).reshape(n, n)
        H = s3[:, None] * Dc
        ev = np.linalg.eigvalsh((H + H.conj().T) / 2)
        return np.sort(np.abs(ev))[:16]

    psi = O.mr(d, w["m0"], w["xi"], U, C, p0, w["N"])
    Uk, _ = O.chiral_truncate(d, b, psi, k)
    P = O.prolongator(d, b, Uk)
    lo = lowest16(*O.coarsen(d, b, w["m0"], w["xi"], U, C, P))
    out = {"lattice": "x".join(map(str, d)), "oracle_mean_abs_lowest16": float(lo.mean())}
    for prec in ("fp32", "mixed", "mixed_fp16"):
        prob = mg.Problem(dims=d, block=b, m0=w["m0"], n_vec=m, k=k, mr_iters=w["N"],
                          csw=w["csw"], xi=w["xi"],
                          precision=PREC_ID[prec])
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()
        Cd = dev(C.reshape(-1, 2, 6, 6)) if C is not None else None
        lv = mg.Level.allocate(prob, dev(U), Cd, dev(p0))
        lv.run()
        mg.mg_sync_status()
        lg = lowest16(lv.X.cpu().numpy().astype(np.complex128),
                      lv.Y.cpu().numpy().astype(np.complex128))
        out[prec] = {"lowest16_max_rel_err": float(np.max(np.abs(lg - lo) / lo)),
                     "mean_abs_lowest16": float(lg.mean())}
    return out


def batch_measure(args, prec="mixed"):
    """The 24-hierarchy batch (mg_inputs.batch_workload): one CUDA graph launch
    per batch (levels fanned out over tuned streams) against the same 24
    levels built one after the other with the single calls."""
    import numpy as np
    import torch

    import mg_inputs as G
    from paper_2502_03091_gb300 import mg

    with open(os.path.join(ROOT, "tests", "golden", "m0.json")) as fh:
        wl = json.load(fh)["workloads"]
    m0s = {v["eps"]: v["m0"] for k, v in wl.items() if k.startswith("Wilson eps=")}
    levels, sites = [], 0
    for h in G.batch_workload(30, m0s):
        p = mg.Problem(dims=h["dims"], block=h["block"], m0=h["m0"], n_vec=h["m"], k=h["k"],
                       mr_iters=h["N"], precision=PREC_ID[prec])
        U = torch.from_numpy(G.gauge_field(h["dims"], h["eps"], h["gauge_seed"], threads=16)
                             .astype(np.complex64)).cuda()
        gen = torch.Generator(device="cuda").manual_seed(h["psi_seed"])
        shape = mg.shape_psi(p)
        p0 = torch.complex(torch.randn(shape, device="cuda", generator=gen),
                           torch.randn(shape, device="cuda", generator=gen))
        levels.append(mg.Level.allocate(p, U, None, p0))
        sites += p.volume
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    batch = mg.Batch(levels, n_streams=0, stream=stream)
    create_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_batch = timed(lambda: batch.launch(stream))
    mg.mg_sync_status(stream)

    def solo():
        for lv in levels:
            lv.run(stream)

    ms_solo = timed(solo)
    out = {"config": "24 hierarchies: 8 each of 8^4, 12^3x24, 16^3x32; m' in {32,48,64}, "
                     "k in {16,24}, aggregates 2^4 or 4^4, eps in [0.15,0.35] (batch seed 30), "
                     f"20 MR iterations, {PRECISION_NOTE[prec]}",
           "ms_per_batch": ms_batch, "levels_per_s": 24e3 / ms_batch,
           "sites_per_s": sites * 1e3 / ms_batch, "n_streams": batch.n_streams,
           "ms_one_after_another": ms_solo, "create_s": create_s,
           "tuned_slab_pairs": sorted({(tuple(lv.prob.dims), lv.prob.n_vec,
                                        mg.mg_tuned_pairs(lv.prob)) for lv in levels})}
    batch.close()
    del levels
    torch.cuda.empty_cache()
    return out


SERVING_RATES = ((2.0, 40), (4.0, 60), (8.0, 100), (20.0, 200))  # (arrivals/s, requests)


def serving_measure(args):
    """Serving under the mixed-volume Poisson load: volumes uniform over
    {8^4, 12^3x24, 16^3x32, 24^3x48, 32^3x64}, (m', k) over {(48,24), (64,24),
    (32,16)}, 4^4 aggregates, eps = 0.25, each hierarchy resident for 4
    coarse applies (nrhs 8); mixed-precision path.  Warm-up: one request per
    volume.  Then, per offered rate (Poisson, seed 40), a stream of requests
    timed in real time: the low rates measure the serving loop's own latency,
    20/s (the workload's rate) is above what one GPU completes, so its queue
    grows over the run."""
    from paper_2502_03091_gb300 import serve

    m0 = _m0_table()["Wilson eps=0.25"]
    warm = [serve.Request(rid=10000 + i, arrival=0.0, dims=list(d), m=64, k=24, m0=m0,
                          seed=10000 + i) for i, d in enumerate(serve.VOLUMES)]
    serve.Server(max_slots=4).run(warm, realtime=False)
    out = {"config": "Poisson arrivals (seed 40) at each offered rate; volumes 8^4, 12^3x24, "
                     "16^3x32, 24^3x48, 32^3x64; (m',k) in {(48,24),(64,24),(32,16)}; 4^4 "
                     "aggregates; eps 0.25; mixed precision; 4 coarse applies (nrhs 8) per "
                     "hierarchy; inputs synthesised on the device per request",
           "latency": "setup complete (host poll of the request's completion event) minus "
                      "arrival, including input synthesis and queueing",
           "rates": []}
    for rate, n in SERVING_RATES:
        reqs = serve.request_stream(n, rate, seed=40, m0=m0)
        st = serve.Server(max_slots=4).run(reqs, realtime=True)
        st["offered_per_s"] = rate
        out["rates"].append(st)
    return out


def run_ours(args, w):
    import numpy as np
    import torch

    import mg_inputs as G
    from paper_2502_03091_gb300 import build as B
    from paper_2502_03091_gb300 import mg

    rep = Replicas()
    world, rank = rep.world, rep.rank
    if rank == 0:
        B.build()
    rep.barrier()
    mg.library()

    # inputs: links from the shared seeded generator (host), starts drawn on the
    # device (a seeded complex Gaussian; 12.9 GB is too large to draw on the host)
    U_host = torch.from_numpy(G.gauge_field(w["dims"], w["eps"], w["gauge_seed"], threads=16)
                              .astype(np.complex64)).pin_memory()
    shape = (G.volume(w["dims"]), 4, 3, w["m"])
    gen = torch.Generator(device="cuda").manual_seed(w["psi_seed"])
    psi0 = torch.complex(torch.randn(shape, device="cuda", generator=gen),
                         torch.randn(shape, device="cuda", generator=gen))

    precs = ["mixed", "fp32", "mixed_fp16"] if args.precision == "all" else [args.precision]
    res = {p: _measure(args, w, p, rep, U_host, psi0,
                       level2=(p == precs[0] and not args.no_level2)) for p in precs}
    if rank != 0:
        rep.close()
        return
    head = precs[0]
    r = res[head]
    stages, top, roofline, dslash = _roofline_table(w, head, r["kern"], args.steps)
    launches = sum(l for l, _ in r["kern"].values())

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        dt_s, scale, threads, desc = oracle_sample(w)
        cpu = {"value": dt_s * scale, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": desc}

    out = {
        "metric": METRIC, "value": per_level(r["ms"], world), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[head],
        "data": "synthetic (seeded random SU(3) links, Gaussian starts)",
        "config": config_of(w, args, head),
        "roofline": roofline,
        "dslash": dslash,
        "top_kernel": top,
        "stages": stages,
        "step_ms": r["step_ms"],
        "gpu_launches": launches,
        "blk_flags_nonzero": r["flags"],
        "sigma_decay_block0": r["sigma_decay"],
        "clocks": r["clocks"],
        "e2e": {"value": per_level(r["e2e_ms"], world), "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "steps": r["e2e_steps"],
                "copies": "pinned host buffers; uploads of step i+1 and downloads of step i "
                          "on a second stream into a second buffer set, overlapping compute"},
        "cpu_baseline": cpu,
    }
    for p in precs[1:]:
        q = res[p]
        st, tp, rf, ds = _roofline_table(w, p, q["kern"], args.steps)
        out["fp32_plain" if p == "fp32" else p] = {
            "value": per_level(q["ms"], world), "ms_per_step": q["ms"],
            "e2e": per_level(q["e2e_ms"], world), "step_ms": q["step_ms"],
            "top_kernel": tp, "roofline": rf,
            "dslash": ds, "stages": {n: v["ms_per_step"] for n, v in st.items()},
            "gpu_launches": sum(l for l, _ in q["kern"].values()), "clocks": q["clocks"],
            "blk_flags_nonzero": q["flags"]}
        if q.get("solve_2level"):
            out["fp32_plain" if p == "fp32" else p]["solve_2level"] = q["solve_2level"]
    if "level2" in r:
        out["level2"] = r["level2"]
    if r.get("solve"):
        out["solve"] = r["solve"]
    # the batch and the server size themselves by the free device memory
    del psi0, U_host
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    if world == 1 and not args.no_accuracy and len(precs) == 3:
        out["accuracy"] = accuracy_check(w)
    if world == 1 and not args.no_batch:
        out["batch"] = {p: batch_measure(args, p) for p in ("mixed", "fp32")}
    if world == 1 and not args.no_serving:
        out["serving"] = serving_measure(args)
    print(json.dumps(out), flush=True)
    rep.close()


# source files of each timed stage's kernels (prefix match, first hit wins);
# every stage also depends on the shared header mg_common.cuh
_STAGE_SOURCES = (("mr_", ("mg_dslash.cu", "mg_bulk.cuh")),
                  ("trunc_gram_tc", ("mg_tc.cu",)),
                  ("trunc_", ("mg_truncate.cu",)),
                  ("prolongator", ("mg_coarsen.cu",)),
                  ("coarsen", ("mg_coarsen.cu",)),
                  ("coarse_apply", ("mg_coarsen.cu",)),
                  ("c_", ("mg_level2.cu", "mg_bulk.cuh")))


def _kernel_sha1(stage: str):
    """Hash of the CUDA sources of one stage's kernels: a stored ncu traffic
    figure is only reported while the kernels it was measured on are
    unchanged."""
    import hashlib
    files = next((f for pre, f in _STAGE_SOURCES if stage.startswith(pre)), None)
    if files is None:
        return None
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2502_03091_gb300", "csrc")
    for f in files + ("mg_common.cuh",):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="32^3x64",
                    choices=["32^3x64", "16^3x32", "16^3x32-aniso"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="all", choices=["all", "fp32", "mixed", "mixed_fp16"],
                    help="all: the mixed path (FP32-accurate) is the headline value; the FP32 "
                         "plain path and the FP16-storage path are reported beside it")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the setup-serving measurement (p50/p99 under Poisson load)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 24-hierarchy batched-setup measurement")
    ap.add_argument("--no-level2", action="store_true",
                    help="skip the second level built on the first level's D_c")
    ap.add_argument("--no-solve", action="store_true",
                    help="skip the K-cycle solves on the built hierarchy")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the lowest-16 eigenvalue check against the oracle")
    args = ap.parse_args()
    w = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
