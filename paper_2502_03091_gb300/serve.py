"""Setup serving: a request loop over the C ABI (continuous batching).

Requests for setups of different lattice volumes, m' and k arrive over time.
The server admits them in arrival order as soon as a slot and device memory
are free (admission by an HBM ledger: inputs, outputs and workspaces of the
setup, with resident hierarchies of finished requests evicted oldest first
when room is needed), runs every admitted request on its own CUDA stream so
that the work of different requests overlaps on the device, polls the
requests' completion events, keeps each built hierarchy (P, X, Y_mu) resident
for its follow-up coarse applies, and reports latency (setup complete minus
arrival) percentiles beside throughput.

Inputs are synthesised on the device per request from a per-request seed,
as part of handling the request, with the counter-based SplitMix64 /
Box-Muller numbers of mg_inputs, by the library (mg_random_links: links
exp(i eps H), H = sum_a h_a lambda_a / 2; mg_random_starts: complex Gaussian
starts), so a request's inputs are those the host generator gives for that
seed, to complex64 rounding.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List

from . import mg

VOLUMES = ([8, 8, 8, 8], [12, 12, 12, 24], [16, 16, 16, 32], [24, 24, 24, 48], [32, 32, 32, 64])
MK = ((48, 24), (64, 24), (32, 16))


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    dims: List[int]
    m: int
    k: int
    eps: float = 0.25
    m0: float = -0.15
    block: List[int] = field(default_factory=lambda: [4, 4, 4, 4])
    mr_iters: int = 20
    seed: int = 0
    # filled in by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    gpu_ms: float = math.nan
    deferred: bool = False
    failed: bool = False      # rejected: a bounded device wait timed out (see Server.run)
    too_large: bool = False   # rejected: needs more device memory than the budget


def request_stream(n: int, rate: float, seed: int = 40, m0: float = -0.15,
                   volumes=VOLUMES, mk=MK) -> List[Request]:
    """n requests with Poisson arrivals (mean `rate` per second); volume and
    (m', k) uniform over the given sets.  Uniforms from the shared counter
    generator (stream MISC of `seed`); request r uses seed 400 + r."""
    import mg_inputs as G
    u = G.uniforms(seed, G.STREAM_MISC, 0, 3 * n).reshape(n, 3)
    out, t = [], 0.0
    for r in range(n):
        t += -math.log(u[r, 0]) / rate
        d = volumes[min(len(volumes) - 1, int(u[r, 1] * len(volumes)))]
        m, k = mk[min(len(mk) - 1, int(u[r, 2] * len(mk)))]
        out.append(Request(rid=r, arrival=t, dims=list(d), m=m, k=k, m0=m0, seed=400 + r))
    return out


def synth_inputs(prob: mg.Problem, eps: float, seed: int, device="cuda"):
    """(U, psi0) complex64 on the device for one request (current stream):
    mg_inputs.gauge_field(dims, eps, seed) and mg_inputs.psi0(dims, m', seed),
    drawn by the library (mg_random_links, mg_random_starts: the same
    counter-based numbers, to complex64 rounding)."""
    import dataclasses

    import torch
    p = dataclasses.replace(prob, seed=seed)
    s = torch.cuda.current_stream()
    U = torch.empty(mg.shape_U(prob), dtype=torch.complex64, device=device)
    mg.mg_random_links(p, eps, U, s)
    psi0 = torch.empty(mg.shape_psi(prob), dtype=torch.complex64, device=device)
    mg.mg_random_starts(p, psi0, s)
    return U, psi0


def need_bytes(prob: mg.Problem) -> int:
    """Device bytes a setup holds while it runs: links, starts, smoothed
    vectors, U_k, sigma, flags, P, X, Y and both workspaces."""
    V, m, k, nb = prob.volume, prob.n_vec, prob.k, prob.n_blocks
    fields = 8 * V * 12 * m * 2                   # psi0, psi (complex64)
    links = 8 * V * 36
    uk_p = 2 * 8 * V * 12 * k                     # U_k and P
    xy = 8 * nb * 9 * (2 * k) ** 2
    small = 8 * nb * 2 * k + 4 * nb * 2
    ws = mg.mg_workspace_size(prob, mg.MG_CALL_SMOOTH) + mg.mg_workspace_size(prob, mg.MG_CALL_TRUNCATE)
    return fields + links + uk_p + xy + small + ws


def resident_bytes(prob: mg.Problem) -> int:
    """Device bytes of a built hierarchy kept for coarse applies (P, X, Y)."""
    V, k, nb = prob.volume, prob.k, prob.n_blocks
    return 8 * V * 12 * k + 8 * nb * 9 * (2 * k) ** 2


class Server:
    """Continuous-batching setup server over one GPU (see the module doc)."""

    def __init__(self, max_slots: int = 4, reserve_bytes: int = 16 << 30,
                 precision: int = mg.MG_PREC_MIXED, applies: int = 4, nrhs: int = 8,
                 keep_results: bool = False, device: str = "cuda"):
        import torch
        self.torch = torch
        self.max_slots = max_slots
        self.precision = precision
        self.applies = applies
        self.nrhs = nrhs
        self.keep_results = keep_results
        self.device = device
        # the device's free memory, counting blocks torch keeps cached but unused
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        self.budget = free - reserve_bytes
        self.used = 0
        self.high_water = 0
        self.results: Dict[int, tuple] = {}
        self.late_timeout = False

    def _problem(self, r: Request) -> mg.Problem:
        return mg.Problem(dims=r.dims, block=r.block, m0=r.m0, n_vec=r.m, k=r.k,
                          mr_iters=r.mr_iters, precision=self.precision)

    def run(self, requests: List[Request], realtime: bool = True) -> dict:
        """Serves the requests (arrival times relative to the call; realtime
        False admits every request at time 0).  Returns the statistics."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        active: List[dict] = []
        applying: List[dict] = []
        resident: "collections.OrderedDict[int, dict]" = collections.OrderedDict()
        done: List[Request] = []
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def evict_until(need):
            while self.used + need > self.budget and resident:
                _, h = resident.popitem(last=False)
                self.used -= h["bytes"]
                h.clear()

        while pending or waiting or active or applying:
            progressed = False
            t = now()
            while pending and (not realtime or pending[0].arrival <= t):
                waiting.append(pending.popleft())
                progressed = True
            # admission in arrival order
            while waiting and len(active) < self.max_slots:
                r = waiting[0]
                prob = self._problem(r)
                need = need_bytes(prob)
                evict_until(need)
                if self.used + need > self.budget:
                    if not active and not applying:
                        # too large even for an idle device: rejected, not queued forever
                        waiting.popleft()
                        r.failed = r.too_large = True
                        r.t_admit = r.t_done = now()
                        done.append(r)
                        progressed = True
                        continue
                    break
                waiting.popleft()
                r.t_admit = now()
                r.deferred = r.t_admit - (r.arrival if realtime else 0.0) > 1e-3
                s = torch.cuda.Stream()
                with torch.cuda.stream(s):
                    U, psi0 = synth_inputs(prob, r.eps, r.seed, self.device)
                    e_in = torch.cuda.Event(enable_timing=True)
                    e_done = torch.cuda.Event(enable_timing=True)
                    e_in.record(s)
                    lv = mg.Level.allocate(prob, U, None, psi0)
                    lv.run(s)
                    e_done.record(s)
                self.used += need
                self.high_water = max(self.high_water, self.used)
                active.append(dict(r=r, s=s, lv=lv, e_in=e_in, e_done=e_done, need=need,
                                   prob=prob))
                progressed = True
            # completions
            for a in list(active):
                if not a["e_done"].query():
                    continue
                r, lv, s = a["r"], a["lv"], a["s"]
                r.t_done = now()
                r.gpu_ms = a["e_in"].elapsed_time(a["e_done"])
                # The library's status word is per device: a bounded wait that
                # timed out in any kernel since the last check shows up here.
                # The request being completed and every request on the device
                # with it are rejected (their results may be the invalid ones).
                try:
                    mg.mg_sync_status(s)
                except mg.MgError as e:
                    if e.status != mg.MG_ERR_TIMEOUT:
                        raise
                    for b in active:
                        b["r"].failed = True
                if r.failed:
                    del lv
                    a.clear()
                    self.used -= need_bytes(self._problem(r))
                    active.remove(a)
                    done.append(r)
                    progressed = True
                    continue
                if self.keep_results:
                    self.results[r.rid] = (lv.sigma.cpu(), lv.X.cpu(), lv.Y.cpu(), lv.psi.cpu())
                # keep the hierarchy, drop the rest of the setup's memory
                h = dict(P=lv.P, X=lv.X, Y=lv.Y, prob=a["prob"], bytes=resident_bytes(a["prob"]))
                del lv
                a.clear()
                self.used -= need_bytes(h["prob"]) - h["bytes"]
                with torch.cuda.stream(s):
                    v = torch.ones((h["prob"].n_blocks, 2 * h["prob"].k, self.nrhs),
                                   dtype=torch.complex64, device=self.device)
                    out = torch.empty_like(v)
                    for _ in range(self.applies):
                        mg.mg_coarse_apply(h["prob"], h["X"], h["Y"], v, out, s)
                    e = torch.cuda.Event()
                    e.record(s)
                applying.append(dict(r=r, h=h, e=e, v=v, out=out))
                active.remove(a)
                done.append(r)
                progressed = True
            for a in list(applying):
                if a["e"].query():
                    resident[a["r"].rid] = a["h"]
                    applying.remove(a)
                    progressed = True
            if not progressed:
                time.sleep(2e-4)
        torch.cuda.synchronize()
        try:
            mg.mg_sync_status()
        except mg.MgError as e:
            if e.status != mg.MG_ERR_TIMEOUT:
                raise
            self.late_timeout = True  # a coarse apply timed out after its request completed
        resident.clear()
        torch.cuda.empty_cache()
        return self._stats(done, realtime)

    def _stats(self, done: List[Request], realtime: bool) -> dict:
        import numpy as np
        failed = sum(r.failed and not r.too_large for r in done)
        too_large = sum(r.too_large for r in done)
        done = [r for r in done if not r.failed]
        if not done:
            return {"requests": 0, "failed": failed, "rejected_too_large": too_large}
        lat = np.array([r.t_done - (r.arrival if realtime else 0.0) for r in done])
        span = max(r.t_done for r in done) - (min(r.arrival for r in done) if realtime else 0.0)
        gpu = np.array([r.gpu_ms for r in done])
        return {"requests": len(done), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "setups_per_s": len(done) / span, "deferred": int(sum(r.deferred for r in done)),
                "admitted_at_arrival": int(sum(not r.deferred for r in done)),
                "gpu_ms_p50": float(np.percentile(gpu, 50)),
                "hbm_high_water_gb": self.high_water / 1e9,
                "max_slots": self.max_slots, "failed": failed,
                "rejected_too_large": too_large, "budget_gb": self.budget / 1e9,
                "late_timeout": self.late_timeout}
