"""Continuous-batching service for many Davidson solves on one GPU.

Requests (a problem: integrals seed, active space, precision) arrive over time.  A
request is admitted as soon as a slot is free and its device memory fits the budget;
its C, sigma and subspace vectors then stay resident until it converges.  Each step,
the sigma products that all active solves need go to the library in one grouped call
(split-precision products with the same slice count share one persistent tcgen05
launch), and every solve then takes its Davidson update (davidson_advance).  Each solve
stages its sigma requests through two fixed vectors (staged_sigma), so while the set of
active solves and their precisions do not change the grouped call is the same list
every step and is replayed from a captured CUDA graph (fci_sigma_grouped_graph).  Solves that finish leave the batch and free their memory; waiting
requests join at the next step.  Reported: time from arrival to converged energy
(p50/p99) and aggregate determinants * sigma / s.

This is scheduling around the library's C ABI; every sigma build and every Davidson
update runs in libfci's kernels.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fci, synth


@dataclass
class Request:
    rid: int
    kind: str                 # "fci" or "das"
    n: int
    na: int
    nb: int
    mixed: bool               # split-precision first phase, FP64-class correction
    seed: int
    arrival: float = 0.0      # seconds after the start of the run
    spaces: tuple = ()
    ref: tuple = ()
    max_transfer: int = 0


@dataclass
class Result:
    rid: int
    energy: float
    converged: bool
    iterations: int
    n_det: int
    n_sigma: int
    arrival: float
    admitted: float
    finished: float
    mixed: bool
    kind: str

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


# Problem shapes of the request mix: plain FCI (6e,6o) .. (12e,12o) and a 16-orbital,
# 4-space DAS problem with 1 alpha + 1 beta electron per space and at most 1 transfer.
MIX = [
    dict(kind="fci", n=6, na=3, nb=3),
    dict(kind="fci", n=8, na=4, nb=4),
    dict(kind="fci", n=10, na=5, nb=5),
    dict(kind="fci", n=12, na=6, nb=6),
    dict(kind="das", n=16, na=4, nb=4, spaces=(4, 4, 4, 4), ref=(1, 1, 1, 1), max_transfer=1),
]


def make_requests(n_req: int, rate: float, seed: int = 5, kinds=None):
    """Poisson arrivals (exponential gaps, mean 1/rate) of a uniform mix; half of the
    requests use the mixed precision.  Integral seed of request i: 1000 + i."""
    st = synth.Stream(seed, tag=0x5E5E)
    u = st.uniform(3 * n_req)
    mix = [m for m in MIX if kinds is None or m["kind"] in kinds]
    t = 0.0
    out = []
    for i in range(n_req):
        t += -math.log(1.0 - u[3 * i]) / rate
        m = mix[int(u[3 * i + 1] * len(mix)) % len(mix)]
        out.append(Request(rid=i, mixed=bool(u[3 * i + 2] < 0.5), seed=1000 + i, arrival=t,
                           **{k: v for k, v in m.items()}))
    return out


class _Active:
    def __init__(self, req: Request, f: fci.FCI, stepper: fci.DavidsonStepper, admitted: float, nbytes: int):
        self.req, self.f, self.stepper, self.admitted, self.nbytes = req, f, stepper, admitted, nbytes


@dataclass
class Server:
    device: int = 0
    max_active: int = 16
    memory_budget: int = 0            # bytes; 0 = 60% of the free device memory at start
    tol_residual: float = 1e-5
    tol_energy: float = 1e-9
    split_slices: int = 3             # first phase of mixed requests
    final_slices: int = 6             # FP64-class correction phase of FCI requests (error < 1e-11
                                      # of ||sigma||); DAS requests correct in FP64
    max_iter: int = 300
    use_graphs: bool = True           # replay the grouped sigma from captured CUDA graphs
    log: list = field(default_factory=list)

    def _opts(self, f: fci.FCI, req: Request):
        kw = dict(max_iter=self.max_iter, tol_residual=self.tol_residual, tol_energy=self.tol_energy,
                  staged_sigma=self.use_graphs)
        if req.mixed and req.kind == "fci" and req.n <= 15:
            return f.davidson_opts(**kw, precision="oz_bf16", n_slices=self.split_slices, switch_residual=1e-4,
                                   final_precision="oz_bf16", final_slices=self.final_slices)
        if req.mixed and req.kind == "das" and req.n <= 17:
            # the DAS split path takes at most 3 slices; the correction phase is FP64
            return f.davidson_opts(**kw, precision="oz_bf16", n_slices=min(self.split_slices, 3),
                                   switch_residual=1e-4, final_precision="fp64")
        return f.davidson_opts(**kw)

    def _build(self, req: Request):
        h, g = synth.real_integrals(req.n, 2 * req.n, req.seed)
        f = fci.FCI(self.device).setup_integrals(h, g).build_strings(req.na, req.nb)
        if req.kind == "das":
            f.build_das(list(req.spaces), list(req.ref), list(req.ref), req.max_transfer)
        return f

    def footprint(self, req: Request) -> int:
        """Device bytes a request holds while active (Davidson workspace + tables)."""
        f = self._build(req)
        nb = f.davidson_workspace_bytes(self._opts(f, req))
        f.close()
        return nb + (8 << 20)

    def run(self, requests, clock=time.perf_counter):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)  # graphs cannot be captured on the legacy stream
        with torch.cuda.stream(stream):
            return self._run(requests, clock, stream)

    def _run(self, requests, clock, stream):
        budget = self.memory_budget
        if budget <= 0:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget = int(0.6 * free)
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting, active, results = [], [], []
        used = 0
        t0 = clock()
        det_sigma = 0
        n_steps = 0
        signatures = set()
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            # admission: FIFO while a slot and the memory budget allow
            while waiting and len(active) < self.max_active:
                req = waiting[0]
                f = self._build(req)
                opts = self._opts(f, req)
                nbytes = f.davidson_workspace_bytes(opts) + (8 << 20)
                if active and used + nbytes > budget:
                    f.close()
                    break
                waiting.pop(0)
                st = fci.DavidsonStepper(f, opts, stream=stream)
                active.append(_Active(req, f, st, clock() - t0, nbytes))
                used += nbytes
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.05, pending[0].arrival - (clock() - t0))))
                continue
            # one step: every active solve's sigma request in one grouped call
            jobs = []
            for a in active:
                x, y, prec, sl, ws, wsb = a.stepper.request()
                jobs.append((a.f, x, y, prec, sl, ws, wsb))
                det_sigma += a.f.n_det
            fci.sigma_grouped(jobs, stream=stream, graph=self.use_graphs)
            signatures.add(tuple((id(j[0]), j[1], j[2], j[3], j[4], j[5]) for j in jobs))
            n_steps += 1
            still = []
            for a in active:
                if a.stepper.advance():
                    r = a.stepper.finish()
                    results.append(Result(a.req.rid, r.energy, r.converged, len(r.iterations), a.f.n_det, r.n_sigma,
                                          a.req.arrival, a.admitted, clock() - t0, a.req.mixed, a.req.kind))
                    used -= a.nbytes
                    a.f.close()
                else:
                    still.append(a)
            active = still
        torch.cuda.synchronize()
        wall = clock() - t0
        lat = np.array([r.latency for r in results])
        stats = {
            "requests": len(results),
            "wall_s": wall,
            "steps": n_steps,
            "det_sigma_per_s": det_sigma / wall,
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "converged": int(sum(r.converged for r in results)),
            "distinct_job_lists": len(signatures),  # graph captures; the other steps replay
        }
        if self.use_graphs:
            fci.clear_grouped_graphs()
        return sorted(results, key=lambda r: r.rid), stats


def solve_alone(req: Request, server: Server):
    """The same request through the same stepper path, on its own."""
    res, _ = Server(device=server.device, max_active=1, memory_budget=server.memory_budget,
                    tol_residual=server.tol_residual, tol_energy=server.tol_energy,
                    split_slices=server.split_slices, final_slices=server.final_slices,
                    max_iter=server.max_iter, use_graphs=server.use_graphs).run([Request(**{**req.__dict__, "arrival": 0.0})])
    return res[0]
