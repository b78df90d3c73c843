"""Continuous-batching service for many Davidson solves on one GPU.

Requests (a problem: integrals seed, active space, precision) arrive over time.  A host
thread builds each request's handle (integrals, strings, DAS layout) as soon as it
arrives, off the step loop.  A built request is admitted as soon as a slot is free and
its device memory fits the budget; its C, sigma and subspace vectors then stay resident
until it converges.  Active solves run in two lanes:
  * split-precision solves (the mixed requests) share one stream: each step their sigma
    products go to the library in one grouped call (products with the same slice count
    share one persistent tcgen05 launch), replayed from a captured CUDA graph while the set
    of solves and their precisions do not change (each solve stages its sigma requests
    through two fixed vectors, staged_sigma), and every solve then takes its Davidson
    update;
  * FP64 solves each have a stream of their own: a solve whose sigma has finished takes its
    update and launches its next sigma at once, so a slow FP64 product (the FP64 DAS
    contraction runs on the FP64 pipe) never holds up the other solves; the large FP64
    products run on low-priority streams, the split lane and the small FP64 solves on high-
    priority ones, so the block scheduler hands freed SMs to the short kernels first.
Solves that finish leave and free their memory; waiting requests join at once.  Reported:
time from arrival to converged energy (p50/p99) and aggregate determinants * sigma / s.

This is scheduling around the library's C ABI; every sigma build and every Davidson
update runs in libfci's kernels.
"""
from __future__ import annotations

import collections
import math
import os
import queue
import threading
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
    def __init__(self, req: Request, f: fci.FCI, stepper: fci.DavidsonStepper, admitted: float, nbytes: int,
                 stream=None):
        self.req, self.f, self.stepper, self.admitted, self.nbytes = req, f, stepper, admitted, nbytes
        self.stream = stream      # FP64 lane: the solve's own stream (None: the split lane)
        self.launched = False     # FP64 lane: a sigma product is in flight


class _Builder(threading.Thread):
    """Builds arrived requests' handles (integrals, strings, DAS layout, Davidson options
    and workspace size) on a stream of its own, in arrival order."""

    def __init__(self, server: "Server"):
        super().__init__(daemon=True)
        self.server = server
        self.todo = queue.Queue()
        self.ready = collections.deque()
        self.lock = threading.Lock()
        self.error = None

    def run(self):
        torch.cuda.set_device(self.server.device)
        st = torch.cuda.Stream(self.server.device, priority=0)  # set-up yields to the solves
        with torch.cuda.stream(st):
            while True:
                req = self.todo.get()
                if req is None:
                    return
                try:
                    f = self.server._build(req)
                    opts = self.server._opts(f, req)
                    nbytes = f.davidson_workspace_bytes(opts) + (8 << 20)
                    st.synchronize()
                except Exception as e:  # reported by the step loop
                    self.error = e
                    return
                with self.lock:
                    self.ready.append((req, f, opts, nbytes))


@dataclass
class Server:
    device: int = 0
    max_active: int = 16
    memory_budget: int = 0            # bytes; 0 = 60% of the free device memory at start
    tol_residual: float = 1e-5
    tol_energy: float = 1e-9
    split_slices: int = 3             # first phase of mixed requests
    final_slices: int = 6             # FP64-class correction phase of mixed requests (error < 1e-11 of
                                      # ||sigma||; the two-pass split form on the DAS layout)
    max_iter: int = 300
    use_graphs: bool = True           # replay the grouped sigma from captured CUDA graphs
    fp64_low_priority: int = 20_000_000  # FP64 solves with n_det_intermediate x n_pair above run at low priority
    fp64_das_chunk: int = 262_144     # FP64 DAS sigma in passes of at most this many intermediate determinants
    log: list = field(default_factory=list)

    def _opts(self, f: fci.FCI, req: Request):
        kw = dict(max_iter=self.max_iter, tol_residual=self.tol_residual, tol_energy=self.tol_energy,
                  staged_sigma=self.use_graphs)
        if req.mixed and ((req.kind == "fci" and req.n <= 15) or (req.kind == "das" and req.n <= 17)):
            return f.davidson_opts(**kw, precision="oz_bf16", n_slices=self.split_slices, switch_residual=1e-4,
                                   final_precision="oz_bf16", final_slices=self.final_slices)
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
        # The persistent tensor-core kernels of the split lane need whole SMs; a long FP64
        # contraction on another stream keeps SMs partly busy until it ends, so the FP64 DAS
        # products run in passes of bounded size (FCI_DAS_FP64_CHUNK_DETS, read by the
        # library at each call) and no FP64 kernel holds the SMs for long.
        old = os.environ.get("FCI_DAS_FP64_CHUNK_DETS")
        if self.fp64_das_chunk > 0:
            os.environ["FCI_DAS_FP64_CHUNK_DETS"] = str(self.fp64_das_chunk)
        try:
            return self._run_on_stream(requests, clock)
        finally:
            if self.fp64_das_chunk > 0:
                if old is None:
                    os.environ.pop("FCI_DAS_FP64_CHUNK_DETS", None)
                else:
                    os.environ["FCI_DAS_FP64_CHUNK_DETS"] = old

    def _run_on_stream(self, requests, clock):
        torch.cuda.set_device(self.device)
        # graphs cannot be captured on the legacy stream; the split lane runs at high priority
        stream = torch.cuda.Stream(self.device, priority=-1)
        with torch.cuda.stream(stream):
            return self._run(requests, clock, stream)

    def _run(self, requests, clock, stream):
        budget = self.memory_budget
        if budget <= 0:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget = int(0.6 * free)
        pending = sorted(requests, key=lambda r: r.arrival)
        builder = _Builder(self)
        builder.start()
        lane_streams = {-1: [], 0: []}  # FP64 lanes' streams by priority, reused
        split, fp64, results = [], [], []
        used = 0
        t0 = clock()
        det_sigma = 0
        n_steps = 0
        signatures = set()

        def finish(a):
            nonlocal used
            r = a.stepper.finish()
            results.append(Result(a.req.rid, r.energy, r.converged, len(r.iterations), a.f.n_det, r.n_sigma,
                                  a.req.arrival, a.admitted, clock() - t0, a.req.mixed, a.req.kind))
            used -= a.nbytes
            a.f.close()
            if a.stream is not None:
                lane_streams[a.prio].append(a.stream)

        try:
            while pending or builder.todo.qsize() or builder.ready or split or fp64 or \
                    len(results) < len(requests):
                if builder.error is not None:
                    raise builder.error
                now = clock() - t0
                while pending and pending[0].arrival <= now:
                    builder.todo.put(pending.pop(0))
                # admission: in arrival order while a slot and the memory budget allow
                while len(split) + len(fp64) < self.max_active:
                    with builder.lock:
                        if not builder.ready:
                            break
                        req, f, opts, nbytes = builder.ready[0]
                        if (split or fp64) and used + nbytes > budget:
                            break
                        builder.ready.popleft()
                    lane, prio = None, 0
                    if opts.precision == fci.FCI_PREC_FP64:
                        # a large FP64 product (long FP64-pipe kernels) runs at low priority, so
                        # that the kernels of the small solves take SMs as soon as blocks retire
                        info = f.info
                        prio = 0 if info["n_det_intermediate"] * info["n_pair"] > self.fp64_low_priority else -1
                        pool = lane_streams[prio]
                        lane = pool.pop() if pool else torch.cuda.Stream(self.device, priority=prio)
                    st = fci.DavidsonStepper(f, opts, stream=lane if lane is not None else stream)
                    a = _Active(req, f, st, clock() - t0, nbytes, lane)
                    a.prio = prio
                    (fp64 if lane is not None else split).append(a)
                    used += nbytes
                if not split and not fp64:
                    time.sleep(0.0005 if (builder.todo.qsize() or builder.ready) else
                               max(0.0, min(0.02, pending[0].arrival - (clock() - t0))) if pending else 0.0005)
                    continue
                # split lane: one grouped sigma call for every split solve
                if split:
                    jobs = []
                    for a in split:
                        x, y, prec, sl, ws, wsb = a.stepper.request()
                        jobs.append((a.f, x, y, prec, sl, ws, wsb))
                        det_sigma += a.f.n_det
                    fci.sigma_grouped(jobs, stream=stream, graph=self.use_graphs)
                    signatures.add(tuple((id(j[0]), j[1], j[2], j[3], j[4], j[5]) for j in jobs))
                    n_steps += 1
                # FP64 lane: launch the sigma of every solve without one in flight, advance
                # the solves whose sigma has finished
                still = []
                for a in fp64:
                    if a.launched and a.stream.query():
                        a.launched = False
                        if a.stepper.advance():
                            finish(a)
                            continue
                    if not a.launched:
                        x, y, prec, sl, ws, wsb = a.stepper.request()
                        if self.use_graphs:  # the solve's own sigma graph (fci_sigma_graph)
                            a.f.sigma_graph_into(x, y, prec, sl, ws, wsb, stream=a.stream)
                        else:
                            fci.sigma_grouped([(a.f, x, y, prec, sl, ws, wsb)], stream=a.stream)
                        det_sigma += a.f.n_det
                        a.launched = True
                    still.append(a)
                fp64 = still
                # split lane: every solve takes its update (waits for the grouped sigma)
                still = []
                for a in split:
                    if a.stepper.advance():
                        finish(a)
                    else:
                        still.append(a)
                split = still
                if not split and fp64 and all(a.launched for a in fp64):
                    time.sleep(0.0002)  # only FP64 products in flight: poll gently
        finally:
            builder.todo.put(None)
            builder.join()
            with builder.lock:
                for _, f, _, _ in builder.ready:
                    f.close()
            if split or fp64:
                # leaving on an error with solves still resident: wait for their kernels,
                # then free each Davidson state before its handle
                try:
                    torch.cuda.synchronize(self.device)
                except Exception:
                    pass
                for a in split + fp64:
                    for release in (a.stepper.finish, a.f.close):
                        try:
                            release()
                        except Exception:
                            pass
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
            "distinct_job_lists": len(signatures),  # graph captures of the split lane; the other steps replay
        }
        if self.use_graphs:
            fci.clear_grouped_graphs()
        return sorted(results, key=lambda r: r.rid), stats


def solve_alone(req: Request, server: Server):
    """The same request through the same stepper path, on its own."""
    res, _ = Server(device=server.device, max_active=1, memory_budget=server.memory_budget,
                    tol_residual=server.tol_residual, tol_energy=server.tol_energy,
                    fp64_das_chunk=server.fp64_das_chunk,
                    split_slices=server.split_slices, final_slices=server.final_slices,
                    max_iter=server.max_iter, use_graphs=server.use_graphs).run([Request(**{**req.__dict__, "arrival": 0.0})])
    return res[0]


def measure_capacity(server: Server, seed: int = 2000):
    """Single-stream capacity of the request mix: one request of every shape in MIX, in
    each precision, solved alone one after another; the mean time to energy of the mix
    (uniform over shapes, half mixed precision) is the mean service time, and its inverse
    the capacity in requests per second.  Returns (mean service seconds, per-request times)."""
    times = {}
    for i, m in enumerate(MIX):
        for mixed in (False, True):
            req = Request(rid=i, mixed=mixed, seed=seed + 2 * i + int(mixed), **{k: v for k, v in m.items()})
            t0 = time.perf_counter()
            solve_alone(req, server)
            times[f"{m['kind']}{m['n']}_{'mixed' if mixed else 'fp64'}"] = time.perf_counter() - t0
    return float(np.mean(list(times.values()))), times

