"""Host logic of the continuous-batching service (CPU only).

The scheduler in paper_2505_20375_gb300/serving.py runs against fakes of the library
binding (handles, step-wise Davidson, grouped sigma) and of the CUDA stream calls, so
that its decisions can be checked without a GPU: admission in arrival order, the slot
limit, the memory budget, the split of solves between the grouped split-precision lane
and the per-solve FP64 streams, that every result belongs to its request, and that a
failure in the request builder reaches the caller without leaking handles.
"""
from __future__ import annotations

import contextlib
import threading
import time
import types

import numpy as np
import pytest
import torch

from paper_2505_20375_gb300 import serving

MiB = 1 << 20
WS_BYTES = 16 * MiB  # Davidson workspace of every fake request; the server adds 8 MiB


class World:
    """Shared record of what the fakes saw."""

    def __init__(self, fail_seed=None, never_finish=False):
        self.lock = threading.Lock()
        self.fail_seed = fail_seed
        self.never_finish = never_finish  # solves stay active until the run ends
        self.fail_when_active = 0         # the failing build waits for this many active solves
        self.handles = []          # every FakeFCI built
        self.active = 0
        self.active_bytes = 0
        self.max_active = 0
        self.over_budget_with_others = False
        self.budget = None
        self.admitted_seeds = []   # stepper creation order
        self.grouped_calls = []    # precisions of each grouped sigma call
        self.fp64_launch_streams = []


def install_fakes(monkeypatch, world: World):
    fci = serving.fci

    class FakeStream:
        def __init__(self, device=None, priority=0):
            self.priority = priority

        def query(self):
            return True

        def synchronize(self):
            pass

    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a, **k: (10 << 30, 20 << 30))
    # the integrals carry the request's seed to the fake handle
    monkeypatch.setattr(serving.synth, "real_integrals", lambda n, n_chol, seed: (("h", seed), ("g", seed)))

    class FakeFCI:
        def __init__(self, device):
            self.closed = False
            self.seed = None
            with world.lock:
                world.handles.append(self)

        def setup_integrals(self, h, g):
            self.seed = h[1]
            return self

        def build_strings(self, na, nb):
            if self.seed == world.fail_seed:
                # fail once the earlier requests hold every slot (bounded wait)
                t_end = time.monotonic() + 10.0
                while world.active < world.fail_when_active and time.monotonic() < t_end:
                    time.sleep(0.001)
                raise RuntimeError("string build failed")
            return self

        def build_das(self, spaces, ref_a, ref_b, max_transfer):
            return self

        @property
        def n_det(self):
            return 100 + self.seed

        @property
        def info(self):
            return {"n_det_intermediate": self.n_det, "n_pair": 10}

        def davidson_opts(self, **kw):
            prec = fci.FCI_PREC_OZ_BF16 if kw.get("precision") == "oz_bf16" else fci.FCI_PREC_FP64
            return types.SimpleNamespace(precision=prec, kw=kw)

        def davidson_workspace_bytes(self, opts):
            return WS_BYTES

        def sigma_graph_into(self, x, y, prec, sl, ws, wsb, stream=None):
            assert prec == fci.FCI_PREC_FP64 and stream is not None
            with world.lock:
                world.fp64_launch_streams.append(stream)

        def close(self):
            self.closed = True

    class FakeStepper:
        def __init__(self, f, opts, guess=None, stream=None):
            self.f, self.opts, self.stream = f, opts, stream
            self.steps = 0
            self.n_steps = 2 + f.seed % 5
            self.nbytes = WS_BYTES + 8 * MiB
            with world.lock:
                world.admitted_seeds.append(f.seed)
                world.active += 1
                world.active_bytes += self.nbytes
                world.max_active = max(world.max_active, world.active)
                if world.active > 1 and world.active_bytes > world.budget:
                    world.over_budget_with_others = True

        def request(self):
            return 1, 2, self.opts.precision, 3, 4, 5

        def advance(self):
            self.steps += 1
            return self.steps >= self.n_steps and not world.never_finish

        def finish(self):
            with world.lock:
                world.active -= 1
                world.active_bytes -= self.nbytes
            return types.SimpleNamespace(energy=-1.0 - 1e-3 * self.f.seed, converged=True,
                                         iterations=[None] * self.steps, n_sigma=self.steps)

    def fake_grouped(jobs, stream=None, graph=False):
        with world.lock:
            world.grouped_calls.append([j[3] for j in jobs])

    monkeypatch.setattr(fci, "FCI", FakeFCI)
    monkeypatch.setattr(fci, "DavidsonStepper", FakeStepper)
    monkeypatch.setattr(fci, "sigma_grouped", fake_grouped)
    monkeypatch.setattr(fci, "clear_grouped_graphs", lambda: None)


def _requests(n=24, rate=400.0):
    return serving.make_requests(n, rate, seed=3)


@pytest.mark.parametrize("max_active,budget_slots", [(16, 2), (3, 100), (1, 100)])
def test_scheduler_admits_in_order_within_slots_and_budget(monkeypatch, max_active, budget_slots):
    world = World()
    world.budget = budget_slots * (WS_BYTES + 8 * MiB)
    install_fakes(monkeypatch, world)
    reqs = _requests()
    server = serving.Server(max_active=max_active, memory_budget=world.budget, use_graphs=True)
    results, stats = server.run(reqs)

    assert stats["requests"] == len(reqs) and stats["converged"] == len(reqs)
    # every result is its own request's (the fake energy encodes the integral seed)
    for r, q in zip(results, sorted(reqs, key=lambda q: q.rid)):
        assert r.rid == q.rid and r.energy == pytest.approx(-1.0 - 1e-3 * q.seed)
        assert r.mixed == q.mixed and r.kind == q.kind
        assert q.arrival <= r.admitted + 1e-9 <= r.finished + 2e-9
        assert r.iterations == 2 + q.seed % 5
    # admission in arrival order, never above the slot limit, within the memory budget
    # whenever more than one solve is resident
    assert world.admitted_seeds == [q.seed for q in sorted(reqs, key=lambda q: q.arrival)]
    assert world.max_active <= min(max_active, budget_slots)
    assert not world.over_budget_with_others
    assert world.active == 0 and world.active_bytes == 0
    # lanes: grouped calls carry split-precision products only; FP64 products go to their
    # solves' own streams
    fp64 = sum(1 for q in reqs if not q.mixed or not (q.kind == "fci" and q.n <= 15 or q.kind == "das" and q.n <= 17))
    assert all(p == serving.fci.FCI_PREC_OZ_BF16 for call in world.grouped_calls for p in call)
    assert (len(world.fp64_launch_streams) > 0) == (fp64 > 0)
    # every handle is closed
    assert all(h.closed for h in world.handles) and len(world.handles) == len(reqs)


def test_make_requests_is_a_seeded_poisson_mix():
    a = serving.make_requests(2000, 50.0, seed=11)
    b = serving.make_requests(2000, 50.0, seed=11)
    assert [(q.arrival, q.kind, q.n, q.mixed) for q in a] == [(q.arrival, q.kind, q.n, q.mixed) for q in b]
    gaps = np.diff([0.0] + [q.arrival for q in a])
    assert np.all(gaps > 0)
    # exponential gaps of mean 1/rate: mean and coefficient of variation near 1/rate and 1
    assert abs(gaps.mean() * 50.0 - 1.0) < 0.1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    # a uniform mix of the shapes, half of it mixed precision
    shapes = {(m["kind"], m["n"]) for m in serving.MIX}
    counts = {s: sum(1 for q in a if (q.kind, q.n) == s) for s in shapes}
    assert all(abs(c / len(a) - 1 / len(shapes)) < 0.05 for c in counts.values())
    assert abs(sum(q.mixed for q in a) / len(a) - 0.5) < 0.05
    assert [q.seed for q in a] == [1000 + i for i in range(len(a))]


def test_builder_failure_reaches_the_caller_and_closes_handles(monkeypatch):
    reqs = [serving.Request(**{**q.__dict__, "arrival": 0.0}) for q in _requests(12)]
    world = World(fail_seed=reqs[6].seed, never_finish=True)
    world.fail_when_active = 4
    world.budget = 100 * (WS_BYTES + 8 * MiB)
    install_fakes(monkeypatch, world)
    server = serving.Server(max_active=4, memory_budget=world.budget)
    with pytest.raises(RuntimeError, match="string build failed"):
        server.run(reqs)
    # no handle stays open: the built but not yet admitted ones, and the active solves
    # (finished first, so that their Davidson state is freed before the handle)
    assert world.max_active == 4
    assert all(h.closed for h in world.handles if h.seed != world.fail_seed)
    assert world.active == 0


def test_solve_alone_and_capacity_use_the_same_stepper_path(monkeypatch):
    """solve_alone runs one request through the same scheduler on its own (arrival reset to
    0, the server's settings kept); measure_capacity solves one request of every shape in
    both precisions and reports the mean service time."""
    world = World()
    world.budget = 100 * (WS_BYTES + 8 * MiB)
    install_fakes(monkeypatch, world)
    server = serving.Server(max_active=8, memory_budget=world.budget, split_slices=3, final_slices=6)
    q = _requests(5)[4]
    r = serving.solve_alone(q, server)
    assert r.rid == q.rid and r.arrival == 0.0 and r.energy == pytest.approx(-1.0 - 1e-3 * q.seed)
    mean, times = serving.measure_capacity(server, seed=2000)
    assert len(times) == 2 * len(serving.MIX) and mean == pytest.approx(np.mean(list(times.values())))
    assert world.active == 0 and all(h.closed for h in world.handles)
    assert server.footprint(q) == WS_BYTES + 8 * MiB
