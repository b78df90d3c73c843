"""GPU tests of the grouped sigma, the step-wise Davidson ABI and the serving loop."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_20375_gb300 import fci, serving, synth

from helpers import ENERGY_TOL, SIGMA_RTOL, fci_problem, gpu_fci, rel_inf

pytestmark = pytest.mark.gpu


def test_grouped_sigma_equals_individual_calls(fci_lib):
    """Split-precision jobs of different sizes in one contraction launch give exactly the
    results of separate calls (integer arithmetic, independent of the CTA split); FP64
    and DAS jobs in the same call run one after another."""
    probs = [fci_problem(6, 3, 3, seed=1), fci_problem(9, 4, 3, seed=2), fci_problem(10, 5, 5, seed=3),
             fci_problem(8, 4, 4, seed=4)]
    fs = [gpu_fci(p) for p in probs]
    Cs = [torch.from_numpy(synth.random_vector(len(p["dets"]), seed=7 + i)).cuda() for i, p in enumerate(probs)]
    precs = [("oz_bf16", 6), ("oz_bf16", 6), ("oz_bf16", 3), ("fp64", 0)]
    ref = [f.sigma(C, precision=pr, n_slices=sl).clone() for f, C, (pr, sl) in zip(fs, Cs, precs)]
    outs = [torch.full_like(C, float("nan")) for C in Cs]
    wss = []
    jobs = []
    for f, C, o, (pr, sl) in zip(fs, Cs, outs, precs):
        nb = f.sigma_workspace_bytes(pr, sl)
        buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        wss.append(buf)
        jobs.append((f, C, o, pr, sl, (buf.data_ptr() + 255) & ~255, nb))
    fci.sigma_grouped(jobs)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)
    # and against the oracle
    for i in range(2):
        p, c = probs[i], Cs[i].cpu().numpy()
        assert rel_inf(outs[i].cpu().numpy(), oracle.sigma(p["hso"], p["gso"], p["dets"], c)) <= SIGMA_RTOL


def test_stepwise_davidson_matches_davidson_solve(fci_lib):
    p = fci_problem(8, 4, 4, n_chol=16, seed=1, e_core=0.5)
    f = gpu_fci(p)
    r1 = f.davidson(tol_residual=1e-6, tol_energy=1e-10)
    st = fci.DavidsonStepper(f, f.davidson_opts(tol_residual=1e-6, tol_energy=1e-10))
    while True:
        x, y, prec, sl, ws, wsb = st.request()
        fci.sigma_grouped([(f, x, y, prec, sl, ws, wsb)])
        if st.advance():
            break
    r2 = st.finish()
    assert r1.converged and r2.converged
    assert abs(r1.energy - r2.energy) < 1e-12
    assert len(r1.iterations) == len(r2.iterations)


def test_serving_results_equal_alone_and_in_the_mix(fci_lib):
    """Requests that arrive while others run are admitted and batched; every energy is
    the same alone and in the mix (to 1e-8 Eh; the arithmetic makes them identical) and
    matches dense diagonalisation for the small ones."""
    reqs = serving.make_requests(10, rate=400.0, seed=7, kinds=("fci",))
    reqs = [r for r in reqs if r.n <= 10]
    srv = serving.Server(max_active=8)
    res, stats = srv.run(reqs)
    assert stats["requests"] == len(reqs) and stats["converged"] == len(reqs)
    assert stats["steps"] < sum(r.iterations for r in res)  # work was batched across solves
    for req, r in zip(reqs, res):
        alone = serving.solve_alone(req, srv)
        assert abs(alone.energy - r.energy) <= ENERGY_TOL
        if req.n <= 8:
            # the lowest eigenvalue of the oracle's dense H
            h, g = synth.real_integrals(req.n, 2 * req.n, req.seed)
            hso, gso = oracle.spin_orbital_integrals(h, g)
            dets = oracle.fci_dets(req.n, req.na, req.nb)
            H = oracle.dense_h(hso, gso, dets).real
            assert abs(np.linalg.eigvalsh(H)[0] - r.energy) < ENERGY_TOL


def test_serving_admission_respects_memory_budget(fci_lib):
    reqs = serving.make_requests(4, rate=1000.0, seed=3, kinds=("fci",))
    srv = serving.Server(max_active=8, memory_budget=1)  # one request at a time
    res, stats = srv.run(reqs)
    assert stats["converged"] == len(reqs)
    spans = sorted((r.admitted, r.finished) for r in res)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-3  # never two solves resident together


@pytest.mark.parametrize("prec,sl", [("fp64", 0), ("oz_bf16", 6)])
def test_sigma_graph_replay_matches_direct_call(fci_lib, prec, sl):
    """The captured sigma graph replays the same kernels: new contents of C (same
    pointer) give the same results as direct calls."""
    p = fci_problem(9, 4, 4, seed=8)
    f = gpu_fci(p)
    st = torch.cuda.Stream()
    N = len(p["dets"])
    C = torch.empty(N, dtype=torch.float64, device="cuda")
    out = torch.empty_like(C)
    with torch.cuda.stream(st):
        for seed in (1, 2, 3):
            C.copy_(torch.from_numpy(synth.random_vector(N, seed=seed)))
            f.sigma_graph(C, out, precision=prec, n_slices=sl, stream=st)
            got = out.clone()
            ref = f.sigma(C, precision=prec, n_slices=sl, stream=st)
            st.synchronize()
            assert torch.equal(got, ref)
    f.clear_graphs()


def test_grouped_graph_replays_with_new_vector_contents(fci_lib):
    """fci_sigma_grouped_graph: the second call with the same job list replays the captured
    graph; new contents of C give the same results as the plain grouped call, and closing
    a handle drops the graphs that name it."""
    probs = [fci_problem(8, 4, 4, seed=21), fci_problem(9, 4, 3, seed=22)]
    fs = [gpu_fci(p) for p in probs]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        Cs = [torch.empty(len(p["dets"]), dtype=torch.float64, device="cuda") for p in probs]
        outs = [torch.empty_like(C) for C in Cs]
        keep, jobs = [], []
        for f, C, o, (pr, sl) in zip(fs, Cs, outs, [("oz_bf16", 6), ("fp64", 0)]):
            nb = f.sigma_workspace_bytes(pr, sl)
            buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
            keep.append(buf)
            jobs.append((f, C, o, pr, sl, (buf.data_ptr() + 255) & ~255, nb))
        for seed in (1, 2, 3):
            for i, C in enumerate(Cs):
                C.copy_(torch.from_numpy(synth.random_vector(C.numel(), seed=seed + 10 * i)))
            fci.sigma_grouped(jobs, stream=st, graph=True)
            got = [o.clone() for o in outs]
            fci.sigma_grouped(jobs, stream=st)
            st.synchronize()
            for g, o in zip(got, outs):
                assert torch.equal(g, o)
    fs[1].close()
    fci.clear_grouped_graphs()


def test_staged_stepper_equals_unstaged(fci_lib):
    """Staging the sigma requests through fixed vectors changes no bit of the solve."""
    p = fci_problem(8, 4, 4, n_chol=16, seed=3, e_core=0.2)
    f = gpu_fci(p)
    res = []
    for staged in (False, True):
        st = fci.DavidsonStepper(f, f.davidson_opts(tol_residual=1e-6, tol_energy=1e-10, precision="oz_bf16",
                                                    n_slices=3, switch_residual=1e-4, final_precision="oz_bf16",
                                                    final_slices=6, staged_sigma=staged))
        ptrs = set()
        while True:
            x, y, prec, sl, ws, wsb = st.request()
            ptrs.add((x, y))
            fci.sigma_grouped([(f, x, y, prec, sl, ws, wsb)])
            if st.advance():
                break
        r = st.finish()
        res.append((r.energy, len(r.iterations), len(ptrs)))
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1]
    assert res[1][2] == 1 and res[0][2] > 1


def test_serving_with_graphs_equals_without(fci_lib):
    reqs = serving.make_requests(8, rate=500.0, seed=11)
    a, sa = serving.Server(max_active=6, use_graphs=True).run(reqs)
    b, sb = serving.Server(max_active=6, use_graphs=False).run(reqs)
    assert sa["converged"] == sb["converged"] == len(reqs)
    for ra, rb in zip(a, b):
        assert ra.energy == rb.energy and ra.iterations == rb.iterations
    assert sa["distinct_job_lists"] < sa["steps"]
