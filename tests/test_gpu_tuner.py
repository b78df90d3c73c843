"""GPU tests of the tile-shape tuner and of the tile shapes it chooses between."""
import pytest
import torch

import oracle
from paper_2505_20375_gb300 import fci, synth

from helpers import SIGMA_RTOL, fci_problem, gpu_fci, rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("s", [2, 3, 6, 7])
@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (9, 4, 3), (11, 6, 4)])
def test_fci_tile_widths_agree(fci_lib, monkeypatch, n, na, nb, s):
    """32 and 64 determinants per tile: the same bits (exact integer arithmetic), ragged
    last tiles included."""
    p = fci_problem(n, na, nb, n_chol=n + 1, seed=50 + n, e_core=0.1)
    f = gpu_fci(p)
    c = torch.from_numpy(synth.random_vector(len(p["dets"]), seed=3)).cuda()
    monkeypatch.setenv("FCI_OZ_TILE", "64")
    a = f.sigma(c, precision="oz_bf16", n_slices=s).clone()
    monkeypatch.setenv("FCI_OZ_TILE", "32")
    b = f.sigma(c, precision="oz_bf16", n_slices=s).clone()
    f.sync_status()
    assert torch.equal(a, b)
    if s >= 6:
        assert rel_inf(b.cpu().numpy(), oracle.sigma(p["hso"], p["gso"], p["dets"], c.cpu().numpy(), e_core=0.1)) <= SIGMA_RTOL


@pytest.mark.parametrize("s", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("n,na,nb", [(1, 1, 1), (5, 0, 3), (6, 3, 3), (9, 4, 3), (11, 6, 4), (13, 6, 6)])
def test_fci_two_pass_path_agrees_with_fused(fci_lib, monkeypatch, n, na, nb, s):
    """The two-pass path (D digit image + bulk-copy GEMM) and the fused kernel compute the
    same integers: identical bits, ragged N tiles and padded K chunks included, for every
    accumulator form (double-buffered s <= 4; one buffer released in two or three level
    groups at s = 5..7) and for a single determinant and an empty alpha string set (one
    tile, one K-chunk)."""
    p = fci_problem(n, na, nb, n_chol=n + 1, seed=90 + n, e_core=-0.2)
    f = gpu_fci(p)
    c = torch.from_numpy(synth.random_vector(len(p["dets"]), seed=6)).cuda()
    monkeypatch.setenv("FCI_OZ_PATH", "fused")
    a = f.sigma(c, precision="oz_bf16", n_slices=s).clone()
    monkeypatch.setenv("FCI_OZ_PATH", "gemm")
    b = f.sigma(c, precision="oz_bf16", n_slices=s).clone()
    f.sync_status()
    assert torch.equal(a, b)


@pytest.mark.parametrize("path", ["fused", "gemm"])
def test_grouped_launch_with_32_wide_tiles_or_two_pass(fci_lib, monkeypatch, path):
    monkeypatch.setenv("FCI_OZ_TILE", "32")
    monkeypatch.setenv("FCI_OZ_PATH", path)
    probs = [fci_problem(7, 3, 3, seed=61), fci_problem(10, 5, 5, seed=62)]
    fs = [gpu_fci(p) for p in probs]
    Cs = [torch.from_numpy(synth.random_vector(len(p["dets"]), seed=8 + i)).cuda() for i, p in enumerate(probs)]
    ref = [f.sigma(C, precision="oz_bf16", n_slices=6).clone() for f, C in zip(fs, Cs)]
    outs = [torch.full_like(C, float("nan")) for C in Cs]
    keep, jobs = [], []
    for f, C, o in zip(fs, Cs, outs):
        nb = f.sigma_workspace_bytes("oz_bf16", 6)
        buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        keep.append(buf)
        jobs.append((f, C, o, "oz_bf16", 6, (buf.data_ptr() + 255) & ~255, nb))
    fci.sigma_grouped(jobs)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)


@pytest.mark.parametrize("kind", ["fci", "das"])
def test_tuner_keeps_the_fastest_and_results_do_not_change(fci_lib, kind):
    if kind == "fci":
        p = fci_problem(10, 5, 5, n_chol=11, seed=70)
        f = gpu_fci(p)
        s = 6
    else:
        h, g = synth.real_integrals(16, 9, 71)
        f = fci.FCI(0).setup_integrals(h, g).build_strings(2, 2).build_das([4, 4, 4, 4], [1, 1, 0, 0], [1, 1, 0, 0], 1)
        s = 3
    c = torch.from_numpy(synth.random_vector(f.n_det, seed=4)).cuda()
    before = f.sigma(c, precision="oz_bf16", n_slices=s).clone()
    rep = f.tune(c, s, reps=2)
    cands = rep["candidates"]
    assert len(cands) >= (3 if kind == "fci" else 1)
    assert rep["chosen"]["ms"] == min(x["ms"] for x in cands)
    after = f.sigma(c, precision="oz_bf16", n_slices=s)
    f.sync_status()
    assert torch.equal(before, after)


def test_tuner_rejects_spinor_strings(fci_lib):
    h, g = synth.complex_integrals(6, 4, 5)
    f = fci.FCI(0).setup_integrals(h, g).build_strings(3, -1)
    c = torch.zeros(f.n_det, dtype=torch.complex128, device="cuda")
    with pytest.raises(fci.FCIError):
        f.tune(c, 6)
