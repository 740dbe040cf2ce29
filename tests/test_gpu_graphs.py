"""CUDA-graph capture of libnbcore steps: a replayed graph gives bitwise the results of
the same calls issued directly (batched force evaluation with PME, and velocity-Verlet
steps with lazy list rebuilds inside the graph)."""
import numpy as np
import pytest

from paper_2503_20541_b300 import nbcore, workloads as wl
from paper_2503_20541_b300.graphs import CapturedStep

from _helpers import dev_xq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_captured_batched_forces_equal_direct_calls():
    systems = [wl.lj_random(700, seed=1), wl.water_box(n_side=9, L=27.9, seed=2, pme_grid=27),
               wl.lj_random(1311, seed=3), wl.water_box_density(400, seed=4)]
    n = sum(s.n for s in systems)
    xq = torch.cat([dev_xq(s) for s in systems])
    fd = torch.empty((n, 3), device="cuda")
    ed = torch.empty((len(systems), 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle(systems) as h:
        h.nonbonded_forces(xq, fd, ed)
        h.check()
    fg = torch.zeros_like(fd)
    eg = torch.zeros_like(ed)
    with nbcore.Handle(systems) as h:
        g = CapturedStep(lambda: h.nonbonded_forces(xq, fg, eg))
        fg.zero_()
        eg.zero_()
        g.replay()
        torch.cuda.synchronize()
        h.check()
    assert torch.equal(fd, fg) and torch.equal(ed, eg)


def test_captured_md_steps_equal_direct_calls():
    s = wl.lj_fcc()
    dt = torch.tensor([0.005], dtype=torch.float32, device="cuda")
    v0 = torch.zeros((s.n, 4), dtype=torch.float32, device="cuda")
    v0[:, :3] = torch.from_numpy(s.v).cuda()
    v0[:, 3] = 1.0 / torch.from_numpy(s.mass).cuda()
    x0 = dev_xq(s)
    xd, vd = x0.clone(), v0.clone()
    with nbcore.Handle([s]) as h:
        for _ in range(5):
            h.md_step(xd, vd, dt, 10, terms=nbcore.NB_TERM_LJ)
        h.check()
        nd = h.rebuild_count()
    xg, vg = x0.clone(), v0.clone()
    with nbcore.Handle([s]) as h:
        g = CapturedStep(lambda: h.md_step(xg, vg, dt, 10, terms=nbcore.NB_TERM_LJ))
        xg.copy_(x0)
        vg.copy_(v0)
        h.nl_build(xg, force_rebuild=True)  # same list state as a fresh handle's first call
        r0 = h.rebuild_count()
        for _ in range(5):
            g.replay()
        torch.cuda.synchronize()
        h.check()
        ng = h.rebuild_count() - r0
    assert torch.equal(xd, xg) and torch.equal(vd, vg)
    assert ng == nd - 1 and ng >= 1  # the lazy rebuilds happened inside the graph
