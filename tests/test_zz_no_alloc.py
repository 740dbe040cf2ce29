"""The allocation-free PME spreading entry point (pme_spread_static).

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator (a framework's memory pool or a fixed arena), or they run where the
device-wide synchronisation of an allocation is not allowed.  pme_spread_static
serves them without a handle, keeping its accumulation mesh in a static device
array.  This file checks, through the C ABI, that two calls in a row each give the
same mesh as the handle-based pme_spread (within the tolerance of the PME spread
test) -- so the shared static mesh is cleared between calls -- that an empty
system gives an all-zero mesh, and that a mesh above the static capacity is refused.  It sits in its own file, collected last.
"""
import numpy as np
import pytest

from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import dev_xq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _handle_mesh(s, xq):
    with nbcore.Handle([s]) as h:
        grid = torch.empty(int(np.prod(s.pme_grid)), dtype=torch.float32, device="cuda")
        h.pme_spread(xq, grid)
        h.check()
    return grid.cpu().numpy()


def test_static_spread_matches_handle_spread_on_two_calls_in_a_row():
    a = wl.water_box(n_side=10, L=31.05, seed=6, pme_grid=32)
    b = wl.water_box(n_side=10, L=31.05, seed=7, pme_grid=32)
    xa, xb = dev_xq(a), dev_xq(b)
    ref_a, ref_b = _handle_mesh(a, xa), _handle_mesh(b, xb)
    ga = torch.full((int(np.prod(a.pme_grid)),), float("nan"), dtype=torch.float32, device="cuda")
    gb = torch.full_like(ga, float("nan"))
    nbcore.pme_spread_static(xa, a.box, a.pme_grid, ga)
    nbcore.pme_spread_static(xb, b.box, b.pme_grid, gb)
    torch.cuda.synchronize()
    for g, ref in ((ga.cpu().numpy(), ref_a), (gb.cpu().numpy(), ref_b)):
        assert np.all(np.isfinite(g))
        assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max()


def test_static_spread_rejects_meshes_beyond_its_capacity():
    s = wl.water_box(n_side=4, L=12.42, seed=1, pme_grid=16)
    xq = dev_xq(s)
    K = (128, 128, 128)  # 2^21 points > NB_STATIC_MESH_MAX
    grid = torch.empty(int(np.prod(K)), dtype=torch.float32, device="cuda")
    with pytest.raises(nbcore.NbError) as ei:
        nbcore.pme_spread_static(xq, s.box, K, grid)
    assert ei.value.status == 1


def test_static_spread_of_an_empty_system_is_an_all_zero_mesh():
    # an empty system spreads no charge; the call after a non-empty one also shows that
    # the previous call's sums left in the shared static mesh do not reach the output
    s = wl.water_box(n_side=4, L=12.42, seed=2, pme_grid=16)
    K = s.pme_grid
    g = torch.empty(int(np.prod(K)), dtype=torch.float32, device="cuda")
    nbcore.pme_spread_static(dev_xq(s), s.box, K, g)
    assert torch.count_nonzero(g).item() > 0
    empty = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    g.fill_(float("nan"))
    nbcore.pme_spread_static(empty, s.box, K, g)
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
