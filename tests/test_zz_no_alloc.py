"""The allocation-free PME spreading entry point (pme_spread_static).

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator (a framework's memory pool or a fixed arena), or they run where the
device-wide synchronisation of an allocation is not allowed.  pme_spread_static
serves them without a handle, keeping its accumulation mesh in a static device
array.  This file checks, through the C ABI, that two calls in a row each give the
same mesh as the handle-based pme_spread (within the tolerance of the PME spread
test) -- so the shared static mesh is cleared between calls -- that its mesh equals the
FP64 oracle's charge mesh, that an empty system gives an all-zero mesh, and that a mesh
above the static capacity is refused, also when the product of its sizes would wrap.
It sits in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_20541_b300 import nbcore, workloads as wl

from oracle import pme as opme

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


def test_static_spread_matches_the_oracle_charge_mesh():
    # Essmann's smooth PME charge mesh Q (order-4 cardinal B-splines), FP64 on the host
    s = wl.water_box(n_side=10, L=31.05, seed=8, pme_grid=32)
    K = s.pme_grid
    Qo = opme.pme(s.x.astype(np.float64), s.q.astype(np.float64), s.box, s.alpha, s.ke, K, return_grid=True)[2]
    g = torch.full((int(np.prod(K)),), float("nan"), dtype=torch.float32, device="cuda")
    for _ in range(2):  # the second call reuses the static mesh the first one filled
        nbcore.pme_spread_static(dev_xq(s), s.box, K, g)
        got = g.cpu().numpy().reshape(K)
        assert np.abs(got - Qo).max() <= 1e-6 * np.abs(Qo).max()


def test_static_spread_refuses_a_mesh_whose_point_count_would_wrap():
    # 2^22 * 2^21 * 2^21 = 2^64 wraps a 64-bit product to 0; the sizes are checked one by
    # one, before the multiplication, and nothing is written to the (small) grid
    s = wl.water_box(n_side=4, L=12.42, seed=1, pme_grid=16)
    xq = dev_xq(s)
    grid = torch.full((16,), 7.0, dtype=torch.float32, device="cuda")
    lib = nbcore.load()
    box = np.ascontiguousarray(np.asarray(s.box, np.float64))
    m = np.array([1 << 22, 1 << 21, 1 << 21], np.int32)
    st = lib.pme_spread_static(ctypes.c_void_p(xq.data_ptr()), int(xq.shape[0]), box.ctypes.data, m.ctypes.data,
                               ctypes.c_void_p(grid.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    torch.cuda.synchronize()
    assert torch.all(grid == 7.0).item()


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
