"""GPU parity: libnbcore (through its C ABI) against the FP64 oracle.

Tolerances (the bar of the hot path: FP32 pair arithmetic against FP64):
  * neighbour pair sets: identical, except pairs whose FP64 r^2 lies within
    8 ulp(fp32) of r_nl^2, which are found by brute force and counted;
  * forces: relative RMS <= 1e-5 against FP64;
  * energies: relative <= 1e-6 per component against FP64 (PME: against the
    FP64 smooth PME with the same mesh);
  * integer/determinism checks are bitwise.
"""
import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from oracle import pme as opme
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import (band, dev_xq, oracle_params, oracle_pme, oracle_real_space, pair_set,
                      pairs_near_boundary, rel_rms)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F_TOL = 1e-5
E_TOL = 1e-6


def _forces(h, s, terms=nbcore.NB_TERM_ALL, xq=None):
    xq = dev_xq(s) if xq is None else xq
    f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    h.nonbonded_forces(xq, f, e, terms=terms)
    h.check()
    return f.cpu().numpy().astype(np.float64), e.cpu().numpy()[0]


def _jittered_fcc(seed=7, jitter=0.05):
    s = wl.lj_fcc()
    rng = np.random.default_rng(seed)
    x = s.x.astype(np.float64) + rng.uniform(-jitter, jitter, s.x.shape)
    s.x = (x - s.box * np.floor(x / s.box)).astype(np.float32)
    return s


# ------------------------------------------------------------ neighbour lists

# tile 256 splits every stencil (864 candidates for cell_div 1) over several
# shared-memory tiles
@pytest.mark.parametrize("tile,cell_div", [(0, 1), (256, 2), (256, 1), (0, 2)])
def test_neighbor_set_lj_fcc_864(tile, cell_div):
    s = _jittered_fcc()
    r_nl = s.r_cut + s.r_skin
    with nbcore.Handle([s], stencil_tile=tile, cell_div=cell_div) as h:
        pairs, n = h.nl_build(dev_xq(s), force_rebuild=True)
        gpu = pair_set(pairs.cpu().numpy())
    ref, n_band = oracle.neighbor_pairs(s.x.astype(np.float64), oracle_params(s), r_nl, band=band(r_nl))
    assert n == len(gpu)
    assert n_band == 0
    assert gpu == pair_set(ref)


def test_neighbor_set_water_with_exclusions_ragged():
    # 1203 molecules on a subset of an 11^3 lattice: ragged cells, exclusions
    s = wl.water_box(n_side=11, L=34.2, seed=3, n_mol=1203)
    r_nl = s.r_cut + s.r_skin
    with nbcore.Handle([s]) as h:
        pairs, n = h.nl_build(dev_xq(s), force_rebuild=True)
        gpu = pair_set(pairs.cpu().numpy())
    ref, n_band = oracle.neighbor_pairs(s.x.astype(np.float64), oracle_params(s), r_nl, excl=s.excl,
                                        band=band(r_nl))
    # pairs whose FP64 r^2 is within 8 ulp(fp32) of r_nl^2 may legitimately differ
    amb = pairs_near_boundary(s.x, s.box, r_nl, band(r_nl))
    assert len(amb) == n_band
    ref = pair_set(ref)
    assert gpu - amb == ref - amb
    assert len(gpu ^ ref) <= n_band


def test_pair_export_counts_again_after_a_rebuild_between_calls():
    # a counting call stores the rows' pair counts for the writing call that usually
    # follows; a writing call that rebuilds the list first (other positions) must not use
    # them: the build clears them and the export counts again
    import ctypes
    s1, s2 = _jittered_fcc(9), _jittered_fcc(10)  # same box and atom count, other positions
    r_nl = s2.r_cut + s2.r_skin
    x1, x2 = dev_xq(s1), dev_xq(s2)
    with nbcore.Handle([s1]) as h:
        n = ctypes.c_int64(0)
        xp1 = nbcore._ptr(x1, torch.float32, (s1.n, 4), "xq")
        xp2 = nbcore._ptr(x2, torch.float32, (s2.n, 4), "xq")
        assert h._lib.nl_build(h._h, xp1, None, 0, ctypes.byref(n), 1, None) == 0
        cap = 2 * int(n.value)
        out = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
        assert h._lib.nl_build(h._h, xp2, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(n), 1, None) == 0
        torch.cuda.synchronize()
        n2 = int(n.value)
        assert n2 <= cap
        gpu = pair_set(out[:n2].cpu().numpy())
        # and the usual sequence on the same list: count, then write from the stored counts
        pairs, n3 = h.nl_build(x2)
        assert n3 == n2 and pair_set(pairs.cpu().numpy()) == gpu
    ref, n_band = oracle.neighbor_pairs(s2.x.astype(np.float64), oracle_params(s2), r_nl, band=band(r_nl))
    assert n_band == 0
    assert len(gpu) == n2 and gpu == pair_set(ref)


def test_neighbor_list_open_system():
    s = _jittered_fcc(5)
    s.periodic = False
    r_nl = s.r_cut + s.r_skin
    with nbcore.Handle([s]) as h:
        pairs, n = h.nl_build(dev_xq(s), force_rebuild=True)
        gpu = pair_set(pairs.cpu().numpy())
    ref, _ = oracle.neighbor_pairs(s.x.astype(np.float64), oracle_params(s), r_nl)
    assert gpu == pair_set(ref)


def test_neighbor_list_rebuild_is_lazy_and_valid():
    s = _jittered_fcc(3)
    xq = dev_xq(s)
    with nbcore.Handle([s]) as h:
        h.nl_build(xq, force_rebuild=True)
        c0 = h.rebuild_count()
        # a displacement below r_skin/2 keeps the list
        xq2 = xq.clone()
        xq2[5, 0] += 0.1
        h.nl_build(xq2)
        assert h.rebuild_count() == c0
        # above r_skin/2 (0.15) triggers a rebuild
        xq2[5, 0] += 0.06
        _, n = h.nl_build(xq2)
        assert h.rebuild_count() == c0 + 1
        s2 = wl.lj_fcc()
        s2.x = xq2[:, :3].cpu().numpy()
        ref, _ = oracle.neighbor_pairs(s2.x.astype(np.float64), oracle_params(s2), s2.r_cut + s2.r_skin)
        assert n == len(ref)


def test_small_box_folds_axes_without_a_stencil():
    # L = 2.4 r_nl: two cells per axis, so every axis is visited whole and folded per pair
    r_nl = 2.8
    s = wl.lj_random(256, seed=17)
    assert 2 * r_nl <= s.box[0] < 3 * r_nl
    with nbcore.Handle([s]) as h:
        pairs, n = h.nl_build(dev_xq(s), force_rebuild=True)
        gpu = pair_set(pairs.cpu().numpy())
        f, e = _forces(h, s, terms=nbcore.NB_TERM_LJ)
    ref, n_band = oracle.neighbor_pairs(s.x.astype(np.float64), oracle_params(s), r_nl, band=band(r_nl))
    assert n_band == 0 and gpu == pair_set(ref)
    eo, fo = oracle_real_space(s)
    assert rel_rms(f, fo) <= F_TOL
    assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0])


@pytest.mark.parametrize("wrap", [False, True])
def test_forces_after_boundary_crossing_without_rebuild(wrap):
    # every atom moves by 0.06..0.14 < r_skin/2 along x: atoms near L leave the box (or,
    # wrapped by the caller, reappear near 0) while the list from the build is kept
    s = _jittered_fcc(5)
    with nbcore.Handle([s]) as h:
        _forces(h, s, terms=nbcore.NB_TERM_LJ)
        c0 = h.rebuild_count()
        step = np.random.default_rng(3).uniform(0.06, 0.14, s.n)
        x = s.x.astype(np.float64)
        x[:, 0] += step
        if wrap:
            x -= s.box * np.floor(x / s.box)
        s.x = x.astype(np.float32)
        f, e = _forces(h, s, terms=nbcore.NB_TERM_LJ)
        assert h.rebuild_count() == c0
    eo, fo = oracle_real_space(s)
    assert rel_rms(f, fo) <= F_TOL
    assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0])


# ---------------------------------------------------------------- forces

@pytest.mark.parametrize("switch", [False, True])
def test_lj_forces_and_energy_864(switch):
    s = _jittered_fcc(11)
    if switch:
        s.r_switch = 2.2
    with nbcore.Handle([s]) as h:
        f, e = _forces(h, s, terms=nbcore.NB_TERM_LJ)
    eo, fo = oracle_real_space(s)
    assert rel_rms(f, fo) <= F_TOL
    assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0])
    assert np.abs(f.sum(axis=0)).max() < 1e-6 * np.abs(fo).max() * np.sqrt(s.n)


# tile 256 splits each ~2250-candidate stencil over nine shared-memory tiles
@pytest.mark.parametrize("tile", [0, 256])
def test_water_real_space_forces_and_energies(tile):
    s = wl.water_box(n_side=10, L=31.05, seed=5, pme_grid=32)
    with nbcore.Handle([s], stencil_tile=tile) as h:
        f, e = _forces(h, s, terms=nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL)
    eo, fo = oracle_real_space(s)
    assert rel_rms(f, fo) <= F_TOL
    for k in range(4):
        assert abs(e[k] - eo[k]) <= E_TOL * abs(eo[k]), (k, e[k], eo[k])
    assert e[4] == 0.0


def test_pme_spread_gather_and_energy():
    s = wl.water_box(n_side=10, L=31.05, seed=6, pme_grid=32)
    K = s.pme_grid
    Eo, Fo, Qo, phio = opme.pme(s.x.astype(np.float64), s.q.astype(np.float64), s.box, s.alpha, s.ke, K,
                                return_grid=True)
    xq = dev_xq(s)
    with nbcore.Handle([s]) as h:
        h.nl_build(xq, force_rebuild=True)
        grid = torch.empty(int(np.prod(K)), dtype=torch.float32, device="cuda")
        h.pme_spread(xq, grid)
        g = grid.cpu().numpy().reshape(K)
        assert np.abs(g - Qo).max() <= 1e-6 * np.abs(Qo).max()
        f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        h.pme_gather(xq, torch.from_numpy(phio.astype(np.float32).ravel()).cuda(), f)
        assert rel_rms(f.cpu().numpy(), Fo) <= F_TOL
        fp, ep = _forces(h, s, terms=nbcore.NB_TERM_PME)
    assert rel_rms(fp, Fo) <= F_TOL
    assert abs(ep[4] - Eo) <= E_TOL * abs(Eo)


@pytest.mark.parametrize("shift", [-2, 4])
def test_caller_coordinates_whole_boxes_away(shift):
    """The list build and the mesh half of PME read the caller's positions, which need
    not lie in the box.  In a box of 31 A with positions on a 2^-16 A grid, moving each
    coordinate of each atom by 0 or `shift` box lengths is exact in FP32, so the wrapped
    positions are the unshifted ones: the real-space energies are bitwise those of the
    unshifted evaluation, and the PME forces and energy (evaluated from the shifted
    coordinates themselves) agree with it and with the oracle."""
    s = wl.water_box(n_side=10, L=31.0, seed=6, pme_grid=32)
    s.x = (np.mod(np.round(s.x.astype(np.float64) * 65536.0) / 65536.0, s.box)).astype(np.float32)
    rng = np.random.default_rng(3)
    k = rng.integers(0, 2, size=(s.n, 3)) * shift
    x_sh = s.x.astype(np.float64) + k * s.box
    x32 = x_sh.astype(np.float32)
    assert np.array_equal(x32.astype(np.float64), x_sh)  # the shift is exact in FP32

    def run(x):
        f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        e = torch.empty((1, 6), dtype=torch.float64, device="cuda")
        with nbcore.Handle([s]) as h:
            h.nonbonded_forces(torch.from_numpy(nbcore.pack_xq(x, s.q)).cuda(), f, e, force_rebuild=True)
            h.check()
        return f.cpu().numpy().astype(np.float64), e.cpu().numpy()[0]
    f0, e0 = run(s.x)
    f1, e1 = run(x32)
    assert np.array_equal(e1[:4], e0[:4])  # LJ, direct, exclusion, self
    assert abs(e1[4] - e0[4]) <= E_TOL * abs(e0[4])
    assert rel_rms(f1, f0) <= F_TOL
    eo, fo = oracle_real_space(s)
    Ep, Fp = oracle_pme(s)
    assert rel_rms(f1, fo + Fp) <= F_TOL
    assert abs(e1[4] - Ep) <= E_TOL * abs(Ep)


def test_water_config2_full_size_sampled():
    """The full 8000-molecule box in the benchmark's configuration; forces checked
    on a sample of 400 atoms (oracle rows), energies from all rows."""
    s = wl.water_box()
    assert s.n == 24000
    with nbcore.Handle([s]) as h:
        f, e = _forces(h, s)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(s.n, 400, replace=False))
    er, fr = oracle.nonbonded_rows(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), rows,
                                   excl=s.excl)
    Ep, Fp = oracle_pme(s)
    fo = fr + Fp[rows]
    assert rel_rms(f[rows], fo) <= F_TOL
    assert abs(e[4] - Ep) <= E_TOL * abs(Ep)
    all_rows = np.arange(s.n)
    er_all, _ = oracle.nonbonded_rows(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s),
                                      all_rows, excl=s.excl)
    eo = er_all.sum(axis=0)
    for k in range(3):
        assert abs(e[k] - eo[k]) <= E_TOL * abs(eo[k]), (k, e[k], eo[k])
    self_o = -s.ke * s.alpha / np.sqrt(np.pi) * np.sum(s.q.astype(np.float64) ** 2)
    assert abs(e[3] - self_o) <= E_TOL * abs(self_o)


def test_forces_bitwise_deterministic():
    s = wl.water_box(n_side=8, L=24.84, seed=9, pme_grid=24)
    xq = dev_xq(s)
    with nbcore.Handle([s]) as h:
        f1, e1 = _forces(h, s, xq=xq)
        h.nl_build(xq, force_rebuild=True)
        f2, e2 = _forces(h, s, xq=xq)
    assert np.array_equal(f1, f2) and np.array_equal(e1, e2)


# ---------------------------------------------------------------- VJP

@pytest.mark.parametrize("tile", [0, 256])
def test_force_vjp_matches_oracle(tile):
    s = wl.water_box(n_side=6, L=18.9, seed=12, r_cut=8.0, r_skin=1.0)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal((s.n, 3)).astype(np.float32)
    gxo, gqo, gso, geo = oracle.force_vjp(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s),
                                          lam, excl=s.excl)
    xq = dev_xq(s)
    with nbcore.Handle([s], stencil_tile=tile) as h:
        gx = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        gq = torch.empty(s.n, dtype=torch.float32, device="cuda")
        gs = torch.empty(s.n, dtype=torch.float32, device="cuda")
        ge = torch.empty(s.n, dtype=torch.float32, device="cuda")
        h.nonbonded_force_vjp(xq, torch.from_numpy(lam).cuda(), gx, gq, gs, ge)
        h.check()
    assert rel_rms(gx.cpu().numpy(), gxo) <= 1e-5
    assert rel_rms(gq.cpu().numpy(), gqo) <= 1e-5
    o = s.sqrt_eps > 0  # LJ parameters only exist on oxygen
    assert rel_rms(gs.cpu().numpy()[o], gso[o]) <= 1e-5
    assert rel_rms(ge.cpu().numpy(), geo) <= 1e-5


def test_force_vjp_lj_switch_matches_oracle():
    s = _jittered_fcc(21)
    s.r_switch = 2.2
    rng = np.random.default_rng(2)
    lam = rng.standard_normal((s.n, 3)).astype(np.float32)
    gxo, _, gso, geo = oracle.force_vjp(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), lam)
    with nbcore.Handle([s]) as h:
        gx = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        gs = torch.empty(s.n, dtype=torch.float32, device="cuda")
        ge = torch.empty(s.n, dtype=torch.float32, device="cuda")
        h.nonbonded_force_vjp(dev_xq(s), torch.from_numpy(lam).cuda(), gx, None, gs, ge)
        h.check()
    assert rel_rms(gx.cpu().numpy(), gxo) <= 1e-5
    assert rel_rms(gs.cpu().numpy(), gso) <= 1e-5
    assert rel_rms(ge.cpu().numpy(), geo) <= 1e-5


def test_force_vjp_small_box_folded_axes():
    # two cells per axis: every axis is folded per pair in the list build and the kernels
    s = wl.lj_random(216, seed=23, n_types=2)
    s.r_switch = 2.2
    rng = np.random.default_rng(4)
    lam = rng.standard_normal((s.n, 3)).astype(np.float32)
    gxo, _, gso, geo = oracle.force_vjp(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), lam)
    with nbcore.Handle([s]) as h:
        gx = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        gs = torch.empty(s.n, dtype=torch.float32, device="cuda")
        ge = torch.empty(s.n, dtype=torch.float32, device="cuda")
        h.nonbonded_force_vjp(dev_xq(s), torch.from_numpy(lam).cuda(), gx, None, gs, ge)
        h.check()
    assert rel_rms(gx.cpu().numpy(), gxo) <= 1e-5
    assert rel_rms(gs.cpu().numpy(), gso) <= 1e-5
    assert rel_rms(ge.cpu().numpy(), geo) <= 1e-5


# ---------------------------------------------------------------- MD

def _dmin(d, box):
    return d - box * np.round(d / box)


def test_md_config1_100_steps_against_oracle():
    s = wl.lj_fcc()  # FCC 864, T* = 0.72 Maxwell-Boltzmann, dt = 0.005
    n_steps, dt = 100, 0.005
    xq = dev_xq(s)
    v = torch.zeros((s.n, 4), dtype=torch.float32, device="cuda")
    v[:, :3] = torch.from_numpy(s.v).cuda()
    v[:, 3] = 1.0 / torch.from_numpy(s.mass).cuda()
    E = torch.zeros((n_steps + 1, 1, 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle([s]) as h:
        h.md_step(xq, v, torch.tensor([dt], dtype=torch.float32, device="cuda"), n_steps, E,
                  terms=nbcore.NB_TERM_LJ)
        h.check()
    p = oracle_params(s)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p)
        return f, float(e[0])
    xo, vo, Uo, Ko = odyn.velocity_verlet(s.x.astype(np.float64), s.v.astype(np.float64),
                                          1.0 / s.mass.astype(np.float64), dt, n_steps, fe)
    Eg = E.cpu().numpy()[:, 0, :]
    np.testing.assert_allclose(Eg[:, 0], Uo, rtol=1e-5)
    np.testing.assert_allclose(Eg[:, 5], Ko, rtol=1e-5)
    xg = xq[:, :3].cpu().numpy().astype(np.float64)
    assert np.sqrt(np.mean(_dmin(xg - xo, s.box) ** 2)) < 1e-4
    # NVE: total energy drift small relative to the kinetic energy
    H = Eg[:, 0] + Eg[:, 5]
    assert np.abs(H - H[0]).max() < 0.02 * Ko[0]


# ---------------------------------------------------------------- batching

def test_batched_systems_match_single_system_bitwise():
    systems = [wl.lj_random(700, seed=1), wl.water_box(n_side=9, L=27.9, seed=2, pme_grid=27),
               wl.lj_random(1311, seed=3), wl.water_box_density(400, seed=4)]
    opts = dict(cell_div=1, max_neighbors=1024)
    xs = [dev_xq(s) for s in systems]
    fb = torch.empty((sum(s.n for s in systems), 3), dtype=torch.float32, device="cuda")
    eb = torch.empty((len(systems), 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle(systems, **opts) as h:
        h.nonbonded_forces(torch.cat(xs), fb, eb)
        h.check()
    off = 0
    for k, s in enumerate(systems):
        with nbcore.Handle([s], **opts) as h1:
            f1, e1 = _forces(h1, s, xq=xs[k])
        assert np.array_equal(fb[off:off + s.n].cpu().numpy().astype(np.float64), f1)
        assert np.array_equal(eb[k].cpu().numpy(), e1)
        off += s.n


def test_batched_systems_take_their_own_cell_size():
    """Without a handle-wide cell size each system takes its own default (cells of edge
    r_nl/2 for the dense 24k water box, r_nl for the LJ fluids): batched forces and
    energies are bitwise those of each system on its own handle."""
    from paper_2503_20541_b300 import autotune
    systems = [wl.lj_random(700, seed=1), wl.water_box(), wl.lj_random(1311, seed=3)]
    assert [autotune.auto_cell_div(s) for s in systems] == [1, 2, 1]
    opts = dict(max_neighbors=1024, stencil_tile=2560)
    xs = [dev_xq(s) for s in systems]
    fb = torch.empty((sum(s.n for s in systems), 3), dtype=torch.float32, device="cuda")
    eb = torch.empty((len(systems), 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle(systems, **opts) as h:
        h.nonbonded_forces(torch.cat(xs), fb, eb)
        h.check()
    off = 0
    for k, s in enumerate(systems):
        with nbcore.Handle([s], **opts) as h1:
            f1, e1 = _forces(h1, s, xq=xs[k])
        assert np.array_equal(fb[off:off + s.n].cpu().numpy().astype(np.float64), f1)
        assert np.array_equal(eb[k].cpu().numpy(), e1)
        off += s.n


# ---------------------------------------------------------------- errors

def test_error_paths_return_status_without_faulting():
    s = wl.water_box(n_side=6, L=18.9, seed=1, r_cut=8.0, r_skin=1.0)
    xq = dev_xq(s)
    with nbcore.Handle([s], max_neighbors=32) as h:
        with pytest.raises(nbcore.NbError) as ei:
            h.nl_build(xq, force_rebuild=True)
        assert ei.value.status == 3
    xbad = xq.clone()
    xbad[7, 1] = float("nan")
    with nbcore.Handle([s]) as h:
        with pytest.raises(nbcore.NbError) as ei:
            h.nl_build(xbad, force_rebuild=True)
        assert ei.value.status == 5
        # the handle stays usable after an error
        _, n = h.nl_build(xq, force_rebuild=True)
        assert n > 0
    small = wl.lj_fcc(n_cells=2)  # L = 3.36 < 2 r_nl
    with pytest.raises(nbcore.NbError) as ei:
        nbcore.Handle([small])
    assert ei.value.status == 2


# ---------------------------------------------------------------- all-pairs baseline

def test_allpairs_baseline_matches_oracle_and_list_path():
    systems = [_jittered_fcc(31), wl.lj_random(1500, seed=32)]
    systems[1].r_switch = 2.2
    n = sum(s.n for s in systems)
    xq = torch.cat([dev_xq(s) for s in systems])
    fa = torch.empty((n, 3), device="cuda")
    ea = torch.empty((2, 6), dtype=torch.float64, device="cuda")
    fl = torch.empty_like(fa)
    el = torch.empty_like(ea)
    with nbcore.Handle(systems) as h:
        h.nonbonded_forces_allpairs(xq, fa, ea)
        h.nonbonded_forces(xq, fl, el, terms=nbcore.NB_TERM_LJ)
        h.check()
    off = 0
    for k, s in enumerate(systems):
        eo, fo = oracle_real_space(s)
        f = fa[off:off + s.n].cpu().numpy().astype(np.float64)
        assert rel_rms(f, fo) <= F_TOL
        assert abs(ea[k, 0].item() - eo[0]) <= E_TOL * abs(eo[0])
        assert rel_rms(f, fl[off:off + s.n].cpu().numpy().astype(np.float64)) <= F_TOL
        off += s.n


def test_md_with_pme_against_oracle():
    """Velocity-Verlet steps of a small water box with the full electrostatics (PME on
    the handle's second stream feeding the integrator) against the FP64 integrator with
    real-space + smooth-PME forces."""
    s = wl.water_box(n_side=10, L=31.05, seed=5, pme_grid=32)
    n_steps, dt = 5, 0.0005
    rng = np.random.default_rng(4)
    v0 = (0.05 * rng.standard_normal((s.n, 3))).astype(np.float32)
    mass = np.where(s.q < 0, 15.999, 1.008).astype(np.float32)
    xq = dev_xq(s)
    v = torch.zeros((s.n, 4), dtype=torch.float32, device="cuda")
    v[:, :3] = torch.from_numpy(v0).cuda()
    v[:, 3] = torch.from_numpy(1.0 / mass).cuda()
    E = torch.zeros((n_steps + 1, 1, 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle([s]) as h:
        h.md_step(xq, v, torch.tensor([dt], dtype=torch.float32, device="cuda"), n_steps, E)
        h.check()

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, oracle_params(s), excl=s.excl)
        ep, fp = opme.pme(x, s.q.astype(np.float64), s.box, s.alpha, s.ke, s.pme_grid)
        return f + fp, float(e.sum() + ep)
    xo, vo, Uo, Ko = odyn.velocity_verlet(s.x.astype(np.float64), v0.astype(np.float64),
                                          1.0 / mass.astype(np.float64), dt, n_steps, fe)
    Eg = E.cpu().numpy()[:, 0, :]
    # per component at the start; the total is a small residual of large components
    # (exclusion and self terms), so per step it is bounded against their magnitudes
    e0, _ = oracle.nonbonded(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), excl=s.excl)
    ep0, _ = opme.pme(s.x.astype(np.float64), s.q.astype(np.float64), s.box, s.alpha, s.ke, s.pme_grid)
    comp = np.concatenate([e0, [ep0]])
    for k in range(5):
        assert abs(Eg[0, k] - comp[k]) <= E_TOL * abs(comp[k]), (k, Eg[0, k], comp[k])
    np.testing.assert_allclose(Eg[:, :5].sum(axis=1), Uo, rtol=0, atol=E_TOL * np.abs(comp).sum())
    np.testing.assert_allclose(Eg[:, 5], Ko, rtol=1e-5)
    xg = xq[:, :3].cpu().numpy().astype(np.float64)
    assert np.sqrt(np.mean(_dmin(xg - xo, s.box) ** 2)) < 1e-5
