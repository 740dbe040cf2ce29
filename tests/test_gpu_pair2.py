"""The LJ-only pair kernel with two atoms per warp (k_pair2) against the warp-per-atom
kernel: an LJ system evaluated alone runs k_pair2; the same system in a handle that also
holds a charged water box runs k_pair (the handle's kernels then carry electrostatics,
skipped for the uncharged system).  Forces and energies must agree bit for bit: on a just
built list, on the kept list after the atoms have moved (the back parts walked through the
queue), with and without energies, with the LJ switch, in a box small enough for per-pair
minimum images, and for several LJ systems of different sizes in one handle.  The kernel
runs on handles large enough for blocks of 16 atoms (9,472 atoms on 148 SMs), so the
LJ-only handles here hold 10,000 atoms or more (the small boxes as a batch of 40)."""
import numpy as np
import pytest

from paper_2503_20541_b300 import nbcore, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(systems, xs_list, energies, **opts):
    xq0 = [nbcore.pack_xq(s.x, s.q) for s in systems]
    n = sum(s.n for s in systems)
    f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((len(systems), 6), dtype=torch.float64, device="cuda")
    out = []
    with nbcore.Handle(systems, **opts) as h:
        for xs in xs_list:
            parts = [nbcore.pack_xq(x, s.q) if x is not None else q for x, s, q in zip(xs, systems, xq0)]
            xq = torch.from_numpy(np.concatenate(parts)).cuda()
            h.nonbonded_forces(xq, f, e if energies else None)
            h.check()
            out.append((f.cpu().numpy().copy(), e.cpu().numpy().copy() if energies else None))
        rebuilds = h.rebuild_count()
    return out, rebuilds


def _moves(s, seed, amps):
    rng = np.random.default_rng(seed)
    return [(s.x.astype(np.float64) + rng.uniform(-a, a, s.x.shape)).astype(np.float32) for a in amps]


def _water():
    return wl.water_box(n_side=8, L=24.84, seed=9, pme_grid=24)


@pytest.mark.parametrize("case", ["random", "switch"])
@pytest.mark.parametrize("energies", [True, False])
def test_two_atoms_per_warp_bitwise_equal(case, energies):
    if case == "random":
        s = wl.lj_random(12000, seed=31)
    else:
        s = wl.lj_random(10000, seed=32, n_types=2)
        s.r_switch = 2.2
    amps = [0.0, 0.03, 0.06]  # below r_skin/2 = 0.15 per atom: the list is kept
    xs = _moves(s, 7, amps)
    w = _water()
    alone, rb1 = _run([s], [[x] for x in xs], energies)
    mixed, rb2 = _run([s, w], [[x, None] for x in xs], energies)
    assert rb1 == 1 and rb2 == 1
    for k, ((fa, ea), (fm, em)) in enumerate(zip(alone, mixed)):
        assert np.array_equal(fa, fm[:s.n]), (case, k, np.abs(fa - fm[:s.n]).max())
        if energies:
            assert np.array_equal(ea[0], em[0]), (case, k, ea[0], em[0])


@pytest.mark.parametrize("kind", ["sizes", "small_boxes"])
def test_several_lj_systems_in_one_handle(kind):
    if kind == "sizes":
        systems = [wl.lj_random(n, seed=40 + n % 97) for n in (3100, 4700, 2900)]
    else:  # 40 boxes of 256 atoms, 2 cells of r_nl per axis: per-pair minimum images
        systems = [wl.lj_fcc(n_cells=4, seed=33 + k) for k in range(40)]
    amps = [0.0, 0.05]
    moves = [_moves(s, 11 + k, amps) for k, s in enumerate(systems)]
    xs_list = [[moves[k][a] for k in range(len(systems))] for a in range(len(amps))]
    batched, _ = _run(systems, xs_list, True)
    offs = np.cumsum([0] + [s.n for s in systems])
    for k, s in enumerate(systems[:3]):
        alone, _ = _run([s, _water()], [[moves[k][a], None] for a in range(len(amps))], True)
        for a in range(len(amps)):
            assert np.array_equal(batched[a][0][offs[k]:offs[k + 1]], alone[a][0][:s.n]), (k, a)
            assert np.array_equal(batched[a][1][k], alone[a][1][0]), (k, a)


def _vjp(systems, xs_list, lam_lj):
    xq0 = [nbcore.pack_xq(s.x, s.q) for s in systems]
    n = sum(s.n for s in systems)
    lam = np.zeros((n, 3), np.float32)
    lam[:lam_lj.shape[0]] = lam_lj
    lam_d = torch.from_numpy(lam).cuda()
    outs = []
    with nbcore.Handle(systems) as h:
        for xs in xs_list:
            parts = [nbcore.pack_xq(x, s.q) if x is not None else q for x, s, q in zip(xs, systems, xq0)]
            xq = torch.from_numpy(np.concatenate(parts)).cuda()
            gx = torch.empty((n, 3), dtype=torch.float32, device="cuda")
            gq, gs, ge = (torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3))
            f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
            h.nonbonded_force_vjp(xq, lam_d, gx, gq, gs, ge, f)
            h.check()
            outs.append([t.cpu().numpy() for t in (gx, gq, gs, ge, f)])
    return outs


def test_force_vjp_two_atoms_per_warp_bitwise_equal():
    s = wl.lj_random(12000, seed=34, n_types=2)
    s.r_switch = 2.2
    xs = _moves(s, 8, [0.0, 0.05])
    lam = np.random.default_rng(3).standard_normal((s.n, 3)).astype(np.float32)
    alone = _vjp([s], [[x] for x in xs], lam)
    mixed = _vjp([s, _water()], [[x, None] for x in xs], lam)
    for k, (a, m) in enumerate(zip(alone, mixed)):
        for name, ta, tm in zip(("gx", "gq", "gsigma", "gsqrt_eps", "f"), a, m):
            assert np.array_equal(ta, tm[:s.n]), (k, name, np.abs(ta - tm[:s.n]).max())


def test_two_atoms_per_warp_with_pruned_lists():
    """Dynamic list pruning on (prune skin 0.1): the kept rows are re-partitioned and the
    back parts skipped, in both kernels alike."""
    s = wl.lj_random(12000, seed=35)
    xs = _moves(s, 9, [0.0, 0.02, 0.045, 0.06])  # past half the prune skin from the third on
    alone, _ = _run([s], [[x] for x in xs], True, prune_skin=0.1)
    mixed, _ = _run([s, _water()], [[x, None] for x in xs], True, prune_skin=0.1)
    for k, ((fa, ea), (fm, em)) in enumerate(zip(alone, mixed)):
        assert np.array_equal(fa, fm[:s.n]), (k, np.abs(fa - fm[:s.n]).max())
        assert np.array_equal(ea[0], em[0]), k
