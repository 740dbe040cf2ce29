"""Dynamic list pruning between builds (nb_options.prune_skin): on the first evaluation after
a build, and whenever an atom has moved more than half the prune skin since, every row of
the Verlet list is re-partitioned at the current positions into the pairs within
r_c + prune_skin and the rest, and the pair kernels skip the rest.  The pair set within
r_c must be exactly the unpruned path's: both take the same FP32 cut-off test on the same
positions, so a pruned and an unpruned handle differ only by summation order, while one
pair within r_c missed by a stale partition moves two atoms by the unswitched LJ force at
r_c (0.039 eps/sigma), far above that rounding.  The sequences below move the atoms by less
than r_skin/2 (no list rebuild) but, at the third evaluation, by more than half the prune
skin since the prune of the second, so the re-partition is exercised; and a batched handle
whose systems re-prune at different evaluations gives each system the results of its own
handle, bit for bit (the prune state is kept per system)."""
import numpy as np
import pytest

from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import oracle_real_space, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRUNE = 0.1  # sigma: half of it (0.05) is crossed from the third evaluation on, r_skin/2 (0.15) never


def _sequence(s, seed, amps):
    """Positions x0 + U(-a, a) per coordinate for each amplitude a (FP32, caller order)."""
    rng = np.random.default_rng(seed)
    out = []
    for a in amps:
        out.append((s.x.astype(np.float64) + rng.uniform(-a, a, s.x.shape)).astype(np.float32))
    return out


def _forces(h, xs_list, q, terms=nbcore.NB_TERM_LJ):
    f = torch.empty((xs_list[0].shape[0], 3), dtype=torch.float32, device="cuda")
    e = torch.empty((h.n_sys, 6), dtype=torch.float64, device="cuda")
    out = []
    for x in xs_list:
        xq = torch.from_numpy(nbcore.pack_xq(x, q)).cuda()
        h.nonbonded_forces(xq, f, e, terms=terms)
        h.check()
        out.append((f.cpu().numpy().copy(), e.cpu().numpy().copy()))
    return out


def test_pruned_forces_equal_unpruned_pair_set():
    s = wl.lj_random(4000, seed=11)
    # amplitudes: the build at x0; 0.02 (pruned at this evaluation, the first after the
    # build); 0.045 and 0.05 (some atom > PRUNE/2 from the prune positions: re-partitioned;
    # every atom < 0.05 sqrt(3) < r_skin/2 from x0)
    xs_list = _sequence(s, 5, [0.0, 0.02, 0.045, 0.05])
    with nbcore.Handle([s], prune_skin=PRUNE) as hp, nbcore.Handle([s], prune_skin=-1.0) as hu:
        got = _forces(hp, xs_list, s.q)
        ref = _forces(hu, xs_list, s.q)
        assert hp.rebuild_count() == 1 and hu.rebuild_count() == 1  # one build: the displacements stay inside r_skin/2
    for k, ((fp, ep), (fu, eu)) in enumerate(zip(got, ref)):
        dev = np.abs(fp.astype(np.float64) - fu).max()
        assert dev < 0.01, (k, dev)  # a missed pair within r_c: ~0.039 on two atoms
        assert abs(ep[0, 0] - eu[0, 0]) <= 1e-6 * abs(eu[0, 0]), k
    # and the last state against the FP64 oracle
    eo, fo = oracle_real_space(s, xs_list[3].astype(np.float64))
    assert rel_rms(got[3][0], fo) <= 1e-5


def test_water_pruned_by_default_matches_oracle():
    s = wl.water_box(n_side=10, L=31.05, seed=5, pme_grid=32)  # r_skin 2.25: prune skin 0.75 by default
    xs_list = _sequence(s, 6, [0.0, 0.1, 0.5])  # 0.5 A per coordinate: > 0.375 from the prune positions
    terms = nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL
    with nbcore.Handle([s]) as hp, nbcore.Handle([s], prune_skin=-1.0) as hu:
        got = _forces(hp, xs_list, s.q, terms)
        ref = _forces(hu, xs_list, s.q, terms)
        assert hp.rebuild_count() == 1
    for k, ((fp, ep), (fu, eu)) in enumerate(zip(got, ref)):
        assert rel_rms(fp, fu) <= 1e-6, k
        # the same pairs summed in another order: FP32 rounding only
        for c in (0, 1):
            assert abs(ep[0, c] - eu[0, c]) <= 1e-5 * abs(eu[0, c]), (k, c)
    eo, fo = oracle_real_space(s, xs_list[2].astype(np.float64))
    assert rel_rms(got[2][0], fo) <= 1e-5


def test_batched_prune_state_is_per_system():
    a = wl.lj_random(2000, seed=21)
    b = wl.lj_random(3000, seed=22)
    rng = np.random.default_rng(7)
    amps_a = [0.0, 0.005, 0.01, 0.012]  # within 0.017 sqrt(3) < PRUNE/2 of the prune positions
    amps_b = [0.0, 0.01, 0.045, 0.05]  # beyond it from the third evaluation on
    xa = [(a.x.astype(np.float64) + rng.uniform(-m, m, a.x.shape)).astype(np.float32) for m in amps_a]
    xb = [(b.x.astype(np.float64) + rng.uniform(-m, m, b.x.shape)).astype(np.float32) for m in amps_b]
    with nbcore.Handle([a, b], prune_skin=PRUNE) as hab:
        both = _forces(hab, [np.concatenate([u, v]) for u, v in zip(xa, xb)], np.concatenate([a.q, b.q]))
    with nbcore.Handle([a], prune_skin=PRUNE) as ha:
        only_a = _forces(ha, xa, a.q)
    with nbcore.Handle([b], prune_skin=PRUNE) as hb:
        only_b = _forces(hb, xb, b.q)
    for k in range(len(xa)):
        fab, eab = both[k]
        assert np.array_equal(fab[:a.n], only_a[k][0]), k
        assert np.array_equal(fab[a.n:], only_b[k][0]), k
        assert eab[0, 0] == only_a[k][1][0, 0] and eab[1, 0] == only_b[k][1][0, 0], k


def test_prune_skin_option_is_validated():
    s = wl.lj_random(500, seed=1)
    with pytest.raises(nbcore.NbError):
        nbcore.Handle([s], prune_skin=float("nan"))
