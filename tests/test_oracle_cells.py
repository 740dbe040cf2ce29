"""The oracle's cell-list sums (Sec. 2.1.2, "Neighborlists") against its all-pairs definition.

``oracle.nonbonded_cells`` visits only the atoms of the 27 cells around each atom's cell
(edge >= r_c) plus every excluded partner, so it must reproduce ``oracle.nonbonded`` (the
O(N^2) definition, pinned in test_oracle_pins.py) up to summation order: the same
energies and forces for the Ewald and reaction-field electrostatics, with and without the
LJ switch, for exclusions at any distance and listed in any way, and through its
all-pairs route for open systems and boxes of fewer than 3 cells.  CPU only.
"""
import numpy as np
import pytest

import oracle
from paper_2503_20541_b300 import workloads as wl


def _both(x, q, sig, sqe, p, excl=None):
    e0, f0 = oracle.nonbonded(x, q, sig, sqe, p, excl=excl)
    e1, f1 = oracle.nonbonded_cells(x, q, sig, sqe, p, excl=excl)
    return e0, f0, e1, f1


def _agree(e0, f0, e1, f1, rtol=1e-11):
    np.testing.assert_allclose(e1, e0, rtol=rtol, atol=1e-12 * max(1.0, np.abs(e0).max()))
    np.testing.assert_allclose(f1, f0, rtol=0, atol=rtol * np.abs(f0).max())


def _water(elec, r_cut=4.6, n_mol=216, seed=7):
    s = wl.water_box_density(n_mol, seed)
    if elec == "rf":
        p = oracle.make_params(s.box, r_cut=r_cut, r_switch=r_cut - 0.6, ke=wl.KE_KJ_MOL_A, eps_rf=78.5)
    else:
        p = oracle.make_params(s.box, r_cut=r_cut, r_switch=r_cut - 0.6, alpha=0.8, ke=wl.KE_KJ_MOL_A)
    return s, p


@pytest.mark.parametrize("elec", ["ewald", "rf"])
def test_cells_equal_all_pairs_on_water(elec):
    s, p = _water(elec)
    assert s.box[0] / 4.6 >= 4.0  # at least 4 cells along each axis: the cell route runs
    x = s.x.astype(np.float64)
    _agree(*_both(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl))


@pytest.mark.parametrize("r_switch", [-1.0, 2.0])
def test_cells_equal_all_pairs_on_lj(r_switch):
    s = wl.lj_random(2000, seed=11, n_types=3)
    rng = np.random.default_rng(3)
    sig = rng.uniform(0.9, 1.1, s.n)
    sqe = np.sqrt(rng.uniform(0.5, 1.5, s.n))
    p = oracle.make_params(s.box, r_cut=2.5, r_switch=r_switch)
    _agree(*_both(s.x.astype(np.float64), np.zeros(s.n), sig, sqe, p))


def test_cells_take_exclusions_at_any_distance_and_listed_any_way():
    s = wl.lj_random(1500, seed=5)
    rng = np.random.default_rng(9)
    q = rng.uniform(-0.8, 0.8, s.n)
    x = s.x.astype(np.float64)
    # pairs far beyond r_c, listed one way, the other way, both ways and twice
    far = []
    while len(far) < 40:
        i, j = (int(v) for v in rng.integers(s.n, size=2))
        d = x[i] - x[j]
        d -= s.box * np.round(d / s.box)
        if i != j and np.linalg.norm(d) > 3.0:
            far.append((i, j))
    lists = [[] for _ in range(s.n)]
    for k, (i, j) in enumerate(far):
        if k % 4 == 0:
            lists[i].append(j)
        elif k % 4 == 1:
            lists[j].append(i)
        elif k % 4 == 2:
            lists[i].append(j)
            lists[j].append(i)
        else:
            lists[i] += [j, j]
    off = np.zeros(s.n + 1, np.int32)
    off[1:] = np.cumsum([len(v) for v in lists])
    idx = np.array([j for v in lists for j in v], np.int32)
    p = oracle.make_params(s.box, r_cut=2.5, alpha=1.1, ke=1.0)
    e0, f0, e1, f1 = _both(x, q, np.ones(s.n), np.ones(s.n), p, excl=(off, idx))
    assert e0[2] != 0.0
    _agree(e0, f0, e1, f1)


def test_cells_fall_back_to_all_pairs_for_open_and_small_boxes():
    s, _ = _water("ewald", n_mol=64)
    x = s.x.astype(np.float64)
    # 12.4 A box: two cells of 4.6 A per axis, below the three the cell route needs
    p = oracle.make_params(s.box, r_cut=4.6, alpha=0.8, ke=wl.KE_KJ_MOL_A)
    assert s.box[0] / 4.6 < 3.0
    _agree(*_both(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl))
    # exactly three cell edges of r_c: the rounding margin drops to two cells (all pairs)
    p3 = oracle.make_params(s.box, r_cut=s.box[0] / 3.0, alpha=0.8, ke=wl.KE_KJ_MOL_A)
    _agree(*_both(x, s.q, s.sigma, s.sqrt_eps, p3, excl=s.excl))
    po = oracle.make_params(s.box, r_cut=4.6, alpha=0.8, ke=wl.KE_KJ_MOL_A, periodic=False)
    _agree(*_both(x, s.q, s.sigma, s.sqrt_eps, po, excl=s.excl))


def test_cells_of_an_empty_and_a_single_atom_system():
    p = oracle.make_params(20.0, r_cut=2.5, alpha=0.5, ke=1.0)
    e, f = oracle.nonbonded_cells(np.zeros((0, 3)), np.zeros(0), np.zeros(0), np.zeros(0), p)
    assert f.shape == (0, 3) and np.all(e == 0.0)
    e, f = oracle.nonbonded_cells(np.array([[1.0, 2.0, 3.0]]), np.array([0.7]), np.ones(1), np.ones(1), p)
    e0, f0 = oracle.nonbonded(np.array([[1.0, 2.0, 3.0]]), np.array([0.7]), np.ones(1), np.ones(1), p)
    np.testing.assert_array_equal(f, f0)
    np.testing.assert_allclose(e, e0, rtol=1e-15)
