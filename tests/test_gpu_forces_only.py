"""GPU parity of the energy-free force evaluation (nonbonded_forces with energies NULL).

Without energies the real-space pass runs another instantiation of the pair kernel: erfc
from a fitted polynomial that shares exp(-x^2) with the Gaussian term, 1/r^2 as the
square of 1/r, and a four-value warp reduction.  Its forces meet the same bar as the
energy kernel's (relative RMS <= 1e-5 against FP64, Sec. 2.1.2) on a list just built
(front entries taken without the cut-off test) and on a kept list (every entry tested),
on every image mode of the list (plain, per-entry image codes, folded axes), and with
LJ, Ewald direct + exclusions, the reaction field and PME.
"""
import numpy as np
import pytest

from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import dev_xq, oracle_pme, oracle_real_space, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F_TOL = 1e-5
LJ = nbcore.NB_TERM_LJ
LJC = nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL


def _pair_forces(h, s, terms, energies, rebuild):
    f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((1, 6), dtype=torch.float64, device="cuda") if energies else None
    h.nonbonded_forces(dev_xq(s), f, e, terms=terms, force_rebuild=rebuild)
    h.check()
    return f.cpu().numpy().astype(np.float64)


def _check(s, terms, f_ref):
    with nbcore.Handle([s]) as h:
        f_fresh = _pair_forces(h, s, terms, False, True)
        assert h.rebuild_count() >= 1
        c0 = h.rebuild_count()
        # same positions, list kept: the load clears the just-built mark
        f_kept = _pair_forces(h, s, terms, False, False)
        assert h.rebuild_count() == c0
        f_en = _pair_forces(h, s, terms, True, False)
    assert rel_rms(f_fresh, f_ref) <= F_TOL
    assert rel_rms(f_kept, f_ref) <= F_TOL
    # the two kernels differ by FP32 rounding only
    assert rel_rms(f_fresh, f_en) <= 1e-6
    assert rel_rms(f_kept, f_en) <= 1e-6
    # the fixed-point sums are order-free: the fresh and kept walks give the same forces
    # up to the roundings of the pairs they evaluate alike
    assert rel_rms(f_fresh, f_kept) <= 1e-6


@pytest.mark.parametrize("switch", [False, True])
def test_lj_fcc(switch):
    s = wl.lj_fcc()
    rng = np.random.default_rng(11)
    x = s.x.astype(np.float64) + rng.uniform(-0.05, 0.05, s.x.shape)
    s.x = (x - s.box * np.floor(x / s.box)).astype(np.float32)
    if switch:
        s.r_switch = 2.2
    _, fo = oracle_real_space(s)
    _check(s, LJ, fo)


def test_water_ewald_real_space():
    s = wl.water_box(n_side=10, L=31.05, seed=5, pme_grid=32)
    _, fo = oracle_real_space(s)
    _check(s, LJC, fo)


def test_water_slab_image_codes():
    # cells of r_nl/2: five along the 31.05 A axes (image codes per entry), four along
    # the 24.8 A axis (folded per pair)
    s = wl.water_slab()
    _, fo = oracle_real_space(s)
    _check(s, LJC, fo)


def test_small_box_folded_axes():
    s = wl.lj_random(256, seed=17)
    _, fo = oracle_real_space(s)
    _check(s, LJ, fo)


def test_water_reaction_field():
    s = wl.water_rf_density(1000, seed=21)
    _, fo = oracle_real_space(s)
    _check(s, LJC, fo)


def test_water_with_pme():
    s = wl.water_box(n_side=10, L=31.05, seed=5, pme_grid=32)
    _, fr = oracle_real_space(s)
    _, fk = oracle_pme(s)
    _check(s, nbcore.NB_TERM_ALL, fr + fk)
