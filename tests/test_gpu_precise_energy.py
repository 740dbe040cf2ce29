"""Precise energies (NB_ENERGY_PRECISE) through the C ABI against the FP64 oracle.

The FP32 pair energies leave relative errors above 1e-6 on boxes whose pair terms cancel
10^3-10^4-fold in the sum (neutral water with Ewald or the reaction field); the precise
evaluation recomputes the real-space and exclusion energies in two-float arithmetic.  Here
every case that the FP32 energies miss is held to the flat 1e-6 relative bar, per energy
component: the reaction-field water box of 1,800 atoms, the smallest water and LJ systems
of the 256-system batch in one batched handle, the orthorhombic water slab, the 24,000-atom
box, kept and pruned lists after the atoms have moved, and an open water cluster without
periodic images.  The forces of a precise call
are bitwise those of the energy-free call, and the two-float erfc itself is checked on the
device against the FP64 erfc."""
import numpy as np
import pytest
from scipy.special import erfc as erfc64

import oracle
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import dev_xq, oracle_params, oracle_pme, oracle_real_space, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 1e-6
F_TOL = 1e-5


def _eval(h, xq, n, terms=nbcore.NB_TERM_ALL, precise=True, force_rebuild=False):
    f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((h.n_sys, 6), dtype=torch.float64, device="cuda")
    h.nonbonded_forces(xq, f, e, terms=terms, precise=precise, force_rebuild=force_rebuild)
    h.check()
    return f.cpu().numpy().astype(np.float64), e.cpu().numpy()


def _check_energies(e, eo, what, comps=(0, 1, 2, 3)):
    for c in comps:
        assert abs(e[c] - eo[c]) <= max(E_TOL * abs(eo[c]), 1e-12), (what, c, e[c], eo[c],
                                                                     abs(e[c] - eo[c]) / max(abs(eo[c]), 1e-300))


def test_erfc_df_against_fp64():
    rng = np.random.default_rng(3)
    xh = np.concatenate([np.linspace(0.0, 8.0, 400_001), rng.uniform(0.0, 6.0, 100_000)]).astype(np.float32)
    # a low part of up to half an ulp of x_hi, as alpha r in two-float carries
    xl = (rng.uniform(-0.5, 0.5, xh.size) * np.spacing(xh)).astype(np.float32)
    hi, lo = nbcore.erfc_df_eval(torch.from_numpy(xh).cuda(), torch.from_numpy(xl).cuda())
    got = hi.cpu().numpy().astype(np.float64) + lo.cpu().numpy().astype(np.float64)
    x = xh.astype(np.float64) + xl.astype(np.float64)
    ref = erfc64(x)
    rel = np.abs(got - ref) / ref
    table = xh < 6.0
    print("two-float erfc: max relative error %.2e on [0, 6), %.2e beyond"
          % (rel[table].max(), rel[~table].max()))
    # two-float roundings of the Horner steps, largest where the series alternates (x ~ 6),
    # and the FP32 first-order term in x_lo (a host emulation of the same arithmetic with
    # a correctly rounded exp: 1.9e-14 for x < 1, 1.9e-13 for x < 3, 7.7e-13 below 6)
    assert rel[xh < 3.0].max() <= 4e-13
    assert rel[table].max() <= 1.5e-12
    # past the table CUDA's erfcf (measured 6.9e-6 relative at 6 <= x <= 8, where erfc < 2.2e-17)
    assert rel[~table].max() <= 2e-5
    assert got[0] == 1.0 or abs(got[0] - 1.0) <= 1e-15


def test_erfc_df_handles_empty_and_bad_arguments():
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    hi, lo = nbcore.erfc_df_eval(e, e)
    assert hi.numel() == 0 and lo.numel() == 0
    lib = nbcore.load()
    assert lib.nb_erfc_df_eval(None, None, None, None, -1, None) == 1


def test_reaction_field_water_1800_precise():
    s = wl.water_rf_density(600, seed=3)  # the FP32 E_RF is 8e-6 off here
    terms = nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL
    with nbcore.Handle([s]) as h:
        xq = dev_xq(s)
        f, e = _eval(h, xq, s.n, terms=terms)
        f0, _ = _eval(h, xq, s.n, terms=terms, precise=False)
        fn = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        h.nonbonded_forces(xq, fn, None, terms=terms)
        h.check()
    eo, fo = oracle_real_space(s)
    _check_energies(e[0], eo, "rf water 1800", comps=(0, 1))
    assert e[0, 2] == 0.0 and e[0, 3] == 0.0
    # forces: the energy-free kernel's, bit for bit
    assert np.array_equal(f, fn.cpu().numpy().astype(np.float64))
    assert rel_rms(f, fo) <= F_TOL
    assert rel_rms(f, f0) <= 1e-6


def test_smallest_batch_systems_precise_batched():
    """The five smallest water (1,149-1,227 atoms, Ewald + PME) and five smallest LJ systems
    (500-548 atoms) of the 256-system batch, in one batched handle."""
    full = wl.batched_mix(256)
    pick = [201, 71, 193, 175, 229, 224, 28, 138, 242, 64]
    systems = [full[k] for k in pick]
    assert all(systems[k].ke for k in range(5)) and not any(systems[k].ke for k in range(5, 10))
    xq = torch.cat([dev_xq(s) for s in systems])
    n = int(xq.shape[0])
    offs = np.cumsum([0] + [s.n for s in systems])
    with nbcore.Handle(systems) as h:
        f, e = _eval(h, xq, n)
    problems = []
    for k, s in enumerate(systems):
        eo, fo = oracle_real_space(s)
        if s.ke:
            Ep, Fp = oracle_pme(s)
            fo = fo + Fp
            if abs(e[k, 4] - Ep) > E_TOL * abs(Ep):
                problems.append(("rec", pick[k], e[k, 4], Ep))
        try:
            _check_energies(e[k], eo, "system %d" % pick[k])
        except AssertionError as err:
            problems.append(str(err)[:200])
        if rel_rms(f[offs[k]:offs[k + 1]], fo) > F_TOL:
            problems.append(("forces", pick[k]))
    assert not problems, problems


def test_orthorhombic_water_slab_precise():
    s = wl.water_slab(seed=7)  # the FP32 E_dir is 1.6e-6 off here
    with nbcore.Handle([s]) as h:
        f, e = _eval(h, dev_xq(s), s.n)
    eo, fo = oracle_real_space(s)
    Ep, Fp = oracle_pme(s)
    _check_energies(e[0], eo, "orthorhombic slab")
    assert abs(e[0, 4] - Ep) <= E_TOL * abs(Ep)
    assert rel_rms(f, fo + Fp) <= F_TOL


def test_water_24k_precise_and_fp32_energies():
    """The benchmark's box: precise energies at 1e-6 per component, the FP32 energies of the
    same call sequence within the same bar here (the box is large enough), and the PME and
    self energies identical between the two modes."""
    s = wl.water_box()
    xq = dev_xq(s)
    with nbcore.Handle([s]) as h:
        f, e = _eval(h, xq, s.n, force_rebuild=True)
        f0, e0 = _eval(h, xq, s.n, precise=False)
    eo = oracle.nonbonded_cells(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s),
                                excl=s.excl)[0]
    _check_energies(e[0], eo, "water 24k precise")
    assert e[0, 3] == e0[0, 3] and e[0, 4] == e0[0, 4]
    print("water 24k relative energy error, precise / FP32: "
          + ", ".join("%.1e / %.1e" % (abs(e[0, c] - eo[c]) / abs(eo[c]), abs(e0[0, c] - eo[c]) / abs(eo[c]))
                      for c in range(3)))


@pytest.mark.parametrize("prune", [0.0, -1.0])
def test_moved_atoms_kept_and_pruned_lists_precise(prune):
    """After the build the atoms move (less than r_skin/2: the list is kept; with pruning on,
    past half the prune skin too, so the rows are re-partitioned): the energies of each
    evaluation at 1e-6 against the oracle at the moved positions, the pair set being the one
    the FP32 cut-off test of the kept list gives."""
    s = wl.water_box(n_side=10, L=31.05, seed=5, pme_grid=32)
    rng = np.random.default_rng(9)
    with nbcore.Handle([s], prune_skin=prune) as h:
        for k, a in enumerate((0.0, 0.1, 0.5)):
            x = (s.x.astype(np.float64) + rng.uniform(-a, a, s.x.shape)).astype(np.float32)
            xq = torch.from_numpy(nbcore.pack_xq(x, s.q)).cuda()
            f, e = _eval(h, xq, s.n)
            eo, fo = oracle_real_space(s, x.astype(np.float64))
            Ep, Fp = oracle_pme(s, x.astype(np.float64))
            _check_energies(e[0], eo, "moved %d prune %g" % (k, prune))
            assert abs(e[0, 4] - Ep) <= E_TOL * abs(Ep)
            assert rel_rms(f, fo + Fp) <= F_TOL
        assert h.rebuild_count() == 1


def test_open_water_cluster_precise():
    """A water cluster without periodic images (no PME): LJ, Ewald direct and exclusion
    energies at 1e-6, the differences taken as plain differences of the caller's positions."""
    s = wl.water_box(n_side=6, L=18.63, seed=4, pme_grid=24)
    s.periodic = False
    s.pme_grid = None
    terms = nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL
    with nbcore.Handle([s]) as h:
        f, e = _eval(h, dev_xq(s), s.n, terms=terms)
    eo, fo = oracle_real_space(s)
    _check_energies(e[0], eo, "open cluster")
    assert rel_rms(f, fo) <= F_TOL
