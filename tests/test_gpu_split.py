"""Several thread blocks per cell of the list build (nb_options.blocks_per_cell) change which
block handles an atom, never its arithmetic: forces, energies, pair sets and the force VJP
are bitwise those of one block per cell, for water with PME and with the reaction field,
plain and multi-tile stencils, and the automatic choice on a small box."""
import numpy as np
import pytest

from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import dev_xq, oracle_real_space, pair_set, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(s, terms, **opt):
    xq = dev_xq(s)
    rng = np.random.default_rng(3)
    lam = torch.from_numpy(rng.standard_normal((s.n, 3)).astype(np.float32)).cuda()
    with nbcore.Handle([s], **opt) as h:
        f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        e = torch.empty((1, 6), dtype=torch.float64, device="cuda")
        h.nonbonded_forces(xq, f, e, terms=terms, force_rebuild=True)
        pairs, n = h.nl_build(xq)
        gx = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        gq = torch.empty(s.n, dtype=torch.float32, device="cuda")
        h.nonbonded_force_vjp(xq, lam, gx, gq, terms=terms & (nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL))
        h.check()
        return f.cpu().numpy(), e.cpu().numpy(), pair_set(pairs[:n].cpu().numpy()), gx.cpu().numpy(), \
            gq.cpu().numpy()


@pytest.mark.parametrize("kind,tile", [("pme", 0), ("pme", 256), ("rf", 0)])
def test_blocks_per_cell_is_bitwise_neutral(kind, tile):
    if kind == "pme":
        s = wl.water_box(n_side=10, L=31.05, seed=5, pme_grid=32)
        terms = nbcore.NB_TERM_ALL
    else:
        s = wl.water_rf_density(1000, seed=8)
        terms = nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL
    ref = _run(s, terms, blocks_per_cell=1, stencil_tile=tile)
    for split in (3, 0):
        got = _run(s, terms, blocks_per_cell=split, stencil_tile=tile)
        for a, b in zip(ref, got):
            if isinstance(a, set):
                assert a == b
            else:
                assert np.array_equal(a, b), split


def test_small_box_uses_several_blocks_and_matches_oracle():
    s = wl.water_rf_density(1000, seed=9)  # 31 A box: 64 cells for 148 SMs
    with nbcore.Handle([s]) as h:
        assert h.blocks_per_cell()[0] > 1 and h.blocks_per_cell()[1] == 1
        f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        h.nonbonded_forces(dev_xq(s), f, None, terms=nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL)
        h.check()
    assert rel_rms(f.cpu().numpy().astype(np.float64), oracle_real_space(s)[1]) <= 1e-5


def test_blocks_per_cell_option_is_validated():
    s = wl.lj_random(500, seed=1)
    for bad in (-1, 33):
        with pytest.raises(nbcore.NbError) as ei:
            nbcore.Handle([s], blocks_per_cell=bad)
        assert ei.value.status == 1
