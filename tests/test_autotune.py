"""Host logic of the autotuner (no GPU): candidate sets, expected stencil sizes and the
selection, with a fake handle factory and a fake timer."""
import math

import pytest

from paper_2503_20541_b300 import autotune, workloads as wl


def test_expected_stencil_matches_density_times_volume():
    s = wl.lj_random(32000, seed=1)
    r_nl = s.r_cut + s.r_skin
    L = float(s.box[0])
    for cd in (1, 2):
        nc = math.floor(L * cd / r_nl)
        want = s.n / L ** 3 * ((2 * cd + 1) * L / nc) ** 3
        assert autotune.expected_stencil([s], cd) == pytest.approx(want, rel=1e-12)
    # an axis with fewer than 2 cd + 1 cells contributes its whole length
    small = wl.lj_random(256, seed=2)
    assert autotune.expected_stencil([small], 1) == pytest.approx(small.n, rel=1e-12)


def test_candidates_cover_both_cell_sizes_with_valid_tiles():
    c = autotune.candidate_options([wl.water_box(n_side=8, L=24.84)])
    assert {o["cell_div"] for o in c} == {1, 2}
    for o in c:
        t = o.get("stencil_tile", 0)
        assert t == 0 or (256 <= t <= 4096 and t % 64 == 0)


def test_mixed_systems_add_the_per_system_cell_size():
    lj, water = wl.lj_random(700, seed=1), wl.water_box()
    assert (autotune.auto_cell_div(lj), autotune.auto_cell_div(water)) == (1, 2)
    assert dict(cell_div=0) in autotune.candidate_options([lj, water])
    assert dict(cell_div=0) not in autotune.candidate_options([water])


def test_autotune_picks_fastest_and_skips_failures():
    systems = [wl.lj_random(500, seed=3)]
    cands = [dict(cell_div=1), dict(cell_div=2), dict(cell_div=2, stencil_tile=512)]
    times = {(1, 0): 3.0, (2, 0): 2.0, (2, 512): 2.5}
    made, closed = [], []

    class FakeHandle:
        def __init__(self, opts):
            self.opts = opts

        def close(self):
            closed.append(self.opts)

    def make(systems, **opts):
        if opts == dict(cell_div=2):
            made.append(opts)
            return FakeHandle(opts)
        if opts.get("stencil_tile") == 512:
            raise RuntimeError("box too small")
        made.append(opts)
        return FakeHandle(opts)

    def timer(h, xq, evals, warmup):
        return times[(h.opts["cell_div"], h.opts.get("stencil_tile", 0))]

    best, table = autotune.autotune(systems, None, candidates=cands, make_handle=make, timer=timer, refine=False)
    assert best == dict(cell_div=2)
    assert [ms for _, ms in table] == [3.0, 2.0, None]
    assert len(closed) == len(made) == 2


def test_autotune_refines_blocks_per_cell_of_the_winner():
    systems = [wl.lj_random(500, seed=3)]
    cands = [dict(cell_div=1), dict(cell_div=2)]
    times = {(1, 0): 3.0, (2, 0): 2.0, (2, 1): 2.5, (2, 2): 1.5, (2, 4): 1.8}

    class FakeHandle:
        def __init__(self, opts):
            self.opts = opts

        def close(self):
            pass

    def timer(h, xq, evals, warmup):
        return times[(h.opts["cell_div"], h.opts.get("blocks_per_cell", 0))]

    best, table = autotune.autotune(systems, None, candidates=cands, make_handle=lambda s, **o: FakeHandle(o),
                                    timer=timer)
    # the second stage times blocks per cell 1, 2, 4 of the first stage's winner only
    assert [o for o, _ in table[2:]] == [dict(cell_div=2, blocks_per_cell=b) for b in (1, 2, 4)]
    assert best == dict(cell_div=2, blocks_per_cell=2)
    assert autotune.refine_options(dict(cell_div=1, blocks_per_cell=2)) == [
        dict(cell_div=1, blocks_per_cell=1), dict(cell_div=1, blocks_per_cell=4)]


def test_choose_raises_when_nothing_ran():
    with pytest.raises(RuntimeError):
        autotune.choose([(dict(cell_div=1), None)])
