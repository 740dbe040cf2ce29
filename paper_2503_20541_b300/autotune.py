"""Autotuner for the handle options of a set of systems: cell size, stencil tile and
thread blocks per cell of the list build.

The first two knobs trade work against occupancy: cells of edge r_nl/2 (cell_div 2)
test ~1.7x fewer stencil candidates than cells of edge r_nl but give more, smaller
blocks; a smaller shared-memory stencil tile raises the number of resident blocks per SM
but sends the densest cells through several tiles.  The third splits a cell's atoms over
several blocks of the list build (results do not depend on it): more blocks fill the
GPU when cells are few, fewer keep the candidate staging of a cell in one block.  The
tuner builds one handle per candidate option set, times a few force evaluations of the
actual systems with CUDA events (list rebuilt every evaluation, so both the build and the
pair kernels count) and keeps the fastest: first over cell size and tile, then over the
blocks per cell of the winner.  Option sets that the systems cannot take (a box too small
for the finer cells) are skipped.
"""
import math


def auto_cell_div(s):
    """The library's default cell size for one system (cell_div 0): cells of edge r_nl/2
    when there are >= 5 of them along every axis and >= 64 atoms per r_nl^3, else r_nl."""
    box = [float(b) for b in (s.box if hasattr(s.box, "__len__") else [s.box] * 3)]
    r_nl = float(s.r_cut) + float(s.r_skin)
    dense = s.n / (box[0] * box[1] * box[2]) * r_nl ** 3 >= 64.0
    return 2 if dense and all(math.floor(L * 2.0 / r_nl) >= 5 for L in box) else 1


def candidate_options(systems):
    """Option sets worth timing for these systems: both cell sizes for all systems, each
    with the automatic tile and a tile about 25% smaller (a multiple of 64, >= 256), and,
    when the systems would take different cell sizes, the per-system default (cell_div 0)."""
    out = []
    if len({auto_cell_div(s) for s in systems}) > 1:
        out.append(dict(cell_div=0))
    for cd in (1, 2):
        base = dict(cell_div=cd)
        out.append(base)
        t = expected_stencil(systems, cd)
        small = int(max(256, 64 * math.floor(0.75 * (t + 3.0 * math.sqrt(t) + 96.0) / 64.0)))
        if small < 4096:
            out.append(dict(cell_div=cd, stencil_tile=small))
    return out


def refine_options(best, splits=(1, 2, 4)):
    """Second stage: the winning option set with each explicit number of list-build blocks
    per cell (the winner itself was timed with the automatic choice)."""
    out = []
    for b in splits:
        if best.get("blocks_per_cell", 0) != b:
            out.append(dict(best, blocks_per_cell=b))
    return out


def expected_stencil(systems, cell_div):
    """Largest expected stencil candidate count over the systems (density x volume of
    the (2 cell_div + 1)^3 cells around a cell, fewer when an axis has fewer cells)."""
    best = 0.0
    for s in systems:
        box = [float(b) for b in (s.box if hasattr(s.box, "__len__") else [s.box] * 3)]
        r_nl = float(s.r_cut) + float(s.r_skin)
        v = s.n / (box[0] * box[1] * box[2])
        for L in box:
            nc = max(1, int(math.floor(L * cell_div / r_nl)))
            v *= min(nc, 2 * cell_div + 1) * L / nc
        best = max(best, v)
    return best


def choose(timings):
    """The option set with the smallest time; ``timings`` is a list of (options, ms)
    with ms None for option sets that failed.  Ties keep the earlier candidate."""
    best, best_ms = None, float("inf")
    for opts, ms in timings:
        if ms is not None and ms < best_ms:
            best, best_ms = opts, ms
    if best is None:
        raise RuntimeError("no candidate option set could be run")
    return best


def autotune(systems, xq, candidates=None, evals=5, warmup=2, make_handle=None, timer=None, refine=True):
    """Time each candidate on ``systems`` (positions ``xq``, a device tensor), then (with
    ``refine``) the blocks-per-cell variants of the fastest, and return
    (best options, [(options, ms or None), ...]).

    ``make_handle(systems, **opts)`` and ``timer(handle, xq, evals, warmup)`` default to
    libnbcore handles and CUDA-event timing; they are parameters so that the selection
    logic can be exercised without a GPU.
    """
    if candidates is None:
        candidates = candidate_options(systems)
    if make_handle is None:
        from . import nbcore

        def make_handle(systems, **opts):
            return nbcore.Handle(systems, **opts)
    if timer is None:
        timer = _event_timer
    results = []

    def run(option_sets):
        for opts in option_sets:
            try:
                h = make_handle(systems, **opts)
            except Exception:  # e.g. a box too small for the finer cells
                results.append((opts, None))
                continue
            try:
                results.append((opts, timer(h, xq, evals, warmup)))
            finally:
                h.close()

    run(candidates)
    if refine:
        run(refine_options(choose(results)))
    return choose(results), results


def _event_timer(h, xq, evals, warmup):
    import torch
    n = xq.shape[0]
    f = torch.empty((n, 3), dtype=torch.float32, device=xq.device)
    e = torch.empty((h.n_sys, 6), dtype=torch.float64, device=xq.device)
    for _ in range(warmup):
        h.nonbonded_forces(xq, f, e, force_rebuild=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(evals):
        h.nonbonded_forces(xq, f, e, force_rebuild=True)
    b.record()
    torch.cuda.synchronize()
    h.check()
    return a.elapsed_time(b) / evals
