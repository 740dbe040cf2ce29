"""Every atom at full size: libnbcore (through its C ABI) against the oracle's cell-list route.

The oracle's cell-list sums (pinned equal to its all-pairs definition in
test_oracle_cells.py) make element-by-element checks affordable at the sizes the
benchmark runs: every force of the 24,000-atom water box in the launch the benchmark
times (graph replays of the evaluation with the list rebuilt every step, and of the one
reusing it), every force of the 8.19M-atom LJ fluid, and every atom of every system of
the 256-system batch.

Bars: forces to relative RMS <= 1e-5 against FP64 and every atom's force error within
1e-3 of the RMS force; energies to 1e-6 relative, and sums that cancel (the pair energies
of small boxes) within that or three standard deviations of the random walk of per-pair
FP32 errors (ULP_DIR, ULP_LJ below), whichever is larger.  Pairs whose FP64 r^2 lies within
the FP32 band of r_c^2 have two correct answers (either side of the cutoff); each such pair
of an atom that is off the oracle takes the side that matches, and the bars apply after.
"""
import numpy as np
import pytest

import oracle
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import EPS32, band, dev_xq, oracle_params, oracle_pme, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F_TOL = 1e-5
F_ATOM_TOL = 1e-3
E_TOL = 1e-6
# Largest relative error of one FP32 pair energy, in ulp: the direct-space term
# ke q_i q_j erfc(alpha r)/r takes erfcf (at most 4 ulp, CUDA's documented bound), an
# approximate 1/r (2 ulp) and three rounded products; the LJ term (sigma/r)^12 raises a
# rounded (sigma/r)^2 to the sixth power (~12 ulp).  One ulp is at most 2 EPS32 relative.
ULP_DIR = 7.5
ULP_LJ = 13.0


def _oracle_cells(s):
    """(E_lj, E_dir, E_excl, E_self) and forces of the real-space terms, FP64 cell list."""
    return oracle.nonbonded_cells(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s),
                                  excl=s.excl)


def _band_partners(s, i):
    """Atom i's partners j whose FP64 r^2 lies within the FP32 band of r_c^2 (8 ulp, the
    band of the neighbour-set tests), excluded partners left out: (j, d_ij, r^2_ij)."""
    x = s.x.astype(np.float64)
    d = x[i] - x
    d -= s.box * np.round(d / s.box)
    r2 = np.einsum("ij,ij->i", d, d)
    rc = float(s.r_cut)
    near = np.nonzero(np.abs(r2 - rc * rc) <= band(rc))[0]
    ex = set()
    if s.excl_off is not None:
        ex = set(int(j) for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]])
    return [(int(j), d[j], float(r2[j])) for j in near if j != i and int(j) not in ex]


def _pair_terms(s, i, j, d, r2):
    """Force on i from j (f(r) d, f = -U'/r) and the pair's LJ and Ewald direct energies, FP64."""
    from scipy.special import erfc
    r = np.sqrt(r2)
    fr = w = t = 0.0
    eps = float(s.sqrt_eps[i]) * float(s.sqrt_eps[j])
    if eps != 0.0 and not (s.r_switch is not None and s.r_switch >= 0):  # a switch is 0 at r_c
        s6 = (0.5 * (float(s.sigma[i]) + float(s.sigma[j])) / r) ** 6
        w = 4.0 * eps * (s6 * s6 - s6)
        fr += 24.0 * eps * (2.0 * s6 * s6 - s6) / r2
    if s.ke and s.alpha:
        a, qq = float(s.alpha), float(s.ke) * float(s.q[i]) * float(s.q[j])
        t = qq * erfc(a * r) / r
        fr += qq * (erfc(a * r) / r + 2.0 * a / np.sqrt(np.pi) * np.exp(-a * a * r2)) / r2
    return fr * d, w, t


def _resolve_cutoff_pairs(f, fo, eo, s):
    """Where several results are correct: a pair whose FP64 r^2 lies within the FP32 band of
    r_c^2 may fall on either side of the FP32 cutoff test, and the unswitched LJ force is not
    zero at r_c (0.039 eps/sigma at 2.5 sigma).  For every atom off the oracle by more than
    1e-4 of the RMS force, each of its band pairs takes the side of the cutoff that matches
    the GPU better (forces on both atoms, and the energies); returns the adjusted oracle
    forces and energies and the number of pairs moved."""
    fo = fo.copy()
    eo = np.array(eo, dtype=np.float64)
    err = np.linalg.norm(f - fo, axis=1)
    rms = np.sqrt(np.mean(np.sum(fo * fo, axis=1)))
    odd = np.nonzero(err > 1e-4 * rms)[0]
    assert odd.size <= 1e-3 * s.n + 8, ("atoms off the oracle", odd.size)
    rc2 = float(s.r_cut) ** 2
    seen, moved = set(), 0
    for i in odd:
        for j, d, r2 in _band_partners(s, int(i)):
            key = (min(int(i), j), max(int(i), j))
            if key in seen:
                continue
            seen.add(key)
            F, w, t = _pair_terms(s, int(i), j, d, r2)
            sgn = -1.0 if r2 < rc2 else 1.0  # the other side: drop an included pair, add an excluded one
            ai, aj = fo[i] + sgn * F, fo[j] - sgn * F
            if np.sum((f[i] - ai) ** 2) + np.sum((f[j] - aj) ** 2) < \
                    np.sum((f[i] - fo[i]) ** 2) + np.sum((f[j] - fo[j]) ** 2):
                fo[i], fo[j] = ai, aj
                eo[0] += sgn * w
                eo[1] += sgn * t
                moved += 1
    return fo, eo, moved


def _check_forces(f, fo, what):
    assert rel_rms(f, fo) <= F_TOL, (what, rel_rms(f, fo))
    err = np.linalg.norm(f - fo, axis=1)
    rms = np.sqrt(np.mean(np.sum(fo * fo, axis=1)))
    i = int(np.argmax(err))
    assert err[i] <= F_ATOM_TOL * rms, (what, i, err[i], rms)


def _check(f, fo, e, eo, s, what):
    """Forces and energies of one system after the cutoff-band pairs are resolved."""
    fo, eo, _ = _resolve_cutoff_pairs(f, fo, eo, s)
    _check_forces(f, fo, what)
    _check_energies(e, eo, s, what)


def _pair_rounding_scales(s):
    """sqrt(sum W_ij^2) and sqrt(sum t_ij^2) over the unordered non-excluded pairs r < r_c:
    the LJ pair energies (Eq. lj, the switch where set) and the Ewald direct pair energies
    ke q_i q_j erfc(alpha r)/r.  Each FP32 pair term rounds at ~EPS32 of itself and the
    roundings of independent pairs add like a random walk."""
    from scipy.spatial import cKDTree
    from scipy.special import erfc
    x = np.mod(s.x.astype(np.float64), s.box)
    p = cKDTree(x, boxsize=s.box).query_pairs(float(s.r_cut), output_type="ndarray")
    if s.excl_off is not None and len(p):
        owner = np.repeat(np.arange(s.n, dtype=np.int64), np.diff(s.excl_off))
        other = s.excl_idx.astype(np.int64)
        ex = np.minimum(owner, other) * s.n + np.maximum(owner, other)
        key = np.minimum(p[:, 0], p[:, 1]).astype(np.int64) * s.n + np.maximum(p[:, 0], p[:, 1])
        p = p[~np.isin(key, ex)]
    if not len(p):
        return 0.0, 0.0
    d = x[p[:, 0]] - x[p[:, 1]]
    d -= s.box * np.round(d / s.box)
    r = np.sqrt(np.sum(d * d, axis=1))
    eps = s.sqrt_eps[p[:, 0]].astype(np.float64) * s.sqrt_eps[p[:, 1]]
    sg = 0.5 * (s.sigma[p[:, 0]].astype(np.float64) + s.sigma[p[:, 1]])
    w = 4.0 * eps * ((sg / r) ** 12 - (sg / r) ** 6)
    t = np.zeros_like(r)
    if s.ke and s.alpha:
        t = s.ke * s.q[p[:, 0]].astype(np.float64) * s.q[p[:, 1]] * erfc(s.alpha * r) / r
    return float(np.sqrt(np.sum(w * w))), float(np.sqrt(np.sum(t * t)))


def _check_energies(e, eo, s, what):
    scales = None
    for c, ulp in ((0, ULP_LJ), (1, ULP_DIR)):
        bound = max(E_TOL * abs(eo[c]), 1e-12)
        if abs(e[c] - eo[c]) > bound:
            # a cancelling sum: independent per-pair errors of at most `ulp` ulp add like a
            # random walk (three standard deviations of it)
            scales = _pair_rounding_scales(s) if scales is None else scales
            bound = max(bound, 3.0 * ulp * 2.0 * EPS32 * scales[c])
        assert abs(e[c] - eo[c]) <= bound, (what, c, e[c], eo[c], bound)
    for c in (2, 3):
        assert abs(e[c] - eo[c]) <= max(E_TOL * abs(eo[c]), 1e-12), (what, c, e[c], eo[c])


def test_water_24k_every_atom_in_the_bench_launch():
    """The 24,000-atom box as the benchmark runs it: a default handle, the evaluation
    with a forced list rebuild and the one reusing the list, each captured as a CUDA
    graph and replayed; every atom's force (real space + PME) against the oracle, the
    energies against the oracle's, and the list-reusing replay bitwise equal to the
    rebuilding one (same positions, same list)."""
    from paper_2503_20541_b300.graphs import CapturedStep
    s = wl.water_box()
    assert s.n == 24000
    xq = dev_xq(s)
    f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle([s]) as h:
        g_rebuild = CapturedStep(lambda: h.nonbonded_forces(xq, f, e, force_rebuild=True))
        g_reuse = CapturedStep(lambda: h.nonbonded_forces(xq, f, e, force_rebuild=False))
        for _ in range(3):
            g_rebuild.replay()
        torch.cuda.synchronize()
        h.check()
        f_rb, e_rb = f.cpu().numpy().astype(np.float64), e.cpu().numpy()[0].copy()
        f.zero_()
        e.zero_()
        for _ in range(3):
            g_reuse.replay()
        torch.cuda.synchronize()
        h.check()
        f_ru, e_ru = f.cpu().numpy().astype(np.float64), e.cpu().numpy()[0].copy()
        del g_rebuild, g_reuse
    assert np.array_equal(f_ru, f_rb)
    assert np.array_equal(e_ru, e_rb)
    eo, fo = _oracle_cells(s)
    Ep, Fp = oracle_pme(s)
    _check(f_rb, fo + Fp, e_rb, eo, s, "water 24k")
    assert abs(e_rb[4] - Ep) <= E_TOL * abs(Ep)


def test_lj_8m_every_atom():
    """The largest LJ sweep point: all 8.19M forces against the oracle's cell list, and
    the LJ energy."""
    s = wl.lj_random(8192000, seed=500 + 8192000 % 997, kT=1.0)
    xq = dev_xq(s)
    with nbcore.Handle([s]) as h:
        f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        e = torch.empty((1, 6), dtype=torch.float64, device="cuda")
        h.nonbonded_forces(xq, f, e, terms=nbcore.NB_TERM_LJ, force_rebuild=True)
        h.check()
        fg = f.cpu().numpy().astype(np.float64)
        eg = e.cpu().numpy()[0]
        del f, xq
    eo, fo = _oracle_cells(s)
    fo, eo, _ = _resolve_cutoff_pairs(fg, fo, eo, s)
    _check_forces(fg, fo, "lj 8.19M")
    assert abs(eg[0] - eo[0]) <= E_TOL * abs(eo[0]), (eg[0], eo[0])


def test_batched_256_every_system_every_atom():
    """The 256-system batch of the benchmark (1.54M atoms, LJ and water, per-system cell
    sizes): every atom of every system (real space + PME for water) against the oracle,
    and every system's energies: the FP32 energies within 1e-6 or their rounding floor, and
    the precise (two-float) energies of a second call within the flat 1e-6."""
    systems = wl.batched_mix(256)
    offs = np.cumsum([0] + [s.n for s in systems])
    xq = torch.cat([dev_xq(s) for s in systems])
    n = int(offs[-1])
    f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((256, 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle(systems) as h:
        h.nonbonded_forces(xq, f, e)
        h.check()
        fb = f.cpu().numpy().astype(np.float64)
        eb = e.cpu().numpy()
        h.nonbonded_forces(xq, f, e, precise=True)
        h.check()
        ebp = e.cpu().numpy()
    problems = []
    worst = 0.0
    for k, s in enumerate(systems):
        try:
            eo, fo = _oracle_cells(s)
            if s.pme_grid and s.pme_grid[0] > 0:
                Ep, Fp = oracle_pme(s)
                fo = fo + Fp
                assert abs(eb[k, 4] - Ep) <= E_TOL * abs(Ep), ("system %d" % k, 4, eb[k, 4], Ep)
            eo_exact = np.array(eo, dtype=np.float64)
            fo, eo, _ = _resolve_cutoff_pairs(fb[offs[k]:offs[k + 1]], fo, eo, s)
            _check_forces(fb[offs[k]:offs[k + 1]], fo, "system %d" % k)
            _check_energies(eb[k], eo, s, "system %d" % k)
            # the precise pass decides r < r_c on its two-float r^2: the oracle's own pair set
            for c in range(4):
                err = abs(ebp[k, c] - eo_exact[c])
                worst = max(worst, err / abs(eo_exact[c]) if eo_exact[c] else 0.0)
                assert err <= max(E_TOL * abs(eo_exact[c]), 1e-12), ("system %d precise" % k, c, ebp[k, c],
                                                                     eo_exact[c])
        except AssertionError as err:
            problems.append(str(err).splitlines()[0][:200])
    print("batched 256: largest relative error of the precise energies %.1e" % worst)
    assert not problems, problems


def test_force_vjp_water_24k_every_atom():
    """The force vector-Jacobian product on the full 24,000-atom box: (dF/dx)^T lam and the
    gradients of lam.F with respect to the charges, sigma and sqrt(eps) of every atom,
    real space (LJ + Ewald direct + exclusion correction) against the FP64 oracle (all
    pairs), and with the PME part added against the oracle's FP64 PME VJP on the same
    mesh (the reciprocal part alone too, as it is small next to real space)."""
    from oracle import pme as opme
    s = wl.water_box()
    rng = np.random.default_rng(24)
    lam = rng.standard_normal((s.n, 3)).astype(np.float32)
    xq = dev_xq(s)
    lam_d = torch.from_numpy(lam).cuda()
    out = {}
    with nbcore.Handle([s]) as h:
        for name, terms in (("real", nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL), ("all", nbcore.NB_TERM_ALL),
                            ("pme", nbcore.NB_TERM_PME)):
            g = [torch.empty((s.n, 3), dtype=torch.float32, device="cuda")] + \
                [torch.empty(s.n, dtype=torch.float32, device="cuda") for _ in range(3)]
            h.nonbonded_force_vjp(xq, lam_d, g[0], g[1], g[2], g[3], terms=terms)
            h.check()
            out[name] = [t.cpu().numpy().astype(np.float64) for t in g]
    x64 = s.x.astype(np.float64)
    gxo, gqo, gso, geo = oracle.force_vjp(x64, s.q, s.sigma, s.sqrt_eps, oracle_params(s), lam, excl=s.excl)
    gxk, gqk = opme.pme_force_vjp(x64, s.q.astype(np.float64), s.box, s.alpha, s.ke, s.pme_grid,
                                  lam.astype(np.float64))
    gx, gq, gs, ge = out["real"]
    o = s.sqrt_eps > 0  # LJ parameters exist on oxygen only
    assert rel_rms(gx, gxo) <= F_TOL
    assert rel_rms(gq, gqo) <= F_TOL
    assert rel_rms(gs[o], gso[o]) <= F_TOL
    assert rel_rms(ge, geo) <= F_TOL
    err = np.linalg.norm(gx - gxo, axis=1)
    rms = np.sqrt(np.mean(np.sum(gxo * gxo, axis=1)))
    assert err.max() <= F_ATOM_TOL * rms, (int(np.argmax(err)), err.max(), rms)
    assert rel_rms(out["all"][0], gxo + gxk) <= F_TOL
    assert rel_rms(out["all"][1], gqo + gqk) <= F_TOL
    assert rel_rms(out["pme"][0], gxk) <= 1e-4
    assert rel_rms(out["pme"][1], gqk) <= 1e-4
