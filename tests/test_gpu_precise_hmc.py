"""HMC with precise end-state energies (NB_ENERGY_PRECISE in hmc_trajectory's terms): dH
against the FP64 oracle's velocity-Verlet proposal from the same start and normals, for
LJ replicas with the switch (the differentiable-HMC configuration) and for a small
water box with Ewald, PME and exclusions (the two-float pass's exclusion energy and the
FP64 reduction of the low parts), with the error of dH from FP32 energies beside it.

What is left of the dH error is the FP32 trajectory: each step rounds positions and
velocities, and every rounding dx moves H by F.dx, a non-Hamiltonian perturbation that the
FP64 trajectory does not have.  For the water box the FP32 energies are the larger part
(measured 1.7e-2 against 2.5e-3 with precise energies); for the LJ replicas the trajectory
already dominates (1.0e-3 either way).  The backward pass with the same terms recomputes
the forward trajectory with the same kernels; its gradients agree with those of a pass
without the flag to the FP32 rounding of the two end-state force evaluations."""
import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from oracle import pme as opme
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu_dh(systems, xi, w, dt, L, kT, terms, ckpt_every=0, u=None):
    R = len(systems)
    n = sum(s.n for s in systems)
    x0 = torch.cat([torch.from_numpy(nbcore.pack_xq(s.x, s.q)) for s in systems]).cuda()
    x1 = torch.empty_like(x0)
    st = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    u = np.zeros(R) if u is None else u
    ck = None
    if ckpt_every:
        ck = torch.empty(nbcore.ckpt_size(n, L, ckpt_every), dtype=torch.float32, device="cuda")
    with nbcore.Handle(systems) as h:
        h.hmc_trajectory(x0, x1, torch.from_numpy(w).cuda(), torch.from_numpy(dt).cuda(), L, kT,
                         torch.from_numpy(xi.reshape(-1, 3)).cuda(), torch.from_numpy(u).cuda(), st, ck,
                         ckpt_every, terms=terms)
        h.check()
        grads = None
        if ckpt_every:
            g_dt = torch.zeros(R, dtype=torch.float64, device="cuda")
            g_w = torch.zeros(n, dtype=torch.float32, device="cuda")
            ga = torch.ones(R, dtype=torch.float64, device="cuda")
            gj = torch.ones(R, dtype=torch.float64, device="cuda")
            h.hmc_trajectory_backward(x0, torch.from_numpy(w).cuda(), torch.from_numpy(dt).cuda(), L, kT,
                                      torch.from_numpy(xi.reshape(-1, 3)).cuda(), ck, ckpt_every, st, ga, gj,
                                      g_dt, g_w, terms=terms)
            h.check()
            grads = (g_dt.cpu().numpy(), g_w.cpu().numpy())
    return st.cpu().numpy(), grads


def test_lj_replicas_precise_dh():
    R, L, n = 2, 32, 2048
    reps = []
    for r in range(R):
        s = wl.lj_random(n, seed=100 + r, n_types=2)
        s.r_switch = 2.2
        reps.append(s)
    xi, _ = wl.hmc_randoms(R, n, seed=5)
    w = np.ones(R * n, np.float32)
    dt = np.full(R, 0.005, np.float32)
    stp, gp = _gpu_dh(reps, xi, w, dt, L, 1.0, nbcore.NB_TERM_LJ | nbcore.NB_ENERGY_PRECISE, ckpt_every=8)
    st32, g32 = _gpu_dh(reps, xi, w, dt, L, 1.0, nbcore.NB_TERM_LJ, ckpt_every=8)
    for r, s in enumerate(reps):
        p = oracle.make_params(s.box, r_cut=s.r_cut, r_switch=s.r_switch)

        def fe(x, s=s, p=p):
            e, f = oracle.nonbonded_cells(x, s.q, s.sigma, s.sqrt_eps, p)
            return f, float(e[0])
        o = odyn.hmc_proposal(s.x.astype(np.float64), xi[r].astype(np.float64), w[r * n:(r + 1) * n].astype(np.float64),
                              float(dt[r]), L, 1.0, fe, s.box)
        err_p, err_32 = abs(stp[r, 0] - o["dH"]), abs(st32[r, 0] - o["dH"])
        print("replica %d: dH %.6f, error precise %.2e, FP32 %.2e (energy scale %.0f)"
              % (r, o["dH"], err_p, err_32, abs(o["U0"]) + o["K0"]))
        scale = abs(o["U0"]) + o["K0"]
        assert err_p <= 2e-7 * scale, (r, stp[r, 0], o["dH"])
        assert abs(stp[r, 0] - st32[r, 0]) <= 2e-7 * scale
    # gradients through the precise forward: the end-state forces come from the energy-free
    # kernel, whose FP32 rounding differs (measured: 1.6e-4 of the largest component), far
    # inside the 2e-3 of the gradient checks against central differences
    for a, b in zip(gp, g32):
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max(), (np.abs(a - b).max(), np.abs(b).max())


def test_water_precise_dh_with_pme_and_exclusions():
    s = wl.water_box(n_side=8, L=24.84, seed=9, pme_grid=24)
    L_steps, kT = 10, 2.494  # kJ/mol at 300 K
    xi, _ = wl.hmc_randoms(1, s.n, seed=11)
    w = (1.0 / s.mass).astype(np.float32)
    dt = np.full(1, 0.0005, np.float32)  # ps
    terms = nbcore.NB_TERM_ALL
    stp, _ = _gpu_dh([s], xi, w, dt, L_steps, kT, terms | nbcore.NB_ENERGY_PRECISE)
    st32, _ = _gpu_dh([s], xi, w, dt, L_steps, kT, terms)
    p = oracle_params(s)

    def fe(x):
        e, f = oracle.nonbonded_cells(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
        Ep, Fp = opme.pme(x, s.q.astype(np.float64), s.box, s.alpha, s.ke, s.pme_grid)
        return f + Fp, float(np.sum(e)) + Ep
    o = odyn.hmc_proposal(s.x.astype(np.float64), xi[0].astype(np.float64), w.astype(np.float64), float(dt[0]),
                          L_steps, kT, fe, s.box)
    err_p, err_32 = abs(stp[0, 0] - o["dH"]), abs(st32[0, 0] - o["dH"])
    print("water: dH %.6f, error precise %.2e, FP32 %.2e (energy scale %.0f)"
          % (o["dH"], err_p, err_32, abs(o["U0"]) + o["K0"]))
    assert err_p <= 1e-6 * (abs(o["U0"]) + o["K0"]), (stp[0, 0], o["dH"])
    assert err_p <= 0.5 * err_32, (err_p, err_32)
