"""FP64 velocity Verlet, HMC proposal and ESJD loss (Sec. 2.2.1 and Sec. 4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

``force_energy(x) -> (F (n,3), U)`` is any oracle force routine (usually the
all-pairs ``oracle.nonbonded`` plus, for charged systems, ``oracle.pme``).
"""
import numpy as np


def kinetic(v, inv_mass):
    """T(v) = 1/2 sum_i m_i |v_i|^2."""
    return 0.5 * float(np.sum(np.sum(v * v, axis=1) / inv_mass))


def velocity_verlet(x, v, inv_mass, dt, n_steps, force_energy):
    """Velocity Verlet, steps 1, 2, 4, 5 of the MD loop of Sec. 2.2.1.

    1. v(t + dt/2) = v(t) + a(t) dt/2     2. x(t + dt) = x(t) + v(t + dt/2) dt
    4. a(t + dt) from the forces          5. v(t + dt) = v(t + dt/2) + a(t + dt) dt/2
    Returns final (x, v) and the potential / kinetic energy at every integer step.
    """
    w = np.asarray(inv_mass, dtype=np.float64)[:, None]
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    F, U = force_energy(x)
    Us, Ks = [U], [kinetic(v, w[:, 0])]
    for _ in range(n_steps):
        v = v + 0.5 * dt * w * F
        x = x + dt * v
        F, U = force_energy(x)
        v = v + 0.5 * dt * w * F
        Us.append(U)
        Ks.append(kinetic(v, w[:, 0]))
    return x, v, np.array(Us), np.array(Ks)


def min_image(d, box):
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    return d - L * np.round(d / L)


def hmc_proposal(x0, xi, inv_mass, dt, n_leap, kT, force_energy, box):
    """One HMC proposal (Sec. 4).

    Velocities are drawn from Maxwell-Boltzmann, v0 = sqrt(kT/m) xi with xi the
    standard-normal deviates passed in; L velocity-Verlet steps give (x', v');
    E = U + T; the Metropolis-Hastings acceptance probability is
    alpha = min(1, exp(-[E(x', v') - E(x, v)]/kT)).  Also returns the squared
    jump |x' - x|^2 (minimum image), the observable O = x of the ESJD loss.
    """
    w = np.asarray(inv_mass, dtype=np.float64)
    v0 = np.sqrt(kT * w)[:, None] * np.asarray(xi, dtype=np.float64)
    xL, vL, Us, Ks = velocity_verlet(x0, v0, w, dt, n_leap, force_energy)
    dH = (Us[-1] + Ks[-1]) - (Us[0] + Ks[0])
    alpha = min(1.0, float(np.exp(-dH / kT)))
    jump = float(np.sum(min_image(xL - np.asarray(x0), box) ** 2))
    return {"x": xL, "v": vL, "dH": float(dH), "alpha": alpha, "jump": jump,
            "U0": float(Us[0]), "U1": float(Us[-1]), "K0": float(Ks[0]), "K1": float(Ks[-1])}


def esjd_loss(alphas, jumps, n_leap):
    """Eq. (loss) per force evaluation: (1/R) sum_i alpha_i |O'_i - O_i|^2 / L."""
    a = np.asarray(alphas, dtype=np.float64)
    j = np.asarray(jumps, dtype=np.float64)
    return float(np.mean(a * j) / n_leap)


def masses_from_logits(logits, types, m_total):
    """Per-type mass repartitioning with the total mass fixed (Sec. 4):
    m_t = M s_t / sum_t n_t s_t, s_t = exp(logit_t)."""
    s = np.exp(np.asarray(logits, dtype=np.float64))
    types = np.asarray(types)
    counts = np.bincount(types, minlength=s.size).astype(np.float64)
    mt = m_total * s / float(np.sum(counts * s))
    return mt[types]


def step_from_folded_normal(mu, eps, rel_sigma=0.01):
    """Reparameterised folded-normal draw dt = |mu + sigma eps|, sigma = 0.01 mu (Sec. 4)."""
    return abs(mu + rel_sigma * mu * eps)
