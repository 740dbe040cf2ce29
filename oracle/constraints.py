"""FP64 reference of rigid-water constraints and Langevin dynamics (Sec. 2.2.1: the MD
loop's position and velocity constraint steps, SETTLE for three-site water, and the
Langevin integrator).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The constraint steps are written as their defining equations, solved directly, not by
SETTLE's geometric construction:
  * positions (SHAKE equations): given constrained positions x_old and unconstrained
    x_new, find multipliers lam_k of the constraints s_k = |x_i - x_j|^2 - d_k^2 with
    x_i = x_new_i + (1/m_i) sum_k lam_k grad_i s_k(x_old) and s_k(x) = 0 for all k; one
    molecule's three equations are solved by Newton's method to rounding level.  SETTLE
    computes the same solution in closed form.
  * velocities (RATTLE): v_i = v_i + (1/m_i) sum_k mu_k grad_i s_k(x) with
    d/dt s_k = 0, a 3x3 linear system per molecule.

Langevin dynamics (reading: the paper cites a unified thermostat scheme and prints no
equations; the scheme taken is its "middle" form in leapfrog variables, velocities at
half steps), one step from x_n, v_{n-1/2} and F(x_n):
  v <- v + dt F / m;  constrain v (RATTLE at x_n)
  x' = x_n + dt/2 v;  v <- c1 v + c2 sqrt(kT/m) xi,  c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2)
  x'' = x' + dt/2 v;  x_{n+1} = SHAKE(x_n, x'');  v <- v + (x_{n+1} - x'')/dt
With gamma = 0 and no constraints this is the leapfrog form of velocity Verlet (the same
positions).  The kinetic energy at step n is reported as the mean of the half-step
values K(v_{n-1/2}) and K(v_{n+1/2}).
"""
import math

import numpy as np


def _pairs(d_oh, d_hh):
    """The three constraints of a water molecule (O, H1, H2): (i, j, d)."""
    return ((0, 1, d_oh), (0, 2, d_oh), (1, 2, d_hh))


def shake_molecule(x_old, x_new, m, d_oh, d_hh, tol=1e-14, max_iter=50):
    """SHAKE solution for one molecule (3x3 arrays, masses m[3])."""
    x_old = np.asarray(x_old, dtype=np.float64)
    x_new = np.asarray(x_new, dtype=np.float64)
    cons = _pairs(d_oh, d_hh)
    g = np.array([x_old[i] - x_old[j] for i, j, _ in cons])  # grad_i s_k / 2 at x_old
    lam = np.zeros(3)

    def positions(lam):
        x = x_new.copy()
        for k, (i, j, _) in enumerate(cons):
            x[i] += lam[k] * g[k] / m[i]
            x[j] -= lam[k] * g[k] / m[j]
        return x

    for _ in range(max_iter):
        x = positions(lam)
        res = np.array([np.dot(x[i] - x[j], x[i] - x[j]) - d * d for i, j, d in cons])
        if np.max(np.abs(res)) < tol * max(d_oh, d_hh) ** 2:
            return x
        J = np.zeros((3, 3))
        for k, (i, j, _) in enumerate(cons):
            r = x[i] - x[j]
            for l, (p, q, _) in enumerate(cons):
                # d x_i / d lam_l = g_l / m_i (i = p), -g_l / m_i (i = q)
                dxi = (g[l] / m[i]) * ((i == p) - (i == q))
                dxj = (g[l] / m[j]) * ((j == p) - (j == q))
                J[k, l] = 2.0 * np.dot(r, dxi - dxj)
        lam = lam - np.linalg.solve(J, res)
    raise RuntimeError("SHAKE did not converge")


def rattle_molecule(x, v, m, d_oh, d_hh):
    """Velocities of one molecule projected onto the constraint manifold at x."""
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64).copy()
    cons = _pairs(d_oh, d_hh)
    g = np.array([x[i] - x[j] for i, j, _ in cons])
    A = np.zeros((3, 3))
    b = np.zeros(3)
    for k, (i, j, _) in enumerate(cons):
        b[k] = -np.dot(g[k], v[i] - v[j])
        for l, (p, q, _) in enumerate(cons):
            dvi = (g[l] / m[i]) * ((i == p) - (i == q))
            dvj = (g[l] / m[j]) * ((j == p) - (j == q))
            A[k, l] = np.dot(g[k], dvi - dvj)
    mu = np.linalg.solve(A, b)
    for k, (i, j, _) in enumerate(cons):
        v[i] += mu[k] * g[k] / m[i]
        v[j] -= mu[k] * g[k] / m[j]
    return v


def constrain_positions(x_old, x_new, mass, mols, d_oh, d_hh):
    """SHAKE every molecule (rows of ``mols``: O, H1, H2 indices); other atoms unchanged."""
    x = np.array(x_new, dtype=np.float64)
    for mol in mols:
        x[mol] = shake_molecule(x_old[mol], x_new[mol], mass[mol], d_oh, d_hh)
    return x


def constrain_velocities(x, v, mass, mols, d_oh, d_hh):
    v = np.array(v, dtype=np.float64)
    for mol in mols:
        v[mol] = rattle_molecule(x[mol], v[mol], mass[mol], d_oh, d_hh)
    return v


def langevin_middle(x, v, mass, dt, gamma, kT, xi, n_steps, force_energy, mols=(), d_oh=1.0, d_hh=1.0):
    """n_steps of the Langevin middle scheme (module header) with normals xi[n_steps][n][3].
    Returns final (x, v) and the potential and kinetic energies at every integer step
    (the kinetic one as the mean of the neighbouring half steps; the last as K(v_{n-1/2}))."""
    m = np.asarray(mass, dtype=np.float64)
    mv = m[:, None]
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    c1 = math.exp(-gamma * dt)
    c2 = math.sqrt(max(0.0, 1.0 - c1 * c1))
    kin = lambda u: 0.5 * float(np.sum(mv * u * u))  # noqa: E731
    F, U = force_energy(x)
    Us, Ks = [], []
    for n in range(n_steps):
        k_prev = kin(v)
        v = v + dt * F / mv
        if len(mols):
            v = constrain_velocities(x, v, m, mols, d_oh, d_hh)
        x1 = x + 0.5 * dt * v
        v = c1 * v + c2 * np.sqrt(kT / mv) * np.asarray(xi[n], dtype=np.float64)
        x2 = x1 + 0.5 * dt * v
        if len(mols):
            x3 = constrain_positions(x, x2, m, mols, d_oh, d_hh)
            v = v + (x3 - x2) / dt
        else:
            x3 = x2
        Us.append(U)
        Ks.append(0.5 * (k_prev + kin(v)))
        x = x3
        F, U = force_energy(x)
    Us.append(U)
    Ks.append(kin(v))
    return x, v, np.array(Us), np.array(Ks)
