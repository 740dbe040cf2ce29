"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds inputs: lattices, molecule placement, seeded random
draws, parameter tables and exclusion lists.  It holds none of the method's
arithmetic (no energies, forces, lists or integrators) and serves both the CUDA
library's tests and benchmark and the FP64 oracle.

Workloads (every one synthetic; the paper's own TIP3P boxes and protein files
are not available, so these stand in for them):
  * ``lj_fcc``       -- LJ fluid on an FCC lattice, rho* = 0.8442 (864 atoms: 6^3 cells).
  * ``lj_random``    -- LJ atoms on a random subset of FCC sites with jitter, any N.
  * ``water_box``    -- 3-site point-charge water (O q=-0.8476, H q=+0.4238,
                        O-H 1.0 A, H-O-H 109.47 deg), randomly oriented molecules on
                        a jittered cubic lattice, LJ on O only, intramolecular
                        exclusions.
  * ``batched_mix``  -- many independent systems of uneven size (log-uniform N),
                        half LJ fluid, half water.
"""
from dataclasses import dataclass, field
import math
import numpy as np

KE_KJ_MOL_A = 1389.35457644  # Coulomb constant in kJ/mol * Angstrom / e^2

WATER_Q_O = -0.8476
WATER_Q_H = 0.4238
WATER_SIGMA_O = 3.166     # Angstrom
WATER_EPS_O = 0.650       # kJ/mol
WATER_ROH = 1.0           # Angstrom
WATER_HOH_DEG = 109.47
MASS_O = 15.999
MASS_H = 1.008
WATER_MOL_DENSITY = 0.03343  # molecules per cubic Angstrom at 1 g/cm^3
WATER_EPS_RF = 78.5          # solvent dielectric of the reaction field (water at 298 K)


def f32(v):
    """Round a scalar parameter to the nearest FP32 value (kept as a Python float).

    The CUDA path holds box lengths, cut-offs, alpha and ke in FP32; giving both
    it and the FP64 oracle the same FP32-exact values makes them evaluate the
    same function (a box that is off by one FP32 ulp shifts every pair that
    crosses the periodic boundary)."""
    return float(np.float32(v))


def f32_box(L):
    return np.array([f32(l) for l in np.broadcast_to(np.asarray(L, np.float64), (3,))])


@dataclass
class System:
    """One periodic system: per-atom arrays plus the interaction settings."""
    name: str
    x: np.ndarray              # (n, 3) float32 positions, wrapped into [0, L)
    q: np.ndarray              # (n,) float32 charges
    sigma: np.ndarray          # (n,) float32 LJ sigma_i
    sqrt_eps: np.ndarray       # (n,) float32 sqrt(eps_i)
    mass: np.ndarray           # (n,) float32
    box: np.ndarray            # (3,) float64
    r_cut: float
    r_skin: float
    alpha: float = 0.0         # Ewald splitting (0: no electrostatics)
    ke: float = 0.0            # Coulomb constant (0: no electrostatics)
    r_switch: float = -1.0     # LJ switching distance (<0: none)
    pme_grid: tuple = (0, 0, 0)
    pme_order: int = 4
    eps_rf: float = 0.0        # reaction field solvent dielectric (0: Ewald / no electrostatics)
    excl_off: np.ndarray = None  # (n+1,) int32 CSR offsets (symmetric)
    excl_idx: np.ndarray = None  # int32 CSR entries
    types: np.ndarray = None     # (n,) int32 atom types (mass sharing)
    v: np.ndarray = None         # (n, 3) float32 initial velocities (MD)
    extra: dict = field(default_factory=dict)

    def __setattr__(self, k, v):
        if k in ("r_cut", "r_skin", "alpha", "ke") or (k == "r_switch" and v is not None and v >= 0):
            v = f32(v)
        elif k == "box":
            v = f32_box(v)
        object.__setattr__(self, k, v)

    @property
    def n(self):
        return int(self.x.shape[0])

    @property
    def excl(self):
        if self.excl_off is None:
            return None
        return (self.excl_off, self.excl_idx)


def fcc_sites(n_cells, a):
    """FCC lattice sites of n_cells^3 conventional cells with lattice constant a."""
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    g = np.arange(n_cells, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return ((cells[:, None, :] + base[None, :, :]).reshape(-1, 3)) * a


def _wrap(x, box):
    return x - box * np.floor(x / box)


def maxwell_boltzmann_initial(mass, kT, seed):
    """Initial MD velocities: N(0, kT/m) per component (seeded), centre-of-mass
    velocity removed, no rescaling."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((mass.size, 3)) * np.sqrt(kT / mass)[:, None]
    p = (v * mass[:, None]).sum(axis=0) / mass.sum()
    return (v - p).astype(np.float32)


def lj_fcc(n_cells=6, rho=0.8442, r_cut=2.5, r_skin=0.3, kT=0.72, seed=1234, r_switch=-1.0):
    """LJ fluid, eps = sigma = m = 1, FCC start (6^3 cells -> 864 atoms, L = 10.0776)."""
    n = 4 * n_cells ** 3
    L = (n / rho) ** (1.0 / 3.0)
    x = fcc_sites(n_cells, L / n_cells)
    box = np.array([L, L, L])
    mass = np.ones(n, dtype=np.float32)
    s = System(name="lj_fcc_%d" % n, x=_wrap(x, box).astype(np.float32), q=np.zeros(n, np.float32),
               sigma=np.ones(n, np.float32), sqrt_eps=np.ones(n, np.float32), mass=mass, box=box,
               r_cut=r_cut, r_skin=r_skin, r_switch=r_switch, types=np.zeros(n, np.int32))
    s.v = maxwell_boltzmann_initial(mass.astype(np.float64), kT, seed)
    return s


def lj_random(n, rho=0.8442, r_cut=2.5, r_skin=0.3, seed=1234, jitter=0.08, n_types=1, kT=1.0):
    """LJ atoms on a random subset of the sites of the smallest FCC lattice with
    >= n sites, each jittered uniformly by +-jitter*sigma (no overlaps)."""
    L = (n / rho) ** (1.0 / 3.0)
    nc = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
    rng = np.random.default_rng(seed)
    sites = fcc_sites(nc, L / nc)
    if sites.shape[0] > n:
        sites = sites[np.sort(rng.choice(sites.shape[0], size=n, replace=False))]
    x = sites + rng.uniform(-jitter, jitter, size=sites.shape)
    box = np.array([L, L, L])
    types = (np.arange(n) % n_types).astype(np.int32)
    mass = np.ones(n, dtype=np.float32)
    s = System(name="lj_random_%d" % n, x=_wrap(x, box).astype(np.float32), q=np.zeros(n, np.float32),
               sigma=np.ones(n, np.float32), sqrt_eps=np.ones(n, np.float32), mass=mass, box=box,
               r_cut=r_cut, r_skin=r_skin, types=types)
    s.v = maxwell_boltzmann_initial(mass.astype(np.float64), kT, seed + 1)
    return s


def _random_rotations(rng, m):
    """Uniform random rotation matrices from uniform quaternions (Shoemake 1992)."""
    u1, u2, u3 = rng.uniform(size=(3, m))
    a = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    b = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    c = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    d = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    R = np.empty((m, 3, 3))
    R[:, 0, 0] = 1 - 2 * (c * c + d * d); R[:, 0, 1] = 2 * (b * c - a * d); R[:, 0, 2] = 2 * (b * d + a * c)
    R[:, 1, 0] = 2 * (b * c + a * d); R[:, 1, 1] = 1 - 2 * (b * b + d * d); R[:, 1, 2] = 2 * (c * d - a * b)
    R[:, 2, 0] = 2 * (b * d - a * c); R[:, 2, 1] = 2 * (c * d + a * b); R[:, 2, 2] = 1 - 2 * (b * b + c * c)
    return R


def water_exclusions(n_mol):
    """Symmetric CSR exclusion list: each atom excludes its two molecule mates."""
    n = 3 * n_mol
    off = np.arange(0, 2 * n + 1, 2, dtype=np.int32)
    idx = np.empty(2 * n, dtype=np.int32)
    base = 3 * np.arange(n_mol)
    for k in range(3):
        others = [o for o in range(3) if o != k]
        idx[2 * (base + k)] = base + others[0]
        idx[2 * (base + k) + 1] = base + others[1]
    return off, idx


def fft_friendly(n):
    """Smallest integer >= n whose prime factors are 2, 3 and 5."""
    k = int(math.ceil(n))
    while True:
        m = k
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return k
        k += 1


def water_box(n_side=20, L=62.1, seed=1234, jitter=0.3, r_cut=9.0, r_skin=2.25, alpha=0.32,
              pme_grid=64, n_mol=None):
    """Point-charge water box (default: 8000 molecules on a 20^3 lattice in 62.1 A).

    With ``n_mol`` < n_side^3, a random subset of lattice sites is used."""
    rng = np.random.default_rng(seed)
    sp = L / n_side
    g = (np.arange(n_side) + 0.5) * sp
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    if n_mol is not None and n_mol < sites.shape[0]:
        sites = sites[np.sort(rng.choice(sites.shape[0], size=n_mol, replace=False))]
    m = sites.shape[0]
    o = sites + rng.uniform(-jitter, jitter, size=sites.shape)
    th = math.radians(WATER_HOH_DEG) / 2.0
    ref = np.array([[0.0, 0.0, 0.0],
                    [WATER_ROH * math.sin(th), WATER_ROH * math.cos(th), 0.0],
                    [-WATER_ROH * math.sin(th), WATER_ROH * math.cos(th), 0.0]])
    R = _random_rotations(rng, m)
    mol = o[:, None, :] + np.einsum("mij,kj->mki", R, ref)
    x = mol.reshape(-1, 3)
    box = np.array([L, L, L])
    n = 3 * m
    q = np.tile(np.array([WATER_Q_O, WATER_Q_H, WATER_Q_H]), m).astype(np.float32)
    sigma = np.tile(np.array([WATER_SIGMA_O, 1.0, 1.0]), m).astype(np.float32)
    sqe = np.tile(np.array([math.sqrt(WATER_EPS_O), 0.0, 0.0]), m).astype(np.float32)
    mass = np.tile(np.array([MASS_O, MASS_H, MASS_H]), m).astype(np.float32)
    off, idx = water_exclusions(m)
    K = pme_grid if pme_grid else fft_friendly(L / 0.97)
    return System(name="water_%d" % n, x=_wrap(x, box).astype(np.float32), q=q, sigma=sigma, sqrt_eps=sqe,
                  mass=mass, box=box, r_cut=r_cut, r_skin=r_skin, alpha=alpha, ke=KE_KJ_MOL_A,
                  pme_grid=(K, K, K), excl_off=off, excl_idx=idx,
                  types=np.tile(np.array([0, 1, 1], np.int32), m))


def water_slab(seed=7, n_layers=8):
    """A non-cubic water box: the molecules of the lowest n_layers of the 10 lattice layers
    of a 31.05 A water box (seed), in a 31.05 x 31.05 x (n_layers * 3.105) A cell (the
    lattice period along z, so the spacing across the boundary stays regular), PME mesh
    32 x 32 x 26 for 8 layers."""
    base = water_box(n_side=10, L=31.05, seed=seed, pme_grid=32)
    m = base.n // 3
    keep = np.where(base.x.reshape(m, 3, 3)[:, 0, 2] < n_layers * 3.105)[0]
    sel = (3 * keep[:, None] + np.arange(3)).ravel()
    off, idx = water_exclusions(len(keep))
    box = np.array([31.05, 31.05, n_layers * 3.105])
    kz = int(math.ceil(n_layers * 3.105 / 0.97))
    s = System(name="water_slab", x=np.zeros((len(sel), 3), np.float32), q=base.q[sel], sigma=base.sigma[sel],
               sqrt_eps=base.sqrt_eps[sel], mass=base.mass[sel], box=box, r_cut=base.r_cut, r_skin=base.r_skin,
               alpha=base.alpha, ke=base.ke, pme_grid=(32, 32, kz), excl_off=off, excl_idx=idx,
               types=base.types[sel])
    s.x = np.mod(base.x[sel].astype(np.float64), s.box).astype(np.float32)
    return s


def water_box_density(n_mol, seed, r_cut=9.0, r_skin=2.25, alpha=0.32, jitter=0.3):
    """Water at 1 g/cm^3 with n_mol molecules; grid K = FFT-friendly >= L/0.97 A."""
    L = (n_mol / WATER_MOL_DENSITY) ** (1.0 / 3.0)
    n_side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    K = fft_friendly(L / 0.97)
    return water_box(n_side=n_side, L=L, seed=seed, jitter=min(jitter, 0.1 * L / n_side), r_cut=r_cut,
                     r_skin=r_skin, alpha=alpha, pme_grid=K, n_mol=n_mol)


def as_reaction_field(s, eps_rf=WATER_EPS_RF):
    """The same system with the reaction field of Eq. RFA (solvent dielectric eps_rf)
    in place of Ewald + PME."""
    s.alpha = 0.0
    s.pme_grid = (0, 0, 0)
    s.eps_rf = float(eps_rf)
    s.name = s.name + "_rf"
    return s


def water_rf_density(n_mol, seed, r_cut=10.0, r_skin=2.5, eps_rf=WATER_EPS_RF, jitter=0.3):
    """Water at 1 g/cm^3 with the reaction field, r_c 10 A: the setting of the paper's
    water scaling benchmark (Sec. 3, electrostatics by RFA)."""
    s = water_box_density(n_mol, seed, r_cut=r_cut, r_skin=r_skin, alpha=0.0, jitter=jitter)
    return as_reaction_field(s, eps_rf)


def batched_mix(n_systems=256, n_min=500, n_max=20000, seed=1234, water_r_nl=11.25):
    """Uneven systems, N log-uniform in [n_min, n_max]; even index LJ, odd index water.

    Water sizes are drawn log-uniformly on [N_min, n_max], N_min the smallest atom
    count whose box holds the minimum image at r_nl (L >= 2 r_nl)."""
    rng = np.random.default_rng(seed)
    n_min_w = int(math.ceil(WATER_MOL_DENSITY * (2 * water_r_nl) ** 3)) * 3
    out = []
    for s in range(n_systems):
        if s % 2 == 0:
            n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
            out.append(lj_random(n, seed=seed + 17 * s))
        else:
            n = int(round(math.exp(rng.uniform(math.log(max(n_min, n_min_w)), math.log(n_max)))))
            out.append(water_box_density(max(1, n // 3), seed=seed + 17 * s))
    return out


def random_cotangent(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, 3)) * scale).astype(np.float32)


def hmc_randoms(n_rep, n, seed):
    """Per-replica standard normals (velocity draws) and uniforms (Metropolis test)."""
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((n_rep, n, 3)).astype(np.float32)
    u = rng.uniform(size=n_rep)
    return xi, u
