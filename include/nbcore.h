/*
 * nbcore.h -- C ABI of libnbcore, the B300 (sm_103a) nonbonded-force / MD / HMC
 * library for the hot path of arXiv 2503.20541 (DIMOS).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Atoms of all systems of a handle are concatenated in system order
 *    ("caller order"); system s owns atoms [offset_s, offset_s + n_s) where
 *    offset_s is the sum of the n of the systems before it.
 *  - Positions are float[N][4] = (x, y, z, q): coordinates plus the charge q in
 *    the fourth slot.  Coordinates may lie anywhere; the library wraps them
 *    into the box internally and never rewrites caller coordinates except in
 *    md_step / hmc_trajectory, whose job is to move them.
 *  - Forces, cotangents and gradients with respect to positions are
 *    float[N][3].
 *  - Every pointer marked (device) is CUDA device memory owned by the caller;
 *    the library keeps no reference past the call.  Pointers marked (host) are
 *    read during the call only.  The handle owns its scratch (cell lists,
 *    neighbour list, fixed-point accumulators, PME meshes, cuFFT plans).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Entry points are asynchronous on that stream unless stated otherwise.
 *  - Errors discovered on the device (list overflow, fixed-point overflow,
 *    non-finite coordinates) are OR-ed into a sticky device word; nb_check
 *    synchronises the stream, returns the first of them as a status and
 *    clears it.  No kernel traps.
 *  - Units are the caller's (reduced LJ, or kJ/mol, Angstrom, e with ke given).
 */
#ifndef NBCORE_H
#define NBCORE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NB_OK = 0,
    NB_ERR_ARG = 1,                 /* invalid argument (NULL, size, unsupported option) */
    NB_ERR_BOX_TOO_SMALL = 2,       /* periodic box edge < 2 r_nl: minimum image is ambiguous */
    NB_ERR_LIST_OVERFLOW = 3,       /* an atom has more neighbours than the list capacity */
    NB_ERR_FIXEDPOINT_OVERFLOW = 4, /* |value| * 2^force_bits does not fit in int64 */
    NB_ERR_NONFINITE = 5,           /* NaN / Inf coordinate */
    NB_ERR_TIMEOUT = 6,             /* reserved for bounded device waits */
    NB_ERR_CUDA = 7,                /* a CUDA runtime or cuFFT call failed */
    NB_ERR_NOMEM = 8                /* device allocation failed */
} nb_status;

/* Bits of the sticky device error word (nb_check maps them to nb_status). */
#define NB_DEVERR_LIST_OVERFLOW 1u
#define NB_DEVERR_FIXEDPOINT 2u
#define NB_DEVERR_NONFINITE 4u
#define NB_DEVERR_ARG 8u          /* a device-side argument out of range (e.g. a proposal length) */

/* Energy components per system, in this order (FP64). */
#define NB_E_LJ 0    /* Lennard-Jones, Eq. (lj), r < r_c, optional switch S(x) */
#define NB_E_DIR 1   /* Ewald direct space, sum ke q_i q_j erfc(alpha r)/r, r < r_c */
#define NB_E_EXCL 2  /* exclusion correction, -sum_excl ke q_i q_j erf(alpha r)/r */
#define NB_E_SELF 3  /* Ewald self energy, -ke alpha/sqrt(pi) sum q_i^2 */
#define NB_E_REC 4   /* PME reciprocal-space energy */
#define NB_E_KIN 5   /* kinetic energy 1/2 sum m v^2 (MD / HMC only) */
#define NB_NE 6

/* Term flags for nonbonded_forces / md_step / hmc_trajectory. */
#define NB_TERM_LJ 1
#define NB_TERM_COUL 2   /* Ewald direct + exclusion correction + self, or the reaction field */
#define NB_TERM_PME 4    /* PME reciprocal space (systems with a PME mesh) */
#define NB_TERM_ALL 7
#define NB_FORCE_REBUILD 256 /* rebuild the neighbour list unconditionally */
#define NB_ENERGY_PRECISE 512 /* nonbonded_forces: energies in two-float arithmetic (see there) */

/*
 * One periodic (or open) system.  Follows Sec. 2.1.2 of the paper:
 *   r_nl = r_cut + r_skin (r_skin is the paper's "ghost radius" r_g, default 0.25 r_c);
 *   the list is rebuilt when an atom has moved more than r_skin/2;
 *   LJ with Lorentz-Berthelot mixing, optional switch from r_switch to r_cut;
 *   Ewald splitting alpha, Coulomb constant ke (ke = 0: no charges);
 *   smooth PME of order 4 on a pme_grid[0] x pme_grid[1] x pme_grid[2] mesh
 *   (all zero: no reciprocal space);
 *   or, with eps_rf >= 1, the reaction field of Eq. RFA instead of Ewald:
 *   ke q_i q_j (1/r + k r^2 - c) for non-excluded pairs with r < r_cut,
 *   k = (eps_rf - 1) / ((2 eps_rf + 1) r_cut^3), c = 3 eps_rf / ((2 eps_rf + 1) r_cut)
 *   (eps_rf the solvent dielectric; excluded pairs do not interact; alpha must be 0 and
 *   pme_grid all zero).  eps_rf = 0 selects Ewald.  The charged systems of one handle
 *   must all use the same electrostatics (NB_ERR_ARG otherwise).
 * Periodic systems need box[d] >= 2 r_nl in every dimension.  Open systems
 * (periodic = 0) must keep every coordinate inside [0, box).
 */
typedef struct {
    int32_t n_atoms;
    int32_t periodic;     /* 1: periodic orthorhombic box; 0: open system embedded in `box` */
    double box[3];
    double r_cut;
    double r_skin;
    double r_switch;      /* < 0: no switch */
    double alpha;
    double ke;
    int32_t pme_grid[3];
    int32_t pme_order;    /* 4 (the only order implemented) */
    double eps_rf;        /* reaction field solvent dielectric (>= 1); 0: Ewald */
} nb_system_desc;

/* Tuning knobs; zero-initialise for defaults. */
typedef struct {
    int32_t max_neighbors;   /* per-atom list capacity (full list), rounded up to a multiple
                                of 128; 0: from density */
    int32_t stencil_tile;    /* stencil candidates per shared-memory tile of the list build
                                (multiple of 64 in [256, 4096]); 0: auto from the density */
    int32_t cell_div;        /* cells of edge >= r_nl / cell_div, cell_div in {1, 2}, for every
                                system; 0: chosen per system (2 for a system with >= 5 cells
                                of edge r_nl/2 along each axis and >= 64 atoms per r_nl^3) */
    int32_t force_bits;      /* fixed-point fraction bits for forces; 0: 32 */
    int32_t blocks_per_cell; /* thread blocks sharing one cell in the list build (each takes a
                                strided share of the cell's atoms), in [1, 32]; 0: auto (more
                                than one only when the cells are too few to fill the GPU).
                                Results do not depend on it.  The pair and VJP kernels are not
                                organised by cell: their blocks take consecutive atoms. */
    double prune_skin;       /* dynamic list pruning between builds: on the first evaluation
                                after a build, and whenever an atom has moved more than
                                prune_skin/2 since, every row is re-partitioned at the current
                                positions into the pairs within r_c + prune_skin and the rest,
                                and the pair and VJP kernels skip the rest (no pair of it can
                                be within r_c before the next re-partition).  The list itself,
                                its build and its rebuild test are unchanged.  > 0: this inner
                                skin for every system (< r_skin); < 0: off; 0: r_skin/3 for
                                systems whose r_skin is >= 0.15 r_c, off for the others. */
} nb_options;

typedef struct nb_handle nb_handle;

/* Human-readable name of a status. */
const char* nb_status_str(nb_status s);

/*
 * Create a handle for n_systems systems on the current CUDA device.
 *   sys[n_systems]        (host) system descriptors.
 *   sigma, sqrt_eps [N]   (host) per-atom LJ sigma_i and sqrt(eps_i), caller order
 *                         (eps_ij = sqrt_eps_i sqrt_eps_j, sigma_ij = (sigma_i + sigma_j)/2).
 *   excl_off [N+1], excl_idx (host, may both be NULL) CSR exclusion lists in caller
 *                         indices; a pair is excluded when either atom lists the other
 *                         (Sec. 2.1.2 "Exclusions and Exceptions"); both atoms must be in
 *                         the same system.
 *   opt                   (host, may be NULL) tuning knobs.
 * Allocates all device scratch.  Returns NB_ERR_BOX_TOO_SMALL / NB_ERR_ARG on invalid
 * systems, NB_ERR_NOMEM / NB_ERR_CUDA on allocation or plan failure (nothing leaks).
 */
nb_status nb_create(nb_handle** out, const nb_system_desc* sys, int32_t n_systems,
                    const float* sigma, const float* sqrt_eps,
                    const int32_t* excl_off, const int32_t* excl_idx,
                    const nb_options* opt);

/* Free a handle and all its device memory (synchronises the device). NULL is a no-op. */
void nb_destroy(nb_handle* h);

/* Total atom count and system count of a handle. */
int64_t nb_num_atoms(const nb_handle* h);
int32_t nb_num_systems(const nb_handle* h);

/*
 * Synchronise `stream`, read and clear the sticky device error word.
 * Returns NB_OK or the status of the first error bit set.
 */
nb_status nb_check(nb_handle* h, void* stream);

/*
 * Neighbour list (Sec. 2.1.2 "Neighborlists"; the NeighborHandling(...).get_neighborlist(pos)
 * call of the paper).  Cell list with cells of edge >= r_nl/cell_div, counting sort of atoms
 * by cell, then a Verlet list of all pairs with |mi(x_i - x_j)| < r_nl = r_cut + r_skin,
 * excluded pairs removed.
 *   xq [N][4]      (device) positions and charges.
 *   pairs_out      (device, may be NULL) receives up to max_pairs unordered pairs
 *                  (i, j), i < j, caller indices, as int32[max_pairs][2]; their order is
 *                  unspecified.
 *   n_pairs_out    (host) number of unordered pairs in the list (may exceed max_pairs).
 *   force_rebuild  0: rebuild only if an atom moved more than r_skin/2 since the last
 *                  build (the paper's validity test); 1: always.
 * Synchronous: returns after the list is built.  Errors: NB_ERR_LIST_OVERFLOW (raise
 * nb_options.max_neighbors), NB_ERR_NONFINITE.
 */
nb_status nl_build(nb_handle* h, const float* xq, int32_t* pairs_out, int64_t max_pairs,
                   int64_t* n_pairs_out, int32_t force_rebuild, void* stream);

/*
 * Nonbonded energies and forces (Sec. 2.1.2): LJ, Ewald direct erfc Coulomb under the
 * minimum image, exclusion correction, self energy and PME reciprocal space, selected
 * by `terms` (NB_TERM_*; add NB_FORCE_REBUILD to force a list rebuild).  The neighbour
 * list is checked and rebuilt on the device when needed.
 *   xq [N][4]            (device) positions and charges.
 *   f_out [N][3]         (device, may be NULL) forces -dE/dx.
 *   energies [n_sys][6]  (device, may be NULL) FP64 components NB_E_* (NB_E_KIN = 0).
 * Forces are accumulated in int64 fixed point (2^force_bits units per force unit), so
 * they are bitwise reproducible run to run.  With energies == NULL the real-space pass
 * runs an energy-free kernel (a polynomial erfc, 1/r^2 from 1/r, a shorter reduction):
 * its forces agree with those of a call that asks for energies to FP32 rounding, not
 * bit for bit.
 * With NB_ENERGY_PRECISE in `terms` (and energies != NULL) the real-space and exclusion
 * energies are recomputed in two-float arithmetic (an FP32 hi + lo pair, ~48 bits: exact
 * coordinate differences, r^2, 1/r, erfc and the LJ powers to 1e-14 - 1e-12 relative, two-float
 * per-atom sums) by a second list pass, and reduced in FP64 as hi + lo.  Energy sums whose
 * pair terms cancel 10^3-10^4-fold (neutral water) then meet 1e-6 relative against FP64
 * where the FP32 energies do not; the forces are the energy-free kernel's (bitwise those of
 * a call with energies == NULL).  The PME reciprocal and self energies are FP64 either way.
 */
nb_status nonbonded_forces(nb_handle* h, const float* xq, float* f_out, double* energies,
                           int32_t terms, void* stream);

/*
 * All-pairs Lennard-Jones forces and energy: every pair (i, j != i) of each system with
 * |mi(x_i - x_j)| < r_cut, same LJ terms and switch as nonbonded_forces, but no cell or
 * Verlet list -- O(N^2) work per system.  It is the comparison baseline of the linear
 * cell-list path (Sec. 3 compares neighbour-list evaluation against all-pairs); the
 * list state of the handle is not touched.
 *   xq [N][4]            (device) positions and charges (caller order; need not be wrapped).
 *   f_out [N][3]         (device, may be NULL) LJ forces.
 *   energies [n_sys][6]  (device, may be NULL) FP64 components; only NB_E_LJ is set.
 * Launches one kernel per system and returns; errors are read with nb_check.
 */
nb_status nonbonded_forces_allpairs(nb_handle* h, const float* xq, float* f_out, double* energies, void* stream);

/*
 * The complementary error function of the Ewald direct-space term ke q_i q_j erfc(alpha r)/r
 * (Sec. 2.1.2) exactly as the pair kernels evaluate it (FP32: a fitted erfcx polynomial in
 * t = 1/(1 + x/2) times exp(-x^2) from the hardware 2^y approximation with a two-float
 * argument), for checking it against a reference erfc.
 *   x [n]    (device) arguments, x >= 0 (alpha r); other values give unspecified results.
 *   out [n]  (device) erfc(x).
 * No handle; launches one kernel on `stream`; NB_ERR_ARG for n < 0 or NULL arrays with n > 0.
 */
nb_status nb_erfc_eval(const float* x, float* out, int32_t n, void* stream);

/*
 * erfc(x) in two-float arithmetic exactly as the precise energies evaluate it
 * (NB_ENERGY_PRECISE): x = x_hi + x_lo, a piecewise degree-15 interpolant with two-float
 * coefficients on [0, 6) (FP32 erfcf beyond), for checking it against a reference erfc.
 *   x_hi, x_lo [n]        (device) the argument as an unevaluated sum, x >= 0, |x_lo| small
 *                         against x_hi (a rounding error); other values give unspecified results.
 *   out_hi, out_lo [n]    (device) erfc(x) = out_hi + out_lo.
 * No handle; launches one kernel on `stream`; NB_ERR_ARG for n < 0 or NULL arrays with n > 0.
 */
nb_status nb_erfc_df_eval(const float* x_hi, const float* x_lo, float* out_hi, float* out_lo, int32_t n,
                          void* stream);

/*
 * PME charge spreading alone (Sec. 2.1.2, smooth PME with order-4 cardinal B-splines):
 *   grid (device) float, for every PME system s the K0*K1*K2 real mesh of system s,
 *   index ((k0 * K1) + k1) * K2 + k2, systems concatenated in system order (systems
 *   without PME take no space).  grid[k] = sum_i q_i M4(u_i0 - k0) M4(u_i1 - k1) M4(u_i2 - k2)
 *   with u_id = K_d x_id / L_d and periodic wrap of k.
 */
nb_status pme_spread(nb_handle* h, const float* xq, float* grid, void* stream);

/*
 * PME force gathering alone: F_i = -q_i sum_k grad_i[M4 M4 M4](k) phi(k) for a caller
 * potential mesh phi (device, same layout as pme_spread's grid).  f_out [N][3] (device)
 * is overwritten (atoms of systems without PME get 0).
 */
nb_status pme_gather(nb_handle* h, const float* xq, const float* phi, float* f_out, void* stream);

/*
 * Velocity-Verlet MD (Sec. 2.2.1, steps 1, 2, 4, 5 of the MD loop; no constraints or
 * thermostat): n_steps steps of every system with its own step dt[s].
 *   xq [N][4]           (device, in/out) positions and charges (charges untouched).
 *   v [N][4]            (device, in/out) (vx, vy, vz, inverse mass) -- the fourth slot
 *                       is read, not written.
 *   dt [n_sys]          (device) time step per system.
 *   energies            (device, may be NULL) FP64 [n_steps+1][n_sys][6]: NB_E_* at every
 *                       integer step including the start.
 *   terms               NB_TERM_* selection of force terms.
 * The neighbour list is checked after every drift and rebuilt on the device when needed.
 */
nb_status md_step(nb_handle* h, float* xq, float* v, const float* dt, int32_t n_steps,
                  double* energies, int32_t terms, void* stream);

/*
 * Rigid three-site water for langevin_step and the constraint calls (Sec. 2.2.1:
 * position and velocity constraints, SETTLE):
 *   mols [n_mol][3] (host) caller indices (O, H1, H2) of each molecule, each atom in at
 *                   most one molecule, the three in one system; both H of a molecule must
 *                   have the same mass.
 *   d_oh, d_hh      the constrained O-H and H-H distances (0 < d_hh < 2 d_oh).
 * n_mol = 0 removes all constraints.  Host work and one copy; NB_ERR_ARG on invalid input.
 */
nb_status nb_set_water_constraints(nb_handle* h, const int32_t* mols, int32_t n_mol, double d_oh, double d_hh);

/*
 * Langevin dynamics (Sec. 2.2.1; the "middle" scheme of the unified thermostat framework the
 * paper cites, in leapfrog variables, velocities at half steps), n_steps steps of
 *   v += dt w F;  constrain v;  x' = x + dt/2 v;  v = c1 v + c2 sqrt(kT w) xi;
 *   x'' = x' + dt/2 v;  x = SETTLE(x, x'');  v += (x - x'') / dt
 * with c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2), the constraints those set by
 * nb_set_water_constraints (none: plain Langevin; gamma = 0: leapfrog velocity Verlet).
 *   xq [N][4]        (device, in/out) positions and charges.
 *   v [N][4]         (device, in/out) (vx, vy, vz, inverse mass): the velocity half a step
 *                    before xq's step (read and written), the inverse mass read only.
 *   dt, gamma [n_sys] (device) step and friction per system.
 *   kT               thermal energy in the energy unit of the force field.
 *   xi               (device) [n_steps][N][3] standard normals, one triple per atom and step.
 *   energies         (device, may be NULL) FP64 [n_steps+1][n_sys][6] as md_step, the kinetic
 *                    energy at step n the mean of the two neighbouring half steps (at the
 *                    last step, the half step before it).
 * A molecule that SETTLE cannot place (a step far too large) makes nb_check return
 * NB_ERR_NONFINITE.
 */
nb_status langevin_step(nb_handle* h, float* xq, float* v, const float* dt, const float* gamma, double kT,
                        int32_t n_steps, const float* xi, double* energies, int32_t terms, void* stream);

/*
 * SETTLE alone: constrains every molecule of x relative to the constrained positions
 * x_ref (both [N][4], device; x overwritten), with inverse masses inv_mass [N] (device);
 * v [N][4] (device, may be NULL) gets the correction / dt added.  Atoms outside molecules
 * are untouched.
 */
nb_status constrain_positions(nb_handle* h, const float* x_ref, float* x, float* v, const float* inv_mass, float dt,
                              void* stream);

/*
 * Velocity constraint alone: v [N][4] (device, (vx, vy, vz, inverse mass)) projected so that
 * every constrained distance of the molecules at x [N][4] has zero rate.
 */
nb_status constrain_velocities(nb_handle* h, const float* x, float* v, void* stream);

/*
 * One HMC proposal per system (Sec. 4): Maxwell-Boltzmann velocities
 * v0 = sqrt(kT w) xi (w = inverse mass), n_leap velocity-Verlet steps of length dt[s],
 * E = U + K in FP64, acceptance alpha = min(1, exp(-(E' - E)/kT)), Metropolis test
 * u[s] < alpha, squared jump |mi(x' - x)|^2 summed over the system's atoms (the
 * observable O = x of the ESJD loss, Eq. loss).
 *   x0 [N][4]        (device) start positions and charges.
 *   x_out [N][4]     (device) the new chain state: the proposal where accepted, x0
 *                    elsewhere.  May not alias x0.
 *   inv_mass [N]     (device) inverse masses w_i.
 *   dt [n_sys]       (device) step per system.
 *   xi [N][3]        (device) standard-normal deviates for the velocity draw.
 *   u [n_sys]        (device, FP64) uniforms in [0,1) for the Metropolis test.
 *   stats [n_sys][4] (device, FP64) out: dH, alpha, jump, accepted (0/1).
 *   ckpt             (device, may be NULL) float[ceil(n_leap/ckpt_every)][2][N][4]:
 *                    (positions, velocities) at steps 0, k, 2k, ... for the backward pass.
 * With checkpoints, the neighbour list is rebuilt at every checkpoint step so that a
 * recomputation from a checkpoint repeats the forward trajectory bit for bit.
 * With NB_ENERGY_PRECISE in `terms`, the potential energies of the two end states (and so
 * dH) are the two-float energies of nonbonded_forces (the forces there come from the
 * energy-free kernel); pass the same `terms` to hmc_trajectory_backward, whose
 * recomputation then runs the same kernels.
 */
nb_status hmc_trajectory(nb_handle* h, const float* x0, float* x_out, const float* inv_mass,
                         const float* dt, int32_t n_leap, double kT, const float* xi,
                         const double* u, double* stats, float* ckpt, int32_t ckpt_every,
                         int32_t terms, void* stream);

/*
 * Reverse-mode derivative of hmc_trajectory (the differentiation of Sec. 4, done with
 * a hand-written adjoint of velocity Verlet and the force VJP instead of autograd).
 * Given cotangents g_alpha[s] and g_jump[s] of each system's acceptance probability
 * and squared jump, accumulates
 *   g_dt [n_sys]     (device, FP64, +=) d/d dt[s],
 *   g_inv_mass [N]   (device, FP32, +=) d/d w_i,
 * recomputing the trajectory segment by segment from `ckpt` (written by the forward
 * call with the same arguments) and applying the force VJP at every state.
 *   stats            (device) the forward call's stats.
 * The first call with a given ckpt_every allocates a segment buffer of
 * 3 (ckpt_every + 1) N float4.  With NB_TERM_PME the reciprocal-space VJP is applied
 * at every state as well.
 */
nb_status hmc_trajectory_backward(nb_handle* h, const float* x0, const float* inv_mass,
                                  const float* dt, int32_t n_leap, double kT, const float* xi,
                                  const float* ckpt, int32_t ckpt_every, const double* stats,
                                  const double* g_alpha, const double* g_jump,
                                  double* g_dt, float* g_inv_mass, int32_t terms, void* stream);

/*
 * HMC with a drawn trajectory length and per-step statistics (Sec. 4, Eq. loss_steps):
 * one trajectory of n_leap = L_q velocity-Verlet steps per system from the
 * Maxwell-Boltzmann draw v0 = sqrt(kT w) xi, recording at every step l = 1..n_leap the
 * statistics of proposing (x_l, v_l), and proposing the state after l_prop[s] steps.
 *   x0 [N][4]           (device) start positions and charges.
 *   x_out [N][4]        (device) the new chain state: x_{l_prop[s]} where accepted, x0
 *                       elsewhere.  May not alias x0.
 *   inv_mass [N], dt [n_sys], xi [N][3], u [n_sys]  as for hmc_trajectory.
 *   l_prop [n_sys]      (device, int32) the proposal length of each system, in
 *                       [1, n_leap] (the caller draws it from the discretised folded
 *                       normal); a value outside that range keeps x0 for the system,
 *                       zeroes its stats and makes nb_check return NB_ERR_ARG.
 *   stats [n_sys][4]    (device, FP64) out: dH, alpha, jump, accepted of the proposal.
 *   step_stats          (device, FP64) out: [n_leap][n_sys][3] (dH_l, alpha_l, jump_l),
 *                       dH_l = E(x_l, v_l) - E(x_0, v_0), alpha_l = min(1, exp(-dH_l/kT)),
 *                       jump_l = |mi(x_l - x_0)|^2 summed over the system's atoms.
 *   ckpt, ckpt_every    as for hmc_trajectory (positions and velocities at steps 0, k, ...).
 * Every system runs all n_leap steps.
 */
nb_status hmc_trajectory_steps(nb_handle* h, const float* x0, float* x_out, const float* inv_mass,
                               const float* dt, int32_t n_leap, const int32_t* l_prop, double kT,
                               const float* xi, const double* u, double* stats, double* step_stats,
                               float* ckpt, int32_t ckpt_every, int32_t terms, void* stream);

/*
 * Reverse-mode derivative of hmc_trajectory_steps: given cotangents
 * g_alpha [n_leap][n_sys] and g_jump [n_leap][n_sys] (device, FP64) of every step's
 * acceptance probability and squared jump, accumulates g_dt [n_sys] (FP64, +=) and
 * g_inv_mass [N] (FP32, +=), recomputing from `ckpt` like hmc_trajectory_backward.
 *   step_stats          (device) the forward call's step_stats.
 */
nb_status hmc_trajectory_steps_backward(nb_handle* h, const float* x0, const float* inv_mass,
                                        const float* dt, int32_t n_leap, double kT, const float* xi,
                                        const float* ckpt, int32_t ckpt_every,
                                        const double* step_stats, const double* g_alpha,
                                        const double* g_jump, double* g_dt, float* g_inv_mass,
                                        int32_t terms, void* stream);

/*
 * Autocorrelation function and exponential autocorrelation time (Sec. 4) of n_series
 * series of n samples each (e.g. the potential energy along HMC chains):
 *   A(k) = (<O_t O_{t+k}> - <O>^2) / (<O^2> - <O>^2),  k = 0..max_lag,
 * estimated about the series mean m: [1/(n-k) sum_{t<n-k} (O_t - m)(O_{t+k} - m)] over
 * [1/n sum_t (O_t - m)^2] (equal in expectation, and invariant under O -> a O + b);
 * tau_exp from A(k) -> exp(-k/tau_exp): the least-squares slope of ln A(k) against k over
 * the lags k >= 1 from the first with A(k) <= a_hi up to the last before A(k) first falls
 * below a_lo; NaN when fewer than two lags qualify.
 *   series [n_series][n]        (device, FP64).
 *   acf [n_series][max_lag+1]   (device, FP64) out.
 *   tau [n_series]              (device, FP64) out (may be NULL).
 * Requires 1 <= max_lag < n and 0 < a_lo < a_hi <= 1.
 */
nb_status autocorrelation(const double* series, int32_t n_series, int32_t n, int32_t max_lag, double a_hi,
                          double a_lo, double* acf, double* tau, void* stream);

/*
 * Force vector-Jacobian product (Sec. 4 differentiates the trajectory through the
 * forces): for a cotangent lam [N][3] and the terms selected by `terms` (NB_TERM_*),
 *   gx = (dF/dx)^T lam           (a Hessian-vector product of -E),
 *   gq, gsigma, gsqrt_eps        gradients of lam . F with respect to q_i, sigma_i and
 *                                sqrt(eps_i) (each may be NULL),
 *   f_out                        the forces F at xq (may be NULL).
 * Real space (LJ, Ewald direct, exclusion correction) in one pass over the list; with
 * NB_TERM_PME the reciprocal part: with psi(k) = sum_i q_i lam_i . grad theta_i(k) spread
 * on a second mesh and chi = C psi (C the PME convolution),
 *   gx_j -= q_j sum_k (Hess theta_j(k) lam_j) phi(k) + q_j sum_k grad theta_j(k) chi(k),
 *   gq_j -= sum_k (lam_j . grad theta_j(k)) phi(k) + sum_k theta_j(k) chi(k).
 * All outputs are overwritten, (device) FP32.
 */
nb_status nonbonded_force_vjp(nb_handle* h, const float* xq, const float* lam, float* gx, float* gq,
                              float* gsigma, float* gsqrt_eps, float* f_out, int32_t terms, void* stream);

/*
 * PME charge spreading without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code whose device
 * memory is owned by another allocator (a framework's memory pool, a fixed arena) and
 * code that must not trigger the device-wide synchronisation an allocation can cause.
 * Every handle-based call in this header needs nb_create, which allocates; this one needs
 * no handle.  It computes the same mesh as pme_spread for one periodic system:
 *   xq [n_atoms][4]   (device) positions and charges; may be NULL when n_atoms is 0,
 *                     which gives an all-zero mesh.
 *   box[3] (host)     box edge lengths;  mesh[3] (host) K0, K1, K2, each >= 4.
 *   grid              (device, caller-owned) float[K0*K1*K2], index ((k0*K1)+k1)*K2+k2.
 * Its int64 accumulation mesh is a library-owned static device array of
 * NB_STATIC_MESH_MAX points (8 MiB on every GPU that loads the library, held until the
 * process exits); a mesh of more points (K0*K1*K2 > NB_STATIC_MESH_MAX, any Kd above it
 * included) returns NB_ERR_ARG before any GPU work.  Every call looks the array's address
 * up in the current context (cudaGetSymbolAddress, which allocates nothing), so a device
 * reset between calls is harmless; the first call on a device may load the library's GPU
 * code, so make it before any stream capture.  Every call clears the part of the array it
 * uses and shares the array with every other call: calls whose executions overlap on the
 * GPU (several streams, or several host threads) race and corrupt each other's result.
 */
#define NB_STATIC_MESH_MAX (1 << 20)
nb_status pme_spread_static(const float* xq, int32_t n_atoms, const double* box, const int32_t* mesh,
                            float* grid, void* stream);

/* Thread blocks per cell the handle uses in the list build (nb_options.blocks_per_cell, or
 * the automatic choice); `pair` is 1 (the pair and VJP kernels take consecutive atoms per
 * block, not cells).  Host only, no GPU work. */
nb_status nb_blocks_per_cell(const nb_handle* h, int32_t* build, int32_t* pair);

/* Cumulative number of neighbour-list rebuilds of a handle (synchronises `stream`). */
int64_t nb_rebuild_count(nb_handle* h, void* stream);

/*
 * Per-stage timing (a profiling aid; the paper reports runtimes only).  While enabled,
 * every entry point brackets the kernels of each stage with CUDA events on its stream.
 * nb_timing_read synchronises `stream`, returns the summed device milliseconds and the
 * number of timed intervals per stage since the previous read (host arrays of
 * NB_NSTAGES), and resets them.  Do not enable it while capturing a CUDA graph.
 */
#define NB_STAGE_CHECK 0     /* list validity test + scatter of positions to slot order */
#define NB_STAGE_REBUILD 1   /* cell binning, scan, scatter, in-cell sort, Verlet list build */
#define NB_STAGE_PAIR 2      /* fused LJ + Ewald-direct + exclusion pair kernel (or its VJP) */
#define NB_STAGE_SPREAD 3    /* PME charge spreading and mesh conversion */
#define NB_STAGE_FFT 4       /* cuFFT transforms (reported separately, not our kernels) */
#define NB_STAGE_CONVOLVE 5  /* PME influence function and reciprocal energy */
#define NB_STAGE_GATHER 6    /* PME force gathering */
#define NB_STAGE_UPDATE 7    /* reductions, force output, integrator updates */
#define NB_STAGE_BUILD 8     /* the Verlet list build kernel alone (also inside NB_STAGE_REBUILD); it
                                also re-partitions the rows of dynamic list pruning when due */
#define NB_NSTAGES 9
nb_status nb_timing_enable(nb_handle* h, int32_t enable);
nb_status nb_timing_read(nb_handle* h, void* stream, double* ms, int64_t* intervals);

#ifdef __cplusplus
}
#endif

#endif /* NBCORE_H */
