/*
 * oracle.c -- plain FP64 CPU reference for the nonbonded force path of
 * arXiv 2503.20541 (DIMOS), Sec. 2.1.2 "Nonbonded Interactions".
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline arm of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA library (paper_2503_20541_b300).
 *
 * Everything here is the literal definition: O(N^2) loops over all atom
 * pairs under the minimum-image convention, no neighbour lists, no blocking,
 * FP64 throughout.  The one exception, orc_nonbonded_cells, visits only the
 * candidates of a plain cell list (for CPU timings at large N) and is pinned
 * equal to the all-pairs routine.  Pins (closed forms, finite differences,
 * lattice sums) live in tests/test_oracle_pins.py.
 *
 * Conventions
 *   positions x[3*i+d]; the pair vector is d_ij = mi(x_i - x_j),
 *   mi(a) = a - L*round(a/L) per axis for periodic systems (orthorhombic box,
 *   the distance routine of Sec. 2.1.1 / Sec. 2.1.2 "Neighborlists").
 *   A pair force is written F_i = f(r) d_ij, F_j = -f(r) d_ij with
 *   f(r) = -U'(r)/r.
 *   Exclusions are a CSR list (ex_off[n+1], ex_idx[]); a pair is excluded if
 *   either atom lists the other (Sec. 2.1.2 "Exclusions and Exceptions").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    double box[3];     /* orthorhombic box edge lengths */
    int32_t periodic;  /* 1: minimum image; 0: open system */
    int32_t pad_;
    double r_cut;      /* r_c: pairs with r < r_c interact (strict) */
    double r_switch;   /* r_s of the LJ switch S(x); < 0 disables it */
    double alpha;      /* Ewald splitting parameter; 0 = bare truncated Coulomb */
    double ke;         /* Coulomb constant 1/(4 pi eps0) in the caller's units */
    double eps_rf;     /* reaction field: solvent dielectric eps_s (> 0 selects it, alpha = 0) */
} orc_params;

static double mi(double a, double L, int periodic) {
    return periodic ? a - L * nearbyint(a / L) : a;
}

static void pair_vec(const double* x, int i, int j, const orc_params* p, double d[3]) {
    for (int k = 0; k < 3; ++k) d[k] = mi(x[3 * i + k] - x[3 * j + k], p->box[k], p->periodic);
}

static int excluded(int i, int j, const int32_t* ex_off, const int32_t* ex_idx) {
    if (!ex_off) return 0;
    for (int32_t e = ex_off[i]; e < ex_off[i + 1]; ++e) if (ex_idx[e] == j) return 1;
    for (int32_t e = ex_off[j]; e < ex_off[j + 1]; ++e) if (ex_idx[e] == i) return 1;
    return 0;
}

/* ---- Lennard-Jones, Eq. (lj), with Lorentz-Berthelot mixing and the ----
 * ---- OpenMM-style switch S(x) = 1 - 6x^5 + 15x^4 - 10x^3 (Sec. 2.1.2) --- */

/* Switch value and derivatives wrt r: S, dS/dr, d2S/dr2. */
static void lj_switch(double r, double rc, double rs, double* S, double* dS, double* d2S) {
    if (rs < 0.0 || r <= rs) { *S = 1.0; *dS = 0.0; *d2S = 0.0; return; }
    double w = rc - rs, x = (r - rs) / w;
    double x2 = x * x, x3 = x2 * x, x4 = x3 * x, x5 = x4 * x;
    *S = 1.0 - 6.0 * x5 + 15.0 * x4 - 10.0 * x3;
    *dS = (-30.0 * x4 + 60.0 * x3 - 30.0 * x2) / w;
    *d2S = (-120.0 * x3 + 180.0 * x2 - 60.0 * x) / (w * w);
}

/* Switched LJ energy W = U*S and W', W''; also dW/dsigma and dW'/dsigma
 * (derivatives with respect to the mixed sigma_ij). */
static void lj_terms(double r, double sig, double eps, double rc, double rs,
                     double* W, double* dW, double* d2W, double* dWs, double* dWps) {
    double sr = sig / r;
    double s6 = pow(sr, 6.0), s12 = s6 * s6;
    double U = 4.0 * eps * (s12 - s6);
    double dU = 4.0 * eps * (-12.0 * s12 + 6.0 * s6) / r;
    double d2U = 4.0 * eps * (156.0 * s12 - 42.0 * s6) / (r * r);
    double Us = 4.0 * eps * (12.0 * s12 - 6.0 * s6) / sig;           /* dU/dsig */
    double dUs = 4.0 * eps * (-144.0 * s12 + 36.0 * s6) / (r * sig);  /* dU'/dsig */
    double S, dS, d2S;
    lj_switch(r, rc, rs, &S, &dS, &d2S);
    *W = U * S;
    *dW = dU * S + U * dS;
    *d2W = d2U * S + 2.0 * dU * dS + U * d2S;
    *dWs = Us * S;
    *dWps = dUs * S + Us * dS;
}

/* ---- Ewald direct-space kernel g(r) = erfc(alpha r)/r and derivatives ---- */
static void erfc_terms(double r, double a, double* g, double* dg, double* d2g) {
    double ec = erfc(a * r);
    double gau = (a > 0.0) ? 2.0 * a / sqrt(ORC_PI) * exp(-a * a * r * r) : 0.0;
    *g = ec / r;
    *dg = -ec / (r * r) - gau / r;
    *d2g = 2.0 * ec / (r * r * r) + 2.0 * gau / (r * r) + 2.0 * a * a * gau;
}

/* ---- Reaction field (RFA, Sec. 2.1.2): g(r) = 1/r + k r^2 - c, r < r_c, with
 * k = (eps_s - 1) / ((2 eps_s + 1) r_c^3) and c = 3 eps_s / ((2 eps_s + 1) r_c), so that
 * g(r_c) = 0 (the printed denominators 2 eps + 1 read as 2 eps_s + 1, which is what makes
 * c = 1/r_c + k r_c^2). ---- */
static void rf_terms(double r, double rc, double eps_s, double* g, double* dg, double* d2g) {
    double k = (eps_s - 1.0) / ((2.0 * eps_s + 1.0) * rc * rc * rc);
    double c = 3.0 * eps_s / ((2.0 * eps_s + 1.0) * rc);
    *g = 1.0 / r + k * r * r - c;
    *dg = -1.0 / (r * r) + 2.0 * k * r;
    *d2g = 2.0 / (r * r * r) + 2.0 * k;
}

/* Coulomb pair kernel of the selected electrostatics: reaction field when eps_rf > 0,
 * else the Ewald direct term (bare 1/r for alpha = 0). */
static void coul_terms(double r, const orc_params* p, double* g, double* dg, double* d2g) {
    if (p->eps_rf > 0.0) rf_terms(r, p->r_cut, p->eps_rf, g, dg, d2g);
    else erfc_terms(r, p->alpha, g, dg, d2g);
}

/*
 * Full nonbonded energy and forces (definition, all pairs i<j):
 *   E_lj   = sum_{r<rc, not excl} 4 eps_ij[(s/r)^12-(s/r)^6] S      Eq. (lj)
 *   E_dir  = sum_{r<rc, not excl} ke q_i q_j erfc(alpha r)/r         Ewald U_dir
 *   E_excl = -sum_{excl} ke q_i q_j erf(alpha r)/r     (excluded pairs leave the
 *            real-space sum but remain in the reciprocal sum; subtracting their
 *            smooth part makes the total equal to "all charges minus the bare
 *            Coulomb of excluded pairs")
 *   E_self = -ke alpha/sqrt(pi) sum_i q_i^2                          Ewald U_self
 * With the reaction field (eps_rf > 0) E_dir is sum_{r<rc, not excl} ke q_i q_j
 * (1/r + k r^2 - c), Eq. (RFA), and excluded pairs do not interact (no reciprocal sum
 * to correct, no self term).
 * energy[0..3] = E_lj, E_dir, E_excl, E_self.  f[3n] = -grad E.
 */
int orc_nonbonded(int n, const double* x, const double* q, const double* sig, const double* sqe,
                  const orc_params* p, const int32_t* ex_off, const int32_t* ex_idx,
                  double* energy, double* f) {
    double elj = 0.0, edir = 0.0, eex = 0.0, eself = 0.0;
    double rc2 = p->r_cut * p->r_cut;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        for (int j = i + 1; j < n; ++j) {
            double d[3];
            pair_vec(x, i, j, p, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            double dU = 0.0;
            if (excluded(i, j, ex_off, ex_idx)) {
                double c = p->ke * q[i] * q[j];
                if (c != 0.0 && p->alpha > 0.0) {
                    double g, dg, d2g;
                    erfc_terms(r, p->alpha, &g, &dg, &d2g);
                    /* -c erf(ar)/r = c (g - 1/r) */
                    eex += c * (g - 1.0 / r);
                    dU += c * (dg + 1.0 / r2);
                }
            } else if (r2 < rc2) {
                double eps = sqe[i] * sqe[j], s = 0.5 * (sig[i] + sig[j]);
                if (eps != 0.0) {
                    double W, dW, d2W, dWs, dWps;
                    lj_terms(r, s, eps, p->r_cut, p->r_switch, &W, &dW, &d2W, &dWs, &dWps);
                    elj += W;
                    dU += dW;
                }
                double c = p->ke * q[i] * q[j];
                if (c != 0.0) {
                    double g, dg, d2g;
                    coul_terms(r, p, &g, &dg, &d2g);
                    edir += c * g;
                    dU += c * dg;
                }
            }
            double fs = -dU / r;
            for (int k = 0; k < 3; ++k) {
                f[3 * i + k] += fs * d[k];
                f[3 * j + k] -= fs * d[k];
            }
        }
    }
    for (int i = 0; i < n; ++i) eself += q[i] * q[i];
    eself *= -p->ke * p->alpha / sqrt(ORC_PI);
    energy[0] = elj; energy[1] = edir; energy[2] = eex; energy[3] = eself;
    return 0;
}

/*
 * Row variant: for each listed atom i, the force on i summed over all j != i
 * (no Newton-III sharing), and half the pair energies of i's pairs
 * (energy_rows[3*r + 0..2] = E_lj, E_dir, E_excl halves).  Rows are
 * independent, so they run in parallel; every row is the same definition as
 * orc_nonbonded.  Used for sampled checks at full size and for the CPU
 * baseline timing.
 */
int orc_nonbonded_rows(int n, const double* x, const double* q, const double* sig, const double* sqe,
                       const orc_params* p, const int32_t* ex_off, const int32_t* ex_idx,
                       int n_rows, const int32_t* rows, double* energy_rows, double* f_rows) {
    double rc2 = p->r_cut * p->r_cut;
#pragma omp parallel for schedule(dynamic, 4)
    for (int rr = 0; rr < n_rows; ++rr) {
        int i = rows[rr];
        double fi[3] = {0.0, 0.0, 0.0}, elj = 0.0, edir = 0.0, eex = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            pair_vec(x, i, j, p, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            double dU = 0.0;
            if (excluded(i, j, ex_off, ex_idx)) {
                double c = p->ke * q[i] * q[j];
                if (c != 0.0 && p->alpha > 0.0) {
                    double g, dg, d2g;
                    erfc_terms(r, p->alpha, &g, &dg, &d2g);
                    eex += 0.5 * c * (g - 1.0 / r);
                    dU += c * (dg + 1.0 / r2);
                }
            } else if (r2 < rc2) {
                double eps = sqe[i] * sqe[j], s = 0.5 * (sig[i] + sig[j]);
                if (eps != 0.0) {
                    double W, dW, d2W, dWs, dWps;
                    lj_terms(r, s, eps, p->r_cut, p->r_switch, &W, &dW, &d2W, &dWs, &dWps);
                    elj += 0.5 * W;
                    dU += dW;
                }
                double c = p->ke * q[i] * q[j];
                if (c != 0.0) {
                    double g, dg, d2g;
                    coul_terms(r, p, &g, &dg, &d2g);
                    edir += 0.5 * c * g;
                    dU += c * dg;
                }
            }
            double fs = -dU / r;
            for (int k = 0; k < 3; ++k) fi[k] += fs * d[k];
        }
        for (int k = 0; k < 3; ++k) f_rows[3 * rr + k] = fi[k];
        energy_rows[3 * rr + 0] = elj;
        energy_rows[3 * rr + 1] = edir;
        energy_rows[3 * rr + 2] = eex;
    }
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops that follow (for single-thread timings). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Cell-list variant of orc_nonbonded_rows over all atoms, the neighbour search of
 * Sec. 2.1.2 "Neighborlists" (cells of edge >= r_c, the 27 cells around an atom's cell):
 * the same pair terms as the row routine, visiting only the candidates the cells can
 * hold within r_c, plus every excluded partner at any distance.  It is a second route to
 * the same definition (pinned equal to orc_nonbonded), kept for CPU timings at sizes the
 * O(N^2) loops cannot reach.  Open systems and boxes with fewer than 3 cells along an
 * axis take the row routine.  Outputs: f[3 n] (force on every atom) and energy[4] (E_lj,
 * E_dir, E_excl from the per-atom halves summed in atom order, and E_self), the layout
 * of orc_nonbonded.
 */
int orc_nonbonded_cells(int n, const double* x, const double* q, const double* sig, const double* sqe,
                        const orc_params* p, const int32_t* ex_off, const int32_t* ex_idx, double* energy,
                        double* f) {
    energy[0] = energy[1] = energy[2] = energy[3] = 0.0;
    if (n <= 0) return 0;
    int nc[3];
    int ok = p->periodic;
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(p->box[k] / p->r_cut);
        /* a cell edge equal to r_c up to rounding could let a pair inside r_c sit two
         * cells apart: keep every edge clearly above r_c */
        while (nc[k] > 0 && p->box[k] / nc[k] < p->r_cut * (1.0 + 1e-9)) --nc[k];
        if (nc[k] < 3) ok = 0;
    }
    double* er = (double*)calloc((size_t)3 * n, sizeof(double));
    if (!er) return -1;
    if (!ok) {
        int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!rows) { free(er); return -1; }
        for (int i = 0; i < n; ++i) rows[i] = i;
        orc_nonbonded_rows(n, x, q, sig, sqe, p, ex_off, ex_idx, n, rows, er, f);
        free(rows);
    } else {
        const int ncell = nc[0] * nc[1] * nc[2];
        int* cell = (int*)malloc(sizeof(int) * (size_t)n);
        int* start = (int*)calloc((size_t)ncell + 1, sizeof(int));
        int* order = (int*)malloc(sizeof(int) * (size_t)n);
        /* symmetric partner lists: j is a partner of i if either lists the other */
        int* pcnt = (int*)calloc((size_t)n + 1, sizeof(int));
        int n_ex = ex_off ? ex_off[n] : 0;
        int* pidx = (int*)malloc(sizeof(int) * (size_t)(2 * n_ex + 1));
        if (!cell || !start || !order || !pcnt || !pidx) {
            free(er); free(cell); free(start); free(order); free(pcnt); free(pidx);
            return -1;
        }
        for (int i = 0; i < n; ++i) {
            int c[3];
            for (int k = 0; k < 3; ++k) {
                double u = x[3 * i + k] - p->box[k] * floor(x[3 * i + k] / p->box[k]);
                c[k] = (int)floor(u * nc[k] / p->box[k]);
                if (c[k] >= nc[k]) c[k] = nc[k] - 1;
                if (c[k] < 0) c[k] = 0;
            }
            cell[i] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
            start[cell[i] + 1] += 1;
        }
        for (int c = 0; c < ncell; ++c) start[c + 1] += start[c];
        {
            int* fill = (int*)malloc(sizeof(int) * (size_t)ncell);
            if (!fill) { free(er); free(cell); free(start); free(order); free(pcnt); free(pidx); return -1; }
            memcpy(fill, start, sizeof(int) * (size_t)ncell);
            for (int i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
            free(fill);
        }
        for (int i = 0; i < n && ex_off; ++i)
            for (int32_t e = ex_off[i]; e < ex_off[i + 1]; ++e) {
                pcnt[i + 1] += 1;
                pcnt[ex_idx[e] + 1] += 1;
            }
        for (int i = 0; i < n; ++i) pcnt[i + 1] += pcnt[i];
        {
            int* fill = (int*)malloc(sizeof(int) * (size_t)(n + 1));
            if (!fill) { free(er); free(cell); free(start); free(order); free(pcnt); free(pidx); return -1; }
            memcpy(fill, pcnt, sizeof(int) * (size_t)(n + 1));
            for (int i = 0; i < n && ex_off; ++i)
                for (int32_t e = ex_off[i]; e < ex_off[i + 1]; ++e) {
                    pidx[fill[i]++] = ex_idx[e];
                    pidx[fill[ex_idx[e]]++] = i;
                }
            free(fill);
        }
        const double rc2 = p->r_cut * p->r_cut;
#pragma omp parallel for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            double fi[3] = {0.0, 0.0, 0.0}, elj = 0.0, edir = 0.0, eex = 0.0;
            const int c0 = cell[i] % nc[0], c1 = (cell[i] / nc[0]) % nc[1], c2 = cell[i] / (nc[0] * nc[1]);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int a = (c0 + dx + nc[0]) % nc[0], b = (c1 + dy + nc[1]) % nc[1];
                        const int cc = (((c2 + dz + nc[2]) % nc[2]) * nc[1] + b) * nc[0] + a;
                        for (int s = start[cc]; s < start[cc + 1]; ++s) {
                            const int j = order[s];
                            if (j == i || excluded(i, j, ex_off, ex_idx)) continue;
                            double d[3];
                            pair_vec(x, i, j, p, d);
                            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (!(r2 < rc2)) continue;
                            double r = sqrt(r2), dU = 0.0;
                            double eps = sqe[i] * sqe[j], sg = 0.5 * (sig[i] + sig[j]);
                            if (eps != 0.0) {
                                double W, dW, d2W, dWs, dWps;
                                lj_terms(r, sg, eps, p->r_cut, p->r_switch, &W, &dW, &d2W, &dWs, &dWps);
                                elj += 0.5 * W;
                                dU += dW;
                            }
                            double cq = p->ke * q[i] * q[j];
                            if (cq != 0.0) {
                                double g, dg, d2g;
                                coul_terms(r, p, &g, &dg, &d2g);
                                edir += 0.5 * cq * g;
                                dU += cq * dg;
                            }
                            double fs = -dU / r;
                            for (int k = 0; k < 3; ++k) fi[k] += fs * d[k];
                        }
                    }
            /* excluded partners at any distance (each once, however often listed) */
            for (int e = pcnt[i]; e < pcnt[i + 1]; ++e) {
                const int j = pidx[e];
                int seen = 0;
                for (int e2 = pcnt[i]; e2 < e; ++e2) seen |= pidx[e2] == j;
                if (seen || j == i) continue;
                double cq = p->ke * q[i] * q[j];
                if (cq == 0.0 || !(p->alpha > 0.0)) continue;
                double d[3];
                pair_vec(x, i, j, p, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
                double g, dg, d2g;
                erfc_terms(r, p->alpha, &g, &dg, &d2g);
                eex += 0.5 * cq * (g - 1.0 / r);
                double fs = -(cq * (dg + 1.0 / r2)) / r;
                for (int k = 0; k < 3; ++k) fi[k] += fs * d[k];
            }
            for (int k = 0; k < 3; ++k) f[3 * i + k] = fi[k];
            er[3 * i + 0] = elj;
            er[3 * i + 1] = edir;
            er[3 * i + 2] = eex;
        }
        free(cell); free(start); free(order); free(pcnt); free(pidx);
    }
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) energy[k] += er[3 * i + k];
        energy[3] += q[i] * q[i];
    }
    energy[3] *= -p->ke * p->alpha / sqrt(ORC_PI);
    free(er);
    return 0;
}

/*
 * Exact Ewald reciprocal-space energy and forces by the structure-factor sum
 * (Ewald U_recip of Sec. 2.1.2, written in its standard form):
 *   E = ke/(2 pi V) sum_{m != 0} exp(-pi^2 |m|^2/alpha^2)/|m|^2 |S(m)|^2,
 *   S(m) = sum_j q_j exp(2 pi i m.x_j),   m = (n1/L1, n2/L2, n3/L3),
 * with |n_d| <= mmax[d].  m and -m give equal terms, so the loop runs over a
 * half space and doubles.
 */
int orc_ewald_recip(int n, const double* x, const double* q, const double* box, double alpha,
                    double ke, const int32_t* mmax, double* energy, double* f) {
    double V = box[0] * box[1] * box[2];
    double e = 0.0;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    double* th = (double*)malloc(sizeof(double) * (size_t)n);
    for (int n1 = 0; n1 <= mmax[0]; ++n1)
        for (int n2 = -mmax[1]; n2 <= mmax[1]; ++n2)
            for (int n3 = -mmax[2]; n3 <= mmax[2]; ++n3) {
                int upper = (n1 > 0) || (n1 == 0 && n2 > 0) || (n1 == 0 && n2 == 0 && n3 > 0);
                if (!upper) continue;
                double m[3] = {n1 / box[0], n2 / box[1], n3 / box[2]};
                double m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
                double pref = exp(-ORC_PI * ORC_PI * m2 / (alpha * alpha)) / m2;
                double A = 0.0, B = 0.0;
                for (int j = 0; j < n; ++j) {
                    th[j] = 2.0 * ORC_PI * (m[0] * x[3 * j] + m[1] * x[3 * j + 1] + m[2] * x[3 * j + 2]);
                    A += q[j] * cos(th[j]);
                    B += q[j] * sin(th[j]);
                }
                e += 2.0 * pref * (A * A + B * B);
                /* -dE/dx_i for the m and -m terms together */
                double c = 2.0 * 2.0 * ke / V * pref;
                for (int i = 0; i < n; ++i) {
                    double t = q[i] * (A * sin(th[i]) - B * cos(th[i]));
                    for (int k = 0; k < 3; ++k) f[3 * i + k] += c * t * m[k];
                }
            }
    free(th);
    *energy = e * ke / (2.0 * ORC_PI * V);
    return 0;
}

/*
 * Neighbour set (Sec. 2.1.2 "Neighborlists"): all unordered pairs i<j, not
 * excluded, with |mi(x_i - x_j)|^2 < r_nl^2, r_nl = r_c + r_g.  Writes up to
 * cap pairs (i, j) and returns the total count.  n_band counts pairs with
 * | r^2 - r_nl^2 | <= band: their membership may legitimately differ between
 * an FP64 and an FP32 evaluation of r^2.
 */
int64_t orc_neighbor_pairs(int n, const double* x, const orc_params* p, double r_nl,
                           const int32_t* ex_off, const int32_t* ex_idx, int64_t cap,
                           int32_t* pairs, double band, int64_t* n_band) {
    int64_t cnt = 0, nb = 0;
    double rn2 = r_nl * r_nl;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double d[3];
            pair_vec(x, i, j, p, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (excluded(i, j, ex_off, ex_idx)) continue;
            if (fabs(r2 - rn2) <= band) ++nb;
            if (r2 < rn2) {
                if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
                ++cnt;
            }
        }
    if (n_band) *n_band = nb;
    return cnt;
}

/*
 * Force vector-Jacobian product of the real-space terms (LJ, Ewald direct or
 * reaction field, exclusion correction).  For the pair Jacobian
 *   J = dF_i/dx_i = f(r) I + (f'(r)/r) d d^T,   dF_i/dx_j = -J,
 * the product with a cotangent lam gives
 *   gx_i += J (lam_i - lam_j),  gx_j -= J (lam_i - lam_j).
 * Parameter gradients of lam.F = sum_pairs f(r) d.(lam_i - lam_j):
 *   gq, gsig (wrt sigma_i), gsqe (wrt sqrt(eps_i)).
 */
int orc_force_vjp(int n, const double* x, const double* q, const double* sig, const double* sqe,
                  const orc_params* p, const int32_t* ex_off, const int32_t* ex_idx,
                  const double* lam, double* gx, double* gq, double* gsig, double* gsqe) {
    double rc2 = p->r_cut * p->r_cut;
    memset(gx, 0, sizeof(double) * 3 * (size_t)n);
    memset(gq, 0, sizeof(double) * (size_t)n);
    memset(gsig, 0, sizeof(double) * (size_t)n);
    memset(gsqe, 0, sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double d[3];
            pair_vec(x, i, j, p, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            double u[3] = {lam[3 * i] - lam[3 * j], lam[3 * i + 1] - lam[3 * j + 1],
                           lam[3 * i + 2] - lam[3 * j + 2]};
            double du = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
            double dU = 0.0, d2U = 0.0;
            if (excluded(i, j, ex_off, ex_idx)) {
                double c = p->ke * q[i] * q[j];
                if (p->alpha > 0.0 && p->ke != 0.0) {
                    double g, dg, d2g;
                    erfc_terms(r, p->alpha, &g, &dg, &d2g);
                    double dUc = dg + 1.0 / r2, d2Uc = d2g - 2.0 / (r2 * r);
                    dU += c * dUc;
                    d2U += c * d2Uc;
                    /* d(f d.u)/dq_i with f = -U'/r, U linear in q_i */
                    gq[i] += -p->ke * q[j] * dUc / r * du;
                    gq[j] += -p->ke * q[i] * dUc / r * du;
                }
            } else if (r2 < rc2) {
                double eps = sqe[i] * sqe[j], s = 0.5 * (sig[i] + sig[j]);
                {
                    /* W is linear in eps = sqe_i sqe_j: evaluate at eps = 1 and scale */
                    double W1, dW1, d2W1, dWs1, dWps1;
                    lj_terms(r, s, 1.0, p->r_cut, p->r_switch, &W1, &dW1, &d2W1, &dWs1, &dWps1);
                    dU += eps * dW1;
                    d2U += eps * d2W1;
                    gsqe[i] += -sqe[j] * dW1 / r * du;
                    gsqe[j] += -sqe[i] * dW1 / r * du;
                    gsig[i] += -0.5 * eps * dWps1 / r * du;
                    gsig[j] += -0.5 * eps * dWps1 / r * du;
                }
                double c = p->ke * q[i] * q[j];
                if (p->ke != 0.0) {
                    double g, dg, d2g;
                    coul_terms(r, p, &g, &dg, &d2g);
                    dU += c * dg;
                    d2U += c * d2g;
                    gq[i] += -p->ke * q[j] * dg / r * du;
                    gq[j] += -p->ke * q[i] * dg / r * du;
                }
            } else {
                continue;
            }
            double fs = -dU / r;
            double dfs = -d2U / r + dU / r2; /* f'(r) */
            double k2 = dfs / r * du;
            for (int k = 0; k < 3; ++k) {
                double ju = fs * u[k] + k2 * d[k];
                gx[3 * i + k] += ju;
                gx[3 * j + k] -= ju;
            }
        }
    return 0;
}
