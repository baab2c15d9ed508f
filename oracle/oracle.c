/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for many-body MD with the
 * Tersoff and Stillinger-Weber potentials.  TEST INFRASTRUCTURE ONLY: it may be
 * called from tests/, from __graft_entry__.smoke() and from bench.py's CPU-baseline /
 * reference legs, and from nothing else.  It shares no code, header, table or constant
 * generator with the CUDA library; the two only see the same seeded inputs.
 *
 * What it computes (Fan, Chen, Vierimaa, Harju, CPC 2017, arXiv:1610.03343):
 *   - neighbour lists by brute force and by a textbook linked-list cell method
 *     (Sec. 2.1: "a Verlet neighbour list ... the standard cell list method"),
 *     minimum image on periodic axes (Algorithm 2 / Algorithm 3 minimum-image step);
 *   - Tersoff energy, Eqs. 1-6, with f_R, f_A, f_C in the forms of Tersoff 1989
 *     (the paper names but does not print them);
 *   - the conventional force loop of Algorithm 1 with the partial forces of
 *     Eqs. 7-11: per-atom energy U_i, forces F_i, the LAMMPS-style per-atom virial of
 *     Eq. 22 and the total virial;
 *   - an independent per-atom derivative routine dU_i/dr_ij (the quantity Eq. 14 and
 *     Eqs. 28-30 are written in; the paper defers its explicit form to its Ref. fan2015,
 *     so it is derived here by differentiating U_i = 1/2 sum_j U_ij with respect to
 *     atom i's own bond vectors);
 *   - the many-body per-atom force, virial and heat current of Eqs. 28-30 from it;
 *   - the same two routes for Stillinger-Weber (Stillinger & Weber 1985 energy; the
 *     three-body term is assigned to its vertex atom);
 *   - velocity-Verlet integration (Sec. 3), neighbour lists rebuilt every step, and
 *     the Berendsen thermostat and barostat of the paper's NPT runs (Sec. 3).
 *
 * Conventions: r_ij = r_j - r_i (Sec. 2.1, below Eq. 6).  Per-atom arrays are SoA
 * (x[0..N), y, z; 3-vectors as F[0..N) = Fx, F[N..2N) = Fy, F[2N..3N) = Fz).  Per-atom
 * tensors are 9 x N, component (a,b) at [(3a+b)N + i], (u (x) w)_ab = u_a w_b.
 * Neighbour lists are "column-major" like the paper's NL_im: NL[m N + i], ascending j.
 * Units: Angstrom, eV, amu, fs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* eV/(Angstrom amu) in Angstrom/fs^2: 1.602176634e-19 J / (1e-10 m 1.66053906660e-27 kg)
 * = 9.648533215665e17 m/s^2, times 1e10 A/m and 1e-30 s^2/fs^2. */
static const double ACC_UNIT = 9.648533215665328e-3;

/* ------------------------------------------------------------------ vectors */
static void vsub(const double *a, const double *b, double *c) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static double vdot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double vnorm(const double *a) { return sqrt(vdot(a, a)); }

static void get_pos(int64_t N, const double *x, const double *y, const double *z, int64_t i, double *r)
{
    (void)N;
    r[0] = x[i]; r[1] = y[i]; r[2] = z[i];
}

/* Minimum image for an orthorhombic box with coordinates wrapped into [0, L):
 * every component then lies in (-L, L), and one shift by L brings it into [-L/2, L/2]. */
static void min_image(const double *box, const int *pbc, double *d)
{
    for (int a = 0; a < 3; ++a) {
        if (!pbc[a]) continue;
        if (d[a] > 0.5 * box[a]) d[a] -= box[a];
        else if (d[a] < -0.5 * box[a]) d[a] += box[a];
    }
}

/* r_ij = minimum image of r_j - r_i */
static void bond(int64_t N, const double *x, const double *y, const double *z,
                 const double *box, const int *pbc, int64_t i, int64_t j, double *rij)
{
    double ri[3], rj[3];
    get_pos(N, x, y, z, i, ri);
    get_pos(N, x, y, z, j, rj);
    vsub(rj, ri, rij);
    min_image(box, pbc, rij);
}

/* --------------------------------------------------------- neighbour lists */
/* Insert j into i's list keeping ascending order.  Returns the new count (which can
 * exceed cap: entries past cap are dropped, the count still reports them). */
static int list_insert(int64_t N, int *NL, int cap, int count, int64_t i, int j)
{
    if (count < cap) {
        int m = count;
        while (m > 0 && NL[(int64_t)(m - 1) * N + i] > j) {
            NL[(int64_t)m * N + i] = NL[(int64_t)(m - 1) * N + i];
            --m;
        }
        NL[(int64_t)m * N + i] = j;
    }
    return count + 1;
}

/* Brute force O(N^2): j in NL_i iff j != i and |r_ij| < rc (minimum image).
 * Returns the largest count over atoms (> cap means some list overflowed). */
int oracle_neighbors_brute(int64_t N, const double *x, const double *y, const double *z,
                           const double *box, const int *pbc, double rc, int cap,
                           int *NN, int *NL)
{
    int maxc = 0;
    for (int64_t i = 0; i < N; ++i) {
        int c = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double rij[3];
            bond(N, x, y, z, box, pbc, i, j, rij);
            if (vdot(rij, rij) < rc * rc) c = list_insert(N, NL, cap, c, i, (int)j);
        }
        NN[i] = c < cap ? c : cap;
        if (c > maxc) maxc = c;
    }
    return maxc;
}

/* Textbook linked-list cells (head/next): cells of edge >= rc on each axis; an atom's
 * candidates are the atoms in its own and the adjacent cells, each distinct cell once
 * (fewer than 3 cells along an axis means fewer distinct neighbours along it).  Atoms
 * outside [0, L) on a non-periodic axis are clamped into the edge cell. */
int oracle_neighbors_cells(int64_t N, const double *x, const double *y, const double *z,
                           const double *box, const int *pbc, double rc, int cap,
                           int *NN, int *NL)
{
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(box[a] / rc);
        if (nc[a] < 1) nc[a] = 1;
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int *cell = (int *)malloc(sizeof(int) * 3 * (size_t)(N > 0 ? N : 1));
    if (!head || !next || !cell) { free(head); free(next); free(cell); return -1; }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = 0; i < N; ++i) {
        double r[3];
        get_pos(N, x, y, z, i, r);
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            int k = (int)floor(r[a] / box[a] * nc[a]);
            if (k < 0) k = 0;
            if (k > nc[a] - 1) k = nc[a] - 1;
            ci[a] = k;
            cell[3 * i + a] = k;
        }
        int64_t c = ((int64_t)ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        next[i] = head[c];
        head[c] = i;
    }
    int maxc = 0;
    for (int64_t i = 0; i < N; ++i) {
        int off[3][3], noff[3];
        for (int a = 0; a < 3; ++a) {
            /* distinct neighbouring cell indices along axis a */
            int cand[3] = {cell[3 * i + a] - 1, cell[3 * i + a], cell[3 * i + a] + 1};
            noff[a] = 0;
            for (int t = 0; t < 3; ++t) {
                int k = cand[t];
                if (pbc[a]) k = ((k % nc[a]) + nc[a]) % nc[a];
                else if (k < 0 || k >= nc[a]) continue;
                int dup = 0;
                for (int u = 0; u < noff[a]; ++u) if (off[a][u] == k) dup = 1;
                if (!dup) off[a][noff[a]++] = k;
            }
        }
        int c = 0;
        for (int p = 0; p < noff[0]; ++p)
            for (int q = 0; q < noff[1]; ++q)
                for (int s = 0; s < noff[2]; ++s) {
                    int64_t cc = ((int64_t)off[0][p] * nc[1] + off[1][q]) * nc[2] + off[2][s];
                    for (int64_t j = head[cc]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double rij[3];
                        bond(N, x, y, z, box, pbc, i, j, rij);
                        if (vdot(rij, rij) < rc * rc) c = list_insert(N, NL, cap, c, i, (int)j);
                    }
                }
        NN[i] = c < cap ? c : cap;
        if (c > maxc) maxc = c;
    }
    free(head); free(next); free(cell);
    return maxc;
}

/* slot of i in j's list, or -1 */
static int find_slot(int64_t N, const int *NN, const int *NL, int64_t j, int64_t i)
{
    for (int m = 0; m < NN[j]; ++m)
        if (NL[(int64_t)m * N + j] == (int)i) return m;
    return -1;
}

/* ------------------------------------------------------------------ Tersoff */
/* Packed parameters: A, B, lambda, mu, beta, n, c, d, h, R, S (Tersoff 1989). */
typedef struct { double A, B, lam, mu, beta, n, c, d, h, R, S; } tersoff_t;

static tersoff_t tersoff_unpack(const double *p)
{
    tersoff_t t = {p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8], p[9], p[10]};
    return t;
}

/* cutoff f_C(r): 1 below R, half-cosine switch on [R, S), 0 from S on */
static double t_fc(const tersoff_t *P, double r)
{
    if (r < P->R) return 1.0;
    if (r >= P->S) return 0.0;
    return 0.5 + 0.5 * cos(ORACLE_PI * (r - P->R) / (P->S - P->R));
}
static double t_dfc(const tersoff_t *P, double r)
{
    if (r < P->R || r >= P->S) return 0.0;
    return -0.5 * ORACLE_PI / (P->S - P->R) * sin(ORACLE_PI * (r - P->R) / (P->S - P->R));
}
static double t_fR(const tersoff_t *P, double r) { return P->A * exp(-P->lam * r); }
static double t_dfR(const tersoff_t *P, double r) { return -P->lam * P->A * exp(-P->lam * r); }
static double t_fA(const tersoff_t *P, double r) { return P->B * exp(-P->mu * r); }
static double t_dfA(const tersoff_t *P, double r) { return -P->mu * P->B * exp(-P->mu * r); }

/* Eq. 5: g(theta) = 1 + c^2/d^2 - c^2 / (d^2 + (h - cos theta)^2) */
static double t_g(const tersoff_t *P, double cs)
{
    double c2 = P->c * P->c, d2 = P->d * P->d, hc = P->h - cs;
    return 1.0 + c2 / d2 - c2 / (d2 + hc * hc);
}
/* dg / d(cos theta) */
static double t_dg(const tersoff_t *P, double cs)
{
    double c2 = P->c * P->c, d2 = P->d * P->d, hc = P->h - cs;
    double den = d2 + hc * hc;
    return -2.0 * c2 * hc / (den * den);
}
/* Eq. 3: b = (1 + beta^n zeta^n)^(-1/(2n)); b = 1 at zeta = 0 */
static double t_b(const tersoff_t *P, double zeta)
{
    if (zeta <= 0.0) return 1.0;
    return pow(1.0 + pow(P->beta, P->n) * pow(zeta, P->n), -1.0 / (2.0 * P->n));
}
/* db/dzeta = -1/2 beta^n zeta^(n-1) (1 + beta^n zeta^n)^(-1/(2n) - 1); taken as 0 at
 * zeta = 0, where every dzeta/dr it multiplies vanishes (no k neighbours). */
static double t_db(const tersoff_t *P, double zeta)
{
    if (zeta <= 0.0) return 0.0;
    double bn = pow(P->beta, P->n);
    return -0.5 * bn * pow(zeta, P->n - 1.0) * pow(1.0 + bn * pow(zeta, P->n), -1.0 / (2.0 * P->n) - 1.0);
}

/* zeta_ij of Eq. 4 for the pair (i, j = NL[mj N + i]); rij is the bond vector */
static double t_zeta(const tersoff_t *P, int64_t N, const double *x, const double *y, const double *z,
                     const double *box, const int *pbc, const int *NN, const int *NL,
                     int64_t i, int mj, const double *rij)
{
    double r1 = vnorm(rij), zeta = 0.0;
    for (int mk = 0; mk < NN[i]; ++mk) {
        if (mk == mj) continue;
        int64_t k = NL[(int64_t)mk * N + i];
        double rik[3];
        bond(N, x, y, z, box, pbc, i, k, rik);
        double r2 = vnorm(rik);
        double cs = vdot(rij, rik) / (r1 * r2);           /* Eq. 6 */
        zeta += t_fc(P, r2) * t_g(P, cs);
    }
    return zeta;
}

/* Algorithm 1 (conventional method) with Eqs. 7-11.
 *   U    [N]  per-atom energy U_i = 1/2 sum_j U_ij          (Algorithm 1, energy line)
 *   F    [3N] forces                                         (Eqs. 7-11 scattered to i, j, k)
 *   Wlmp [9N] LAMMPS-style per-atom virial (Eq. 22), or NULL
 *   Wtot [9]  total virial sum over all interactions of sum_a r_a (x) F_a, or NULL
 * Reading of the two-body virial line: the printed line adds -1/2 r_ij (x) F^(ij)_i to
 * W_i only; the ordered-pair term's full virial is -r_ij (x) F^(ij)_i, and LAMMPS (whose
 * virial Eq. 22 describes) gives half of it to each of the two atoms.  Both halves are
 * assigned here, so that sum_i W_i equals the true virial.  The three-body part is
 * split in thirds over i, j, k exactly as printed.  Returns 0. */
int oracle_tersoff_conventional(int64_t N, const double *x, const double *y, const double *z,
                                const double *box, const int *pbc, const double *params,
                                const int *NN, const int *NL,
                                double *U, double *F, double *Wlmp, double *Wtot)
{
    tersoff_t P = tersoff_unpack(params);
    for (int64_t i = 0; i < N; ++i) {
        U[i] = 0.0;
        F[i] = F[N + i] = F[2 * N + i] = 0.0;
        if (Wlmp) for (int c = 0; c < 9; ++c) Wlmp[c * N + i] = 0.0;
    }
    if (Wtot) for (int c = 0; c < 9; ++c) Wtot[c] = 0.0;

    for (int64_t i = 0; i < N; ++i) {
        for (int mj = 0; mj < NN[i]; ++mj) {
            int64_t j = NL[(int64_t)mj * N + i];
            double rij[3];
            bond(N, x, y, z, box, pbc, i, j, rij);
            double r = vnorm(rij);
            if (r >= P.S) continue;                          /* f_C(r_ij) = 0 */
            double zeta = t_zeta(&P, N, x, y, z, box, pbc, NN, NL, i, mj, rij);
            double b = t_b(&P, zeta), db = t_db(&P, zeta);
            double fc = t_fc(&P, r), dfc = t_dfc(&P, r);
            double fR = t_fR(&P, r), dfR = t_dfR(&P, r);
            double fA = t_fA(&P, r), dfA = t_dfA(&P, r);
            U[i] += 0.5 * fc * (fR - b * fA);                /* Eq. 2, U_i += U_ij / 2 */

            /* Eq. 7: F^(ij)_i = -1/2 d(fC fR)/dr_i + 1/2 b d(fC fA)/dr_i, with
             * d phi(r_ij)/dr_i = -phi'(r) r_ij / r.  Eq. 8: F^(ij)_j = -F^(ij)_i. */
            double dR = dfc * fR + fc * dfR, dA = dfc * fA + fc * dfA;
            double Fi[3];
            for (int a = 0; a < 3; ++a) Fi[a] = (0.5 * dR - 0.5 * b * dA) * rij[a] / r;
            for (int a = 0; a < 3; ++a) { F[a * N + i] += Fi[a]; F[a * N + j] -= Fi[a]; }
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    double w = -rij[a] * Fi[c];              /* virial of this ordered pair */
                    if (Wlmp) { Wlmp[(3 * a + c) * N + i] += 0.5 * w; Wlmp[(3 * a + c) * N + j] += 0.5 * w; }
                    if (Wtot) Wtot[3 * a + c] += w;
                }

            /* Eqs. 9-11: three-body partial forces from b_ij's dependence on r_i, r_j, r_k */
            double pref = 0.5 * fc * fA * db;
            for (int mk = 0; mk < NN[i]; ++mk) {
                if (mk == mj) continue;
                int64_t k = NL[(int64_t)mk * N + i];
                double rik[3];
                bond(N, x, y, z, box, pbc, i, k, rik);
                double r2 = vnorm(rik);
                double cs = vdot(rij, rik) / (r * r2);
                double fck = t_fc(&P, r2), dfck = t_dfc(&P, r2);
                double gk = t_g(&P, cs), dgk = t_dg(&P, cs);
                double Fj[3], Fk[3], Fi3[3];
                for (int a = 0; a < 3; ++a) {
                    double dcos_drj = (rik[a] / r2 - cs * rij[a] / r) / r;   /* d cos / d r_j */
                    double dcos_drk = (rij[a] / r - cs * rik[a] / r2) / r2;  /* d cos / d r_k */
                    double dj = fck * dgk * dcos_drj;                        /* d(fC(r_ik) g)/d r_j */
                    double dk = dfck * gk * rik[a] / r2 + fck * dgk * dcos_drk; /* d(...)/d r_k */
                    Fj[a] = pref * dj;                                       /* Eq. 10 */
                    Fk[a] = pref * dk;                                       /* Eq. 11 */
                    Fi3[a] = -pref * (dj + dk);                              /* Eq. 9  */
                }
                for (int a = 0; a < 3; ++a) {
                    F[a * N + i] += Fi3[a]; F[a * N + j] += Fj[a]; F[a * N + k] += Fk[a];
                }
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) {
                        double w = rij[a] * Fj[c] + rik[a] * Fk[c];
                        if (Wlmp) {
                            Wlmp[(3 * a + c) * N + i] += w / 3.0;
                            Wlmp[(3 * a + c) * N + j] += w / 3.0;
                            Wlmp[(3 * a + c) * N + k] += w / 3.0;
                        }
                        if (Wtot) Wtot[3 * a + c] += w;
                    }
            }
        }
    }
    return 0;
}

/* Per-atom derivative route for Tersoff.  U_i = 1/2 sum_j f_C(r_ij)[f_R(r_ij) - b_ij f_A(r_ij)]
 * is a function of atom i's bond vectors {r_ij} only; this returns, for every list slot,
 *   D[m N + i] (3 components at D, D + cap N, D + 2 cap N) = dU_i / dr_ij,  j = NL[m N + i]
 * obtained by the chain rule through r_ij, b_ij and every b_ik (k != j), whose zeta_ik
 * contains the term f_C(r_ij) g(cos theta_ikj):
 *   dU_i/dr_ij = 1/2 [ (f_C f_R)' - b_ij (f_C f_A)' ] r_ij/r_ij
 *              - 1/2 f_C(r_ij) f_A(r_ij) b'_ij  dzeta_ij/dr_ij
 *              - 1/2 sum_{k != j} f_C(r_ik) f_A(r_ik) b'_ik dzeta_ik/dr_ij,
 *   dzeta_ij/dr_ij = sum_{k != j} f_C(r_ik) g'(cos) (r_ik/r_ik - cos r_ij/r_ij) / r_ij,
 *   dzeta_ik/dr_ij = f_C'(r_ij) g(cos) r_ij/r_ij + f_C(r_ij) g'(cos) (r_ik/r_ik - cos r_ij/r_ij)/r_ij.
 * Also returns U_i.  Slots with r_ij >= S get D = 0. */
int oracle_tersoff_dUdr(int64_t N, const double *x, const double *y, const double *z,
                        const double *box, const int *pbc, const double *params,
                        int cap, const int *NN, const int *NL, double *U, double *D)
{
    tersoff_t P = tersoff_unpack(params);
    int64_t CN = (int64_t)cap * N;
    double *zeta = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    if (!zeta) return -1;
    for (int64_t i = 0; i < N; ++i) {
        int nn = NN[i];
        /* bond order of each of i's bonds */
        for (int mj = 0; mj < nn; ++mj) {
            double rij[3];
            bond(N, x, y, z, box, pbc, i, NL[(int64_t)mj * N + i], rij);
            zeta[mj] = t_zeta(&P, N, x, y, z, box, pbc, NN, NL, i, mj, rij);
        }
        U[i] = 0.0;
        for (int mj = 0; mj < nn; ++mj) {
            double rij[3];
            bond(N, x, y, z, box, pbc, i, NL[(int64_t)mj * N + i], rij);
            double r = vnorm(rij);
            double fc = t_fc(&P, r), dfc = t_dfc(&P, r);
            double fR = t_fR(&P, r), dfR = t_dfR(&P, r);
            double fA = t_fA(&P, r), dfA = t_dfA(&P, r);
            double b = t_b(&P, zeta[mj]), db = t_db(&P, zeta[mj]);
            U[i] += 0.5 * fc * (fR - b * fA);
            double d[3];
            double radial = 0.5 * ((dfc * fR + fc * dfR) - b * (dfc * fA + fc * dfA));
            for (int a = 0; a < 3; ++a) d[a] = radial * rij[a] / r;
            for (int mk = 0; mk < nn; ++mk) {
                if (mk == mj) continue;
                double rik[3];
                bond(N, x, y, z, box, pbc, i, NL[(int64_t)mk * N + i], rik);
                double r2 = vnorm(rik);
                double cs = vdot(rij, rik) / (r * r2);
                double fck = t_fc(&P, r2), fAk = t_fA(&P, r2);
                double g = t_g(&P, cs), dg = t_dg(&P, cs);
                double bk = t_db(&P, zeta[mk]);
                for (int a = 0; a < 3; ++a) {
                    double dcos = (rik[a] / r2 - cs * rij[a] / r) / r;
                    d[a] += -0.5 * fc * fA * db * fck * dg * dcos;                    /* via zeta_ij */
                    d[a] += -0.5 * fck * fAk * bk * (dfc * g * rij[a] / r + fc * dg * dcos); /* via zeta_ik */
                }
            }
            for (int a = 0; a < 3; ++a) D[a * CN + (int64_t)mj * N + i] = (r < P.S) ? d[a] : 0.0;
        }
        for (int mj = nn; mj < cap; ++mj)
            for (int a = 0; a < 3; ++a) D[a * CN + (int64_t)mj * N + i] = 0.0;
    }
    free(zeta);
    return 0;
}

/* ------------------------------------------------ multi-element Tersoff */
/* Tersoff's multicomponent form (J. Tersoff, Phys. Rev. B 39, 5566 (1989)); the paper
 * presents the single-element form and notes that its method covers systems with several
 * kinds of atoms (end of Sec. 2.1).  For atoms i, j of elements a = t_i, b = t_j:
 *   U_ij   = f_C^{ab}(r_ij) [ f_R^{ab}(r_ij) - b_ij f_A^{ab}(r_ij) ],   U_i = 1/2 sum_j U_ij,
 *   f_R^{ab} = A_ab e^{-lambda_ab r},  f_A^{ab} = B_ab e^{-mu_ab r},  f_C^{ab}: R_ab, S_ab,
 *   A_ab = sqrt(A_a A_b), B_ab = sqrt(B_a B_b), R_ab = sqrt(R_a R_b), S_ab = sqrt(S_a S_b),
 *   lambda_ab = (lambda_a + lambda_b)/2, mu_ab = (mu_a + mu_b)/2,
 *   b_ij   = chi_ab (1 + beta_a^{n_a} zeta_ij^{n_a})^{-1/(2 n_a)},
 *   zeta_ij = sum_{k != j} f_C^{a t_k}(r_ik) g_a(theta_ijk)        (omega = 1),
 *   g_a(theta) = 1 + c_a^2/d_a^2 - c_a^2 / (d_a^2 + (h_a - cos theta)^2).
 * One element with chi = 1 gives Eqs. 2-6.  Arguments: types[N] element of each atom
 * (0 .. n_types-1, n_types <= 4); params[n_types x 11] per element in the packing of the
 * single-element routines; chi[n_types x n_types].
 * Implementation: a table of tersoff_t per ordered element pair (a, b), whose radial
 * fields (A, B, lambda, mu, R, S) are the mixed ones and whose angular and bond-order
 * fields (beta, n, c, d, h) are element a's, so the single-element helpers apply. */
#define ORACLE_MAXT 4
typedef struct {
    int nt;
    tersoff_t P[ORACLE_MAXT][ORACLE_MAXT];
    double chi[ORACLE_MAXT][ORACLE_MAXT];
} tersoff_multi_t;

static int tersoff_multi_unpack(int n_types, const double *params, const double *chi, tersoff_multi_t *T)
{
    if (n_types < 1 || n_types > ORACLE_MAXT) return -1;
    T->nt = n_types;
    for (int a = 0; a < n_types; ++a)
        for (int b = 0; b < n_types; ++b) {
            tersoff_t ea = tersoff_unpack(params + 11 * a), eb = tersoff_unpack(params + 11 * b);
            tersoff_t m = ea;
            m.A = sqrt(ea.A * eb.A);
            m.B = sqrt(ea.B * eb.B);
            m.lam = 0.5 * (ea.lam + eb.lam);
            m.mu = 0.5 * (ea.mu + eb.mu);
            m.R = sqrt(ea.R * eb.R);
            m.S = sqrt(ea.S * eb.S);
            T->P[a][b] = m;
            T->chi[a][b] = chi[a * n_types + b];
        }
    return 0;
}

/* zeta_ij for the pair (i, j = NL[mj N + i]) of atom i (element a) */
static double tm_zeta(const tersoff_multi_t *T, const int *types, int64_t N, const double *x, const double *y,
                      const double *z, const double *box, const int *pbc, const int *NN, const int *NL,
                      int64_t i, int mj, const double *rij)
{
    int a = types[i];
    double r1 = vnorm(rij), zeta = 0.0;
    for (int mk = 0; mk < NN[i]; ++mk) {
        if (mk == mj) continue;
        int64_t k = NL[(int64_t)mk * N + i];
        double rik[3];
        bond(N, x, y, z, box, pbc, i, k, rik);
        double r2 = vnorm(rik);
        double cs = vdot(rij, rik) / (r1 * r2);
        zeta += t_fc(&T->P[a][types[k]], r2) * t_g(&T->P[a][a], cs);
    }
    return zeta;
}

/* Algorithm 1 (Eqs. 7-11) for the multicomponent form: U_i, F_i and the total virial
 * (Wtot may be NULL).  Same loop structure as oracle_tersoff_conventional, each radial
 * function taken with the pair's mixed parameters, g and the bond order with atom i's
 * element, b_ij and its derivative scaled by chi_ij.  Returns 0, -1 on bad n_types. */
int oracle_tersoff_multi_conventional(int64_t N, const double *x, const double *y, const double *z,
                                      const double *box, const int *pbc, const int *types, int n_types,
                                      const double *params, const double *chi, const int *NN, const int *NL,
                                      double *U, double *F, double *Wtot)
{
    tersoff_multi_t T;
    if (tersoff_multi_unpack(n_types, params, chi, &T) != 0) return -1;
    for (int64_t i = 0; i < N; ++i) {
        U[i] = 0.0;
        F[i] = F[N + i] = F[2 * N + i] = 0.0;
    }
    if (Wtot) for (int c = 0; c < 9; ++c) Wtot[c] = 0.0;

    for (int64_t i = 0; i < N; ++i) {
        int a = types[i];
        const tersoff_t *Pa = &T.P[a][a];
        for (int mj = 0; mj < NN[i]; ++mj) {
            int64_t j = NL[(int64_t)mj * N + i];
            const tersoff_t *Pij = &T.P[a][types[j]];
            double chi_ij = T.chi[a][types[j]];
            double rij[3];
            bond(N, x, y, z, box, pbc, i, j, rij);
            double r = vnorm(rij);
            if (r >= Pij->S) continue;
            double zeta = tm_zeta(&T, types, N, x, y, z, box, pbc, NN, NL, i, mj, rij);
            double b = chi_ij * t_b(Pa, zeta), db = chi_ij * t_db(Pa, zeta);
            double fc = t_fc(Pij, r), dfc = t_dfc(Pij, r);
            double fR = t_fR(Pij, r), dfR = t_dfR(Pij, r);
            double fA = t_fA(Pij, r), dfA = t_dfA(Pij, r);
            U[i] += 0.5 * fc * (fR - b * fA);

            double dR = dfc * fR + fc * dfR, dA = dfc * fA + fc * dfA;
            double Fi[3];
            for (int q = 0; q < 3; ++q) Fi[q] = (0.5 * dR - 0.5 * b * dA) * rij[q] / r;     /* Eq. 7 */
            for (int q = 0; q < 3; ++q) { F[q * N + i] += Fi[q]; F[q * N + j] -= Fi[q]; } /* Eq. 8 */
            if (Wtot)
                for (int q = 0; q < 3; ++q)
                    for (int c = 0; c < 3; ++c) Wtot[3 * q + c] += -rij[q] * Fi[c];

            double pref = 0.5 * fc * fA * db;
            for (int mk = 0; mk < NN[i]; ++mk) {
                if (mk == mj) continue;
                int64_t k = NL[(int64_t)mk * N + i];
                const tersoff_t *Pik = &T.P[a][types[k]];
                double rik[3];
                bond(N, x, y, z, box, pbc, i, k, rik);
                double r2 = vnorm(rik);
                double cs = vdot(rij, rik) / (r * r2);
                double fck = t_fc(Pik, r2), dfck = t_dfc(Pik, r2);
                double gk = t_g(Pa, cs), dgk = t_dg(Pa, cs);
                double Fj[3], Fk[3];
                for (int q = 0; q < 3; ++q) {
                    double dcos_drj = (rik[q] / r2 - cs * rij[q] / r) / r;
                    double dcos_drk = (rij[q] / r - cs * rik[q] / r2) / r2;
                    double dj = fck * dgk * dcos_drj;
                    double dk = dfck * gk * rik[q] / r2 + fck * dgk * dcos_drk;
                    Fj[q] = pref * dj;                                          /* Eq. 10 */
                    Fk[q] = pref * dk;                                          /* Eq. 11 */
                    F[q * N + i] += -pref * (dj + dk);                          /* Eq. 9  */
                }
                for (int q = 0; q < 3; ++q) { F[q * N + j] += Fj[q]; F[q * N + k] += Fk[q]; }
                if (Wtot)
                    for (int q = 0; q < 3; ++q)
                        for (int c = 0; c < 3; ++c) Wtot[3 * q + c] += rij[q] * Fj[c] + rik[q] * Fk[c];
            }
        }
    }
    return 0;
}

/* dU_i/dr_ij for the multicomponent form, per list slot (layout of oracle_tersoff_dUdr):
 *   dU_i/dr_ij = 1/2 [ (f_C f_R)'_ij - b_ij (f_C f_A)'_ij ] r_ij/r_ij
 *              - 1/2 f_C^{ij} f_A^{ij} b'_ij dzeta_ij/dr_ij
 *              - 1/2 sum_{k != j} f_C^{ik} f_A^{ik} b'_ik dzeta_ik/dr_ij,
 *   dzeta_ik/dr_ij = f_C^{ij}'(r_ij) g_a(cos) r_ij/r_ij + f_C^{ij}(r_ij) g_a'(cos) dcos/dr_ij,
 * b' = chi db/dzeta.  Also U_i.  Slots with r_ij >= S_ij get D = 0.  Returns 0, -1 on
 * allocation failure or bad n_types. */
int oracle_tersoff_multi_dUdr(int64_t N, const double *x, const double *y, const double *z,
                              const double *box, const int *pbc, const int *types, int n_types,
                              const double *params, const double *chi, int cap, const int *NN, const int *NL,
                              double *U, double *D)
{
    tersoff_multi_t T;
    if (tersoff_multi_unpack(n_types, params, chi, &T) != 0) return -1;
    int64_t CN = (int64_t)cap * N;
    double *zeta = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    if (!zeta) return -1;
    for (int64_t i = 0; i < N; ++i) {
        int a = types[i], nn = NN[i];
        const tersoff_t *Pa = &T.P[a][a];
        for (int mj = 0; mj < nn; ++mj) {
            double rij[3];
            bond(N, x, y, z, box, pbc, i, NL[(int64_t)mj * N + i], rij);
            zeta[mj] = tm_zeta(&T, types, N, x, y, z, box, pbc, NN, NL, i, mj, rij);
        }
        U[i] = 0.0;
        for (int mj = 0; mj < nn; ++mj) {
            int64_t j = NL[(int64_t)mj * N + i];
            const tersoff_t *Pij = &T.P[a][types[j]];
            double chi_ij = T.chi[a][types[j]];
            double rij[3];
            bond(N, x, y, z, box, pbc, i, j, rij);
            double r = vnorm(rij);
            double fc = t_fc(Pij, r), dfc = t_dfc(Pij, r);
            double fR = t_fR(Pij, r), dfR = t_dfR(Pij, r);
            double fA = t_fA(Pij, r), dfA = t_dfA(Pij, r);
            double b = chi_ij * t_b(Pa, zeta[mj]), db = chi_ij * t_db(Pa, zeta[mj]);
            U[i] += 0.5 * fc * (fR - b * fA);
            double d[3];
            double radial = 0.5 * ((dfc * fR + fc * dfR) - b * (dfc * fA + fc * dfA));
            for (int q = 0; q < 3; ++q) d[q] = radial * rij[q] / r;
            for (int mk = 0; mk < nn; ++mk) {
                if (mk == mj) continue;
                int64_t k = NL[(int64_t)mk * N + i];
                const tersoff_t *Pik = &T.P[a][types[k]];
                double chi_ik = T.chi[a][types[k]];
                double rik[3];
                bond(N, x, y, z, box, pbc, i, k, rik);
                double r2 = vnorm(rik);
                double cs = vdot(rij, rik) / (r * r2);
                double fck = t_fc(Pik, r2), fAk = t_fA(Pik, r2);
                double g = t_g(Pa, cs), dg = t_dg(Pa, cs);
                double bk = chi_ik * t_db(Pa, zeta[mk]);
                for (int q = 0; q < 3; ++q) {
                    double dcos = (rik[q] / r2 - cs * rij[q] / r) / r;
                    d[q] += -0.5 * fc * fA * db * fck * dg * dcos;
                    d[q] += -0.5 * fck * fAk * bk * (dfc * g * rij[q] / r + fc * dg * dcos);
                }
            }
            for (int q = 0; q < 3; ++q) D[q * CN + (int64_t)mj * N + i] = (r < Pij->S) ? d[q] : 0.0;
        }
        for (int mj = nn; mj < cap; ++mj)
            for (int q = 0; q < 3; ++q) D[q * CN + (int64_t)mj * N + i] = 0.0;
    }
    free(zeta);
    return 0;
}

/* ------------------------------------------------------- Stillinger-Weber */
/* Packed parameters: epsilon, sigma, a, lambda, gamma, A, B, p, q (SW 1985). */
typedef struct { double eps, sig, a, lam, gam, A, B, p, q; } sw_t;

static sw_t sw_unpack(const double *p)
{
    sw_t s = {p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8]};
    return s;
}

/* two-body phi2(r) = A eps [B (sigma/r)^p - (sigma/r)^q] exp(sigma / (r - a sigma)), r < a sigma */
static double sw_phi2(const sw_t *S, double r)
{
    double rc = S->a * S->sig;
    if (r >= rc) return 0.0;
    return S->A * S->eps * (S->B * pow(S->sig / r, S->p) - pow(S->sig / r, S->q)) * exp(S->sig / (r - rc));
}
static double sw_dphi2(const sw_t *S, double r)
{
    double rc = S->a * S->sig;
    if (r >= rc) return 0.0;
    double e = exp(S->sig / (r - rc));
    double poly = S->B * pow(S->sig / r, S->p) - pow(S->sig / r, S->q);
    double dpoly = (-S->p * S->B * pow(S->sig / r, S->p) + S->q * pow(S->sig / r, S->q)) / r;
    double de = -S->sig / ((r - rc) * (r - rc)) * e;
    return S->A * S->eps * (dpoly * e + poly * de);
}
/* radial factor of the three-body term, exp(gamma sigma / (r - a sigma)), r < a sigma */
static double sw_E(const sw_t *S, double r)
{
    double rc = S->a * S->sig;
    if (r >= rc) return 0.0;
    return exp(S->gam * S->sig / (r - rc));
}
static double sw_dE(const sw_t *S, double r)
{
    double rc = S->a * S->sig;
    if (r >= rc) return 0.0;
    return -S->gam * S->sig / ((r - rc) * (r - rc)) * exp(S->gam * S->sig / (r - rc));
}

/* Conventional (scatter) SW evaluation in the style of Algorithm 1.  Per-atom energy
 * U_i = 1/2 sum_j phi2(r_ij) + sum_{j<k} phi3(r_ij, r_ik, theta_jik): the three-body term
 * belongs to its vertex atom i.  F from -dU/dr of every term, scattered to its atoms;
 * Wtot as in the Tersoff routine.  (The LAMMPS-style per-atom virial is a Tersoff-only
 * contrast quantity here.) */
int oracle_sw_conventional(int64_t N, const double *x, const double *y, const double *z,
                           const double *box, const int *pbc, const double *params,
                           const int *NN, const int *NL, double *U, double *F, double *Wtot)
{
    sw_t S = sw_unpack(params);
    double rc = S.a * S.sig;
    for (int64_t i = 0; i < N; ++i) { U[i] = 0.0; F[i] = F[N + i] = F[2 * N + i] = 0.0; }
    if (Wtot) for (int c = 0; c < 9; ++c) Wtot[c] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        for (int mj = 0; mj < NN[i]; ++mj) {
            int64_t j = NL[(int64_t)mj * N + i];
            double rij[3];
            bond(N, x, y, z, box, pbc, i, j, rij);
            double r1 = vnorm(rij);
            if (r1 >= rc) continue;
            U[i] += 0.5 * sw_phi2(&S, r1);
            double Fi[3];
            for (int a = 0; a < 3; ++a) Fi[a] = 0.5 * sw_dphi2(&S, r1) * rij[a] / r1;
            for (int a = 0; a < 3; ++a) { F[a * N + i] += Fi[a]; F[a * N + j] -= Fi[a]; }
            if (Wtot) for (int a = 0; a < 3; ++a) for (int c = 0; c < 3; ++c) Wtot[3 * a + c] += -rij[a] * Fi[c];
            for (int mk = mj + 1; mk < NN[i]; ++mk) {
                int64_t k = NL[(int64_t)mk * N + i];
                double rik[3];
                bond(N, x, y, z, box, pbc, i, k, rik);
                double r2 = vnorm(rik);
                if (r2 >= rc) continue;
                double cs = vdot(rij, rik) / (r1 * r2);
                double E1 = sw_E(&S, r1), E2 = sw_E(&S, r2), dE1 = sw_dE(&S, r1), dE2 = sw_dE(&S, r2);
                double t = cs + 1.0 / 3.0;
                U[i] += S.lam * S.eps * t * t * E1 * E2;
                double Fj[3], Fk[3];
                for (int a = 0; a < 3; ++a) {
                    double dcos_drj = (rik[a] / r2 - cs * rij[a] / r1) / r1;
                    double dcos_drk = (rij[a] / r1 - cs * rik[a] / r2) / r2;
                    double dphi_drj = S.lam * S.eps * (2.0 * t * dcos_drj * E1 * E2 + t * t * dE1 * rij[a] / r1 * E2);
                    double dphi_drk = S.lam * S.eps * (2.0 * t * dcos_drk * E1 * E2 + t * t * E1 * dE2 * rik[a] / r2);
                    Fj[a] = -dphi_drj;
                    Fk[a] = -dphi_drk;
                }
                for (int a = 0; a < 3; ++a) {
                    F[a * N + j] += Fj[a]; F[a * N + k] += Fk[a]; F[a * N + i] -= Fj[a] + Fk[a];
                }
                if (Wtot) for (int a = 0; a < 3; ++a) for (int c = 0; c < 3; ++c)
                    Wtot[3 * a + c] += rij[a] * Fj[c] + rik[a] * Fk[c];
            }
        }
    }
    return 0;
}

/* Per-atom derivative route for SW: D = dU_i/dr_ij for every slot, U_i as above.
 *   dU_i/dr_ij = 1/2 phi2'(r_ij) r_ij/r_ij + sum_{k != j} d phi3(r_ij, r_ik, theta_jik)/d r_ij,
 *   d phi3/d r_ij = lambda eps [ 2 (cos + 1/3) (r_ik/r_ik - cos r_ij/r_ij)/r_ij E(r_ij) E(r_ik)
 *                               + (cos + 1/3)^2 E'(r_ij) E(r_ik) r_ij/r_ij ]. */
int oracle_sw_dUdr(int64_t N, const double *x, const double *y, const double *z,
                   const double *box, const int *pbc, const double *params,
                   int cap, const int *NN, const int *NL, double *U, double *D)
{
    sw_t S = sw_unpack(params);
    double rc = S.a * S.sig;
    int64_t CN = (int64_t)cap * N;
    for (int64_t i = 0; i < N; ++i) {
        U[i] = 0.0;
        for (int mj = 0; mj < cap; ++mj)
            for (int a = 0; a < 3; ++a) D[a * CN + (int64_t)mj * N + i] = 0.0;
        for (int mj = 0; mj < NN[i]; ++mj) {
            double rij[3];
            bond(N, x, y, z, box, pbc, i, NL[(int64_t)mj * N + i], rij);
            double r1 = vnorm(rij);
            if (r1 >= rc) continue;
            U[i] += 0.5 * sw_phi2(&S, r1);
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = 0.5 * sw_dphi2(&S, r1) * rij[a] / r1;
            for (int mk = 0; mk < NN[i]; ++mk) {
                if (mk == mj) continue;
                double rik[3];
                bond(N, x, y, z, box, pbc, i, NL[(int64_t)mk * N + i], rik);
                double r2 = vnorm(rik);
                if (r2 >= rc) continue;
                double cs = vdot(rij, rik) / (r1 * r2);
                double t = cs + 1.0 / 3.0;
                double E1 = sw_E(&S, r1), E2 = sw_E(&S, r2), dE1 = sw_dE(&S, r1);
                if (mk > mj) U[i] += S.lam * S.eps * t * t * E1 * E2;  /* each unordered pair once */
                for (int a = 0; a < 3; ++a) {
                    double dcos = (rik[a] / r2 - cs * rij[a] / r1) / r1;
                    d[a] += S.lam * S.eps * (2.0 * t * dcos * E1 * E2 + t * t * dE1 * rij[a] / r1 * E2);
                }
            }
            for (int a = 0; a < 3; ++a) D[a * CN + (int64_t)mj * N + i] = d[a];
        }
    }
    return 0;
}

/* --------------------------------------------- many-body F, W, J (Eqs. 28-30) */
/* From per-slot D = dU_i/dr_ij (any many-body potential):
 *   F_i = sum_j (dU_i/dr_ij - dU_j/dr_ji)                         Eq. 28
 *   W_i = -1/2 sum_j r_ij (x) (dU_i/dr_ij - dU_j/dr_ji)             Eq. 29
 *   J_i = sum_j r_ij (dU_j/dr_ji . v_i)                            Eq. 30
 * dU_j/dr_ji is looked up in j's own list.  Any output may be NULL.  v may be NULL
 * (then J is not computed).  Returns 0, or -2 if a pair is missing from j's list. */
int oracle_manybody_fwj(int64_t N, const double *x, const double *y, const double *z,
                        const double *box, const int *pbc, int cap, const int *NN, const int *NL,
                        const double *D, const double *vx, const double *vy, const double *vz,
                        double *F, double *W, double *J)
{
    int64_t CN = (int64_t)cap * N;
    for (int64_t i = 0; i < N; ++i) {
        double f[3] = {0, 0, 0}, w[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, jj[3] = {0, 0, 0};
        double vi[3] = {0, 0, 0};
        if (vx) { vi[0] = vx[i]; vi[1] = vy[i]; vi[2] = vz[i]; }
        for (int m = 0; m < NN[i]; ++m) {
            int64_t j = NL[(int64_t)m * N + i];
            int mr = find_slot(N, NN, NL, j, i);
            if (mr < 0) return -2;
            double rij[3], dij[3], dji[3];
            bond(N, x, y, z, box, pbc, i, j, rij);
            for (int a = 0; a < 3; ++a) {
                dij[a] = D[a * CN + (int64_t)m * N + i];
                dji[a] = D[a * CN + (int64_t)mr * N + j];
            }
            double dv = vdot(dji, vi);
            for (int a = 0; a < 3; ++a) {
                f[a] += dij[a] - dji[a];
                jj[a] += rij[a] * dv;
                for (int c = 0; c < 3; ++c) w[3 * a + c] += -0.5 * rij[a] * (dij[c] - dji[c]);
            }
        }
        if (F) for (int a = 0; a < 3; ++a) F[a * N + i] = f[a];
        if (W) for (int c = 0; c < 9; ++c) W[c * N + i] = w[c];
        if (J && vx) for (int a = 0; a < 3; ++a) J[a * N + i] = jj[a];
    }
    return 0;
}

/* ------------------------------------------------------------ time stepping */
enum { ORACLE_TERSOFF = 1, ORACLE_SW = 2, ORACLE_TERSOFF_MULTI = 3 };

/* the potential of a run: one element (Tersoff or SW), or multi-element Tersoff */
typedef struct {
    int kind;
    const double *params;
    const int *types;     /* multi-element only */
    int n_types;
    const double *chi;
} pot_t;

static double pot_cutoff(const pot_t *pot)
{
    if (pot->kind == ORACLE_TERSOFF) return pot->params[10];
    if (pot->kind == ORACLE_SW) return pot->params[1] * pot->params[2];
    double rc = 0.0;   /* largest mixed S_ab */
    for (int a = 0; a < pot->n_types; ++a)
        for (int b = 0; b < pot->n_types; ++b) {
            double s = sqrt(pot->params[11 * a + 10] * pot->params[11 * b + 10]);
            if (s > rc) rc = s;
        }
    return rc;
}

static int build_list(int64_t N, const double *x, const double *y, const double *z,
                      const double *box, const int *pbc, double rc, int cap, int *NN, int *NL)
{
    if (N <= 4096) return oracle_neighbors_brute(N, x, y, z, box, pbc, rc, cap, NN, NL);
    return oracle_neighbors_cells(N, x, y, z, box, pbc, rc, cap, NN, NL);
}

static void conventional_forces(const pot_t *pot, int64_t N, const double *x, const double *y, const double *z,
                                const double *box, const int *pbc, const int *NN, const int *NL, double *U,
                                double *F)
{
    if (pot->kind == ORACLE_TERSOFF)
        oracle_tersoff_conventional(N, x, y, z, box, pbc, pot->params, NN, NL, U, F, NULL, NULL);
    else if (pot->kind == ORACLE_SW)
        oracle_sw_conventional(N, x, y, z, box, pbc, pot->params, NN, NL, U, F, NULL);
    else
        oracle_tersoff_multi_conventional(N, x, y, z, box, pbc, pot->types, pot->n_types, pot->params, pot->chi,
                                          NN, NL, U, F, NULL);
}

static void pair_derivatives(const pot_t *pot, int64_t N, const double *x, const double *y, const double *z,
                             const double *box, const int *pbc, int cap, const int *NN, const int *NL, double *U,
                             double *D)
{
    if (pot->kind == ORACLE_TERSOFF) oracle_tersoff_dUdr(N, x, y, z, box, pbc, pot->params, cap, NN, NL, U, D);
    else if (pot->kind == ORACLE_SW) oracle_sw_dUdr(N, x, y, z, box, pbc, pot->params, cap, NN, NL, U, D);
    else
        oracle_tersoff_multi_dUdr(N, x, y, z, box, pbc, pot->types, pot->n_types, pot->params, pot->chi, cap, NN,
                                  NL, U, D);
}

/* Velocity Verlet (Sec. 3): per step
 *   v += F/m dt/2;  x += v dt (wrapped into [0, L) on periodic axes);
 *   neighbour list rebuilt from scratch at the potential cutoff; F(x) by Algorithm 1;
 *   v += F/m dt/2;  [damped relaxation: v *= (1 - damp dt)];
 *   heat current J = sum_i J_i (Eq. 30) from x(t+dt), v(t+dt).
 * series (n_steps x 5, or NULL) receives U, K, Jx, Jy, Jz after every step.
 * masses: per-atom masses (amu).  x, y, z, vx, vy, vz are updated in place.
 * Returns 0, -1 on allocation failure, -3 on neighbour overflow. */
/* Berendsen weak coupling (Berendsen et al., J. Chem. Phys. 81, 3684 (1984)), the NPT
 * ensemble the paper's benchmarks run in (Sec. 3: 300 K, 0 Pa).  At the end of step s,
 * with K = sum_i m_i v_i^2 / 2, K_aa = sum_i m_i v_ia^2 / 2, the total virial W (the sum of
 * the Eq. 29 per-atom virials) and V = Lx Ly Lz:
 *     T      = 2 K / (k_B (3N - 3)),
 *     lambda = sqrt(1 + (dt / tau_T) (T0 / T - 1)),
 *     P_aa   = (2 K_aa + W_aa) / V                      (converted to GPa),
 *     mu_a   = cbrt(1 - (beta dt / tau_P) (P0 - P_aa))  on each coupled periodic axis, else 1.
 * The velocities are multiplied by lambda and every coordinate and box edge along a by
 * mu_a at the start of step s + 1, before its half-kick; the scaling computed at the last
 * step of a run is not applied (it stays pending).  tau_T <= 0 or tau_P <= 0 switches that
 * half off.  npt = {T0 (K), P0 (GPa), tau_T (fs), tau_P (fs), beta (1/GPa), couple_x,
 * couple_y, couple_z}. */
static const double K_BOLTZMANN = 8.617333262e-5;            /* eV / K */
static const double EV_PER_A3_IN_GPA = 160.21766340;          /* 1.602176634e-19 J / 1e-30 m^3 */

static int run_core(int64_t N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                    const double *masses, double *box, const int *pbc, const pot_t *pot, int cap,
                    int64_t n_steps, double dt, double damp, const double *npt, double *series)
{
    double rc = pot_cutoff(pot);
    size_t n1 = (size_t)(N > 0 ? N : 1);
    int *NN = (int *)malloc(sizeof(int) * n1);
    int *NL = (int *)malloc(sizeof(int) * (size_t)cap * n1);
    double *U = (double *)malloc(sizeof(double) * n1);
    double *F = (double *)malloc(sizeof(double) * 3 * n1);
    double *D = (double *)malloc(sizeof(double) * 3 * (size_t)cap * n1);
    double *Jv = (double *)malloc(sizeof(double) * 3 * n1);
    double *Wv = (double *)malloc(sizeof(double) * 9 * n1);
    double *Ud = (double *)malloc(sizeof(double) * n1);
    double lam = 1.0, mu[3] = {1.0, 1.0, 1.0};
    int pending = 0;
    int rc_status = 0;
    if (!NN || !NL || !U || !F || !D || !Jv || !Wv || !Ud) { rc_status = -1; goto done; }
    if (build_list(N, x, y, z, box, pbc, rc, cap, NN, NL) > cap) { rc_status = -3; goto done; }
    conventional_forces(pot, N, x, y, z, box, pbc, NN, NL, U, F);
    for (int64_t s = 0; s < n_steps; ++s) {
        if (pending) {   /* Berendsen scaling computed at the end of the previous step */
            double *c[3] = {x, y, z};
            for (int64_t i = 0; i < N; ++i) {
                vx[i] *= lam; vy[i] *= lam; vz[i] *= lam;
                for (int a = 0; a < 3; ++a) c[a][i] *= mu[a];
            }
            for (int a = 0; a < 3; ++a) box[a] *= mu[a];
            pending = 0;
        }
        for (int64_t i = 0; i < N; ++i) {
            double h = 0.5 * dt * ACC_UNIT / masses[i];
            vx[i] += h * F[i]; vy[i] += h * F[N + i]; vz[i] += h * F[2 * N + i];
            x[i] += dt * vx[i]; y[i] += dt * vy[i]; z[i] += dt * vz[i];
            double *c[3] = {x, y, z};
            for (int a = 0; a < 3; ++a) {
                if (!pbc[a]) continue;
                if (c[a][i] >= box[a]) c[a][i] -= box[a];
                else if (c[a][i] < 0.0) c[a][i] += box[a];
            }
        }
        if (build_list(N, x, y, z, box, pbc, rc, cap, NN, NL) > cap) { rc_status = -3; goto done; }
        conventional_forces(pot, N, x, y, z, box, pbc, NN, NL, U, F);
        double Ut = 0.0, K = 0.0, Kaa[3] = {0, 0, 0}, Jt[3] = {0, 0, 0}, Waa[3] = {0, 0, 0};
        for (int64_t i = 0; i < N; ++i) {
            double h = 0.5 * dt * ACC_UNIT / masses[i];
            vx[i] += h * F[i]; vy[i] += h * F[N + i]; vz[i] += h * F[2 * N + i];
            if (damp > 0.0) {
                double f = 1.0 - damp * dt;
                vx[i] *= f; vy[i] *= f; vz[i] *= f;
            }
            Ut += U[i];
            K += 0.5 * masses[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]) / ACC_UNIT;
            Kaa[0] += 0.5 * masses[i] * vx[i] * vx[i] / ACC_UNIT;
            Kaa[1] += 0.5 * masses[i] * vy[i] * vy[i] / ACC_UNIT;
            Kaa[2] += 0.5 * masses[i] * vz[i] * vz[i] / ACC_UNIT;
        }
        pair_derivatives(pot, N, x, y, z, box, pbc, cap, NN, NL, Ud, D);
        oracle_manybody_fwj(N, x, y, z, box, pbc, cap, NN, NL, D, vx, vy, vz, NULL, npt ? Wv : NULL, Jv);
        for (int64_t i = 0; i < N; ++i) for (int a = 0; a < 3; ++a) Jt[a] += Jv[a * N + i];
        if (series) {
            series[5 * s + 0] = Ut; series[5 * s + 1] = K;
            series[5 * s + 2] = Jt[0]; series[5 * s + 3] = Jt[1]; series[5 * s + 4] = Jt[2];
        }
        if (npt) {
            for (int64_t i = 0; i < N; ++i) for (int a = 0; a < 3; ++a) Waa[a] += Wv[(4 * a) * N + i];
            double T0 = npt[0], P0 = npt[1], tauT = npt[2], tauP = npt[3], beta = npt[4];
            double ndof = 3.0 * (double)N - 3.0;
            double T = ndof > 0 ? 2.0 * K / (K_BOLTZMANN * ndof) : 0.0;
            lam = 1.0;
            if (tauT > 0.0 && T > 0.0) {
                double l2 = 1.0 + dt / tauT * (T0 / T - 1.0);
                lam = l2 > 0.0 ? sqrt(l2) : 0.0;
            }
            double V = box[0] * box[1] * box[2];
            for (int a = 0; a < 3; ++a) {
                mu[a] = 1.0;
                if (tauP > 0.0 && pbc[a] && npt[5 + a] != 0.0) {
                    double P = (2.0 * Kaa[a] + Waa[a]) / V * EV_PER_A3_IN_GPA;
                    mu[a] = cbrt(1.0 - beta * dt / tauP * (P0 - P));
                }
            }
            pending = 1;
        }
    }
done:
    free(NN); free(NL); free(U); free(F); free(D); free(Jv); free(Wv); free(Ud);
    return rc_status;
}

int oracle_run_ex(int64_t N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                  const double *masses, double *box, const int *pbc, int kind, const double *params, int cap,
                  int64_t n_steps, double dt, double damp, const double *npt, double *series)
{
    pot_t pot = {kind, params, NULL, 1, NULL};
    return run_core(N, x, y, z, vx, vy, vz, masses, box, pbc, &pot, cap, n_steps, dt, damp, npt, series);
}

/* The same integrator for multi-element Tersoff (types, n_types, params, chi as in
 * oracle_tersoff_multi_conventional). */
int oracle_run_multi(int64_t N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                     const double *masses, double *box, const int *pbc, const int *types, int n_types,
                     const double *params, const double *chi, int cap, int64_t n_steps, double dt, double damp,
                     const double *npt, double *series)
{
    if (n_types < 1 || n_types > ORACLE_MAXT) return -1;
    pot_t pot = {ORACLE_TERSOFF_MULTI, params, types, n_types, chi};
    return run_core(N, x, y, z, vx, vy, vz, masses, box, pbc, &pot, cap, n_steps, dt, damp, npt, series);
}

int oracle_run(int64_t N, double *x, double *y, double *z, double *vx, double *vy, double *vz,
               const double *masses, const double *box, const int *pbc, int kind,
               const double *params, int cap, int64_t n_steps, double dt, double damp, double *series)
{
    double b[3] = {box[0], box[1], box[2]};
    return oracle_run_ex(N, x, y, z, vx, vy, vz, masses, b, pbc, kind, params, cap, n_steps, dt, damp, NULL,
                         series);
}
