/*
 * nb_oracle.c -- the oracle for the short-range non-bonded forces.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load or call this file.  It shares no
 * code, header, table or constant with the CUDA library, and the library
 * never calls it.
 *
 * What it computes is the plain definition of the quantity that the paper's
 * cluster-pair method evaluates (Introduction: each particle's electrostatic
 * and van der Waals forces from all other particles inside a spherical
 * cut-off; Section 3.2: the cluster-pair list only adds interactions that are
 * known to be zero, so the method reaches the same sum):
 *
 *   for every unordered atom pair (i, j), i < j, that is not excluded:
 *     d   = x_i - x_j, reduced to the minimum image of the periodic box
 *           (rectangular, or triclinic with rows a, b, c; see pair_image)
 *     r^2 = |d|^2;  the pair contributes only if r^2 < rc^2 (strict)
 *     Lennard-Jones  V = c12 / r^12 - c6 / r^6
 *                    F/r = (12 c12 / r^12 - 6 c6 / r^6) / r^2
 *     reaction field V = f qi qj / eps_r (1/r + k_rf r^2 - c_rf)
 *                    F/r = f qi qj / eps_r (1/r^3 - 2 k_rf)
 *                    k_rf = (eps_rf - eps_r) / ((2 eps_rf + eps_r) rc^3),
 *                    c_rf = 1/rc + k_rf rc^2  (eps_rf = 0 means infinity:
 *                    k_rf = 1 / (2 rc^3))
 *     Ewald real     V = f qi qj / eps_r erfc(beta r) / r
 *                    F/r = f qi qj / eps_r (erfc(beta r)/r
 *                          + 2 beta/sqrt(pi) exp(-beta^2 r^2)) / r^2
 *     force on i = (F/r) d, force on j = -(F/r) d
 *     virial Xi -= 1/2 (F/r) d (x) d
 *
 * Optional potential modifiers (bits of `mods`; all off by default):
 *   OR_MOD_LJ_SHIFT     every interacting pair's Lennard-Jones energy is taken
 *                       relative to its value at the cut-off:
 *                       V = c12 (1/r^12 - 1/rc^12) - c6 (1/r^6 - 1/rc^6);
 *                       forces unchanged
 *   OR_MOD_EWALD_SHIFT  likewise for the Ewald real-space term:
 *                       V = f qi qj / eps_r (erfc(beta r)/r - erfc(beta rc)/rc)
 *   OR_MOD_RF_EXCL      reaction-field correction of excluded pairs: every
 *                       excluded pair (i, j) with r^2 < rc^2 contributes
 *                       V = f qi qj / eps_r (k_rf r^2 - c_rf) and the force
 *                       of that potential, F/r = -2 f qi qj / eps_r k_rf
 *                       (no self term)
 *
 * Everything is double precision.  Inputs are the same float32 values the
 * CUDA path receives, promoted exactly by the caller.  Exclusions are a CSR
 * list over atoms; a pair is excluded if either atom lists the other.
 *
 * The interaction forms, the strict cut-off test, the virial convention and
 * the treatment of excluded pairs (they contribute nothing) are readings of
 * a paper that states none of them; each one is pinned by the oracle tests.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_RF 0
#define OR_EWALD 1
#define OR_MOD_LJ_SHIFT 1
#define OR_MOD_EWALD_SHIFT 2
#define OR_MOD_RF_EXCL 4

static double min_image(double d, double L) { return d - L * round(d / L); }

/*
 * Minimum image of d = x_i - x_j.  box = (ax, by, cz, bx, cx, cy): the rows
 * a = (ax, 0, 0), b = (bx, by, 0), c = (cx, cy, cz) of the periodic lattice.
 * A rectangular box (bx = cx = cy = 0) reduces each component; a triclinic
 * one is reduced by c, b, a in turn and then the shortest of the 27
 * neighbouring images is taken (brute force).
 */
static void pair_image(const double *box, double dx, double dy, double dz, double *ox, double *oy,
                       double *oz) {
    const double ax = box[0], by = box[1], cz = box[2], bx = box[3], cx = box[4], cy = box[5];
    if (bx == 0.0 && cx == 0.0 && cy == 0.0) {
        *ox = min_image(dx, ax);
        *oy = min_image(dy, by);
        *oz = min_image(dz, cz);
        return;
    }
    double k = round(dz / cz);
    dx -= k * cx;
    dy -= k * cy;
    dz -= k * cz;
    k = round(dy / by);
    dx -= k * bx;
    dy -= k * by;
    dx -= round(dx / ax) * ax;
    double best = dx * dx + dy * dy + dz * dz, bxo = dx, byo = dy, bzo = dz;
    for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j)
            for (int l = -1; l <= 1; ++l) {
                double ex = dx + i * ax + j * bx + l * cx;
                double ey = dy + j * by + l * cy;
                double ez = dz + l * cz;
                double r2 = ex * ex + ey * ey + ez * ez;
                if (r2 < best) {
                    best = r2;
                    bxo = ex;
                    byo = ey;
                    bzo = ez;
                }
            }
    *ox = bxo;
    *oy = byo;
    *oz = bzo;
}

static int excluded(int i, int j, const int *ei, const int *ea) {
    if (!ei) return 0;
    for (int k = ei[i]; k < ei[i + 1]; ++k)
        if (ea[k] == j) return 1;
    for (int k = ei[j]; k < ei[j + 1]; ++k)
        if (ea[k] == i) return 1;
    return 0;
}

typedef struct {
    double rc, rc2, krf, crf, beta, fpre;
    int coul, ntypes, mods;
    const double *c6, *c12;
} setup_t;

static setup_t make_setup(double rc, int coul, double eps_r, double eps_rf, double beta,
                          double fcoul, int ntypes, const double *c6, const double *c12, int mods) {
    setup_t s;
    s.rc = rc;
    s.rc2 = rc * rc;
    s.mods = mods;
    if (eps_rf == 0.0)
        s.krf = 1.0 / (2.0 * rc * rc * rc);
    else
        s.krf = (eps_rf - eps_r) / ((2.0 * eps_rf + eps_r) * rc * rc * rc);
    s.crf = 1.0 / rc + s.krf * rc * rc;
    s.beta = beta;
    s.fpre = fcoul / eps_r;
    s.coul = coul;
    s.ntypes = ntypes;
    s.c6 = c6;
    s.c12 = c12;
    return s;
}

/* One pair at squared distance r2 (already known to be inside the cut-off).
 * Returns F/r; writes the energy parts. */
static double pair_terms(const setup_t *s, double r2, double qq, int ti, int tj, double *v_lj,
                         double *v_c, double *e12, double *e6, double *fr_lj, double *fr_c) {
    double r = sqrt(r2);
    double c6 = s->c6[ti * s->ntypes + tj];
    double c12 = s->c12[ti * s->ntypes + tj];
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    double t12 = c12 * ir6 * ir6;
    double t6 = c6 * ir6;
    *e12 = t12;
    *e6 = t6;
    *v_lj = t12 - t6;
    if (s->mods & OR_MOD_LJ_SHIFT) {
        double irc6 = 1.0 / (s->rc2 * s->rc2 * s->rc2);
        *v_lj -= c12 * irc6 * irc6 - c6 * irc6;
    }
    double flj = (12.0 * t12 - 6.0 * t6) * ir2;
    double fc, vc;
    double fq = s->fpre * qq;
    if (s->coul == OR_RF) {
        vc = fq * (1.0 / r + s->krf * r2 - s->crf);
        fc = fq * (1.0 / (r2 * r) - 2.0 * s->krf);
    } else {
        double br = s->beta * r;
        double ec = erfc(br);
        vc = fq * ec / r;
        if (s->mods & OR_MOD_EWALD_SHIFT) vc -= fq * erfc(s->beta * s->rc) / s->rc;
        fc = fq * (ec / r + 2.0 * s->beta / sqrt(M_PI) * exp(-br * br)) * ir2;
    }
    *v_c = vc;
    *fr_lj = flj;
    *fr_c = fc;
    return flj + fc;
}

/* Reaction-field correction of one excluded pair inside the cut-off:
 * returns F/r and writes the energy. */
static double excl_rf_terms(const setup_t *s, double r2, double qq, double *v_c) {
    double fq = s->fpre * qq;
    *v_c = fq * (s->krf * r2 - s->crf);
    return -2.0 * fq * s->krf;
}

/*
 * Energies and virial over all unordered pairs.
 * out[0] = E_LJ, out[1] = E_Coulomb, out[2..10] = virial (row-major 3x3),
 * out[11] = sum c12/r^12, out[12] = sum c6/r^6,
 * out[13] = sum over pairs of d.F (LJ part), out[14] = the same for Coulomb.
 * npairs[0] = number of interacting pairs.
 */
int or_energy_virial_rows(int n, const double *x, const double *q, const int *type, const double *box,
                          double rc, int coul, double eps_r, double eps_rf, double beta, double fcoul,
                          int ntypes, const double *c6, const double *c12, const int *excl_index,
                          const int *excl_atoms, int mods, int i0, int i1, double *out, long long *npairs);

int or_energy_virial(int n, const double *x, const double *q, const int *type, const double *box,
                     double rc, int coul, double eps_r, double eps_rf, double beta, double fcoul,
                     int ntypes, const double *c6, const double *c12, const int *excl_index,
                     const int *excl_atoms, int mods, double *out, long long *npairs) {
    return or_energy_virial_rows(n, x, q, type, box, rc, coul, eps_r, eps_rf, beta, fcoul, ntypes, c6, c12,
                                 excl_index, excl_atoms, mods, 0, n, out, npairs);
}

/*
 * The same sums restricted to the pairs (i, j) with i in [i0, i1), j > i:
 * the sums over consecutive row ranges add up to those of all pairs (a
 * long evaluation can be taken in pieces).
 */
int or_energy_virial_rows(int n, const double *x, const double *q, const int *type, const double *box,
                          double rc, int coul, double eps_r, double eps_rf, double beta, double fcoul,
                          int ntypes, const double *c6, const double *c12, const int *excl_index,
                          const int *excl_atoms, int mods, int i0, int i1, double *out, long long *npairs) {
    if (n < 0 || !out || i0 < 0 || i1 > n || i0 > i1) return 1;
    setup_t s = make_setup(rc, coul, eps_r, eps_rf, beta, fcoul, ntypes, c6, c12, mods);
    double elj = 0, ec = 0, e12 = 0, e6 = 0, rf_lj = 0, rf_c = 0;
    double vxx = 0, vxy = 0, vxz = 0, vyy = 0, vyz = 0, vzz = 0;
    long long np = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : elj, ec, e12, e6, rf_lj, rf_c, vxx, vxy, vxz, vyy, vyz, vzz, np)
    for (int i = i0; i < i1; ++i) {
        for (int j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            pair_image(box, x[3 * i + 0] - x[3 * j + 0], x[3 * i + 1] - x[3 * j + 1],
                       x[3 * i + 2] - x[3 * j + 2], &dx, &dy, &dz);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < s.rc2)) continue;
            double fr;
            if (excluded(i, j, excl_index, excl_atoms)) {
                if (!(s.mods & OR_MOD_RF_EXCL) || s.coul != OR_RF) continue;
                double vc;
                fr = excl_rf_terms(&s, r2, q[i] * q[j], &vc);
                ec += vc;
                rf_c += fr * r2;
            } else {
                double vl, vc, a12, a6, fl, fc;
                fr = pair_terms(&s, r2, q[i] * q[j], type[i], type[j], &vl, &vc, &a12, &a6, &fl, &fc);
                elj += vl;
                ec += vc;
                e12 += a12;
                e6 += a6;
                rf_lj += fl * r2;
                rf_c += fc * r2;
                np += 1;
            }
            vxx -= 0.5 * fr * dx * dx;
            vxy -= 0.5 * fr * dx * dy;
            vxz -= 0.5 * fr * dx * dz;
            vyy -= 0.5 * fr * dy * dy;
            vyz -= 0.5 * fr * dy * dz;
            vzz -= 0.5 * fr * dz * dz;
        }
    }
    out[0] = elj;
    out[1] = ec;
    out[2] = vxx; out[3] = vxy; out[4] = vxz;
    out[5] = vxy; out[6] = vyy; out[7] = vyz;
    out[8] = vxz; out[9] = vyz; out[10] = vzz;
    out[11] = e12;
    out[12] = e6;
    out[13] = rf_lj;
    out[14] = rf_c;
    if (npairs) npairs[0] = np;
    return 0;
}

/*
 * Total force on each selected atom: sum over every other atom j of the pair
 * force (no use of Newton's third law, so every row is independent).
 * sel == NULL selects all atoms (nsel must then equal n).  f: nsel*3.
 */
int or_forces(int n, const double *x, const double *q, const int *type, const double *box,
              double rc, int coul, double eps_r, double eps_rf, double beta, double fcoul,
              int ntypes, const double *c6, const double *c12, const int *excl_index,
              const int *excl_atoms, int mods, int nsel, const int *sel, double *f) {
    if (n < 0 || nsel < 0 || !f) return 1;
    if (!sel && nsel != n) return 1;
    setup_t s = make_setup(rc, coul, eps_r, eps_rf, beta, fcoul, ntypes, c6, c12, mods);
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < nsel; ++k) {
        int i = sel ? sel[k] : k;
        double fx = 0, fy = 0, fz = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx, dy, dz;
            pair_image(box, x[3 * i + 0] - x[3 * j + 0], x[3 * i + 1] - x[3 * j + 1],
                       x[3 * i + 2] - x[3 * j + 2], &dx, &dy, &dz);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < s.rc2)) continue;
            double fr;
            if (excluded(i, j, excl_index, excl_atoms)) {
                if (!(s.mods & OR_MOD_RF_EXCL) || s.coul != OR_RF) continue;
                double vc;
                fr = excl_rf_terms(&s, r2, q[i] * q[j], &vc);
            } else {
                double vl, vc, a12, a6, fl, fc;
                fr = pair_terms(&s, r2, q[i] * q[j], type[i], type[j], &vl, &vc, &a12, &a6, &fl, &fc);
            }
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
        }
        f[3 * k + 0] = fx;
        f[3 * k + 1] = fy;
        f[3 * k + 2] = fz;
    }
    return 0;
}

/*
 * The set of interacting pairs: every unordered pair i < j, not excluded,
 * with minimum-image r^2 < r_cut^2 (evaluated in double precision).
 * counts: n entries (pairs whose lower index is i).  If pairs != NULL it
 * receives 2 ints per pair (i, j), ordered by i then j, and must hold the
 * total given by a previous count-only call.  Returns the total, or -1.
 */
long long or_pairs(int n, const double *x, const double *box, double r_cut, const int *excl_index,
                   const int *excl_atoms, long long *counts, int *pairs) {
    if (n < 0 || !counts) return -1;
    double rc2 = r_cut * r_cut;
    if (!pairs) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            long long c = 0;
            for (int j = i + 1; j < n; ++j) {
                double dx, dy, dz;
                pair_image(box, x[3 * i + 0] - x[3 * j + 0], x[3 * i + 1] - x[3 * j + 1],
                           x[3 * i + 2] - x[3 * j + 2], &dx, &dy, &dz);
                if (!(dx * dx + dy * dy + dz * dz < rc2)) continue;
                if (excluded(i, j, excl_index, excl_atoms)) continue;
                ++c;
            }
            counts[i] = c;
        }
    }
    long long total = 0;
    for (int i = 0; i < n; ++i) total += counts[i];
    if (!pairs) return total;
    long long *start = (long long *)malloc(sizeof(long long) * (size_t)(n + 1));
    if (!start) return -1;
    start[0] = 0;
    for (int i = 0; i < n; ++i) start[i + 1] = start[i] + counts[i];
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        long long w = start[i];
        for (int j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            pair_image(box, x[3 * i + 0] - x[3 * j + 0], x[3 * i + 1] - x[3 * j + 1],
                       x[3 * i + 2] - x[3 * j + 2], &dx, &dy, &dz);
            if (!(dx * dx + dy * dy + dz * dz < rc2)) continue;
            if (excluded(i, j, excl_index, excl_atoms)) continue;
            pairs[2 * w + 0] = i;
            pairs[2 * w + 1] = j;
            ++w;
        }
    }
    free(start);
    return total;
}

/*
 * The interacting pairs of selected atoms: for each selected atom i =
 * sel[k], every other atom j (either side of i), not excluded, with
 * minimum-image r^2 < r_cut^2 (double precision), reported as the unordered
 * pair (min(i, j), max(i, j)).  This is the row i of the plain definition
 * above, so the union over all atoms is the set or_pairs gives; it costs
 * O(N) per selected atom and so reaches boxes where the full O(N^2) set is
 * out of reach.  counts: nsel entries.  If pairs != NULL it receives 2 ints
 * per pair, ordered by k then j, and must hold the total of a previous
 * count-only call.  Returns the total, or -1.  A pair of two selected atoms
 * appears under both of them.
 */
long long or_pairs_rows(int n, const double *x, const double *box, double r_cut, const int *excl_index,
                        const int *excl_atoms, int nsel, const int *sel, long long *counts, int *pairs) {
    if (n < 0 || nsel < 0 || !counts || !sel) return -1;
    for (int k = 0; k < nsel; ++k)
        if (sel[k] < 0 || sel[k] >= n) return -1;
    double rc2 = r_cut * r_cut;
    if (!pairs) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int k = 0; k < nsel; ++k) {
            int i = sel[k];
            long long c = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double dx, dy, dz;
                pair_image(box, x[3 * i + 0] - x[3 * j + 0], x[3 * i + 1] - x[3 * j + 1],
                           x[3 * i + 2] - x[3 * j + 2], &dx, &dy, &dz);
                if (!(dx * dx + dy * dy + dz * dz < rc2)) continue;
                if (excluded(i, j, excl_index, excl_atoms)) continue;
                ++c;
            }
            counts[k] = c;
        }
    }
    long long total = 0;
    for (int k = 0; k < nsel; ++k) total += counts[k];
    if (!pairs) return total;
    long long *start = (long long *)malloc(sizeof(long long) * (size_t)(nsel + 1));
    if (!start) return -1;
    start[0] = 0;
    for (int k = 0; k < nsel; ++k) start[k + 1] = start[k] + counts[k];
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < nsel; ++k) {
        int i = sel[k];
        long long w = start[k];
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx, dy, dz;
            pair_image(box, x[3 * i + 0] - x[3 * j + 0], x[3 * i + 1] - x[3 * j + 1],
                       x[3 * i + 2] - x[3 * j + 2], &dx, &dy, &dz);
            if (!(dx * dx + dy * dy + dz * dz < rc2)) continue;
            if (excluded(i, j, excl_index, excl_atoms)) continue;
            pairs[2 * w + 0] = i < j ? i : j;
            pairs[2 * w + 1] = i < j ? j : i;
            ++w;
        }
    }
    free(start);
    return total;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
