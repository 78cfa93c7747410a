/*
 * md_oracle.c -- plain, slow FP64 CPU oracle for the united-atom polyethylene
 * MD step of Xu et al., "Molecular Dynamics Simulation of Macromolecules Using
 * Graphics Processing Unit".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything is double precision and written as the definitions read:
 *   - Eq. (1)-(3): E = E_nb + E_b + E_a + E_d
 *   - Eq. (2): Lennard-Jones 4 eps [(s/r)^12 - (s/r)^6], truncated at r_c
 *     (pairs with r^2 >= r_c^2 contribute nothing, Sec. 3.2 listing), with
 *     1-2 and 1-3 bonded neighbours excluded (Sec. 3.1, Dreiding II);
 *     lj_form = 1 selects a force-shifted variant (not the paper's) used
 *     only by the gradient checks
 *   - Eq. (4): 1/2 k_b (r - b)^2
 *   - Eq. (5): 1/2 k_a (theta - theta0)^2, harmonic in theta
 *   - Eq. (6): k_phi (1 + cos(n phi - phi_s)), IUPAC phi (trans = 180 deg)
 *   - Sec. 3.3: per-molecule-type topology lists (t_bonds, t_angles and the
 *     dihedral analogue) built from a bond graph, and t_exclusions
 *   - Sec. 3.1: binning into cubic cells by position, cell index per atom
 *   - Sec. 3 / 3.4: time integration (velocity Verlet, which gives the same
 *     positions as the Leap-Frog scheme the paper names)
 * Readings of the paper where it is silent or garbled (parameter table,
 * mixing rule, thermostat) are taken by the caller, which passes parameters.
 *
 * Build with -ffp-contract=off so that no a*b+c is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* force-field parameters; index 0 = C_32 (CH2), 1 = C_33 (CH3) */
typedef struct {
    double eps[2], sigma[2], mass[2];
    double kb, b0;           /* Eq. (4): kJ/mol/nm^2, nm */
    double ka, theta0;       /* Eq. (5): kJ/mol/rad^2, rad */
    double kphi, phis;       /* Eq. (6): kJ/mol, rad */
    int32_t n_mult, pad;     /* Eq. (6): periodicity n */
    double rc;               /* LJ cutoff, nm */
    int32_t lj_form, pad2;   /* 0: Eq. (2) truncated at r_c (the paper's);
                                1: force-shifted variant for gradient checks */
} orc_ff;

/* ------------------------------------------------------------------ */
/* Topology (Sec. 3.3).  One molecule type with `naom` atoms (NAOM, Table II)
 * and an undirected bond list.  Angles are the paths a-b-c (vertex b), listed
 * by ascending vertex, then ascending (a, c); dihedrals are the paths a-b-c-d
 * over each bond b-c (b < c, in bond-list order).                          */

static int cmp_int(const void *a, const void *b) { return (*(const int *)a > *(const int *)b) - (*(const int *)a < *(const int *)b); }

/* neighbours of every atom, sorted ascending: nb_index[naom+1], nb[2*nbond] */
static void adjacency(int naom, int nbond, const int32_t *bonds, int *nb_index, int *nb) {
    int *deg = (int *)calloc(naom, sizeof(int));
    for (int k = 0; k < nbond; ++k) { deg[bonds[2 * k]]++; deg[bonds[2 * k + 1]]++; }
    nb_index[0] = 0;
    for (int a = 0; a < naom; ++a) nb_index[a + 1] = nb_index[a] + deg[a];
    int *fill = (int *)calloc(naom, sizeof(int));
    for (int k = 0; k < nbond; ++k) {
        int a = bonds[2 * k], b = bonds[2 * k + 1];
        nb[nb_index[a] + fill[a]++] = b;
        nb[nb_index[b] + fill[b]++] = a;
    }
    for (int a = 0; a < naom; ++a) qsort(nb + nb_index[a], deg[a], sizeof(int), cmp_int);
    free(deg); free(fill);
}

/* t_bonds (Sec. 3.3): index[naom+1], bond[2*nbond] (neighbour atom ids) */
int orc_topo_bonds(int naom, int nbond, const int32_t *bonds, int32_t *index, int32_t *bond) {
    int *nbi = (int *)malloc(sizeof(int) * (naom + 1)), *nb = (int *)malloc(sizeof(int) * 2 * nbond);
    adjacency(naom, nbond, bonds, nbi, nb);
    for (int a = 0; a <= naom; ++a) index[a] = nbi[a];
    for (int k = 0; k < 2 * nbond; ++k) bond[k] = nb[k];
    free(nbi); free(nb);
    return 0;
}

/* t_exclusions (Sec. 3.1): per atom, its 1-2 and 1-3 neighbours, ascending */
int orc_topo_exclusions(int naom, int nbond, const int32_t *bonds, int32_t *index, int32_t *excl, int cap) {
    int *nbi = (int *)malloc(sizeof(int) * (naom + 1)), *nb = (int *)malloc(sizeof(int) * 2 * nbond);
    adjacency(naom, nbond, bonds, nbi, nb);
    int *tmp = (int *)malloc(sizeof(int) * (naom + 1));
    int n = 0;
    index[0] = 0;
    for (int a = 0; a < naom; ++a) {
        int t = 0;
        for (int p = nbi[a]; p < nbi[a + 1]; ++p) {
            int b = nb[p];
            tmp[t++] = b;
            for (int q = nbi[b]; q < nbi[b + 1]; ++q) if (nb[q] != a) tmp[t++] = nb[q];
        }
        qsort(tmp, t, sizeof(int), cmp_int);
        for (int s = 0; s < t; ++s) {
            if (s > 0 && tmp[s] == tmp[s - 1]) continue;
            if (n >= cap) { free(nbi); free(nb); free(tmp); return -1; }
            excl[n++] = tmp[s];
        }
        index[a + 1] = n;
    }
    free(nbi); free(nb); free(tmp);
    return n;
}

/* unique angles (a,b,c), vertex b; returns count (<= cap) */
int orc_topo_angles(int naom, int nbond, const int32_t *bonds, int32_t *angles, int cap) {
    int *nbi = (int *)malloc(sizeof(int) * (naom + 1)), *nb = (int *)malloc(sizeof(int) * 2 * nbond);
    adjacency(naom, nbond, bonds, nbi, nb);
    int n = 0;
    for (int b = 0; b < naom; ++b)
        for (int p = nbi[b]; p < nbi[b + 1]; ++p)
            for (int q = p + 1; q < nbi[b + 1]; ++q) {
                if (n >= cap) { free(nbi); free(nb); return -1; }
                angles[3 * n] = nb[p]; angles[3 * n + 1] = b; angles[3 * n + 2] = nb[q];
                ++n;
            }
    free(nbi); free(nb);
    return n;
}

/* unique dihedrals (a,b,c,d) around each bond b-c */
int orc_topo_dihedrals(int naom, int nbond, const int32_t *bonds, int32_t *dih, int cap) {
    int *nbi = (int *)malloc(sizeof(int) * (naom + 1)), *nb = (int *)malloc(sizeof(int) * 2 * nbond);
    adjacency(naom, nbond, bonds, nbi, nb);
    int n = 0;
    for (int k = 0; k < nbond; ++k) {
        int b = bonds[2 * k], c = bonds[2 * k + 1];
        if (b > c) { int t = b; b = c; c = t; }
        for (int p = nbi[b]; p < nbi[b + 1]; ++p) {
            int a = nb[p];
            if (a == c) continue;
            for (int q = nbi[c]; q < nbi[c + 1]; ++q) {
                int d = nb[q];
                if (d == b || d == a) continue;
                if (n >= cap) { free(nbi); free(nb); return -1; }
                dih[4 * n] = a; dih[4 * n + 1] = b; dih[4 * n + 2] = c; dih[4 * n + 3] = d;
                ++n;
            }
        }
    }
    free(nbi); free(nb);
    return n;
}

/*
 * Per-home-atom view of a list of `width`-atom terms (Sec. 3.3, Fig. 5):
 * for each atom, the terms it belongs to in ascending term index, with the
 * atom's 1-based position in the term and the other atoms in term order.
 * index[naom+1]; rows of (term_idx, pos, other_1 .. other_{width-1}).
 */
int orc_topo_home_view(int naom, int nterm, int width, const int32_t *terms, int32_t *index, int32_t *rows) {
    int n = 0;
    index[0] = 0;
    for (int a = 0; a < naom; ++a) {
        for (int t = 0; t < nterm; ++t)
            for (int p = 0; p < width; ++p)
                if (terms[width * t + p] == a) {
                    int32_t *r = rows + (width + 1) * n;
                    r[0] = t; r[1] = p + 1;
                    int o = 2;
                    for (int q = 0; q < width; ++q) if (q != p) r[o++] = terms[width * t + q];
                    ++n;
                }
        index[a + 1] = n;
    }
    return n;
}

/* ------------------------------------------------------------------ */
/* Lennard-Jones (Eq. 2) with geometric mixing of eps and sigma.         */

/* e_rc = E(r_c); dphi_rc = dE/dr at r_c, used by the force-shifted variant
 * E_sf(r) = E(r) - E(r_c) - (r - r_c) dE/dr(r_c), whose force vanishes at
 * r_c (not part of the paper's method; it makes the trajectory a smooth
 * function of the parameters for the gradient checks). */
typedef struct { double c6, c12, e_rc, dphi_rc, rc; int form; } lj_pair;

static void lj_table(const orc_ff *ff, lj_pair tab[2][2]) {
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double eps = sqrt(ff->eps[a] * ff->eps[b]);
            double sig = sqrt(ff->sigma[a] * ff->sigma[b]);
            double s6 = sig * sig * sig * sig * sig * sig;
            tab[a][b].c6 = 4.0 * eps * s6;
            tab[a][b].c12 = 4.0 * eps * s6 * s6;
            double ir6 = 1.0 / (ff->rc * ff->rc * ff->rc * ff->rc * ff->rc * ff->rc);
            tab[a][b].e_rc = tab[a][b].c12 * ir6 * ir6 - tab[a][b].c6 * ir6;
            tab[a][b].dphi_rc = (-12.0 * tab[a][b].c12 * ir6 * ir6 + 6.0 * tab[a][b].c6 * ir6) / ff->rc;
            tab[a][b].rc = ff->rc;
            tab[a][b].form = ff->lj_form;
        }
}

static double min_image(double d, double L) { return d - L * floor(d / L + 0.5); }

/* is MAIDX b an excluded partner of MAIDX a within one molecule? */
static int excluded(int a, int b, const int32_t *ei, const int32_t *ex) {
    if (a == b) return 1;
    for (int p = ei[a]; p < ei[a + 1]; ++p) if (ex[p] == b) return 1;
    return 0;
}

/* one pair: returns 1 if inside the cutoff; fills F on i (along d = x_i - x_j) */
static int lj_one(const lj_pair *P, double rc2, const double d[3], double fi[3], double *e, double *es) {
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 >= rc2) return 0;
    double ir2 = 1.0 / r2, ir6 = ir2 * ir2 * ir2;
    double fr = ir2 * ir6 * (12.0 * P->c12 * ir6 - 6.0 * P->c6);   /* |F|/r */
    *e = P->c12 * ir6 * ir6 - P->c6 * ir6;
    *es = *e - P->e_rc;
    if (P->form == 1) {
        double r = sqrt(r2);
        fr += P->dphi_rc / r;
        *es -= (r - P->rc) * P->dphi_rc;
    }
    for (int a = 0; a < 3; ++a) fi[a] = fr * d[a];
    return 1;
}

/* common arguments describing a system of n = n_mol * naom atoms */
#define SYS_ARGS int64_t n, const double *x, double L, int32_t naom, const int32_t *type_m, \
                 const int32_t *excl_index, const int32_t *excl, const orc_ff *ff

/* All pairs i < j under the minimum image (the definition). */
int orc_lj_brute(SYS_ARGS, double *f, double *en, double *vir) {
    lj_pair tab[2][2];
    lj_table(ff, tab);
    double rc2 = ff->rc * ff->rc, E = 0.0, ES = 0.0, W[6] = { 0 };
    memset(f, 0, sizeof(double) * 3 * n);
    for (int64_t i = 0; i < n; ++i) {
        int mi = (int)(i / naom), ai = (int)(i % naom);
        for (int64_t j = i + 1; j < n; ++j) {
            int mj = (int)(j / naom), aj = (int)(j % naom);
            if (mi == mj && excluded(ai, aj, excl_index, excl)) continue;
            double d[3], fi[3], e, es;
            for (int a = 0; a < 3; ++a) d[a] = min_image(x[3 * i + a] - x[3 * j + a], L);
            if (!lj_one(&tab[type_m[ai]][type_m[aj]], rc2, d, fi, &e, &es)) continue;
            for (int a = 0; a < 3; ++a) { f[3 * i + a] += fi[a]; f[3 * j + a] -= fi[a]; }
            E += e; ES += es;
            W[0] += d[0] * fi[0]; W[1] += d[1] * fi[1]; W[2] += d[2] * fi[2];
            W[3] += d[0] * fi[1]; W[4] += d[0] * fi[2]; W[5] += d[1] * fi[2];
        }
    }
    en[0] = E; en[1] = ES;
    for (int a = 0; a < 6; ++a) vir[a] = W[a];
    return 0;
}

/* Force on selected atoms only, each summed over all other atoms. */
int orc_lj_atoms(SYS_ARGS, int64_t n_sel, const int64_t *sel, double *f_sel, int32_t nthreads) {
    lj_pair tab[2][2];
    lj_table(ff, tab);
    double rc2 = ff->rc * ff->rc;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < n_sel; ++s) {
        int64_t i = sel[s];
        int mi = (int)(i / naom), ai = (int)(i % naom);
        double acc[3] = { 0, 0, 0 };
        for (int64_t j = 0; j < n; ++j) {
            int mj = (int)(j / naom), aj = (int)(j % naom);
            if (j == i || (mi == mj && excluded(ai, aj, excl_index, excl))) continue;
            double d[3], fi[3], e, es;
            for (int a = 0; a < 3; ++a) d[a] = min_image(x[3 * i + a] - x[3 * j + a], L);
            if (lj_one(&tab[type_m[ai]][type_m[aj]], rc2, d, fi, &e, &es))
                for (int a = 0; a < 3; ++a) acc[a] += fi[a];
        }
        for (int a = 0; a < 3; ++a) f_sel[3 * s + a] = acc[a];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Binning (Sec. 3.1): cubic cells of side L/M; cell index per atom from its
 * wrapped position, then atoms listed cell by cell, in atom order inside a
 * cell (a stable counting sort).                                         */

void orc_cell_coords(const double *xi, double L, int32_t M, int c[3]) {
    double inv_h = (double)M / L;
    for (int a = 0; a < 3; ++a) {
        double s = xi[a] - L * floor(xi[a] / L);
        int k = (int)floor(s * inv_h);
        if (k < 0) k = 0;
        if (k > M - 1) k = M - 1;
        c[a] = k;
    }
}

int orc_bin(int64_t n, const double *x, double L, int32_t M, int32_t *cell_of, int32_t *cell_start, int32_t *perm) {
    if (M < 1 || M > 1024) return -1;
    int64_t nc = (int64_t)M * M * M;
    for (int64_t c = 0; c <= nc; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        orc_cell_coords(x + 3 * i, L, M, c);
        cell_of[i] = (c[2] * M + c[1]) * M + c[0];
        cell_start[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) cell_start[c + 1] += cell_start[c];
    int32_t *fill = (int32_t *)calloc((size_t)nc, sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) perm[cell_start[cell_of[i]] + fill[cell_of[i]]++] = (int32_t)i;
    free(fill);
    return 0;
}

/* Cell-list form of orc_lj_brute: same pair set (cells of side >= r_c, the
 * home cell and its 26 neighbours), each atom's force summed over its own
 * neighbours; energy and virial are half-sums over atoms. */
int orc_lj_cells(SYS_ARGS, double *f, double *en, double *vir, int32_t nthreads) {
    int32_t M = (int32_t)floor(L / ff->rc);
    if (M < 3) return orc_lj_brute(n, x, L, naom, type_m, excl_index, excl, ff, f, en, vir);
    lj_pair tab[2][2];
    lj_table(ff, tab);
    double rc2 = ff->rc * ff->rc;
    int64_t nc = (int64_t)M * M * M;
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (nc + 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * n);
    orc_bin(n, x, L, M, cell_of, start, perm);
    double *ea = (double *)calloc(2 * n, sizeof(double));
    double *wa = (double *)calloc(6 * n, sizeof(double));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t i = 0; i < n; ++i) {
        int mi = (int)(i / naom), ai = (int)(i % naom);
        int c[3];
        orc_cell_coords(x + 3 * i, L, M, c);
        double acc[3] = { 0, 0, 0 };
        for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int cx = (c[0] + dx + M) % M, cy = (c[1] + dy + M) % M, cz = (c[2] + dz + M) % M;
            int cell = (cz * M + cy) * M + cx;
            for (int p = start[cell]; p < start[cell + 1]; ++p) {
                int64_t j = perm[p];
                int mj = (int)(j / naom), aj = (int)(j % naom);
                if (j == i || (mi == mj && excluded(ai, aj, excl_index, excl))) continue;
                double d[3], fi[3], e, es;
                for (int a = 0; a < 3; ++a) d[a] = min_image(x[3 * i + a] - x[3 * j + a], L);
                if (!lj_one(&tab[type_m[ai]][type_m[aj]], rc2, d, fi, &e, &es)) continue;
                for (int a = 0; a < 3; ++a) acc[a] += fi[a];
                ea[2 * i] += 0.5 * e; ea[2 * i + 1] += 0.5 * es;
                wa[6 * i + 0] += 0.5 * d[0] * fi[0]; wa[6 * i + 1] += 0.5 * d[1] * fi[1];
                wa[6 * i + 2] += 0.5 * d[2] * fi[2]; wa[6 * i + 3] += 0.5 * d[0] * fi[1];
                wa[6 * i + 4] += 0.5 * d[0] * fi[2]; wa[6 * i + 5] += 0.5 * d[1] * fi[2];
            }
        }
        for (int a = 0; a < 3; ++a) f[3 * i + a] = acc[a];
    }
    en[0] = en[1] = 0.0;
    for (int a = 0; a < 6; ++a) vir[a] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        en[0] += ea[2 * i]; en[1] += ea[2 * i + 1];
        for (int a = 0; a < 6; ++a) vir[a] += wa[6 * i + a];
    }
    free(cell_of); free(start); free(perm); free(ea); free(wa);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Bonded terms, Eqs. (4)-(6).  Term lists are per molecule type and are
 * applied to every molecule (atom = molecule * naom + MAIDX).            */

static void sub_mi(const double *a, const double *b, double L, double *o) {
    for (int q = 0; q < 3; ++q) o[q] = min_image(a[q] - b[q], L);
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void add_vir(double W[6], const double r[3], const double fo[3]) {
    W[0] += r[0] * fo[0]; W[1] += r[1] * fo[1]; W[2] += r[2] * fo[2];
    W[3] += r[0] * fo[1]; W[4] += r[0] * fo[2]; W[5] += r[1] * fo[2];
}

/* Eq. (4).  d = x_b - x_a; F_a = k (r - b0) d/r; F_b = -F_a. */
static double bond_term(const orc_ff *ff, const double *xa, const double *xb, double L, double fa[3], double fb[3], double W[6]) {
    double d[3];
    sub_mi(xb, xa, L, d);
    double r = sqrt(dot3(d, d)), dr = r - ff->b0;
    double g = ff->kb * dr / r;
    for (int q = 0; q < 3; ++q) { fa[q] = g * d[q]; fb[q] = -g * d[q]; }
    add_vir(W, d, fb);   /* positions relative to atom a */
    return 0.5 * ff->kb * dr * dr;
}

/* Eq. (5), vertex b.  u = x_a - x_b, w = x_c - x_b, theta = angle(u, w);
 * dtheta/dx_a = -(w^ - cos u^)/(|u| sin), likewise for c; F = -dE/dtheta * grad. */
static double angle_term(const orc_ff *ff, const double *xa, const double *xb, const double *xc, double L,
                         double fa[3], double fb[3], double fc[3], double W[6]) {
    double u[3], w[3], cr[3];
    sub_mi(xa, xb, L, u);
    sub_mi(xc, xb, L, w);
    double lu = sqrt(dot3(u, u)), lw = sqrt(dot3(w, w));
    cross3(u, w, cr);
    double s = sqrt(dot3(cr, cr)), c = dot3(u, w);
    double th = atan2(s, c);
    double dth = th - ff->theta0;
    double E = 0.5 * ff->ka * dth * dth;
    double sin_t = s / (lu * lw), cos_t = c / (lu * lw);
    if (sin_t < 1e-12) {   /* collinear: gradient direction undefined, force set to 0 */
        for (int q = 0; q < 3; ++q) fa[q] = fb[q] = fc[q] = 0.0;
        return E;
    }
    double g = ff->ka * dth / sin_t;
    for (int q = 0; q < 3; ++q) {
        double uh = u[q] / lu, wh = w[q] / lw;
        fa[q] = g * (wh - cos_t * uh) / lu;
        fc[q] = g * (uh - cos_t * wh) / lw;
        fb[q] = -fa[q] - fc[q];
    }
    add_vir(W, u, fa);
    add_vir(W, w, fc);
    return E;
}

/* Eq. (6).  b1 = x_b - x_a, b2 = x_c - x_b, b3 = x_d - x_c, m = b1 x b2,
 * n = b2 x b3, phi = atan2(|b2| b1.n, m.n) (trans = 180 deg).  Gradient of
 * phi after Blondel & Karplus, J. Comput. Chem. 17, 1132 (1996):
 *   dphi/dx_a = -|b2|/|m|^2 m,  dphi/dx_d = |b2|/|n|^2 n,
 *   dphi/dx_b = (|b2|/|m|^2 + b1.b2/(|b2||m|^2)) m + b2.b3/(|b2||n|^2) n,
 *   dphi/dx_c = -(dphi/dx_a + dphi/dx_b + dphi/dx_d).                   */
static double dihedral_term(const orc_ff *ff, const double *xa, const double *xb, const double *xc, const double *xd,
                            double L, double fa[3], double fb[3], double fc[3], double fd[3], double W[6]) {
    double b1[3], b2[3], b3[3], m[3], nn[3];
    sub_mi(xb, xa, L, b1);
    sub_mi(xc, xb, L, b2);
    sub_mi(xd, xc, L, b3);
    cross3(b1, b2, m);
    cross3(b2, b3, nn);
    double lb2 = sqrt(dot3(b2, b2)), m2 = dot3(m, m), n2 = dot3(nn, nn);
    double phi = atan2(lb2 * dot3(b1, nn), dot3(m, nn));
    double arg = ff->n_mult * phi - ff->phis;
    double E = ff->kphi * (1.0 + cos(arg));
    if (m2 < 1e-24 || n2 < 1e-24) {   /* collinear triple: phi undefined, force set to 0 */
        for (int q = 0; q < 3; ++q) fa[q] = fb[q] = fc[q] = fd[q] = 0.0;
        return E;
    }
    double dEdphi = -ff->kphi * ff->n_mult * sin(arg);
    double ca = -lb2 / m2, cd = lb2 / n2;
    double cbm = lb2 / m2 + dot3(b1, b2) / (lb2 * m2), cbn = dot3(b2, b3) / (lb2 * n2);
    for (int q = 0; q < 3; ++q) {
        double ga = ca * m[q], gd = cd * nn[q], gb = cbm * m[q] + cbn * nn[q];
        double gc = -(ga + gb + gd);
        fa[q] = -dEdphi * ga; fb[q] = -dEdphi * gb; fc[q] = -dEdphi * gc; fd[q] = -dEdphi * gd;
    }
    /* virial with positions relative to atom a */
    double rb[3] = { b1[0], b1[1], b1[2] };
    double rc_[3] = { b1[0] + b2[0], b1[1] + b2[1], b1[2] + b2[2] };
    double rd[3] = { rc_[0] + b3[0], rc_[1] + b3[1], rc_[2] + b3[2] };
    add_vir(W, rb, fb); add_vir(W, rc_, fc); add_vir(W, rd, fd);
    return E;
}

/* Sum of Eqs. (4)-(6) over all molecules.  en[3] = bond, angle, dihedral.
 * f is overwritten. */
int orc_bonded(int64_t n_mol, int32_t naom, const double *x, double L,
               int32_t nb, const int32_t *bonds, int32_t na, const int32_t *angles,
               int32_t nd, const int32_t *dih, const orc_ff *ff, double *f, double *en, double *vir) {
    int64_t n = n_mol * naom;
    memset(f, 0, sizeof(double) * 3 * n);
    double Eb = 0, Ea = 0, Ed = 0, W[6] = { 0 };
    for (int64_t mol = 0; mol < n_mol; ++mol) {
        int64_t o = mol * naom;
        for (int t = 0; t < nb; ++t) {
            int64_t a = o + bonds[2 * t], b = o + bonds[2 * t + 1];
            double fa[3], fb[3];
            Eb += bond_term(ff, x + 3 * a, x + 3 * b, L, fa, fb, W);
            for (int q = 0; q < 3; ++q) { f[3 * a + q] += fa[q]; f[3 * b + q] += fb[q]; }
        }
        for (int t = 0; t < na; ++t) {
            int64_t a = o + angles[3 * t], b = o + angles[3 * t + 1], c = o + angles[3 * t + 2];
            double fa[3], fb[3], fc[3];
            Ea += angle_term(ff, x + 3 * a, x + 3 * b, x + 3 * c, L, fa, fb, fc, W);
            for (int q = 0; q < 3; ++q) { f[3 * a + q] += fa[q]; f[3 * b + q] += fb[q]; f[3 * c + q] += fc[q]; }
        }
        for (int t = 0; t < nd; ++t) {
            int64_t a = o + dih[4 * t], b = o + dih[4 * t + 1], c = o + dih[4 * t + 2], d = o + dih[4 * t + 3];
            double fa[3], fb[3], fc[3], fd[3];
            Ed += dihedral_term(ff, x + 3 * a, x + 3 * b, x + 3 * c, x + 3 * d, L, fa, fb, fc, fd, W);
            for (int q = 0; q < 3; ++q) {
                f[3 * a + q] += fa[q]; f[3 * b + q] += fb[q]; f[3 * c + q] += fc[q]; f[3 * d + q] += fd[q];
            }
        }
    }
    en[0] = Eb; en[1] = Ea; en[2] = Ed;
    for (int a = 0; a < 6; ++a) vir[a] = W[a];
    return 0;
}

/* ------------------------------------------------------------------ */
/* A whole system and its time integration.                             */

typedef struct {
    int64_t n_mol;
    int32_t naom;
    int32_t nb, na, nd, pad;
    const int32_t *type_m, *excl_index, *excl, *bonds, *angles, *dih;
    double L;
    int32_t use_cells, nthreads;
} orc_sys;

/* total force and energies: en[7] = lj, lj_shifted, bond, angle, dihedral,
 * (unused), (unused); vir[6] = total virial */
int orc_forces(const orc_sys *S, const orc_ff *ff, const double *x, double *f, double *en, double *vir) {
    int64_t n = S->n_mol * S->naom;
    double *fb = (double *)malloc(sizeof(double) * 3 * n);
    double enl[2], vl[6], enb[3], vb[6];
    if (S->use_cells)
        orc_lj_cells(n, x, S->L, S->naom, S->type_m, S->excl_index, S->excl, ff, f, enl, vl, S->nthreads);
    else
        orc_lj_brute(n, x, S->L, S->naom, S->type_m, S->excl_index, S->excl, ff, f, enl, vl);
    orc_bonded(S->n_mol, S->naom, x, S->L, S->nb, S->bonds, S->na, S->angles, S->nd, S->dih, ff, fb, enb, vb);
    for (int64_t i = 0; i < 3 * n; ++i) f[i] += fb[i];
    en[0] = enl[0]; en[1] = enl[1]; en[2] = enb[0]; en[3] = enb[1]; en[4] = enb[2]; en[5] = en[6] = 0.0;
    for (int a = 0; a < 6; ++a) vir[a] = vl[a] + vb[a];
    free(fb);
    return 0;
}

/*
 * Velocity Verlet for n_steps (same positions as Leap-Frog, Sec. 3.4).
 * Optional weak-coupling velocity rescaling (the paper names Nose-Hoover
 * but fixes no thermostat for a quench; this is the reading used here):
 * at the start of step k the full-step velocities v(t_k) are multiplied by
 *     lambda_{k-1} = sqrt(1 + (dt/tau) (T0/T_{k-1} - 1)),
 * where T_{k-1} is the temperature of the unscaled v(t_{k-1}); lambda is 1
 * before any temperature is known (*lambda on entry carries it between calls).
 * Temperature uses 3N-3 degrees of freedom.
 *
 * x is unwrapped (minimum images are taken inside the force routines).
 * Every `sample_every` steps (and at step 0) a row of 8 numbers is written to
 * samples: step, lj, lj_shifted, bond, angle, dihedral, kinetic, T.  The
 * energies of row k are those of x(t_k) and of the unscaled v(t_k).
 * Returns the number of rows written.
 */
int orc_run(const orc_sys *S, const orc_ff *ff, const double *mass_m, double *x, double *v, double *f,
            double dt, int64_t n_steps, int32_t thermostat, double T0, double tau, double kB,
            double *lambda, int64_t sample_every, double *samples) {
    int64_t n = S->n_mol * S->naom;
    double *m = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) m[i] = mass_m[i % S->naom];
    double en[7], vir[6];
    orc_forces(S, ff, x, f, en, vir);
    double dof = 3.0 * (double)n - 3.0;
    double lam = *lambda;
    int rows = 0;
    for (int64_t k = 0; k <= n_steps; ++k) {
        double ke = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 3; ++q) ke += 0.5 * m[i] * v[3 * i + q] * v[3 * i + q];
        double T = 2.0 * ke / (dof * kB);
        if (sample_every > 0 && (k % sample_every == 0)) {
            double *r = samples + 8 * rows++;
            r[0] = (double)k; r[1] = en[0]; r[2] = en[1]; r[3] = en[2]; r[4] = en[3]; r[5] = en[4];
            r[6] = ke; r[7] = T;
        }
        if (k == n_steps) break;
        /* scale v(t_k) by the factor from the previous temperature */
        for (int64_t i = 0; i < 3 * n; ++i) v[i] *= lam;
        lam = thermostat ? sqrt(1.0 + dt / tau * (T0 / T - 1.0)) : 1.0;
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 3; ++q) {
                v[3 * i + q] += 0.5 * dt * f[3 * i + q] / m[i];
                x[3 * i + q] += dt * v[3 * i + q];
            }
        orc_forces(S, ff, x, f, en, vir);
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 3; ++q) v[3 * i + q] += 0.5 * dt * f[3 * i + q] / m[i];
    }
    *lambda = lam;
    free(m);
    return rows;
}

/*
 * NVT run with the paper's integrator and thermostat: Leap-Frog (Sec. 2,
 * Sec. 3.4) with Nose-Hoover coupling (the extended-ensemble method of
 * Sec. 2), and removal of the centre-of-mass translation (Sec. 2).  The paper
 * prints no formulas; this is the standard leap-frog Nose-Hoover scheme for
 *   dv/dt = F/m - xi v,   dxi/dt = (T - T0) / Q,   Q = tau^2 T0 / (4 pi^2):
 *   v_{k+1/2} = [v_{k-1/2} (1 - c_k) + dt F_k / m] / (1 + c_k),  c_k = dt xi_k / 2,
 *   x_{k+1}   = x_k + dt v_{k+1/2},
 *   xi_{k+1}  = xi_k + dt (T_{k+1/2} - T0) / Q    (midpoint rule),
 * T_{k+1/2} the temperature (3N - 3 degrees of freedom) of v_{k+1/2}.  The
 * step goes through the on-step velocity
 *   v_k = (v_{k-1/2} + dt F_k / (2m)) / (1 + c_k),
 * from which v_{k+1/2} = (1 - c_k) v_k + dt F_k / (2m) is the same update.
 * After the drift and T_{k+1/2}, the centre-of-mass velocity of v_{k+1/2} is
 * subtracted.
 * In: v = v_0 (on step), *xi_io = xi_0.  Out: x_K, v_K, F_K, *xi_io = xi_K.
 * Sample rows (10 values): k, lj, lj_shifted, bond, angle, dihedral, kinetic,
 * T, xi_k, eta_k with eta the trapezoidal integral of xi; with them
 *   H = K + U + g kB Q xi^2 / 2 + g kB T0 eta,  g = 3N - 3,
 * is the conserved energy of the extended system.
 */
int orc_run_nh(const orc_sys *S, const orc_ff *ff, const double *mass_m, double *x, double *v, double *f,
               double dt, int64_t n_steps, double T0, double tau, double kB, double *xi_io, int64_t sample_every,
               double *samples) {
    int64_t n = S->n_mol * S->naom;
    double *m = (double *)malloc(sizeof(double) * n);
    double M = 0.0;
    for (int64_t i = 0; i < n; ++i) { m[i] = mass_m[i % S->naom]; M += m[i]; }
    const double pi = 3.14159265358979323846;
    const double dof = 3.0 * (double)n - 3.0;
    const double Q = tau * tau * T0 / (4.0 * pi * pi);
    double xi = *xi_io, eta = 0.0;
    double en[7], vir[6];
    orc_forces(S, ff, x, f, en, vir);
    int rows = 0;
    for (int64_t k = 0; k <= n_steps; ++k) {
        const double c = 0.5 * dt * xi;
        if (k > 0)                                   /* v holds v_{k-1/2}: the on-step velocity */
            for (int64_t i = 0; i < n; ++i)
                for (int q = 0; q < 3; ++q) v[3 * i + q] = (v[3 * i + q] + 0.5 * dt * f[3 * i + q] / m[i]) / (1.0 + c);
        double ke = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 3; ++q) ke += 0.5 * m[i] * v[3 * i + q] * v[3 * i + q];
        const double T = 2.0 * ke / (dof * kB);       /* on-step T_k, reported */
        if (sample_every > 0 && (k % sample_every == 0)) {
            double *r = samples + 10 * rows++;
            r[0] = (double)k; r[1] = en[0]; r[2] = en[1]; r[3] = en[2]; r[4] = en[3]; r[5] = en[4];
            r[6] = ke; r[7] = T; r[8] = xi; r[9] = eta;
        }
        if (k == n_steps) break;
        /* v_{k+1/2} and the drift */
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 3; ++q) {
                v[3 * i + q] = (1.0 - c) * v[3 * i + q] + 0.5 * dt * f[3 * i + q] / m[i];
                x[3 * i + q] += dt * v[3 * i + q];
            }
        /* T_{k+1/2}, then the centre-of-mass translation of v_{k+1/2} removed */
        double ke_h = 0.0, P[3] = { 0.0, 0.0, 0.0 };
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 3; ++q) {
                ke_h += 0.5 * m[i] * v[3 * i + q] * v[3 * i + q];
                P[q] += m[i] * v[3 * i + q];
            }
        for (int64_t i = 0; i < n; ++i)
            for (int q = 0; q < 3; ++q) v[3 * i + q] -= P[q] / M;
        const double T_h = 2.0 * ke_h / (dof * kB);
        const double xi_next = xi + dt * (T_h - T0) / Q;
        eta += 0.5 * dt * (xi + xi_next);
        xi = xi_next;
        orc_forces(S, ff, x, f, en, vir);
    }
    *xi_io = xi;
    free(m);
    return rows;
}

/* Kinetic energy and instantaneous temperature (3N-3 dof). */
double orc_kinetic(int64_t n, int32_t naom, const double *mass_m, const double *v) {
    double ke = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) ke += 0.5 * mass_m[i % naom] * v[3 * i + q] * v[3 * i + q];
    return ke;
}

/*
 * Trajectory means used by the gradient checks.  Two observables of an NVE
 * velocity-Verlet run of n_steps from (x0, v0), x0 unwrapped:
 *   out[0] = 1/(K+1) sum_{k=0..K} U(x_k), U = shifted LJ + bond + angle
 *            + dihedral (Eqs. 1-6, each LJ pair shifted by -E(r_c));
 *   out[1] = 1/(K+1) sum_{k=0..K} 1/n_mol sum_mol |x_last - x_first|^2,
 *            the mean-square end-to-end distance of the chains (the
 *            end-to-end vector of Sec. 4, Fig. 8), from the unwrapped
 *            positions of MAIDX 0 and MAIDX naom-1.
 * x0 and v0 are not modified.
 */
int orc_traj_means(const orc_sys *S, const orc_ff *ff, const double *mass_m, const double *x0, const double *v0,
                   double dt, int64_t n_steps, double *out) {
    int64_t n = S->n_mol * S->naom;
    double *x = (double *)malloc(sizeof(double) * 3 * n);
    double *v = (double *)malloc(sizeof(double) * 3 * n);
    double *f = (double *)malloc(sizeof(double) * 3 * n);
    memcpy(x, x0, sizeof(double) * 3 * n);
    memcpy(v, v0, sizeof(double) * 3 * n);
    double en[7], vir[6], sum_u = 0.0, sum_r2 = 0.0;
    orc_forces(S, ff, x, f, en, vir);
    for (int64_t k = 0; k <= n_steps; ++k) {
        sum_u += en[1] + en[2] + en[3] + en[4];
        double r2 = 0.0;
        for (int64_t mol = 0; mol < S->n_mol; ++mol) {
            const double *a = x + 3 * (mol * S->naom), *b = x + 3 * (mol * S->naom + S->naom - 1);
            double e[3] = { b[0] - a[0], b[1] - a[1], b[2] - a[2] };
            r2 += dot3(e, e);
        }
        sum_r2 += r2 / (double)S->n_mol;
        if (k == n_steps) break;
        for (int64_t i = 0; i < n; ++i) {
            double m = mass_m[i % S->naom];
            for (int q = 0; q < 3; ++q) {
                v[3 * i + q] += 0.5 * dt * f[3 * i + q] / m;
                x[3 * i + q] += dt * v[3 * i + q];
            }
        }
        orc_forces(S, ff, x, f, en, vir);
        for (int64_t i = 0; i < n; ++i) {
            double m = mass_m[i % S->naom];
            for (int q = 0; q < 3; ++q) v[3 * i + q] += 0.5 * dt * f[3 * i + q] / m;
        }
    }
    out[0] = sum_u / (double)(n_steps + 1);
    out[1] = sum_r2 / (double)(n_steps + 1);
    free(x); free(v); free(f);
    return 0;
}
