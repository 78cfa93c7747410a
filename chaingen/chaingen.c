/*
 * chaingen.c -- seeded synthetic inputs for united-atom polyethylene melts.
 *
 * This module builds INPUTS only: chain coordinates grown as random walks and
 * Maxwell velocities.  It contains none of the force field or integrator
 * arithmetic (no energies, no forces); both the CUDA path and the FP64 oracle
 * consume what it writes.
 *
 * Geometry follows the model of Sec. 2: chains of `sites` united atoms, bond
 * length b, tetrahedral bond angle (cos = -1/3, i.e. 109.47 deg, Table I) and
 * dihedrals drawn from {trans (180 deg), gauche+ (+60), gauche- (-60)}.
 * The paper takes its initial structures from earlier work and does not say
 * how they were built; the growth rules below (uniform chain starts, overlap
 * rejection with backtracking, trans/gauche weights) are this generator's own
 * choices.
 *
 * Determinism across x86-64 and aarch64: only +,-,*,/ and sqrt are used (all
 * correctly rounded in IEEE 754), the natural log needed by the Gaussian
 * sampler is a fixed series written below, and the file must be compiled with
 * -ffp-contract=off so no platform fuses a*b+c.  Random numbers come from
 * SplitMix64 (Steele, Lea, Flood 2014; constants as published by Vigna).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---------------- SplitMix64 ---------------- */
typedef struct { uint64_t s; } cg_rng;

static uint64_t cg_next(cg_rng *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* uniform in [0,1) with 53 random bits */
static double cg_unif(cg_rng *r) { return (double)(cg_next(r) >> 11) * (1.0 / 9007199254740992.0); }

uint64_t cg_splitmix64(uint64_t x) { cg_rng r = { x }; return cg_next(&r); }

/* ---------------- portable natural log ----------------
 * ln(x) = e*ln2 + 2*atanh(t), x = m*2^e with m in [sqrt(1/2), sqrt(2)),
 * t = (m-1)/(m+1), |t| < 0.1716; the odd series in t is summed to 1e-18. */
static double cg_ln(double x) {
    int e;
    double m = frexp(x, &e);                /* exact: m in [0.5,1) */
    if (m < 0.70710678118654752) { m *= 2.0; e -= 1; }
    double t = (m - 1.0) / (m + 1.0), t2 = t * t, term = t, s = 0.0;
    for (int k = 0; k < 40; ++k) {
        s += term / (double)(2 * k + 1);
        term *= t2;
    }
    return (double)e * 0.69314718055994530942 + 2.0 * s;
}
/* portable exp for |x| < 50: x = k ln2 + r, Taylor in r, scale by 2^k */
static double cg_exp(double x) {
    double kf = floor(x / 0.69314718055994530942 + 0.5);
    double r = x - kf * 0.69314718055994530942;
    double s = 1.0, term = 1.0;
    for (int n = 1; n < 30; ++n) { term *= r / (double)n; s += term; }
    return ldexp(s, (int)kf);
}
double cg_ln_export(double x) { return cg_ln(x); }
double cg_exp_export(double x) { return cg_exp(x); }

/* standard normal by the Marsaglia polar method */
static double cg_gauss(cg_rng *r, double *spare, int *has_spare) {
    if (*has_spare) { *has_spare = 0; return *spare; }
    double u, v, s;
    do {
        u = 2.0 * cg_unif(r) - 1.0;
        v = 2.0 * cg_unif(r) - 1.0;
        s = u * u + v * v;
    } while (s >= 1.0 || s == 0.0);
    double f = sqrt(-2.0 * cg_ln(s) / s);
    *spare = v * f; *has_spare = 1;
    return u * f;
}

/* ---------------- small vector helpers ---------------- */
static void v_sub(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double v_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v_cross(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void v_unit(double *a) { double n = sqrt(v_dot(a, a)); a[0] /= n; a[1] /= n; a[2] /= n; }

static double wrap(double x, double L) {
    double s = x - L * floor(x / L);
    if (s >= L) s -= L;
    if (s < 0.0) s = 0.0;
    return s;
}

/* random unit vector: rejection from the cube, then normalise */
static void rand_dir(cg_rng *r, double *d) {
    for (;;) {
        d[0] = 2.0 * cg_unif(r) - 1.0; d[1] = 2.0 * cg_unif(r) - 1.0; d[2] = 2.0 * cg_unif(r) - 1.0;
        double s = v_dot(d, d);
        if (s > 1e-4 && s <= 1.0) { v_unit(d); return; }
    }
}

/* ---------------- occupancy grid for overlap tests ---------------- */
typedef struct {
    int G;            /* cells per side */
    double L, g;      /* box, cell side */
    int32_t *head;    /* G^3 */
    int32_t *next;    /* per placed atom */
    int32_t *chain, *idx;
    double *x;        /* unwrapped positions of placed atoms (3n) */
} grid_t;

static int cell_of(const grid_t *gr, const double *p) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
        int k = (int)(wrap(p[a], gr->L) / gr->g);
        if (k >= gr->G) k = gr->G - 1;
        c[a] = k;
    }
    return (c[2] * gr->G + c[1]) * gr->G + c[0];
}

/* smallest minimum-image distance^2 from p to placed atoms, ignoring atoms of
 * chain `ch` whose index is within `skip` of `k` */
static double min_d2(const grid_t *gr, const double *p, int ch, int k, int skip) {
    double best = 1e300;
    int G = gr->G, c0[3];
    for (int a = 0; a < 3; ++a) {
        int q = (int)(wrap(p[a], gr->L) / gr->g);
        if (q >= G) q = G - 1;
        c0[a] = q;
    }
    int span = G >= 3 ? 1 : 0;
    for (int dz = -span; dz <= span; ++dz)
    for (int dy = -span; dy <= span; ++dy)
    for (int dx = -span; dx <= span; ++dx) {
        int cx = (c0[0] + dx + G) % G, cy = (c0[1] + dy + G) % G, cz = (c0[2] + dz + G) % G;
        for (int a = gr->head[(cz * G + cy) * G + cx]; a >= 0; a = gr->next[a]) {
            if (gr->chain[a] == ch && abs(gr->idx[a] - k) <= skip) continue;
            double d[3];
            v_sub(p, gr->x + 3 * a, d);
            for (int q = 0; q < 3; ++q) d[q] -= gr->L * floor(d[q] / gr->L + 0.5);
            double d2 = v_dot(d, d);
            if (d2 < best) best = d2;
        }
    }
    if (G < 3) { /* tiny box: brute force over everything placed */
        best = 1e300;
        for (int c = 0; c < G * G * G; ++c)
            for (int a = gr->head[c]; a >= 0; a = gr->next[a]) {
                if (gr->chain[a] == ch && abs(gr->idx[a] - k) <= skip) continue;
                double d[3];
                v_sub(p, gr->x + 3 * a, d);
                for (int q = 0; q < 3; ++q) d[q] -= gr->L * floor(d[q] / gr->L + 0.5);
                double d2 = v_dot(d, d);
                if (d2 < best) best = d2;
            }
    }
    return best;
}

static void grid_add(grid_t *gr, int a) {
    int c = cell_of(gr, gr->x + 3 * a);
    gr->next[a] = gr->head[c];
    gr->head[c] = a;
}
/* remove atom a (it is always at the head of its cell's list, because atoms
 * are removed in reverse order of insertion) */
static void grid_remove(grid_t *gr, int a) {
    int c = cell_of(gr, gr->x + 3 * a);
    if (gr->head[c] == a) { gr->head[c] = gr->next[a]; return; }
    for (int b = gr->head[c]; b >= 0; b = gr->next[b])
        if (gr->next[b] == a) { gr->next[b] = gr->next[a]; return; }
}

/*
 * Candidate position of site k of a chain whose earlier sites are at
 * x[k-1], x[k-2], x[k-3] (unwrapped).  `choice` selects the dihedral:
 * 0 trans, 1 gauche+, 2 gauche-.  The bond angle at x[k-1] is tetrahedral:
 * the new bond makes cos = 1/3 with the previous bond direction.
 */
static void place_dihedral(const double *xa, const double *xb, const double *xc, double b, int choice, double *out) {
    /* xa = x[k-3], xb = x[k-2], xc = x[k-1] */
    double u[3], w[3], e[3], t[3];
    v_sub(xc, xb, u); v_unit(u);               /* previous bond direction */
    double q[3]; v_sub(xa, xb, q);             /* towards x[k-3] */
    double qu = v_dot(q, u);
    for (int a = 0; a < 3; ++a) w[a] = q[a] - qu * u[a];
    v_unit(w);                                  /* in-plane, pointing to x[k-3] side */
    for (int a = 0; a < 3; ++a) w[a] = -w[a];   /* trans side */
    v_cross(u, w, t);                           /* completes the frame */
    double c, s;
    if (choice == 0) { c = 1.0; s = 0.0; }
    else { c = -0.5; s = (choice == 1 ? 1.0 : -1.0) * sqrt(3.0) * 0.5; }
    for (int a = 0; a < 3; ++a) e[a] = c * w[a] + s * t[a];
    double cb = 1.0 / 3.0, sb = sqrt(8.0) / 3.0;
    for (int a = 0; a < 3; ++a) out[a] = xc[a] + b * (cb * u[a] + sb * e[a]);
}

/* site at tetrahedral angle from the bond x0->x1, direction otherwise random */
static void place_angle(cg_rng *r, const double *x0, const double *x1, double b, double *out) {
    double u[3], d[3], e[3];
    v_sub(x1, x0, u); v_unit(u);
    for (;;) {
        rand_dir(r, d);
        double du = v_dot(d, u);
        for (int a = 0; a < 3; ++a) e[a] = d[a] - du * u[a];
        if (v_dot(e, e) > 1e-3) break;
    }
    v_unit(e);
    double cb = 1.0 / 3.0, sb = sqrt(8.0) / 3.0;
    for (int a = 0; a < 3; ++a) out[a] = x1[a] + b * (cb * u[a] + sb * e[a]);
}

/*
 * Grow n_chains chains of `sites` atoms in a periodic cube of side L.
 *   r_min     : non-bonded sites (other chains, or |di| >= 4 in the chain)
 *               are kept at least r_min apart (minimum image) when possible
 *   p_trans   : probability of the trans dihedral; gauche+/- share the rest
 * Output (caller-allocated): pos[3*N] wrapped into [0,L), in chain-major
 * order (atom = chain*sites + index).  Returns the number of sites that had
 * to be placed with a relaxed spacing (0 if every rejection test passed).
 */
int cg_grow_chains(int32_t n_chains, int32_t sites, double L, double bond, double r_min,
                   double p_trans, uint64_t seed, double *pos) {
    int64_t N = (int64_t)n_chains * sites;
    cg_rng rng = { seed };
    grid_t gr;
    gr.L = L;
    gr.G = (int)(L / r_min);
    if (gr.G < 1) gr.G = 1;
    if (gr.G > 512) gr.G = 512;
    gr.g = L / gr.G;
    int64_t G3 = (int64_t)gr.G * gr.G * gr.G;
    gr.head = (int32_t *)malloc(sizeof(int32_t) * G3);
    gr.next = (int32_t *)malloc(sizeof(int32_t) * N);
    gr.chain = (int32_t *)malloc(sizeof(int32_t) * N);
    gr.idx = (int32_t *)malloc(sizeof(int32_t) * N);
    gr.x = (double *)malloc(sizeof(double) * 3 * N);
    for (int64_t c = 0; c < G3; ++c) gr.head[c] = -1;
    int relaxed = 0;
    double rmin2 = r_min * r_min;

    for (int ch = 0; ch < n_chains; ++ch) {
        int base = ch * sites;
        double r2 = rmin2;         /* relaxed after repeated failures */
        int restarts = 0;
        for (;;) {                 /* whole-chain attempts */
            int k = 0, backtracks = 0, ok_chain = 1;
            while (k < sites) {
                int a = base + k;
                gr.chain[a] = ch; gr.idx[a] = k;
                double cand[3], best[3], bestd = -1.0;
                int placed = 0;
                if (k < 3) {
                    for (int t = 0; t < 30 && !placed; ++t) {
                        if (k == 0) for (int q = 0; q < 3; ++q) cand[q] = L * cg_unif(&rng);
                        else if (k == 1) {
                            double d[3]; rand_dir(&rng, d);
                            for (int q = 0; q < 3; ++q) cand[q] = gr.x[3 * (a - 1) + q] + bond * d[q];
                        } else place_angle(&rng, gr.x + 3 * (a - 2), gr.x + 3 * (a - 1), bond, cand);
                        double d2 = min_d2(&gr, cand, ch, k, 3);
                        if (d2 >= r2) placed = 1;
                        else if (d2 > bestd) { bestd = d2; memcpy(best, cand, sizeof best); }
                    }
                } else {
                    int order[3];
                    double u = cg_unif(&rng);
                    double pg = 0.5 * (1.0 - p_trans);
                    order[0] = u < p_trans ? 0 : (u < p_trans + pg ? 1 : 2);
                    int o1 = (order[0] + 1) % 3, o2 = (order[0] + 2) % 3;
                    if (cg_unif(&rng) < 0.5) { order[1] = o1; order[2] = o2; } else { order[1] = o2; order[2] = o1; }
                    for (int t = 0; t < 3 && !placed; ++t) {
                        place_dihedral(gr.x + 3 * (a - 3), gr.x + 3 * (a - 2), gr.x + 3 * (a - 1), bond, order[t], cand);
                        double d2 = min_d2(&gr, cand, ch, k, 3);
                        if (d2 >= r2) placed = 1;
                        else if (d2 > bestd) { bestd = d2; memcpy(best, cand, sizeof best); }
                    }
                }
                if (placed) {
                    memcpy(gr.x + 3 * a, cand, sizeof cand);
                    grid_add(&gr, a);
                    ++k;
                    continue;
                }
                /* after many restarts accept the least-bad candidate, but
                 * never one closer than a hard floor (the discrete angles put
                 * a chain on a diamond lattice, so exact self-overlaps exist) */
                double hard2 = restarts < 200 ? 0.0625 : (restarts < 400 ? 0.0484 : (restarts < 1000 ? 0.04 : 0.0));
                if (restarts >= 40 && bestd > hard2) {
                    memcpy(gr.x + 3 * a, best, sizeof best);
                    grid_add(&gr, a);
                    ++relaxed; ++k;
                    continue;
                }
                /* backtrack a few sites */
                if (++backtracks > 60 || k == 0) { ok_chain = 0; break; }
                int back = 1 + (int)(cg_unif(&rng) * 4.0);
                if (back > k) back = k;
                for (int q = 0; q < back; ++q) { --k; grid_remove(&gr, base + k); }
            }
            if (ok_chain) break;
            for (int q = k - 1; q >= 0; --q) grid_remove(&gr, base + q);
            ++restarts;
            if (restarts % 10 == 0 && r2 > 0.0484) r2 *= 0.9;
        }
    }
    for (int64_t i = 0; i < 3 * N; ++i) pos[i] = wrap(gr.x[i], L);
    free(gr.head); free(gr.next); free(gr.chain); free(gr.idx); free(gr.x);
    return relaxed;
}

/*
 * Maxwell-Boltzmann velocities at temperature T (kelvin) in nm/ps for masses
 * in amu (kB in kJ/mol/K), then the centre-of-mass momentum is removed.
 */
void cg_maxwell(int64_t n, const double *mass, double T, double kB, uint64_t seed, double *vel) {
    cg_rng rng = { seed };
    double spare = 0.0; int has = 0;
    double P[3] = { 0, 0, 0 }, M = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = sqrt(kB * T / mass[i]);
        for (int a = 0; a < 3; ++a) {
            vel[3 * i + a] = s * cg_gauss(&rng, &spare, &has);
            P[a] += mass[i] * vel[3 * i + a];
        }
        M += mass[i];
    }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) vel[3 * i + a] -= P[a] / M;
}

/* uniform numbers for the replica recipe (chain counts, temperatures) */
void cg_uniforms(uint64_t seed, int64_t n, double *out) {
    cg_rng rng = { seed };
    for (int64_t i = 0; i < n; ++i) out[i] = cg_unif(&rng);
}
