/*
 * traphic_oracle.c -- plain, slow FP64 CPU oracle of one TRAPHIC step with transport of
 * ionizing recombination radiation (Raicevic et al., Sec. 2).  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the CPU-baseline leg of the benchmark are its only
 * callers.  It is written for a reader checking it against the paper: one sequential
 * loop per step of the method, in the paper's order, with no blocking or fusion.
 * Compile with -ffp-contract=off so that every floating-point operation is rounded as
 * written.
 *
 * Where the paper leaves a detail to the TRAPHIC papers it cites (Pawlik & Schaye 2008,
 * 2011), the reading taken is stated at the function that implements it.
 *
 * Parity unpinned (no printed number or closed form fixes them; checked only through
 * the physical limits): the normalisations of the collisional ionisation and collisional
 * excitation fits (their activation energies, the ionisation cooling's tie to the
 * ionisation energy, and the free-free normalisation and sqrt(T) scaling are pinned).  Where a virtual particle lands is checked statistically against the
 * uniform law of its reading; the rest of its step (its interpolated n_HI, projected length,
 * clock and the sharing of its absorptions) by invariants of a uniform medium and by brute
 * force of whole chains on tiny boxes.  The equal split among cone members and the
 * photon-weighted merge of arriving packets are readings the paper does not fix; a
 * brute-force computation of one hop on tiny boxes checks that this code does what they
 * say.  The chemistry update is checked by its convergence to a stiff integration of its
 * own rate equations.
 */
#include "traphic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 1048576LL /* 2^20 quantisation cells per box side */
#define MAXK 32

static const double K_B = 1.380649e-16;    /* erg/K */
static const double C_LIGHT = 2.99792458e10; /* cm/s */
static const double T_HI = 157807.0;       /* K, hydrogen ionisation temperature */

enum { PURPOSE_RECEPTION = 1, PURPOSE_EMISSION = 2, PURPOSE_VIRTUAL = 3, PURPOSE_REC_EMISSION = 4 };

/* ------------------------------------------------------------------------------ */
/* Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).    */
/* ------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_key(uint64_t seed, uint32_t purpose, uint32_t key[2]) {
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32) ^ purpose;
}

/* SplitMix64 output function (Steele, Lea & Flood 2014): identities of virtual
   particles descending from earlier virtual particles. */
uint64_t orc_mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------------ */
/* Isotropic direction sets for emission and reception cones (Sec. 2.1).  The      */
/* paper does not give the construction.  Reading: 8 cones = the cube diagonals;   */
/* 32 cones = icosahedron (12) + dodecahedron (20) vertices.                      */
/* ------------------------------------------------------------------------------ */
int orc_axis_set(int n, double *out) {
    if (n == 8) {
        double r = 1.0 / sqrt(3.0);
        for (int b = 0; b < 8; ++b) {
            out[3 * b + 0] = (b & 4) ? -r : r;
            out[3 * b + 1] = (b & 2) ? -r : r;
            out[3 * b + 2] = (b & 1) ? -r : r;
        }
        return 0;
    }
    if (n == 32) {
        double phi = (1.0 + sqrt(5.0)) / 2.0;
        double a = 1.0 / sqrt(1.0 + phi * phi);
        double r = 1.0 / sqrt(3.0);
        double iphi = 1.0 / phi;
        int v = 0;
        /* icosahedron: cyclic permutations of (0, +-1, +-phi) */
        for (int g = 0; g < 3; ++g)
            for (int i1 = 0; i1 < 2; ++i1)
                for (int i2 = 0; i2 < 2; ++i2) {
                    double s1 = i1 ? -1.0 : 1.0, s2 = i2 ? -1.0 : 1.0;
                    double e[3];
                    if (g == 0) { e[0] = 0.0; e[1] = s1 * a; e[2] = s2 * (phi * a); }
                    else if (g == 1) { e[0] = s1 * a; e[1] = s2 * (phi * a); e[2] = 0.0; }
                    else { e[0] = s2 * (phi * a); e[1] = 0.0; e[2] = s1 * a; }
                    out[3 * v + 0] = e[0]; out[3 * v + 1] = e[1]; out[3 * v + 2] = e[2];
                    ++v;
                }
        /* dodecahedron: the cube (+-1,+-1,+-1) ... */
        for (int b = 0; b < 8; ++b) {
            out[3 * v + 0] = (b & 4) ? -r : r;
            out[3 * v + 1] = (b & 2) ? -r : r;
            out[3 * v + 2] = (b & 1) ? -r : r;
            ++v;
        }
        /* ... and cyclic permutations of (0, +-1/phi, +-phi), all of norm sqrt(3) */
        for (int g = 0; g < 3; ++g)
            for (int i1 = 0; i1 < 2; ++i1)
                for (int i2 = 0; i2 < 2; ++i2) {
                    double s1 = i1 ? -1.0 : 1.0, s2 = i2 ? -1.0 : 1.0;
                    double e[3];
                    if (g == 0) { e[0] = 0.0; e[1] = s1 * (iphi * r); e[2] = s2 * (phi * r); }
                    else if (g == 1) { e[0] = s1 * (iphi * r); e[1] = s2 * (phi * r); e[2] = 0.0; }
                    else { e[0] = s2 * (phi * r); e[1] = 0.0; e[2] = s1 * (iphi * r); }
                    out[3 * v + 0] = e[0]; out[3 * v + 1] = e[1]; out[3 * v + 2] = e[2];
                    ++v;
                }
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------------ */
/* Random rotation before each emission and for the reception cones (Sec. 2.1:     */
/* directions "randomly rotated" before each emission; reception directions        */
/* "frequently rotated"; the cadence read as once per RT step).  A uniform unit    */
/* quaternion by rejection from the 4-cube, at most 16 draws, else the identity.    */
/* ------------------------------------------------------------------------------ */
void orc_rotation(uint64_t seed, uint32_t purpose, uint32_t c0, uint32_t c1, uint32_t c2,
                  double R[9]) {
    uint32_t key[2];
    philox_key(seed, purpose, key);
    double q0 = 1.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
    for (uint32_t attempt = 0; attempt < 16; ++attempt) {
        uint32_t ctr[4] = {c0, c1, c2, attempt}, u[4];
        orc_philox4x32_10(ctr, key, u);
        double v[4];
        for (int k = 0; k < 4; ++k) v[k] = (double)(u[k] >> 8) * (1.0 / 8388608.0) - 1.0;
        double s = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
        if (s > 1e-6 && s <= 1.0) {
            double n = sqrt(s);
            q0 = v[0] / n; q1 = v[1] / n; q2 = v[2] / n; q3 = v[3] / n;
            break;
        }
    }
    R[0] = 1.0 - 2.0 * (q2 * q2 + q3 * q3);
    R[1] = 2.0 * (q1 * q2 - q0 * q3);
    R[2] = 2.0 * (q1 * q3 + q0 * q2);
    R[3] = 2.0 * (q1 * q2 + q0 * q3);
    R[4] = 1.0 - 2.0 * (q1 * q1 + q3 * q3);
    R[5] = 2.0 * (q2 * q3 - q0 * q1);
    R[6] = 2.0 * (q1 * q3 - q0 * q2);
    R[7] = 2.0 * (q2 * q3 + q0 * q1);
    R[8] = 1.0 - 2.0 * (q1 * q1 + q2 * q2);
}

/* direction of axis D rotated by R: R * D */
static void rotate_axis(const double R[9], const double *D, double out[3]) {
    out[0] = R[0] * D[0] + R[1] * D[1] + R[2] * D[2];
    out[1] = R[3] * D[0] + R[4] * D[1] + R[5] * D[2];
    out[2] = R[6] * D[0] + R[7] * D[1] + R[8] * D[2];
}

/* Transmission cone (Sec. 2.1): the regular cone of solid angle 4 pi / N_TC about the
   propagation direction d, i.e. half-opening angle with cos = 1 - 2/N_TC.  A neighbour
   at integer offset delta is inside when delta . d > 0 and
   (delta . d)^2 >= cos^2 |delta|^2.  A coincident neighbour is never inside. */
int orc_in_cone(const int64_t delta[3], const double d[3], int n_tc) {
    if (delta[0] == 0 && delta[1] == 0 && delta[2] == 0) return 0;
    double t = (double)delta[0] * d[0] + (double)delta[1] * d[1] + (double)delta[2] * d[2];
    if (!(t > 0.0)) return 0;
    double r2 = (double)(delta[0] * delta[0] + delta[1] * delta[1] + delta[2] * delta[2]);
    double c = 1.0 - 2.0 / (double)n_tc;
    return t * t >= (c * c) * r2;
}

/* Reception cone of direction d at a particle with rotation R (Sec. 2.1, Fig. 1a):
   the bin whose rotated axis R*D_b is nearest to d, i.e. argmax_b (R^T d) . D_b, the
   first maximum winning ties. */
int orc_bin(const double R[9], const double *axes, int n_rc, const double d[3]) {
    double e0 = R[0] * d[0] + R[3] * d[1] + R[6] * d[2];
    double e1 = R[1] * d[0] + R[4] * d[1] + R[7] * d[2];
    double e2 = R[2] * d[0] + R[5] * d[1] + R[8] * d[2];
    int best = 0;
    double bs = 0.0;
    for (int b = 0; b < n_rc; ++b) {
        double sc = e0 * axes[3 * b] + e1 * axes[3 * b + 1] + e2 * axes[3 * b + 2];
        if (b == 0 || sc > bs) { bs = sc; best = b; }
    }
    return best;
}

/* ------------------------------------------------------------------------------ */
/* Rates (Sec. 2.1, penultimate paragraph).  Recombination coefficients, their     */
/* cooling and collisional ionisation: the fits of Hui & Gnedin (1997) with        */
/* lambda = 2 T_HI / T.  Collisional excitation cooling: Cen (1992).  Free-free:   */
/* 1.42e-27 g_ff sqrt(T) with g_ff = 1.3.  Compton cooling off the CMB is left out  */
/* (static, non-cosmological test fields).  The coefficients, their values at 1e4,  */
/* 2e4, 3e4 and 1e5 K and their sources are tabulated in docs/rates; the case-A and */
/* case-B coefficients are checked against Osterbrock & Ferland (2006, Table 2.1)   */
/* with the values in tests/golden/published_rates.txt.                            */
/* ------------------------------------------------------------------------------ */
void orc_rates(double T, double out[8]) {
    double lam = 2.0 * T_HI / T;
    double aA = 1.269e-13 * pow(lam, 1.503) / pow(1.0 + pow(lam / 0.522, 0.470), 1.923);
    double aB = 2.753e-14 * pow(lam, 1.500) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
    double beta = 21.11 * pow(T, -1.5) * exp(-lam / 2.0) * pow(lam, -1.089) /
                  pow(1.0 + pow(lam / 0.354, 0.874), 1.101);
    double LA = 1.778e-29 * T * pow(lam, 1.965) / pow(1.0 + pow(lam / 0.541, 0.502), 2.697);
    double LB = 3.435e-30 * T * pow(lam, 1.970) / pow(1.0 + pow(lam / 2.250, 0.376), 3.720);
    double Lce = 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1e5));
    double Lci = K_B * T_HI * beta;
    double Lff = 1.42e-27 * 1.3 * sqrt(T);
    out[0] = aA; out[1] = aB; out[2] = beta; out[3] = LA;
    out[4] = LB; out[5] = Lce; out[6] = Lci; out[7] = Lff;
}

/* ------------------------------------------------------------------------------ */
/* Chemistry of one particle over dt (Sec. 2.1 "Once the transport step has        */
/* completed ..."; Sec. 2.2).  Photoionisation rate per neutral atom               */
/* Gamma = N_abs / (N_HI dt), photoheating per neutral atom H = E_abs / (N_HI dt),   */
/* both with N_HI at the start of the step.  The solver itself lives in Pawlik &   */
/* Schaye (2011); reading: subcycles with the electron density frozen inside each,  */
/* the exact exponential solution for x_HI within a subcycle,                      */
/*   dx/dt = alpha n_e (1 - x) - (Gamma + beta n_e) x,                             */
/* explicit Euler for the energy density u = 1.5 k T n_H (1 + x_HII) with a          */
/* subcycle no longer than 0.1 u/|du/dt| (floor dt/sub_cap).  Case B coefficients   */
/* with on-the-spot, case A with case-A cooling otherwise; with transport of        */
/* recombination radiation the ground-level recombinations, at rate                 */
/* alpha_1 = alpha_A - alpha_B, are the photons to emit (Sec. 2.2).                 */
/* ------------------------------------------------------------------------------ */
void orc_chem_particle(const orc_config *cfg, double nH, double NH, double phot,
                       double heat, double *x_io, double *T_io, double out[3]) {
    double dt = cfg->dt;
    double x = *x_io, T = *T_io;
    double NHI = x * NH;
    double Gam = 0.0, Hh = 0.0;
    if (NHI > 0.0) {
        Gam = phot / (NHI * dt);
        Hh = heat / (NHI * dt);
    }
    double dtmin = dt / (double)cfg->sub_cap;
    double t = 0.0, Nrec = 0.0;
    long long nsub = 0, nfloor = 0;
    int last = 0;
    while (!last) {
        double r[8];
        orc_rates(T, r);
        double alpha = (cfg->rec_mode == ORC_REC_OTS_CASE_B) ? r[1] : r[0];
        double ne = (1.0 - x) * nH;
        double lamx = Gam + r[2] * ne + alpha * ne;
        double h = dt - t;
        double u = 0.0, dudt = 0.0;
        if (cfg->evolve_T) {
            double xII = 1.0 - x;
            u = 1.5 * K_B * T * nH * (1.0 + xII);
            double Lrec = (cfg->rec_mode == ORC_REC_OTS_CASE_B) ? r[4] : r[3];
            double cool = 0.0;
            if (cfg->cool_flags & ORC_COOL_REC) cool += ne * (xII * nH) * Lrec;
            if (cfg->cool_flags & ORC_COOL_CEX) cool += ne * (x * nH) * r[5];
            if (cfg->cool_flags & ORC_COOL_CION) cool += ne * (x * nH) * r[6];
            if (cfg->cool_flags & ORC_COOL_FF) cool += ne * (xII * nH) * r[7];
            dudt = x * nH * Hh - cool;
            if (dudt != 0.0) {
                double ht = 0.1 * u / fabs(dudt);
                if (ht < h) h = ht;
            }
            /* the floor binds only when the 10% limit, not the time left in the step, made
               the subcycle shorter than dt/sub_cap: the subcycle taken then changes u by more
               than 10% */
            if (h < dtmin) {
                if (h < dt - t) ++nfloor;
                h = dtmin;
            }
        }
        if (h >= dt - t) { h = dt - t; last = 1; }
        double xn, intII;
        if (lamx > 0.0) {
            double xeq = alpha * ne / lamx;
            double e = exp(-lamx * h);
            xn = xeq + (x - xeq) * e;
            intII = (1.0 - xeq) * h - (x - xeq) * (1.0 - e) / lamx; /* integral of 1-x */
        } else {
            xn = x;
            intII = (1.0 - x) * h;
        }
        if (cfg->rec_mode == ORC_REC_TRANSPORT || cfg->rec_mode == ORC_REC_EMISSION_CONES)
            Nrec += (r[0] - r[1]) * ne * NH * intII;
        if (cfg->evolve_T) {
            double un = u + h * dudt;
            T = un / (1.5 * K_B * nH * (1.0 + (1.0 - xn)));
            if (!(T >= cfg->T_floor)) T = cfg->T_floor;
        }
        x = xn;
        t += h;
        ++nsub;
    }
    *x_io = x;
    *T_io = T;
    out[0] = Nrec;
    out[1] = (double)nsub;
    out[2] = (double)nfloor;
}

/* ------------------------------------------------------------------------------ */
/* Exact k nearest neighbours (Sec. 2.1: a packet searches the neighbours within   */
/* the smoothing volume of the particle it is attached to; the smoothing volume    */
/* holds the N_ngb nearest particles).  Order: squared integer distance, then      */
/* index.  Brute force, or a uniform grid searched in growing shells of cells       */
/* until no unsearched cell can hold a closer point.                               */
/* ------------------------------------------------------------------------------ */
typedef struct {
    int G;            /* cells per side */
    int64_t cs;       /* cell side in quantised units */
    long long *start; /* [G^3 + 1] */
    long long *items; /* point indices, grouped by cell */
} grid_t;

static int cell_of(int64_t v, const grid_t *g) {
    int64_t c = v / g->cs;
    if (c < 0) c = 0;
    if (c >= g->G) c = g->G - 1;
    return (int)c;
}

static void grid_build(grid_t *g, long long n, const int64_t *pts) {
    int G = (int)cbrt((double)n / 2.0);
    if (G < 1) G = 1;
    if (G > 256) G = 256;
    g->G = G;
    g->cs = (ORC_Q + G - 1) / G;
    long long nc = (long long)G * G * G;
    g->start = (long long *)calloc((size_t)nc + 1, sizeof(long long));
    g->items = (long long *)malloc(sizeof(long long) * (size_t)(n > 0 ? n : 1));
    long long *fill = (long long *)calloc((size_t)nc, sizeof(long long));
    for (long long i = 0; i < n; ++i) {
        long long c = ((long long)cell_of(pts[3 * i], g) * G + cell_of(pts[3 * i + 1], g)) * G +
                      cell_of(pts[3 * i + 2], g);
        g->start[c + 1]++;
    }
    for (long long c = 0; c < nc; ++c) g->start[c + 1] += g->start[c];
    for (long long i = 0; i < n; ++i) {
        long long c = ((long long)cell_of(pts[3 * i], g) * G + cell_of(pts[3 * i + 1], g)) * G +
                      cell_of(pts[3 * i + 2], g);
        g->items[g->start[c] + fill[c]++] = i;
    }
    free(fill);
}

static void grid_free(grid_t *g) {
    free(g->start);
    free(g->items);
    g->start = NULL;
    g->items = NULL;
}

typedef struct {
    int k, m;
    int64_t d2[MAXK];
    long long idx[MAXK];
} topk_t;

static int key_less(int64_t da, long long ia, int64_t db, long long ib) {
    return da < db || (da == db && ia < ib);
}

static void topk_insert(topk_t *t, int64_t d2, long long idx) {
    if (t->m == t->k && !key_less(d2, idx, t->d2[t->k - 1], t->idx[t->k - 1])) return;
    int p = (t->m < t->k) ? t->m++ : t->k - 1;
    while (p > 0 && key_less(d2, idx, t->d2[p - 1], t->idx[p - 1])) {
        t->d2[p] = t->d2[p - 1];
        t->idx[p] = t->idx[p - 1];
        --p;
    }
    t->d2[p] = d2;
    t->idx[p] = idx;
}

static int64_t dist2(const int64_t *a, const int64_t *b) {
    int64_t dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* exclude: index to skip (the query particle itself) or -1 */
static void knn_brute(long long n, const int64_t *pts, const int64_t *q, long long exclude,
                      topk_t *t) {
    for (long long j = 0; j < n; ++j)
        if (j != exclude) topk_insert(t, dist2(q, pts + 3 * j), j);
}

static void knn_grid(const grid_t *g, const int64_t *pts, const int64_t *q, long long exclude,
                     topk_t *t) {
    int G = g->G;
    int c0[3];
    for (int a = 0; a < 3; ++a) c0[a] = cell_of(q[a], g);
    for (int r = 0; r <= G; ++r) {
        for (int dx = -r; dx <= r; ++dx)
            for (int dy = -r; dy <= r; ++dy)
                for (int dz = -r; dz <= r; ++dz) {
                    int ax = abs(dx), ay = abs(dy), az = abs(dz);
                    int m = ax > ay ? ax : ay;
                    if (az > m) m = az;
                    if (m != r) continue;
                    int cx = c0[0] + dx, cy = c0[1] + dy, cz = c0[2] + dz;
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= G || cy >= G || cz >= G) continue;
                    long long c = ((long long)cx * G + cy) * G + cz;
                    for (long long p = g->start[c]; p < g->start[c + 1]; ++p) {
                        long long j = g->items[p];
                        if (j != exclude) topk_insert(t, dist2(q, pts + 3 * j), j);
                    }
                }
        /* distance from q to the outside of the searched block of cells */
        int64_t b = -1;
        for (int a = 0; a < 3; ++a) {
            if (c0[a] - r > 0) {
                int64_t lo = q[a] - (int64_t)(c0[a] - r) * g->cs;
                if (b < 0 || lo < b) b = lo;
            }
            if (c0[a] + r + 1 < G) {
                int64_t hi = (int64_t)(c0[a] + r + 1) * g->cs - q[a];
                if (b < 0 || hi < b) b = hi;
            }
        }
        if (b < 0) break; /* the whole grid was searched */
        if (t->m == t->k && t->d2[t->k - 1] < b * b) break;
    }
}

int orc_knn(long long n_pts, const int64_t *pts, long long n_q, const int64_t *qpts,
            long long self_offset, int k, int use_grid, int32_t *out_idx, int64_t *out_d2) {
    if (k < 1 || k > MAXK) return ORC_ERR_INVALID;
    grid_t g = {0};
    if (use_grid) grid_build(&g, n_pts, pts);
    for (long long i = 0; i < n_q; ++i) {
        topk_t t;
        t.k = k;
        t.m = 0;
        long long ex = self_offset >= 0 ? self_offset + i : -1;
        if (use_grid) knn_grid(&g, pts, qpts + 3 * i, ex, &t);
        else knn_brute(n_pts, pts, qpts + 3 * i, ex, &t);
        for (int m = 0; m < k; ++m) {
            out_idx[i * k + m] = m < t.m ? (int32_t)t.idx[m] : -1;
            out_d2[i * k + m] = m < t.m ? t.d2[m] : -1;
        }
    }
    if (use_grid) grid_free(&g);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* Simulation state                                                                */
/* ------------------------------------------------------------------------------ */
typedef struct {
    int box;
    int64_t q[3];
    int32_t nbr[MAXK]; /* global gas indices */
    int64_t h2;
    double N, d[3], clock, eps;
    double sig;        /* cross-section of its photons, cm^2 */
    int nu;
    uint64_t fid;
} freep_t; /* a packet not held by a gas particle: a source packet or a virtual particle */

typedef struct {
    freep_t *p;
    long long n, cap;
} freelist_t;

static void fl_push(freelist_t *l, const freep_t *p) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 1024;
        l->p = (freep_t *)realloc(l->p, sizeof(freep_t) * (size_t)l->cap);
    }
    l->p[l->n++] = *p;
}

/* An artificial photon barrier (Sec. 4): a disk perpendicular to a coordinate axis that
   removes every packet whose path crosses it.  In doubled quantised units: the plane sits at
   the odd coordinate p2 along `axis` (no particle lies on it), the centre at (c1, c2) in the
   other two axes (cyclic order), the radius is r2. */
typedef struct {
    int axis;
    int64_t p2, c1, c2, r2;
} barrier_t;

struct orc_sim {
    orc_config cfg;
    int nb;
    long long *box_off;
    double *box_L;
    long long n;
    int nf, S, K;
    int64_t *q;
    int *box;
    double *nH, *NH, *xHI, *T;
    int ns;
    int *sbox;
    /* identities in the random streams: particle i of box b draws as particle
       gid0[b] + (i - box_off[b]) and source j as source sid[j] (by default their own indices),
       so that the boxes of a larger workload, run apart, repeat their draws */
    long long *gid0;
    long long *sid;
    int64_t *sq;
    double *ndot, *sigma, *eps;
    double *sdir;  /* [ns*3] fixed emission direction of a directed source, 0: isotropic */
    int *sgate;    /* [ns] 1: emits only while its nearest gas particle has x_HI < 0.5 */
    barrier_t *bar; /* [nb] photon barrier of each box (axis < 0: none) */
    int32_t *nbr, *snbr;
    int64_t *h2, *sh2;
    grid_t *grids;
    double *R, *Rs;
    double axes_rc[3 * 32], axes_ec[3 * 32];
    double *sl[6], *nx[6];
    /* shared frequency bin (Sec. 2.2, last paragraph): recombination photons travel in source
       bin 0 (rbin = 0), and each slot of that bin carries G = sum N sigma of the photons merged
       into it ([n*n_rc], current and next hop); without it rbin is the extra last bin */
    int rbin;
    double *sg, *nsg;
    double *abs_, *absE, *pass, *nHI, *Nrec, *epsrec;
    double *tally; /* [nb*4] running sums (Neumaier compensated with tallc) */
    double *tallc;
    freelist_t cur, nxt;
    long long st_hops, st_virtual, st_escaped_v, st_sub, st_sends, st_floor;
    int built;
};

/* Neumaier's compensated sum: photon tallies add ~10^7 terms per step and must close
   to 1e-12 relative */
static void kadd(double *sum, double *comp, double v) {
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
    else *comp += (v - t) + *sum;
    *sum = t;
}

static void tally_add(orc_sim *s, int box, int f, double v) {
    kadd(&s->tally[4 * box + f], &s->tallc[4 * box + f], v);
}

static int64_t quantise(double x, double L) {
    double f = x / L;
    f = f * (double)ORC_Q;
    double fl = floor(f);
    int64_t q = (int64_t)fl;
    if (!(fl >= 0.0)) q = 0;
    if (q > ORC_Q - 1) q = ORC_Q - 1;
    return q;
}

/* identity of particle i in the random streams */
static uint64_t gid(const orc_sim *s, long long i) {
    int b = s->box[i];
    return (uint64_t)(s->gid0[b] + (i - s->box_off[b]));
}

orc_sim *orc_create(const orc_config *cfg, int n_boxes, const long long *box_off,
                    const double *box_L, const double *x, const double *y, const double *z,
                    const double *n_H, const double *N_H, const double *x_HI,
                    const double *T, int n_src, const int *src_box, const double *sx,
                    const double *sy, const double *sz, const double *ndot,
                    const double *sigma, const double *eps) {
    if (cfg->n_ngb < 1 || cfg->n_ngb > MAXK || cfg->n_tc < 2 || cfg->n_freq_src < 0)
        return NULL;
    if ((cfg->n_rc != 8 && cfg->n_rc != 32) || (cfg->n_ec != 8 && cfg->n_ec != 32))
        return NULL;
    if (cfg->rec_shared_bin && cfg->n_freq_src < 1) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->cfg = *cfg;
    s->nb = n_boxes;
    s->n = box_off[n_boxes];
    s->nf = cfg->n_freq_src + (cfg->rec_shared_bin ? 0 : 1);
    s->rbin = cfg->rec_shared_bin ? 0 : cfg->n_freq_src;
    s->S = s->nf * cfg->n_rc;
    long long K = (long long)llround(cfg->dt / cfg->dt_em);
    s->K = K < 1 ? 1 : (int)K;
    long long n = s->n;
    s->box_off = (long long *)malloc(sizeof(long long) * (size_t)(n_boxes + 1));
    memcpy(s->box_off, box_off, sizeof(long long) * (size_t)(n_boxes + 1));
    s->box_L = (double *)malloc(sizeof(double) * (size_t)n_boxes);
    memcpy(s->box_L, box_L, sizeof(double) * (size_t)n_boxes);
    s->q = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)n);
    s->box = (int *)malloc(sizeof(int) * (size_t)n);
    s->nH = (double *)malloc(sizeof(double) * (size_t)n);
    s->NH = (double *)malloc(sizeof(double) * (size_t)n);
    s->xHI = (double *)malloc(sizeof(double) * (size_t)n);
    s->T = (double *)malloc(sizeof(double) * (size_t)n);
    for (int b = 0; b < n_boxes; ++b)
        for (long long i = box_off[b]; i < box_off[b + 1]; ++i) {
            s->box[i] = b;
            s->q[3 * i + 0] = quantise(x[i], box_L[b]);
            s->q[3 * i + 1] = quantise(y[i], box_L[b]);
            s->q[3 * i + 2] = quantise(z[i], box_L[b]);
        }
    memcpy(s->nH, n_H, sizeof(double) * (size_t)n);
    memcpy(s->NH, N_H, sizeof(double) * (size_t)n);
    memcpy(s->xHI, x_HI, sizeof(double) * (size_t)n);
    memcpy(s->T, T, sizeof(double) * (size_t)n);
    s->ns = n_src;
    int nfs = cfg->n_freq_src;
    s->sbox = (int *)malloc(sizeof(int) * (size_t)(n_src + 1));
    s->sq = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(n_src + 1));
    s->ndot = (double *)malloc(sizeof(double) * (size_t)(n_src * nfs + 1));
    for (int i = 0; i < n_src; ++i) {
        s->sbox[i] = src_box[i];
        double L = box_L[src_box[i]];
        s->sq[3 * i + 0] = quantise(sx[i], L);
        s->sq[3 * i + 1] = quantise(sy[i], L);
        s->sq[3 * i + 2] = quantise(sz[i], L);
        for (int f = 0; f < nfs; ++f) s->ndot[i * nfs + f] = ndot[i * nfs + f];
    }
    s->gid0 = (long long *)malloc(sizeof(long long) * (size_t)n_boxes);
    for (int b = 0; b < n_boxes; ++b) s->gid0[b] = box_off[b];
    s->sid = (long long *)malloc(sizeof(long long) * (size_t)(n_src + 1));
    for (int j = 0; j < n_src; ++j) s->sid[j] = j;
    s->sdir = (double *)calloc((size_t)(3 * n_src + 3), sizeof(double));
    s->sgate = (int *)calloc((size_t)(n_src + 1), sizeof(int));
    s->bar = (barrier_t *)calloc((size_t)n_boxes, sizeof(barrier_t));
    for (int b = 0; b < n_boxes; ++b) s->bar[b].axis = -1;
    s->sigma = (double *)malloc(sizeof(double) * (size_t)(nfs + 1));
    s->eps = (double *)malloc(sizeof(double) * (size_t)(nfs + 1));
    for (int f = 0; f < nfs; ++f) {
        s->sigma[f] = sigma[f];
        s->eps[f] = eps[f];
    }
    s->sigma[nfs] = cfg->sigma_rec;   /* the recombination bin (unused with a shared bin) */
    s->eps[nfs] = 0.0;
    orc_axis_set(cfg->n_rc, s->axes_rc);
    orc_axis_set(cfg->n_ec, s->axes_ec);
    int k = cfg->n_ngb;
    s->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * k));
    s->h2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    s->snbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)((n_src + 1) * k));
    s->sh2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_src + 1));
    s->grids = (grid_t *)calloc((size_t)n_boxes, sizeof(grid_t));
    s->R = (double *)calloc((size_t)(9 * n), sizeof(double));
    s->Rs = (double *)calloc((size_t)(9 * (n_src * s->K + 1)), sizeof(double));
    for (int f = 0; f < 6; ++f) {
        s->sl[f] = (double *)calloc((size_t)(n * s->S), sizeof(double));
        s->nx[f] = (double *)calloc((size_t)(n * s->S), sizeof(double));
    }
    if (cfg->rec_shared_bin) {
        s->sg = (double *)calloc((size_t)(n * cfg->n_rc), sizeof(double));
        s->nsg = (double *)calloc((size_t)(n * cfg->n_rc), sizeof(double));
    }
    s->abs_ = (double *)calloc((size_t)(n * s->nf), sizeof(double));
    s->pass = (double *)calloc((size_t)(n * s->nf), sizeof(double));
    s->absE = (double *)calloc((size_t)n, sizeof(double));
    s->nHI = (double *)calloc((size_t)n, sizeof(double));
    s->Nrec = (double *)calloc((size_t)n, sizeof(double));
    s->epsrec = (double *)calloc((size_t)n, sizeof(double));
    s->tally = (double *)calloc((size_t)(4 * n_boxes), sizeof(double));
    s->tallc = (double *)calloc((size_t)(4 * n_boxes), sizeof(double));
    /* identity rotations until orc_rotate is called */
    for (long long i = 0; i < n; ++i) s->R[9 * i] = s->R[9 * i + 4] = s->R[9 * i + 8] = 1.0;
    return s;
}

int orc_set_identities(orc_sim *s, const long long *box_first_id, const long long *src_id) {
    for (int b = 0; b < s->nb; ++b) s->gid0[b] = box_first_id ? box_first_id[b] : s->box_off[b];
    for (int j = 0; j < s->ns; ++j) s->sid[j] = src_id ? src_id[j] : j;
    return ORC_OK;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->box_off); free(s->box_L); free(s->q); free(s->box); free(s->nH); free(s->NH);
    free(s->xHI); free(s->T); free(s->sbox); free(s->sq); free(s->ndot); free(s->sigma);
    free(s->sdir); free(s->sgate); free(s->bar); free(s->gid0); free(s->sid);
    free(s->eps); free(s->nbr); free(s->h2); free(s->snbr); free(s->sh2);
    for (int b = 0; b < s->nb; ++b) grid_free(&s->grids[b]);
    free(s->grids); free(s->R); free(s->Rs);
    for (int f = 0; f < 6; ++f) { free(s->sl[f]); free(s->nx[f]); }
    free(s->sg); free(s->nsg);
    free(s->abs_); free(s->pass); free(s->absE); free(s->nHI); free(s->Nrec);
    free(s->epsrec); free(s->tally); free(s->tallc); free(s->cur.p); free(s->nxt.p);
    free(s);
}

void orc_set_source_options(orc_sim *s, const double *dir, const int *gate) {
    for (int j = 0; j < s->ns; ++j) {
        for (int a = 0; a < 3; ++a) s->sdir[3 * j + a] = dir ? dir[3 * j + a] : 0.0;
        s->sgate[j] = gate ? gate[j] : 0;
    }
}

void orc_set_barrier(orc_sim *s, int box, int axis, const double centre[3], double radius) {
    barrier_t *B = &s->bar[box];
    if (!(radius > 0.0) || axis < 0 || axis > 2) {
        B->axis = -1;
        return;
    }
    double L = s->box_L[box];
    B->axis = axis;
    B->p2 = 2 * quantise(centre[axis], L) + 1;
    B->c1 = 2 * quantise(centre[(axis + 1) % 3], L);
    B->c2 = 2 * quantise(centre[(axis + 2) % 3], L);
    B->r2 = (int64_t)llround(2.0 * radius / L * (double)ORC_Q);
}

/* Does the straight path from a to b (quantised) cross the box's barrier disk?  Exact
   integer test: the plane separates a and b, and the crossing point (a rational point) lies
   within the radius; 128-bit products keep every term exact. */
static int barrier_crosses(const barrier_t *B, const int64_t *a, const int64_t *b) {
    if (B->axis < 0) return 0;
    int ax = B->axis, i1 = (ax + 1) % 3, i2 = (ax + 2) % 3;
    int64_t sa = 2 * a[ax] - B->p2, sb = 2 * b[ax] - B->p2;   /* odd: never 0 */
    if ((sa < 0) == (sb < 0)) return 0;
    int64_t D = sa - sb;
    __int128 y = (__int128)(2 * a[i1] - B->c1) * D + (__int128)sa * (2 * (b[i1] - a[i1]));
    __int128 z = (__int128)(2 * a[i2] - B->c2) * D + (__int128)sa * (2 * (b[i2] - a[i2]));
    __int128 rD = (__int128)B->r2 * D;
    return (unsigned __int128)(y * y) + (unsigned __int128)(z * z) <=
           (unsigned __int128)(rD * rD);
}

int orc_barrier_test(const int64_t a[3], const int64_t b[3], int axis, int64_t p2, int64_t c1,
                     int64_t c2, int64_t r2) {
    barrier_t B = {axis, p2, c1, c2, r2};
    return barrier_crosses(&B, a, b);
}

/* k nearest gas particles of point q in box b; returns global indices */
static int box_knn(const orc_sim *s, int b, const int64_t *q, long long exclude_global,
                   int32_t *nbr, int64_t *d2) {
    long long o = s->box_off[b], nb = s->box_off[b + 1] - o;
    topk_t t;
    t.k = s->cfg.n_ngb;
    t.m = 0;
    long long ex = exclude_global >= 0 ? exclude_global - o : -1;
    knn_grid(&s->grids[b], s->q + 3 * o, q, ex, &t);
    (void)nb;
    if (t.m < t.k) return ORC_ERR_INVALID;
    for (int m = 0; m < t.k; ++m) {
        nbr[m] = (int32_t)(t.idx[m] + o);
        if (d2) d2[m] = t.d2[m];
    }
    return ORC_OK;
}

int orc_build_neighbours(orc_sim *s) {
    int k = s->cfg.n_ngb;
    for (int b = 0; b < s->nb; ++b) {
        long long o = s->box_off[b], nb = s->box_off[b + 1] - o;
        if (nb < k + 1) return ORC_ERR_INVALID;
        grid_free(&s->grids[b]);
        grid_build(&s->grids[b], nb, s->q + 3 * o);
    }
    int64_t d2[MAXK];
    for (long long i = 0; i < s->n; ++i) {
        if (box_knn(s, s->box[i], s->q + 3 * i, i, s->nbr + i * k, d2)) return ORC_ERR_INVALID;
        s->h2[i] = d2[k - 1];
    }
    for (int i = 0; i < s->ns; ++i) {
        if (box_knn(s, s->sbox[i], s->sq + 3 * i, -1, s->snbr + i * k, d2)) return ORC_ERR_INVALID;
        s->sh2[i] = d2[k - 1];
    }
    s->built = 1;
    return ORC_OK;
}

void orc_get_neighbours(const orc_sim *s, int32_t *nbr, int64_t *h2, int32_t *src_nbr,
                        int64_t *src_h2) {
    int k = s->cfg.n_ngb;
    if (nbr) memcpy(nbr, s->nbr, sizeof(int32_t) * (size_t)(s->n * k));
    if (h2) memcpy(h2, s->h2, sizeof(int64_t) * (size_t)s->n);
    if (src_nbr) memcpy(src_nbr, s->snbr, sizeof(int32_t) * (size_t)(s->ns * k));
    if (src_h2) memcpy(src_h2, s->sh2, sizeof(int64_t) * (size_t)s->ns);
}

void orc_get_quantised(const orc_sim *s, int64_t *q) {
    memcpy(q, s->q, sizeof(int64_t) * 3 * (size_t)s->n);
}

/* Rotations of step `step`: reception cones of every gas particle and the emission
   cones of every source for each of its K emission sub-steps. */
void orc_rotate(orc_sim *s, long long step) {
    for (long long i = 0; i < s->n; ++i)
        orc_rotation(s->cfg.seed, PURPOSE_RECEPTION, (uint32_t)step, (uint32_t)(step >> 32),
                     (uint32_t)gid(s, i), s->R + 9 * i);
    for (int j = 0; j < s->ns; ++j)
        for (int k = 0; k < s->K; ++k)
            orc_rotation(s->cfg.seed, PURPOSE_EMISSION, (uint32_t)step, (uint32_t)k,
                         (uint32_t)s->sid[j], s->Rs + 9 * ((long long)j * s->K + k));
}

void orc_get_rotations(const orc_sim *s, double *R, double *Rs) {
    if (R) memcpy(R, s->R, sizeof(double) * 9 * (size_t)s->n);
    if (Rs) memcpy(Rs, s->Rs, sizeof(double) * 9 * (size_t)(s->ns * s->K));
}

/* unit direction of a packet from its summed momentum M (luminosity-weighted mean
   direction of the merged packets, Sec. 2.1 and Fig. 1b) */
static void packet_dir(const double M[3], double d[3]) {
    double n = sqrt(M[0] * M[0] + M[1] * M[1] + M[2] * M[2]);
    if (n > 0.0) {
        d[0] = M[0] / n; d[1] = M[1] / n; d[2] = M[2] / n;
    } else {
        d[0] = 1.0; d[1] = 0.0; d[2] = 0.0;
    }
}

static int slot_active(const orc_sim *s, long long i, int sl, double *clock) {
    long long p = i * s->S + sl;
    double N = s->sl[0][p];
    if (!(N > 0.0)) return 0;
    double c = s->sl[4][p] / N;
    if (clock) *clock = c;
    return c < s->cfg.dt;
}

/* Start of an RT step: clocks restart at the beginning of the step (Sec. 2.1: the
   clock is initialised with the time at the beginning of the current RT step) and the
   packets held by each particle are re-sorted into its freshly rotated reception
   cones, merging those that share a cone (Sec. 2.1, Fig. 1a,b). */
void orc_rebin(orc_sim *s) {
    int S = s->S, nrc = s->cfg.n_rc;
    double *tmp = (double *)malloc(sizeof(double) * 6 * (size_t)S);
    double gold[32];
    for (long long i = 0; i < s->n; ++i) {
        for (int f = 0; f < 6; ++f)
            for (int sl = 0; sl < S; ++sl) {
                tmp[f * S + sl] = s->sl[f][i * S + sl];
                s->sl[f][i * S + sl] = 0.0;
            }
        if (s->sg)
            for (int b = 0; b < nrc; ++b) {
                gold[b] = s->sg[i * nrc + b];
                s->sg[i * nrc + b] = 0.0;
            }
        for (int sl = 0; sl < S; ++sl) {
            double N = tmp[sl];
            if (!(N > 0.0)) continue;
            int nu = sl / nrc;
            double M[3] = {tmp[S + sl], tmp[2 * S + sl], tmp[3 * S + sl]}, d[3];
            packet_dir(M, d);
            int b = orc_bin(s->R + 9 * i, s->axes_rc, nrc, d);
            long long p = i * S + nu * nrc + b;
            s->sl[0][p] += N;
            s->sl[1][p] += M[0];
            s->sl[2][p] += M[1];
            s->sl[3][p] += M[2];
            s->sl[4][p] += 0.0;
            s->sl[5][p] += tmp[5 * S + sl];
            if (s->sg && nu == 0) s->sg[i * nrc + b] += gold[sl];
        }
    }
    free(tmp);
}

/* Emission at the start of an RT step.
   (1) Recombination radiation of the last chemistry step (Sec. 2.2, Fig. 1c,d): each
       particle adds N_rec/N_RC photons to every reception cone of the recombination
       frequency bin, along the cone's rotated axis, merging instantly with the packets
       already there; each carries excess energy eps_rr (kT of the emitting gas).
   (2) Source packets (Sec. 2.1): K = dt/dt_em emissions of N_EC packets per source
       frequency bin, N = Ndot_nu dt_em / N_EC photons each, along the randomly rotated
       emission axes; their clocks start at the beginning of the step. They leave the
       source in the first hop.
   Absorption and pass counters restart, and the neutral density seen by the transport
   is frozen at its value at the start of the step (operator split, Sec. 2.1).
   With rec_mode ORC_REC_EMISSION_CONES, (1) is replaced by (3) below.
   With a shared bin (Sec. 2.2, last paragraph) the recombination photons go into source bin
   0 instead of a bin of their own, and add N sigma_rec to the slot's cross-section sum. */
void orc_emit(orc_sim *s, long long step) {
    int S = s->S, nrc = s->cfg.n_rc, nfs = s->cfg.n_freq_src;
    for (long long i = 0; i < s->n * s->nf; ++i) { s->abs_[i] = 0.0; s->pass[i] = 0.0; }
    for (long long i = 0; i < s->n; ++i) {
        s->absE[i] = 0.0;
        s->nHI[i] = s->xHI[i] * s->nH[i];
    }
    for (long long i = 0; i < s->n && s->cfg.rec_mode != ORC_REC_EMISSION_CONES; ++i) {
        double Nr = s->Nrec[i];
        if (!(Nr > 0.0)) continue;
        double e = Nr / (double)nrc;
        for (int b = 0; b < nrc; ++b) {
            double A[3];
            rotate_axis(s->R + 9 * i, s->axes_rc + 3 * b, A);
            long long p = i * S + s->rbin * nrc + b;
            s->sl[0][p] += e;
            s->sl[1][p] += e * A[0];
            s->sl[2][p] += e * A[1];
            s->sl[3][p] += e * A[2];
            s->sl[5][p] += e * s->epsrec[i];
            if (s->sg) s->sg[i * nrc + b] += e * s->cfg.sigma_rec;
            tally_add(s, s->box[i], 0, e);
        }
    }
    s->cur.n = 0;
    int kn = s->cfg.n_ngb, nec = s->cfg.n_ec;
    for (int j = 0; j < s->ns; ++j) {
        /* a gated source (the boundary emitters of Sec. 4 and App. B) emits only once the
           I-front has passed it: its nearest gas particle is more than half ionised */
        if (s->sgate[j] && !(s->xHI[s->snbr[(long long)j * kn]] < 0.5)) continue;
        const double *dir = s->sdir + 3 * j;
        int directed = dir[0] != 0.0 || dir[1] != 0.0 || dir[2] != 0.0;
        for (int k = 0; k < s->K; ++k)
            for (int nu = 0; nu < nfs; ++nu)
                for (int e = 0; e < nec; ++e) {
                    /* a directed source (a packet of the plane-parallel front of Sec. 4) sends
                       one packet per emission and frequency along its direction */
                    if (directed && e > 0) continue;
                    uint64_t idx = (((uint64_t)s->sid[j] * s->K + k) * nfs + nu) * nec + e;
                    freep_t p;
                    memset(&p, 0, sizeof(p));
                    p.box = s->sbox[j];
                    p.q[0] = s->sq[3 * j]; p.q[1] = s->sq[3 * j + 1]; p.q[2] = s->sq[3 * j + 2];
                    memcpy(p.nbr, s->snbr + (long long)j * kn, sizeof(int32_t) * (size_t)kn);
                    p.h2 = s->sh2[j];
                    if (directed) {
                        p.N = s->ndot[j * nfs + nu] * s->cfg.dt_em;
                        p.d[0] = dir[0]; p.d[1] = dir[1]; p.d[2] = dir[2];
                    } else {
                        p.N = s->ndot[j * nfs + nu] * s->cfg.dt_em / (double)nec;
                        rotate_axis(s->Rs + 9 * ((long long)j * s->K + k), s->axes_ec + 3 * e,
                                    p.d);
                    }
                    p.clock = 0.0;
                    p.eps = s->eps[nu];
                    p.sig = s->sigma[nu];
                    p.nu = nu;
                    p.fid = (1ull << 62) | idx;
                    tally_add(s, p.box, 0, p.N);
                    fl_push(&s->cur, &p);
                }
    }
    /* (3) The original implementation of recombination radiation (Sec. 2.2): every particle
       with recombination photons is a source with its own N_EC emission cones, rotated at
       random before each of the K emissions of the step, like a star; its packets carry
       N_rec / (K N_EC) photons each, stay separate from the packets the particle holds, and
       leave it in the first hop through its own neighbours.  Packet identities follow
       (particle, emission, cone) whether or not a particle emits. */
    if (s->cfg.rec_mode == ORC_REC_EMISSION_CONES) {
        int nrb = s->rbin;                         /* the recombination frequency bin */
        for (long long i = 0; i < s->n; ++i) {
            double Nr = s->Nrec[i];
            if (!(Nr > 0.0)) continue;
            for (int k = 0; k < s->K; ++k) {
                double R[9];
                orc_rotation(s->cfg.seed, PURPOSE_REC_EMISSION, (uint32_t)step, (uint32_t)k,
                             (uint32_t)gid(s, i), R);
                for (int e = 0; e < nec; ++e) {
                    freep_t p;
                    memset(&p, 0, sizeof(p));
                    p.box = s->box[i];
                    p.q[0] = s->q[3 * i]; p.q[1] = s->q[3 * i + 1]; p.q[2] = s->q[3 * i + 2];
                    memcpy(p.nbr, s->nbr + i * kn, sizeof(int32_t) * (size_t)kn);
                    p.h2 = s->h2[i];
                    p.N = Nr / (double)(s->K * nec);
                    rotate_axis(R, s->axes_ec + 3 * e, p.d);
                    p.clock = 0.0;
                    p.eps = s->epsrec[i];
                    p.sig = s->cfg.sigma_rec;
                    p.nu = nrb;
                    p.fid = (2ull << 62) | (uint64_t)((gid(s, i) * s->K + k) * nec + e);
                    tally_add(s, p.box, 0, p.N);
                    fl_push(&s->cur, &p);
                }
            }
        }
    }
}

/* N_abs = N_in (1 - exp(-tau)) and the transmitted rest (Sec. 2.1), evaluated so that both
   parts keep full relative precision: the smaller of the two is computed directly and the other
   as the difference, which keeps N_abs + N_out = N_in. */
static void split_absorbed(double N, double tau, double *A, double *T) {
    if (tau < 1.0) {
        *A = -N * expm1(-tau);
        *T = N - *A;
    } else {
        *T = N * exp(-tau);
        *A = N - *T;
    }
}

/* Deliver w photons of a packet (direction d, clock, eps, cross-section sig, frequency nu)
   from a sender at integer position qs to gas neighbour j (Sec. 2.1): optical depth
   tau = sig n_HI,j l with l the distance projected on the propagation direction (sig is the
   bin's grey cross-section sigma_nu, or in a shared bin the packet's photon-weighted mean),
   absorbed N_in (1 - exp(-tau)), the rest arriving at j after l/c and merged into the
   reception cone of its direction. */
static void deliver(orc_sim *s, const int64_t *qs, long long j, double w, const double d[3],
                    double clock, double eps, double sig, int nu) {
    int nrc = s->cfg.n_rc, S = s->S;
    int b = s->box[j];
    if (barrier_crosses(&s->bar[b], qs, s->q + 3 * j)) {   /* removed (Sec. 4): leaves the box */
        tally_add(s, b, 2, w);
        return;
    }
    double u = s->box_L[b] / (double)ORC_Q;
    const int64_t *qj = s->q + 3 * j;
    double t = (double)(qj[0] - qs[0]) * d[0] + (double)(qj[1] - qs[1]) * d[1] +
               (double)(qj[2] - qs[2]) * d[2];
    double l = t * u;
    double tau = (sig * s->nHI[j]) * l;
    double A, T;
    split_absorbed(w, tau, &A, &T);
    s->abs_[j * s->nf + nu] += A;
    s->absE[j] += A * eps;
    s->pass[j * s->nf + nu] += w;
    tally_add(s, b, 1, A);
    int bb = orc_bin(s->R + 9 * j, s->axes_rc, nrc, d);
    long long p = j * S + nu * nrc + bb;
    s->nx[0][p] += T;
    s->nx[1][p] += T * d[0];
    s->nx[2][p] += T * d[1];
    s->nx[3][p] += T * d[2];
    s->nx[4][p] += T * (clock + l / C_LIGHT);
    s->nx[5][p] += T * eps;
    /* shared bin: the merged packet's cross-section is the photon-weighted mean */
    if (s->nsg && nu == 0) s->nsg[j * nrc + bb] += T * sig;
}

/* M4 cubic spline of compact support h (the GADGET form), without its normalisation,
   which cancels in the interpolation below. */
static double kernel_w(double q) {
    if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
    if (q <= 1.0) {
        double a = 1.0 - q;
        return 2.0 * a * a * a;
    }
    return 0.0;
}

/* Where a virtual particle is placed, as an integer offset from its sender (Sec. 2.1;
   reading at make_virtual): the first of 64 counter-based draws, uniform over the integer
   points of [-H, H]^3 with H = floor(sqrt(h2)), that lies in the sender's smoothing sphere and
   in the transmission cone about d; when none does, the point on the axis at H/2. */
void orc_virtual_offset(uint64_t seed, long long step, int hop, uint64_t fid, int64_t h2,
                        const double d[3], int n_tc, int64_t del[3]) {
    uint32_t key[2];
    philox_key(seed, PURPOSE_VIRTUAL, key);
    int64_t H = (int64_t)floor(sqrt((double)h2));
    int64_t span = 2 * H + 1;
    int found = 0;
    for (uint32_t a = 0; a < 64 && !found; ++a) {
        uint32_t ctr[4] = {(uint32_t)step, ((uint32_t)hop << 8) | a, (uint32_t)fid,
                           (uint32_t)(fid >> 32)},
                 r[4];
        orc_philox4x32_10(ctr, key, r);
        for (int c = 0; c < 3; ++c)
            del[c] = (int64_t)(((uint64_t)r[c] * (uint64_t)span) >> 32) - H;
        int64_t r2 = del[0] * del[0] + del[1] * del[1] + del[2] * del[2];
        if (r2 > 0 && r2 <= h2 && orc_in_cone(del, d, n_tc)) found = 1;
    }
    if (!found) {
        double f = 0.5 * (double)H;
        if (f < 1.0) f = 1.0;
        for (int c = 0; c < 3; ++c) del[c] = (int64_t)rint(d[c] * f);
    }
}

/* Virtual particle (Sec. 2.1): created at random inside the transmission cone, its
   properties SPH-interpolated from its own neighbours, absorptions on the way to it
   shared among those neighbours; it then passes the packet on and is deleted.
   Readings: the point is drawn uniformly in the part of the sender's smoothing sphere
   inside the cone (integer rejection sampling, 64 draws, else on the axis at h/2);
   a point outside the box means the photons leave the box (the only escape route);
   n_HI at the point is the Shepard-normalised SPH estimate with weights V_k W_k,
   V_k = N_H,k/n_H,k; absorptions are shared in proportion to V_k W_k n_HI,k; the
   packet is passed on in the next hop, from the virtual particle's position, whatever
   its clock. */
static void make_virtual(orc_sim *s, long long step, int hop, int box, const int64_t *qs,
                         int64_t h2, double N, const double d[3], double clock, double eps,
                         double sig, int nu, uint64_t fid) {
    s->st_virtual++;
    int64_t del[3];
    orc_virtual_offset(s->cfg.seed, step, hop, fid, h2, d, s->cfg.n_tc, del);
    int64_t qv[3] = {qs[0] + del[0], qs[1] + del[1], qs[2] + del[2]};
    if (qv[0] < 0 || qv[1] < 0 || qv[2] < 0 || qv[0] >= ORC_Q || qv[1] >= ORC_Q ||
        qv[2] >= ORC_Q) {
        tally_add(s, box, 2, N);
        s->st_escaped_v++;
        return;
    }
    if (barrier_crosses(&s->bar[box], qs, qv)) {   /* removed on the way to the point */
        tally_add(s, box, 2, N);
        return;
    }
    freep_t v;
    memset(&v, 0, sizeof(v));
    v.box = box;
    v.q[0] = qv[0]; v.q[1] = qv[1]; v.q[2] = qv[2];
    int64_t d2[MAXK];
    box_knn(s, box, qv, -1, v.nbr, d2);
    int kn = s->cfg.n_ngb;
    v.h2 = d2[kn - 1];
    double om[MAXK], sw = 0.0, swn = 0.0;
    for (int k = 0; k < kn; ++k) {
        long long j = v.nbr[k];
        double qk = v.h2 > 0 ? sqrt((double)d2[k] / (double)v.h2) : 0.0;
        om[k] = (s->NH[j] / s->nH[j]) * kernel_w(qk);
        sw += om[k];
    }
    if (!(sw > 0.0)) {
        sw = 0.0;
        for (int k = 0; k < kn; ++k) {
            long long j = v.nbr[k];
            om[k] = s->NH[j] / s->nH[j];
            sw += om[k];
        }
    }
    for (int k = 0; k < kn; ++k) swn += om[k] * s->nHI[v.nbr[k]];
    double nHIv = swn / sw;
    double u = s->box_L[box] / (double)ORC_Q;
    double t = (double)del[0] * d[0] + (double)del[1] * d[1] + (double)del[2] * d[2];
    double l = t * u;
    double tau = (sig * nHIv) * l;
    double A, T;
    split_absorbed(N, tau, &A, &T);
    if (swn > 0.0) {
        for (int k = 0; k < kn; ++k) {
            long long j = v.nbr[k];
            double Ak = A * ((om[k] * s->nHI[j]) / swn);
            s->abs_[j * s->nf + nu] += Ak;
            s->absE[j] += Ak * eps;
            tally_add(s, box, 1, Ak);
        }
    }
    v.N = T;
    v.d[0] = d[0]; v.d[1] = d[1]; v.d[2] = d[2];
    v.clock = clock + l / C_LIGHT;
    v.eps = eps;
    v.sig = sig;
    v.nu = nu;
    v.fid = orc_mix64(fid);
    fl_push(&s->nxt, &v);
}

/* One packet sent from a sender (gas particle, source or virtual particle) holding the
   neighbour list nbr: the neighbours inside its transmission cone share it equally
   (reading: the paper only says the packet is distributed among them), in neighbour
   order; an empty cone creates a virtual particle. */
static void send_packet(orc_sim *s, long long step, int hop, int box, const int64_t *qs,
                        const int32_t *nbr, int64_t h2, double N, const double d[3],
                        double clock, double eps, double sig, int nu, uint64_t fid) {
    s->st_sends++;
    int kn = s->cfg.n_ngb, members[MAXK], m = 0;
    for (int k = 0; k < kn; ++k) {
        const int64_t *qj = s->q + 3 * (long long)nbr[k];
        int64_t del[3] = {qj[0] - qs[0], qj[1] - qs[1], qj[2] - qs[2]};
        if (orc_in_cone(del, d, s->cfg.n_tc)) members[m++] = k;
    }
    if (m == 0) {
        make_virtual(s, step, hop, box, qs, h2, N, d, clock, eps, sig, nu, fid);
        return;
    }
    double w = N / (double)m;
    for (int a = 0; a < m; ++a) deliver(s, qs, nbr[members[a]], w, d, clock, eps, sig, nu);
}

/* Transport (Sec. 2.1): every packet whose clock has not reached the end of the step
   moves forward one neighbour at a time until all clocks have run out or all photons
   have been absorbed or have left the box.  Packets that arrive at a particle merge
   per reception cone and frequency; a packet whose clock has run out waits at its
   particle (and may be carried forward again when a younger packet merges into its
   cone, the merged clock being the photon-weighted mean). */
int orc_transport(orc_sim *s, long long step) {
    long long n = s->n;
    int S = s->S, nrc = s->cfg.n_rc, kn = s->cfg.n_ngb;
    int status = ORC_OK;
    s->st_hops = 0;
    s->st_virtual = 0;
    s->st_escaped_v = 0;
    s->st_sends = 0;
    for (int hop = 0;; ++hop) {
        long long nact = 0;
        for (long long i = 0; i < n; ++i)
            for (int sl = 0; sl < S; ++sl) nact += slot_active(s, i, sl, NULL);
        long long nfree = 0;
        for (long long f = 0; f < s->cur.n; ++f) nfree += s->cur.p[f].N > 0.0;
        if (nact == 0 && nfree == 0) break;
        if (hop >= s->cfg.hop_cap) {
            status = ORC_ERR_HOP_LIMIT;
            for (long long f = 0; f < s->cur.n; ++f)
                if (s->cur.p[f].N > 0.0) tally_add(s, s->cur.p[f].box, 2, s->cur.p[f].N);
            s->cur.n = 0;
            break;
        }
        /* waiting packets stay where they are */
        for (int f = 0; f < 6; ++f) memset(s->nx[f], 0, sizeof(double) * (size_t)(n * S));
        if (s->nsg) memset(s->nsg, 0, sizeof(double) * (size_t)(n * nrc));
        for (long long i = 0; i < n; ++i)
            for (int sl = 0; sl < S; ++sl) {
                long long p = i * S + sl;
                if (s->sl[0][p] > 0.0 && !slot_active(s, i, sl, NULL)) {
                    for (int f = 0; f < 6; ++f) s->nx[f][p] = s->sl[f][p];
                    if (s->nsg && sl < nrc) s->nsg[i * nrc + sl] = s->sg[i * nrc + sl];
                }
            }
        s->nxt.n = 0;
        /* gas particles send, in index order */
        for (long long i = 0; i < n; ++i)
            for (int sl = 0; sl < S; ++sl) {
                double clock;
                if (!slot_active(s, i, sl, &clock)) continue;
                long long p = i * S + sl;
                double N = s->sl[0][p];
                double M[3] = {s->sl[1][p], s->sl[2][p], s->sl[3][p]}, d[3];
                packet_dir(M, d);
                double eps = s->sl[5][p] / N;
                /* shared bin: the packet's mean cross-section; else its bin's */
                double sig = (s->sg && sl < nrc) ? s->sg[i * nrc + sl] / N : s->sigma[sl / nrc];
                send_packet(s, step, hop, s->box[i], s->q + 3 * i, s->nbr + i * kn, s->h2[i],
                            N, d, clock, eps, sig, sl / nrc, gid(s, i) * S + sl + 1);
            }
        /* then sources (first hop) and virtual particles, in creation order */
        for (long long f = 0; f < s->cur.n; ++f) {
            freep_t *p = &s->cur.p[f];
            if (!(p->N > 0.0)) continue;
            send_packet(s, step, hop, p->box, p->q, p->nbr, p->h2, p->N, p->d, p->clock,
                        p->eps, p->sig, p->nu, p->fid);
        }
        for (int f = 0; f < 6; ++f) {
            double *t = s->sl[f];
            s->sl[f] = s->nx[f];
            s->nx[f] = t;
        }
        double *tg = s->sg;
        s->sg = s->nsg;
        s->nsg = tg;
        freelist_t t = s->cur;
        s->cur = s->nxt;
        s->nxt = t;
        s->st_hops++;
    }
    return status;
}

/* Chemistry step of every particle (Sec. 2.1, Sec. 2.2); the recombination photons
   found here are emitted at the start of the next RT step.  Returns
   ORC_ERR_SUBCYCLE_LIMIT when some particle's energy step was held at the subcycle floor
   dt/sub_cap (the state is still updated). */
int orc_chemistry(orc_sim *s) {
    long long nsub = 0, nfloor = 0;
    for (long long i = 0; i < s->n; ++i) {
        double phot = 0.0;
        for (int nu = 0; nu < s->nf; ++nu) phot += s->abs_[i * s->nf + nu];
        double out[3];
        orc_chem_particle(&s->cfg, s->nH[i], s->NH[i], phot, s->absE[i], &s->xHI[i], &s->T[i],
                          out);
        s->Nrec[i] = out[0];
        s->epsrec[i] = s->cfg.eps_rr_fixed >= 0.0 ? s->cfg.eps_rr_fixed : K_B * s->T[i];
        nsub += (long long)out[1];
        nfloor += (long long)out[2];
    }
    s->st_sub = nsub;
    s->st_floor = nfloor;
    return nfloor > 0 ? ORC_ERR_SUBCYCLE_LIMIT : ORC_OK;
}

int orc_step(orc_sim *s, long long step) {
    if (!s->built) return ORC_ERR_INVALID;
    orc_rotate(s, step);
    orc_rebin(s);
    orc_emit(s, step);
    int st = orc_transport(s, step);
    int cs = orc_chemistry(s);
    return st != ORC_OK ? st : cs;
}

void orc_cone_masks(const orc_sim *s, uint32_t *mask) {
    int S = s->S, kn = s->cfg.n_ngb;
    for (long long i = 0; i < s->n; ++i)
        for (int sl = 0; sl < S; ++sl) {
            uint32_t m = 0;
            if (slot_active(s, i, sl, NULL)) {
                long long p = i * S + sl;
                double M[3] = {s->sl[1][p], s->sl[2][p], s->sl[3][p]}, d[3];
                packet_dir(M, d);
                for (int k = 0; k < kn; ++k) {
                    const int64_t *qj = s->q + 3 * (long long)s->nbr[i * kn + k];
                    const int64_t *qi = s->q + 3 * i;
                    int64_t del[3] = {qj[0] - qi[0], qj[1] - qi[1], qj[2] - qi[2]};
                    if (orc_in_cone(del, d, s->cfg.n_tc)) m |= 1u << k;
                }
            }
            mask[i * S + sl] = m;
        }
}

/* The same membership test with the packet directions given ([n * S * 3], row per slot)
   instead of formed from the held momenta: the masks of a transport whose direction
   arithmetic differs from FP64 (the FP32 packets), evaluated with the exact test (Sec. 2.1:
   the cone of solid angle 4 pi / N_TC about the packet direction). */
void orc_cone_masks_dir(const orc_sim *s, const double *dirs, uint32_t *mask) {
    int S = s->S, kn = s->cfg.n_ngb;
    for (long long i = 0; i < s->n; ++i)
        for (int sl = 0; sl < S; ++sl) {
            uint32_t m = 0;
            if (slot_active(s, i, sl, NULL)) {
                const double *d = dirs + 3 * (i * S + sl);
                for (int k = 0; k < kn; ++k) {
                    const int64_t *qj = s->q + 3 * (long long)s->nbr[i * kn + k];
                    const int64_t *qi = s->q + 3 * i;
                    int64_t del[3] = {qj[0] - qi[0], qj[1] - qi[1], qj[2] - qi[2]};
                    if (orc_in_cone(del, d, s->cfg.n_tc)) m |= 1u << k;
                }
            }
            mask[i * S + sl] = m;
        }
}

void orc_get_slots(const orc_sim *s, double *f) {
    long long m = s->n * s->S;
    for (int k = 0; k < 6; ++k) memcpy(f + k * m, s->sl[k], sizeof(double) * (size_t)m);
}

void orc_set_slots(orc_sim *s, const double *f) {
    long long m = s->n * s->S;
    for (int k = 0; k < 6; ++k) memcpy(s->sl[k], f + k * m, sizeof(double) * (size_t)m);
}

void orc_get_shared_sigma(const orc_sim *s, double *G) {
    if (s->sg) memcpy(G, s->sg, sizeof(double) * (size_t)(s->n * s->cfg.n_rc));
}

void orc_set_shared_sigma(orc_sim *s, const double *G) {
    if (s->sg) memcpy(s->sg, G, sizeof(double) * (size_t)(s->n * s->cfg.n_rc));
}

void orc_get_state(const orc_sim *s, double *x_HI, double *T, double *N_rec,
                   double *eps_rec) {
    size_t b = sizeof(double) * (size_t)s->n;
    if (x_HI) memcpy(x_HI, s->xHI, b);
    if (T) memcpy(T, s->T, b);
    if (N_rec) memcpy(N_rec, s->Nrec, b);
    if (eps_rec) memcpy(eps_rec, s->epsrec, b);
}

void orc_set_state(orc_sim *s, const double *x_HI, const double *T, const double *N_rec,
                   const double *eps_rec) {
    size_t b = sizeof(double) * (size_t)s->n;
    if (x_HI) memcpy(s->xHI, x_HI, b);
    if (T) memcpy(s->T, T, b);
    if (N_rec) memcpy(s->Nrec, N_rec, b);
    if (eps_rec) memcpy(s->epsrec, eps_rec, b);
}

void orc_get_deposits(const orc_sim *s, double *abs_, double *absE, double *pass) {
    if (abs_) memcpy(abs_, s->abs_, sizeof(double) * (size_t)(s->n * s->nf));
    if (absE) memcpy(absE, s->absE, sizeof(double) * (size_t)s->n);
    if (pass) memcpy(pass, s->pass, sizeof(double) * (size_t)(s->n * s->nf));
}

void orc_get_budget(const orc_sim *s, double *out) {
    for (int b = 0; b < s->nb; ++b) {
        for (int f = 0; f < 3; ++f) out[4 * b + f] = s->tally[4 * b + f] + s->tallc[4 * b + f];
        double fl = 0.0, fc = 0.0;
        for (long long i = s->box_off[b]; i < s->box_off[b + 1]; ++i)
            for (int sl = 0; sl < s->S; ++sl) kadd(&fl, &fc, s->sl[0][i * s->S + sl]);
        for (long long f = 0; f < s->cur.n; ++f)
            if (s->cur.p[f].box == b) kadd(&fl, &fc, s->cur.p[f].N);
        out[4 * b + 3] = fl + fc;
    }
}

void orc_get_stats(const orc_sim *s, long long out[6]) {
    out[0] = s->st_hops;
    out[1] = s->st_virtual;
    out[2] = s->st_escaped_v;
    out[3] = s->st_sub;
    out[4] = s->st_sends;
    out[5] = s->st_floor;
}
