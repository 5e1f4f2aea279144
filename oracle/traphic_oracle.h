/*
 * traphic_oracle.h -- plain, slow FP64 CPU oracle of one TRAPHIC radiative-transfer
 * step with transport of ionizing recombination radiation (Raicevic, Pawlik, Schaye &
 * Rahmati, "The effect of recombination radiation on the temperature and ionization
 * state of partially ionized gas", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no source, header, table or
 * constant generator with the CUDA library; both follow the same written readings of
 * the paper.
 *
 * Units are cgs throughout.  Positions are given per box in [0, L_b) and quantised to
 * ORC_Q = 2^20 integer cells per box side (a reading: the paper fixes no position
 * arithmetic; integers make neighbour and cone decisions exact and reproducible).
 */
#ifndef TRAPHIC_ORACLE_H
#define TRAPHIC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_HOP_LIMIT = 4, ORC_ERR_SUBCYCLE_LIMIT = 9 };
/* recombination radiation: transported through the reception cones (Sec. 2.2, the new
   implementation); on-the-spot case B; case A; transported through N_EC per-particle emission
   cones whose packets stay separate (Sec. 2.2, the original implementation) */
enum { ORC_REC_TRANSPORT = 0, ORC_REC_OTS_CASE_B = 1, ORC_REC_CASE_A = 2,
       ORC_REC_EMISSION_CONES = 3 };
/* cooling terms (bit flags): recombination, collisional excitation,
   collisional ionisation, free-free */
enum { ORC_COOL_REC = 1, ORC_COOL_CEX = 2, ORC_COOL_CION = 4, ORC_COOL_FF = 8 };

typedef struct {
    int n_ngb;            /* SPH neighbours per particle, 1..32 (Sec. 2.1) */
    int n_ec, n_tc, n_rc; /* emission / transmission / reception cones (Sec. 2.1) */
    int n_freq_src;       /* source frequency bins; one recombination bin is added */
    double dt, dt_em;     /* RT step and emission step, s (Sec. 2.1) */
    int rec_mode;         /* ORC_REC_* (Sec. 2.1 last paragraphs; Sec. 2.2) */
    int evolve_T;         /* 0: temperature held fixed */
    uint64_t seed;
    int hop_cap;          /* maximum hops per RT step */
    int sub_cap;          /* maximum chemistry subcycles per step */
    int cool_flags;       /* ORC_COOL_* */
    double T_floor;       /* K */
    double eps_rr_fixed;  /* erg; < 0 selects kT of the emitting gas (Sec. 2.2) */
    double sigma_rec;     /* grey cross-section of the recombination photons, cm^2 (Sec. 2.2) */
    int rec_shared_bin;   /* 1: recombination photons travel in source bin 0 (no bin of their
                             own); each packet of that bin carries its photon-weighted mean
                             cross-section, averaged on every merge (Sec. 2.2, last paragraph);
                             needs n_freq_src >= 1 */
} orc_config;

typedef struct orc_sim orc_sim;

/* --- building blocks, exposed for pinning tests ------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t orc_mix64(uint64_t z);
int orc_axis_set(int n, double *out /* [n*3] */);
/* random rotation matrix (row-major) drawn from the counter-based generator */
void orc_rotation(uint64_t seed, uint32_t purpose, uint32_t c0, uint32_t c1, uint32_t c2,
                  double R[9]);
int orc_in_cone(const int64_t delta[3], const double d[3], int n_tc);
int orc_bin(const double R[9], const double *axes, int n_rc, const double d[3]);
/* offset of a virtual particle from its sender (h2: the sender's squared smoothing length in
   quantised units; fid: the packet's identity in the generator's counter) */
void orc_virtual_offset(uint64_t seed, long long step, int hop, uint64_t fid, int64_t h2,
                        const double d[3], int n_tc, int64_t del[3]);
/* rate coefficients at T: alpha_A, alpha_B, beta_col, Lrec_A, Lrec_B, L_cex, L_cion, L_ff */
void orc_rates(double T, double out[8]);
/* one particle's chemistry update over dt.  On return x and T hold the new state;
   out[0] = recombination photons to emit, out[1] = subcycles, out[2] = floor hits */
void orc_chem_particle(const orc_config *cfg, double nH, double NH, double phot,
                       double heat, double *x, double *T, double out[3]);
/* exact k nearest neighbours of query points among points (integer coordinates).
   self_offset >= 0: query q is point (self_offset + q) and is excluded. use_grid
   selects the uniform-grid search instead of brute force. */
int orc_knn(long long n_pts, const int64_t *pts /* [n*3] */, long long n_q,
            const int64_t *qpts /* [n_q*3] */, long long self_offset, int k, int use_grid,
            int32_t *out_idx /* [n_q*k] */, int64_t *out_d2 /* [n_q*k] */);

/* --- the full step ------------------------------------------------------------ */
orc_sim *orc_create(const orc_config *cfg, int n_boxes, const long long *box_off,
                    const double *box_L, const double *x, const double *y, const double *z,
                    const double *n_H, const double *N_H, const double *x_HI,
                    const double *T, int n_src, const int *src_box, const double *sx,
                    const double *sy, const double *sz, const double *ndot,
                    const double *sigma, const double *eps);
void orc_destroy(orc_sim *s);
/* per source: a fixed unit emission direction (dir [ns*3], zero vector: isotropic emission
   cones) and a gate (1: emits only while its nearest gas particle has x_HI < 0.5); NULL
   resets to isotropic / ungated (Sec. 4 and App. B: the plane-parallel front and the
   boundary emitters) */
void orc_set_source_options(orc_sim *s, const double *dir, const int *gate);
/* an artificial barrier in box `box` (Sec. 4): the disk of the given radius (cm) centred at
   `centre` (box coordinates, cm), perpendicular to coordinate axis `axis`, removes every
   packet whose straight path crosses it (counted as escaped); radius <= 0 removes it */
void orc_set_barrier(orc_sim *s, int box, int axis, const double centre[3], double radius);
/* the barrier test on its own (doubled quantised units, see orc_set_barrier): does the path
   from a to b cross the disk? */
int orc_barrier_test(const int64_t a[3], const int64_t b[3], int axis, int64_t p2, int64_t c1,
                     int64_t c2, int64_t r2);
int orc_build_neighbours(orc_sim *s);
void orc_get_neighbours(const orc_sim *s, int32_t *nbr, int64_t *h2, int32_t *src_nbr,
                        int64_t *src_h2);
void orc_get_quantised(const orc_sim *s, int64_t *q);
void orc_rotate(orc_sim *s, long long step);       /* reception + emission rotations */
void orc_get_rotations(const orc_sim *s, double *R /* [n*9] */, double *Rs /* [ns*K*9] */);
void orc_rebin(orc_sim *s);                        /* clock reset + re-bin (Sec. 2.1) */
void orc_emit(orc_sim *s, long long step);         /* recombination + source emission */
int orc_transport(orc_sim *s, long long step);     /* hop loop; returns status */
int orc_chemistry(orc_sim *s);     /* ORC_ERR_SUBCYCLE_LIMIT at the subcycle floor */
int orc_step(orc_sim *s, long long step);
/* masks of the current packets: bit k set when neighbour k of particle i lies in the
   transmission cone of slot sl; entries of inactive slots are 0 */
/* Identities in the random streams (rotations, packet identities): particle i of box b draws
   as particle box_first_id[b] + (i - box_off[b]) and source j as source src_id[j]; NULL keeps
   the own indices.  A box cut out of a larger workload with its identities repeats the draws
   it makes there. */
int orc_set_identities(orc_sim *s, const long long *box_first_id, const long long *src_id);
void orc_cone_masks(const orc_sim *s, uint32_t *mask /* [n*S] */);
void orc_cone_masks_dir(const orc_sim *s, const double *dirs, uint32_t *mask); /* given directions [n*S*3] */
/* state access; slot fields are N, Mx, My, Mz, C (= N * clock), E (= N * eps) */
void orc_get_slots(const orc_sim *s, double *f /* [6*n*S] */);
void orc_set_slots(orc_sim *s, const double *f);
/* with rec_shared_bin: the cross-section field G = sum of N sigma of the slots of bin 0,
   [n*n_rc], slot (i, b) at i*n_rc + b; no-ops otherwise */
void orc_get_shared_sigma(const orc_sim *s, double *G);
void orc_set_shared_sigma(orc_sim *s, const double *G);
void orc_get_state(const orc_sim *s, double *x_HI, double *T, double *N_rec,
                   double *eps_rec);
void orc_set_state(orc_sim *s, const double *x_HI, const double *T, const double *N_rec,
                   const double *eps_rec);
void orc_get_deposits(const orc_sim *s, double *abs_ /* [n*nf] */, double *absE /* [n] */,
                      double *pass /* [n*nf] */);
/* per box: emitted, absorbed, escaped, in flight (cumulative photon counts) */
void orc_get_budget(const orc_sim *s, double *out /* [n_boxes*4] */);
/* hops, virtual particles, escaped virtuals, chemistry subcycles, and packets sent (by gas
   particles, sources and virtual particles) of the last step */
void orc_get_stats(const orc_sim *s, long long out[6]);

#ifdef __cplusplus
}
#endif
#endif
