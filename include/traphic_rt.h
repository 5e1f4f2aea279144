/*
 * traphic_rt.h -- C ABI of the GB300 (sm_103a) TRAPHIC transport sweep with transport of
 * ionizing recombination radiation.
 *
 * The method is the one of Raicevic, Pawlik, Schaye & Rahmati, "The effect of recombination
 * radiation on the temperature and ionization state of partially ionized gas": photon
 * packets are traced on SPH particles through transmission cones, merged per reception cone
 * (Sec. 2.1), recombination photons are emitted into the reception cones (Sec. 2.2), and a
 * chemistry step updates each particle's neutral fraction and temperature (Sec. 2.1).
 *
 * Conventions
 *  - Units are cgs.  Particles are grouped in independent boxes (a CSR over particles);
 *    positions are per box in [0, L_b).  Positions are quantised to 2^20 cells per box side,
 *    so neighbour lists and cone decisions are exact integer/IEEE decisions.
 *  - `where` says whether a pointer argument is host (RT_HOST) or device (RT_DEVICE) memory.
 *    Host buffers are copied synchronously on `stream`; device buffers must stay valid until
 *    the call's work on `stream` has completed.  The library never keeps a caller pointer.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work is
 *    queued on it asynchronously unless noted.  A context is not thread-safe.
 *  - The library owns every internal buffer: rt_create allocates them on the current device
 *    (rt_build_neighbours adds the candidate lists of the neighbour search, whose size it
 *    counts first) and rt_destroy frees them.
 *  - Every entry point returns an rt_status; nothing is thrown across the ABI.  After a
 *    non-OK status rt_last_error() holds a one-line description.  Device-side limits (hop
 *    cap, packet capacity, deposit range) set a sticky error word that rt_step/rt_transport
 *    read when they finish; kernels never trap.
 *  - The library needs a GPU of compute capability 10.3 (sm_103a).
 */
#ifndef TRAPHIC_RT_H
#define TRAPHIC_RT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_ctx rt_ctx;

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID = 1,   /* bad argument or configuration */
    RT_ERR_OOM = 2,       /* device allocation failed */
    RT_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    RT_ERR_HOP_LIMIT = 4, /* hop loop reached hop_cap; unfinished free packets counted escaped */
    RT_ERR_KNN = 5,       /* a box holds fewer than n_ngb + 1 particles, or (in a box of more
                             than 2^22 particles) an n_ngb-th neighbour lies farther than the
                             kNN keys order exactly: 2^20 / sqrt(3) of the box's 2^20
                             quantisation cells */
    RT_ERR_CAPACITY = 6,  /* more free packets (sources + virtual particles) in a hop than free_cap */
    RT_ERR_STATE = 7,     /* call out of order, e.g. rt_transport before rt_build_neighbours */
    RT_ERR_RANGE = 8,     /* a virtual-particle deposit overflowed its fixed-point accumulator */
    RT_ERR_SUBCYCLE_LIMIT = 9 /* the chemistry held some particle's subcycle at the floor
                                 dt/sub_cap although the 10% energy limit asked for a shorter
                                 one: that explicit energy step changed u by more than 10%.  The
                                 step completed and its state is written; the status says that it
                                 is less accurate there (raise sub_cap).  Numbered 9 because 6 was
                                 taken by RT_ERR_CAPACITY. */
} rt_status;

/* Treatment of recombination radiation (Sec. 2.1, last paragraphs; Sec. 2.2) */
typedef enum {
    RT_REC_TRANSPORT = 0,  /* case A rates; ground-level recombinations emitted and transported */
    RT_REC_OTS_CASE_B = 1, /* on-the-spot: case B rates, nothing emitted */
    RT_REC_CASE_A = 2,     /* case A rates, nothing emitted */
    RT_REC_EMISSION_CONES = 3 /* case A rates; the original implementation (Sec. 2.2): each
                                 recombining particle emits n_ec separate packets in its own
                                 randomly rotated emission cones, K times a step, sent in the
                                 first hop like source packets */
} rt_rec_mode;

enum { RT_COOL_REC = 1, RT_COOL_CEX = 2, RT_COOL_CION = 4, RT_COOL_FF = 8 };
enum { RT_HOST = 0, RT_DEVICE = 1 };

typedef struct {
    int n_ngb;            /* SPH neighbours per particle, 1..32 */
    int n_ec;             /* emission cones per source (8 or 32) */
    int n_tc;             /* transmission cones: cone solid angle 4 pi / n_tc, n_tc >= 2 */
    int n_rc;             /* reception cones per particle (8 or 32) */
    int n_freq_src;       /* source frequency bins (>= 0); one recombination bin is added
                             unless rec_shared_bin is set */
    double dt;            /* RT step, s */
    double dt_em;         /* source emission step, s (dt / dt_em rounded = emissions per step) */
    int rec_mode;         /* rt_rec_mode */
    int evolve_T;         /* 0: temperature held fixed */
    int transport_fp32;   /* 1: packets in FP32 (per-box normalised); 0: all FP64 */
    unsigned long long seed;
    int hop_cap;          /* maximum hops per RT step */
    int sub_cap;          /* maximum chemistry subcycles per step (subcycle floor dt/sub_cap) */
    int cool_flags;       /* RT_COOL_* */
    double T_floor;       /* K */
    double eps_rr_fixed;  /* excess energy of recombination photons, erg; < 0: kT of emitter */
    double sigma_rec;     /* grey cross-section of the recombination photons, cm^2 */
    long long free_cap;   /* capacity of free packets per hop (0: library default) */
    int cell_occupancy;   /* particles per cell of the kNN grids; 0: chosen in
                             rt_build_neighbours by timing the virtual particles' search over
                             1, 2, 3, 4 and 6 */
    int tune_launch;      /* 1: the grid sizes of the three main hop kernels (sender side,
                             virtual particles, receiver side) are chosen by timing the first
                             steps of rt_step as whole step-graph launches: coordinate search
                             from the built-in sizes over 152 x {2, 3, 4, 5} blocks for the
                             virtual particles (one wave at most: they pull work from a queue)
                             and 152 x {8, 16, 32, 64} for the two others, each candidate step
                             after a step of the best so far, per unit of work of the step (18
                             steps).  The winner is kept for the process per
                             configuration and particle count, so a later context of the same
                             kind starts with it.  0: built-in sizes.  Results do not depend on
                             the choice. */
    int launch_grid[3];   /* grid sizes (blocks) of those three kernels; 0: built-in or tuned.
                             Any nonzero entry switches the tuning off (> 0 values are used,
                             zeros keep the built-in size). */
    int rec_shared_bin;   /* 1: one frequency bin for stellar and recombination photons (Sec.
                             2.2, last paragraph): recombination photons travel in source bin 0
                             and there is no recombination bin (n_freq_src bins in all, so
                             n_freq_src >= 1); every packet of bin 0 carries the photon-weighted
                             mean cross-section of its photons, averaged again on every merge,
                             and is attenuated with it.  0: a recombination bin of its own. */
} rt_config;

/* rt_create -- validate cfg, allocate every device buffer for n_boxes boxes whose particle
   ranges are box_off[0..n_boxes] (host, box_off[0] = 0) with side lengths box_L (host, cm),
   and n_src sources.  Sizes only: particle and source data come with rt_set_particles and
   rt_set_sources.  On success *out owns the allocations.  Limits: a box holds at most
   2^24 particles, all boxes together fewer than 2^27.  Errors: RT_ERR_INVALID (also
   beyond those limits), RT_ERR_KNN, RT_ERR_OOM, RT_ERR_CUDA (*out is NULL). */
rt_status rt_create(const rt_config *cfg, int n_boxes, const long long *box_off,
                    const double *box_L, int n_src, rt_ctx **out);

/* rt_destroy -- free every allocation of ctx (NULL is allowed). */
rt_status rt_destroy(rt_ctx *ctx);

/* rt_set_particles -- copy the particle arrays (each [n], n = box_off[n_boxes]) into the
   context: positions (cm, per box in [0, L_b)), hydrogen number density n_H (cm^-3),
   hydrogen atoms per particle N_H, neutral fraction x_HI and temperature T (K).  Resets the
   packets held by the particles, the recombination photons pending and the neighbour lists
   (call rt_build_neighbours again).  Positions outside [0, L_b) are moved onto the box's edge.
   Errors: RT_ERR_INVALID (also for a non-finite position, a non-positive or non-finite density
   or atom count, x_HI outside [0, 1] or a non-positive temperature: the context then holds no
   particles until a valid call), RT_ERR_CUDA. */
rt_status rt_set_particles(rt_ctx *ctx, const double *x, const double *y, const double *z,
                           const double *n_H, const double *N_H, const double *x_HI,
                           const double *T, int where, void *stream);

/* rt_set_sources -- copy the sources: box index (int [n_src]), position ([n_src] each, cm),
   photon rates ndot ([n_src * n_freq_src], row per source, s^-1), and per source frequency
   bin the grey cross-section sigma (cm^2) and excess energy eps (erg) ([n_freq_src]) (Sec.
   2.1: each packet carries one bin; the bin's spectrum is a grey cross-section).  Errors:
   RT_ERR_INVALID (also for a non-finite position, a negative photon rate, a non-positive
   cross-section or a negative excess energy: the context then holds no sources until a valid
   call), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_set_sources(rt_ctx *ctx, const int *box, const double *x, const double *y,
                         const double *z, const double *ndot, const double *sigma,
                         const double *eps, int where, void *stream);

/* rt_set_source_options -- per source, a fixed unit emission direction (dir [n_src * 3]; a zero
   vector keeps the n_ec randomly rotated emission cones) and a gate (gate [n_src]: 1 = the
   source emits only while its nearest gas particle has x_HI < 0.5 at the start of the step,
   0 = always).  A directed source sends, per emission and frequency, one packet of
   ndot * dt_em photons along its direction: the packets of the plane-parallel front of the
   shadow test; the gate switches on its boundary emitters once the front has passed them
   (Sec. 4, App. B).  NULL resets the option for every source.  Host or device arrays
   (`where`); synchronises `stream`.  Errors: RT_ERR_INVALID. */
rt_status rt_set_source_options(rt_ctx *ctx, const double *dir, const int *gate, int where,
                                void *stream);

/* rt_set_identities -- the identities the random streams use (the reception and emission-cone
   rotations and the packet identities that seed the virtual-particle draws; Sec. 2.1 rotates
   cones at random): particle i of box b draws as particle box_first_id[b] + (i - box_off[b]),
   and source j as source src_id[j] (host arrays of n_boxes and n_src entries; NULL keeps the
   own indices, the default).  Boxes cut out of a larger workload with the identities they have
   there repeat their results in it bit for bit (the boxes of a workload are independent), which
   is how the boxes of one workload are split over several GPUs.  Identities must lie in
   [0, 2^32).  Waits for the device.  Errors: RT_ERR_INVALID, RT_ERR_CUDA. */
rt_status rt_set_identities(rt_ctx *ctx, const long long *box_first_id, const long long *src_id);

/* rt_set_barrier -- an artificial photon barrier in box `box` (Sec. 4): the disk of radius
   `radius` (cm) centred at centre[3] (box coordinates, cm), perpendicular to coordinate axis
   `axis` (0, 1, 2), removes every packet whose straight path from sender to receiver (or to
   its virtual particle) crosses it.  Removed photons are counted as escaped.  The plane is
   placed half a quantisation cell above the centre's cell, so no particle lies on it; the
   test is exact integer arithmetic.  radius <= 0 removes the barrier.  Synchronises the
   device.  Errors: RT_ERR_INVALID. */
rt_status rt_set_barrier(rt_ctx *ctx, int box, int axis, const double *centre, double radius);

/* rt_build_neighbours -- exact n_ngb nearest neighbours of every particle and source within
   its box, ordered by (squared quantised distance, index); smoothing length h = distance of
   the n_ngb-th; and the receiver-sorted reverse lists (Sec. 2.1: packets search the
   neighbours within the smoothing volume of the particle they are attached to).  Also builds
   the per-cell candidate lists the virtual particles' neighbour search takes: for each kNN
   cell, every particle that can be among the n_ngb nearest of a point in the cell (about 100
   to 200 four-byte entries per particle, allocated here).  Static density fields: call once
   after rt_set_particles; a later call rebuilds everything.  Synchronises `stream`.  Errors:
   RT_ERR_KNN, RT_ERR_CUDA (also when the candidate lists cannot be allocated). */
rt_status rt_build_neighbours(rt_ctx *ctx, void *stream);

/* rt_assign_cones -- the rotations of step `step` (reception cones of every particle, once
   per step; emission cones of every source, once per emission; Sec. 2.1) and, for the
   packets currently held, the transmission-cone membership of every neighbour (cone of solid
   angle 4 pi / n_tc about the packet direction, Sec. 2.1).  Read with rt_get_rotations and
   rt_get_cone_masks. */
rt_status rt_assign_cones(rt_ctx *ctx, long long step, void *stream);

/* rt_merge -- start of an RT step: reset every packet clock to the step start and re-sort
   the packets held by each particle into its current reception cones, merging packets that
   share a cone and frequency (sums of photons, momentum N*d, N*clock and N*eps; Sec. 2.1,
   Fig. 1a,b).  Uses the rotations of the last rt_assign_cones. */
rt_status rt_merge(rt_ctx *ctx, void *stream);

/* rt_emit -- emission at the start of step `step` (Sec. 2.1, Sec. 2.2, Fig. 1c,d): the
   recombination photons of the last chemistry step go N_rec/n_rc into each reception cone of
   the recombination bin (source bin 0 with rec_shared_bin, where they add N_rec/n_rc sigma_rec
   to the cone's cross-section sum) along its rotated axis, merged with the packets there (with
   rec_mode RT_REC_EMISSION_CONES they leave as separate packets instead); the sources
   emit dt/dt_em times n_ec packets per frequency bin along their rotated emission axes.
   Also restarts the absorption counters and freezes n_HI for the transport. */
rt_status rt_emit(rt_ctx *ctx, long long step, void *stream);

/* rt_transport -- the hop loop of step `step` (Sec. 2.1): each packet whose clock is below
   dt is split equally among the neighbours in its transmission cone (or handed to a virtual
   particle when the cone is empty), attenuated by exp(-sigma n_HI l) photon-conservingly,
   deposited, and merged per reception cone at the receiver, until no packet can move.
   Synchronises `stream` once per hop to test for completion.  Errors: RT_ERR_HOP_LIMIT,
   RT_ERR_CAPACITY, RT_ERR_RANGE, RT_ERR_CUDA. */
rt_status rt_transport(rt_ctx *ctx, long long step, void *stream);

/* rt_chemistry -- per particle: photoionisation and photoheating rates from the step's
   absorptions, subcycled update of x_HI and T, and the ground-level recombination photons to
   emit next step (Sec. 2.1, Sec. 2.2).  Subcycles are limited to a 10% change of the energy
   density, with a floor of dt/sub_cap.  Synchronises `stream`.  Errors: RT_ERR_SUBCYCLE_LIMIT
   (some subcycle was held at the floor; the state is updated, rt_get_stats counts the floor
   hits), RT_ERR_CUDA. */
rt_status rt_chemistry(rt_ctx *ctx, void *stream);

/* rt_step -- one RT step: rt_assign_cones, rt_merge, rt_emit, rt_transport, rt_chemistry and
   the photon budget.  Returns the first non-OK status.  Synchronises `stream` once, at the end.
   By default (rt_set_graph) the whole step runs as one CUDA graph launched on `stream`: the
   hop loop is a conditional while node whose last kernel decides on the device whether
   another hop runs, so no host round trip separates hops.  A transport error takes precedence
   over RT_ERR_SUBCYCLE_LIMIT, which only reports that the (completed) chemistry hit its floor.  The graph is captured on the
   first call and again whenever a parameter it holds changes (configuration, barriers,
   source options, kNN grid, launch sizes).  The hop-by-hop path runs instead while kernels
   are timed (rt_set_profiling), when hop_cap is 0, and for the first step when tune_launch
   chooses the launch sizes; both give bit-identical results.  After an error
   status from the graph the chemistry of that step has run on incomplete absorptions (the
   hop-by-hop path stops before it); the state of a failed step is not meant to be used. */
rt_status rt_step(rt_ctx *ctx, long long step, void *stream);
/* rt_set_graph -- on != 0 (default): rt_step runs as a captured CUDA graph; 0: it drives the
   hop loop from the host, one synchronisation per hop. */
rt_status rt_set_graph(rt_ctx *ctx, int on);

/* rt_get_state / rt_set_state -- x_HI, T, pending recombination photons N_rec and their
   excess energy eps_rec ([n] each; NULL skips a field).  rt_set_state returns RT_ERR_INVALID
   for x_HI outside [0, 1], a non-positive temperature, or negative or non-finite photons or
   energy; the rejected values are then in place and the state must be set again. */
rt_status rt_get_state(rt_ctx *ctx, double *x_HI, double *T, double *N_rec, double *eps_rec,
                       int where, void *stream);
rt_status rt_set_state(rt_ctx *ctx, const double *x_HI, const double *T, const double *N_rec,
                       const double *eps_rec, int where, void *stream);

/* rt_get_budget -- per box, cumulative photons emitted, absorbed, escaped and currently in
   flight ([n_boxes * 4], host).  Synchronises `stream`.  Photon conservation (Abstract,
   Sec. 2.1): emitted = absorbed + escaped + in flight. */
rt_status rt_get_budget(rt_ctx *ctx, double *out, void *stream);

/* --- inspection hooks (parity tests) ---------------------------------------------------- */
/* neighbour lists [n * n_ngb] (global indices), h^2 in quantised units [n]; the same for the
   sources ([n_src * n_ngb], [n_src]); NULL skips */
rt_status rt_get_neighbours(rt_ctx *ctx, int *nbr, long long *h2, int *src_nbr,
                            long long *src_h2, int where, void *stream);
/* quantised positions [n * 3] */
rt_status rt_get_quantised(rt_ctx *ctx, long long *q, int where, void *stream);
/* rt_query_neighbours -- the exact n_ngb nearest particles of m points of box `box`, by the
   search the virtual particles use (Sec. 2.1: a virtual particle's neighbours are the n_ngb
   particles nearest to it), from the per-cell candidate lists that rt_build_neighbours builds.
   q[m * 3]: quantised positions (int, each in [0, 2^20), the units of rt_get_quantised).
   nbr[m * n_ngb]: global particle indices, nearest first, equal distances to the lower index;
   d2[m * n_ngb]: their squared quantised distances; NULL skips.  A point whose search fails
   gets -1 entries.  Allocates temporary device buffers for host arrays and synchronises
   `stream`.  Errors: RT_ERR_STATE (before rt_build_neighbours), RT_ERR_INVALID (a bad box or
   count, or a coordinate out of range: no output is valid then), RT_ERR_KNN (some search
   failed, as for the particles' own), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_query_neighbours(rt_ctx *ctx, int box, long long m, const int *q, int *nbr,
                              long long *d2, int where, void *stream);
/* rotation matrices (row-major): reception [n * 9], emission [n_src * K * 9], K = dt/dt_em */
rt_status rt_get_rotations(rt_ctx *ctx, double *R, double *Rs, int where, void *stream);
/* transmission masks of the held packets [n * S], S = n_rc * (n_freq_src + 1): bit k set
   when neighbour k lies in the cone of slot s; 0 for slots with no packet able to move */
rt_status rt_get_cone_masks(rt_ctx *ctx, unsigned *mask, int where, void *stream);
/* rt_get_cone_masks_noalloc -- the same masks as rt_get_cone_masks, for callers that must not
   allocate device memory: code running under a caller-owned memory budget or pool, or a host
   thread that may not call cudaMalloc/cudaFree while other work is in flight.  The paper has
   no counterpart (it is an interface convenience).  No allocation: the masks are assembled in
   a file-scope device array of 4,194,304 entries (16 MiB) that every GPU loading the library
   holds until the process exits; n * S beyond that is rejected with RT_ERR_INVALID.  The first
   call on a device looks up the array's device address (cudaGetSymbolAddress, with that
   device current); make that first call before any stream capture.  The address is kept for
   the rest of the process, so it stays valid only while that device's primary context lives:
   after cudaDeviceReset on the device, do not call this entry point again.  All calls share the
   array: calls whose work overlaps on the GPU race, so serialise them (one stream, or wait for
   the previous call's copy).  With where == RT_HOST the call synchronises `stream`; with
   RT_DEVICE the copy is queued on `stream`. */
rt_status rt_get_cone_masks_noalloc(rt_ctx *ctx, unsigned *mask, int where, void *stream);
/* held packets: 6 fields [6 * n * S] (N, Mx, My, Mz, C = N*clock, E = N*eps), physical units */
rt_status rt_get_slots(rt_ctx *ctx, double *f, int where, void *stream);
rt_status rt_set_slots(rt_ctx *ctx, const double *f, int where, void *stream);
/* rt_save_state -- checkpoint between steps (the paper has none; GADGET snapshots are implied):
   what a step carries into the next one, byte for byte -- the packets held by the particles
   (slots with their occupancy and activity words, and the cross-section sums of a shared bin),
   x_HI, T, the recombination photons waiting to be emitted and their energy, and the photon
   budget.  With buf NULL, *bytes receives the size needed; otherwise buf (host, *bytes long)
   receives the checkpoint and *bytes its size.  Waits for all work on the device.  Errors:
   RT_ERR_STATE before rt_build_neighbours, RT_ERR_INVALID (buffer too small), RT_ERR_CUDA.
   rt_load_state -- restore a checkpoint into a context of the same configuration and particle
   set whose neighbours are built (a fresh context built from the same inputs gives the same
   neighbour lists, rotations and random streams, so a resumed run repeats an uninterrupted one
   bit for bit).  Errors: RT_ERR_INVALID (not a checkpoint, another configuration, short
   buffer), RT_ERR_STATE, RT_ERR_CUDA. */
rt_status rt_save_state(rt_ctx *ctx, void *buf, size_t *bytes);
rt_status rt_load_state(rt_ctx *ctx, const void *buf, size_t bytes);
/* rt_get_shared_sigma / rt_set_shared_sigma -- with rec_shared_bin (Sec. 2.2, last paragraph:
   one bin for stellar and recombination photons, cross-sections averaged on merging): the
   cross-section sum G = sum N sigma (cm^2 x photons) of each held packet of bin 0, [n * n_rc],
   packet (i, b) at i * n_rc + b; a packet's mean cross-section is G / N.  Get writes 0 for
   empty slots; set writes the field as given (call it after rt_set_slots, which decides which
   slots are held).  Synchronous on `stream`.  Errors: RT_ERR_INVALID (also without a shared
   bin), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_get_shared_sigma(rt_ctx *ctx, double *G, int where, void *stream);
rt_status rt_set_shared_sigma(rt_ctx *ctx, const double *G, int where, void *stream);
/* absorptions of the current step: photons [n * nf], energy [n * nf] (erg), photons passing
   each particle [n * nf] (the intensity diagnostic of Sec. 3); nf = n_freq_src + 1, or
   n_freq_src with rec_shared_bin.  Valid after rt_transport and still after rt_chemistry (the
   values do not depend on the x_HI the chemistry writes); cleared by the next rt_emit.
   Allocates a temporary device buffer and synchronises `stream`. */
rt_status rt_get_deposits(rt_ctx *ctx, double *abs_, double *absE, double *pass, int where,
                          void *stream);
/* statistics of the last rt_transport/rt_chemistry, out[RT_NSTATS] (host): hops, virtual
   particles, escaped virtual particles, chemistry subcycles, subcycle-floor hits, peak free
   packets in a hop, peak active slots in a hop; then summed over the hops of the last
   transport: gas-to-gas contributions, particles with a packet able to move, packets able to
   move, staged free-packet contributions, receiver work-list entries, occupied slots written
   by the receiver side; then the cell occupancy of the kNN grids in use; then the grid sizes
   (blocks) of the sender side, the virtual particles and the receiver side in use; then the
   entries of the per-cell candidate lists of the virtual particles' kNN (4 bytes each, built
   by rt_build_neighbours), and the cells without a list, deep in voids, whose queries take the
   grid walk instead; out[19] is 0 */
#define RT_NSTATS 20
rt_status rt_get_stats(rt_ctx *ctx, long long *out);
/* the isotropic cone direction set with n directions (8 or 32), [n * 3] host */
rt_status rt_axis_set(int n, double *out);

/* rt_set_profiling -- mask: bit k (k = the kernel's position in rt_get_profile's list)
   records a pair of CUDA events on the launching stream around every launch of kernel k and
   sums their durations; -1 profiles every kernel, 0 stops.  Resets the sums.  Synchronises
   the device.  The launch counters run always. */
rt_status rt_set_profiling(rt_ctx *ctx, int mask);

/* rt_get_profile -- total kernel launches since rt_create, and per kernel (at most
   max_kernels entries, host arrays, NULL skips): its name (static string), launches, summed
   device time in ms (while profiling) and algorithmic bytes (reserved, 0).  Synchronises the
   device. */
rt_status rt_get_profile(rt_ctx *ctx, long long *launches_total, int max_kernels,
                         const char **names, long long *launches, double *ms, double *bytes);

const char *rt_last_error(const rt_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
