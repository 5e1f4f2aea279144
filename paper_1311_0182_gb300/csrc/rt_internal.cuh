// rt_internal.cuh -- internal state and device helpers of the TRAPHIC transport library.
//
// The whole library is compiled with -fmad=false (and the host part with -ffp-contract=off):
// every FP64 expression that decides an integer (neighbour order, cone membership, reception
// cone, rotation, virtual-particle position) is evaluated with the operation order written
// here, so that it matches a plain IEEE evaluation of the same formula.  Where a fused
// multiply-add is wanted for speed it is written out as __fmaf_rn.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/traphic_rt.h"

#define RT_Q 1048576          // 2^20 quantisation cells per box side
#define RT_BUDGET_CHUNK 4096
#define RT_OCC_MIN 1           // finest kNN grid the occupancy search tries
#define RT_MAXK 32            // maximum neighbours per particle
#define RT_FREE_BIT (1ull << 63)
#define RT_SCAN_NB 608         // blocks of every prefix-sum launch (4 per SM)

// error bits of the sticky device error word
enum { ERRB_FREE_CAP = 1, ERRB_STAGE_CAP = 2, ERRB_RANGE = 4, ERRB_KNN = 8 };

// device counters
enum {
    CNT_ACTIVE = 0,     // active slots after the hop
    CNT_NREQ = 1,       // virtual-particle requests of the hop (= free packets of the next hop)
    CNT_LIVE = 2,       // live free packets for the next hop
    CNT_STAGE = 3,      // staged free-packet contributions of the hop
    CNT_ERR = 4,        // sticky error bits
    CNT_VIRT = 5,       // virtual particles this step
    CNT_VESC = 6,       // escaped virtual particles this step
    CNT_GAS = 7,        // gas-to-gas contributions this step
    CNT_SUB = 8,        // chemistry subcycles
    CNT_FLOOR = 9,      // subcycle-floor hits
    CNT_NFREE = 10,     // free packets of the current hop
    CNT_ACTP = 11,      // particles with a packet able to move, summed over hops
    CNT_ACTS = 12,      // packets able to move (slots), summed over hops
    CNT_GCON = 13,      // gas-to-gas contributions, summed over hops
    CNT_STG = 14,       // staged free-packet contributions, summed over hops
    CNT_WLS = 15,       // receiver work-list entries, summed over hops
    CNT_OUT = 16,       // occupied slots written by the receiver side, summed over hops
    // hop state: kept on the device so that a captured graph replays the hop loop unchanged
    // (19: unused)
    CNT_CUR = 17,       // slot buffer holding the current packets (0 or 1)
    CNT_FCUR = 18,      // free-packet buffer of the current hop (0 or 1)
    CNT_HOP = 20,       // hops done in this step
    CNT_STEP = 21,      // step number (random streams of the rotations and virtual particles)
    CNT_DROP = 22,      // 1: the hop cap stopped the loop with packets still moving
    CNT_PKFREE = 23,    // largest request count of a hop in this step
    CNT_PKACT = 24,     // largest active-slot count after a hop in this step
    CNT_VQ = 25,        // the virtual particles' work queue: requests taken in this hop
    CNT_N = 32
};


// fixed-point scales of the virtual-particle deposits (relative to the receiver's neutral
// atoms N_HI at the start of the step) and of the escaped tally (relative to the box's
// photon reference)
#define FX_ABS_SCALE 1099511627776.0   // 2^40
#define FX_E_SCALE 68719476736.0       // 2^36 (energy in eV)
#define FX_ESC_SCALE 1125899906842624.0 // 2^50
#define FX_LO_SCALE 4294967296.0        // 2^32: second word of the photon deposits

struct FreeBuf {  // packets not held by gas particles: source packets and virtual particles
    int *box, *qx, *qy, *qz, *nu;
    int *nbr;                 // [cap * kn]
    long long *h2;
    unsigned long long *fid;
    void *N, *dx, *dy, *dz, *clock, *eps;  // Real [cap]
    void *sig;                // Real [cap]: cross-section of the photons in units of sunit
                              // (shared frequency bin only, else null)
};

struct Grid {                 // per-box uniform cell lists (device arrays)
    int *G;                   // cells per side, per box
    int *cs;                  // cell side (quantised units), per box
    long long *coff;          // first cell of the box
    int *start;               // [ncells + 1] offsets into items
    int4 *items;              // (qx, qy, qz, local index) sorted by cell
    long long ncells;
    int *tab;                 // cell offsets of the kNN search, nearest first (rt_knn.cuh)
    // per-cell candidate lists of the virtual particles' kNN (rt_knn.cuh): cand_off[ncells + 1]
    // offsets into cand; an entry is ring << 24 | the item's position among the box's items
    long long *cand_off;
    unsigned *cand;
    long long cand_cap;       // entries allocated
};

struct HopScratch {           // per-hop scratch: [0] free packets, [1] n + free, [2] requests, [3] staged
    int *lens;
    unsigned *fmask;
    int *stcnt, *stoff;
    unsigned long long *esc_r;
    unsigned char *vstat;
};

// Artificial photon barrier of a box (Sec. 4): a disk perpendicular to coordinate `axis`, in
// doubled quantised units: plane at the odd coordinate p2, centre (c1, c2) in the next two
// axes (cyclic order), radius r2.  axis < 0: none.
struct Barrier {
    int axis;
    long long p2, c1, c2, r2;
};

// Does the straight path from a to b cross the barrier?  The plane separates a and b, and
// the crossing point lies within the radius: exact in 128-bit integers (|terms| < 2^91).
__host__ __device__ __forceinline__ bool barrier_crosses(const Barrier &B, int ax, int ay, int az,
                                                         int bx, int by, int bz) {
    if (B.axis < 0) return false;
    long long a[3] = {ax, ay, az}, b[3] = {bx, by, bz};
    int i0 = B.axis, i1 = (B.axis + 1) % 3, i2 = (B.axis + 2) % 3;
    long long sa = 2 * a[i0] - B.p2, sb = 2 * b[i0] - B.p2;   // odd: never 0
    if ((sa < 0) == (sb < 0)) return false;
    long long D = sa - sb;
    __int128 y = (__int128)(2 * a[i1] - B.c1) * D + (__int128)sa * (2 * (b[i1] - a[i1]));
    __int128 z = (__int128)(2 * a[i2] - B.c2) * D + (__int128)sa * (2 * (b[i2] - a[i2]));
    __int128 rD = (__int128)B.r2 * D;
    return (unsigned __int128)(y * y) + (unsigned __int128)(z * z) <=
           (unsigned __int128)(rD * rD);
}

// the kernels call it out of line: its 128-bit arithmetic would otherwise raise the register
// pressure of every hop kernel, and it runs only in boxes with a barrier
static __device__ __noinline__ bool barrier_crosses_call(const Barrier &B, int ax, int ay,
                                                         int az, int bx, int by, int bz) {
    return barrier_crosses(B, ax, ay, az, bx, by, bz);
}

struct DevPtrs {              // plain pointers handed to kernels (by value)
    // sizes and parameters
    long long n;
    int nb, ns, nf, S, K, kn, nrc, nec, ntc, nfs;
    int fp32;
    double dt, dt_em, sigma_rec, T_floor, eps_rr_fixed;
    double eunit;             // energy unit of the slot field E: 1 erg (FP64), 1 eV (FP32)
    int rec_mode, evolve_T, sub_cap, cool_flags;
    // shared frequency bin (Sec. 2.2, last paragraph): recombination photons in source bin
    // rbin = 0 (else rbin = nf - 1, a bin of their own); each slot of bin 0 carries
    // G = sum N sigma (slG, Real [n * nrc], slot (i, b) at i * nrc + b) in units of
    // sunit * the slot's photon unit: 1 cm^2 (FP64), 1e-18 cm^2 (FP32)
    int shared, rbin;
    double sunit;
    unsigned long long seed;
    long long F_cap, ST_cap;
    // boxes
    long long *box_off;
    double *box_L, *box_u, *norm, *ref, *vunit;
    unsigned long long *esc_fx;
    double *tally;            // [nb * 4]
    // budget reduction: fixed chunks of RT_BUDGET_CHUNK particles (CSR over boxes)
    int nbch;
    int *box_bch;             // [nb + 1] first chunk of each box
    long long *bch_lo;        // [nbch + 1] particle ranges
    double *bpart;            // [nbch * 2]
    // particles
    int *pbox, *qx, *qy, *qz;
    double *nH, *NH, *xHI, *T, *Nrec, *epsrec, *nHI, *phot;
    void *nHIr, *Vr, *depE_s;  // Real [n]
    void *dep_s;               // Real [n]: fixed-point scale of photon deposits
    // sources
    int *sbox, *sqx, *sqy, *sqz;
    // identities in the random streams: particle i of box b draws as gid0[b] + (i - box_off[b]),
    // source j as sid[j] (by default their own indices)
    long long *gid0, *sid;
    double *ndot, *sigma, *eps;  // [ns*nfs], [nf], [nf]
    float *sigmaf, *box_uf, *escf;  // FP32 copies: sigma [nf], box unit [nb], escape scale [nb]
    float *passf;                // [n * nf] photons passing (FP32 path, slot units)
    // neighbours
    int *nbr, *snbr;
    long long *h2, *sh2;
    double *sdir;             // [ns * 3] fixed direction of a directed source (0: isotropic)
    int *sgate;               // [ns] 1: emits only while its nearest gas particle is ionised
    Barrier *bar;             // [nb] photon barriers
    int any_bar;              // some box has a barrier
    int kwide;                // some box holds more than 2^22 particles (24-bit kNN keys)
    int gated;                // some source has a gate
    float *fdx, *fdy, *fdz;   // forward offsets q_j - q_i, [n * kn]
    int *rev_off;
    unsigned *rev_ent;        // (i << 5) | k
    float *rdx, *rdy, *rdz;   // offsets in reverse order
    Grid grid;
    // rotations
    double *R, *Rs;
    float *Rf;
    // slots (double-buffered): 6 Real fields + occupancy/activity words per (i, nu)
    void *sl[2][6];
    void *slG[2];             // shared bin: cross-section sums of bin 0 (null otherwise)
    unsigned *occ[2], *act[2];
    // phase-A records, one per slot, 8 Real each (w, dx, dy, dz, clock, eps, sigma, unused;
    // sigma in units of sunit, written for bin 0 with a shared bin only):
    // the receiver side reads a record as one aligned 32-byte (FP32) or 64-byte (FP64) piece;
    // and transposed cone bitmaps
    void *rec;
    unsigned *bm;             // receiver-ordered cone bitmaps [nu * n * kn + p], p = reverse position
    int *revpos;              // position of forward entry (i, k) in the reverse lists
    unsigned *emp;            // empty-cone bits [n * nf]
    int *touched;             // per (j, nu): 1 when a gas sender wrote a bitmap word this hop
    // requests
    int *reqcnt, *reqoff;     // [n + F_cap]
    unsigned long long *req;  // [F_cap]
    FreeBuf fr[2];
    // staged free-packet contributions
    int *st_key;              // receiver key j*nf+nu
    long long *st_ord;        // ordering key f*kn + k
    int *st_bin;
    void *st_v[10];           // T, T dx, T dy, T dz, T clock, T eps, A, A eps, w, T sigma (Real;
                              // the last with a shared bin only)
    int *seg_cnt, *seg_off, *seg_fill, *seg_idx;
    // accumulators
    double *abs, *absE, *pass;                // [n * nf]
    unsigned long long *fx_abs, *fx_lo, *fx_E;  // [n * nf]: photons (2 words), energy
    long long *cnt;                           // CNT_N counters
    int ax_rc, ax_ec;         // index of the reception / emission direction set in c_axes*
    int *worklist;            // (particle, nu) keys a hop's receiver side has to visit
};

// the low word of a device counter, loaded where it is used (volatile: the load is neither
// hoisted nor kept in a register across the caller's loops)
__device__ __forceinline__ unsigned cnt_word(const DevPtrs &P, int k) {
    unsigned v;
    asm volatile("ld.global.b32 %0, [%1];" : "=r"(v) : "l"(P.cnt + k));
    return v;
}

// identity of particle i (of box b) in the random streams
__device__ __forceinline__ unsigned long long gid_of(const DevPtrs &P, long long i, int b) {
    return (unsigned long long)(P.gid0[b] + (i - P.box_off[b]));
}

// kernel identities for the launch counter and the optional per-kernel timer
enum {
    KT_ROTATE, KT_REBIN, KT_EMIT_REC, KT_EMIT_SRC, KT_PHASE_A, KT_FREE_A, KT_SCAN, KT_EXPAND,
    KT_FREE_C, KT_VIRTUAL, KT_SEG_FILL, KT_SEG_SORT, KT_PHASE_B, KT_HOP_COUNT, KT_HOP_LENS,
    KT_DROP, KT_CHEM, KT_BUDGET, KT_KNN, KT_WORKLIST, KT_MASKS, KT_N
};

struct KStat {
    double ms = 0.0, bytes = 0.0;
    long long launches = 0;
};

// state of the launch-size tuning on whole steps (tune_launch)
struct TuneState {
    int phase = 0;            // 0: not started; 1: next step runs the best; 2: the candidate; 3: done
    int best[3] = {0, 0, 0};  // grid sizes of the sender side, virtual particles, receiver side
    double best_cost = 0.0;   // ms per unit of work of the best's last step
    std::vector<std::pair<int, int>> cand;   // (kernel, grid size) still to try
    int steps = 0;
};

struct rt_ctx {
    rt_config cfg;
    DevPtrs d;
    std::vector<long long> box_off_h;
    std::vector<double> box_L_h;
    std::vector<int> gridG_h;
    std::vector<Barrier> bar_h;    // host copy of the barriers
    int cell_occ = 9;              // particles per cell of the kNN grids in use
    long long grid_cap = 0;        // cells allocated (the finest grid that can be chosen)
    bool grid_tuned = false;       // occupancy chosen (or fixed by the configuration)
    long long cand_entries = 0;    // entries of the candidate lists in use
    long long cand_fallback = 0;   // cells without a list (their queries take the grid walk)
    long long *cnt_h = nullptr;   // pinned
    std::vector<void *> allocs;
    bool have_particles = false, have_sources = false, built = false;
    bool bm_dirty = false;        // cone bitmaps left by rt_assign_cones (cleared before a hop loop)
    int cur = 0;                  // slot buffer holding the current packets
    int fcur = 0;                 // free buffer of the current hop
    long long nfree_h = 0;        // free packets of the current hop (host copy)
    long long step_dev = -1ll << 63;  // step number held in the device counters (LLONG_MIN: unknown)
    long long stats[RT_NSTATS] = {0};
    std::string err;
    // scan scratch
    int *scan_tmp = nullptr;
    long long scan_tmp_n = 0;
    int *scan_tmp2 = nullptr;     // scratch of the scans on the second stream
    // second stream of the hop loop (work independent of the caller's stream's kernels) and
    // the events that order the two
    cudaStream_t st2 = nullptr;
    cudaEvent_t hev[4] = {nullptr, nullptr, nullptr, nullptr};
    HopScratch hop = {};
    // launch counter and optional per-kernel timing (CUDA events on the launching stream)
    long long launches = 0;
    unsigned prof = 0;         // bit mask of the kernels timed with events
    KStat kstat[KT_N];
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    size_t ev_next = 0;
    // the whole step as one CUDA graph (conditional while node around the hop body); rebuilt
    // when the kernel parameters it captured change
    bool use_graph = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t st_cap = nullptr;     // capture stream
    DevPtrs graph_P;                   // parameters the graph was captured with
    int graph_hop_cap = -1;
    long long graph_launch_step[KT_N] = {0}, graph_launch_hop[KT_N] = {0};
    bool capturing = false;            // launches counted into graph_launch_* while capturing
    bool in_hop_body = false;
    // grid sizes (blocks) of the sender side, the virtual particles and the receiver side
    // (0: the built-in ones), chosen by timing the first hop loop when cfg.tune_launch is set:
    // its hops cycle through the candidates, each of the three kernels is timed with events,
    // and the candidate with the least time per item wins
    int grid_hop[3] = {0, 0, 0};
    bool launch_tuned = false;
    TuneState tune;
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    double *src_emit = nullptr;   // device [nb]: source photons of one step per box
    std::vector<double> src_emit_h, box_NH_h;
};

// ---- helpers shared by the .cu files (host side) ----
rt_status rt_fail(rt_ctx *c, rt_status s, const std::string &msg);
rt_status rt_cuda_check(rt_ctx *c, cudaError_t e, const char *what);
void rt_scan_exclusive(rt_ctx *c, const int *in, int *out, long long n, const int *d_len,
                       int *d_total, cudaStream_t st, int *tmp = nullptr);
void rt_scan_exclusive64(const int *in, long long *out, long long n, long long *tmp,
                         cudaStream_t st);
rt_status rt_knn_build(rt_ctx *c, cudaStream_t st);
// per-box cell grids for a target occupancy; host-synchronous copies: no kernel that reads
// the grids may be in flight
void rt_set_grid(rt_ctx *c, int occupancy);
rt_status rt_run_step_parts(rt_ctx *c, int part, long long step, cudaStream_t st);
// one whole step through the captured graph (captured again when its parameters changed)
rt_status rt_step_graph(rt_ctx *c, long long step, cudaStream_t st);
rt_status rt_step_graph_tuned(rt_ctx *c, long long step, cudaStream_t st);
void rt_graph_destroy(rt_ctx *c);
// the grid sizes (blocks) of the sender side, the virtual particles and the receiver side
void rt_launch_grids(const rt_ctx *c, long long out[3]);
rt_status rt_chem_launch(rt_ctx *c, cudaStream_t st);
// RT_ERR_SUBCYCLE_LIMIT (with its message) when the last chemistry counted floor hits, else RT_OK
rt_status rt_subcycle_status(rt_ctx *c);
rt_status rt_budget_launch(rt_ctx *c, int phase, cudaStream_t st);
void rt_host_axis_set(int n, double *out);
void rt_upload_axes();
// launch bookkeeping: call kt_begin before and kt_end after the launches of kernel `id`
void kt_begin(rt_ctx *c, int id, cudaStream_t st);
void kt_end(rt_ctx *c, int id, cudaStream_t st, int nlaunch = 1);
void kt_resolve(rt_ctx *c);   // after a synchronisation: fold finished event pairs into kstat

// ---- device helpers ----
#define FULLMASK 0xffffffffu

__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11)
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint2 philox_key(unsigned long long seed, unsigned purpose) {
    return make_uint2((unsigned)seed, (unsigned)(seed >> 32) ^ purpose);
}

// SplitMix64 output function (Steele, Lea & Flood 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// random rotation (row-major R) from a uniform quaternion drawn by rejection in the 4-cube
__device__ inline void random_rotation(unsigned long long seed, unsigned purpose, unsigned c0,
                                       unsigned c1, unsigned c2, double *R) {
    uint2 key = philox_key(seed, purpose);
    double q0 = 1.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
    for (unsigned a = 0; a < 16; ++a) {
        uint4 u = philox4x32_10(make_uint4(c0, c1, c2, a), key);
        double v0 = xsub(xmul((double)(u.x >> 8), 1.0 / 8388608.0), 1.0);
        double v1 = xsub(xmul((double)(u.y >> 8), 1.0 / 8388608.0), 1.0);
        double v2 = xsub(xmul((double)(u.z >> 8), 1.0 / 8388608.0), 1.0);
        double v3 = xsub(xmul((double)(u.w >> 8), 1.0 / 8388608.0), 1.0);
        double s = xadd(xadd(xadd(xmul(v0, v0), xmul(v1, v1)), xmul(v2, v2)), xmul(v3, v3));
        if (s > 1e-6 && s <= 1.0) {
            double nn = __dsqrt_rn(s);
            q0 = __ddiv_rn(v0, nn); q1 = __ddiv_rn(v1, nn);
            q2 = __ddiv_rn(v2, nn); q3 = __ddiv_rn(v3, nn);
            break;
        }
    }
    R[0] = xsub(1.0, xmul(2.0, xadd(xmul(q2, q2), xmul(q3, q3))));
    R[1] = xmul(2.0, xsub(xmul(q1, q2), xmul(q0, q3)));
    R[2] = xmul(2.0, xadd(xmul(q1, q3), xmul(q0, q2)));
    R[3] = xmul(2.0, xadd(xmul(q1, q2), xmul(q0, q3)));
    R[4] = xsub(1.0, xmul(2.0, xadd(xmul(q1, q1), xmul(q3, q3))));
    R[5] = xmul(2.0, xsub(xmul(q2, q3), xmul(q0, q1)));
    R[6] = xmul(2.0, xsub(xmul(q1, q3), xmul(q0, q2)));
    R[7] = xmul(2.0, xadd(xmul(q2, q3), xmul(q0, q1)));
    R[8] = xsub(1.0, xmul(2.0, xadd(xmul(q1, q1), xmul(q2, q2))));
}

// R * D (emission direction along a rotated cone axis)
__device__ __forceinline__ void rot_apply(const double *R, const double *D, double *o) {
    o[0] = xadd(xadd(xmul(R[0], D[0]), xmul(R[1], D[1])), xmul(R[2], D[2]));
    o[1] = xadd(xadd(xmul(R[3], D[0]), xmul(R[4], D[1])), xmul(R[5], D[2]));
    o[2] = xadd(xadd(xmul(R[6], D[0]), xmul(R[7], D[1])), xmul(R[8], D[2]));
}

// Transmission cone, exact form: delta . d > 0 and (delta . d)^2 >= (1 - 2/n_tc)^2 |delta|^2
static __device__ __noinline__ bool cone_exact(int dx, int dy, int dz, double d0, double d1,
                                        double d2, int ntc) {
    if ((dx | dy | dz) == 0) return false;
    double t = xadd(xadd(xmul((double)dx, d0), xmul((double)dy, d1)), xmul((double)dz, d2));
    if (!(t > 0.0)) return false;
    long long r2i = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
    double c = xsub(1.0, __ddiv_rn(2.0, (double)ntc));
    return xmul(t, t) >= xmul(xmul(c, c), (double)r2i);
}

// Fast FP32 test with a guard band; falls back to the exact test inside the band.  The
// FP32 cosine estimate is within ~1e-6 of the exact value, far inside the 2e-5 band.
#define CONE_BAND 2e-5f
// (the direction comes in the packet's own precision; conversions to FP64 run on the FP64
// pipe, so they happen only inside the band)
template <typename Real>
__device__ __forceinline__ bool cone_test(int dx, int dy, int dz, float fx, float fy, float fz,
                                          Real d0, Real d1, Real d2, float cf, int ntc) {
    if ((dx | dy | dz) == 0) return false;
    float r2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, fz * fz));
    float cs = __fmaf_rn(fx, (float)d0, __fmaf_rn(fy, (float)d1, fz * (float)d2)) * rsqrtf(r2);
    if (cs > cf + CONE_BAND) return true;
    if (cs < cf - CONE_BAND) return false;
    return cone_exact(dx, dy, dz, (double)d0, (double)d1, (double)d2, ntc);
}

// Reception cone of direction d at a particle with rotation R: argmax_b (R^T d) . D_b,
// first maximum on ties.  Exact (FP64) form.
static __device__ __noinline__ int bin_exact(const double *R, const double *axes, int nrc, double d0,
                                      double d1, double d2) {
    double e0 = xadd(xadd(xmul(R[0], d0), xmul(R[3], d1)), xmul(R[6], d2));
    double e1 = xadd(xadd(xmul(R[1], d0), xmul(R[4], d1)), xmul(R[7], d2));
    double e2 = xadd(xadd(xmul(R[2], d0), xmul(R[5], d1)), xmul(R[8], d2));
    int best = 0;
    double bs = 0.0;
#pragma unroll 1
    for (int b = 0; b < nrc; ++b) {
        double sc = xadd(xadd(xmul(e0, axes[3 * b]), xmul(e1, axes[3 * b + 1])),
                         xmul(e2, axes[3 * b + 2]));
        if (b == 0 || sc > bs) { bs = sc; best = b; }
    }
    return best;
}

// octahedral-map candidate table of the reception cones (bin_fast, rt_transport.cu)
#define BIN_TAB_M 32
#define BIN_TAB_ALL 0xfefefefeu   // table entry: scan every direction

// M4 cubic spline of support 1 (unnormalised)
template <typename Real>
__device__ __forceinline__ Real kernel_w(Real q) {
    if (q <= Real(0.5)) return Real(1) - Real(6) * q * q + Real(6) * q * q * q;
    if (q <= Real(1)) {
        Real a = Real(1) - q;
        return Real(2) * a * a * a;
    }
    return Real(0);
}

template <typename Real> __device__ __forceinline__ Real rt_exp(Real x);
template <> __device__ __forceinline__ float rt_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double rt_exp<double>(double x) { return exp(x); }
template <typename Real> __device__ __forceinline__ Real rt_expm1(Real x);
template <> __device__ __forceinline__ float rt_expm1<float>(float x) { return expm1f(x); }
template <> __device__ __forceinline__ double rt_expm1<double>(double x) { return expm1(x); }
template <typename Real> __device__ __forceinline__ Real rt_sqrt(Real x);
template <> __device__ __forceinline__ float rt_sqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rt_sqrt<double>(double x) { return sqrt(x); }

// N_abs = N (1 - exp(-tau)) and the transmitted rest (Sec. 2.1), the smaller part computed
// directly so that both keep full relative precision and A + T = N
template <typename Real>
__device__ __forceinline__ void split_absorbed(Real N, Real tau, Real &A, Real &T) {
    if (tau < Real(1)) {
        A = -N * rt_expm1<Real>(-tau);
        T = N - A;
    } else {
        T = N * rt_exp<Real>(-tau);
        A = N - T;
    }
}

// Split a photon deposit, already scaled to units of 2^-40 N_HI, into the two fixed-point
// words (units 1 and 2^-32).  Returns false when the value is outside the accumulator range.
__device__ __forceinline__ bool fx_split(double fa, unsigned long long &qh, unsigned long long &ql) {
    if (!(fa < 4.0e18)) return false;
    double hi = floor(fa);
    qh = (unsigned long long)hi;
    ql = (unsigned long long)llrint((fa - hi) * 4294967296.0);
    return true;
}
// Conversions built from 32-bit pieces: on GB300 conversions between 64-bit integers and
// floating point issue to the (narrow) FP64 pipe.
__device__ __forceinline__ unsigned long long f2u64_rz(float v) {   // 0 <= v < 2^64
    float hi = floorf(v * 2.3283064365386963e-10f);                 // v / 2^32
    float lo = v - hi * 4294967296.0f;
    return ((unsigned long long)__float2uint_rz(hi) << 32) + __float2uint_rz(lo);
}
__device__ __forceinline__ float i64_to_f(long long v) {            // |v| < 2^52
    long long hi = v >> 21;
    return (float)(int)hi * 2097152.0f + (float)(int)(v - (hi << 21));
}
// floor(sqrt(v)) for 0 <= v < 2^52, exact, without FP64
__device__ __forceinline__ long long isqrt64(long long v) {
    long long s = (long long)__float2uint_rz(sqrtf(i64_to_f(v)));
    while (s * s > v) --s;
    while ((s + 1) * (s + 1) <= v) ++s;
    return s;
}
__device__ __forceinline__ bool fx_split(float fa, unsigned long long &qh, unsigned long long &ql) {
    if (!(fa < 4.0e18f)) return false;
    float hi = floorf(fa);
    qh = f2u64_rz(hi);
    ql = __float2uint_rn((fa - hi) * 4294967296.0f);   // < 2^32
    return true;
}

// Kahan-compensated accumulator (FP32 path); plain sums for FP64
template <typename Real> struct KSum {
    Real s, c;
    __device__ __forceinline__ void init(Real v) { s = v; c = Real(0); }
    __device__ __forceinline__ void add(Real v) {
        Real y = v - c;
        Real t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ Real get() const { return s; }
};
template <> struct KSum<double> {
    double s;
    __device__ __forceinline__ void init(double v) { s = v; }
    __device__ __forceinline__ void add(double v) { s = s + v; }
    __device__ __forceinline__ double get() const { return s; }
};

static inline int rt_blocks(long long items, int per_block, int cap = 152 * 32) {
    long long b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}
