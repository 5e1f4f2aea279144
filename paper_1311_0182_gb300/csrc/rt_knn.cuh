// rt_knn.cuh -- exact k-nearest-neighbour search by one warp over a box's uniform cell list.
//
// The result is the k smallest (squared quantised distance, local index) pairs, a unique set,
// held sorted across the lanes: lane l has the l-th nearest.  The search first visits the cells
// within Chebyshev radius KNN_TAB_R of the query's cell, 32 at a time, nearest first (a fixed
// table of offsets sorted by the smallest distance a cell at that offset can have), skipping
// every cell farther than the current k-th distance, and stops as soon as no remaining cell can
// be nearer; when the k-th distance still reaches beyond that block, growing shells of cells
// follow until it is below the distance to the outside of the visited block.
//
// A pair is one 64-bit key, d2 * 2^ib + index, with ib index bits per box: 22 for a box of up
// to 2^22 particles, 24 up to 2^24 (the most a box may hold, checked when the context is
// created).  Quantised offsets are below 2^20 per axis, so d2 < 3 * 2^40 < 2^42: with 22 index
// bits d2 always fits.  With 24, d2 is saturated at 2^40 - 2, which only points farther apart
// than 2^20 / sqrt(3) of the box's 2^20 cells reach; a search whose k-th neighbour is that far
// reports failure instead of a possibly wrong order.  Key order is the (d2, index) order, and
// one compare or shuffle pair moves it.
#pragma once
#include "rt_internal.cuh"

#define KNN_INF 0x7fffffffffffffffll
#define KNN_IB_SMALL 22        // index bits of a box of up to 2^22 particles
#define KNN_IB_LARGE 24        // index bits of a larger box (up to 2^24 particles)
#define KNN_KEY_NONE 0xffffffffffffffffull
// merge by insertion when at most this many candidates of a batch pass the k-th key
#ifndef KNN_INSERT_MAX
#define KNN_INSERT_MAX 16
#endif

// the largest d2 a key with IB index bits holds
template <int IB> __device__ __forceinline__ long long knn_d2max() { return (1ll << (64 - IB)) - 2; }

template <int IB>
__device__ __forceinline__ unsigned long long knn_key(long long d2, int idx) {
    // with 22 index bits every d2 (< 3 * 2^40) fits; with 24 it saturates
    if (IB > KNN_IB_SMALL && d2 > knn_d2max<IB>()) d2 = knn_d2max<IB>();
    return ((unsigned long long)d2 << IB) | (unsigned long long)idx;
}

// bitonic sort (ascending) of one key per lane across the warp
__device__ __forceinline__ void warp_sort(unsigned long long &k) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 2; s <= 32; s <<= 1) {
#pragma unroll
        for (int j = s >> 1; j > 0; j >>= 1) {
            unsigned long long o = __shfl_xor_sync(FULLMASK, k, j);
            bool up = ((lane & s) == 0);
            bool lower = (lane & j) == 0;
            bool take_min = (lower == up);
            if (take_min ? o < k : o > k) k = o;
        }
    }
}

// top (sorted ascending across lanes) <- the 32 smallest of top U batch (batch unsorted)
__device__ __forceinline__ void warp_merge(unsigned long long &t, unsigned long long b) {
    int lane = threadIdx.x & 31;
    warp_sort(b);
    unsigned long long r = __shfl_sync(FULLMASK, b, 31 - lane);
    if (r < t) t = r;
    // t is now bitonic: merge down
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        unsigned long long o = __shfl_xor_sync(FULLMASK, t, j);
        bool lower = (lane & j) == 0;
        if (lower ? o < t : o > t) t = o;
    }
}

// insert key c (unique) into the sorted top list; a key above every entry changes nothing
__device__ __forceinline__ void warp_insert(unsigned long long &t, unsigned long long c) {
    int lane = threadIdx.x & 31;
    unsigned long long p = __shfl_up_sync(FULLMASK, t, 1);
    if (t > c) t = (lane == 0 || p < c) ? c : p;
}

// Merge one batch of candidate keys (one per lane, KNN_KEY_NONE for none; pass: the lane's key
// is below the current k-th key) into the sorted top list t, and update kth (the key held by lane
// kn - 1).  Few passing candidates are inserted one by one (one that no longer beats the list's
// last entry falls off its end); more are sorted and merged.
__device__ __forceinline__ void knn_merge_batch(unsigned long long ck, bool pass, int kn,
                                                unsigned long long &t, unsigned long long &kth) {
    unsigned m = __ballot_sync(FULLMASK, pass);
    if (!m) return;
    if (__popc(m) <= KNN_INSERT_MAX) {
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1u;
            warp_insert(t, __shfl_sync(FULLMASK, ck, src));
        }
    } else if (__shfl_sync(FULLMASK, t, 0) == KNN_KEY_NONE) {
        // first candidates: the sorted batch is the list
        t = pass ? ck : KNN_KEY_NONE;
        warp_sort(t);
    } else {
        warp_merge(t, pass ? ck : KNN_KEY_NONE);
    }
    kth = __shfl_sync(FULLMASK, t, kn - 1);
}

// the table of cell offsets: all of [-KNN_TAB_R, KNN_TAB_R]^3, each entry
// (ox + 4) | (oy + 4) << 4 | (oz + 4) << 8 | dmin << 12, sorted by dmin, then by |o|^2, where
// dmin = sum_a max(|o_a| - 1, 0)^2: a point in the query's cell is at least dmin * cs^2 from
// any point of the cell at offset o (squared quantised units)
#define KNN_TAB_R 3
#define KNN_TAB_N 343
void knn_offset_table(int *out);   // host: fills KNN_TAB_N entries

struct BoxGrid {
    int G, cs;
    long long coff;
    const int *start;
    const int4 *items;
    const int *tab;           // the offset table (device)
};

// Exact kNN with the key width of the box: the searches of one launch that may meet boxes of
// more than 2^22 particles are compiled with 24 index bits, the others with 22
__device__ __forceinline__ bool knn_wide_box(long long box_particles) {
    return box_particles > (1ll << KNN_IB_SMALL);
}

__device__ __forceinline__ int cell_coord(int v, int cs, int G) {
    int c = v / cs;
    return c < G ? c : G - 1;
}

// squared distance from q to the integer box [lo, hi] (inclusive), 0 inside
__device__ __forceinline__ long long box_d2(int qx, int qy, int qz, int lx, int ly, int lz,
                                            int hx, int hy, int hz) {
    long long dx = qx < lx ? lx - qx : (qx > hx ? qx - hx : 0);
    long long dy = qy < ly ? ly - qy : (qy > hy ? qy - hy : 0);
    long long dz = qz < lz ? lz - qz : (qz > hz ? qz - hz : 0);
    return dx * dx + dy * dy + dz * dz;
}

// Item base + lane of the concatenated ranges (lane l owns [rs, rs + rc), starting at position
// excl of the concatenation); out-of-range lanes get index -2.  The lanes whose range starts
// inside this batch publish (item start - position) at that batch position in sdelta (one
// 32-entry array per warp); a lane takes the value of the last start at or before it, else
// `carry`, the value in force at the end of the previous batch (updated here).
__device__ __forceinline__ int4 knn_fetch(const BoxGrid &g, int base, int total, int rs, int rc,
                                          int excl, int *sdelta, int &carry) {
    int lane = threadIdx.x & 31;
    bool st = rc > 0 && excl >= base && excl < base + 32;
    if (st) sdelta[excl - base] = rs - excl;
    unsigned sm = __reduce_or_sync(FULLMASK, st ? 1u << (excl - base) : 0u);
    __syncwarp();
    unsigned below = sm & (0xffffffffu >> (31 - lane));
    int delta = below ? sdelta[31 - __clz(below)] : carry;
    carry = __shfl_sync(FULLMASK, delta, 31);
    __syncwarp();
    int c = base + lane;
    int4 it = make_int4(0, 0, 0, -2);
    if (c < total) it = g.items[c + delta];
    return it;
}

// Merge the candidates of a list of contiguous item ranges, one per lane, into the running
// top list t; kth is the key held by lane kn - 1 (uniform), bkey the largest key allowed.
// The items of the next batch of 32 are loaded before the current batch is merged, so the
// load latency overlaps the merge.
template <int IB>
__device__ inline void knn_visit(const BoxGrid &g, int qx, int qy, int qz, int exclude, int kn,
                                 int rs, int rc, unsigned long long bkey, unsigned long long &t,
                                 unsigned long long &kth, int *sdelta) {
    int lane = threadIdx.x & 31;
    // inclusive scan of range counts
    int incl = rc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += v;
    }
    int total = __shfl_sync(FULLMASK, incl, 31);
    int excl = incl - rc;
    if (total == 0) return;
    int carry = 0;
    int4 nxt = knn_fetch(g, 0, total, rs, rc, excl, sdelta, carry);
    for (int base = 0; base < total; base += 32) {
        int4 it = nxt;
        if (base + 32 < total) nxt = knn_fetch(g, base + 32, total, rs, rc, excl, sdelta, carry);
        unsigned long long ck = KNN_KEY_NONE;
        if (it.w >= 0 && it.w != exclude) {
            long long dx = it.x - qx, dy = it.y - qy, dz = it.z - qz;
            ck = knn_key<IB>(dx * dx + dy * dy + dz * dz, it.w);
        }
        knn_merge_batch(ck, ck < kth && ck <= bkey, kn, t, kth);
    }
}

// Shells of cells at Chebyshev radius r0, r0 + 1, ... around the query's cell, merged into the
// running list t (k-th key kth), until the k-th distance is below the distance from q to the
// outside of the visited block (every cell of radius < r0 has been visited or shown not to
// matter).  r0 = 1 visits the whole 3x3x3 block first.
template <int IB>
__device__ inline void knn_shells(const BoxGrid &g, int qx, int qy, int qz, int exclude, int kn,
                                  int r0, long long bound, unsigned long long bkey,
                                  unsigned long long &t, unsigned long long &kth, int *sdelta) {
    int G = g.G, cs = g.cs;
    int cx = cell_coord(qx, cs, G), cy = cell_coord(qy, cs, G), cz = cell_coord(qz, cs, G);
    for (int r = r0; r <= G; ++r) {
        // the columns (x, y) of the shell at Chebyshev radius r (r = 1: the whole 3x3x3 block)
        int side = 2 * r + 1;
        int ncol = side * side;
        // cells farther than the current k-th distance (or the bound) cannot help
        long long prune = kth == KNN_KEY_NONE ? KNN_INF : (long long)(kth >> IB);
        if (bound < prune) prune = bound;
        for (int cb = 0; cb < ncol; cb += 32) {
            int col = cb + (threadIdx.x & 31);
            // up to two z-ranges per column
            int rs0 = 0, rc0 = 0, rs1 = 0, rc1 = 0;
            if (col < ncol) {
                int ix, iy;
                if (r == 1) {
                    // the 3x3 block: the query's column first, then the four sharing a face
                    // with it, then the corners (near points first make the k-th distance tight
                    // sooner); offsets + 1 packed two bits per column
                    ix = cx - 1 + (int)((0x28251u >> (2 * col)) & 3u);
                    iy = cy - 1 + (int)((0x22185u >> (2 * col)) & 3u);
                } else {
                    ix = cx - r + col / side;
                    iy = cy - r + col % side;
                }
                if (ix >= 0 && iy >= 0 && ix < G && iy < G) {
                    bool edge = (r == 1) || ix == cx - r || ix == cx + r || iy == cy - r ||
                                iy == cy + r;
                    long long colbase = g.coff + ((long long)ix * G + iy) * G;
                    int lx = ix * cs, ly = iy * cs, hx = lx + cs - 1, hy = ly + cs - 1;
                    if (edge) {
                        int z0 = max(cz - r, 0), z1 = min(cz + r, G - 1);
                        if (box_d2(qx, qy, qz, lx, ly, z0 * cs, hx, hy, z1 * cs + cs - 1) <= prune) {
                            rs0 = g.start[colbase + z0];
                            rc0 = g.start[colbase + z1 + 1] - rs0;
                        }
                    } else {
                        int z0 = cz - r, z1 = cz + r;
                        if (z0 >= 0 && box_d2(qx, qy, qz, lx, ly, z0 * cs, hx, hy, z0 * cs + cs - 1) <= prune) {
                            rs0 = g.start[colbase + z0];
                            rc0 = g.start[colbase + z0 + 1] - rs0;
                        }
                        if (z1 < G && box_d2(qx, qy, qz, lx, ly, z1 * cs, hx, hy, z1 * cs + cs - 1) <= prune) {
                            rs1 = g.start[colbase + z1];
                            rc1 = g.start[colbase + z1 + 1] - rs1;
                        }
                    }
                }
            }
            knn_visit<IB>(g, qx, qy, qz, exclude, kn, rs0, rc0, bkey, t, kth, sdelta);
            if (__any_sync(FULLMASK, rc1 > 0))
                knn_visit<IB>(g, qx, qy, qz, exclude, kn, rs1, rc1, bkey, t, kth, sdelta);
        }
        // distance from q to the outside of the visited block [c - r, c + r]^3
        long long b = -1;
        int cc[3] = {cx, cy, cz}, qq[3] = {qx, qy, qz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (cc[a] - r > 0) {
                long long lo = (long long)qq[a] - (long long)(cc[a] - r) * cs;
                if (b < 0 || lo < b) b = lo;
            }
            if (cc[a] + r + 1 < G) {
                long long hi = (long long)(cc[a] + r + 1) * cs - qq[a];
                if (b < 0 || hi < b) b = hi;
            }
        }
        if (b < 0) break;
        if (kth != KNN_KEY_NONE && (long long)(kth >> IB) < b * b) break;
    }
}

// Exact kNN of point q (quantised, inside [0, RT_Q)^3) among the box's points, excluding the
// point with local index `exclude` (-1: none).  Lane l < kn returns the l-th nearest.
// `bound` is an upper bound on the squared distance of the kn-th neighbour (KNN_INF when none
// is known): points and cells beyond it are skipped, which leaves the result unchanged.
// sdelta: 32 ints of shared memory owned by the calling warp.
// Returns false when the box holds fewer than kn candidates, or when the kn-th distance
// saturated the key (the order among the farthest candidates is then not certain).
template <int IB>
__device__ inline bool warp_knn(const BoxGrid &g, int qx, int qy, int qz, int exclude, int kn,
                                long long &out_d2, int &out_idx, int *sdelta,
                                long long bound = KNN_INF) {
    unsigned long long t = KNN_KEY_NONE, kth = KNN_KEY_NONE;
    unsigned long long bkey = bound >= knn_d2max<IB>() ? KNN_KEY_NONE - 1ull
                                                       : knn_key<IB>(bound, (1 << IB) - 1);
    int G = g.G, cs = g.cs;
    int cx = cell_coord(qx, cs, G), cy = cell_coord(qy, cs, G), cz = cell_coord(qz, cs, G);
    const long long cs2 = (long long)cs * cs;
    // cells outside the table are at Chebyshev radius > KNN_TAB_R: dmin >= KNN_TAB_R^2
    const int dout = KNN_TAB_R * KNN_TAB_R;
    bool done = false;
    for (int e0 = 0; e0 < KNN_TAB_N; e0 += 32) {
        // cells farther than the current k-th distance (or the bound) cannot help
        long long lim = kth == KNN_KEY_NONE ? KNN_INF : (long long)(kth >> IB);
        if (bound < lim) lim = bound;
        // the table is sorted by dmin: once the next entry (and every cell outside the table)
        // is beyond the limit, nothing nearer remains
        int dnext = __ldg(g.tab + e0) >> 12;
        if (lim < KNN_INF && (long long)min(dnext, dout) * cs2 > lim) {
            done = true;
            break;
        }
        int rs = 0, rc = 0;
        int k = e0 + (int)(threadIdx.x & 31);
        if (k < KNN_TAB_N) {
            int e = __ldg(g.tab + k);
            int ix = cx + (e & 15) - 4, iy = cy + ((e >> 4) & 15) - 4, iz = cz + ((e >> 8) & 15) - 4;
            if (ix >= 0 && iy >= 0 && iz >= 0 && ix < G && iy < G && iz < G) {
                int lx = ix * cs, ly = iy * cs, lz = iz * cs;
                if (box_d2(qx, qy, qz, lx, ly, lz, lx + cs - 1, ly + cs - 1, lz + cs - 1) <= lim) {
                    long long c = g.coff + ((long long)ix * G + iy) * G + iz;
                    rs = g.start[c];
                    rc = g.start[c + 1] - rs;
                }
            }
        }
        knn_visit<IB>(g, qx, qy, qz, exclude, kn, rs, rc, bkey, t, kth, sdelta);
    }
    if (!done) knn_shells<IB>(g, qx, qy, qz, exclude, kn, KNN_TAB_R + 1, bound, bkey, t, kth, sdelta);
    if (t == KNN_KEY_NONE) {
        out_d2 = KNN_INF;
        out_idx = 0x7fffffff;
    } else {
        out_d2 = (long long)(t >> IB);
        out_idx = (int)(t & ((1ull << IB) - 1ull));
    }
    return kth != KNN_KEY_NONE && (IB == KNN_IB_SMALL || (long long)(kth >> IB) < knn_d2max<IB>());
}

// ---- per-cell candidate lists (the virtual particles' search) ---------------------------------
// Gas particles do not move, so for every cell of a box's grid the particles that can be among
// the kn nearest of some point of the cell are listed once, after the neighbour build.  With
// lo and hi = lo + cs - 1 the cell's corners and U the largest distance from any point of the
// cell to any of the kn nearest particles of the cell's centre point (computed per particle as
// its distance to the farthest corner), every point of the cell has kn particles within U, so
// its kn nearest lie within U of it, and hence within U of the cell: the list holds every
// particle whose distance to the cell is at most U.  Entries are ordered by ring, the distance
// from the centre point m in units of w, rounded down (ring * w <= |p - m|, capped at 255).  A
// query q in the cell takes the list 32 entries at a time; a particle p of ring r is at least
// r * w - |q - m| from q, so once the first entry of a batch has r * w - |q - m| above the
// current k-th distance, no later entry can enter the result, which is the exact kn nearest
// either way.

// ring width of a box's lists: a sixteenth of the cell side
#ifndef CAND_RING_SHIFT
#define CAND_RING_SHIFT 4
#endif
__device__ __forceinline__ int cand_ring_width(int cs) {
    return cs >= (1 << (CAND_RING_SHIFT + 1)) ? cs >> CAND_RING_SHIFT : 1;
}

// the centre point of the cell starting at lo (inside the quantised range)
__device__ __forceinline__ int cand_centre(int lo, int cs) {
    int m = lo + (cs >> 1);
    return m < RT_Q - 1 ? m : RT_Q - 1;
}

// an upper bound on sqrt(x) for 0 <= x < 2^42, from 32-bit operations with upward rounding
__device__ __forceinline__ float sqrt_up(long long x) {
    float hi = __uint2float_rn((unsigned)(x >> 21));           // < 2^21: exact
    float lo = __uint2float_rn((unsigned)(x & 0x1fffffll));    // < 2^21: exact
    return __fsqrt_ru(__fmaf_ru(hi, 2097152.0f, lo));
}

// Exact kNN of q (quantised) from the candidate list [a, e) of its cell: the result and the
// return value are those of warp_knn over the whole box.  items: the box's grid items (an entry's
// low 24 bits index them); w: the box's ring width; rq_up: an upper bound on |q - m|.
template <int IB>
__device__ inline bool cand_knn(const int4 *items, const unsigned *cand, long long a, long long e,
                                int qx, int qy, int qz, float rq_up, int w, int kn,
                                long long &out_d2, int &out_idx) {
    int lane = threadIdx.x & 31;
    unsigned long long t = KNN_KEY_NONE, kth = KNN_KEY_NONE;
    // entries and items of the next batch are loaded before the current batch is merged
    unsigned ent = a + lane < e ? __ldg(cand + a + lane) : 0xffffffffu;
    int4 nxt = make_int4(0, 0, 0, -1);
    if (a + lane < e) nxt = __ldg(items + (ent & 0xffffffu));
    for (long long base = a; base < e; base += 32) {
        unsigned cur = ent;
        int4 it = nxt;
        bool have = base + lane < e;
        if (kth != KNN_KEY_NONE) {
            // the batch's first entry has the smallest ring of what is left
            int r0 = (int)(__shfl_sync(FULLMASK, cur, 0) >> 24);
            float reach = __fadd_ru(sqrt_up((long long)(kth >> IB)), rq_up);
            if (__int2float_rd(r0 * w) > reach) break;
        }
        if (base + 32 + lane < e) {
            ent = __ldg(cand + base + 32 + lane);
            nxt = __ldg(items + (ent & 0xffffffu));
        }
        unsigned long long ck = KNN_KEY_NONE;
        if (have) {
            long long dx = it.x - qx, dy = it.y - qy, dz = it.z - qz;
            ck = knn_key<IB>(dx * dx + dy * dy + dz * dz, it.w);
        }
        knn_merge_batch(ck, ck < kth, kn, t, kth);
    }
    if (t == KNN_KEY_NONE) {
        out_d2 = KNN_INF;
        out_idx = 0x7fffffff;
    } else {
        out_d2 = (long long)(t >> IB);
        out_idx = (int)(t & ((1ull << IB) - 1ull));
    }
    return kth != KNN_KEY_NONE && (IB == KNN_IB_SMALL || (long long)(kth >> IB) < knn_d2max<IB>());
}

// A cell keeps a candidate list when its walk radius (in cells, from U) is at most CAND_R_MAX
// and the list holds at most CAND_MAX entries.  Other cells (deep in a void, where the n_ngb
// nearest lie far away and U takes in a large part of a distant cluster) get an empty list; a
// query there takes the grid walk.  A kept list is never empty: it holds the centre point's
// n_ngb nearest.
#define CAND_R_MAX 8
#define CAND_MAX 4096

// The query of a virtual particle at (qx, qy, qz) in box b: its cell's list, ring width and
// the bound on its distance to the cell's centre point.
struct CandQuery {
    const int4 *items;
    long long a, e;
    int w;
    float rq_up;
};
__device__ __forceinline__ CandQuery cand_query(const Grid &gr, int b, int qx, int qy, int qz) {
    CandQuery Q;
    int G = gr.G[b], cs = gr.cs[b];
    long long coff = gr.coff[b];
    int cx = cell_coord(qx, cs, G), cy = cell_coord(qy, cs, G), cz = cell_coord(qz, cs, G);
    long long cell = coff + ((long long)cx * G + cy) * G + cz;
    Q.a = gr.cand_off[cell];
    Q.e = gr.cand_off[cell + 1];
    Q.items = gr.items + gr.start[coff];
    Q.w = cand_ring_width(cs);
    long long mx = cand_centre(cx * cs, cs) - qx, my = cand_centre(cy * cs, cs) - qy,
              mz = cand_centre(cz * cs, cs) - qz;
    Q.rq_up = sqrt_up(mx * mx + my * my + mz * mz);
    return Q;
}

// the grid description of box b, for the grid walk
__device__ __forceinline__ BoxGrid grid_of_box(const Grid &gr, int b) {
    BoxGrid g;
    g.G = gr.G[b];
    g.cs = gr.cs[b];
    g.coff = gr.coff[b];
    g.start = gr.start;
    g.items = gr.items;
    g.tab = gr.tab;
    return g;
}

struct KnnOut {
    long long d2;
    int idx;
    bool ok;
};

// The grid walk for a query in a cell without a candidate list, kept out of line: it is rare,
// and inlined it would take registers from the common path.  Called by the whole warp.
template <int IB>
__device__ __noinline__ KnnOut knn_walk_query(BoxGrid g, int qx, int qy, int qz, int kn,
                                              int *sdelta) {
    KnnOut o;
    o.ok = warp_knn<IB>(g, qx, qy, qz, -1, kn, o.d2, o.idx, sdelta);
    return o;
}

// The virtual particles' exact kNN of (qx, qy, qz) in box b: from the cell's candidate list,
// or by the grid walk where the cell has none.  Both give warp_knn's result.  sdelta: 32 ints
// of shared memory owned by the calling warp (the grid walk's).
template <int IB>
__device__ __forceinline__ bool vp_knn(const Grid &gr, int b, int qx, int qy, int qz, int kn,
                                       long long &d2, int &idx, int *sdelta) {
    CandQuery Q = cand_query(gr, b, qx, qy, qz);
    if (Q.e > Q.a)
        return cand_knn<IB>(Q.items, gr.cand, Q.a, Q.e, qx, qy, qz, Q.rq_up, Q.w, kn, d2, idx);
    KnnOut o = knn_walk_query<IB>(grid_of_box(gr, b), qx, qy, qz, kn, sdelta);
    d2 = o.d2;
    idx = o.idx;
    return o.ok;
}
