// rt_knn.cuh -- exact k-nearest-neighbour search by one warp over a box's uniform cell list.
//
// The result is the k smallest (squared quantised distance, local index) pairs, a unique set,
// held sorted across the lanes: lane l has the l-th nearest.  The search visits the 3x3x3 block
// of cells around the query, then growing shells of cells (skipping cells that cannot hold a
// point at or below the current k-th distance) until the k-th distance is below the distance
// to the outside of the visited block.
#pragma once
#include "rt_internal.cuh"

#define KNN_INF 0x7fffffffffffffffll

struct KKey {
    long long d2;
    int idx;
};

__device__ __forceinline__ bool kless(long long da, int ia, long long db, int ib) {
    return da < db || (da == db && ia < ib);
}

__device__ __forceinline__ void kshfl(long long &d2, int &idx, int src_lane, long long &od2,
                                      int &oidx) {
    od2 = __shfl_sync(FULLMASK, d2, src_lane);
    oidx = __shfl_sync(FULLMASK, idx, src_lane);
}

// bitonic sort (ascending) of one key per lane across the warp
__device__ __forceinline__ void warp_sort(long long &d2, int &idx) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            long long od2;
            int oidx;
            kshfl(d2, idx, lane ^ j, od2, oidx);
            bool up = ((lane & k) == 0);
            bool lower = (lane & j) == 0;
            bool take_min = (lower == up);
            bool o_less = kless(od2, oidx, d2, idx);
            if (take_min ? o_less : !o_less) { d2 = od2; idx = oidx; }
        }
    }
}

// top (sorted ascending across lanes) <- the 32 smallest of top U batch (batch unsorted)
__device__ __forceinline__ void warp_merge(long long &td2, int &tidx, long long bd2, int bidx) {
    int lane = threadIdx.x & 31;
    warp_sort(bd2, bidx);
    long long rd2;
    int ridx;
    kshfl(bd2, bidx, 31 - lane, rd2, ridx);
    if (kless(rd2, ridx, td2, tidx)) { td2 = rd2; tidx = ridx; }
    // td2 is now bitonic: merge down
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        long long od2;
        int oidx;
        kshfl(td2, tidx, lane ^ j, od2, oidx);
        bool lower = (lane & j) == 0;
        bool o_less = kless(od2, oidx, td2, tidx);
        if (lower ? o_less : !o_less) { td2 = od2; tidx = oidx; }
    }
}

struct BoxGrid {
    int G, cs;
    long long coff;
    const int *start;
    const int4 *items;
};

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

// Visit a list of contiguous item ranges, one per lane (lane l owns [rs, rs + rc)); merge the
// candidates into the running top-k.
__device__ inline void knn_visit(const BoxGrid &g, int qx, int qy, int qz, int exclude, int kn,
                                 int rs, int rc, long long bound, long long &td2, int &tidx) {
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
    for (int base = 0; base < total; base += 32) {
        int c = base + lane;
        // owner lane: the last lane whose exclusive start is <= c
        int lo = 0, hi = 31;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            int mid = (lo + hi + 1) >> 1;
            int em = __shfl_sync(FULLMASK, excl, mid);
            if (em <= c) lo = mid; else hi = mid - 1;
        }
        int o_rs = __shfl_sync(FULLMASK, rs, lo);
        int o_ex = __shfl_sync(FULLMASK, excl, lo);
        long long cd2 = KNN_INF;
        int cidx = 0x7fffffff;
        if (c < total) {
            int4 it = g.items[o_rs + (c - o_ex)];
            if (it.w != exclude) {
                long long dx = it.x - qx, dy = it.y - qy, dz = it.z - qz;
                cd2 = dx * dx + dy * dy + dz * dz;
                cidx = it.w;
            }
        }
        long long kd2 = __shfl_sync(FULLMASK, td2, kn - 1);
        int kidx = __shfl_sync(FULLMASK, tidx, kn - 1);
        bool better = cd2 <= bound && kless(cd2, cidx, kd2, kidx);
        if (__any_sync(FULLMASK, better)) {
            if (!better) { cd2 = KNN_INF; cidx = 0x7fffffff; }
            warp_merge(td2, tidx, cd2, cidx);
        }
    }
}

// Exact kNN of point q (quantised, inside [0, RT_Q)^3) among the box's points, excluding the
// point with local index `exclude` (-1: none).  Lane l < kn returns the l-th nearest.
// `bound` is an upper bound on the squared distance of the kn-th neighbour (KNN_INF when none
// is known): points and cells beyond it are skipped, which leaves the result unchanged.
// Returns false when the box holds fewer than kn candidates.
__device__ inline bool warp_knn(const BoxGrid &g, int qx, int qy, int qz, int exclude, int kn,
                                long long &out_d2, int &out_idx, long long bound = KNN_INF) {
    int lane = threadIdx.x & 31;
    long long td2 = KNN_INF;
    int tidx = 0x7fffffff;
    int G = g.G, cs = g.cs;
    int cx = cell_coord(qx, cs, G), cy = cell_coord(qy, cs, G), cz = cell_coord(qz, cs, G);
    for (int r = 1; r <= G; ++r) {
        // the columns (x, y) of the shell at Chebyshev radius r (r = 1: the whole 3x3x3 block)
        int side = 2 * r + 1;
        int ncol = side * side;
        long long prune = __shfl_sync(FULLMASK, td2, kn - 1);   // cells farther cannot help
        if (bound < prune) prune = bound;
        for (int cb = 0; cb < ncol; cb += 32) {
            int col = cb + lane;
            // up to two z-ranges per column
            int rs0 = 0, rc0 = 0, rs1 = 0, rc1 = 0;
            if (col < ncol) {
                int ix = cx - r + col / side, iy = cy - r + col % side;
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
            knn_visit(g, qx, qy, qz, exclude, kn, rs0, rc0, bound, td2, tidx);
            if (__any_sync(FULLMASK, rc1 > 0))
                knn_visit(g, qx, qy, qz, exclude, kn, rs1, rc1, bound, td2, tidx);
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
        long long kd2 = __shfl_sync(FULLMASK, td2, kn - 1);
        if (b < 0) break;
        if (kd2 != KNN_INF && kd2 < b * b) break;
    }
    out_d2 = td2;
    out_idx = tidx;
    long long kd2 = __shfl_sync(FULLMASK, td2, kn - 1);
    return kd2 != KNN_INF;
}
