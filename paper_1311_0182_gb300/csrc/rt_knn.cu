// rt_knn.cu -- quantisation, per-box cell lists, exact kNN of particles and sources, and the
// receiver-sorted reverse neighbour lists (Sec. 2.1: a packet at particle i is passed to the
// neighbours within i's smoothing volume, the n_ngb nearest particles).
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "rt_knn.cuh"

__global__ void k_quantise(DevPtrs P, const double *x, const double *y, const double *z) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    int lo = 0, hi = P.nb - 1;          // box of particle i: box_off[b] <= i < box_off[b+1]
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.box_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    double L = P.box_L[lo];
    double v[3] = {x[i], y[i], z[i]};
    int q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f = __ddiv_rn(v[a], L);
        f = __dmul_rn(f, (double)RT_Q);
        double fl = floor(f);
        long long qq = (long long)fl;
        if (!(fl >= 0.0)) qq = 0;
        if (qq > RT_Q - 1) qq = RT_Q - 1;
        q[a] = (int)qq;
    }
    P.pbox[i] = lo;
    P.qx[i] = q[0]; P.qy[i] = q[1]; P.qz[i] = q[2];
}

__global__ void k_quantise_src(DevPtrs P, const double *x, const double *y, const double *z) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.ns) return;
    double L = P.box_L[P.sbox[i]];
    double v[3] = {x[i], y[i], z[i]};
    int q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f = __dmul_rn(__ddiv_rn(v[a], L), (double)RT_Q);
        double fl = floor(f);
        long long qq = (long long)fl;
        if (!(fl >= 0.0)) qq = 0;
        if (qq > RT_Q - 1) qq = RT_Q - 1;
        q[a] = (int)qq;
    }
    P.sqx[i] = q[0]; P.sqy[i] = q[1]; P.sqz[i] = q[2];
}

__device__ __forceinline__ long long cell_of_particle(const DevPtrs &P, long long i) {
    int b = P.pbox[i];
    int G = P.grid.G[b], cs = P.grid.cs[b];
    int cx = cell_coord(P.qx[i], cs, G), cy = cell_coord(P.qy[i], cs, G),
        cz = cell_coord(P.qz[i], cs, G);
    return P.grid.coff[b] + ((long long)cx * G + cy) * G + cz;
}

__global__ void k_cell_count(DevPtrs P, int *cnt) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    atomicAdd(&cnt[cell_of_particle(P, i)], 1);
}

__global__ void k_cell_fill(DevPtrs P, int *fill) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    long long c = cell_of_particle(P, i);
    int pos = P.grid.start[c] + atomicAdd(&fill[c], 1);
    int b = P.pbox[i];
    P.grid.items[pos] = make_int4(P.qx[i], P.qy[i], P.qz[i], (int)(i - P.box_off[b]));
}

void knn_offset_table(int *out) {
    struct E { int d, r2, code; };
    std::vector<E> es;
    for (int ox = -KNN_TAB_R; ox <= KNN_TAB_R; ++ox)
        for (int oy = -KNN_TAB_R; oy <= KNN_TAB_R; ++oy)
            for (int oz = -KNN_TAB_R; oz <= KNN_TAB_R; ++oz) {
                int o[3] = {ox, oy, oz}, d = 0;
                for (int a = 0; a < 3; ++a) {
                    int m = std::abs(o[a]) - 1;
                    if (m > 0) d += m * m;
                }
                int code = (ox + 4) | (oy + 4) << 4 | (oz + 4) << 8 | d << 12;
                es.push_back({d, ox * ox + oy * oy + oz * oz, code});
            }
    std::stable_sort(es.begin(), es.end(), [](const E &a, const E &b) {
        return a.d != b.d ? a.d < b.d : a.r2 < b.r2;
    });
    for (int k = 0; k < KNN_TAB_N; ++k) out[k] = es[k].code;
}

__device__ __forceinline__ BoxGrid box_grid(const DevPtrs &P, int b) {
    BoxGrid g;
    g.G = P.grid.G[b];
    g.cs = P.grid.cs[b];
    g.coff = P.grid.coff[b];
    g.start = P.grid.start;
    g.tab = P.grid.tab;
    g.items = P.grid.items;
    return g;
}

// one warp per gas particle (exclude itself) or source
__global__ void __launch_bounds__(256) k_knn(DevPtrs P, int sources) {
    __shared__ int sdelta[8][32];
    int lane = threadIdx.x & 31;
    long long nq = sources ? P.ns : P.n;
    long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = w0; w < nq; w += nw) {
        int b, qx, qy, qz, ex;
        if (sources) {
            b = P.sbox[w]; qx = P.sqx[w]; qy = P.sqy[w]; qz = P.sqz[w]; ex = -1;
        } else {
            b = P.pbox[w]; qx = P.qx[w]; qy = P.qy[w]; qz = P.qz[w];
            ex = (int)(w - P.box_off[b]);
        }
        long long d2;
        int idx;
        bool ok = knn_wide_box(P.box_off[b + 1] - P.box_off[b])
                      ? warp_knn<KNN_IB_LARGE>(box_grid(P, b), qx, qy, qz, ex, P.kn, d2, idx,
                                               sdelta[threadIdx.x >> 5])
                      : warp_knn<KNN_IB_SMALL>(box_grid(P, b), qx, qy, qz, ex, P.kn, d2, idx,
                                               sdelta[threadIdx.x >> 5]);
        if (!ok) {
            if (lane == 0) atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_KNN);
            continue;
        }
        long long g = P.box_off[b] + idx;
        long long kd2 = __shfl_sync(FULLMASK, d2, P.kn - 1);
        if (lane < P.kn) {
            if (sources) {
                P.snbr[w * P.kn + lane] = (int)g;
            } else {
                P.nbr[w * P.kn + lane] = (int)g;
                P.fdx[w * P.kn + lane] = (float)(P.qx[g] - qx);
                P.fdy[w * P.kn + lane] = (float)(P.qy[g] - qy);
                P.fdz[w * P.kn + lane] = (float)(P.qz[g] - qz);
            }
        }
        if (lane == 0) {
            if (sources) P.sh2[w] = kd2; else P.h2[w] = kd2;
        }
    }
}

__global__ void k_rev_count(DevPtrs P, int *cnt) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.n * P.kn) return;
    atomicAdd(&cnt[P.nbr[e]], 1);
}

__global__ void k_rev_fill(DevPtrs P, int *fill) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.n * P.kn) return;
    long long i = e / P.kn;
    int k = (int)(e % P.kn);
    int j = P.nbr[e];
    int pos = P.rev_off[j] + atomicAdd(&fill[j], 1);
    P.rev_ent[pos] = ((unsigned)i << 5) | (unsigned)k;
}

// order each receiver's senders by index (the fill order is arbitrary) and copy the offsets
__global__ void k_rev_sort(DevPtrs P) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n) return;
    int a = P.rev_off[j], b = P.rev_off[j + 1];
    for (int p = a + 1; p < b; ++p) {
        unsigned v = P.rev_ent[p];
        int q = p - 1;
        while (q >= a && P.rev_ent[q] > v) {
            P.rev_ent[q + 1] = P.rev_ent[q];
            --q;
        }
        P.rev_ent[q + 1] = v;
    }
    for (int p = a; p < b; ++p) {
        unsigned v = P.rev_ent[p];
        long long f = (long long)(v >> 5) * P.kn + (v & 31);
        P.revpos[f] = p;
        P.rdx[p] = P.fdx[f];
        P.rdy[p] = P.fdy[f];
        P.rdz[p] = P.fdz[f];
    }
}

// Timing probe of the occupancy search: the kNN search of virtual-particle-like points, one
// per fourth particle, up to 0.44 smoothing lengths from it in a hashed direction, from the
// candidate list of its cell (or the grid walk where it has none) like the virtual particles'
// search.  Writes one word no one reads,
// so that the search is not dropped.
template <bool FB>
__global__ void __launch_bounds__(256) k_knn_probe(DevPtrs P, unsigned long long *sink) {
    __shared__ int sdelta[FB ? 8 : 1][32];
    int lane = threadIdx.x & 31;
    long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (long long w = w0; 4 * w < P.n; w += nw) {
        long long i = 4 * w;
        int b = P.pbox[i];
        long long H = (long long)sqrt((double)P.h2[i]);
        unsigned long long hsh = mix64((unsigned long long)i);
        int o[3];
        for (int a = 0; a < 3; ++a) {
            int u = (int)((hsh >> (16 * a)) & 0xffff) - 32768;       // in [-2^15, 2^15)
            o[a] = (int)((long long)u * (H / 4) / 32768);             // |o| < 0.44 H
        }
        int qx = min(max(P.qx[i] + o[0], 0), RT_Q - 1);
        int qy = min(max(P.qy[i] + o[1], 0), RT_Q - 1);
        int qz = min(max(P.qz[i] + o[2], 0), RT_Q - 1);
        long long d2;
        int idx;
        int *sd = sdelta[FB ? threadIdx.x >> 5 : 0];
        bool wide = knn_wide_box(P.box_off[b + 1] - P.box_off[b]);
        if (FB) {
            if (wide) vp_knn<KNN_IB_LARGE>(P.grid, b, qx, qy, qz, P.kn, d2, idx, sd);
            else vp_knn<KNN_IB_SMALL>(P.grid, b, qx, qy, qz, P.kn, d2, idx, sd);
        } else {
            CandQuery Q = cand_query(P.grid, b, qx, qy, qz);
            if (wide)
                cand_knn<KNN_IB_LARGE>(Q.items, P.grid.cand, Q.a, Q.e, qx, qy, qz, Q.rq_up, Q.w,
                                       P.kn, d2, idx);
            else
                cand_knn<KNN_IB_SMALL>(Q.items, P.grid.cand, Q.a, Q.e, qx, qy, qz, Q.rq_up, Q.w,
                                       P.kn, d2, idx);
        }
        acc += (unsigned long long)idx;
    }
    if (lane == 0 && acc == 0xffffffffffffffffull) *sink = acc;
}

// ---- per-cell candidate lists (rt_knn.cuh) ----------------------------------------------------
// the box and coordinates of global cell index c
__device__ __forceinline__ int cell_box(const DevPtrs &P, long long c) {
    int lo = 0, hi = P.nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.grid.coff[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Chebyshev radius (in cells) of the cells that can hold a particle within sqrt(u2) of a
// cell: a cell at offset o >= 2 is at least (o - 1) cs + 1 from it
__device__ __forceinline__ int cand_radius(long long u2, int cs, int G) {
    if (u2 >= KNN_INF) return G;
    long long u = (long long)sqrt((double)u2) + 1;
    long long r = u / cs + 1;
    return r < G ? (int)r : G;
}

// Calls f(position of the item among the box's items, item) for every particle of box b whose
// squared distance to the cell box [lo, lo + cs - 1]^3 is at most u2 (lane = grid column; a
// column's cells are consecutive, so its candidate cells are one range of items).
template <typename F>
__device__ __forceinline__ void cand_walk(const DevPtrs &P, int b, int cx, int cy, int cz,
                                          long long u2, F f) {
    int lane = threadIdx.x & 31;
    int G = P.grid.G[b], cs = P.grid.cs[b];
    long long coff = P.grid.coff[b];
    int ibase = P.grid.start[coff];
    int R = cand_radius(u2, cs, G);
    int lx = cx * cs, ly = cy * cs, lz = cz * cs;
    int hx = lx + cs - 1, hy = ly + cs - 1, hz = lz + cs - 1;
    int side = 2 * R + 1;
    long long ncol = (long long)side * side;
    int z0 = max(cz - R, 0), z1 = min(cz + R, G - 1);
    for (long long cb = 0; cb < ncol; cb += 32) {
        long long col = cb + lane;
        if (col >= ncol) continue;
        int ix = cx - R + (int)(col / side), iy = cy - R + (int)(col % side);
        if (ix < 0 || iy < 0 || ix >= G || iy >= G) continue;
        long long gx = ix < cx ? lx - (ix * cs + cs - 1) : (ix > cx ? ix * cs - hx : 0);
        long long gy = iy < cy ? ly - (iy * cs + cs - 1) : (iy > cy ? iy * cs - hy : 0);
        if (gx * gx + gy * gy > u2) continue;
        long long colbase = coff + ((long long)ix * G + iy) * G;
        int p0 = P.grid.start[colbase + z0], p1 = P.grid.start[colbase + z1 + 1];
        for (int pos = p0; pos < p1; ++pos) {
            int4 it = P.grid.items[pos];
            if (box_d2(it.x, it.y, it.z, lx, ly, lz, hx, hy, hz) <= u2) f(pos - ibase, it);
        }
    }
}

// one warp per cell: U^2 (the kn nearest of the cell's centre point, each at its distance to
// the farthest corner of the cell) and the number of candidates, 0 for a cell without a list
// (counted in *nfall)
__global__ void __launch_bounds__(256) k_cand_count(DevPtrs P, long long *u2out, int *cnt,
                                                    unsigned long long *nfall) {
    __shared__ int sdelta[8][32];
    int lane = threadIdx.x & 31;
    long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = w0; c < P.grid.ncells; c += nw) {
        int b = cell_box(P, c);
        int G = P.grid.G[b], cs = P.grid.cs[b];
        long long lc = c - P.grid.coff[b];
        int cx = (int)(lc / ((long long)G * G)), cy = (int)((lc / G) % G), cz = (int)(lc % G);
        int lx = cx * cs, ly = cy * cs, lz = cz * cs;
        int mx = cand_centre(lx, cs), my = cand_centre(ly, cs), mz = cand_centre(lz, cs);
        long long d2;
        int idx;
        if (knn_wide_box(P.box_off[b + 1] - P.box_off[b]))
            warp_knn<KNN_IB_LARGE>(box_grid(P, b), mx, my, mz, -1, P.kn, d2, idx,
                                   sdelta[threadIdx.x >> 5]);
        else
            warp_knn<KNN_IB_SMALL>(box_grid(P, b), mx, my, mz, -1, P.kn, d2, idx,
                                   sdelta[threadIdx.x >> 5]);
        // any kn particles bound U, so a search whose keys saturated (a k-th distance beyond
        // their range) still gives one; only a box of fewer than kn particles has none
        bool ok = __all_sync(FULLMASK, lane >= P.kn || idx != 0x7fffffff);
        long long u2 = 0;
        if (ok && lane < P.kn) {
            long long j = P.box_off[b] + idx;
            long long ex = max(P.qx[j] - lx, lx + cs - 1 - P.qx[j]);
            long long ey = max(P.qy[j] - ly, ly + cs - 1 - P.qy[j]);
            long long ez = max(P.qz[j] - lz, lz + cs - 1 - P.qz[j]);
            u2 = ex * ex + ey * ey + ez * ez;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            long long v = __shfl_xor_sync(FULLMASK, u2, o);
            u2 = v > u2 ? v : u2;
        }
        // fewer than kn particles in the box: the whole box
        if (!ok) u2 = KNN_INF;
        int n = 0;
        bool keep = cand_radius(u2, cs, G) <= CAND_R_MAX;   // (always in a box of G <= 8)
        if (keep) {
            cand_walk(P, b, cx, cy, cz, u2, [&](int, const int4 &) { ++n; });
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(FULLMASK, n, o);
            keep = n <= CAND_MAX;
        }
        if (lane == 0) {
            u2out[c] = u2;
            cnt[c] = keep ? n : 0;
            if (!keep) atomicAdd(nfall, 1ull);
        }
    }
}

// one warp per cell: the entries, by ring (a counting sort in shared memory)
__global__ void __launch_bounds__(256) k_cand_fill(DevPtrs P, const long long *u2in) {
    __shared__ int bins[8][256];
    int lane = threadIdx.x & 31;
    int *bin = bins[threadIdx.x >> 5];
    long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = w0; c < P.grid.ncells; c += nw) {
        int b = cell_box(P, c);
        int G = P.grid.G[b], cs = P.grid.cs[b];
        long long lc = c - P.grid.coff[b];
        int cx = (int)(lc / ((long long)G * G)), cy = (int)((lc / G) % G), cz = (int)(lc % G);
        int mx = cand_centre(cx * cs, cs), my = cand_centre(cy * cs, cs), mz = cand_centre(cz * cs, cs);
        int w = cand_ring_width(cs);
        long long u2 = u2in[c];
        long long a = P.grid.cand_off[c], e = P.grid.cand_off[c + 1];
        if (e == a) continue;   // no list: its queries take the grid walk
        auto ring_of = [&](const int4 &it) {
            long long dx = it.x - mx, dy = it.y - my, dz = it.z - mz;
            long long d2 = dx * dx + dy * dy + dz * dz;
            long long r = (long long)(sqrt((double)d2) / (double)w);
            if (r > 255) r = 255;
            while (r > 0 && (r * w) * (r * w) > d2) --r;   // r w <= |p - m|
            return (int)r;
        };
        for (int k = lane; k < 256; k += 32) bin[k] = 0;
        __syncwarp();
        cand_walk(P, b, cx, cy, cz, u2, [&](int, const int4 &it) { atomicAdd(&bin[ring_of(it)], 1); });
        __syncwarp();
        // exclusive scan of the 256 bins: 8 per lane
        int loc[8], s = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) { loc[k] = s; s += bin[lane * 8 + k]; }
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(FULLMASK, incl, o);
            if (lane >= o) incl += v;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; ++k) bin[lane * 8 + k] = incl - s + loc[k];
        __syncwarp();
        bool over = false;
        cand_walk(P, b, cx, cy, cz, u2, [&](int ipos, const int4 &it) {
            int r = ring_of(it);
            long long pos = a + atomicAdd(&bin[r], 1);
            if (pos < e) P.grid.cand[pos] = ((unsigned)r << 24) | (unsigned)ipos;
            else over = true;
        });
        if (over) atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_KNN);
        __syncwarp();
    }
}

static void cell_lists(rt_ctx *c, cudaStream_t st) {
    DevPtrs &P = c->d;
    int tb = 256;
    unsigned nbk = (unsigned)((P.n + tb - 1) / tb);
    int *cnt = P.seg_cnt, *fill = P.seg_fill;   // scratch, sized >= max(ncells, n)
    cudaMemsetAsync(cnt, 0, sizeof(int) * (P.grid.ncells + 1), st);
    cudaMemsetAsync(fill, 0, sizeof(int) * (P.grid.ncells + 1), st);
    k_cell_count<<<nbk, tb, 0, st>>>(P, cnt);
    rt_scan_exclusive(c, cnt, P.grid.start, P.grid.ncells + 1, nullptr, nullptr, st);
    k_cell_fill<<<nbk, tb, 0, st>>>(P, fill);
}

// The candidate lists of the current grid: counts and U^2 per cell, 64-bit offsets, storage
// (grown when needed), entries.  Setup work: it synchronises the stream to size the storage.
static rt_status cand_lists(rt_ctx *c, cudaStream_t st) {
    DevPtrs &P = c->d;
    long long nc = P.grid.ncells;
    int tb = 256;
    int *cnt = P.seg_cnt;   // scratch, sized >= ncells + 1
    long long *tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof(long long) * (size_t)(nc + RT_SCAN_NB + 1));
    if (e != cudaSuccess) return rt_cuda_check(c, e, "candidate lists");
    long long *u2 = tmp + RT_SCAN_NB;
    unsigned long long *nfall = (unsigned long long *)(tmp + RT_SCAN_NB + nc);
    cudaMemsetAsync(cnt + nc, 0, sizeof(int), st);
    cudaMemsetAsync(nfall, 0, sizeof(unsigned long long), st);
    k_cand_count<<<rt_blocks(nc * 32, tb, 152 * 64), tb, 0, st>>>(P, u2, cnt, nfall);
    rt_scan_exclusive64(cnt, P.grid.cand_off, nc + 1, tmp, st);
    long long total = 0, fall = 0;
    cudaMemcpyAsync(&total, P.grid.cand_off + nc, sizeof(long long), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&fall, nfall, sizeof(long long), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && total > P.grid.cand_cap) {
        if (P.grid.cand) cudaFree(P.grid.cand);
        P.grid.cand = nullptr;
        P.grid.cand_cap = 0;
        e = cudaMalloc(&P.grid.cand, sizeof(unsigned) * (size_t)(total > 0 ? total : 1));
        if (e == cudaSuccess) P.grid.cand_cap = total;
        else P.grid.cand = nullptr;
    }
    if (e == cudaSuccess)
        k_cand_fill<<<rt_blocks(nc * 32, tb, 152 * 64), tb, 0, st>>>(P, u2);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(tmp);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGetLastError();
    c->cand_entries = total;
    c->cand_fallback = fall;
    return rt_cuda_check(c, e, "candidate lists");
}

// The occupancy of the kNN cell grids (the cells whose candidate lists the virtual particles'
// search takes) is picked on the particle set itself: after the first neighbour build, the
// search of points placed like virtual particles (the hot use of the grids) is timed on each
// candidate grid, with its candidate lists, and the fastest wins.  Done once per context; any
// grid gives the same exact neighbours, so only the time depends on the choice.
static rt_status tune_grid(rt_ctx *c, cudaStream_t st) {
    static const int cand[] = {1, 2, 3, 4, 6};
    DevPtrs &P = c->d;
    int tb = 256;
    // rt_set_grid rewrites the grid description with plain copies, which do not wait for
    // kernels on the caller's (possibly non-blocking) stream: let the neighbour build finish
    cudaStreamSynchronize(st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 0.f;
    int best = c->cell_occ;
    rt_status s = RT_OK;
    for (int occ : cand) {
        rt_set_grid(c, occ);
        cell_lists(c, st);
        if ((s = cand_lists(c, st)) != RT_OK) break;
        cudaEventRecord(e0, st);
        // the probe takes the instance the virtual particles will (with the grid-walk
        // fallback only when some cell has no list)
        unsigned long long *sink = (unsigned long long *)&P.cnt[CNT_N - 1];   // an unused counter
        int pb = rt_blocks((P.n / 4 + 1) * 32, tb, 152 * 64);
        if (c->cand_fallback > 0) k_knn_probe<true><<<pb, tb, 0, st>>>(P, sink);
        else k_knn_probe<false><<<pb, tb, 0, st>>>(P, sink);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (occ == cand[0] || ms < best_ms) { best_ms = ms; best = occ; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != RT_OK) return s;
    rt_set_grid(c, best);
    cell_lists(c, st);
    if ((s = cand_lists(c, st)) != RT_OK) return s;
    c->grid_tuned = true;
    return RT_OK;
}

rt_status rt_knn_build(rt_ctx *c, cudaStream_t st) {
    DevPtrs &P = c->d;
    long long n = P.n;
    int tb = 256;
    unsigned nbk = (unsigned)((n + tb - 1) / tb);
    int *cnt = P.seg_cnt, *fill = P.seg_fill;
    // cell lists
    cell_lists(c, st);
    // neighbours of particles and sources
    k_knn<<<rt_blocks(n * 32, tb, 152 * 64), tb, 0, st>>>(P, 0);
    if (P.ns > 0) k_knn<<<rt_blocks((long long)P.ns * 32, tb), tb, 0, st>>>(P, 1);
    // reverse lists
    cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), st);
    cudaMemsetAsync(fill, 0, sizeof(int) * (n + 1), st);
    long long ne = n * P.kn;
    unsigned nbe = (unsigned)((ne + tb - 1) / tb);
    k_rev_count<<<nbe, tb, 0, st>>>(P, cnt);
    rt_scan_exclusive(c, cnt, P.rev_off, n + 1, nullptr, nullptr, st);
    k_rev_fill<<<nbe, tb, 0, st>>>(P, fill);
    k_rev_sort<<<nbk, tb, 0, st>>>(P);
    rt_status s = rt_cuda_check(c, cudaGetLastError(), "neighbour build");
    if (s != RT_OK) return s;
    // the virtual particles' candidate lists, on the grid the occupancy search picks (it needs
    // the smoothing lengths just computed)
    s = c->grid_tuned ? cand_lists(c, st) : tune_grid(c, st);
    // the step graph holds the grid description by value
    rt_graph_destroy(c);
    return s;
}

// rt_query_neighbours: one warp per point; fail bit 1: a coordinate out of range, bit 2: a
// failed search
__global__ void __launch_bounds__(256) k_query(DevPtrs P, int b, long long m, const int *q,
                                               int *nbr, long long *d2out, int *fail) {
    __shared__ int sdelta[8][32];
    int lane = threadIdx.x & 31;
    long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    bool wide = knn_wide_box(P.box_off[b + 1] - P.box_off[b]);
    for (long long w = w0; w < m; w += nw) {
        int qx = q[3 * w], qy = q[3 * w + 1], qz = q[3 * w + 2];
        bool ok = qx >= 0 && qy >= 0 && qz >= 0 && qx < RT_Q && qy < RT_Q && qz < RT_Q;
        if (!ok && lane == 0) atomicOr(fail, 1);
        long long d2 = -1;
        int idx = 0;
        if (ok) {
            int *sd = sdelta[threadIdx.x >> 5];
            ok = wide ? vp_knn<KNN_IB_LARGE>(P.grid, b, qx, qy, qz, P.kn, d2, idx, sd)
                      : vp_knn<KNN_IB_SMALL>(P.grid, b, qx, qy, qz, P.kn, d2, idx, sd);
            if (!ok && lane == 0) atomicOr(fail, 2);
        }
        if (lane < P.kn) {
            if (nbr) nbr[w * P.kn + lane] = ok ? (int)(P.box_off[b] + idx) : -1;
            if (d2out) d2out[w * P.kn + lane] = ok ? d2 : -1;
        }
    }
}

void rt_launch_query(rt_ctx *c, int b, long long m, const int *q, int *nbr, long long *d2,
                     int *fail, cudaStream_t st) {
    if (m > 0) k_query<<<rt_blocks(m * 32, 256, 152 * 64), 256, 0, st>>>(c->d, b, m, q, nbr, d2, fail);
}

// launchers used by the API for particle/source upload
void rt_launch_quantise(rt_ctx *c, const double *x, const double *y, const double *z,
                        cudaStream_t st) {
    long long n = c->d.n;
    k_quantise<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->d, x, y, z);
}

void rt_launch_quantise_src(rt_ctx *c, const double *x, const double *y, const double *z,
                            cudaStream_t st) {
    if (c->d.ns > 0) k_quantise_src<<<(c->d.ns + 255) / 256, 256, 0, st>>>(c->d, x, y, z);
}
