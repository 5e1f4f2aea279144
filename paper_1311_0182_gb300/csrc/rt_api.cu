// rt_api.cu -- the C ABI declared in include/traphic_rt.h: context life cycle, uploads, the
// step sequence, and inspection hooks.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "rt_knn.cuh"

rt_status rt_fail(rt_ctx *c, rt_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

rt_status rt_cuda_check(rt_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return RT_OK;
    return rt_fail(c, RT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Isotropic cone direction sets (reading of Sec. 2.1): 8 = cube diagonals; 32 = the 12
// icosahedron vertices followed by the 20 dodecahedron vertices.
void rt_host_axis_set(int n, double *out) {
    if (n == 8) {
        double r = 1.0 / sqrt(3.0);
        for (int b = 0; b < 8; ++b) {
            out[3 * b + 0] = (b & 4) ? -r : r;
            out[3 * b + 1] = (b & 2) ? -r : r;
            out[3 * b + 2] = (b & 1) ? -r : r;
        }
        return;
    }
    double phi = (1.0 + sqrt(5.0)) / 2.0;
    double a = 1.0 / sqrt(1.0 + phi * phi);
    double pa = phi * a;
    double r = 1.0 / sqrt(3.0);
    double ir = (1.0 / phi) * r, pr = phi * r;
    int v = 0;
    // (0, +-1, +-phi) and its cyclic permutations, normalised
    for (int g = 0; g < 3; ++g)
        for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2) {
                double A = s1 ? -a : a, B = s2 ? -pa : pa;
                double e[3] = {0.0, 0.0, 0.0};
                if (g == 0) { e[1] = A; e[2] = B; }
                else if (g == 1) { e[0] = A; e[1] = B; }
                else { e[0] = B; e[2] = A; }
                out[3 * v] = e[0]; out[3 * v + 1] = e[1]; out[3 * v + 2] = e[2];
                ++v;
            }
    for (int b = 0; b < 8; ++b) {
        out[3 * v + 0] = (b & 4) ? -r : r;
        out[3 * v + 1] = (b & 2) ? -r : r;
        out[3 * v + 2] = (b & 1) ? -r : r;
        ++v;
    }
    // (0, +-1/phi, +-phi) and its cyclic permutations, normalised by 1/sqrt(3)
    for (int g = 0; g < 3; ++g)
        for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2) {
                double A = s1 ? -ir : ir, B = s2 ? -pr : pr;
                double e[3] = {0.0, 0.0, 0.0};
                if (g == 0) { e[1] = A; e[2] = B; }
                else if (g == 1) { e[0] = A; e[1] = B; }
                else { e[0] = B; e[2] = A; }
                out[3 * v] = e[0]; out[3 * v + 1] = e[1]; out[3 * v + 2] = e[2];
                ++v;
            }
}

static cudaEvent_t ev_take(rt_ctx *c) {
    if (c->ev_next == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_next++];
}

void kt_begin(rt_ctx *c, int id, cudaStream_t st) {
    if (c->capturing || !((c->prof >> id) & 1)) return;
    cudaEvent_t e0 = ev_take(c), e1 = ev_take(c);
    cudaEventRecord(e0, st);
    c->ev_pending.push_back({id, {e0, e1}});
}

void kt_end(rt_ctx *c, int id, cudaStream_t st, int nlaunch) {
    if (c->capturing) {   // counted per step (and per hop) when the graph runs
        (c->in_hop_body ? c->graph_launch_hop : c->graph_launch_step)[id] += nlaunch;
        return;
    }
    c->launches += nlaunch;
    c->kstat[id].launches += nlaunch;
    if (!((c->prof >> id) & 1)) return;
    cudaEventRecord(c->ev_pending.back().second.second, st);
}

void kt_resolve(rt_ctx *c) {
    for (auto &p : c->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess)
            c->kstat[p.first].ms += ms;
    }
    c->ev_pending.clear();
    c->ev_next = 0;
}

static const char *KT_NAMES[KT_N] = {
    "rotate", "rebin", "emit_rec", "emit_src", "phase_a_send", "free_a_send", "scan",
    "expand_requests", "free_c_stage", "virtual_particles", "seg_fill", "seg_sort",
    "phase_b_merge", "hop_counts", "hop_lens", "drop_free", "chemistry", "budget", "knn_build",
    "worklist", "cone_masks"};

extern "C" rt_status rt_set_graph(rt_ctx *c, int on) {
    if (!c) return RT_ERR_INVALID;
    c->use_graph = on != 0;
    return RT_OK;
}

extern "C" rt_status rt_set_profiling(rt_ctx *c, int on) {
    if (!c) return RT_ERR_INVALID;
    cudaDeviceSynchronize();
    kt_resolve(c);
    c->prof = (unsigned)on & ((1u << KT_N) - 1u);
    for (int k = 0; k < KT_N; ++k) c->kstat[k] = KStat();
    return RT_OK;
}

extern "C" rt_status rt_get_profile(rt_ctx *c, long long *launches_total, int max_kernels,
                                    const char **names, long long *launches, double *ms,
                                    double *bytes) {
    if (!c) return RT_ERR_INVALID;
    cudaDeviceSynchronize();
    kt_resolve(c);
    if (launches_total) *launches_total = c->launches;
    for (int k = 0; k < KT_N && k < max_kernels; ++k) {
        if (names) names[k] = KT_NAMES[k];
        if (launches) launches[k] = c->kstat[k].launches;
        if (ms) ms[k] = c->kstat[k].ms;
        if (bytes) bytes[k] = c->kstat[k].bytes;
    }
    return RT_OK;
}

static void *dalloc(rt_ctx *c, size_t bytes, bool *ok) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        *ok = false;
        return nullptr;
    }
    cudaMemset(p, 0, bytes);
    c->allocs.push_back(p);
    return p;
}

void rt_launch_quantise(rt_ctx *c, const double *x, const double *y, const double *z,
                        cudaStream_t st);
void rt_launch_quantise_src(rt_ctx *c, const double *x, const double *y, const double *z,
                            cudaStream_t st);

extern "C" rt_status rt_axis_set(int n, double *out) {
    if (!out || (n != 8 && n != 32)) return RT_ERR_INVALID;
    rt_host_axis_set(n, out);
    return RT_OK;
}

// cells per box side for a target occupancy
static int grid_side(long long nb, int occupancy) {
    int g = (int)cbrt((double)nb / (double)occupancy);
    return std::max(1, std::min(g, 512));
}

void rt_set_grid(rt_ctx *c, int occupancy) {
    DevPtrs &P = c->d;
    int nb = P.nb;
    std::vector<int> G(nb), cs(nb);
    std::vector<long long> coff(nb);
    long long ncell = 0;
    for (int b = 0; b < nb; ++b) {
        int g = grid_side(c->box_off_h[b + 1] - c->box_off_h[b], occupancy);
        G[b] = g;
        cs[b] = (int)((RT_Q + g - 1) / g);
        coff[b] = ncell;
        ncell += (long long)g * g * g;
    }
    P.grid.ncells = ncell;   // <= grid_cap: occupancy >= the smallest one allocated for
    c->gridG_h = G;
    c->cell_occ = occupancy;
    cudaMemcpy(P.grid.G, G.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    cudaMemcpy(P.grid.cs, cs.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    cudaMemcpy(P.grid.coff, coff.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice);
}

extern "C" rt_status rt_create(const rt_config *cfg, int n_boxes, const long long *box_off,
                               const double *box_L, int n_src, rt_ctx **out) {
    if (!out) return RT_ERR_INVALID;
    *out = nullptr;
    if (!cfg || n_boxes < 1 || !box_off || !box_L || n_src < 0) return RT_ERR_INVALID;
    if (cfg->n_ngb < 1 || cfg->n_ngb > RT_MAXK || cfg->n_tc < 2 || cfg->n_freq_src < 0 ||
        (cfg->n_rc != 8 && cfg->n_rc != 32) || (cfg->n_ec != 8 && cfg->n_ec != 32) ||
        !(cfg->dt > 0.0) || !(cfg->dt_em > 0.0) || cfg->hop_cap < 1 || cfg->sub_cap < 1 ||
        cfg->rec_mode < 0 || cfg->rec_mode > 3 || cfg->rec_shared_bin < 0 ||
        cfg->rec_shared_bin > 1 || (cfg->rec_shared_bin && cfg->n_freq_src < 1) ||
        cfg->launch_grid[0] < 0 || cfg->launch_grid[1] < 0 || cfg->launch_grid[2] < 0 ||
        cfg->cell_occupancy < 0)
        return RT_ERR_INVALID;
    if (box_off[0] != 0) return RT_ERR_INVALID;
    for (int b = 0; b < n_boxes; ++b) {
        if (box_off[b + 1] < box_off[b] + cfg->n_ngb + 1) return RT_ERR_KNN;
        // the kNN search packs a box-local index into 22 bits
        if (box_off[b + 1] - box_off[b] > (1ll << 24)) return RT_ERR_INVALID;
        if (!(box_L[b] > 0.0)) return RT_ERR_INVALID;
    }
    long long n = box_off[n_boxes];
    // particle indices < 2^27 (packed with the neighbour rank), and slot codes and (particle,
    // frequency) keys < 2^31 (32-bit index arithmetic in the kernels)
    long long n_slots = n * (long long)(cfg->n_freq_src + 1) * cfg->n_rc;
    if (n >= (1ll << 27) || n * cfg->n_ngb >= (1ll << 31) || n_slots >= (1ll << 31))
        return RT_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RT_ERR_CUDA;

    rt_ctx *c = new rt_ctx();
    c->cfg = *cfg;
    rt_ctx *x = c;
    DevPtrs &P = c->d;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.nb = n_boxes;
    P.ns = n_src;
    P.nfs = cfg->n_freq_src;
    P.shared = cfg->rec_shared_bin;
    for (int b = 0; b < n_boxes; ++b)
        if (box_off[b + 1] - box_off[b] > (1ll << 22)) P.kwide = 1;
    P.nf = cfg->n_freq_src + (P.shared ? 0 : 1);
    P.rbin = P.shared ? 0 : P.nf - 1;
    P.nrc = cfg->n_rc;
    P.nec = cfg->n_ec;
    P.ntc = cfg->n_tc;
    P.kn = cfg->n_ngb;
    P.S = P.nf * P.nrc;
    long long K = llround(cfg->dt / cfg->dt_em);
    P.K = K < 1 ? 1 : (int)K;
    P.fp32 = cfg->transport_fp32 ? 1 : 0;
    P.dt = cfg->dt;
    P.dt_em = cfg->dt_em;
    P.sigma_rec = cfg->sigma_rec;
    P.T_floor = cfg->T_floor;
    P.eps_rr_fixed = cfg->eps_rr_fixed;
    P.eunit = P.fp32 ? 1.602176634e-12 : 1.0;
    P.sunit = P.fp32 ? 1e-18 : 1.0;
    P.rec_mode = cfg->rec_mode;
    P.evolve_T = cfg->evolve_T;
    P.sub_cap = cfg->sub_cap;
    P.cool_flags = cfg->cool_flags;
    P.seed = cfg->seed;
    long long np_src = (long long)n_src * P.K * P.nfs * P.nec;
    // the original recombination implementation adds K * n_ec packets per particle
    if (cfg->rec_mode == RT_REC_EMISSION_CONES) np_src += n * P.K * P.nec;
    long long fc = cfg->free_cap > 0 ? cfg->free_cap : std::max<long long>(65536, n * P.nrc / 2);
    fc = std::max(fc, np_src);
    P.F_cap = fc;
    long long mem_per = std::max<long long>(4, 2 * ((P.kn + P.ntc - 1) / P.ntc) + 2);
    P.ST_cap = std::max<long long>(fc * mem_per, np_src * P.kn);
    if (P.F_cap >= (1ll << 30) || P.ST_cap >= (1ll << 31)) {
        delete c;
        return RT_ERR_INVALID;
    }
    c->box_off_h.assign(box_off, box_off + n_boxes + 1);
    c->box_L_h.assign(box_L, box_L + n_boxes);
    P.ax_rc = P.nrc == 8 ? 0 : 1;
    P.ax_ec = P.nec == 8 ? 0 : 1;
    rt_upload_axes();

    bool ok = true;
    size_t R = P.fp32 ? 4 : 8;
    long long nkey = n * P.nf, nslot = n * P.S;
    // per-box grids: storage for the finest grid that can be chosen
    if (cfg->cell_occupancy < 0) {
        delete c;
        return RT_ERR_INVALID;
    }
    c->cell_occ = cfg->cell_occupancy > 0 ? cfg->cell_occupancy : 9;
    // launch sizes of the hop kernels given by the caller: no tuning
    for (int k = 0; k < 3; ++k) {
        c->grid_hop[k] = cfg->launch_grid[k];
        if (cfg->launch_grid[k] > 0) c->launch_tuned = true;
    }
    c->grid_tuned = cfg->cell_occupancy > 0;
    long long ncell = 0;
    for (int b = 0; b < n_boxes; ++b) {
        long long nb = box_off[b + 1] - box_off[b];
        int gmax = grid_side(nb, cfg->cell_occupancy > 0 ? cfg->cell_occupancy : RT_OCC_MIN);
        ncell += (long long)gmax * gmax * gmax;
    }
#define A(ptr, T, cnt) ptr = (T *)dalloc(c, sizeof(T) * (size_t)(cnt), &ok)
    A(P.box_off, long long, n_boxes + 1);
    A(P.box_L, double, n_boxes);
    A(P.box_u, double, n_boxes);
    A(P.norm, double, n_boxes);
    A(P.ref, double, n_boxes);
    A(P.vunit, double, n_boxes);
    A(P.esc_fx, unsigned long long, n_boxes);
    A(P.tally, double, 4 * n_boxes);
    // budget chunks: each box cut into ranges of at most RT_BUDGET_CHUNK particles
    std::vector<int> box_bch(n_boxes + 1, 0);
    std::vector<long long> bch_lo;
    for (int b = 0; b < n_boxes; ++b) {
        box_bch[b] = (int)bch_lo.size();
        for (long long i = box_off[b]; i < box_off[b + 1]; i += RT_BUDGET_CHUNK) bch_lo.push_back(i);
    }
    box_bch[n_boxes] = (int)bch_lo.size();
    P.nbch = (int)bch_lo.size();
    bch_lo.push_back(n);
    A(P.box_bch, int, n_boxes + 1);
    A(P.bch_lo, long long, P.nbch + 1);
    A(P.bpart, double, 2 * (long long)P.nbch);
    A(x->src_emit, double, n_boxes);
    A(P.pbox, int, n);
    A(P.qx, int, n); A(P.qy, int, n); A(P.qz, int, n);
    A(P.nH, double, n); A(P.NH, double, n); A(P.xHI, double, n); A(P.T, double, n);
    A(P.Nrec, double, n); A(P.epsrec, double, n); A(P.nHI, double, n); A(P.phot, double, n);
    P.nHIr = dalloc(c, R * n, &ok);
    P.Vr = dalloc(c, R * n, &ok);
    P.dep_s = dalloc(c, R * n, &ok);
    P.depE_s = dalloc(c, R * n, &ok);
    A(P.sbox, int, n_src + 1);
    A(P.gid0, long long, n_boxes);
    A(P.sid, long long, n_src + 1);
    A(P.sqx, int, n_src + 1); A(P.sqy, int, n_src + 1); A(P.sqz, int, n_src + 1);
    A(P.ndot, double, (long long)n_src * P.nfs + 1);
    A(P.sigma, double, P.nfs + 1);
    A(P.eps, double, P.nfs + 1);
    A(P.sigmaf, float, P.nfs + 1);
    A(P.box_uf, float, n_boxes);
    A(P.escf, float, n_boxes);
    A(P.nbr, int, n * P.kn);
    A(P.snbr, int, (long long)(n_src + 1) * P.kn);
    A(P.h2, long long, n);
    A(P.sh2, long long, n_src + 1);
    A(P.sdir, double, 3 * (long long)n_src + 3);
    A(P.sgate, int, n_src + 1);
    A(P.bar, Barrier, n_boxes);
    A(P.fdx, float, n * P.kn); A(P.fdy, float, n * P.kn); A(P.fdz, float, n * P.kn);
    A(P.rev_off, int, n + 1);
    A(P.rev_ent, unsigned, n * P.kn);
    A(P.rdx, float, n * P.kn); A(P.rdy, float, n * P.kn); A(P.rdz, float, n * P.kn);
    A(P.grid.G, int, n_boxes);
    A(P.grid.cs, int, n_boxes);
    A(P.grid.coff, long long, n_boxes);
    A(P.grid.start, int, ncell + 1);
    A(P.grid.cand_off, long long, ncell + 1);
    P.grid.cand = nullptr;       // sized and filled by the neighbour build
    P.grid.cand_cap = 0;
    c->grid_cap = ncell;
    A(P.grid.items, int4, n);
    A(P.grid.tab, int, KNN_TAB_N);
    A(P.R, double, 9 * n);
    A(P.Rf, float, 9 * n);
    A(P.Rs, double, 9 * ((long long)n_src * P.K + 1));
    for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < 6; ++f) P.sl[b][f] = dalloc(c, R * nslot, &ok);
        if (P.shared) P.slG[b] = dalloc(c, R * n * P.nrc, &ok);
        A(P.occ[b], unsigned, nkey);
        A(P.act[b], unsigned, nkey);
    }
    P.rec = dalloc(c, 8 * R * nslot, &ok);
    A(P.bm, unsigned, n * P.kn * P.nf);
    A(P.revpos, int, n * P.kn);
    A(P.worklist, int, nkey);
    A(P.emp, unsigned, nkey);
    A(P.touched, int, nkey);
    A(P.reqcnt, int, n + fc);
    A(P.reqoff, int, n + fc);
    A(P.req, unsigned long long, fc);
    for (int b = 0; b < 2; ++b) {
        FreeBuf &F = P.fr[b];
        A(F.box, int, fc); A(F.qx, int, fc); A(F.qy, int, fc); A(F.qz, int, fc);
        A(F.nu, int, fc);
        A(F.nbr, int, fc * P.kn);
        A(F.h2, long long, fc);
        A(F.fid, unsigned long long, fc);
        F.N = dalloc(c, R * fc, &ok); F.dx = dalloc(c, R * fc, &ok);
        F.dy = dalloc(c, R * fc, &ok); F.dz = dalloc(c, R * fc, &ok);
        F.clock = dalloc(c, R * fc, &ok); F.eps = dalloc(c, R * fc, &ok);
        if (P.shared) F.sig = dalloc(c, R * fc, &ok);
    }
    A(P.st_key, int, P.ST_cap);
    A(P.st_bin, int, P.ST_cap);
    for (int f = 0; f < 9; ++f) P.st_v[f] = dalloc(c, R * P.ST_cap, &ok);
    if (P.shared) P.st_v[9] = dalloc(c, R * P.ST_cap, &ok);
    long long segn = std::max<long long>(nkey, ncell) + 1;
    A(P.seg_cnt, int, segn);
    A(P.seg_off, int, segn);
    A(P.seg_fill, int, segn);
    A(P.seg_idx, int, P.ST_cap);
    A(P.abs, double, nkey); A(P.absE, double, nkey); A(P.pass, double, nkey);
    A(P.passf, float, nkey);
    A(P.fx_abs, unsigned long long, nkey);
    A(P.fx_E, unsigned long long, nkey);
    A(P.fx_lo, unsigned long long, nkey);
    A(P.cnt, long long, CNT_N);
    A(x->hop.lens, int, 8);
    A(x->hop.fmask, unsigned, fc);
    A(x->hop.stcnt, int, fc);
    A(x->hop.stoff, int, fc);
    A(x->hop.esc_r, unsigned long long, fc);
    A(x->hop.vstat, unsigned char, fc);
#undef A
    // the scan scratch: one partial sum per block of a scan (no allocation later)
    c->scan_tmp_n = RT_SCAN_NB;
    if (cudaMalloc(&c->scan_tmp, sizeof(int) * c->scan_tmp_n) != cudaSuccess) ok = false;
    if (cudaMalloc(&c->scan_tmp2, sizeof(int) * c->scan_tmp_n) != cudaSuccess) ok = false;
    if (cudaMallocHost(&c->cnt_h, sizeof(long long) * CNT_N) != cudaSuccess) ok = false;
    // the hop loop's second stream, at the highest priority: its receiver-side kernels take
    // SM slots ahead of the virtual-particle kernel that runs beside them
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&c->st2, cudaStreamNonBlocking, prio_hi) != cudaSuccess)
        ok = false;
    for (int k = 0; k < 4; ++k)
        if (cudaEventCreateWithFlags(&c->hev[k], cudaEventDisableTiming) != cudaSuccess) ok = false;
    for (int k = 0; k < 6; ++k)
        if (k < 2 && cudaEventCreate(&c->tune_ev[k]) != cudaSuccess) ok = false;
    // the stream the step graph is captured on (it never runs work itself)
    if (cudaStreamCreateWithFlags(&c->st_cap, cudaStreamNonBlocking) != cudaSuccess) ok = false;
    if (!ok) {
        rt_destroy(c);
        return RT_ERR_OOM;
    }
    std::vector<double> u(n_boxes);
    for (int b = 0; b < n_boxes; ++b) u[b] = box_L[b] / (double)RT_Q;
    cudaMemcpy(P.box_off, box_off, sizeof(long long) * (n_boxes + 1), cudaMemcpyHostToDevice);
    {
        int tab[KNN_TAB_N];
        knn_offset_table(tab);
        cudaMemcpy(P.grid.tab, tab, sizeof(tab), cudaMemcpyHostToDevice);
    }
    cudaMemcpy(P.box_bch, box_bch.data(), sizeof(int) * (n_boxes + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(P.bch_lo, bch_lo.data(), sizeof(long long) * (P.nbch + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(P.box_L, box_L, sizeof(double) * n_boxes, cudaMemcpyHostToDevice);
    cudaMemcpy(P.box_u, u.data(), sizeof(double) * n_boxes, cudaMemcpyHostToDevice);
    std::vector<float> uf(u.begin(), u.end());
    cudaMemcpy(P.box_uf, uf.data(), sizeof(float) * n_boxes, cudaMemcpyHostToDevice);
    // unit of particle volumes N_H/n_H: the mean particle volume on the FP32 path (volumes in
    // cm^3 exceed the FP32 range), 1 on the FP64 path
    std::vector<double> vu(n_boxes, 1.0);
    if (P.fp32)
        for (int b = 0; b < n_boxes; ++b)
            vu[b] = box_L[b] * box_L[b] * box_L[b] / (double)(box_off[b + 1] - box_off[b]);
    cudaMemcpy(P.vunit, vu.data(), sizeof(double) * n_boxes, cudaMemcpyHostToDevice);
    rt_set_grid(c, c->cell_occ);
    {
        std::vector<Barrier> nob(n_boxes, Barrier{-1, 0, 0, 0, 0});
        cudaMemcpy(P.bar, nob.data(), sizeof(Barrier) * n_boxes, cudaMemcpyHostToDevice);
        c->bar_h = nob;
    }
    x->src_emit_h.assign(n_boxes, 0.0);
    x->box_NH_h.assign(n_boxes, 0.0);
    if (rt_set_identities(c, nullptr, nullptr) != RT_OK) {
        rt_destroy(c);
        return RT_ERR_CUDA;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rt_destroy(c);
        return RT_ERR_CUDA;
    }
    *out = c;
    return RT_OK;
}

extern "C" rt_status rt_destroy(rt_ctx *c) {
    if (!c) return RT_OK;
    cudaDeviceSynchronize();
    rt_graph_destroy(c);
    if (c->st_cap) cudaStreamDestroy(c->st_cap);
    for (size_t k = 0; k < c->allocs.size(); ++k) cudaFree(c->allocs[k]);
    if (c->d.grid.cand) cudaFree(c->d.grid.cand);
    if (c->scan_tmp) cudaFree(c->scan_tmp);
    if (c->scan_tmp2) cudaFree(c->scan_tmp2);
    if (c->cnt_h) cudaFreeHost(c->cnt_h);
    if (c->st2) {
        cudaStreamSynchronize(c->st2);
        cudaStreamDestroy(c->st2);
    }
    for (int k = 0; k < 4; ++k)
        if (c->hev[k]) cudaEventDestroy(c->hev[k]);
    for (int k = 0; k < 2; ++k)
        if (c->tune_ev[k]) cudaEventDestroy(c->tune_ev[k]);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return RT_OK;
}

static rt_status copy_in(rt_ctx *c, void *dst, const void *src, size_t bytes, int where,
                         cudaStream_t st) {
    if (!src) return RT_OK;
    cudaMemcpyKind k = where == RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, k, st);
    if (e == cudaSuccess && where == RT_HOST) e = cudaStreamSynchronize(st);
    return rt_cuda_check(c, e, "copy in");
}

static rt_status copy_out(rt_ctx *c, void *dst, const void *src, size_t bytes, int where,
                          cudaStream_t st) {
    if (!dst) return RT_OK;
    cudaMemcpyKind k = where == RT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, k, st);
    if (e == cudaSuccess && where == RT_HOST) e = cudaStreamSynchronize(st);
    return rt_cuda_check(c, e, "copy out");
}

static void set_norms(rt_ctx *c) {
    // slot unit per box: the box's source photons of one step (FP32 path), else 1 (FP64);
    // fixed-point reference of the escaped tally: the same photon count
    rt_ctx &x = *c;
    int nb = c->d.nb;
    std::vector<double> ref(nb), norm(nb);
    for (int b = 0; b < nb; ++b) {
        double r = x.src_emit_h[b];
        if (!(r > 0.0)) r = 1e-3 * x.box_NH_h[b];
        if (!(r > 0.0)) r = 1.0;
        ref[b] = r;
        norm[b] = c->d.fp32 ? r : 1.0;
    }
    cudaMemcpy(c->d.ref, ref.data(), sizeof(double) * nb, cudaMemcpyHostToDevice);
    std::vector<float> escf(nb);
    for (int b = 0; b < nb; ++b) escf[b] = (float)(FX_ESC_SCALE * norm[b] / ref[b]);
    cudaMemcpy(c->d.escf, escf.data(), sizeof(float) * nb, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d.norm, norm.data(), sizeof(double) * nb, cudaMemcpyHostToDevice);
    cudaMemcpy(x.src_emit, x.src_emit_h.data(), sizeof(double) * nb, cudaMemcpyHostToDevice);
}

// ---- input validation ---------------------------------------------------------------------
// Values the method cannot use, found on the device copies (host and device inputs alike):
// non-finite positions; non-positive or non-finite densities and atom counts; neutral
// fractions outside [0, 1]; non-positive or non-finite temperatures; negative or non-finite
// recombination photons and energies.  Reads only; a NULL array is not checked.
__global__ void k_check_inputs(long long n, const double *x, const double *y, const double *z,
                               const double *nH, const double *NH, const double *xHI,
                               const double *T, const double *Nrec, const double *epsrec,
                               long long *bad) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    if (x) ok = ok && isfinite(x[i]) && isfinite(y[i]) && isfinite(z[i]);
    if (nH) ok = ok && nH[i] > 0.0 && isfinite(nH[i]);
    if (NH) ok = ok && NH[i] > 0.0 && isfinite(NH[i]);
    if (xHI) ok = ok && xHI[i] >= 0.0 && xHI[i] <= 1.0;
    if (T) ok = ok && T[i] > 0.0 && isfinite(T[i]);
    if (Nrec) ok = ok && Nrec[i] >= 0.0 && isfinite(Nrec[i]);
    if (epsrec) ok = ok && epsrec[i] >= 0.0 && isfinite(epsrec[i]);
    if (!ok) atomicOr((unsigned long long *)bad, 1ull);
}

static const int CNT_CHECK = CNT_N - 2;   // device word of the input checks

// true when every value passes (synchronises st)
static bool inputs_ok(rt_ctx *c, long long n, const double *x, const double *y, const double *z,
                      const double *nH, const double *NH, const double *xHI, const double *T,
                      const double *Nrec, const double *epsrec, cudaStream_t st) {
    long long *flag = c->d.cnt + CNT_CHECK;
    cudaMemsetAsync(flag, 0, sizeof(long long), st);
    if (n > 0)
        k_check_inputs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y, z, nH, NH, xHI, T,
                                                                    Nrec, epsrec, flag);
    long long bad = 0;
    cudaMemcpyAsync(&bad, flag, sizeof(long long), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return bad == 0;
}

extern "C" rt_status rt_set_particles(rt_ctx *c, const double *x, const double *y,
                                      const double *z, const double *n_H, const double *N_H,
                                      const double *x_HI, const double *T, int where,
                                      void *stream) {
    if (!c || !x || !y || !z || !n_H || !N_H || !x_HI || !T) return RT_ERR_INVALID;
    if (where != RT_HOST && where != RT_DEVICE) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    DevPtrs &P = c->d;
    size_t nb = sizeof(double) * (size_t)P.n;
    double *tx = nullptr, *ty = nullptr, *tz = nullptr;
    if (cudaMalloc(&tx, 3 * nb) != cudaSuccess) return rt_fail(c, RT_ERR_OOM, "position staging");
    ty = tx + P.n;
    tz = ty + P.n;
    rt_status s = RT_OK;
    if ((s = copy_in(c, tx, x, nb, where, st)) || (s = copy_in(c, ty, y, nb, where, st)) ||
        (s = copy_in(c, tz, z, nb, where, st)) || (s = copy_in(c, P.nH, n_H, nb, where, st)) ||
        (s = copy_in(c, P.NH, N_H, nb, where, st)) || (s = copy_in(c, P.xHI, x_HI, nb, where, st)) ||
        (s = copy_in(c, P.T, T, nb, where, st))) {
        cudaFree(tx);
        return s;
    }
    if (!inputs_ok(c, P.n, tx, ty, tz, P.nH, P.NH, P.xHI, P.T, nullptr, nullptr, st)) {
        cudaFree(tx);
        c->have_particles = false;
        c->built = false;
        return rt_fail(c, RT_ERR_INVALID,
                       "rt_set_particles: a non-finite position, a non-positive density or atom "
                       "count, x_HI outside [0, 1] or a non-positive temperature");
    }
    rt_launch_quantise(c, tx, ty, tz, st);
    cudaStreamSynchronize(st);
    cudaFree(tx);
    // per-box atom totals (fallback photon unit for boxes without sources)
    std::vector<double> NHh(P.n);
    cudaMemcpy(NHh.data(), P.NH, nb, cudaMemcpyDeviceToHost);
    rt_ctx &xe = *c;
    for (int b = 0; b < P.nb; ++b) {
        double t = 0.0;
        for (long long i = c->box_off_h[b]; i < c->box_off_h[b + 1]; ++i) t += NHh[i];
        xe.box_NH_h[b] = t;
    }
    for (int b = 0; b < 2; ++b) {
        cudaMemsetAsync(P.occ[b], 0, sizeof(unsigned) * P.n * P.nf, st);
        cudaMemsetAsync(P.act[b], 0, sizeof(unsigned) * P.n * P.nf, st);
    }
    cudaMemsetAsync(P.Nrec, 0, nb, st);
    cudaMemsetAsync(P.epsrec, 0, nb, st);
    cudaMemsetAsync(P.tally, 0, sizeof(double) * 4 * P.nb, st);
    cudaMemsetAsync(P.esc_fx, 0, sizeof(unsigned long long) * P.nb, st);
    c->have_particles = true;
    c->built = false;
    set_norms(c);
    return rt_cuda_check(c, cudaStreamSynchronize(st), "set particles");
}

extern "C" rt_status rt_set_sources(rt_ctx *c, const int *box, const double *x, const double *y,
                                    const double *z, const double *ndot, const double *sigma,
                                    const double *eps, int where, void *stream) {
    if (!c) return RT_ERR_INVALID;
    if (where != RT_HOST && where != RT_DEVICE) return RT_ERR_INVALID;
    DevPtrs &P = c->d;
    cudaStream_t st = (cudaStream_t)stream;
    if (P.nfs > 0 && (!sigma || !eps)) return RT_ERR_INVALID;
    if (P.ns > 0 && (!box || !x || !y || !z || (P.nfs > 0 && !ndot))) return RT_ERR_INVALID;
    size_t sb = sizeof(double) * (size_t)P.ns;
    std::vector<int> boxh(P.ns);
    std::vector<double> ndh((size_t)P.ns * P.nfs);
    rt_status s;
    if (P.ns > 0) {
        if (where == RT_HOST) {
            memcpy(boxh.data(), box, sizeof(int) * P.ns);
            if (P.nfs) memcpy(ndh.data(), ndot, sizeof(double) * P.ns * P.nfs);
        } else {
            cudaMemcpy(boxh.data(), box, sizeof(int) * P.ns, cudaMemcpyDeviceToHost);
            if (P.nfs) cudaMemcpy(ndh.data(), ndot, sizeof(double) * P.ns * P.nfs, cudaMemcpyDeviceToHost);
        }
        for (int j = 0; j < P.ns; ++j)
            if (boxh[j] < 0 || boxh[j] >= P.nb) return rt_fail(c, RT_ERR_INVALID, "source box index");
        double *t = nullptr;
        if (cudaMalloc(&t, 3 * sb) != cudaSuccess) return rt_fail(c, RT_ERR_OOM, "source staging");
        cudaMemcpy(P.sbox, boxh.data(), sizeof(int) * P.ns, cudaMemcpyHostToDevice);
        if ((s = copy_in(c, t, x, sb, where, st)) || (s = copy_in(c, t + P.ns, y, sb, where, st)) ||
            (s = copy_in(c, t + 2 * P.ns, z, sb, where, st))) {
            cudaFree(t);
            return s;
        }
        if (!inputs_ok(c, P.ns, t, t + P.ns, t + 2 * P.ns, nullptr, nullptr, nullptr, nullptr,
                       nullptr, nullptr, st)) {
            cudaFree(t);
            c->have_sources = false;
            c->built = false;
            return rt_fail(c, RT_ERR_INVALID, "rt_set_sources: a non-finite position");
        }
        rt_launch_quantise_src(c, t, t + P.ns, t + 2 * P.ns, st);
        cudaStreamSynchronize(st);
        cudaFree(t);
        if (P.nfs) cudaMemcpy(P.ndot, ndh.data(), sizeof(double) * P.ns * P.nfs, cudaMemcpyHostToDevice);
    }
    std::vector<double> sg(P.nfs + 1), ep(P.nfs + 1);
    if (P.nfs > 0) {
        if (where == RT_HOST) {
            memcpy(sg.data(), sigma, sizeof(double) * P.nfs);
            memcpy(ep.data(), eps, sizeof(double) * P.nfs);
        } else {
            cudaMemcpy(sg.data(), sigma, sizeof(double) * P.nfs, cudaMemcpyDeviceToHost);
            cudaMemcpy(ep.data(), eps, sizeof(double) * P.nfs, cudaMemcpyDeviceToHost);
        }
    }
    for (int f = 0; f < P.nfs; ++f)
        if (!(sg[f] > 0.0) || !std::isfinite(sg[f]) || !(ep[f] >= 0.0) || !std::isfinite(ep[f]))
        {
            c->have_sources = false;
            c->built = false;
            return rt_fail(c, RT_ERR_INVALID, "rt_set_sources: a non-positive cross-section or a "
                                              "negative excess energy");
        }
    for (double v : ndh)
        if (!(v >= 0.0) || !std::isfinite(v))
        {
            c->have_sources = false;
            c->built = false;
            return rt_fail(c, RT_ERR_INVALID, "rt_set_sources: a negative photon rate");
        }
    sg[P.nfs] = c->cfg.sigma_rec;
    ep[P.nfs] = 0.0;
    // entry nfs: the recombination photons' (their bin's, unless the bin is shared)
    cudaMemcpy(P.sigma, sg.data(), sizeof(double) * (P.nfs + 1), cudaMemcpyHostToDevice);
    std::vector<float> sgf(sg.begin(), sg.end());
    cudaMemcpy(P.sigmaf, sgf.data(), sizeof(float) * (P.nfs + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(P.eps, ep.data(), sizeof(double) * (P.nfs + 1), cudaMemcpyHostToDevice);
    // source photons of one step per box, summed packet by packet as they are emitted
    rt_ctx &xe = *c;
    std::fill(xe.src_emit_h.begin(), xe.src_emit_h.end(), 0.0);
    for (int j = 0; j < P.ns; ++j)
        for (int k = 0; k < P.K; ++k)
            for (int nu = 0; nu < P.nfs; ++nu) {
                double Np = ndh[(size_t)j * P.nfs + nu] * P.dt_em / (double)P.nec;
                for (int e = 0; e < P.nec; ++e) xe.src_emit_h[boxh[j]] += Np;
            }
    c->have_sources = true;
    c->built = false;
    set_norms(c);
    return rt_cuda_check(c, cudaStreamSynchronize(st), "set sources");
}

extern "C" rt_status rt_set_identities(rt_ctx *c, const long long *box_first_id,
                                       const long long *src_id) {
    if (!c) return RT_ERR_INVALID;
    DevPtrs &P = c->d;
    int nb = P.nb, ns = P.ns;
    std::vector<long long> g(nb), sd(ns + 1, 0);
    for (int b = 0; b < nb; ++b) {
        long long cnt = c->box_off_h[b + 1] - c->box_off_h[b];
        g[b] = box_first_id ? box_first_id[b] : c->box_off_h[b];
        // the rotation counters take 32-bit identities
        if (g[b] < 0 || g[b] + cnt > (1ll << 32))
            return rt_fail(c, RT_ERR_INVALID, "rt_set_identities: box identities outside [0, 2^32)");
    }
    for (int j = 0; j < ns; ++j) {
        sd[j] = src_id ? src_id[j] : j;
        if (sd[j] < 0 || sd[j] >= (1ll << 32))
            return rt_fail(c, RT_ERR_INVALID, "rt_set_identities: source identities outside [0, 2^32)");
    }
    cudaDeviceSynchronize();   // no kernel of this context may be reading the identities
    cudaMemcpy(P.gid0, g.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice);
    cudaMemcpy(P.sid, sd.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice);
    return rt_cuda_check(c, cudaGetLastError(), "identities");
}

extern "C" rt_status rt_set_source_options(rt_ctx *c, const double *dir, const int *gate,
                                           int where, void *stream) {
    if (!c) return RT_ERR_INVALID;
    if (where != RT_HOST && where != RT_DEVICE) return RT_ERR_INVALID;
    DevPtrs &P = c->d;
    cudaStream_t st = (cudaStream_t)stream;
    if (P.ns == 0) return RT_OK;
    rt_status s;
    if (dir) {
        if ((s = copy_in(c, P.sdir, dir, sizeof(double) * 3 * P.ns, where, st))) return s;
    } else {
        cudaMemsetAsync(P.sdir, 0, sizeof(double) * 3 * P.ns, st);
    }
    if (gate) {
        if ((s = copy_in(c, P.sgate, gate, sizeof(int) * P.ns, where, st))) return s;
    } else {
        cudaMemsetAsync(P.sgate, 0, sizeof(int) * P.ns, st);
    }
    if ((s = rt_cuda_check(c, cudaStreamSynchronize(st), "source options"))) return s;
    std::vector<int> g(P.ns);
    cudaMemcpy(g.data(), P.sgate, sizeof(int) * P.ns, cudaMemcpyDeviceToHost);
    P.gated = 0;
    for (int v : g) P.gated |= v != 0;
    return rt_cuda_check(c, cudaGetLastError(), "source options");
}

// quantised coordinate of a box position (floor of x / L * 2^20, clamped into the box)
static long long host_quantise(double x, double L) {
    double f = x / L;
    f = f * (double)RT_Q;
    double fl = floor(f);
    long long q = (long long)fl;
    if (!(fl >= 0.0)) q = 0;
    if (q > RT_Q - 1) q = RT_Q - 1;
    return q;
}

extern "C" rt_status rt_set_barrier(rt_ctx *c, int box, int axis, const double *centre,
                                    double radius) {
    if (!c) return RT_ERR_INVALID;
    DevPtrs &P = c->d;
    if (box < 0 || box >= P.nb) return RT_ERR_INVALID;
    Barrier B{-1, 0, 0, 0, 0};
    if (radius > 0.0) {
        if (axis < 0 || axis > 2 || !centre) return RT_ERR_INVALID;
        double L = c->box_L_h[box];
        B.axis = axis;
        B.p2 = 2 * host_quantise(centre[axis], L) + 1;
        B.c1 = 2 * host_quantise(centre[(axis + 1) % 3], L);
        B.c2 = 2 * host_quantise(centre[(axis + 2) % 3], L);
        B.r2 = llround(2.0 * radius / L * (double)RT_Q);
        if (B.r2 >= (1ll << 23)) return RT_ERR_INVALID;   // keeps the exact test in 128 bits
    }
    c->bar_h[box] = B;
    cudaDeviceSynchronize();   // no hop kernel of this context may be reading the barriers
    cudaMemcpy(P.bar + box, &B, sizeof(Barrier), cudaMemcpyHostToDevice);
    P.any_bar = 0;
    for (const Barrier &x : c->bar_h) P.any_bar |= x.axis >= 0;
    return rt_cuda_check(c, cudaGetLastError(), "barrier");
}

extern "C" rt_status rt_build_neighbours(rt_ctx *c, void *stream) {
    if (!c) return RT_ERR_INVALID;
    if (!c->have_particles || !c->have_sources)
        return rt_fail(c, RT_ERR_STATE, "rt_set_particles and rt_set_sources come first");
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(&c->d.cnt[CNT_ERR], 0, sizeof(long long), st);
    rt_status s = rt_knn_build(c, st);
    if (s) return s;
    long long err = 0;
    cudaMemcpyAsync(&err, &c->d.cnt[CNT_ERR], sizeof(long long), cudaMemcpyDeviceToHost, st);
    s = rt_cuda_check(c, cudaStreamSynchronize(st), "neighbour build");
    if (s) return s;
    if (err & ERRB_KNN)
        return rt_fail(c, RT_ERR_KNN, "a box holds too few particles, or a neighbour lies "
                                      "beyond the kNN key range");
    c->built = true;
    return RT_OK;
}

static rt_status need_built(rt_ctx *c) {
    if (!c) return RT_ERR_INVALID;
    if (!c->built) return rt_fail(c, RT_ERR_STATE, "rt_build_neighbours has not run");
    return RT_OK;
}

extern "C" rt_status rt_assign_cones(rt_ctx *c, long long step, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = rt_run_step_parts(c, 0, step, st))) return s;
    return rt_run_step_parts(c, 3, step, st);
}

extern "C" rt_status rt_merge(rt_ctx *c, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    return rt_run_step_parts(c, 1, 0, (cudaStream_t)stream);
}

extern "C" rt_status rt_emit(rt_ctx *c, long long step, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = rt_run_step_parts(c, 2, step, st))) return s;
    return rt_budget_launch(c, 0, st);
}

extern "C" rt_status rt_transport(rt_ctx *c, long long step, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    return rt_run_step_parts(c, 4, step, (cudaStream_t)stream);
}

// the chemistry and the end-of-step tally; RT_OK even when the subcycle floor was hit (the
// floor hits are in c->stats[4] afterwards)
static rt_status chemistry_run(rt_ctx *c, cudaStream_t st) {
    rt_status s;
    if ((s = rt_chem_launch(c, st))) return s;
    if ((s = rt_budget_launch(c, 1, st))) return s;
    cudaMemcpyAsync(c->cnt_h, c->d.cnt, sizeof(long long) * CNT_N, cudaMemcpyDeviceToHost, st);
    s = rt_cuda_check(c, cudaStreamSynchronize(st), "chemistry");
    c->stats[3] = c->cnt_h[CNT_SUB];
    c->stats[4] = c->cnt_h[CNT_FLOOR];
    return s;
}

rt_status rt_subcycle_status(rt_ctx *c) {
    if (c->stats[4] <= 0) return RT_OK;
    return rt_fail(c, RT_ERR_SUBCYCLE_LIMIT,
                   std::to_string(c->stats[4]) + " chemistry subcycles were held at the floor "
                   "dt/sub_cap with a larger than 10% energy change (raise sub_cap)");
}

extern "C" rt_status rt_chemistry(rt_ctx *c, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    if ((s = chemistry_run(c, (cudaStream_t)stream))) return s;
    return rt_subcycle_status(c);
}

extern "C" rt_status rt_step(rt_ctx *c, long long step, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the captured step graph, unless kernels are being timed one by one (events cannot sit
    // inside the graph's conditional hop loop) or the hop cap allows no hop; while the launch
    // sizes are being tuned (tune_launch), the graph steps are timed whole
    if (c->use_graph && c->prof == 0 && c->cfg.hop_cap > 0) {
        if (c->cfg.tune_launch && !c->launch_tuned) return rt_step_graph_tuned(c, step, st);
        return rt_step_graph(c, step, st);
    }
    if ((s = rt_run_step_parts(c, 0, step, st))) return s;
    if ((s = rt_run_step_parts(c, 1, step, st))) return s;
    if ((s = rt_emit(c, step, stream))) return s;
    rt_status ts = rt_run_step_parts(c, 4, step, st);
    if (ts != RT_OK && ts != RT_ERR_HOP_LIMIT) return ts;
    if ((s = chemistry_run(c, st))) return s;
    return ts != RT_OK ? ts : rt_subcycle_status(c);
}

extern "C" rt_status rt_get_state(rt_ctx *c, double *x_HI, double *T, double *N_rec,
                                  double *eps_rec, int where, void *stream) {
    if (!c) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    size_t b = sizeof(double) * (size_t)c->d.n;
    rt_status s;
    if ((s = copy_out(c, x_HI, c->d.xHI, b, where, st)) || (s = copy_out(c, T, c->d.T, b, where, st)) ||
        (s = copy_out(c, N_rec, c->d.Nrec, b, where, st)) ||
        (s = copy_out(c, eps_rec, c->d.epsrec, b, where, st)))
        return s;
    return RT_OK;
}

extern "C" rt_status rt_set_state(rt_ctx *c, const double *x_HI, const double *T,
                                  const double *N_rec, const double *eps_rec, int where,
                                  void *stream) {
    if (!c) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    size_t b = sizeof(double) * (size_t)c->d.n;
    rt_status s;
    if ((s = copy_in(c, c->d.xHI, x_HI, b, where, st)) || (s = copy_in(c, c->d.T, T, b, where, st)) ||
        (s = copy_in(c, c->d.Nrec, N_rec, b, where, st)) ||
        (s = copy_in(c, c->d.epsrec, eps_rec, b, where, st)))
        return s;
    DevPtrs &P = c->d;
    if (!inputs_ok(c, P.n, nullptr, nullptr, nullptr, nullptr, nullptr, x_HI ? P.xHI : nullptr,
                   T ? P.T : nullptr, N_rec ? P.Nrec : nullptr, eps_rec ? P.epsrec : nullptr, st))
        return rt_fail(c, RT_ERR_INVALID,
                       "rt_set_state: x_HI outside [0, 1], a non-positive temperature, or negative "
                       "recombination photons or energy (the rejected values are in place: set "
                       "the state again before the next step)");
    return RT_OK;
}

extern "C" rt_status rt_get_budget(rt_ctx *c, double *out, void *stream) {
    if (!c || !out) return RT_ERR_INVALID;
    return copy_out(c, out, c->d.tally, sizeof(double) * 4 * c->d.nb, RT_HOST, (cudaStream_t)stream);
}

// ---- checkpoint / resume ------------------------------------------------------------------
// A checkpoint taken between steps holds what a step carries into the next one, byte for byte:
// the packets held by the particles (the current slot buffer with its occupancy and activity
// words, and the cross-section sums of a shared bin), the particle state (x_HI, T, and the
// recombination photons and their energy waiting to be emitted), the photon budget and the
// fixed-point escape word.  Everything else (rotations, deposits, bitmaps, free packets) is
// rebuilt or cleared by the next step.  The header records the sizes it was taken with.
struct CkptHeader {
    char magic[8];
    int version, fp32, shared, nf, S, nrc, nb, pad;
    long long n, bytes;
};

static const char CKPT_MAGIC[8] = {'T', 'R', 'P', 'H', 'C', 'K', 'P', '1'};

struct CkptPart {
    void *dev;
    size_t bytes;
};

static std::vector<CkptPart> ckpt_parts(rt_ctx *c) {
    DevPtrs &P = c->d;
    size_t R = P.fp32 ? 4 : 8, nslot = (size_t)P.n * P.S, nkey = (size_t)P.n * P.nf;
    std::vector<CkptPart> v;
    for (int f = 0; f < 6; ++f) v.push_back({P.sl[c->cur][f], R * nslot});
    v.push_back({P.occ[c->cur], sizeof(unsigned) * nkey});
    v.push_back({P.act[c->cur], sizeof(unsigned) * nkey});
    if (P.shared) v.push_back({P.slG[c->cur], R * (size_t)P.n * P.nrc});
    for (double *a : {P.xHI, P.T, P.Nrec, P.epsrec}) v.push_back({a, sizeof(double) * (size_t)P.n});
    v.push_back({P.tally, sizeof(double) * 4 * (size_t)P.nb});
    v.push_back({P.esc_fx, sizeof(unsigned long long) * (size_t)P.nb});
    return v;
}

static CkptHeader ckpt_header(rt_ctx *c) {
    DevPtrs &P = c->d;
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, CKPT_MAGIC, 8);
    h.version = 1;
    h.fp32 = P.fp32; h.shared = P.shared; h.nf = P.nf; h.S = P.S; h.nrc = P.nrc; h.nb = P.nb;
    h.n = P.n;
    size_t b = sizeof(CkptHeader);
    for (auto &q : ckpt_parts(c)) b += q.bytes;
    h.bytes = (long long)b;
    return h;
}

extern "C" rt_status rt_save_state(rt_ctx *c, void *buf, size_t *bytes) {
    rt_status s = need_built(c);
    if (s) return s;
    if (!bytes) return RT_ERR_INVALID;
    CkptHeader h = ckpt_header(c);
    if (!buf) {
        *bytes = (size_t)h.bytes;
        return RT_OK;
    }
    if (*bytes < (size_t)h.bytes)
        return rt_fail(c, RT_ERR_INVALID, "rt_save_state: buffer of " + std::to_string(*bytes) +
                                              " bytes, " + std::to_string(h.bytes) + " needed");
    // every queued step on every stream has finished before the copies
    if ((s = rt_cuda_check(c, cudaDeviceSynchronize(), "save state"))) return s;
    char *o = (char *)buf;
    memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    for (auto &q : ckpt_parts(c)) {
        if ((s = rt_cuda_check(c, cudaMemcpy(o, q.dev, q.bytes, cudaMemcpyDeviceToHost), "save state")))
            return s;
        o += q.bytes;
    }
    *bytes = (size_t)h.bytes;
    return RT_OK;
}

extern "C" rt_status rt_load_state(rt_ctx *c, const void *buf, size_t bytes) {
    rt_status s = need_built(c);
    if (s) return s;
    if (!buf || bytes < sizeof(CkptHeader)) return RT_ERR_INVALID;
    CkptHeader h = ckpt_header(c), g;
    memcpy(&g, buf, sizeof(g));
    if (memcmp(g.magic, CKPT_MAGIC, 8) != 0 || g.version != 1)
        return rt_fail(c, RT_ERR_INVALID, "rt_load_state: not a checkpoint of this library");
    if (g.fp32 != h.fp32 || g.shared != h.shared || g.nf != h.nf || g.S != h.S ||
        g.nrc != h.nrc || g.nb != h.nb || g.n != h.n || g.bytes != h.bytes || bytes < (size_t)h.bytes)
        return rt_fail(c, RT_ERR_INVALID, "rt_load_state: checkpoint of another configuration");
    if ((s = rt_cuda_check(c, cudaDeviceSynchronize(), "load state"))) return s;
    const char *o = (const char *)buf + sizeof(CkptHeader);
    for (auto &q : ckpt_parts(c)) {
        if ((s = rt_cuda_check(c, cudaMemcpy(q.dev, o, q.bytes, cudaMemcpyHostToDevice), "load state")))
            return s;
        o += q.bytes;
    }
    return RT_OK;
}

extern "C" rt_status rt_get_neighbours(rt_ctx *c, int *nbr, long long *h2, int *src_nbr,
                                       long long *src_h2, int where, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    DevPtrs &P = c->d;
    if ((s = copy_out(c, nbr, P.nbr, sizeof(int) * P.n * P.kn, where, st)) ||
        (s = copy_out(c, h2, P.h2, sizeof(long long) * P.n, where, st)) ||
        (s = copy_out(c, src_nbr, P.snbr, sizeof(int) * (size_t)P.ns * P.kn, where, st)) ||
        (s = copy_out(c, src_h2, P.sh2, sizeof(long long) * P.ns, where, st)))
        return s;
    return RT_OK;
}

__global__ void k_get_q(DevPtrs P, long long *q) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    q[3 * i] = P.qx[i]; q[3 * i + 1] = P.qy[i]; q[3 * i + 2] = P.qz[i];
}

template <typename T> static T *dtmp(size_t n) {
    T *p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) return nullptr;
    return p;
}

void rt_launch_query(rt_ctx *c, int b, long long m, const int *q, int *nbr, long long *d2,
                     int *fail, cudaStream_t st);

extern "C" rt_status rt_query_neighbours(rt_ctx *c, int box, long long m, const int *q, int *nbr,
                                         long long *d2, int where, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    if (box < 0 || box >= c->d.nb || m < 0 || (m > 0 && !q) ||
        (where != RT_HOST && where != RT_DEVICE))
        return rt_fail(c, RT_ERR_INVALID, "rt_query_neighbours: bad box, count or pointer");
    if (m == 0) return RT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    size_t kn = (size_t)c->d.kn;
    int *qd = (int *)q, *nd = nbr, *fd = dtmp<int>(1);
    long long *dd = d2;
    bool host = where == RT_HOST;
    if (host) {
        qd = dtmp<int>(3 * (size_t)m);
        nd = nbr ? dtmp<int>(kn * m) : nullptr;
        dd = d2 ? dtmp<long long>(kn * m) : nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!fd || !qd || (nbr && !nd) || (d2 && !dd)) {
        s = rt_fail(c, RT_ERR_OOM, "temp");
    } else {
        cudaMemsetAsync(fd, 0, sizeof(int), st);
        if (host) e = cudaMemcpyAsync(qd, q, sizeof(int) * 3 * m, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            rt_launch_query(c, box, m, qd, nd, dd, fd, st);
            e = cudaGetLastError();
        }
        int fail = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&fail, fd, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && host && nbr)
            e = cudaMemcpyAsync(nbr, nd, sizeof(int) * kn * m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && host && d2)
            e = cudaMemcpyAsync(d2, dd, sizeof(long long) * kn * m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        s = rt_cuda_check(c, e, "rt_query_neighbours");
        if (s == RT_OK && (fail & 1))
            s = rt_fail(c, RT_ERR_INVALID, "rt_query_neighbours: a coordinate out of [0, 2^20)");
        else if (s == RT_OK && (fail & 2))
            s = rt_fail(c, RT_ERR_KNN, "rt_query_neighbours: a search found too few particles");
    }
    cudaStreamSynchronize(st);
    if (fd) cudaFree(fd);
    if (host) {
        if (qd) cudaFree(qd);
        if (nd) cudaFree(nd);
        if (dd) cudaFree(dd);
    }
    return s;
}

extern "C" rt_status rt_get_quantised(rt_ctx *c, long long *q, int where, void *stream) {
    if (!c || !q || !c->have_particles) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    long long *t = dtmp<long long>(3 * c->d.n);
    if (!t) return rt_fail(c, RT_ERR_OOM, "temp");
    k_get_q<<<(unsigned)((c->d.n + 255) / 256), 256, 0, st>>>(c->d, t);
    rt_status s = copy_out(c, q, t, sizeof(long long) * 3 * c->d.n, where, st);
    cudaStreamSynchronize(st);
    cudaFree(t);
    return s;
}

extern "C" rt_status rt_get_rotations(rt_ctx *c, double *R, double *Rs, int where, void *stream) {
    if (!c) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    DevPtrs &P = c->d;
    rt_status s;
    if ((s = copy_out(c, R, P.R, sizeof(double) * 9 * P.n, where, st)) ||
        (s = copy_out(c, Rs, P.Rs, sizeof(double) * 9 * (size_t)P.ns * P.K, where, st)))
        return s;
    return RT_OK;
}

__global__ void k_masks(DevPtrs P, int cur, unsigned *out) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.n * P.S) return;
    long long i = t / P.S;
    int s = (int)(t % P.S);
    int nu = s / P.nrc, b = s % P.nrc;
    unsigned a = P.act[cur][i * P.nf + nu];
    unsigned m = 0;
    const unsigned *bmr = P.bm + (long long)nu * P.n * P.kn;
    if ((a >> b) & 1u)
        for (int k = 0; k < P.kn; ++k)
            m |= ((bmr[P.revpos[i * P.kn + k]] >> b) & 1u) << k;
    out[t] = m;
}

extern "C" rt_status rt_get_cone_masks(rt_ctx *c, unsigned *mask, int where, void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    if (!mask || (where != RT_HOST && where != RT_DEVICE)) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    long long m = c->d.n * c->d.S;
    unsigned *t = dtmp<unsigned>(m);
    if (!t) return rt_fail(c, RT_ERR_OOM, "temp");
    k_masks<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(c->d, c->cur, t);
    s = rt_cuda_check(c, cudaGetLastError(), "mask kernel");
    if (s == RT_OK) s = copy_out(c, mask, t, sizeof(unsigned) * m, where, st);
    cudaStreamSynchronize(st);
    cudaFree(t);
    return s;
}

// ---- cone masks without allocation -----------------------------------------------------------
// The same masks as rt_get_cone_masks, assembled in a file-scope device array instead of a
// buffer obtained from cudaMalloc, for callers that must not allocate device memory.
#define RT_STATIC_MASKS (1 << 22)   // 4,194,304 masks (16 MiB), held by every device that loads the library
static __device__ __align__(256) unsigned g_mask_scratch[RT_STATIC_MASKS];

// device address of g_mask_scratch, looked up once per device (with that device current)
static unsigned *mask_scratch(int dev, cudaError_t *err) {
    static std::mutex mu;
    static unsigned *addr[128] = {nullptr};
    *err = cudaSuccess;
    if (dev < 0 || dev >= 128) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_mask_scratch);
        if (*err != cudaSuccess) return nullptr;
        addr[dev] = (unsigned *)p;
    }
    return addr[dev];
}

extern "C" rt_status rt_get_cone_masks_noalloc(rt_ctx *c, unsigned *mask, int where,
                                               void *stream) {
    rt_status s = need_built(c);
    if (s) return s;
    if (!mask || (where != RT_HOST && where != RT_DEVICE)) return RT_ERR_INVALID;
    long long m = c->d.n * c->d.S;
    if (m > RT_STATIC_MASKS)
        return rt_fail(c, RT_ERR_INVALID,
                       "rt_get_cone_masks_noalloc: n * S = " + std::to_string(m) +
                           " masks exceed the static scratch of 4194304");
    int dev = 0;
    if ((s = rt_cuda_check(c, cudaGetDevice(&dev), "cudaGetDevice"))) return s;
    cudaError_t e;
    unsigned *t = mask_scratch(dev, &e);
    if (!t) return rt_cuda_check(c, e, "cudaGetSymbolAddress(g_mask_scratch)");
    cudaStream_t st = (cudaStream_t)stream;
    // every entry of [0, m) is written, so the previous call's contents need no clearing
    kt_begin(c, KT_MASKS, st);
    k_masks<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(c->d, c->cur, t);
    kt_end(c, KT_MASKS, st);
    if ((s = rt_cuda_check(c, cudaGetLastError(), "mask kernel"))) return s;
    return copy_out(c, mask, t, sizeof(unsigned) * m, where, st);
}

template <typename Real>
__global__ void k_slots_io(DevPtrs P, int cur, double *f, int to_dev) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long m = P.n * P.S;
    if (t >= m) return;
    long long i = t / P.S;
    int s = (int)(t % P.S);
    int nu = s / P.nrc, b = s % P.nrc;
    double nm = P.norm[P.pbox[i]];
    Real *F[6];
    for (int k = 0; k < 6; ++k) F[k] = (Real *)P.sl[cur][k];
    long long key = i * P.nf + nu;
    if (to_dev) {
        double N = f[t];
        for (int k = 0; k < 5; ++k) F[k][t] = (Real)(f[k * m + t] / nm);
        F[5][t] = (Real)(f[5 * m + t] / nm / P.eunit);
        bool occ = N > 0.0;
        bool act = occ && (f[4 * m + t] / N < P.dt);
        if (occ) atomicOr(&P.occ[cur][key], 1u << b);
        if (act) atomicOr(&P.act[cur][key], 1u << b);
    } else {
        bool occ = (P.occ[cur][key] >> b) & 1u;
        for (int k = 0; k < 6; ++k) f[k * m + t] = occ ? (double)F[k][t] * nm : 0.0;
        f[5 * m + t] *= P.eunit;
    }
}

extern "C" rt_status rt_get_slots(rt_ctx *c, double *f, int where, void *stream) {
    if (!c || !f) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    long long m = c->d.n * c->d.S;
    double *t = dtmp<double>(6 * m);
    if (!t) return rt_fail(c, RT_ERR_OOM, "temp");
    unsigned nb = (unsigned)((m + 255) / 256);
    if (c->d.fp32) k_slots_io<float><<<nb, 256, 0, st>>>(c->d, c->cur, t, 0);
    else k_slots_io<double><<<nb, 256, 0, st>>>(c->d, c->cur, t, 0);
    rt_status s = copy_out(c, f, t, sizeof(double) * 6 * m, where, st);
    cudaStreamSynchronize(st);
    cudaFree(t);
    return s;
}

extern "C" rt_status rt_set_slots(rt_ctx *c, const double *f, int where, void *stream) {
    if (!c || !f) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    long long m = c->d.n * c->d.S;
    double *t = dtmp<double>(6 * m);
    if (!t) return rt_fail(c, RT_ERR_OOM, "temp");
    rt_status s = copy_in(c, t, f, sizeof(double) * 6 * m, where, st);
    if (s) { cudaFree(t); return s; }
    cudaMemsetAsync(c->d.occ[c->cur], 0, sizeof(unsigned) * c->d.n * c->d.nf, st);
    cudaMemsetAsync(c->d.act[c->cur], 0, sizeof(unsigned) * c->d.n * c->d.nf, st);
    unsigned nb = (unsigned)((m + 255) / 256);
    if (c->d.fp32) k_slots_io<float><<<nb, 256, 0, st>>>(c->d, c->cur, t, 1);
    else k_slots_io<double><<<nb, 256, 0, st>>>(c->d, c->cur, t, 1);
    s = rt_cuda_check(c, cudaStreamSynchronize(st), "set slots");
    cudaFree(t);
    return s;
}

// the cross-section sums of the shared frequency bin (bin 0), [n * nrc], in cm^2 x photons
template <typename Real>
__global__ void k_shared_sigma_io(DevPtrs P, int cur, double *f, int to_dev) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.n * P.nrc) return;
    long long i = t / P.nrc;
    int b = (int)(t % P.nrc);
    double nm = P.norm[P.pbox[i]];
    Real *G = (Real *)P.slG[cur];
    if (to_dev) {
        G[t] = (Real)(f[t] / nm / P.sunit);
    } else {
        bool occ = (P.occ[cur][i * P.nf] >> b) & 1u;
        f[t] = occ ? (double)G[t] * nm * P.sunit : 0.0;
    }
}

static rt_status shared_sigma_io(rt_ctx *c, double *f, int to_dev, int where, void *stream) {
    if (!c || !f || (where != RT_HOST && where != RT_DEVICE)) return RT_ERR_INVALID;
    if (!c->d.shared) return rt_fail(c, RT_ERR_INVALID, "no shared frequency bin in this context");
    cudaStream_t st = (cudaStream_t)stream;
    long long m = c->d.n * c->d.nrc;
    double *t = dtmp<double>(m);
    if (!t) return rt_fail(c, RT_ERR_OOM, "temp");
    rt_status s = RT_OK;
    if (to_dev && (s = copy_in(c, t, f, sizeof(double) * m, where, st))) {
        cudaFree(t);
        return s;
    }
    unsigned nb = (unsigned)((m + 255) / 256);
    if (c->d.fp32) k_shared_sigma_io<float><<<nb, 256, 0, st>>>(c->d, c->cur, t, to_dev);
    else k_shared_sigma_io<double><<<nb, 256, 0, st>>>(c->d, c->cur, t, to_dev);
    if (!to_dev) s = copy_out(c, f, t, sizeof(double) * m, where, st);
    rt_status s2 = rt_cuda_check(c, cudaStreamSynchronize(st), "shared sigma");
    cudaFree(t);
    return s ? s : s2;
}

extern "C" rt_status rt_get_shared_sigma(rt_ctx *c, double *G, int where, void *stream) {
    return shared_sigma_io(c, G, 0, where, stream);
}

extern "C" rt_status rt_set_shared_sigma(rt_ctx *c, const double *G, int where, void *stream) {
    return shared_sigma_io(c, const_cast<double *>(G), 1, where, stream);
}

__global__ void k_deposits(DevPtrs P, double *a, double *e, double *ps) {
    long long key = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= P.n * P.nf) return;
    long long i = key / P.nf;
    ps[key] = P.pass[key] + (double)P.passf[key] * P.norm[P.pbox[i]];
    // the fixed-point words count in units of the neutral atoms at the start of the step (the
    // n_HI frozen for the transport), not of the x_HI the chemistry has written since
    double NHI = P.nH[i] > 0.0 ? P.nHI[i] / P.nH[i] * P.NH[i] : 0.0;
    a[key] = P.abs[key] + ((double)P.fx_abs[key] + (double)P.fx_lo[key] / FX_LO_SCALE) *
                              (NHI / FX_ABS_SCALE);
    e[key] = P.absE[key] + (double)P.fx_E[key] * (NHI * 1.602176634e-12 / FX_E_SCALE);
}

extern "C" rt_status rt_get_deposits(rt_ctx *c, double *abs_, double *absE, double *pass,
                                     int where, void *stream) {
    if (!c) return RT_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    long long m = c->d.n * c->d.nf;
    double *t = dtmp<double>(3 * m);
    if (!t) return rt_fail(c, RT_ERR_OOM, "temp");
    k_deposits<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(c->d, t, t + m, t + 2 * m);
    rt_status s;
    if ((s = copy_out(c, abs_, t, sizeof(double) * m, where, st)) ||
        (s = copy_out(c, absE, t + m, sizeof(double) * m, where, st)) ||
        (s = copy_out(c, pass, t + 2 * m, sizeof(double) * m, where, st))) {
        cudaFree(t);
        return s;
    }
    cudaStreamSynchronize(st);
    cudaFree(t);
    return RT_OK;
}

extern "C" rt_status rt_get_stats(rt_ctx *c, long long *out) {
    if (!c || !out) return RT_ERR_INVALID;
    for (int k = 0; k < RT_NSTATS; ++k) out[k] = c->stats[k];
    out[13] = c->cell_occ;
    rt_launch_grids(c, out + 14);
    out[17] = c->cand_entries;
    out[18] = c->cand_fallback;
    return RT_OK;
}

extern "C" const char *rt_last_error(const rt_ctx *c) { return c ? c->err.c_str() : "null context"; }
