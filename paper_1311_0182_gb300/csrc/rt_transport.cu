// rt_transport.cu -- one RT step on the GPU (Sec. 2.1 and Sec. 2.2 of the paper).
//
// Packets live in per-particle slots (reception cone b, frequency bin nu), double-buffered
// across hops.  One hop:
//   A  sender side, warp per gas particle (lanes = neighbours): for every packet able to move,
//      the transmission-cone membership of each neighbour (ballot), the equal share w = N/n,
//      and a transposed bitmap (sender, neighbour, nu) -> bins; empty cones request a virtual
//      particle.  Free packets (source packets in the first hop, virtual particles after) do
//      the same with their own neighbour lists and stage their contributions.
//   V  warp per virtual-particle request: position inside the cone (counter-based draws),
//      escape test, exact kNN of the point, SPH-interpolated n_HI, attenuation; absorptions
//      go to the neighbours as fixed-point integer sums (order-independent, so reproducible);
//      the transmitted packet becomes a free packet of the next hop.
//   B  receiver side, group of n_rc lanes per (particle, nu), lane = reception cone: walks the
//      particle's reverse neighbour list in sender order, expands the bitmap bits into
//      contributions, attenuates, picks the reception cone, and merges in a fixed order
//      (sender, slot); then the staged free-packet contributions in (packet, neighbour) order.
//      No floating-point atomics: every sum has one fixed order.
#include <algorithm>
#include <climits>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "rt_knn.cuh"

static const double C_LIGHT = 2.99792458e10;
static const double EV_ERG = 1.602176634e-12;

// the two isotropic direction sets (index 0: 8 directions, 1: 32), FP64 and FP32 copies
__constant__ double c_axd[2][96];
__constant__ float c_axf[2][96];
// FP32 copy in global memory for lane-divergent reads, and the candidate table of each set
__device__ float g_axf[2][96];
__device__ unsigned g_bin_tab[2][BIN_TAB_M * BIN_TAB_M];

// Candidate table of a direction set.  Cell (i, j) of the octahedral map covers
// u in [-1 + 2i/M, -1 + 2(i+1)/M], v likewise; its entry lists (one byte each, 0xff unused) the
// directions D_b that can be the nearest for some direction p of the cell, i.e. whose gap
// f_b(p) = p.D_b - max_a p.D_a comes near zero there.  f_b is 2-Lipschitz in p, and the
// inverse map (u, v) -> p is 3-Lipschitz (the point on the octahedron moves by at most
// sqrt(3) |d(u, v)| and has norm >= 1/sqrt(3)), so sampling the cell on a grid of spacing sp
// bounds f_b everywhere in it to within 2 * 3 * sp / sqrt(2) of the sampled maximum.
static void build_bin_table(const double *D, int nax, unsigned *tab) {
    const int M = BIN_TAB_M, S = 17;
    const double sp = 2.0 / (M * (S - 1.0));
    const double thr = -(6.0 * sp / sqrt(2.0) + 1e-3);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double fmax[32];
            for (int k = 0; k < nax; ++k) fmax[k] = -1e30;
            for (int a = 0; a < S; ++a)
                for (int b = 0; b < S; ++b) {
                    double u = -1.0 + 2.0 * (i + a / (S - 1.0)) / M;
                    double v = -1.0 + 2.0 * (j + b / (S - 1.0)) / M;
                    double x = u, y = v, z = 1.0 - fabs(u) - fabs(v);
                    if (z < 0.0) {
                        x = (u < 0.0 ? -1.0 : 1.0) * (1.0 - fabs(v));
                        y = (v < 0.0 ? -1.0 : 1.0) * (1.0 - fabs(u));
                    }
                    double nn = sqrt(x * x + y * y + z * z);
                    x /= nn; y /= nn; z /= nn;
                    double sc[32], best = -2.0;
                    for (int k = 0; k < nax; ++k) {
                        sc[k] = x * D[3 * k] + y * D[3 * k + 1] + z * D[3 * k + 2];
                        best = std::max(best, sc[k]);
                    }
                    for (int k = 0; k < nax; ++k) fmax[k] = std::max(fmax[k], sc[k] - best);
                }
            unsigned w = 0xffffffffu;
            int cnt = 0;
            for (int k = 0; k < nax; ++k) {
                if (!(fmax[k] > thr)) continue;
                if (cnt < 4) w = (w & ~(0xffu << (8 * cnt))) | ((unsigned)k << (8 * cnt));
                ++cnt;
            }
            tab[i * M + j] = cnt <= 4 ? w : BIN_TAB_ALL;
        }
}

#define BIN_BAND 2e-5f
// Reception cone of direction d at a particle with rotation R: argmax_b (R^T d) . D_b, first
// maximum on ties.  FP32 scores of the cell's candidates with a guard band on the margin
// between the two best; inside the band (or for a tie) the exact FP64 scan decides.  Every
// direction left out of a cell is more than 1e-3 below the best everywhere in the cell, far
// beyond the FP32 error (~1e-6), so the fast answer is the exact argmax.
template <typename Real>
__device__ inline int bin_fast(const float *Rf, const double *Rd, int ax, int nrc, Real d0,
                               Real d1, Real d2) {
    float f0 = (float)d0, f1 = (float)d1, f2 = (float)d2;
    float e0 = __fmaf_rn(Rf[0], f0, __fmaf_rn(Rf[3], f1, Rf[6] * f2));
    float e1 = __fmaf_rn(Rf[1], f0, __fmaf_rn(Rf[4], f1, Rf[7] * f2));
    float e2 = __fmaf_rn(Rf[2], f0, __fmaf_rn(Rf[5], f1, Rf[8] * f2));
    // octahedral map of e onto [-1, 1]^2
    float is = __fdividef(1.0f, fabsf(e0) + fabsf(e1) + fabsf(e2));
    float u = e0 * is, v = e1 * is;
    if (e2 < 0.0f) {
        float uu = copysignf(1.0f - fabsf(v), u), vv = copysignf(1.0f - fabsf(u), v);
        u = uu;
        v = vv;
    }
    int cu = min(max(__float2int_rd((u + 1.0f) * (0.5f * BIN_TAB_M)), 0), BIN_TAB_M - 1);
    int cv = min(max(__float2int_rd((v + 1.0f) * (0.5f * BIN_TAB_M)), 0), BIN_TAB_M - 1);
    unsigned c = __ldg(&g_bin_tab[ax][cu * BIN_TAB_M + cv]);
    const float *axf = g_axf[ax];
    float b1 = -3.0f, b2 = -3.0f;
    int best = 0;
    int nk = c == BIN_TAB_ALL ? nrc : 4;
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        int b = c == BIN_TAB_ALL ? k : (int)((c >> (8 * k)) & 0xffu);
        if (b == 0xff) break;
        float sc = __fmaf_rn(e0, __ldg(&axf[3 * b]),
                             __fmaf_rn(e1, __ldg(&axf[3 * b + 1]), e2 * __ldg(&axf[3 * b + 2])));
        if (sc > b1) { b2 = b1; b1 = sc; best = b; }
        else if (sc > b2) b2 = sc;
    }
    if (b1 - b2 > BIN_BAND) return best;
    return bin_exact(Rd, c_axd[ax], nrc, (double)d0, (double)d1, (double)d2);
}

struct BinTables {
    unsigned t[2][BIN_TAB_M * BIN_TAB_M];
};

void rt_upload_axes() {
    double d[2][96] = {{0}};
    float f[2][96];
    rt_host_axis_set(8, d[0]);
    rt_host_axis_set(32, d[1]);
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 96; ++k) f[a][k] = (float)d[a][k];
    static const BinTables *tab = [&d] {   // built once (thread-safe static initialisation)
        BinTables *t = new BinTables;
        build_bin_table(d[0], 8, t->t[0]);
        build_bin_table(d[1], 32, t->t[1]);
        return t;
    }();
    cudaMemcpyToSymbol(c_axd, d, sizeof(d));
    cudaMemcpyToSymbol(c_axf, f, sizeof(f));
    cudaMemcpyToSymbol(g_axf, f, sizeof(f));
    cudaMemcpyToSymbol(g_bin_tab, tab->t, sizeof(tab->t));
}

// Resident 256-thread blocks per SM asked of the hop kernels: four (64 registers a thread)
// for FP32 packets; three for FP64, whose wider values would otherwise spill.  The virtual
// particles take five with FP32 packets (48 registers, some spilled): the extra warps hide
// more latency than the spills cost (measured on the 64^3 step graph).
#define HOP_MINB(Real) (sizeof(Real) == 4 ? 4 : 3)
#ifndef VIRT_MINB_F32
#define VIRT_MINB_F32 5
#endif
#define VIRT_MINB(Real) (sizeof(Real) == 4 ? VIRT_MINB_F32 : 3)
// Largest grids (blocks) of the sender side, the virtual particles and the receiver side.  On
// the sender and receiver sides each block takes a contiguous chunk of the live items; the
// sizes were set by a measured sweep on the 64^3 HII-region step: fewer, longer-lived blocks
// than one per 32 items, while still several blocks per SM turn over during a launch.
#ifndef GRID_A
#define GRID_A (152 * 16)
#endif
#ifndef GRID_V
#define GRID_V (152 * VIRT_MINB_F32)   // one wave: the virtual particles pull from a work queue
#endif
#ifndef GRID_B
#define GRID_B (152 * 8)
#endif

template <typename Real> struct Slots {
    Real *N, *X, *Y, *Z, *C, *E;
    __device__ __forceinline__ Slots(const DevPtrs &P, int b) {
        N = (Real *)P.sl[b][0]; X = (Real *)P.sl[b][1]; Y = (Real *)P.sl[b][2];
        Z = (Real *)P.sl[b][3]; C = (Real *)P.sl[b][4]; E = (Real *)P.sl[b][5];
    }
};

// phase-A record of a slot: (w, d, clock, eps) in one aligned piece of 8 Real, and with `sg`
// (a slot of a shared frequency bin) the packet's mean cross-section in the seventh
__device__ __forceinline__ void rec_store(void *rec, long long s, float w, float d0, float d1,
                                          float d2, float c, float e, bool sg, float sig) {
    float4 *p = (float4 *)rec + 2 * s;
    p[0] = make_float4(w, d0, d1, d2);
    if (sg) p[1] = make_float4(c, e, sig, 0.0f);
    else *(float2 *)(p + 1) = make_float2(c, e);
}
__device__ __forceinline__ void rec_store(void *rec, long long s, double w, double d0, double d1,
                                          double d2, double c, double e, bool sg, double sig) {
    double2 *p = (double2 *)rec + 4 * s;
    p[0] = make_double2(w, d0);
    p[1] = make_double2(d1, d2);
    p[2] = make_double2(c, e);
    if (sg) p[3] = make_double2(sig, 0.0);
}
__device__ __forceinline__ void rec_load(const void *rec, long long s, float &w, float &d0,
                                         float &d1, float &d2, float &c, float &e, bool sg,
                                         float &sig) {
    const float4 *p = (const float4 *)rec + 2 * s;
    float4 a = p[0];
    w = a.x; d0 = a.y; d1 = a.z; d2 = a.w;
    if (sg) {
        float4 b = p[1];
        c = b.x; e = b.y; sig = b.z;
    } else {
        float2 b = *(const float2 *)(p + 1);
        c = b.x; e = b.y;
    }
}
__device__ __forceinline__ void rec_load(const void *rec, long long s, double &w, double &d0,
                                         double &d1, double &d2, double &c, double &e, bool sg,
                                         double &sig) {
    const double2 *p = (const double2 *)rec + 4 * s;
    double2 a = p[0], b = p[1], d = p[2];
    w = a.x; d0 = a.y; d1 = b.x; d2 = b.y; c = d.x; e = d.y;
    if (sg) sig = p[3].x;
}

// unit direction of a packet from its summed momentum M (the luminosity-weighted mean
// direction of merged packets, Sec. 2.1, Fig. 1b)
__device__ __forceinline__ void packet_dir(double Mx, double My, double Mz, double &d0, double &d1,
                                           double &d2) {
    double nn = sqrt(Mx * Mx + My * My + Mz * Mz);
    if (nn > 0.0) { d0 = Mx / nn; d1 = My / nn; d2 = Mz / nn; }
    else { d0 = 1.0; d1 = 0.0; d2 = 0.0; }
}

// FP32: normalised photon counts can be small enough for |M|^2 to underflow, so scale first.
// Every operation is a correctly rounded IEEE single-precision operation in a fixed order
// (reciprocal, products, (a^2 + b^2) + c^2, square root, reciprocal, products), so the FP32
// direction is a reproducible function of the stored momentum: the exact cone test (FP64, on
// this direction) then decides every membership the same way wherever it is evaluated.
__device__ __forceinline__ void packet_dir(float Mx, float My, float Mz, float &d0, float &d1,
                                           float &d2) {
    float s = fmaxf(fabsf(Mx), fmaxf(fabsf(My), fabsf(Mz)));
    if (s > 0.0f) {
        float is = __frcp_rn(s);
        float a = __fmul_rn(Mx, is), b = __fmul_rn(My, is), c = __fmul_rn(Mz, is);
        float q = __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
        float rn = __frcp_rn(__fsqrt_rn(q));
        d0 = __fmul_rn(a, rn); d1 = __fmul_rn(b, rn); d2 = __fmul_rn(c, rn);
    } else {
        d0 = 1.0f; d1 = 0.0f; d2 = 0.0f;
    }
}

// a / b: IEEE division on the FP64 path (the oracle's arithmetic), a times the correctly
// rounded reciprocal on the FP32 path
template <typename Real> __device__ __forceinline__ Real rdiv(Real a, Real b);
template <> __device__ __forceinline__ double rdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float rdiv<float>(float a, float b) { return a * __frcp_rn(b); }

// precision-matched constants: FP64 values on the FP64 path, FP32 copies on the FP32 path
template <typename Real> __device__ __forceinline__ Real box_unit(const DevPtrs &P, int b);
template <> __device__ __forceinline__ double box_unit<double>(const DevPtrs &P, int b) { return P.box_u[b]; }
template <> __device__ __forceinline__ float box_unit<float>(const DevPtrs &P, int b) { return P.box_uf[b]; }
template <typename Real> __device__ __forceinline__ Real sigma_of(const DevPtrs &P, int nu);
template <> __device__ __forceinline__ double sigma_of<double>(const DevPtrs &P, int nu) { return P.sigma[nu]; }
template <> __device__ __forceinline__ float sigma_of<float>(const DevPtrs &P, int nu) { return P.sigmaf[nu]; }
// the cross-section of a bin in the unit of the shared-bin fields (sunit)
template <typename Real> __device__ __forceinline__ Real sigma_units(const DevPtrs &P, int nu);
template <> __device__ __forceinline__ double sigma_units<double>(const DevPtrs &P, int nu) {
    return P.sigma[nu] / P.sunit;
}
template <> __device__ __forceinline__ float sigma_units<float>(const DevPtrs &P, int nu) {
    return (float)(P.sigma[nu] / P.sunit);
}
template <typename Real> __device__ __forceinline__ Real to_real(long long v);
template <> __device__ __forceinline__ double to_real<double>(long long v) { return (double)v; }
template <> __device__ __forceinline__ float to_real<float>(long long v) { return i64_to_f(v); }

__device__ __forceinline__ unsigned long long to_fixed(double v) { return (unsigned long long)llrint(v); }
__device__ __forceinline__ unsigned long long to_fixed(float v) { return f2u64_rz(v + 0.5f); }

// escaped photons in the fixed-point unit of the box's escape tally
__device__ __forceinline__ unsigned long long esc_fixed(double N, const DevPtrs &P, int box) {
    return (unsigned long long)llrint(N * P.norm[box] / P.ref[box] * FX_ESC_SCALE);
}
__device__ __forceinline__ unsigned long long esc_fixed(float N, const DevPtrs &P, int box) {
    return f2u64_rz(N * P.escf[box] + 0.5f);
}

// ------------------------------------------------------------------------------------------
// per-step kernels
// ------------------------------------------------------------------------------------------
__global__ void k_rotate(DevPtrs P) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long step = P.cnt[CNT_STEP];
    long long nsrc = (long long)P.ns * P.K;
    if (i < P.n) {
        double R[9];
        random_rotation(P.seed, 1u, (unsigned)step, (unsigned)(step >> 32),
                        (unsigned)gid_of(P, i, P.pbox[i]), R);
#pragma unroll
        for (int a = 0; a < 9; ++a) { P.R[i * 9 + a] = R[a]; P.Rf[i * 9 + a] = (float)R[a]; }
    } else if (i < P.n + nsrc) {
        long long t = i - P.n;
        int j = (int)((unsigned)t / (unsigned)P.K), k = (int)((unsigned)t % (unsigned)P.K);
        double R[9];
        random_rotation(P.seed, 2u, (unsigned)step, (unsigned)k, (unsigned)P.sid[j], R);
#pragma unroll
        for (int a = 0; a < 9; ++a) P.Rs[t * 9 + a] = R[a];
    }
}

// Start of step: clock reset and re-binning of held packets into the new reception cones.
template <typename Real, int NRC>
__global__ void k_rebin(DevPtrs P) {
    long long key = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= P.n * P.nf) return;
    int cur = (int)P.cnt[CNT_CUR];
    unsigned o = P.occ[cur][key];
    if (!o) { P.act[cur][key] = 0; return; }
    long long i = (unsigned)key / (unsigned)P.nf;   // keys < 2^31: 32-bit division
    int nu = (int)((unsigned)key % (unsigned)P.nf);
    Slots<Real> S(P, cur);
    long long s0 = i * P.S + (long long)nu * NRC;
    Real nN[NRC], nX[NRC], nY[NRC], nZ[NRC], nE[NRC], nG[NRC];
    Real oN[NRC], oX[NRC], oY[NRC], oZ[NRC], oE[NRC], oG[NRC];
    // a shared frequency bin carries the cross-section sums of bin 0 along
    Real *SG = (P.shared && nu == 0) ? (Real *)P.slG[cur] + i * NRC : nullptr;
    for (int b = 0; b < NRC; ++b) {
        nN[b] = nX[b] = nY[b] = nZ[b] = nE[b] = nG[b] = Real(0);
        if ((o >> b) & 1) {
            oN[b] = S.N[s0 + b]; oX[b] = S.X[s0 + b]; oY[b] = S.Y[s0 + b];
            oZ[b] = S.Z[s0 + b]; oE[b] = S.E[s0 + b];
            oG[b] = SG ? SG[b] : Real(0);
        }
    }
    const double *Rd = P.R + i * 9;
    const float *Rf = P.Rf + i * 9;
    for (int b = 0; b < NRC; ++b) {
        if (!((o >> b) & 1) || !(oN[b] > Real(0))) continue;
        Real d0, d1, d2;
        packet_dir(oX[b], oY[b], oZ[b], d0, d1, d2);
        int nb = bin_fast<Real>(Rf, Rd, P.ax_rc, NRC, d0, d1, d2);
        nN[nb] += oN[b]; nX[nb] += oX[b]; nY[nb] += oY[b]; nZ[nb] += oZ[b]; nE[nb] += oE[b];
        nG[nb] += oG[b];
    }
    unsigned no = 0;
    for (int b = 0; b < NRC; ++b) {
        if (nN[b] > Real(0)) {
            no |= 1u << b;
            S.N[s0 + b] = nN[b]; S.X[s0 + b] = nX[b]; S.Y[s0 + b] = nY[b];
            S.Z[s0 + b] = nZ[b]; S.C[s0 + b] = Real(0); S.E[s0 + b] = nE[b];
            if (SG) SG[b] = nG[b];
        }
    }
    P.occ[cur][key] = no;
    P.act[cur][key] = no;   // clocks restart: every held packet can move again
}

// Recombination emission into the reception cones, counter reset, frozen n_HI.
template <typename Real, int NRC>
__global__ void k_emit_rec(DevPtrs P) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    int cur = (int)P.cnt[CNT_CUR];
    int b = P.pbox[i];
    double nm = P.norm[b];
    for (int nu = 0; nu < P.nf; ++nu) {
        long long key = i * P.nf + nu;
        P.abs[key] = 0.0; P.absE[key] = 0.0; P.pass[key] = 0.0;
        P.fx_abs[key] = 0ull; P.fx_lo[key] = 0ull; P.fx_E[key] = 0ull; P.passf[key] = 0.0f;
    }
    double x = P.xHI[i], nH = P.nH[i], NH = P.NH[i];
    double nHI = __dmul_rn(x, nH);
    P.nHI[i] = nHI;
    ((Real *)P.nHIr)[i] = (Real)nHI;
    ((Real *)P.Vr)[i] = (Real)(NH / nH / P.vunit[b]);   // volume in the box's volume unit
    double NHI = x * NH;
    ((Real *)P.dep_s)[i] = NHI > 0.0 ? (Real)(FX_ABS_SCALE * nm / NHI) : Real(0);
    ((Real *)P.depE_s)[i] = NHI > 0.0 ? (Real)(FX_E_SCALE * nm * P.eunit / (NHI * EV_ERG)) : Real(0);
    double Nr = P.Nrec[i];
    if (!(Nr > 0.0) || P.rec_mode == RT_REC_EMISSION_CONES) return;
    double e_phys = Nr / (double)NRC;
    Real e = (Real)(e_phys / nm);
    Real epsr = (Real)(P.epsrec[i] / P.eunit);
    int nu = P.rbin;       // the recombination bin, or source bin 0 when the bin is shared
    long long key = i * P.nf + nu;
    unsigned o = P.occ[cur][key], a = P.act[cur][key];
    Slots<Real> S(P, cur);
    long long s0 = i * P.S + (long long)nu * NRC;
    // shared bin: each cone gains e sigma_rec of cross-section sum
    Real *SG = P.shared ? (Real *)P.slG[cur] + i * NRC : nullptr;
    Real eg = e * (Real)(P.sigma_rec / P.sunit);
    const double *R = P.R + i * 9;
    for (int bb = 0; bb < NRC; ++bb) {
        double A[3];
        rot_apply(R, c_axd[P.ax_rc] + 3 * bb, A);
        long long s = s0 + bb;
        if ((o >> bb) & 1) {
            S.N[s] += e; S.X[s] += e * (Real)A[0]; S.Y[s] += e * (Real)A[1];
            S.Z[s] += e * (Real)A[2]; S.E[s] += e * epsr;
            if (SG) SG[bb] += eg;
        } else {
            S.N[s] = e; S.X[s] = e * (Real)A[0]; S.Y[s] = e * (Real)A[1];
            S.Z[s] = e * (Real)A[2]; S.C[s] = Real(0); S.E[s] = e * epsr;
            if (SG) SG[bb] = eg;
        }
        if (e > Real(0)) { o |= 1u << bb; a |= 1u << bb; }
    }
    P.occ[cur][key] = o;
    P.act[cur][key] = a;
}

// Source packets of the step: K emissions x n_freq_src bins x n_ec cones per source, written
// to free buffer 0 (the first hop's).
template <typename Real>
__global__ void k_emit_src(DevPtrs P) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long per_src = (long long)P.K * P.nfs * P.nec;
    if (p >= (long long)P.ns * per_src) return;
    unsigned ps = (unsigned)per_src, tt = (unsigned)(p % ps);
    int j = (int)((unsigned)p / ps);
    int k = (int)(tt / (unsigned)(P.nfs * P.nec));
    int nu = (int)((tt / (unsigned)P.nec) % (unsigned)P.nfs);
    int e = (int)(tt % (unsigned)P.nec);
    FreeBuf F = P.fr[0];
    int b = P.sbox[j];
    // a gated source emits only while its nearest gas particle is more than half ionised; a
    // directed source sends one packet per emission and frequency (cone 0) along its direction
    const double *dir = P.sdir + 3 * (long long)j;
    bool directed = dir[0] != 0.0 || dir[1] != 0.0 || dir[2] != 0.0;
    bool on = !P.sgate[j] || P.xHI[P.snbr[(long long)j * P.kn]] < 0.5;
    double nd = P.ndot[(long long)j * P.nfs + nu];
    double N = 0.0, d[3];
    if (directed) {
        if (on && e == 0) N = __dmul_rn(nd, P.dt_em);
        d[0] = dir[0]; d[1] = dir[1]; d[2] = dir[2];
    } else {
        if (on) N = __ddiv_rn(__dmul_rn(nd, P.dt_em), (double)P.nec);
        rot_apply(P.Rs + ((long long)j * P.K + k) * 9, c_axd[P.ax_ec] + 3 * e, d);
    }
    F.box[p] = b;
    F.qx[p] = P.sqx[j]; F.qy[p] = P.sqy[j]; F.qz[p] = P.sqz[j];
    for (int a = 0; a < P.kn; ++a) F.nbr[p * P.kn + a] = P.snbr[(long long)j * P.kn + a];
    F.h2[p] = P.sh2[j];
    ((Real *)F.N)[p] = (Real)(N / P.norm[b]);
    ((Real *)F.dx)[p] = (Real)d[0];
    ((Real *)F.dy)[p] = (Real)d[1];
    ((Real *)F.dz)[p] = (Real)d[2];
    ((Real *)F.clock)[p] = Real(0);
    ((Real *)F.eps)[p] = (Real)(P.eps[nu] / P.eunit);
    if (P.shared) ((Real *)F.sig)[p] = sigma_units<Real>(P, nu);
    F.nu[p] = nu;
    // identity (source, emission, frequency, cone), with the source's identity
    F.fid[p] = (1ull << 62) |
               ((((unsigned long long)P.sid[j] * P.K + k) * P.nfs + nu) * P.nec + e);
}

// The original implementation of recombination radiation (Sec. 2.2): particle i emits, K
// times a step, n_ec packets of N_rec / (K n_ec) photons along its emission axes, rotated at
// random before each emission; they are free packets at the particle's position with its
// neighbour list, written to free buffer 0 after the source packets (index
// base + (i K + k) n_ec + e).
// Particles without recombination photons leave packets of N = 0, which never move.
template <typename Real>
__global__ void k_emit_rec_cones(DevPtrs P, long long base) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long per = (long long)P.K * P.nec;
    if (p >= P.n * per) return;
    long long step = P.cnt[CNT_STEP];
    long long i = p / per;
    int k = (int)((p % per) / P.nec), e = (int)(p % P.nec);
    FreeBuf F = P.fr[0];
    long long f = base + p;
    int b = P.pbox[i];
    double Nr = P.Nrec[i];
    double N = Nr > 0.0 ? __ddiv_rn(Nr, (double)per) : 0.0;
    double R[9], d[3];
    const unsigned long long gi = gid_of(P, i, b);
    random_rotation(P.seed, 4u, (unsigned)step, (unsigned)k, (unsigned)gi, R);
    rot_apply(R, c_axd[P.ax_ec] + 3 * e, d);
    F.box[f] = b;
    F.qx[f] = P.qx[i]; F.qy[f] = P.qy[i]; F.qz[f] = P.qz[i];
    for (int a = 0; a < P.kn; ++a) F.nbr[f * P.kn + a] = P.nbr[i * P.kn + a];
    F.h2[f] = P.h2[i];
    ((Real *)F.N)[f] = (Real)(N / P.norm[b]);
    ((Real *)F.dx)[f] = (Real)d[0];
    ((Real *)F.dy)[f] = (Real)d[1];
    ((Real *)F.dz)[f] = (Real)d[2];
    ((Real *)F.clock)[f] = Real(0);
    ((Real *)F.eps)[f] = (Real)(P.epsrec[i] / P.eunit);
    if (P.shared) ((Real *)F.sig)[f] = (Real)(P.sigma_rec / P.sunit);
    F.nu[f] = P.rbin;
    F.fid[f] = (2ull << 62) | ((gi * P.K + k) * P.nec + e);   // (particle, emission, cone)
}

// ------------------------------------------------------------------------------------------
// hop kernels
// ------------------------------------------------------------------------------------------
// Sender side.  Warp per particle.  The particle's packets able to move are taken 32 at a
// time (lane = packet: load, direction, clock), then tested one after the other against the
// neighbours (lane = neighbour k: cone membership, ballot).  For each (frequency, neighbour)
// the bits of the packets whose cone holds the neighbour go to the neighbour's receiver-ordered
// bitmap word; empty cones become virtual-particle requests.
// cur: the slot buffer holding the hop's packets.  Receivers of a bitmap word are flagged in
// `touched` (cleared again by the work-list kernel).
// SH: the shared frequency bin (a separate instance keeps its code out of the common case)
template <typename Real, int NRC, bool SH>
__global__ void __launch_bounds__(256, HOP_MINB(Real)) k_phaseA(DevPtrs P, int cur) {
    int lane = threadIdx.x & 31;
    Slots<Real> S(P, cur);
    float cf = 1.0f - 2.0f / (float)P.ntc;
    long long nrev = P.n * P.kn;
    long long ncon = 0;
    // each block takes one contiguous chunk of particles; its warps pull particles from it
    // through a shared counter, so that they finish together (particles hold from none to
    // hundreds of packets)
    __shared__ int snext;
    long long chunk = (P.n + gridDim.x - 1) / gridDim.x;
    long long ib0 = (long long)blockIdx.x * chunk;
    long long ib1 = ib0 + chunk < P.n ? ib0 + chunk : P.n;
    if (threadIdx.x == 0) snext = 0;
    __syncthreads();
    auto next_particle = [&]() {
        long long v = 0;
        if (lane == 0) v = ib0 + atomicAdd(&snext, 1);
        return __shfl_sync(FULLMASK, v, 0);
    };
    for (long long i = next_particle(); i < ib1; i = next_particle()) {
        unsigned aw = (lane < P.nf) ? P.act[cur][i * P.nf + lane] : 0u;
        if (__ballot_sync(FULLMASK, aw != 0u) == 0u) {
            if (lane == 0) P.reqcnt[i] = 0;
            continue;
        }
        // neighbour k = lane
        int nb = 0, dx = 0, dy = 0, dz = 0, rp = 0;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        bool valid = lane < P.kn;
        if (valid) {
            long long f = i * P.kn + lane;
            nb = P.nbr[f];
            rp = P.revpos[f];
            fx = P.fdx[f]; fy = P.fdy[f]; fz = P.fdz[f];
            dx = (int)fx; dy = (int)fy; dz = (int)fz;
        }
        // active packets in (nu, b) order: prefix of the per-frequency counts
        int cnt = __popc(aw);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(FULLMASK, incl, o);
            if (lane >= o) incl += v;
        }
        int total = __shfl_sync(FULLMASK, incl, 31);
        int excl = incl - cnt;
        int nreq = 0;
        unsigned emp_acc = 0u;        // lane nu: empty-cone bits of frequency nu
        unsigned word = 0u;           // lane k: the current bitmap word and its frequency
        int cur_nu = -1;
        for (int cb = 0; cb < total; cb += 32) {
            // lane t takes packet cb + t: its frequency (owner lane) and bin
            int t = cb + lane;
            int onu = 0;
            for (int q = 1; q < P.nf; ++q) {
                int eq = __shfl_sync(FULLMASK, excl, q);
                if (eq <= t) onu = q;
            }
            unsigned ow = __shfl_sync(FULLMASK, aw, onu);
            int oex = __shfl_sync(FULLMASK, excl, onu);
            bool has = t < total;
            int ob = has ? __fns(ow, 0, t - oex + 1) : 0;
            long long s = i * P.S + (long long)onu * NRC + ob;
            Real N = Real(0), d0 = Real(1), d1 = Real(0), d2 = Real(0), C = Real(0), E = Real(0);
            Real sgr = Real(0);
            bool sgs = SH && onu == 0;   // a slot of the shared bin: its mean cross-section
            if (has) {
                N = S.N[s];
                packet_dir(S.X[s], S.Y[s], S.Z[s], d0, d1, d2);
                C = S.C[s];
                E = S.E[s];
                if (sgs) sgr = ((Real *)P.slG[cur])[i * NRC + ob] / N;
            }
            int nb_chunk = min(32, total - cb);
            int my_cm = 0;
            // the chunk's packets one after the other (lane = neighbour k): cone membership; the
            // bitmap word of lane k collects, frequency by frequency, the bins whose cone holds
            // k (a word continues across chunks while the frequency does); a cone with no member
            // adds its bin to the empty-cone word of its frequency, held on lane nu
            for (int u = 0; u < nb_chunk; ++u) {
                Real e0 = __shfl_sync(FULLMASK, d0, u), e1 = __shfl_sync(FULLMASK, d1, u),
                     e2 = __shfl_sync(FULLMASK, d2, u);
                int unu = __shfl_sync(FULLMASK, onu, u);
                int ub = __shfl_sync(FULLMASK, ob, u);
                bool in = valid && cone_test<Real>(dx, dy, dz, fx, fy, fz, e0, e1, e2, cf, P.ntc);
                unsigned m = __ballot_sync(FULLMASK, in);
                if (lane == u) my_cm = __popc(m);
                if (unu != cur_nu) {
                    if (valid && word) {
                        P.bm[(long long)cur_nu * nrev + rp] = word;
                        P.touched[(long long)nb * P.nf + cur_nu] = 1;
                    }
                    word = 0u;
                    cur_nu = unu;
                }
                if (in) word |= 1u << ub;
                if (m == 0u && lane == unu) emp_acc |= 1u << ub;
            }
            ncon += (lane < nb_chunk) ? my_cm : 0;
            if (has && my_cm > 0)
                rec_store(P.rec, s, rdiv<Real>(N, (Real)my_cm), d0, d1, d2, rdiv<Real>(C, N),
                          rdiv<Real>(E, N), sgs, sgr);
            nreq += __popc(__ballot_sync(FULLMASK, has && my_cm == 0));
        }
        // every word starts the hop at zero (the receiver side clears the words it reads), and
        // each (frequency, neighbour) word is written once: a plain store
        if (valid && word) {
            P.bm[(long long)cur_nu * nrev + rp] = word;
            P.touched[(long long)nb * P.nf + cur_nu] = 1;
        }
        if (lane < P.nf) P.emp[i * P.nf + lane] = emp_acc;
        if (lane == 0) P.reqcnt[i] = nreq;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ncon += __shfl_down_sync(FULLMASK, ncon, o);
    if (lane == 0 && ncon) atomicAdd((unsigned long long *)&P.cnt[CNT_GCON], (unsigned long long)ncon);
}

// Free packets: cone membership over their own neighbour lists.
template <typename Real>
__global__ void __launch_bounds__(256) k_freeA(DevPtrs P, int fcur, const int *lens,
                                               unsigned *fmask, int *stcnt) {
    int lane = threadIdx.x & 31;
    long long nfree = lens[0];
    long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    FreeBuf F = P.fr[fcur];
    float cf = 1.0f - 2.0f / (float)P.ntc;
    for (long long f = w0; f < nfree; f += nw) {
        Real N = ((Real *)F.N)[f];
        if (!(N > Real(0))) {
            if (lane == 0) { fmask[f] = 0u; stcnt[f] = 0; P.reqcnt[P.n + f] = 0; }
            continue;
        }
        Real d0 = ((Real *)F.dx)[f], d1 = ((Real *)F.dy)[f], d2 = ((Real *)F.dz)[f];
        bool in = false;
        if (lane < P.kn) {
            long long j = F.nbr[f * P.kn + lane];
            int dx = P.qx[j] - F.qx[f], dy = P.qy[j] - F.qy[f], dz = P.qz[j] - F.qz[f];
            in = cone_test<Real>(dx, dy, dz, (float)dx, (float)dy, (float)dz, d0, d1, d2, cf, P.ntc);
        }
        unsigned m = __ballot_sync(FULLMASK, in);
        if (lane == 0) {
            fmask[f] = m;
            stcnt[f] = __popc(m);
            P.reqcnt[P.n + f] = (m == 0u) ? 1 : 0;
        }
    }
}

// Free packets with cone members: stage one contribution per member, in (packet, neighbour)
// order at the positions given by the scan of the member counts.
template <typename Real, int NRC, bool BAR, bool SH>
__global__ void __launch_bounds__(256) k_freeC(DevPtrs P, int fcur, const int *lens,
                                               const unsigned *fmask, const int *stoff) {
    int lane = threadIdx.x & 31;
    long long nfree = lens[0];
    long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    FreeBuf F = P.fr[fcur];
    for (long long f = w0; f < nfree; f += nw) {
        unsigned m = fmask[f];
        if (!m) continue;
        if (!((m >> lane) & 1u)) continue;
        int rank = __popc(m & ((1u << lane) - 1u));
        long long s = (long long)stoff[f] + rank;
        if (s >= P.ST_cap) {
            atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_STAGE_CAP);
            continue;
        }
        Real N = ((Real *)F.N)[f];
        Real w = N / (Real)__popc(m);
        Real d0 = ((Real *)F.dx)[f], d1 = ((Real *)F.dy)[f], d2 = ((Real *)F.dz)[f];
        Real clk = ((Real *)F.clock)[f], eps = ((Real *)F.eps)[f];
        int nu = F.nu[f];
        // the packet's cross-section: its own mean in a shared bin, else its bin's
        bool sgs = SH && nu == 0;
        Real sg = sgs ? ((Real *)F.sig)[f] : Real(0);
        long long j = F.nbr[f * P.kn + lane];
        int b = P.pbox[j];
        long long key = j * P.nf + nu;
        Real **V = (Real **)P.st_v;
        if (BAR && barrier_crosses_call(P.bar[b], F.qx[f], F.qy[f], F.qz[f], P.qx[j], P.qy[j],
                                         P.qz[j])) {
            // the share crosses the barrier: removed (counted escaped); the staged
            // contribution is empty
            atomicAdd(&P.esc_fx[b], esc_fixed(w, P, b));
            P.st_key[s] = (int)key;
            P.st_bin[s] = -1;            // the receiver side skips it
            atomicAdd(&P.seg_cnt[key], 1);
            continue;
        }
        Real t = (Real)(P.qx[j] - F.qx[f]) * d0 + (Real)(P.qy[j] - F.qy[f]) * d1 +
                 (Real)(P.qz[j] - F.qz[f]) * d2;
        Real l = t * box_unit<Real>(P, b);
        Real sig = sgs ? sg * (Real)P.sunit : sigma_of<Real>(P, nu);
        Real tau = (sig * ((Real *)P.nHIr)[j]) * l;
        Real A, T;
        split_absorbed<Real>(w, tau, A, T);
        int bt = bin_fast<Real>(P.Rf + j * 9, P.R + j * 9, P.ax_rc, NRC, d0, d1, d2);
        P.st_key[s] = (int)key;
        P.st_bin[s] = bt;
        V[0][s] = T;
        V[1][s] = T * d0;
        V[2][s] = T * d1;
        V[3][s] = T * d2;
        V[4][s] = T * (clk + l / (Real)C_LIGHT);
        V[5][s] = T * eps;
        V[6][s] = A;
        V[7][s] = A * eps;
        V[8][s] = w;
        if (sgs) V[9][s] = T * sg;
        atomicAdd(&P.seg_cnt[key], 1);
    }
}

// request list: gas slots with empty cones (particle order, slot order), then free packets
// (grid-stride: a launch sized for the free-packet capacity covers any count).  Its first
// thread also books the hop's request count and checks the capacities (after the request
// scan and the staging scan).
__global__ void k_expand(DevPtrs P, const int *lens) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long *cnt = P.cnt;
        long long nr = lens[2];
        if (nr > P.F_cap)
            atomicOr((unsigned long long *)&cnt[CNT_ERR], (unsigned long long)ERRB_FREE_CAP);
        cnt[CNT_NREQ] = nr;
        cnt[CNT_VIRT] += nr < P.F_cap ? nr : P.F_cap;
        if (lens[3] > P.ST_cap)
            atomicOr((unsigned long long *)&cnt[CNT_ERR], (unsigned long long)ERRB_STAGE_CAP);
    }
    long long nfree = lens[0];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < P.n + nfree;
         t += (long long)gridDim.x * blockDim.x) {
        if (!P.reqcnt[t]) continue;
        long long o = P.reqoff[t];
        if (t < P.n) {
            for (int nu = 0; nu < P.nf; ++nu) {
                unsigned e = P.emp[t * P.nf + nu];
                while (e) {
                    int b = __ffs(e) - 1;
                    e &= e - 1u;
                    if (o < P.F_cap) P.req[o] = (unsigned long long)(t * P.S + (long long)nu * P.nrc + b);
                    else atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_FREE_CAP);
                    ++o;
                }
            }
        } else {
            long long f = t - P.n;
            if (o < P.F_cap) P.req[o] = RT_FREE_BIT | (unsigned long long)f;
            else atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_FREE_CAP);
        }
    }
}

// No accepted draw: the point on the packet's axis at h/2 (at least one quantum), rounded to
// the nearest integer offset.  FP64 path: in FP64.  FP32 path: in FP32 (fh = H/2 is exact,
// the product is rounded once), so no FP64 instruction runs in the hop loop.
__device__ __forceinline__ void axis_offset(double d0, double d1, double d2, long long H,
                                            int &Dx, int &Dy, int &Dz) {
    double fh = 0.5 * (double)H;
    if (fh < 1.0) fh = 1.0;
    Dx = (int)rint(__dmul_rn(d0, fh));
    Dy = (int)rint(__dmul_rn(d1, fh));
    Dz = (int)rint(__dmul_rn(d2, fh));
}
__device__ __forceinline__ void axis_offset(float d0, float d1, float d2, long long H,
                                            int &Dx, int &Dy, int &Dz) {
    float fh = fmaxf(0.5f * (float)(int)H, 1.0f);   // H < 2^21
    Dx = __float2int_rn(__fmul_rn(d0, fh));
    Dy = __float2int_rn(__fmul_rn(d1, fh));
    Dz = __float2int_rn(__fmul_rn(d2, fh));
}

// A virtual-particle request decoded: the packet, its sender's position and smoothing length,
// and the per-box and per-frequency values the request needs.
template <typename Real> struct VDec {
    long long h2, boff;
    unsigned long long fid;
    Real N, d0, d1, d2, clk, eps, sg, sig, bu;
    int box, qx, qy, qz, nu, H;
};
// requests a warp takes together: one lane decodes each, into shared memory
#ifndef VREQ_GROUP
#define VREQ_GROUP 4
#endif

// Virtual particles (Sec. 2.1): one warp per request.
// BAR: some box has a barrier (a separate instance keeps the test out of the common case);
// SH: the shared frequency bin (likewise); IB: index bits of the kNN keys (24 when a box holds
// more than 2^22 particles); FB: some cell has no candidate list, and queries there take the
// grid walk (a separate instance keeps that call, and the registers it costs, out of the
// common case)
// cur, fcur: the hop's slot and free-packet buffers (launch parameters, so that buffer
// pointers are re-read from the parameter space instead of being held in registers); the
// step and hop of the random draws are read from the device counters where they are used.
template <typename Real, int NRC, bool BAR, bool SH, int IB, bool FB>
__global__ void __launch_bounds__(256, VIRT_MINB(Real)) k_virtual(DevPtrs P, int cur, int fcur,
                                                 const int *lens, unsigned long long *esc_r,
                                                 unsigned char *vstat) {
    int lane = threadIdx.x & 31;
    long long nreq = lens[2];
    if (nreq > P.F_cap) nreq = P.F_cap;
    FreeBuf Fi = P.fr[fcur], Fo = P.fr[fcur ^ 1];
    Slots<Real> S(P, cur);
    uint2 key = philox_key(P.seed, 3u);
    // A warp takes VREQ_GROUP consecutive requests at a time; lane v decodes request v of the
    // group (slot or free packet, direction, clock, identity, per-box and per-frequency values)
    // into shared memory, so that the group's loads and divisions run side by side instead of
    // once per request on every lane.  Then the warp serves the requests one after the other.
    // Latency: the kNN search loads each batch of its cell's candidates before merging the
    // previous one; the four per-neighbour inputs of the interpolation and deposit are gathered
    // together; the values returned by the deposit atomics are checked one request later.
    // Work queue: every warp of the launch takes its next group from one device counter
    // (CNT_VQ, set to zero before the hop), so all resident warps stay busy until the requests
    // run out, whatever each request costs; the grid is one wave of resident blocks.  (Blocks
    // that own a fixed chunk each leave most of their warps idle while the slowest finishes:
    // 25 of 40 warps per SM were active.)  Results do not depend on which warp takes a request.
    __shared__ VDec<Real> sdec[8][VREQ_GROUP];
    __shared__ int sdelta[FB ? 8 : 1][32];   // the grid walk of cells without a candidate list
    VDec<Real> *mine = sdec[threadIdx.x >> 5];
    unsigned long long *queue = (unsigned long long *)&P.cnt[CNT_VQ];
    const float cf = 1.0f - 2.0f / (float)P.ntc;
    unsigned long long pend_a = 0ull, pend_e = 0ull;   // words before this lane's last adds
    bool bad = false, bad_knn = false;
    for (;;) {
        long long g0 = 0;
        if (lane == 0) g0 = (long long)atomicAdd(queue, (unsigned long long)VREQ_GROUP);
        g0 = __shfl_sync(FULLMASK, g0, 0);
        if (g0 >= nreq) break;
        const int gn = (int)(nreq - g0 < VREQ_GROUP ? nreq - g0 : VREQ_GROUP);
        if (lane < gn) {
            unsigned long long code = P.req[g0 + lane];
            VDec<Real> D;
            D.sg = Real(0);          // shared bin: the packet's mean cross-section (sunit)
            if (!(code & RT_FREE_BIT)) {
                long long i = (unsigned)code / (unsigned)P.S;   // slot codes < 2^31
                int s = (int)((unsigned)code % (unsigned)P.S);
                D.nu = s / NRC;
                D.box = P.pbox[i];
                D.qx = P.qx[i]; D.qy = P.qy[i]; D.qz = P.qz[i];
                D.h2 = P.h2[i];
                D.N = S.N[code];
                packet_dir(S.X[code], S.Y[code], S.Z[code], D.d0, D.d1, D.d2);
                D.clk = S.C[code] / D.N;
                D.eps = S.E[code] / D.N;
                if (SH && D.nu == 0) D.sg = ((Real *)P.slG[cur])[i * NRC + s] / D.N;
                D.fid = gid_of(P, i, D.box) * P.S + (code - (unsigned long long)i * P.S) + 1ull;
            } else {
                long long f = (long long)(code & ~RT_FREE_BIT);
                D.box = Fi.box[f]; D.qx = Fi.qx[f]; D.qy = Fi.qy[f]; D.qz = Fi.qz[f];
                D.h2 = Fi.h2[f];
                D.N = ((Real *)Fi.N)[f];
                D.d0 = ((Real *)Fi.dx)[f]; D.d1 = ((Real *)Fi.dy)[f]; D.d2 = ((Real *)Fi.dz)[f];
                D.clk = ((Real *)Fi.clock)[f];
                D.eps = ((Real *)Fi.eps)[f];
                D.nu = Fi.nu[f];
                if (SH && D.nu == 0) D.sg = ((Real *)Fi.sig)[f];
                D.fid = Fi.fid[f];
            }
            D.boff = P.box_off[D.box];
            D.sig = (SH && D.nu == 0) ? D.sg * (Real)P.sunit : sigma_of<Real>(P, D.nu);
            D.bu = box_unit<Real>(P, D.box);
            D.H = (int)isqrt64(D.h2);   // = floor(sqrt(h2)) exactly (h2 < 3 * 2^40), < 2^21
            mine[lane] = D;
        }
        __syncwarp();
        for (int v = 0; v < gn; ++v) {
            const long long r = g0 + v;
            const int box = mine[v].box, qx = mine[v].qx, qy = mine[v].qy, qz = mine[v].qz,
                      nu = mine[v].nu;
            const long long h2 = mine[v].h2, boff = mine[v].boff;
            const Real N = mine[v].N, d0 = mine[v].d0, d1 = mine[v].d1, d2 = mine[v].d2,
                       clk = mine[v].clk, eps = mine[v].eps, sg = mine[v].sg, sig = mine[v].sig,
                       bu = mine[v].bu;
            const unsigned long long fid = mine[v].fid;
            const bool sgs = SH && nu == 0;
            // position: first accepted of 64 counter-based draws in [-H, H]^3, else on the axis
            const long long H = mine[v].H;
            unsigned span = (unsigned)(2 * H + 1);   // < 2^22
            int Dx = 0, Dy = 0, Dz = 0;   // |D| <= H < 2^21
            bool found = false;
            for (int a0 = 0; a0 < 64 && !found; a0 += 32) {
                unsigned a = (unsigned)(a0 + lane);
                // counter: (step, hop << 8 | draw, packet id); step and hop from the device counters
                uint4 u = philox4x32_10(make_uint4(cnt_word(P, CNT_STEP), (cnt_word(P, CNT_HOP) << 8) | a,
                                                   (unsigned)fid, (unsigned)(fid >> 32)), key);
                // floor(u * span / 2^32) - H, |e| <= H < 2^21: 32-bit integers (a 64-bit integer to
                // float conversion would run on the FP64 pipe)
                int ix = (int)__umulhi(u.x, span) - (int)H;
                int iy = (int)__umulhi(u.y, span) - (int)H;
                int iz = (int)__umulhi(u.z, span) - (int)H;
                long long ex = ix, ey = iy, ez = iz;
                long long r2 = ex * ex + ey * ey + ez * ez;
                bool ok = r2 > 0 && r2 <= h2 &&
                          cone_test<Real>(ix, iy, iz, (float)ix, (float)iy, (float)iz, d0, d1, d2, cf,
                                          P.ntc);
                unsigned m = __ballot_sync(FULLMASK, ok);
                if (m) {
                    int src = __ffs(m) - 1;
                    Dx = __shfl_sync(FULLMASK, ix, src);
                    Dy = __shfl_sync(FULLMASK, iy, src);
                    Dz = __shfl_sync(FULLMASK, iz, src);
                    found = true;
                }
            }
            if (!found) axis_offset(d0, d1, d2, H, Dx, Dy, Dz);
            int vx = qx + Dx, vy = qy + Dy, vz = qz + Dz;
            // outside the box: the photons escape (vstat 1); on a path through the barrier they
            // are removed, counted with the escapes (vstat 3)
            int gone = (vx < 0 || vy < 0 || vz < 0 || vx >= RT_Q || vy >= RT_Q || vz >= RT_Q) ? 1
                     : (BAR && barrier_crosses_call(P.bar[box], qx, qy, qz, vx, vy, vz)) ? 3 : 0;
            if (gone) {
                if (lane == 0) {
                    esc_r[r] = esc_fixed(N, P, box);
                    vstat[r] = (unsigned char)gone;
                    Fo.box[r] = box;
                    ((Real *)Fo.N)[r] = Real(0);
                }
                continue;
            }
            bad |= pend_a > (1ull << 62) || pend_e > (1ull << 62);
            // exact kNN from the candidate list of the virtual particle's cell (the grid walk
            // in a cell without one)
            long long kd2;
            int kidx;
            bool kok;
            if (FB) {
                kok = vp_knn<IB>(P.grid, box, vx, vy, vz, P.kn, kd2, kidx,
                                 sdelta[FB ? threadIdx.x >> 5 : 0]);
            } else {
                CandQuery Q = cand_query(P.grid, box, vx, vy, vz);
                kok = cand_knn<IB>(Q.items, P.grid.cand, Q.a, Q.e, vx, vy, vz, Q.rq_up, Q.w, P.kn,
                                   kd2, kidx);
            }
            if (!kok) {
                // a k-th neighbour beyond the key range: reported; indices kept inside the box
                bad_knn = true;
                long long nbx = P.box_off[box + 1] - boff;
                if (kidx < 0 || kidx >= nbx) { kidx = 0; kd2 = 0; }
            }
            long long h2v = __shfl_sync(FULLMASK, kd2, P.kn - 1);
            bool valid = lane < P.kn;
            long long j = valid ? boff + kidx : 0;
            Real om = Real(0), nhj = Real(0), Vj = Real(0), dsj = Real(0), dej = Real(0);
            if (valid) {
                Vj = ((Real *)P.Vr)[j];
                nhj = ((Real *)P.nHIr)[j];
                dsj = ((Real *)P.dep_s)[j];
                dej = ((Real *)P.depE_s)[j];
                Real q = h2v > 0 ? rt_sqrt<Real>(to_real<Real>(kd2) / to_real<Real>(h2v)) : Real(0);
                om = Vj * kernel_w<Real>(q);
            }
            Real sw = om;
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(FULLMASK, sw, o);
            if (!(sw > Real(0))) {
                om = Vj;
                sw = om;
    #pragma unroll
                for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(FULLMASK, sw, o);
            }
            Real wn = om * nhj;
            Real swn = wn;
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) swn += __shfl_xor_sync(FULLMASK, swn, o);
            Real nHIv = swn / sw;
            Real t = (Real)Dx * d0 + (Real)Dy * d1 + (Real)Dz * d2;
            Real l = t * bu;
            Real tau = (sig * nHIv) * l;
            Real A, T;
            split_absorbed<Real>(N, tau, A, T);
            if (valid && swn > Real(0) && wn > Real(0)) {
                Real Ak = A * (wn / swn);
                long long key2 = j * P.nf + nu;
                // two fixed-point words: units of 2^-40 N_HI and 2^-72 N_HI (integer sums do not
                // depend on their order)
                Real fa = Ak * dsj;
                Real fe = Ak * eps * dej;
                pend_a = 0ull;
                pend_e = 0ull;
                if (fa > Real(0)) {
                    unsigned long long qh = 0, ql = 0;
                    bad |= !fx_split(fa, qh, ql);
                    if (qh) pend_a = atomicAdd(&P.fx_abs[key2], qh);
                    if (ql) atomicAdd(&P.fx_lo[key2], ql);
                }
                if (fe > Real(0)) {
                    bad |= fe > Real(4.0e18);
                    pend_e = atomicAdd(&P.fx_E[key2], to_fixed(fe));
                }
            }
            if (valid) Fo.nbr[r * P.kn + lane] = (int)j;
            if (lane == 0) {
                esc_r[r] = 0ull;
                vstat[r] = T > Real(0) ? 0 : 2;
                Fo.box[r] = box;
                Fo.qx[r] = vx; Fo.qy[r] = vy; Fo.qz[r] = vz;
                Fo.h2[r] = h2v;
                ((Real *)Fo.N)[r] = T;
                ((Real *)Fo.dx)[r] = d0; ((Real *)Fo.dy)[r] = d1; ((Real *)Fo.dz)[r] = d2;
                ((Real *)Fo.clock)[r] = clk + l / (Real)C_LIGHT;
                ((Real *)Fo.eps)[r] = eps;
                if (sgs) ((Real *)Fo.sig)[r] = sg;
                Fo.nu[r] = nu;
                Fo.fid[r] = mix64(fid);
            }
        }
        __syncwarp();   // the group's decoded requests are read before the next group's decode
    }
    bad |= pend_a > (1ull << 62) || pend_e > (1ull << 62);
    if (bad) atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_RANGE);
    if (bad_knn) atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_KNN);
}

// receiver segments of the staged contributions
__global__ void k_seg_fill(DevPtrs P, const int *lens) {
    long long nst = lens[3];
    if (nst > P.ST_cap) nst = P.ST_cap;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nst;
         s += (long long)gridDim.x * blockDim.x) {
        int key = P.st_key[s];
        int pos = P.seg_off[key] + atomicAdd(&P.seg_fill[key], 1);
        P.seg_idx[pos] = (int)s;
    }
}

__global__ void k_seg_sort(DevPtrs P) {
    long long key = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= P.n * P.nf) return;
    int c = P.seg_cnt[key];
    if (c < 2) return;
    int a = P.seg_off[key], b = a + c;
    for (int p = a + 1; p < b; ++p) {
        int v = P.seg_idx[p];
        int q = p - 1;
        while (q >= a && P.seg_idx[q] > v) {
            P.seg_idx[q + 1] = P.seg_idx[q];
            --q;
        }
        P.seg_idx[q + 1] = v;
    }
}

// The receiver groups with work this hop: receivers touched by a gas sender, receivers of
// staged free-packet contributions, and particles holding waiting packets.  Block-level
// compaction with one atomic per block; the order of the list does not matter.  An entry is
// the key, with bit 31 set when a gas sender touched it (the flag is cleared here).  The next
// slot buffer's occupancy and activity words are cleared here for the receiver side.
__global__ void __launch_bounds__(256) k_worklist(DevPtrs P, int cur, int *wl_n) {
    __shared__ int wcount[8], wbase[8], bbase;
    long long nkey = P.n * P.nf;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned *occ_n = P.occ[cur ^ 1], *act_n = P.act[cur ^ 1];
    for (long long k0 = (long long)blockIdx.x * blockDim.x; k0 < nkey;
         k0 += (long long)gridDim.x * blockDim.x) {
        long long key = k0 + threadIdx.x;
        bool f = false, t = false;
        if (key < nkey) {
            t = P.touched[key] != 0;
            if (t) P.touched[key] = 0;
            f = t || P.seg_cnt[key] > 0 || (P.occ[cur][key] & ~P.act[cur][key]) != 0u;
            occ_n[key] = 0u;
            act_n[key] = 0u;
        }
        unsigned m = __ballot_sync(FULLMASK, f);
        if (lane == 0) wcount[w] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < 8; ++k) { wbase[k] = t; t += wcount[k]; }
            bbase = t ? atomicAdd(wl_n, t) : 0;
        }
        __syncthreads();
        if (f)
            P.worklist[bbase + wbase[w] + __popc(m & ((1u << lane) - 1u))] =
                (int)((unsigned)key | (t ? 0x80000000u : 0u));
        __syncthreads();
    }
}

// absorptions of one receiver group in one hop.  FP64 path: FP64 sums.  FP32 path: the
// group's (fixed-order) sums go into the particle's fixed-point words, like the virtual-particle
// deposits, so no FP64 instruction runs in the hop loop; pass counts stay in FP32.  Returns the
// high absorption word before the add (0 on the FP64 path), which the caller range-checks one
// group later, so that the group does not wait for the atomic's round trip.
template <typename Real>
__device__ __forceinline__ unsigned long long deposit_group(const DevPtrs &P, long long key,
                                                            long long j, int box, Real a, Real ae,
                                                            Real w);
template <>
__device__ __forceinline__ unsigned long long deposit_group<double>(const DevPtrs &P,
                                                                    long long key, long long j,
                                                                    int box, double a, double ae,
                                                                    double w) {
    double nm = P.norm[box];
    P.abs[key] += a * nm;
    P.absE[key] += ae * nm * P.eunit;
    P.pass[key] += w * nm;
    return 0ull;
}
template <>
__device__ __forceinline__ unsigned long long deposit_group<float>(const DevPtrs &P,
                                                                   long long key, long long j,
                                                                   int box, float a, float ae,
                                                                   float w) {
    // atomics: virtual-particle deposits into the same words may run at the same time
    unsigned long long old = 0ull;
    float fa = a * ((float *)P.dep_s)[j];
    if (fa > 0.0f) {
        unsigned long long qh, ql;
        if (fx_split(fa, qh, ql)) {
            old = atomicAdd(&P.fx_abs[key], qh);
            atomicAdd(&P.fx_lo[key], ql);
        } else {
            atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_RANGE);
        }
    }
    float fe = ae * ((float *)P.depE_s)[j];
    if (fe > 0.0f) atomicAdd(&P.fx_E[key], f2u64_rz(fe + 0.5f));
    P.passf[key] += w;
    return old;
}

// Receiver side.  Group of G = n_rc lanes per (particle j, frequency nu); lane = reception
// cone.  Contributions are computed in parallel and merged in their fixed order by a
// broadcast loop (the lane owning the target cone adds).  Groups come from the work list;
// the next buffer's occupancy words were cleared by the work-list kernel.
// cur: the slot buffer holding the hop's packets.
template <typename Real, int G, bool BAR, bool SH>
__global__ void __launch_bounds__(256, HOP_MINB(Real)) k_phaseB(DevPtrs P, int cur, const int *wl_n) {
    // contributions of the current chunk, one per lane: 6 values (T, T d, T clock, T eps), and
    // T sigma in a shared frequency bin; and per reception cone of each group, the mask of the
    // chunk's lanes that feed it
    __shared__ Real sv[SH ? 7 : 6][256];
    __shared__ unsigned sm[256];
    // the current chunk of reverse edges: offset and sender; bitmap word and first
    // contribution; and per contribution chunk, the edge lane where each range starts
    __shared__ float4 se[256];
    __shared__ uint2 sw2[256];
    __shared__ int sown[256];
    int gl = threadIdx.x & (G - 1);
    int gbase = threadIdx.x - gl;               // first thread of this group in the block
    unsigned base = (threadIdx.x & 31) & ~(unsigned)(G - 1);
    unsigned gmask = (G == 32) ? FULLMASK : (((1u << G) - 1u) << base);
    long long ng = *wl_n;
    int nxt = cur ^ 1;
    // each block takes one contiguous chunk of the work list; its groups pull entries from it
    // through a shared counter, so that they finish together
    __shared__ int snext;
    long long chunk = (ng + gridDim.x - 1) / gridDim.x;
    long long gb0 = (long long)blockIdx.x * chunk;
    long long gb1 = gb0 + chunk < ng ? gb0 + chunk : ng;
    if (threadIdx.x == 0) snext = 0;
    __syncthreads();
    auto next_group = [&]() {
        long long v = 0;
        if (gl == 0) v = gb0 + atomicAdd(&snext, 1);
        return __shfl_sync(gmask, v, 0, G);
    };
    unsigned long long pend = 0ull;   // the high absorption word before the last deposit
    bool bad = false;
    for (long long gi = next_group(); gi < gb1; gi = next_group()) {
        unsigned wv = (unsigned)P.worklist[gi];
        long long key = wv & 0x7fffffffu;
        bool touched = (wv >> 31) != 0u;
        long long j = (unsigned)key / (unsigned)P.nf;
        int nu = (int)((unsigned)key % (unsigned)P.nf);
        unsigned park = P.occ[cur][key] & ~P.act[cur][key];
        int fc = P.seg_cnt[key];
        Slots<Real> So(P, cur), Sn(P, nxt);
        long long sidx = j * P.S + (long long)nu * G + gl;
        // a group of the shared frequency bin also merges the cross-section sums
        bool sgs = SH && nu == 0;
        long long gidx = j * G + gl;
        KSum<Real> aN, aX, aY, aZ, aC, aE, aG, sA, sAE, sW;
        if ((park >> gl) & 1u) {
            aN.init(So.N[sidx]); aX.init(So.X[sidx]); aY.init(So.Y[sidx]);
            aZ.init(So.Z[sidx]); aC.init(So.C[sidx]); aE.init(So.E[sidx]);
            aG.init(sgs ? ((Real *)P.slG[cur])[gidx] : Real(0));
        } else {
            aN.init(Real(0)); aX.init(Real(0)); aY.init(Real(0));
            aZ.init(Real(0)); aC.init(Real(0)); aE.init(Real(0));
            aG.init(Real(0));
        }
        sA.init(Real(0)); sAE.init(Real(0)); sW.init(Real(0));
        int box = P.pbox[j];
        // merge this chunk's contributions: lane gl of the group holds one for reception cone
        // mybin (-1: none).  Lanes of equal cone find each other (match), the lowest of them
        // publishes the set, and lane b adds the contributions to cone b in lane order.
        auto merge_chunk = [&](int mybin) {
            unsigned peers = __match_any_sync(gmask, mybin >= 0 ? mybin : G + gl);
            sm[threadIdx.x] = 0u;
            __syncwarp(gmask);
            if (mybin >= 0 && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0u)
                sm[gbase + mybin] = peers >> base;
            __syncwarp(gmask);
            unsigned m = sm[threadIdx.x];
            while (m) {
                int t2 = gbase + __ffs(m) - 1;
                m &= m - 1u;
                aN.add(sv[0][t2]); aX.add(sv[1][t2]); aY.add(sv[2][t2]);
                aZ.add(sv[3][t2]); aC.add(sv[4][t2]); aE.add(sv[5][t2]);
                if (sgs) aG.add(sv[SH ? 6 : 0][t2]);
            }
            __syncwarp(gmask);
        };
        if (touched) {
            Real u = box_unit<Real>(P, box);
            Real sig_nhi = sigma_of<Real>(P, nu) * ((Real *)P.nHIr)[j];
            const float *Rf = P.Rf + j * 9;
            const double *Rd = P.R + j * 9;
            int e0 = P.rev_off[j], e1 = P.rev_off[j + 1];
            unsigned *bmr = P.bm + (long long)nu * P.n * P.kn;
            for (int eb = e0; eb < e1; eb += G) {
                int e = eb + gl;
                unsigned word = 0u;
                int si = 0;
                float fx = 0.f, fy = 0.f, fz = 0.f;
                unsigned xb = 0u;   // 1u << 31: the edge's path crosses the box's barrier
                if (e < e1) {   // the edge's data is loaded with its word (one memory round)
                    word = bmr[e];
                    si = (int)(P.rev_ent[e] >> 5);
                    fx = P.rdx[e]; fy = P.rdy[e]; fz = P.rdz[e];
                    if (word) bmr[e] = 0u;
                    if (BAR && word) {
                        int jx = P.qx[j], jy = P.qy[j], jz = P.qz[j];
                        if (barrier_crosses_call(P.bar[box], jx - (int)fx, jy - (int)fy,
                                                 jz - (int)fz, jx, jy, jz))
                            xb = 1u << 31;
                    }
                }
                int cw = __popc(word);
                int incl = cw;
#pragma unroll
                for (int o = 1; o < G; o <<= 1) {
                    int v = __shfl_up_sync(gmask, incl, o, G);
                    if (gl >= o) incl += v;
                }
                int total = __shfl_sync(gmask, incl, G - 1, G);
                int excl = incl - cw;
                // the chunk's edges in shared memory; contribution c belongs to the edge whose
                // range [excl, excl + cw) holds it
                se[threadIdx.x] = make_float4(fx, fy, fz, __int_as_float(si));
                sw2[threadIdx.x] = make_uint2(word, (unsigned)excl | xb);
                int carry = 0;   // owner of the last contribution of the previous chunk
                for (int cb = 0; cb < total; cb += G) {
                    bool st = cw > 0 && excl >= cb && excl < cb + G;
                    if (st) sown[gbase + excl - cb] = gl;
                    unsigned smk = __reduce_or_sync(gmask, st ? 1u << (excl - cb) : 0u);
                    __syncwarp(gmask);
                    unsigned below = smk & (0xffffffffu >> (31 - gl));
                    int own = below ? sown[gbase + 31 - __clz(below)] : carry;
                    carry = __shfl_sync(gmask, own, G - 1, G);
                    int c = cb + gl;
                    int mybin = -1;
                    bool keep = c < total;
                    Real w, d0, d1, d2, clk, eps, sgc = Real(0);
                    float4 ed;
                    if (keep) {
                        ed = se[gbase + own];
                        uint2 ow = sw2[gbase + own];
                        int bsrc = __fns(ow.x, 0, c - (int)(ow.y & 0x7fffffffu) + 1);
                        long long ridx = (long long)__float_as_int(ed.w) * P.S + (long long)nu * G + bsrc;
                        rec_load(P.rec, ridx, w, d0, d1, d2, clk, eps, sgs, sgc);
                        if (ow.y >> 31) {   // through the barrier: removed (counted escaped)
                            atomicAdd(&P.esc_fx[box], esc_fixed(w, P, box));
                            keep = false;
                        }
                    }
                    if (keep) {
                        Real t = (Real)ed.x * d0 + (Real)ed.y * d1 + (Real)ed.z * d2;
                        Real l = t * u;
                        Real A, T;
                        // in a shared bin each packet carries its own mean cross-section
                        Real sn = sgs ? (sgc * (Real)P.sunit) * ((Real *)P.nHIr)[j] : sig_nhi;
                        split_absorbed<Real>(w, sn * l, A, T);
                        sA.add(A);
                        sAE.add(A * eps);
                        sW.add(w);
                        mybin = bin_fast<Real>(Rf, Rd, P.ax_rc, G, d0, d1, d2);
                        sv[0][threadIdx.x] = T;
                        sv[1][threadIdx.x] = T * d0;
                        sv[2][threadIdx.x] = T * d1;
                        sv[3][threadIdx.x] = T * d2;
                        sv[4][threadIdx.x] = T * (clk + l / (Real)C_LIGHT);
                        sv[5][threadIdx.x] = T * eps;
                        if (sgs) sv[SH ? 6 : 0][threadIdx.x] = T * sgc;
                    }
                    merge_chunk(mybin);
                }
            }
        }
        if (fc > 0) {
            int so = P.seg_off[key];
            Real *const *V = (Real *const *)P.st_v;
            for (int cb = 0; cb < fc; cb += G) {
                int c = cb + gl;
                int mybin = -1;
                if (c < fc) {
                    int s = P.seg_idx[so + c];
                    mybin = P.st_bin[s];           // -1: removed by a barrier
                    if (mybin >= 0) {
                        for (int f = 0; f < 6; ++f) sv[f][threadIdx.x] = V[f][s];
                        if (sgs) sv[SH ? 6 : 0][threadIdx.x] = V[9][s];
                        sA.add(V[6][s]);
                        sAE.add(V[7][s]);
                        sW.add(V[8][s]);
                    }
                }
                merge_chunk(mybin);
            }
        }
        Real N = aN.get();
        bool occ = N > Real(0);
        bool act = occ && (aC.get() / N < (Real)P.dt);
        unsigned lmask = (G == 32) ? FULLMASK : ((1u << G) - 1u);
        unsigned bo = (__ballot_sync(gmask, occ) >> base) & lmask;
        unsigned ba = (__ballot_sync(gmask, act) >> base) & lmask;
        if (occ) {
            Sn.N[sidx] = N; Sn.X[sidx] = aX.get(); Sn.Y[sidx] = aY.get();
            Sn.Z[sidx] = aZ.get(); Sn.C[sidx] = aC.get(); Sn.E[sidx] = aE.get();
            if (sgs) ((Real *)P.slG[nxt])[gidx] = aG.get();
        }
        Real a = sA.get(), ae = sAE.get(), w = sW.get();
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) {
            a += __shfl_down_sync(gmask, a, o, G);
            ae += __shfl_down_sync(gmask, ae, o, G);
            w += __shfl_down_sync(gmask, w, o, G);
        }
        if (gl == 0) {
            P.occ[nxt][key] = bo;
            P.act[nxt][key] = ba;
            if (touched || fc > 0) {
                bad |= pend > (1ull << 62);
                pend = deposit_group<Real>(P, key, j, box, a, ae, w);
            }
        }
    }
    bad |= pend > (1ull << 62);
    if (bad) atomicOr((unsigned long long *)&P.cnt[CNT_ERR], (unsigned long long)ERRB_RANGE);
}

// After a hop: active slots, live free packets, escaped photons per box (fixed point).
__global__ void k_hop_counts(DevPtrs P, int nxt, int fnxt, const int *lens,
                             const unsigned long long *esc_r, const unsigned char *vstat) {
    __shared__ long long sh[5][8];
    long long act = 0, live = 0, nesc = 0, actp = 0, occs = 0;
    long long nreq = lens[2];
    if (nreq > P.F_cap) nreq = P.F_cap;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = t0; i < P.n; i += stride) {
        unsigned any = 0u;
        for (int nu = 0; nu < P.nf; ++nu) {
            unsigned a = P.act[nxt][i * P.nf + nu];
            any |= a;
            act += __popc(a);
            occs += __popc(P.occ[nxt][i * P.nf + nu]);
        }
        actp += (any != 0u);
    }
    FreeBuf F = P.fr[fnxt];
    for (long long r = t0; r < nreq; r += stride) {
        unsigned char s = vstat[r];
        live += (s == 0);
        if (s == 1 || s == 3) {
            nesc += (s == 1);
            unsigned long long v = esc_r[r];
            int b = F.box[r];
            // aggregate equal boxes within the warp before the atomic
            unsigned peers = __match_any_sync(__activemask(), b);
            int leader = __ffs(peers) - 1;
            unsigned long long tot = 0;
            for (unsigned m = peers; m; m &= m - 1) {
                int src = __ffs(m) - 1;
                tot += __shfl_sync(peers, v, src);
            }
            if ((int)(threadIdx.x & 31) == leader) atomicAdd(&P.esc_fx[b], tot);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        act += __shfl_down_sync(FULLMASK, act, o);
        live += __shfl_down_sync(FULLMASK, live, o);
        nesc += __shfl_down_sync(FULLMASK, nesc, o);
        actp += __shfl_down_sync(FULLMASK, actp, o);
        occs += __shfl_down_sync(FULLMASK, occs, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = act; sh[1][w] = live; sh[2][w] = nesc; sh[3][w] = actp; sh[4][w] = occs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, l = 0, e = 0, ap = 0, oc = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += sh[0][k]; l += sh[1][k]; e += sh[2][k]; ap += sh[3][k]; oc += sh[4][k];
        }
        if (a) atomicAdd((unsigned long long *)&P.cnt[CNT_ACTIVE], (unsigned long long)a);
        if (a) atomicAdd((unsigned long long *)&P.cnt[CNT_ACTS], (unsigned long long)a);
        if (l) atomicAdd((unsigned long long *)&P.cnt[CNT_LIVE], (unsigned long long)l);
        if (e) atomicAdd((unsigned long long *)&P.cnt[CNT_VESC], (unsigned long long)e);
        if (ap) atomicAdd((unsigned long long *)&P.cnt[CNT_ACTP], (unsigned long long)ap);
        if (oc) atomicAdd((unsigned long long *)&P.cnt[CNT_OUT], (unsigned long long)oc);
    }
}

// bookkeeping of the hop loop (single thread)
enum { HL_BEGIN = 0, HL_END = 2, HL_EMIT = 3, HL_TRANSPORT = 4, HL_STEP = 5 };
// in_graph: the launch is a node of the step graph, and `handle` the conditional it sets
// (HL_BEGIN: the buffer switch; HL_END: the hop loop)
__global__ void k_hop_lens(DevPtrs P, int *lens, int phase, long long arg, int in_graph,
                           cudaGraphConditionalHandle handle) {
    long long *cnt = P.cnt;
    if (phase == HL_BEGIN) {            // before the hop: counters, scan length
        cnt[CNT_ACTIVE] = 0;
        cnt[CNT_LIVE] = 0;
        cnt[CNT_VQ] = 0;                // the virtual particles' work queue
        lens[1] = (int)(P.n + lens[0]);
        // in the graph: which of the four copies of the hop (slot and free-packet buffers) runs
        if (in_graph) cudaGraphSetConditional(handle, (unsigned)(cnt[CNT_CUR] | (cnt[CNT_FCUR] << 1)));
    } else if (phase == HL_END) {       // after the hop (arg = hop cap)
        long long nr = lens[2];
        lens[0] = (int)(nr < P.F_cap ? nr : P.F_cap);
        cnt[CNT_STG] += lens[3];
        cnt[CNT_WLS] += lens[4];
        if (nr > cnt[CNT_PKFREE]) cnt[CNT_PKFREE] = nr;
        if (cnt[CNT_ACTIVE] > cnt[CNT_PKACT]) cnt[CNT_PKACT] = cnt[CNT_ACTIVE];
        cnt[CNT_CUR] ^= 1;              // the receivers' buffers hold the next hop's packets
        cnt[CNT_FCUR] ^= 1;
        long long hop = ++cnt[CNT_HOP];
        // another hop while packets still move and no error stopped the step; at the hop cap
        // the free packets in flight are dropped (counted escaped) and the step reports it
        bool moving = cnt[CNT_ACTIVE] != 0 || cnt[CNT_LIVE] != 0;
        bool more = moving && cnt[CNT_ERR] == 0;
        if (more && hop >= arg) {
            more = false;
            cnt[CNT_DROP] = 1;
        }
        if (in_graph) cudaGraphSetConditional(handle, more ? 1u : 0u);
    } else if (phase == HL_EMIT) {      // emission (arg = packets): free buffer 0 holds them
        lens[0] = (int)arg;
        cnt[CNT_FCUR] = 0;
    } else if (phase == HL_TRANSPORT) { // start of the hop loop (arg = hop cap)
        cnt[CNT_VIRT] = 0;
        cnt[CNT_VESC] = 0;
        cnt[CNT_GAS] = 0;
        for (int k = CNT_ACTP; k <= CNT_OUT; ++k) cnt[k] = 0;
        cnt[CNT_HOP] = 0;
        cnt[CNT_PKFREE] = 0;
        cnt[CNT_PKACT] = 0;
        cnt[CNT_DROP] = arg <= 0 ? 1 : 0;
    } else {                            // HL_STEP: the step number (arg)
        cnt[CNT_STEP] = arg;
    }
}

// Hop cap reached: the free packets still in flight leave the box (counted escaped).  Does
// nothing unless the hop loop set the drop flag.
template <typename Real>
__global__ void k_drop_free(DevPtrs P, const int *lens) {
    if (!P.cnt[CNT_DROP]) return;
    FreeBuf F = P.fr[(int)P.cnt[CNT_FCUR]];
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < lens[0];
         f += (long long)gridDim.x * blockDim.x) {
        Real N = ((Real *)F.N)[f];
        if (N > Real(0)) {
            int b = F.box[f];
            atomicAdd(&P.esc_fx[b], esc_fixed(N, P, b));
            ((Real *)F.N)[f] = Real(0);
        }
    }
}

// ------------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------------

#define LAUNCH_ON(sx, id, n, ...)   \
    do {                            \
        kt_begin(c, id, sx);        \
        __VA_ARGS__;                \
        kt_end(c, id, sx, n);       \
    } while (0)
#define LAUNCH(id, n, ...) LAUNCH_ON(st, id, n, __VA_ARGS__)

// the step number the rotations and virtual particles draw with (kept on the device)
static void set_step(rt_ctx *c, long long step, cudaStream_t st) {
    if (c->step_dev == step && step != LLONG_MIN) return;
    LAUNCH(KT_HOP_LENS, 1, (k_hop_lens<<<1, 1, 0, st>>>(c->d, c->hop.lens, HL_STEP, step, 0, 0)));
    c->step_dev = step;
}

// The virtual-particle kernel of the hop: the instance with the grid-walk fallback only when
// some cell of the context has no candidate list.
template <typename Real, int NRC, bool BAR, bool SH, int IB>
static void launch_virtual(rt_ctx *c, cudaStream_t st, int GV, int cur, int fcur) {
    DevPtrs &P = c->d;
    HopScratch &H = c->hop;
    const int tb = 256;
    int nb = rt_blocks(P.F_cap * 32, tb, GV);
    if (c->cand_fallback > 0)
        k_virtual<Real, NRC, BAR, SH, IB, true><<<nb, tb, 0, st>>>(P, cur, fcur, H.lens, H.esc_r,
                                                                   H.vstat);
    else
        k_virtual<Real, NRC, BAR, SH, IB, false><<<nb, tb, 0, st>>>(P, cur, fcur, H.lens, H.esc_r,
                                                                    H.vstat);
}

// One hop.  Two streams: st: gas senders, the request list, virtual particles, the hop counts.
// s2: free-packet senders and staging, receiver segments, work list, receiver side.  s2 starts
// after everything before this hop on st; the work list waits for the gas senders (touched
// flags, bitmaps, records); the request scan and its length check wait for the free-packet
// cone tests; the hop counts wait for the receiver side.  nfr bounds the free packets of the
// hop (their count is on the device); cur and fcur are the hop's slot and free-packet buffers.
// The bookkeeping kernels before and after (k_hop_lens HL_BEGIN, HL_END) are not part of it.
template <typename Real, int NRC>
static void hop_core(rt_ctx *c, cudaStream_t st, long long nfr, int cur, int fcur) {
    DevPtrs &P = c->d;
    const int GA = c->grid_hop[0] ? c->grid_hop[0] : GRID_A;
    const int GV = c->grid_hop[1] ? c->grid_hop[1] : GRID_V;
    const int GB = c->grid_hop[2] ? c->grid_hop[2] : GRID_B;
    HopScratch &H = c->hop;
    const int tb = 256, gb = 152 * 64;
    long long n = P.n, nkey = n * P.nf;
    cudaStream_t s2 = c->st2;
    cudaEvent_t evFork = c->hev[0], evA = c->hev[1], evFree = c->hev[2], evB = c->hev[3];
    if (nfr < 1) nfr = 1;
    cudaEventRecord(evFork, st);
    cudaStreamWaitEvent(s2, evFork, 0);
    cudaMemsetAsync(P.seg_cnt, 0, sizeof(int) * nkey, s2);
    cudaMemsetAsync(P.seg_fill, 0, sizeof(int) * nkey, s2);
    LAUNCH_ON(s2, KT_FREE_A, 1, (k_freeA<Real><<<rt_blocks(nfr * 32, tb, gb), tb, 0, s2>>>(P, fcur, H.lens, H.fmask, H.stcnt)));
    LAUNCH_ON(s2, KT_SCAN, 2, (rt_scan_exclusive(c, H.stcnt, H.stoff, nfr, H.lens, H.lens + 3, s2, c->scan_tmp2)));
    cudaEventRecord(evFree, s2);
    // instances: the common case; with a barrier; with a shared frequency bin (whose instance
    // also takes the barrier test, which is a no-op in boxes without one)
    if (P.shared)
        LAUNCH_ON(s2, KT_FREE_C, 1, (k_freeC<Real, NRC, true, true><<<rt_blocks(nfr * 32, tb, gb), tb, 0, s2>>>(P, fcur, H.lens, H.fmask, H.stoff)));
    else if (P.any_bar)
        LAUNCH_ON(s2, KT_FREE_C, 1, (k_freeC<Real, NRC, true, false><<<rt_blocks(nfr * 32, tb, gb), tb, 0, s2>>>(P, fcur, H.lens, H.fmask, H.stoff)));
    else
        LAUNCH_ON(s2, KT_FREE_C, 1, (k_freeC<Real, NRC, false, false><<<rt_blocks(nfr * 32, tb, gb), tb, 0, s2>>>(P, fcur, H.lens, H.fmask, H.stoff)));
    if (P.shared)
        LAUNCH(KT_PHASE_A, 1, (k_phaseA<Real, NRC, true><<<rt_blocks(n * 32, tb, GA), tb, 0, st>>>(P, cur)));
    else
        LAUNCH(KT_PHASE_A, 1, (k_phaseA<Real, NRC, false><<<rt_blocks(n * 32, tb, GA), tb, 0, st>>>(P, cur)));
    cudaEventRecord(evA, st);
    cudaStreamWaitEvent(st, evFree, 0);
    LAUNCH(KT_SCAN, 2, (rt_scan_exclusive(c, P.reqcnt, P.reqoff, n + nfr, H.lens + 1, H.lens + 2, st)));
    LAUNCH(KT_EXPAND, 1, (k_expand<<<rt_blocks(n + nfr, tb, gb), tb, 0, st>>>(P, H.lens)));
    const int IS = KNN_IB_SMALL, IL = KNN_IB_LARGE;
    if (P.kwide && P.shared)   // boxes above 2^22 particles: the general instance, 24-bit keys
        LAUNCH(KT_VIRTUAL, 1, (launch_virtual<Real, NRC, true, true, IL>(c, st, GV, cur, fcur)));
    else if (P.kwide)
        LAUNCH(KT_VIRTUAL, 1, (launch_virtual<Real, NRC, true, false, IL>(c, st, GV, cur, fcur)));
    else if (P.shared)
        LAUNCH(KT_VIRTUAL, 1, (launch_virtual<Real, NRC, true, true, IS>(c, st, GV, cur, fcur)));
    else if (P.any_bar)
        LAUNCH(KT_VIRTUAL, 1, (launch_virtual<Real, NRC, true, false, IS>(c, st, GV, cur, fcur)));
    else
        LAUNCH(KT_VIRTUAL, 1, (launch_virtual<Real, NRC, false, false, IS>(c, st, GV, cur, fcur)));
    LAUNCH_ON(s2, KT_SCAN, 2, (rt_scan_exclusive(c, P.seg_cnt, P.seg_off, nkey, nullptr, nullptr, s2, c->scan_tmp2)));
    LAUNCH_ON(s2, KT_SEG_FILL, 1, (k_seg_fill<<<rt_blocks(P.ST_cap, tb, 152 * 16), tb, 0, s2>>>(P, H.lens)));
    LAUNCH_ON(s2, KT_SEG_SORT, 1, (k_seg_sort<<<(unsigned)((nkey + tb - 1) / tb), tb, 0, s2>>>(P)));
    cudaMemsetAsync(H.lens + 4, 0, sizeof(int), s2);
    cudaStreamWaitEvent(s2, evA, 0);
    LAUNCH_ON(s2, KT_WORKLIST, 1, (k_worklist<<<rt_blocks(nkey, tb, 152 * 16), tb, 0, s2>>>(P, cur, H.lens + 4)));
    if (P.shared)
        LAUNCH_ON(s2, KT_PHASE_B, 1, (k_phaseB<Real, NRC, true, true><<<rt_blocks(nkey * NRC, tb, GB), tb, 0, s2>>>(P, cur, H.lens + 4)));
    else if (P.any_bar)
        LAUNCH_ON(s2, KT_PHASE_B, 1, (k_phaseB<Real, NRC, true, false><<<rt_blocks(nkey * NRC, tb, GB), tb, 0, s2>>>(P, cur, H.lens + 4)));
    else
        LAUNCH_ON(s2, KT_PHASE_B, 1, (k_phaseB<Real, NRC, false, false><<<rt_blocks(nkey * NRC, tb, GB), tb, 0, s2>>>(P, cur, H.lens + 4)));
    cudaEventRecord(evB, s2);
    cudaStreamWaitEvent(st, evB, 0);
    LAUNCH(KT_HOP_COUNT, 1, (k_hop_counts<<<304, 256, 0, st>>>(P, cur ^ 1, fcur ^ 1, H.lens, H.esc_r, H.vstat)));
}

static void graph_destroy(rt_ctx *c);
void rt_launch_grids(const rt_ctx *c, long long out[3]) {
    const int def[3] = {GRID_A, GRID_V, GRID_B};
    for (int k = 0; k < 3; ++k) out[k] = c->grid_hop[k] ? c->grid_hop[k] : def[k];
}

// cone bitmaps and receiver flags back to zero (as every hop leaves them)
static void clear_cone_bits(rt_ctx *c, cudaStream_t st) {
    DevPtrs &P = c->d;
    cudaMemsetAsync(P.bm, 0, sizeof(unsigned) * P.n * P.kn * P.nf, st);
    cudaMemsetAsync(P.touched, 0, sizeof(int) * P.n * P.nf, st);
}

// start of the hop loop: cone bits cleared if an inspection pass left some, counters reset
static void transport_begin(rt_ctx *c, cudaStream_t st) {
    DevPtrs &P = c->d;
    if (c->bm_dirty) {
        clear_cone_bits(c, st);
        c->bm_dirty = false;
    }
    LAUNCH(KT_HOP_LENS, 1, (k_hop_lens<<<1, 1, 0, st>>>(P, c->hop.lens, HL_TRANSPORT, c->cfg.hop_cap, 0, 0)));
}

// after the hop loop (the counters are in cnt_h): statistics, modelled bytes, status
static rt_status transport_end(rt_ctx *c, bool fp32) {
    DevPtrs &P = c->d;
    long long hops = c->cnt_h[CNT_HOP];
    // the active packets of the first hop were made by the emission: add them to the model
    // counts below (CNT_ACTS/ACTP count those produced by each hop's receiver side)
    {
        const double R = fp32 ? 4.0 : 8.0, kn = P.kn;
        double actp = (double)c->cnt_h[CNT_ACTP], acts = (double)c->cnt_h[CNT_ACTS];
        double gcon = (double)c->cnt_h[CNT_GCON], stg = (double)c->cnt_h[CNT_STG];
        double wls = (double)c->cnt_h[CNT_WLS], outs = (double)c->cnt_h[CNT_OUT];
        double vreq = (double)c->cnt_h[CNT_VIRT];
        // algorithmic bytes: each input read once and each output written once
        c->kstat[KT_PHASE_A].bytes += actp * (kn * (4 + 4 + 12) + P.nf * 4) + acts * 12 * R +
                                      gcon * 8 + (double)hops * (double)P.n * 4;
        c->kstat[KT_PHASE_B].bytes += wls * (16 + 8 + 48 + kn * 4) + gcon * (16 + 6 * R + 4) +
                                      stg * (8 + 9 * R) + outs * 6 * R;
        c->kstat[KT_VIRTUAL].bytes += vreq * (8 + 6 * R + 40 + kn * (16 + 4 * R + 16 + 4) +
                                              6 * R + 40);
    }
    c->stats[0] = hops;
    c->stats[1] = c->cnt_h[CNT_VIRT];
    c->stats[2] = c->cnt_h[CNT_VESC];
    c->stats[5] = c->cnt_h[CNT_PKFREE];
    c->stats[6] = c->cnt_h[CNT_PKACT];
    c->stats[7] = c->cnt_h[CNT_GCON];
    c->stats[8] = c->cnt_h[CNT_ACTP];
    c->stats[9] = c->cnt_h[CNT_ACTS];
    c->stats[10] = c->cnt_h[CNT_STG];
    c->stats[11] = c->cnt_h[CNT_WLS];
    c->stats[12] = c->cnt_h[CNT_OUT];
    long long e = c->cnt_h[CNT_ERR];
    if (e & ERRB_FREE_CAP) return rt_fail(c, RT_ERR_CAPACITY, "free packets exceeded free_cap");
    if (e & ERRB_STAGE_CAP) return rt_fail(c, RT_ERR_CAPACITY, "staged contributions exceeded capacity");
    if (e & ERRB_RANGE) return rt_fail(c, RT_ERR_RANGE, "virtual deposit overflowed its accumulator");
    if (e & ERRB_KNN)
        return rt_fail(c, RT_ERR_KNN, "a virtual particle's n_ngb-th neighbour lies beyond the kNN key range");
    if (c->cnt_h[CNT_DROP]) return rt_fail(c, RT_ERR_HOP_LIMIT, "hop loop reached hop_cap");
    return RT_OK;
}

template <typename Real, int NRC>
static rt_status run_parts(rt_ctx *c, int part, long long step, cudaStream_t st) {
    DevPtrs &P = c->d;
    const int tb = 256;
    long long n = P.n;
    long long nkey = n * P.nf;
    HopScratch &H = c->hop;
    if (part == 0) {  // rotations
        if (!c->capturing) set_step(c, step, st);
        long long t = n + (long long)P.ns * P.K;
        LAUNCH(KT_ROTATE, 1, (k_rotate<<<(unsigned)((t + tb - 1) / tb), tb, 0, st>>>(P)));
        return rt_cuda_check(c, cudaGetLastError(), "rotate");
    }
    if (part == 1) {  // re-bin held packets
        LAUNCH(KT_REBIN, 1, (k_rebin<Real, NRC><<<(unsigned)((nkey + tb - 1) / tb), tb, 0, st>>>(P)));
        return rt_cuda_check(c, cudaGetLastError(), "rebin");
    }
    if (part == 2) {  // emission
        long long np_s = (long long)P.ns * P.K * P.nfs * P.nec;
        long long np_r = P.rec_mode == RT_REC_EMISSION_CONES ? n * P.K * P.nec : 0;
        long long np = np_s + np_r;
        if (np > P.F_cap) return rt_fail(c, RT_ERR_CAPACITY, "source packets exceed free_cap");
        if (!c->capturing) set_step(c, step, st);
        LAUNCH(KT_EMIT_REC, 1, (k_emit_rec<Real, NRC><<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(P)));
        LAUNCH(KT_HOP_LENS, 1, (k_hop_lens<<<1, 1, 0, st>>>(P, H.lens, HL_EMIT, np, 0, 0)));
        c->fcur = 0;
        if (np_s > 0)
            LAUNCH(KT_EMIT_SRC, 1, (k_emit_src<Real><<<(unsigned)((np_s + tb - 1) / tb), tb, 0, st>>>(P)));
        if (np_r > 0)
            LAUNCH(KT_EMIT_SRC, 1, (k_emit_rec_cones<Real><<<(unsigned)((np_r + tb - 1) / tb), tb, 0, st>>>(P, np_s)));
        c->nfree_h = np;
        return rt_cuda_check(c, cudaGetLastError(), "emit");
    }
    if (part == 3) {  // cone masks of the held packets only (inspection)
        clear_cone_bits(c, st);
        c->bm_dirty = true;
        if (P.shared)
            LAUNCH(KT_PHASE_A, 1, (k_phaseA<Real, NRC, true><<<rt_blocks(n * 32, tb, 152 * 64), tb, 0, st>>>(P, c->cur)));
        else
            LAUNCH(KT_PHASE_A, 1, (k_phaseA<Real, NRC, false><<<rt_blocks(n * 32, tb, 152 * 64), tb, 0, st>>>(P, c->cur)));
        return rt_cuda_check(c, cudaGetLastError(), "cone masks");
    }
    // part 4: the hop loop, driven from the host (one synchronisation per hop)
    set_step(c, step, st);
    transport_begin(c, st);
    for (int hop = 0;; ++hop) {
        if (hop >= c->cfg.hop_cap) {
            LAUNCH(KT_DROP, 1, (k_drop_free<Real><<<rt_blocks(P.F_cap, tb, 152 * 64), tb, 0, st>>>(P, H.lens)));
            break;
        }
        LAUNCH(KT_HOP_LENS, 1, (k_hop_lens<<<1, 1, 0, st>>>(P, H.lens, HL_BEGIN, 0, 0, 0)));
        hop_core<Real, NRC>(c, st, c->nfree_h, c->cur, c->fcur);
        LAUNCH(KT_HOP_LENS, 1, (k_hop_lens<<<1, 1, 0, st>>>(P, H.lens, HL_END, c->cfg.hop_cap, 0, 0)));
        c->cur ^= 1;
        c->fcur ^= 1;
        cudaMemcpyAsync(c->cnt_h, P.cnt, sizeof(long long) * CNT_N, cudaMemcpyDeviceToHost, st);
        rt_status hs = rt_cuda_check(c, cudaStreamSynchronize(st), "hop");
        if (hs != RT_OK) return hs;
        kt_resolve(c);
        if (c->cnt_h[CNT_ERR]) break;
        c->nfree_h = std::min<long long>(c->cnt_h[CNT_NREQ], P.F_cap);
        if (c->cnt_h[CNT_ACTIVE] == 0 && c->cnt_h[CNT_LIVE] == 0) break;
    }
    cudaMemcpyAsync(c->cnt_h, P.cnt, sizeof(long long) * CNT_N, cudaMemcpyDeviceToHost, st);
    rt_status hs = rt_cuda_check(c, cudaStreamSynchronize(st), "hop loop");
    if (hs != RT_OK) return hs;
    kt_resolve(c);
    return transport_end(c, sizeof(Real) == 4);
}

// ---- the whole step as one CUDA graph --------------------------------------------------
// Prologue (rotations, re-binning, emission, emitted-photon tally, counter reset), a
// conditional while node whose body is one hop (its last kernel decides whether another hop
// runs), and the epilogue (drop at the hop cap, chemistry, end-of-step tally).  Captured on
// the context's own streams.  What changes from step to step or hop to hop is on the device:
// the step and hop numbers (read where they are used), and the buffer pair of the hop, which
// selects one of four captured copies of the hop through a switch node, so that inside a
// copy the buffers are launch parameters.  One capture serves every step.
static void graph_destroy(rt_ctx *c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
}

static rt_status capture_segment(rt_ctx *c, cudaGraph_t *out, rt_status (*body)(rt_ctx *, cudaStream_t)) {
    cudaStream_t sc = c->st_cap;
    cudaError_t e = cudaStreamBeginCapture(sc, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return rt_cuda_check(c, e, "graph capture");
    rt_status s = body(c, sc);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(sc, &g);
    if (s != RT_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e2 != cudaSuccess) return rt_cuda_check(c, e2, "graph capture");
    *out = g;
    return RT_OK;
}

template <typename Real, int NRC>
static rt_status seg_prologue(rt_ctx *c, cudaStream_t st) {
    rt_status s;
    if ((s = run_parts<Real, NRC>(c, 0, 0, st))) return s;
    if ((s = run_parts<Real, NRC>(c, 1, 0, st))) return s;
    if ((s = run_parts<Real, NRC>(c, 2, 0, st))) return s;
    if ((s = rt_budget_launch(c, 0, st))) return s;
    LAUNCH(KT_HOP_LENS, 1, (k_hop_lens<<<1, 1, 0, st>>>(c->d, c->hop.lens, HL_TRANSPORT, c->cfg.hop_cap, 0, 0)));
    return rt_cuda_check(c, cudaGetLastError(), "graph prologue");
}

template <typename Real>
static rt_status seg_epilogue(rt_ctx *c, cudaStream_t st) {
    LAUNCH(KT_DROP, 1, (k_drop_free<Real><<<rt_blocks(c->d.F_cap, 256, 152 * 64), 256, 0, st>>>(c->d, c->hop.lens)));
    rt_status s;
    if ((s = rt_chem_launch(c, st))) return s;
    if ((s = rt_budget_launch(c, 1, st))) return s;
    return rt_cuda_check(c, cudaGetLastError(), "graph epilogue");
}

// a single-thread bookkeeping kernel as an explicit node of a graph
static cudaError_t add_lens_node(rt_ctx *c, cudaGraphNode_t *node, cudaGraph_t g,
                                 const cudaGraphNode_t *dep, int phase, long long arg,
                                 cudaGraphConditionalHandle handle) {
    DevPtrs P = c->d;
    int *lens = c->hop.lens;
    int in_graph = 1;
    void *args[] = {&P, &lens, &phase, &arg, &in_graph, &handle};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)k_hop_lens;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    c->graph_launch_hop[KT_HOP_LENS] += 1;
    return cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &kp);
}

// The while node's body: HL_BEGIN (sets the buffer switch) -> a switch node over the four
// (slot buffer, free-packet buffer) pairs, each body one capture of the hop with those buffers
// as launch parameters -> HL_END (sets the loop condition).
template <typename Real, int NRC>
static cudaError_t build_hop_body(rt_ctx *c, cudaGraph_t body, cudaGraphConditionalHandle loop) {
    cudaGraphNode_t nbeg, nsw, nend;
    cudaGraphConditionalHandle sw;
    cudaError_t e = cudaGraphConditionalHandleCreate(&sw, body, 0, 0);
    if (e == cudaSuccess) e = add_lens_node(c, &nbeg, body, nullptr, HL_BEGIN, 0, sw);
    cudaGraphNodeParams cp = {};
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = sw;
        cp.conditional.type = cudaGraphCondTypeSwitch;
        cp.conditional.size = 4;
        e = cudaGraphAddNode(&nsw, body, &nbeg, nullptr, 1, &cp);
    }
    c->in_hop_body = true;
    long long once[KT_N];
    for (int par = 0; par < 4 && e == cudaSuccess; ++par) {
        e = cudaStreamBeginCaptureToGraph(c->st_cap, cp.conditional.phGraph_out[par], nullptr,
                                          nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        hop_core<Real, NRC>(c, c->st_cap, c->d.F_cap, par & 1, par >> 1);
        cudaGraph_t b = cp.conditional.phGraph_out[par];
        e = cudaStreamEndCapture(c->st_cap, &b);
        // one copy runs per hop: its launches are counted once
        if (par == 0) memcpy(once, c->graph_launch_hop, sizeof(once));
        else memcpy(c->graph_launch_hop, once, sizeof(once));
    }
    if (e == cudaSuccess) e = add_lens_node(c, &nend, body, &nsw, HL_END, c->cfg.hop_cap, loop);
    c->in_hop_body = false;
    return e;
}

template <typename Real, int NRC>
static rt_status capture_step(rt_ctx *c) {
    graph_destroy(c);
    for (int k = 0; k < KT_N; ++k) c->graph_launch_step[k] = c->graph_launch_hop[k] = 0;
    c->capturing = true;
    cudaGraph_t pro = nullptr, epi = nullptr, g = nullptr;
    rt_status s = capture_segment(c, &pro, seg_prologue<Real, NRC>);
    if (s == RT_OK) s = capture_segment(c, &epi, seg_epilogue<Real>);
    cudaError_t e = cudaSuccess;
    if (s == RT_OK) {
        cudaGraphNode_t npro, nloop, nepi;
        cudaGraphConditionalHandle loop;
        e = cudaGraphCreate(&g, 0);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&npro, g, nullptr, 0, pro);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams cp = {};
        if (e == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = loop;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&nloop, g, &npro, nullptr, 1, &cp);
        }
        if (e == cudaSuccess) e = build_hop_body<Real, NRC>(c, cp.conditional.phGraph_out[0], loop);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&nepi, g, &nloop, 1, epi);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    }
    c->capturing = false;
    c->in_hop_body = false;
    if (pro) cudaGraphDestroy(pro);
    if (epi) cudaGraphDestroy(epi);
    if (s != RT_OK || e != cudaSuccess) {
        if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
        if (g) cudaGraphDestroy(g);
        c->graph_exec = nullptr;
        cudaGetLastError();
        return s != RT_OK ? s : rt_cuda_check(c, e, "graph build");
    }
    c->graph = g;
    c->graph_P = c->d;
    c->graph_hop_cap = c->cfg.hop_cap;
    return RT_OK;
}

template <typename Real, int NRC>
static rt_status step_graph(rt_ctx *c, long long step, cudaStream_t st) {
    bool stale = !c->graph_exec || c->graph_hop_cap != c->cfg.hop_cap ||
                 memcmp(&c->graph_P, &c->d, sizeof(DevPtrs)) != 0;
    rt_status s;
    if (stale && (s = capture_step<Real, NRC>(c))) return s;
    set_step(c, step, st);
    if (c->bm_dirty) {
        clear_cone_bits(c, st);
        c->bm_dirty = false;
    }
    cudaError_t e = cudaGraphLaunch(c->graph_exec, st);
    if (e != cudaSuccess) return rt_cuda_check(c, e, "graph launch");
    cudaMemcpyAsync(c->cnt_h, c->d.cnt, sizeof(long long) * CNT_N, cudaMemcpyDeviceToHost, st);
    if ((s = rt_cuda_check(c, cudaStreamSynchronize(st), "graph step"))) return s;
    long long hops = c->cnt_h[CNT_HOP];
    for (int k = 0; k < KT_N; ++k) {
        long long l = c->graph_launch_step[k] + hops * c->graph_launch_hop[k];
        c->kstat[k].launches += l;
        c->launches += l;
    }
    c->cur = (int)c->cnt_h[CNT_CUR];
    c->fcur = (int)c->cnt_h[CNT_FCUR];
    c->nfree_h = std::min<long long>(c->cnt_h[CNT_NREQ], c->d.F_cap);
    c->stats[3] = c->cnt_h[CNT_SUB];
    c->stats[4] = c->cnt_h[CNT_FLOOR];
    rt_status ts = transport_end(c, sizeof(Real) == 4);
    return ts != RT_OK ? ts : rt_subcycle_status(c);
}

rt_status rt_step_graph(rt_ctx *c, long long step, cudaStream_t st) {
    int nrc = c->d.nrc;
    if (c->d.fp32) return nrc == 8 ? step_graph<float, 8>(c, step, st) : step_graph<float, 32>(c, step, st);
    return nrc == 8 ? step_graph<double, 8>(c, step, st) : step_graph<double, 32>(c, step, st);
}

// ---- launch-size tuning on whole steps -------------------------------------------------------
// With tune_launch the first steps run as the captured step graph, each with one triple of grid
// sizes of the sender side, the virtual particles and the receiver side, and are timed with CUDA
// events around the graph launch, so that the overlap of the two streams is in the objective.
// The time of a step is divided by its work (packets moved, particles sending, virtual
// particles: device counters of that step).  Coordinate search from the built-in sizes, the
// virtual particles first (152 x {2, 3, 4, 5} blocks: at most one wave, since its warps pull
// from a work queue; fewer blocks leave room for the receiver side beside it), then the sender
// and the receiver side (152 x {8, 16, 32, 64} blocks); each candidate step follows a step of
// the current best, so that the pair sees nearly the same work, and replaces it when it costs
// 1% less per unit of work.  The winner is kept
// for the process per (configuration, particles, boxes): a later context of the same kind
// starts with it and does not tune.  The steps run while tuning are ordinary steps: results do
// not depend on the launch sizes.
static std::mutex g_tune_mu;
static std::map<std::string, std::array<int, 3>> g_tune_cache;

static std::string tune_key(const rt_ctx *c) {
    const DevPtrs &P = c->d;
    char buf[256];
    snprintf(buf, sizeof(buf), "%lld/%d/%d/%d/%d/%d/%d/%d/%d", P.n, P.nb, P.kn, P.ntc, P.nrc,
             P.nf, P.fp32, P.rec_mode, P.shared);
    return buf;
}

static void set_grids(rt_ctx *c, const int g[3]) {
    bool same = true;
    for (int k = 0; k < 3; ++k) same &= c->grid_hop[k] == g[k];
    if (same) return;
    for (int k = 0; k < 3; ++k) c->grid_hop[k] = g[k];
    graph_destroy(c);     // the sizes are captured in the graph
}

rt_status rt_step_graph_tuned(rt_ctx *c, long long step, cudaStream_t st) {
    TuneState &U = c->tune;
    if (U.phase == 0) {   // start: a cached winner, or the candidates from the built-in sizes
        const int def[3] = {GRID_A, GRID_V, GRID_B};
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(tune_key(c));
            if (it != g_tune_cache.end()) {
                set_grids(c, it->second.data());
                c->launch_tuned = true;
                return rt_step_graph(c, step, st);
            }
        }
        for (int k = 0; k < 3; ++k) U.best[k] = def[k];
        U.cand.clear();
        const int order[3] = {1, 0, 2};
        for (int kk : order)
            for (int q = 0; q < 4; ++q) {
                int g = kk == 1 ? 152 * (2 + q) : 152 * (8 << q);
                if (g != def[kk]) U.cand.push_back({kk, g});
            }
        U.phase = 1;
        U.steps = 0;
    }
    int g[3] = {U.best[0], U.best[1], U.best[2]};
    if (U.phase == 2) g[U.cand.front().first] = U.cand.front().second;
    set_grids(c, g);
    cudaEventRecord(c->tune_ev[0], st);
    rt_status s = rt_step_graph(c, step, st);
    cudaEventRecord(c->tune_ev[1], st);
    cudaError_t e = cudaEventSynchronize(c->tune_ev[1]);
    if (s != RT_OK) return s;
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->tune_ev[0], c->tune_ev[1]);
    if (e != cudaSuccess) return rt_cuda_check(c, e, "launch-size tuning");
    double work = (double)(c->cnt_h[CNT_ACTS] + c->cnt_h[CNT_ACTP] + c->cnt_h[CNT_VIRT]);
    double cost = (double)ms / (work > 0.0 ? work : 1.0);
    ++U.steps;
    if (U.phase == 1) {
        U.best_cost = cost;
        U.phase = 2;
        return s;
    }
    if (cost < 0.99 * U.best_cost) {
        for (int k = 0; k < 3; ++k) U.best[k] = g[k];
    }
    U.cand.erase(U.cand.begin());
    // the next candidate of the same kernel is compared with the best found so far
    if (U.cand.empty()) {
        set_grids(c, U.best);
        c->launch_tuned = true;
        U.phase = 3;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[tune_key(c)] = {U.best[0], U.best[1], U.best[2]};
    } else {
        U.phase = 1;
    }
    return s;
}

void rt_graph_destroy(rt_ctx *c) { graph_destroy(c); }

rt_status rt_run_step_parts(rt_ctx *c, int part, long long step, cudaStream_t st) {
    int nrc = c->d.nrc;
    if (c->d.fp32) {
        return nrc == 8 ? run_parts<float, 8>(c, part, step, st) : run_parts<float, 32>(c, part, step, st);
    }
    return nrc == 8 ? run_parts<double, 8>(c, part, step, st) : run_parts<double, 32>(c, part, step, st);
}
