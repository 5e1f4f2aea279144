// rt_chem.cu -- per-particle chemistry/thermal update and the per-box photon budget.
//
// Chemistry (Sec. 2.1, Sec. 2.2): photoionisation rate per neutral atom
// Gamma = N_abs / (N_HI dt) and photoheating per neutral atom H = E_abs / (N_HI dt) from the
// step's absorptions; subcycles with the electron density frozen inside each; inside a
// subcycle the exact exponential solution of dx/dt = alpha n_e (1 - x) - (Gamma + beta n_e) x
// and an explicit step of u = 1.5 k T n_H (1 + x_HII) limited to a 10% change (floor dt/sub_cap;
// a subcycle held at the floor is counted, and the step then reports RT_ERR_SUBCYCLE_LIMIT).
// Rates: Hui & Gnedin (1997) recombination, recombination cooling and collisional ionisation;
// Cen (1992) collisional-excitation cooling; free-free with g_ff = 1.3.  The coefficients, their
// values at 1e4, 2e4, 3e4 and 1e5 K and their sources are tabulated in docs/rates (the same table
// as the CPU oracle's); the case-A and case-B coefficients are checked against Osterbrock &
// Ferland (2006, Table 2.1), tests/golden/published_rates.txt.  Case B with
// on-the-spot, case A otherwise; with transport of recombination radiation the ground-level
// recombinations (alpha_A - alpha_B) are the photons emitted next step.
//
// The stiff solve runs in FP64.  The rate fits run in FP64 on the all-FP64 path and in FP32 on
// the mixed path (relative error ~1e-6, far below the 1e-3 tolerance on x_HI and T).
#include "rt_internal.cuh"

static const double K_B = 1.380649e-16;
static const double EV_ERG = 1.602176634e-12;
static const double T_HI = 157807.0;

struct Rates {
    double aA, aB, beta, LA, LB, Lce, Lci, Lff;
};

__device__ __forceinline__ void rates64(double T, Rates &r) {
    double lam = 2.0 * T_HI / T;
    r.aA = 1.269e-13 * pow(lam, 1.503) / pow(1.0 + pow(lam / 0.522, 0.470), 1.923);
    r.aB = 2.753e-14 * pow(lam, 1.500) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
    r.beta = 21.11 * pow(T, -1.5) * exp(-lam / 2.0) * pow(lam, -1.089) /
             pow(1.0 + pow(lam / 0.354, 0.874), 1.101);
    r.LA = 1.778e-29 * T * pow(lam, 1.965) / pow(1.0 + pow(lam / 0.541, 0.502), 2.697);
    r.LB = 3.435e-30 * T * pow(lam, 1.970) / pow(1.0 + pow(lam / 2.250, 0.376), 3.720);
    r.Lce = 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1e5));
    r.Lci = K_B * T_HI * r.beta;
    r.Lff = 1.42e-27 * 1.3 * sqrt(T);
}

// the same fits evaluated in FP32; prefactors below the FP32 range are applied in FP64
__device__ __forceinline__ void rates32(double Td, Rates &r) {
    float T = (float)Td;
    float lam = 2.0f * (float)T_HI / T;
    r.aA = 1.269e-13 * (double)(powf(lam, 1.503f) / powf(1.0f + powf(lam / 0.522f, 0.470f), 1.923f));
    r.aB = 2.753e-14 * (double)(powf(lam, 1.500f) / powf(1.0f + powf(lam / 2.740f, 0.407f), 2.242f));
    r.beta = 21.11 * (double)powf(T, -1.5f) * (double)expf(-0.5f * lam) *
             (double)powf(lam, -1.089f) / (double)powf(1.0f + powf(lam / 0.354f, 0.874f), 1.101f);
    r.LA = 1.778e-29 * Td * (double)(powf(lam, 1.965f) / powf(1.0f + powf(lam / 0.541f, 0.502f), 2.697f));
    r.LB = 3.435e-30 * Td * (double)(powf(lam, 1.970f) / powf(1.0f + powf(lam / 2.250f, 0.376f), 3.720f));
    r.Lce = 7.5e-19 * (double)(expf(-118348.0f / T) / (1.0f + sqrtf(T / 1e5f)));
    r.Lci = K_B * T_HI * r.beta;
    r.Lff = 1.42e-27 * 1.3 * (double)sqrtf(T);
}

template <typename RR>
__global__ void k_chem(DevPtrs P) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nsub = 0, nfloor = 0;
    if (i < P.n) {
        double x = P.xHI[i], T = P.T[i], nH = P.nH[i], NH = P.NH[i];
        double NHI = x * NH;
        double phot = 0.0, heat = 0.0;
        for (int nu = 0; nu < P.nf; ++nu) {
            long long key = i * P.nf + nu;
            phot += P.abs[key] + ((double)P.fx_abs[key] + (double)P.fx_lo[key] / FX_LO_SCALE) *
                                     (NHI / FX_ABS_SCALE);
            heat += P.absE[key] + (double)P.fx_E[key] * (NHI * EV_ERG / FX_E_SCALE);
        }
        P.phot[i] = phot;
        double dt = P.dt;
        double Gam = 0.0, Hh = 0.0;
        if (NHI > 0.0) {
            Gam = phot / (NHI * dt);
            Hh = heat / (NHI * dt);
        }
        double dtmin = dt / (double)P.sub_cap;
        double t = 0.0, Nrec = 0.0;
        bool last = false;
        while (!last) {
            Rates r;
            if (sizeof(RR) == 8) rates64(T, r);
            else rates32(T, r);
            double alpha = (P.rec_mode == RT_REC_OTS_CASE_B) ? r.aB : r.aA;
            double ne = (1.0 - x) * nH;
            double lamx = Gam + r.beta * ne + alpha * ne;
            double h = dt - t;
            double u = 0.0, dudt = 0.0;
            if (P.evolve_T) {
                double xII = 1.0 - x;
                u = 1.5 * K_B * T * nH * (1.0 + xII);
                double Lrec = (P.rec_mode == RT_REC_OTS_CASE_B) ? r.LB : r.LA;
                double cool = 0.0;
                if (P.cool_flags & RT_COOL_REC) cool += ne * (xII * nH) * Lrec;
                if (P.cool_flags & RT_COOL_CEX) cool += ne * (x * nH) * r.Lce;
                if (P.cool_flags & RT_COOL_CION) cool += ne * (x * nH) * r.Lci;
                if (P.cool_flags & RT_COOL_FF) cool += ne * (xII * nH) * r.Lff;
                dudt = x * nH * Hh - cool;
                if (dudt != 0.0) {
                    double ht = 0.1 * u / fabs(dudt);
                    if (ht < h) h = ht;
                }
                // the floor binds only when the 10% limit, not the time left in the step,
                // made the subcycle shorter than dt/sub_cap
                if (h < dtmin) {
                    if (h < dt - t) ++nfloor;
                    h = dtmin;
                }
            }
            if (h >= dt - t) { h = dt - t; last = true; }
            double xn, intII;
            if (lamx > 0.0) {
                double xeq = alpha * ne / lamx;
                double e = exp(-lamx * h);
                xn = xeq + (x - xeq) * e;
                intII = (1.0 - xeq) * h - (x - xeq) * (1.0 - e) / lamx;
            } else {
                xn = x;
                intII = (1.0 - x) * h;
            }
            if (P.rec_mode == RT_REC_TRANSPORT || P.rec_mode == RT_REC_EMISSION_CONES)
                Nrec += (r.aA - r.aB) * ne * NH * intII;
            if (P.evolve_T) {
                double un = u + h * dudt;
                T = un / (1.5 * K_B * nH * (1.0 + (1.0 - xn)));
                if (!(T >= P.T_floor)) T = P.T_floor;
            }
            x = xn;
            t += h;
            ++nsub;
        }
        P.xHI[i] = x;
        P.T[i] = T;
        P.Nrec[i] = Nrec;
        P.epsrec[i] = P.eps_rr_fixed >= 0.0 ? P.eps_rr_fixed : K_B * T;
    }
    // warp-aggregated statistics
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nsub += __shfl_down_sync(FULLMASK, nsub, o);
        nfloor += __shfl_down_sync(FULLMASK, nfloor, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nsub) atomicAdd((unsigned long long *)&P.cnt[CNT_SUB], (unsigned long long)nsub);
        if (nfloor) atomicAdd((unsigned long long *)&P.cnt[CNT_FLOOR], (unsigned long long)nfloor);
    }
}

rt_status rt_chem_launch(rt_ctx *c, cudaStream_t st) {
    DevPtrs &P = c->d;
    cudaMemsetAsync(&P.cnt[CNT_SUB], 0, 2 * sizeof(long long), st);
    unsigned nb = (unsigned)((P.n + 255) / 256);
    kt_begin(c, KT_CHEM, st);
    if (P.fp32) k_chem<float><<<nb, 256, 0, st>>>(P);
    else k_chem<double><<<nb, 256, 0, st>>>(P);
    kt_end(c, KT_CHEM, st);
    return rt_cuda_check(c, cudaGetLastError(), "chemistry");
}

// ---- photon budget: fixed chunks of particles, fixed reduction order --------------------
__device__ double block_sum(double v, double *sh) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    __syncthreads();
    return t;
}

// One block per chunk (a fixed particle range inside one box): partial sums of
// phase 0: the recombination photons of the last chemistry step;
// phase 1: the absorptions, and the photons held in slots.
template <typename Real>
__global__ void k_budget_part(DevPtrs P, int phase) {
    __shared__ double sh[32];
    const int cur = (int)P.cnt[CNT_CUR];
    int ch = blockIdx.x;
    long long i0 = P.bch_lo[ch], i1 = P.bch_lo[ch + 1];
    if (phase == 0) {
        double s = 0.0;
        // the packets' photon counts as emitted: N_rec split over the reception cones, or over
        // K emissions of n_ec emission cones in the original implementation
        double parts = P.rec_mode == RT_REC_EMISSION_CONES ? (double)P.K * P.nec : (double)P.nrc;
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            double Nr = P.Nrec[i];
            if (Nr > 0.0) s += (Nr / parts) * parts;
        }
        double t = block_sum(s, sh);
        if (threadIdx.x == 0) P.bpart[2 * ch] = t;
        return;
    }
    double a = 0.0, fl = 0.0;
    Real *SN = (Real *)P.sl[cur][0];
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        a += P.phot[i];
        for (int nu = 0; nu < P.nf; ++nu) {
            unsigned o = P.occ[cur][i * P.nf + nu];
            while (o) {
                int bb = __ffs(o) - 1;
                o &= o - 1u;
                fl += (double)SN[i * P.S + (long long)nu * P.nrc + bb];
            }
        }
    }
    double ta = block_sum(a, sh);
    double tf = block_sum(fl, sh);
    if (threadIdx.x == 0) {
        P.bpart[2 * ch] = ta;
        P.bpart[2 * ch + 1] = tf;
    }
}

// One thread per box: the box's chunk sums in chunk order.
// phase 0 (at emission): emitted += recombination photons + the box's source photons of one
// step.  phase 1 (end of step): absorbed += absorptions; escaped += fixed-point escapes;
// in flight = photons held in slots.
__global__ void k_budget_fin(DevPtrs P, int phase, const double *src_emit) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= P.nb) return;
    double s0 = 0.0, s1 = 0.0;
    for (int ch = P.box_bch[b]; ch < P.box_bch[b + 1]; ++ch) {
        s0 += P.bpart[2 * ch];
        s1 += P.bpart[2 * ch + 1];
    }
    if (phase == 0) {
        // the box's source photons of this step: sources switched off by their gate send
        // nothing (a directed source sends ndot dt_em per emission, an isotropic one n_ec
        // packets of ndot dt_em / n_ec)
        double src = 0.0;
        if (!P.gated) {
            src = src_emit[b];
        } else {
            for (int j = 0; j < P.ns; ++j) {
                if (P.sbox[j] != b) continue;
                if (P.sgate[j] && !(P.xHI[P.snbr[(long long)j * P.kn]] < 0.5)) continue;
                for (int nu = 0; nu < P.nfs; ++nu)
                    src += P.ndot[(long long)j * P.nfs + nu] * P.dt_em * (double)P.K;
            }
        }
        P.tally[4 * b + 0] += s0 + src;
        return;
    }
    P.tally[4 * b + 1] += s0;
    P.tally[4 * b + 2] += (double)P.esc_fx[b] * (P.ref[b] / FX_ESC_SCALE);
    P.esc_fx[b] = 0ull;
    P.tally[4 * b + 3] = s1 * P.norm[b];
}

rt_status rt_budget_launch(rt_ctx *c, int phase, cudaStream_t st) {
    DevPtrs &P = c->d;
    kt_begin(c, KT_BUDGET, st);
    if (P.fp32) k_budget_part<float><<<P.nbch, 256, 0, st>>>(P, phase);
    else k_budget_part<double><<<P.nbch, 256, 0, st>>>(P, phase);
    k_budget_fin<<<(P.nb + 127) / 128, 128, 0, st>>>(P, phase, c->src_emit);
    kt_end(c, KT_BUDGET, st);
    return rt_cuda_check(c, cudaGetLastError(), "budget");
}
