"""Seeded synthetic inputs shaped like the paper's tests.

This module holds no step of the transport method: it only lays out particles, densities, sources
and their spectra.  Both the CUDA library and the CPU oracle take its output as input.

Workloads (seed = 1000 + number):
  1  Strömgren sphere, Sec. 3 geometry (Iliev et al. 2006 Test 1): 16^3 jittered grid, 13.2 kpc box,
     n_H = 1e-3, T = 1e4 K fixed, 5e48 s^-1 at 13.6 eV, sigma = 6.3e-18, 8 cones, 200 steps of 2.5 Myr.
  2  the same HII region at 64^3 with T evolving, a 1e5 K blackbody in 8 grey bins, 32 cones,
     0.5 Myr steps.
  3  128^3 equal-mass particles, background n_H = 2e-4 with a 0.8 kpc clump at 200x, 5 kpc from a
     3e51 s^-1 source; grey 1e5 K bin (Sec. 4 values); 0.1 Myr steps.
  4  512 independent boxes of 8^3..40^3 particles (log-uniform count), lognormal density fields.
  5  256^3 equal-mass particles sampled from a lognormal field in a 20 Mpc box, 256 sources.
  6  the shadow test of Sec. 4: a plane-parallel front, a disk barrier and boundary emitters
     of recombination radiation (App. B) in a 32^3 box.

All quantities are cgs.  Positions are per box in [0, L).
"""
from __future__ import annotations

import math

import numpy as np

KPC = 3.0857e21
MYR = 3.15576e13
EV = 1.602176634e-12
K_B = 1.380649e-16
T_HI = 157807.0

REC_TRANSPORT, REC_OTS_CASE_B, REC_CASE_A, REC_EMISSION_CONES = 0, 1, 2, 3
COOL_REC, COOL_CEX, COOL_CION, COOL_FF = 1, 2, 4, 8


def default_params(**kw) -> dict:
    p = dict(n_ngb=32, n_ec=8, n_tc=8, n_rc=8, n_freq_src=1, dt=2.5 * MYR, dt_em=2.5 * MYR,
             rec_mode=REC_TRANSPORT, evolve_T=0, seed=1001, hop_cap=4096, sub_cap=100000000,
             cool_flags=COOL_REC | COOL_CEX, T_floor=10.0, eps_rr_fixed=-1.0, sigma_rec=6.3e-18,
             transport_fp32=0, rec_shared_bin=0, tune_launch=0)
    p.update(kw)
    return p


# --- source spectra ------------------------------------------------------------------------
def verner_hi(E_eV):
    """Photoionisation cross-section of H I (Verner et al. 1996 fit), cm^2; 0 below 13.6 eV."""
    E = np.asarray(E_eV, dtype=np.float64)
    E0, s0, ya, P = 4.298e-1, 5.475e-14, 3.288e1, 2.963
    x = E / E0
    y = x
    F = (x - 1.0) ** 2 * y ** (0.5 * P - 5.5) * (1.0 + np.sqrt(y / ya)) ** (-P)
    return np.where(E >= 13.6, s0 * F, 0.0)


def blackbody_bins(T_bb: float, edges_eV) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Grey bins of a blackbody photon spectrum (Sec. 2.1, the grey approximation; optically thin).

    For each bin [E_a, E_b): the fraction of ionising photons in it, the photon-weighted mean
    cross-section <sigma> and the excess energy per photoionisation <eps> = <sigma (E - 13.6 eV)> /
    <sigma>, in erg.  A bin edge of inf integrates to 100 kT.
    """
    kT = K_B * T_bb / EV
    lo = 13.6
    hi_all = 100.0 * kT + lo

    def photons(E):  # photon number per unit energy, up to a constant
        return E * E / np.expm1(E / kT)

    def integ(f, a, b):
        g = np.geomspace(a, b, 200001)
        return np.trapezoid(f(g), g)

    total = integ(photons, lo, hi_all)
    frac, sig, eps = [], [], []
    for a, b in zip(edges_eV[:-1], edges_eV[1:]):
        b = min(b, hi_all)
        n = integ(photons, a, b)
        s = integ(lambda E: photons(E) * verner_hi(E), a, b)
        e = integ(lambda E: photons(E) * verner_hi(E) * (E - 13.6), a, b)
        frac.append(n / total)
        sig.append(s / n)
        eps.append(e / s * EV)
    return np.array(frac), np.array(sig), np.array(eps)


# --- particle layouts -------------------------------------------------------------------------
def jittered_grid(n_side: int, L: float, rng, jitter=0.3):
    s = L / n_side
    i = np.arange(n_side)
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    pos = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1).astype(np.float64) + 0.5
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    pos *= s
    return np.clip(pos, 0.0, np.nextafter(L, 0.0))


def _pack(params, box_L, box_off, pos, n_H, N_H, x_HI, T, src_box, src_pos, src_ndot, sigma, eps):
    return dict(
        params=params, box_L=np.asarray(box_L, float), box_off=np.asarray(box_off, np.int64),
        x=np.ascontiguousarray(pos[:, 0]), y=np.ascontiguousarray(pos[:, 1]),
        z=np.ascontiguousarray(pos[:, 2]), n_H=np.asarray(n_H, float), N_H=np.asarray(N_H, float),
        x_HI=np.asarray(x_HI, float), T=np.asarray(T, float),
        src_box=np.asarray(src_box, np.int32), src_x=np.ascontiguousarray(src_pos[:, 0]),
        src_y=np.ascontiguousarray(src_pos[:, 1]), src_z=np.ascontiguousarray(src_pos[:, 2]),
        src_ndot=np.ascontiguousarray(src_ndot, dtype=float).reshape(-1),
        sigma=np.asarray(sigma, float), eps=np.asarray(eps, float))


def hii_region_state(pos, centre, n_H, ndot, sigma, r_front, x_floor=1e-6):
    """Synthetic mid-expansion HII region: optically thin case-B ionisation balance
    Gamma x = alpha_B n_H (1 - x)^2 inside r_front, neutral outside, T = 1e4 K inside and 100 K
    outside.  Used as the starting state of timed runs; alpha_B = 2.59e-13 (t_rec = 122.4 Myr)."""
    r = np.linalg.norm(pos - centre, axis=1)
    gam = sigma * ndot / (4 * math.pi * np.maximum(r, 1e-3 * KPC) ** 2)
    a = 2.59e-13 * n_H
    # a (1-x)^2 = gam x  ->  a x^2 - (2a + gam) x + a = 0, smaller root
    b = 2 * a + gam
    x_eq = (b - np.sqrt(b * b - 4 * a * a)) / (2 * a)
    x = np.where(r < r_front, np.maximum(x_eq, x_floor), 1.0)
    T = np.where(r < r_front, 1e4, 100.0)
    return x, T


def stromgren_radius(ndot, n_H, alpha_B=2.59e-13):
    return (3 * ndot / (4 * math.pi * alpha_B * n_H * n_H)) ** (1.0 / 3.0)


def cfg1(n_side=16, seed=1001, **kw):
    """Workload 1: Strömgren sphere, 16^3, T = 1e4 K fixed, 13.6 eV source (Sec. 3)."""
    rng = np.random.default_rng(seed)
    L = 13.2 * KPC
    n = n_side ** 3
    pos = jittered_grid(n_side, L, rng)
    nH = np.full(n, 1e-3)
    NH = np.full(n, 1e-3 * L ** 3 / n)
    params = default_params(seed=seed, n_ngb=32, n_ec=8, n_tc=8, n_rc=8, n_freq_src=1,
                            dt=2.5 * MYR, dt_em=2.5 * MYR, evolve_T=0)
    params.update(kw)
    return _pack(params, [L], [0, n], pos, nH, NH, np.ones(n), np.full(n, 1e4), [0],
                 np.array([[0.5 * L, 0.5 * L, 0.5 * L]]), [5e48], [6.3e-18], [0.0])


BB_EDGES_8 = np.concatenate([13.6 * 10.0 ** (np.arange(8) / 7.0), [np.inf]])


def cfg2(n_side=64, seed=1002, ionised=True, **kw):
    """Workload 2: the HII region at 64^3, T evolving, 1e5 K blackbody in 8 bins, 32 cones.

    ionised=True starts from a synthetic mid-expansion state (front at 0.8 R_S), the state the
    timed steps are measured on; False starts neutral at 100 K."""
    rng = np.random.default_rng(seed)
    L = 13.2 * KPC
    n = n_side ** 3
    pos = jittered_grid(n_side, L, rng)
    nH = np.full(n, 1e-3)
    NH = np.full(n, 1e-3 * L ** 3 / n)
    frac, sig, eps = blackbody_bins(1e5, BB_EDGES_8)
    ndot = 5e48 * frac
    centre = np.array([0.5 * L] * 3)
    if ionised:
        s_mean = float(np.sum(frac * sig))
        x, T = hii_region_state(pos, centre, nH, 5e48, s_mean,
                                0.8 * stromgren_radius(5e48, 1e-3))
    else:
        x, T = np.ones(n), np.full(n, 100.0)
    params = default_params(seed=seed, n_ngb=32, n_ec=32, n_tc=32, n_rc=32, n_freq_src=8,
                            dt=0.5 * MYR, dt_em=0.5 * MYR, evolve_T=1, transport_fp32=1)
    params.update(kw)
    return _pack(params, [L], [0, n], pos, nH, NH, x, T, [0], centre[None, :], ndot, sig, eps)


def cfg3(n_total=128 ** 3, seed=1003, rec_mode=REC_TRANSPORT, **kw):
    """Workload 3: clump 200x background, 0.8 kpc radius, 5 kpc from a 3e51 s^-1 source."""
    rng = np.random.default_rng(seed)
    L = 13.2 * KPC
    nb, contrast, rc = 2e-4, 200.0, 0.8 * KPC
    c = np.array([6.6, 6.6, 6.6]) * KPC
    vol_c = 4.0 / 3.0 * math.pi * rc ** 3
    m_c = contrast * nb * vol_c
    m_b = nb * (L ** 3 - vol_c)
    n_c = int(round(n_total * m_c / (m_c + m_b)))
    # background: jittered grid with the clump excluded, thinned to n_total - n_c
    n_side = int(math.ceil(((n_total - n_c) * L ** 3 / (L ** 3 - vol_c)) ** (1 / 3)))
    bg = jittered_grid(n_side, L, rng)
    bg = bg[np.linalg.norm(bg - c, axis=1) >= rc]
    bg = bg[rng.permutation(len(bg))[: n_total - n_c]]
    # clump: finer jittered grid inside the sphere
    s_c = (vol_c / n_c) ** (1 / 3)
    m = int(math.ceil(2 * rc / s_c)) + 2
    g = jittered_grid(m, m * s_c, rng) - 0.5 * m * s_c + c
    g = g[np.linalg.norm(g - c, axis=1) < rc]
    g = g[rng.permutation(len(g))[:n_c]]
    pos = np.concatenate([bg, g])
    inside = np.arange(len(pos)) >= len(bg)
    nH = np.where(inside, contrast * nb, nb)
    N_H = np.full(len(pos), (m_c + m_b) / len(pos))
    params = default_params(seed=seed, n_ec=8, n_tc=8, n_rc=8, n_freq_src=1, dt=0.1 * MYR,
                            dt_em=0.1 * MYR, evolve_T=1, rec_mode=rec_mode, transport_fp32=1)
    params.update(kw)
    n = len(pos)
    return _pack(params, [L], [0, n], pos, nH, N_H, np.ones(n), np.full(n, 100.0), [0],
                 np.array([[1.6 * KPC, 6.6 * KPC, 6.6 * KPC]]), [3e51], [1.6e-18], [6.3 * EV])


def _lognormal_field(G, sigma_ln, slope, rng):
    k = np.fft.fftfreq(G) * G
    kx, ky, kz = np.meshgrid(k, k, k[: G // 2 + 1], indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.where(kk > 0, np.power(np.maximum(kk, 1e-12), slope / 2.0), 0.0)
    noise = rng.standard_normal((G, G, G))
    f = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=(G, G, G), axes=(0, 1, 2))
    f = (f - f.mean()) / f.std() * sigma_ln
    rho = np.exp(f)
    return rho / rho.mean()


def _trilinear(field, pos_frac):
    G = field.shape[0]
    p = pos_frac * G - 0.5
    i0 = np.floor(p).astype(np.int64)
    t = p - i0
    out = np.zeros(len(p))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = (np.where(dx, t[:, 0], 1 - t[:, 0]) * np.where(dy, t[:, 1], 1 - t[:, 1]) *
                     np.where(dz, t[:, 2], 1 - t[:, 2]))
                out += w * field[(i0[:, 0] + dx) % G, (i0[:, 1] + dy) % G, (i0[:, 2] + dz) % G]
    return out


def cfg4(n_boxes=512, seed=1004, n_min=512, n_max=64000, **kw):
    """Workload 4: many independent boxes of uneven size, lognormal densities, central sources."""
    rng = np.random.default_rng(seed)
    L = 13.2 * KPC
    counts = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_boxes)).astype(np.int64)
    box_off = np.concatenate([[0], np.cumsum(counts)])
    pos_all, nH_all, NH_all = [], [], []
    ndot = np.exp(rng.uniform(math.log(1e47), math.log(1e50), n_boxes))
    for b in range(n_boxes):
        n = int(counts[b])
        pos = rng.uniform(0.0, L, size=(n, 3))
        rho = _lognormal_field(32, 1.0, -2.5, rng)
        mean_n = math.exp(rng.uniform(math.log(1e-4), math.log(1e-2)))
        nH = mean_n * _trilinear(rho, pos / L)
        pos_all.append(pos)
        nH_all.append(nH)
        NH_all.append(nH * L ** 3 / n)
    params = default_params(seed=seed, n_ec=8, n_tc=8, n_rc=8, n_freq_src=1, dt=0.5 * MYR,
                            dt_em=0.5 * MYR, evolve_T=1, transport_fp32=1)
    params.update(kw)
    n = int(box_off[-1])
    src = np.tile([0.5 * L] * 3, (n_boxes, 1))
    return _pack(params, np.full(n_boxes, L), box_off, np.concatenate(pos_all),
                 np.concatenate(nH_all), np.concatenate(NH_all), np.ones(n), np.full(n, 100.0),
                 np.arange(n_boxes), src, ndot[:, None], [1.6e-18], [6.3 * EV])


def cfg5(n_side=256, seed=1005, n_src=256, **kw):
    """Workload 5: 256^3 equal-mass particles sampled from a lognormal field, 256 sources."""
    rng = np.random.default_rng(seed)
    L = 20000.0 * KPC
    G = n_side
    rho = _lognormal_field(G, 1.5, -2.5, rng)
    n = n_side ** 3
    p = (rho / rho.sum()).ravel()
    cells = rng.choice(p.size, size=n, p=p)
    ci = np.stack(np.unravel_index(cells, (G, G, G)), 1).astype(np.float64)
    pos = (ci + rng.uniform(0, 1, size=(n, 3))) * (L / G)
    nH = 2e-4 * rho.ravel()[cells]
    N_H = np.full(n, 2e-4 * L ** 3 / n)
    dens_cut = np.quantile(nH, 0.99)
    cand = np.nonzero(nH >= dens_cut)[0]
    pick = rng.choice(cand, size=n_src, replace=False)
    off = rng.normal(size=(n_src, 3))
    off *= 0.25 * (L / n_side) / np.linalg.norm(off, axis=1, keepdims=True)
    src = np.clip(pos[pick] + off, 0.0, np.nextafter(L, 0))
    ndot = np.exp(rng.normal(math.log(1e50), 1.0, n_src))
    params = default_params(seed=seed, n_ec=8, n_tc=8, n_rc=8, n_freq_src=1, dt=1.0 * MYR,
                            dt_em=1.0 * MYR, evolve_T=1, transport_fp32=1)
    params.update(kw)
    return _pack(params, [L], [0, n], pos, nH, N_H, np.ones(n), np.full(n, 100.0),
                 np.zeros(n_src, np.int32), src, ndot[:, None], [1.6e-18], [6.3 * EV])


def shadow(n_side=32, seed=1006, n_front=100, n_bnd=50, barrier=True, boundary=True,
           rec_mode=REC_TRANSPORT, **kw):
    """Workload 6, the shadow test of Sec. 4 (App. B).

    A 13.2 kpc box of n_H = 1e-3 hydrogen on an n_side^3 jittered grid, neutral at 100 K,
    T evolving.  A plane-parallel front of flux F = 1e6 s^-1 cm^-2 enters through x = 0: n_front^2
    directed emitters on that face send their packets along +x (grey 1e5 K bin: sigma = 1.6e-18,
    eps = 6.3 eV).  A disk barrier of radius 0.2 L at (0.27, 0.5, 0.5) L, perpendicular to x,
    removes the packets that cross it.  The recombination radiation of the ionised gas outside
    the box enters from the four sides parallel to x: n_bnd^2 isotropic emitters per side, each
    switched on once the front has passed it, in their own bin (sigma = 6.3e-18, eps = 2.3 eV),
    with the App. B intensity I = 0.63 lambda_mfp E_RR, E_RR = alpha_1 n_H^2 x_HII^2 and
    lambda_mfp = 1251.37 kpc (App. B); alpha_1 = (2/3) alpha_B with alpha_B from t_rec = 122.4
    Myr (Sec. 3) and alpha_1 / alpha_A ~ 0.4 (Sec. 1).  N_TC = 128, N_RC = N_EC = 8,
    dt = dt_em = 0.1 Myr (Sec. 4)."""
    rng = np.random.default_rng(seed)
    L = 13.2 * KPC
    n = n_side ** 3
    pos = jittered_grid(n_side, L, rng)
    nH = np.full(n, 1e-3)
    NH = np.full(n, 1e-3 * L ** 3 / n)
    F = 1e6
    # front emitters on the x = 0 face
    g = (np.arange(n_front) + 0.5) / n_front * L
    fy, fz = np.meshgrid(g, g, indexing="ij")
    front = np.stack([np.zeros(n_front ** 2), fy.ravel(), fz.ravel()], 1)
    # boundary emitters on the y = 0, y = L, z = 0, z = L faces
    gb = (np.arange(n_bnd) + 0.5) / n_bnd * L
    bx, bo = np.meshgrid(gb, gb, indexing="ij")
    bx, bo = bx.ravel(), bo.ravel()
    top = np.nextafter(L, 0.0)
    sides = [np.stack([bx, np.zeros_like(bx), bo], 1), np.stack([bx, np.full_like(bx, top), bo], 1),
             np.stack([bx, bo, np.zeros_like(bx)], 1), np.stack([bx, bo, np.full_like(bx, top)], 1)]
    bnd = np.concatenate(sides) if boundary else np.zeros((0, 3))
    alpha_B = 1.0 / (122.4 * MYR * 1e-3)
    alpha_1 = (2.0 / 3.0) * alpha_B
    I = 0.63 * 1251.37 * KPC * alpha_1 * 1e-3 ** 2          # x_HII ~ 1 in front of the barrier
    src = np.concatenate([front, bnd])
    ndot = np.zeros((len(src), 2))
    ndot[: len(front), 0] = F * (L / n_front) ** 2
    ndot[len(front):, 1] = I * L ** 2 / n_bnd ** 2
    params = default_params(seed=seed, n_ngb=32, n_ec=8, n_tc=128, n_rc=8, n_freq_src=2,
                            dt=0.1 * MYR, dt_em=0.1 * MYR, evolve_T=1, rec_mode=rec_mode,
                            cool_flags=COOL_REC | COOL_CEX)
    params.update(kw)
    wl = _pack(params, [L], [0, n], pos, nH, NH, np.ones(n), np.full(n, 100.0),
               np.zeros(len(src), int), src, ndot, [1.6e-18, 6.3e-18],
               [6.3 * EV, 2.3 * EV])
    wl["src_dir"] = np.zeros((len(src), 3))
    wl["src_dir"][: len(front), 0] = 1.0
    wl["src_gate"] = np.zeros(len(src), np.int32)
    wl["src_gate"][len(front):] = 1
    wl["barriers"] = [(0, 0, np.array([0.27 * L, 0.5 * L, 0.5 * L]), 0.2 * L)] if barrier else []
    return wl


def split_sources(wl: dict, n_src: int, spread=0.02, seed=11) -> dict:
    """The same workload with its first source's photons split equally over n_src sources
    placed uniformly within +-spread of the box side around it (one cluster of sources where
    one sat); the total luminosity per frequency bin is unchanged."""
    if n_src <= 1:
        return wl
    rng = np.random.default_rng(seed)
    b = int(wl["src_box"][0])
    L = float(wl["box_L"][b])
    c = np.array([wl["src_x"][0], wl["src_y"][0], wl["src_z"][0]])
    pos = np.clip(c + rng.uniform(-spread, spread, (n_src, 3)) * L, 0.0, np.nextafter(L, 0.0))
    nfs = wl["params"]["n_freq_src"]
    ndot = np.asarray(wl["src_ndot"], dtype=np.float64).reshape(len(wl["src_box"]), nfs)[0]
    out = dict(wl)
    out.update(src_box=np.full(n_src, b, np.int32), src_x=pos[:, 0].copy(), src_y=pos[:, 1].copy(),
               src_z=pos[:, 2].copy(), src_ndot=np.tile(ndot / n_src, n_src))
    return out


def tiny(n=200, seed=7, n_ngb=16, L=1.0 * KPC, **kw):
    """Small random box for brute-force and edge-case checks."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, size=(n, 3))
    nH = np.exp(rng.normal(math.log(1e-3), 0.5, n))
    NH = nH * L ** 3 / n
    params = default_params(seed=seed, n_ngb=n_ngb, dt=0.05 * MYR, dt_em=0.05 * MYR)
    params.update(kw)
    return _pack(params, [L], [0, n], pos, nH, NH, np.full(n, 0.5), np.full(n, 1e4), [0],
                 np.array([[0.5 * L] * 3]), [1e47], [6.3e-18], [0.0])
