"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test would fail on a plausible mistake in the oracle: a wrong generator constant, a cone of
the wrong opening angle, a transposed rotation, a dropped N_HI or dt in the rates, a wrong energy
normalisation, a photon leak, a wrong recombination coefficient, an unequal split or a merge
weighted before absorption, a virtual particle drawn outside its cone or weighted wrongly, a
packet left in its old cone at the step start, or a source emission of the wrong size.
Brute-force tests recompute small cases directly from the definitions; copies of the oracle
with such mistakes planted in them fail those tests.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1311_0182_gb300 import workloads as W
from conftest import golden, paper_values

KPC, MYR, EV, K_B = W.KPC, W.MYR, W.EV, W.K_B


# --- generator --------------------------------------------------------------------------------
def test_philox_known_answers():
    n = 0
    for line in open(golden("philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert list(oracle.philox(v[0:4], v[4:6])) == v[6:10]
        n += 1
    assert n == 3


def test_splitmix_known_answers():
    g = 0x9E3779B97F4A7C15
    for line in open(golden("splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, val = line.split()
        assert oracle.mix64((int(k) - 1) * g % (1 << 64)) == int(val, 16)


# --- cone direction sets and rotations ----------------------------------------------------------
@pytest.mark.parametrize("n", [8, 32])
def test_axis_sets_isotropic(n):
    A = oracle.axis_set(n)
    assert np.allclose(np.linalg.norm(A, axis=1), 1.0, atol=1e-15)
    assert np.allclose(A.sum(0), 0.0, atol=1e-14)               # no preferred direction
    assert np.allclose(A.T @ A / n, np.eye(3) / 3, atol=1e-14)  # isotropic second moment
    # every direction's antipode is in the set
    for a in A:
        assert np.min(np.linalg.norm(A + a, axis=1)) < 1e-14
    G = A @ A.T
    np.fill_diagonal(G, -2)
    nearest = G.max(1)
    if n == 8:   # cube diagonals: nearest neighbours at cos = 1/3
        assert np.allclose(nearest, 1 / 3)
    else:        # icosahedron vertices (first 12) and dodecahedron vertices (last 20)
        ico, dod = A[:12], A[12:]
        Gi = ico @ ico.T
        np.fill_diagonal(Gi, -2)
        assert np.allclose(Gi.max(1), 1 / math.sqrt(5))
        Gd = dod @ dod.T
        np.fill_diagonal(Gd, -2)
        assert np.allclose(Gd.max(1), math.sqrt(5) / 3)


def test_rotations_are_uniform_rotations():
    Rs = np.array([oracle.rotation(1234, 1, 7, 0, i) for i in range(4000)])
    for R in Rs[:50]:
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
    # Haar measure: E[R] = 0 and the image of a fixed axis is uniform on the sphere
    assert np.abs(Rs.mean(0)).max() < 4 / math.sqrt(4000)
    v = Rs[:, :, 2]
    assert np.allclose(v.T @ v / len(v), np.eye(3) / 3, atol=0.03)
    # different counters give different rotations
    assert not np.allclose(Rs[0], Rs[1])


def test_transmission_cone_solid_angle():
    """The cone holds the directions within arccos(1 - 2/N_TC) of the axis: solid angle 4pi/N_TC."""
    rng = np.random.default_rng(3)
    for n_tc in (2, 8, 32, 128):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        dirs = rng.normal(size=(20000, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        delta = np.rint(dirs * 1e5).astype(np.int64)
        inside = np.array([oracle.in_cone(x, d, n_tc) for x in delta])
        frac = inside.mean()
        sd = math.sqrt((1 / n_tc) * (1 - 1 / n_tc) / len(dirs))
        assert abs(frac - 1 / n_tc) < 5 * sd + 1e-4
        # agreement with the angle computed from scratch, away from the cone edge
        ang = np.degrees(np.arccos(np.clip(delta @ d / np.linalg.norm(delta, axis=1), -1, 1)))
        half = math.degrees(math.acos(1 - 2 / n_tc))
        far = np.abs(ang - half) > 1e-3
        assert np.array_equal(inside[far], (ang < half)[far])
    assert not oracle.in_cone([0, 0, 0], [1.0, 0, 0], 8)   # coincident neighbour never inside


def test_reception_bin_is_nearest_rotated_axis():
    rng = np.random.default_rng(4)
    for n in (8, 32):
        A = oracle.axis_set(n)
        R = oracle.rotation(99, 1, 1, 2, 3)
        counts = np.zeros(n)
        for _ in range(4000):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            b = oracle.recv_bin(R, A, d)
            assert b == int(np.argmax((R @ A.T).T @ d))
            counts[b] += 1
        if n == 8:  # cube-diagonal cones are the 8 octants of the rotated frame
            assert np.all(np.abs(counts / 4000 - 1 / 8) < 0.03)


# --- neighbours ---------------------------------------------------------------------------------
def _brute_knn(pts, q, k, self_idx=None):
    d2 = ((pts - q) ** 2).sum(1)
    idx = np.arange(len(pts))
    keep = idx != self_idx if self_idx is not None else np.ones(len(pts), bool)
    order = np.lexsort((idx[keep], d2[keep]))[:k]
    return idx[keep][order], d2[keep][order]


@pytest.mark.parametrize("kind", ["uniform", "clustered", "lattice"])
def test_knn_grid_equals_brute_force(kind):
    rng = np.random.default_rng(5)
    Q = 1 << 20
    if kind == "uniform":
        pts = rng.integers(0, Q, size=(1500, 3))
    elif kind == "clustered":   # tight clumps, exact duplicates and empty space
        c = rng.integers(0, Q, size=(6, 3))
        pts = np.clip(c[rng.integers(0, 6, 1500)] + rng.normal(0, 3000, (1500, 3)), 0, Q - 1)
        pts = pts.astype(np.int64)
        pts[100:140] = pts[99]
    else:                       # exact lattice: many equal distances, ties go to the lower index
        g = np.arange(11) * (Q // 11)
        pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    k = 32
    i_grid, d_grid = oracle.knn(pts, pts, k, self_offset=0, use_grid=True)
    i_br, d_br = oracle.knn(pts, pts, k, self_offset=0, use_grid=False)
    assert np.array_equal(i_grid, i_br) and np.array_equal(d_grid, d_br)
    for t in range(0, len(pts), 97):
        ib, db = _brute_knn(pts, pts[t], k, self_idx=t)
        assert np.array_equal(i_grid[t], ib) and np.array_equal(d_grid[t], db)
    # arbitrary query points (virtual particles, sources)
    qs = rng.integers(0, Q, size=(200, 3))
    i_g, d_g = oracle.knn(pts, qs, k, use_grid=True)
    for t in range(200):
        ib, db = _brute_knn(pts, qs[t], k)
        assert np.array_equal(i_g[t], ib) and np.array_equal(d_g[t], db)


# --- rates and chemistry ---------------------------------------------------------------------------
def test_recombination_coefficients_match_paper():
    pv = paper_values()
    r = oracle.rates(1e4)
    t_rec = 1 / (r["alpha_B"] * 1e-3) / MYR
    v, tol = pv["t_rec_Myr"]
    assert abs(t_rec / v - 1) < tol
    v, tol = pv["alphaB_over_alphaA"]
    assert abs(r["alpha_B"] / r["alpha_A"] / v - 1) < tol
    v, tol = pv["ionising_recomb_fraction"]
    assert abs((r["alpha_A"] - r["alpha_B"]) / r["alpha_A"] / v - 1) < tol
    # mean energy carried off by a recombining electron is below ~kT (Osterbrock's beta/alpha)
    for case in ("A", "B"):
        ratio = r[f"Lrec_{case}"] / (K_B * 1e4 * r[f"alpha_{case}"])
        assert 0.5 < ratio < 1.0
    # recombination slows with temperature; collisional ionisation and excitation grow
    r2 = oracle.rates(2e4)
    assert r2["alpha_A"] < r["alpha_A"] and r2["beta"] > r["beta"] and r2["L_cex"] > r["L_cex"]


def test_recombination_coefficients_match_published_tables():
    """The case-A and case-B recombination coefficients of the chemistry (Hui & Gnedin 1997
    fits, named in Sec. 2.1) against the tabulated values of Osterbrock & Ferland (2006) at
    5000, 10^4 and 2 x 10^4 K (tests/golden/published_rates.txt)."""
    n = 0
    with open(golden("published_rates.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, T, v, tol = line.split()[:4]
            got = oracle.rates(float(T))[name]
            assert abs(got / float(v) - 1) < float(tol), (name, T, got, v)
            n += 1
    assert n == 6


def test_recombination_cooling_energy_per_recombination():
    """Recombination cooling removes a fraction of kT per recombination that falls with T
    (the recombining electrons are the slow ones): between 0.45 and 0.8 kT over 10^4-10^5 K,
    more per case-A recombination than per case-B one."""
    k = 1.380649e-16
    prev = None
    for T in (1e4, 2e4, 3e4, 1e5):
        r = oracle.rates(T)
        eA = r["Lrec_A"] / (k * T * r["alpha_A"])
        eB = r["Lrec_B"] / (k * T * r["alpha_B"])
        assert 0.45 < eB < eA < 0.8
        if prev is not None:
            assert eB < prev
        prev = eB


def test_collisional_ionisation_cooling_removes_the_ionisation_energy():
    """Each collisional ionisation takes the 13.598 eV ionisation energy of hydrogen out of the
    gas, so its cooling rate coefficient is that energy times the ionisation coefficient; the
    free-free rate grows as sqrt(T) (constant Gaunt factor)."""
    for T in (1e4, 3e4, 1e5, 1e6):
        r = oracle.rates(T)
        assert abs(r["L_cion"] / r["beta"] / EV / 13.598 - 1) < 2e-4
        assert abs(oracle.rates(4 * T)["L_ff"] / r["L_ff"] - 2) < 1e-12


def _activation_temperature(name, T, h=1e-3):
    """-d ln(rate) / d(1/T) at T, by a central difference in 1/T."""
    u = 1.0 / T
    a = oracle.rates(1.0 / (u * (1 + h)))[name]
    b = oracle.rates(1.0 / (u * (1 - h)))[name]
    return -(math.log(a) - math.log(b)) / (2 * h * u)


def test_collisional_rates_have_the_atomic_activation_energies():
    """A collisional rate of H I is a Boltzmann factor exp(-E/kT) times a slowly varying
    function of T, with E the energy the collision must supply.  So -d ln(rate)/d(1/T) tends to
    E/k as T falls, with corrections of order T:
    - collisional ionisation (beta): the ionisation energy of hydrogen, 13.598 eV;
    - collisional excitation cooling: the excitation of the n = 2 level, 3/4 of 13.598 eV
      (the Lyman-alpha energy, 10.2 eV).
    A fit with the wrong level, the wrong energy or a mistyped exponent fails."""
    E_ion = 13.598 * EV / K_B
    E_12 = 0.75 * E_ion
    for T, tol in ((1000.0, 0.005), (2000.0, 0.01)):
        assert abs(_activation_temperature("beta", T) / E_ion - 1) < tol
        assert abs(_activation_temperature("L_cex", T) / E_12 - 1) < tol / 2


def test_free_free_cooling_has_the_textbook_normalisation():
    """Thermal bremsstrahlung of a hydrogen plasma emits 1.4e-27 T^(1/2) n_e n_p g_B erg cm^-3
    s^-1, with the frequency-averaged Gaunt factor g_B between 1.1 and 1.5 (Rybicki & Lightman
    1979, Eq. 5.15b and the text after it)."""
    for T in (1e4, 3e4, 1e5, 1e6):
        g = oracle.rates(T)["L_ff"] / (1.4e-27 * math.sqrt(T))
        assert 1.1 <= g <= 1.5, (T, g)


def test_recombination_heating_energy():
    v, tol = paper_values()["kT_27000K_eV"]
    assert abs(K_B * 27000 / EV / v - 1) < tol


def _params(**kw):
    return W.default_params(**kw)


def test_chemistry_equilibrium_reproduces_appendix_b():
    """Plane-parallel front of App. B: Gamma = sigma F, case B, T = 1e4 K; the converged neutral
    fraction gives lambda_mfp and the Stromgren distance printed in the paper."""
    pv = paper_values()
    sigma, F, nH = 1.6e-18, 1e6, 1e-3
    p = _params(rec_mode=W.REC_OTS_CASE_B, evolve_T=0, dt=0.1 * MYR)
    NH = 1e60
    x, T = 1.0, 1e4
    for _ in range(20000):      # 2 Gyr: many recombination times
        phot = sigma * F * (x * NH) * p["dt"]
        x, T, nrec, nsub, _f = oracle.chem_particle(p, nH, NH, phot, 0.0, x, T)
    r = oracle.rates(1e4)
    aB = r["alpha_B"]
    # the quadratic of the ion balance sigma F x = alpha_B n_H (1-x)^2 (App. B) ...
    a, b = aB * nH, sigma * F
    x_quad = ((2 * a + b) - math.sqrt((2 * a + b) ** 2 - 4 * a * a)) / (2 * a)
    assert abs(x / x_quad - 1) < 2e-6
    # ... plus collisional ionisation beta n_e x, which App. B leaves out (beta n_e/Gamma ~ 6e-7)
    xs = x_quad
    for _ in range(50):
        g = b + r["beta"] * nH * (1 - xs)
        xs = ((2 * a + g) - math.sqrt((2 * a + g) ** 2 - 4 * a * a)) / (2 * a)
    assert abs(x / xs - 1) < 1e-9
    lam = 1 / (sigma * nH * x) / KPC
    v, tol = pv["lambda_mfp_kpc"]
    assert abs(lam / v - 1) < tol
    v, tol = pv["L_strom_kpc"]
    assert abs(F / (aB * nH * nH) / KPC / v - 1) < tol
    assert nrec == 0.0       # no recombination photons emitted on the spot


def test_chemistry_photon_accounting_and_recombination_photons():
    p = _params(rec_mode=W.REC_TRANSPORT, evolve_T=0, dt=0.01 * MYR)
    nH, NH = 1e-3, 1e60
    # small photon dose into neutral gas: every absorbed photon ionises one atom
    phot = 1e-4 * NH
    x, T, nrec, _, _ = oracle.chem_particle(p, nH, NH, phot, 0.0, 1.0, 1e4)
    assert abs((1 - x) * NH / phot - 1) < 1e-3
    # partially ionised gas: the rate is per neutral atom, so the absorbed photons still ionise
    # as many atoms (against the same step without photons, which recombines a little)
    x0 = 0.3
    dose = 1e-5 * x0 * NH
    xa = oracle.chem_particle(p, nH, NH, 0.0, 0.0, x0, 1e4)[0]
    xb = oracle.chem_particle(p, nH, NH, dose, 0.0, x0, 1e4)[0]
    assert abs((xa - xb) * NH / dose - 1) < 1e-2
    # fully ionised gas without photons: ground-level recombinations alpha_1 n_e n_HII V dt
    x, T, nrec, _, _ = oracle.chem_particle(p, nH, NH, 0.0, 0.0, 0.0, 1e4)
    r = oracle.rates(1e4)
    expect = (r["alpha_A"] - r["alpha_B"]) * nH * NH * p["dt"]
    assert abs(nrec / expect - 1) < 2e-3
    assert abs(x - r["alpha_A"] * nH * p["dt"]) < 2e-3 * x
    # case A and on-the-spot modes emit nothing
    for mode in (W.REC_OTS_CASE_B, W.REC_CASE_A):
        q = _params(rec_mode=mode, evolve_T=0, dt=0.01 * MYR)
        assert oracle.chem_particle(q, nH, NH, 0.0, 0.0, 0.0, 1e4)[2] == 0.0


def test_chemistry_heating_normalisation():
    """Absorbed energy E raises T by E / (1.5 k N_H (1 + x_HII)) when nothing else happens."""
    p = _params(evolve_T=1, cool_flags=0, dt=0.01 * MYR, sub_cap=100000)
    nH, NH = 1e-3, 1e60
    E = 1e-6 * NH * EV * 13.6
    x0 = 0.999999
    x, T, _, nsub, _ = oracle.chem_particle(p, nH, NH, 1e-12 * NH, E, x0, 100.0)
    dT = E / (1.5 * K_B * NH * (1 + (1 - x0)))
    assert abs((T - 100.0) / dT - 1) < 1e-3
    assert nsub >= 1


def test_chemistry_cooling_reaches_floor_and_subcycles_bounded():
    p = _params(evolve_T=1, cool_flags=15, dt=5 * MYR, sub_cap=2000)
    x, T, _, nsub, nfloor = oracle.chem_particle(p, 1.0, 1e60, 0.0, 0.0, 0.01, 1e6)
    assert T < 1e6 and T >= p["T_floor"]
    assert nsub <= p["sub_cap"] + 1


def test_subcycle_floor_hits_are_the_subcycles_the_floor_lengthened():
    """A floor hit is counted exactly when the floor dt/sub_cap made a subcycle longer than the
    10% energy limit allowed: with no hit counted, a floor 1000 times lower gives the same
    result bit for bit (the last, shortened subcycle of a step is not a hit); with a hit it
    gives another result."""
    rng = np.random.default_rng(5)
    hits = quiet = 0
    for _ in range(400):
        sc = int(rng.choice([20, 200, 2000]))
        p = _params(evolve_T=1, cool_flags=3, dt=0.5 * MYR, sub_cap=sc)
        nH, NH = 10 ** rng.uniform(-4, -2), 1e60
        x0, T0 = rng.uniform(0.01, 1.0), 10 ** rng.uniform(2, 4.5)
        phot = 10 ** rng.uniform(-6, 0) * x0 * NH
        heat = phot * 10 ** rng.uniform(0, 1.5) * EV
        r1 = oracle.chem_particle(p, nH, NH, phot, heat, x0, T0)
        r2 = oracle.chem_particle(dict(p, sub_cap=1000 * sc), nH, NH, phot, heat, x0, T0)
        if r1[4] == 0:
            quiet += 1
            assert r1[:3] == r2[:3]
        else:
            hits += 1
            assert r1[:3] != r2[:3]
    assert hits >= 10 and quiet >= 10


def test_subcycle_floor_is_an_error_status_of_the_step():
    """Sec. 2.1 chemistry with a floor too high for the heating at the front: the step still
    completes (state written, budget closed) and reports the floor (status 9)."""
    wl = W.cfg2(n_side=12, sub_cap=4)
    s = oracle.Sim(wl)
    s.build_neighbours()
    assert s.step(0) == 9
    assert s.stats()["floor_hits"] > 0
    b = s.budget()[0]
    assert abs(b[0] - b[1:].sum()) <= 1e-12 * b[0]
    s2 = oracle.Sim(W.cfg2(n_side=12))
    s2.build_neighbours()
    assert s2.step(0) == 0 and s2.stats()["floor_hits"] == 0


# --- transport ------------------------------------------------------------------------------------
def test_grey_bins_of_1e5K_blackbody_match_paper():
    pv = paper_values()
    frac, sig, eps = W.blackbody_bins(1e5, [13.6, np.inf])
    v, tol = pv["grey_sigma_1e5K_cm2"]
    assert abs(sig[0] / v - 1) < tol
    v, tol = pv["grey_eps_1e5K_eV"]
    assert abs(eps[0] / EV / v - 1) < tol
    v, tol = pv["sigma_13p6_cm2"]
    assert abs(W.verner_hi(13.6) / v - 1) < tol
    frac8, sig8, eps8 = W.blackbody_bins(1e5, W.BB_EDGES_8)
    assert abs(frac8.sum() - 1) < 1e-6 and np.all(np.diff(sig8) < 0)


def _run(wl, steps):
    s = oracle.Sim(wl)
    s.build_neighbours()
    for st in range(steps):
        assert s.step(st) == 0
    return s


def test_photon_conservation_cfg1():
    s = _run(W.cfg1(), 12)
    e, a, esc, fl = s.budget()[0]
    assert e > 0 and a > 0 and esc > 0
    assert abs(e - a - esc - fl) <= 1e-12 * e


def test_photon_conservation_virtual_heavy():
    wl = W.tiny(n=600, n_ngb=16, n_tc=64, n_rc=32, n_ec=32)
    wl["x_HI"][:] = 0.05
    s = _run(wl, 4)
    st = s.stats()
    assert st["virtual"] > 100
    e, a, esc, fl = s.budget()[0]
    assert abs(e - a - esc - fl) <= 1e-12 * e


def test_optically_thin_box_lets_every_photon_escape():
    wl = W.cfg1()
    wl["x_HI"][:] = 0.0
    s = _run(wl, 1)       # one step: afterwards the gas has recombined and is no longer thin
    e, a, esc, fl = s.budget()[0]
    assert a == 0.0 and fl == 0.0
    assert abs(esc / e - 1) < 1e-12
    assert np.all(s.deposits()[0] == 0.0)


def test_recombination_emission_is_isotropic_and_complete():
    wl = W.cfg1()
    s = oracle.Sim(wl)
    s.build_neighbours()
    n = s.n
    nrec = np.zeros(n)
    nrec[[5, 77, 2000]] = [1e55, 3e54, 7e53]
    s.set_state(N_rec=nrec, eps_rec=np.full(n, 2 * EV))
    s.rotate(3)
    s.rebin()
    s.emit(3)
    f = s.slots()
    rec = slice(8, 16)   # recombination bin: the last 8 slots
    N = f[0][:, rec].sum(1)
    assert np.allclose(N[[5, 77, 2000]], nrec[[5, 77, 2000]], rtol=1e-14)
    for i in (5, 77, 2000):
        M = f[1:4, i, rec].sum(1)
        assert np.linalg.norm(M) < 1e-13 * N[i]          # isotropic: net momentum cancels
        assert np.allclose(f[5, i, rec].sum(), 2 * EV * N[i], rtol=1e-14)
        assert np.all(f[4, i, rec] == 0.0)                # clocks start at the step start


def _chain(n_part=40, spacing=0.1 * KPC, nH=1e-3, xHI=1e-2, steps_dt=None):
    """Particles on a line with two neighbours each: a packet sent along the line can only reach
    the next particle, so its photon count follows Beer-Lambert hop by hop."""
    L = (n_part + 1) * spacing
    x = (np.arange(n_part) + 0.5) * spacing
    yz = np.full(n_part, 0.5 * L)
    wl = W.tiny(n=n_part, n_ngb=2, L=L, n_tc=64)
    wl.update(x=x, y=yz.copy(), z=yz.copy(), n_H=np.full(n_part, nH),
              N_H=np.full(n_part, nH * spacing ** 3), x_HI=np.full(n_part, xHI),
              T=np.full(n_part, 1e4), src_box=np.zeros(0, np.int32), src_x=np.zeros(0),
              src_y=np.zeros(0), src_z=np.zeros(0), src_ndot=np.zeros(0))
    if steps_dt is not None:
        wl["params"]["dt"] = wl["params"]["dt_em"] = steps_dt
    return wl


def _put_packet(s, i, N, d):
    f = np.zeros((6, s.n, s.S))
    b = oracle.recv_bin(s.rotations()[0][i].reshape(3, 3), oracle.axis_set(s.params["n_rc"]), d)
    f[0, i, b] = N
    f[1:4, i, b] = N * np.asarray(d)
    s.set_slots(f)


def test_beer_lambert_chain():
    wl = _chain()
    s = oracle.Sim(wl)
    s.build_neighbours()
    s.rotate(0)
    s.emit(0)
    N0 = 1e50
    # particle 1's two neighbours are particles 0 and 2: only 2 lies in a +x cone, and so on
    _put_packet(s, 1, N0, [1.0, 0.0, 0.0])
    assert s.transport(0) == 0
    a = s.deposits()[0][:, 0]
    sigma = wl["sigma"][0]
    q = s.quantised()
    u = wl["box_L"][0] / (1 << 20)
    l = np.diff(q[1:, 0]) * u                     # projected hop lengths 1->2, 2->3, ...
    tau = sigma * wl["x_HI"][2:] * wl["n_H"][2:] * l
    N = N0 * np.exp(-np.concatenate([[0.0], np.cumsum(tau)]))   # photons arriving at 1, 2, ...
    assert a[0] == 0.0 and a[1] == 0.0
    # arrivals up to the second-to-last particle (the last one has no neighbour ahead and hands
    # its photons to a virtual particle, which may still deposit some near the end of the chain)
    assert np.allclose(a[2:-2], N[:-3] - N[1:-2], rtol=1e-12, atol=0)
    e, ab, esc, fl = s.budget()[0]
    assert abs(ab + esc - N0) <= 1e-12 * N0 and fl == 0.0
    assert esc <= N[-1] * (1 + 1e-12)


def test_clock_stops_packet_after_c_dt():
    spacing = 0.1 * KPC
    m = 7
    dt = (m - 0.5) * spacing / 2.99792458e10     # light crosses 6.5 spacings in one step
    wl = _chain(xHI=0.0, steps_dt=dt)
    s = oracle.Sim(wl)
    s.build_neighbours()
    s.rotate(0)
    s.emit(0)
    _put_packet(s, 1, 1e50, [1.0, 0.0, 0.0])
    assert s.transport(0) == 0
    f = s.slots()
    held = np.nonzero(f[0].sum(1))[0]
    assert list(held) == [m + 1]                  # stopped at the first particle past c dt
    i = held[0]
    clock = f[4, i].sum() / f[0, i].sum()
    q = s.quantised()
    u = wl["box_L"][0] / (1 << 20)
    assert abs(clock - (q[m + 1, 0] - q[1, 0]) * u / 2.99792458e10) < 1e-9 * clock
    # the next step restarts its clock and carries it further
    s.rotate(1)
    s.rebin()
    assert np.all(s.slots()[4] == 0.0)


def _one_hop_box(seed, n=12, n_tc=8, n_emit=5):
    """A box of n particles, each the neighbour of all the others (n_ngb = n - 1), with packets
    planted at n_emit of them, pointing within a few degrees of one common direction (so that
    arrivals share reception cones), each with a non-empty transmission cone, clocks already
    started, and dt short enough that every packet stops after one hop.  Returns None when
    some neighbour lies within 1e-9 of a cone's edge in cos, or too few emitters qualify."""
    rng = np.random.default_rng(seed)
    L = 1.0 * KPC
    wl = W.tiny(n=n, seed=seed, n_ngb=n - 1, L=L, n_tc=n_tc)
    wl.update(x_HI=rng.uniform(0.0, 0.9, n), src_box=np.zeros(0, np.int32), src_x=np.zeros(0),
              src_y=np.zeros(0), src_z=np.zeros(0), src_ndot=np.zeros(0))
    s = oracle.Sim(wl)
    q = s.quantised().astype(np.float64)
    u = L / (1 << 20)
    cmin = 1.0 - 2.0 / n_tc
    d0 = rng.normal(size=3)
    d0 /= np.linalg.norm(d0)
    pk = []
    for e in rng.permutation(n):
        d = d0 + rng.normal(0.0, 0.05, 3)
        d /= np.linalg.norm(d)
        members, l = [], []
        for j in range(n):
            if j == e:
                continue
            delta = q[j] - q[e]
            cosang = delta @ d / np.linalg.norm(delta)
            if abs(cosang - cmin) < 1e-9:
                return None
            if cosang > cmin:
                members.append(j)
                l.append((delta @ d) * u)
        if not members:
            continue
        pk.append(dict(e=e, d=d, members=members, l=np.array(l), N=rng.uniform(1e48, 1e50),
                       eps=rng.uniform(1.0, 5.0) * EV))
        if len(pk) == n_emit:
            break
    if len(pk) < n_emit:
        return None
    dt = 0.5 * min(p["l"].min() for p in pk) / 2.99792458e10
    for p in pk:
        p["clock"] = rng.uniform(0.0, 0.3) * dt
    wl["params"]["dt"] = wl["params"]["dt_em"] = dt
    return wl, pk


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_one_hop_splits_equally_among_cone_members_and_merges_photon_weighted(seed):
    """Brute force on tiny boxes (Sec. 2.1): a packet of N photons shares them equally among the
    k neighbours inside its transmission cone; each share loses 1 - exp(-sigma n_HI l) on the way
    (l the hop projected on the packet's direction) and arrives in the reception cone of its
    direction at the receiver, where the arrivals merge.  The merged packet's photons, momentum
    and energy are the sums; its clock is the photon-weighted mean of the arriving clocks, each
    the sender's clock plus l / c."""
    made = None
    for k in range(20):
        made = _one_hop_box(1000 * seed + k)
        if made is not None:
            break
    wl, pk = made
    s = oracle.Sim(wl)
    s.build_neighbours()
    s.rotate(0)
    s.emit(0)
    axes = oracle.axis_set(wl["params"]["n_rc"])
    R = s.rotations()[0]
    f = np.zeros((6, s.n, s.S))
    for p in pk:
        b = oracle.recv_bin(R[p["e"]].reshape(3, 3), axes, p["d"])
        f[0, p["e"], b] = p["N"]
        f[1:4, p["e"], b] = p["N"] * p["d"]
        f[4, p["e"], b] = p["N"] * p["clock"]
        f[5, p["e"], b] = p["N"] * p["eps"]
    s.set_slots(f)
    assert s.transport(0) == 0
    sigma = wl["sigma"][0]
    nHI = wl["x_HI"] * wl["n_H"]
    want = np.zeros((6, s.n, s.S))
    absorbed = np.zeros(s.n)
    arrivals = np.zeros((s.n, s.S), int)
    for p in pk:
        w = p["N"] / len(p["members"])
        for j, l in zip(p["members"], p["l"]):
            T = w * math.exp(-sigma * nHI[j] * l)
            absorbed[j] += w - T
            b = oracle.recv_bin(R[j].reshape(3, 3), axes, p["d"])
            want[0, j, b] += T
            want[1:4, j, b] += T * p["d"]
            want[4, j, b] += T * (p["clock"] + l / 2.99792458e10)
            want[5, j, b] += T * p["eps"]
            arrivals[j, b] += 1
    assert arrivals.max() >= 2          # some slot merges packets from two senders
    got = s.slots()
    scale = np.abs(want).max(axis=(1, 2), keepdims=True)
    assert np.all(np.abs(got - want) <= 1e-12 * scale)
    held = want[0] > 0
    assert np.allclose(got[4][held] / got[0][held], want[4][held] / want[0][held], rtol=1e-12)
    assert np.allclose(s.deposits()[0][:, 0], absorbed, rtol=1e-11, atol=1e-12 * absorbed.max())
    e, ab, esc, fl = s.budget()[0]
    total = sum(p["N"] for p in pk)
    assert esc == 0.0 and abs(ab - absorbed.sum()) <= 1e-12 * total
    st = s.stats()
    assert st["virtual"] == 0 and st["hops"] == 1   # no empty cone; every packet stopped


def _virtual_hop_receivers(seed):
    """One packet sent into an empty cone in a uniform medium; returns its receiver count."""
    rng = np.random.default_rng(seed)
    L = 1.0 * KPC
    c0 = np.full(3, 0.5)
    d = np.array([1.0, 0.0, 0.0])

    def dirs(m, cos_lo, cos_hi):
        ct = rng.uniform(cos_lo, cos_hi, m)
        ph = rng.uniform(0.0, 2 * np.pi, m)
        st = np.sqrt(1 - ct ** 2)
        return np.stack([ct, st * np.cos(ph), st * np.sin(ph)], 1)

    n_ngb = 8
    behind = c0 + rng.uniform(0.04, 0.05, (n_ngb, 1)) * dirs(n_ngb, -1.0, -0.1)
    ahead = c0 + rng.uniform(0.09, 0.2, (14, 1)) * dirs(14, 0.8, 1.0)
    side = c0 + rng.uniform(0.08, 0.15, (10, 1)) * dirs(10, -0.6, 0.6)
    pos = np.concatenate([[c0], behind, ahead, side]) * L
    n = len(pos)
    wl = W.tiny(n=n, seed=seed, n_ngb=n_ngb, L=L, n_tc=8)
    nH = 1e-3
    wl.update(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
              n_H=np.full(n, nH), N_H=np.full(n, nH * (0.05 * L) ** 3), x_HI=np.full(n, 0.08),
              T=np.full(n, 1e4), src_box=np.zeros(0, np.int32), src_x=np.zeros(0),
              src_y=np.zeros(0), src_z=np.zeros(0), src_ndot=np.zeros(0))
    wl["params"]["dt"] = wl["params"]["dt_em"] = 1.0   # 1 s: every packet stops at the first gas
    s = oracle.Sim(wl)
    s.build_neighbours()
    q = s.quantised().astype(np.float64)
    nbr = s.neighbours()[0][0]
    assert set(nbr) == set(range(1, n_ngb + 1))
    assert all((q[j] - q[0]) @ d < 0 for j in nbr)     # the sender's cone is empty
    s.rotate(0)
    s.emit(0)
    N0 = 1e50
    _put_packet(s, 0, N0, d)
    assert s.transport(0) == 0
    st = s.stats()
    assert st["virtual"] >= 1 and st["escaped_virtual"] == 0
    f = s.slots()
    Nj = f[0].sum(1)
    recv = np.nonzero(Nj)[0]
    assert len(recv) >= 1 and 0 not in recv
    u = L / (1 << 20)
    lj = ((q[recv] - q[0]) @ d) * u
    assert np.all(lj > 0)
    tau = wl["sigma"][0] * 0.08 * nH * lj
    share = Nj[recv] * np.exp(tau)
    assert np.allclose(share, N0 / len(recv), rtol=1e-12)
    assert np.allclose(f[4][recv].sum(1) / Nj[recv], lj / 2.99792458e10, rtol=1e-12)
    assert np.allclose(f[1:4][:, recv].sum(2), np.outer(d, Nj[recv]), rtol=1e-12, atol=0)
    e, ab, esc, fl = s.budget()[0]
    assert esc == 0.0 and abs(ab + Nj.sum() - N0) <= 1e-12 * N0
    assert abs(s.deposits()[0][:, 0].sum() - ab) <= 1e-12 * N0
    return len(recv)


def test_virtual_particle_hop_in_a_uniform_medium_is_independent_of_its_position():
    """A packet whose transmission cone holds no neighbour is handed to a virtual particle
    (Sec. 2.1), drawn at random in the cone.  In a medium of uniform n_HI and V = N_H/n_H
    the outcome at every receiver depends on where that point landed only through the
    number k of receivers:
    - the SPH estimate at the point is exactly the uniform n_HI (the weights are normalised);
    - the projected lengths of the hops add up, so the optical depth and the clock at
      receiver j are those of the straight projected path (q_j - q_sender) . d;
    - the last virtual particle splits what is left equally among its cone members.
    So N_j exp(tau_j) is the same for every receiver, these sum to the N sent, and every
    receiver's clock is (q_j - q_sender) . d u / c."""
    counts = [_virtual_hop_receivers(seed) for seed in range(21, 29)]
    assert sum(c >= 2 for c in counts) >= 3, counts   # the split is exercised


@pytest.mark.parametrize("n_tc", [8, 32])
def test_virtual_particle_lands_uniformly_in_the_cone_part_of_the_smoothing_sphere(n_tc):
    """The point of a virtual particle (Sec. 2.1, reading: uniform over the part of the sender's
    smoothing sphere inside the transmission cone).  Uniform in that solid cone means three
    independent uniform variables: (r/h)^3 on [0, 1], cos(angle to the axis) on [1 - 2/N_TC, 1]
    and the azimuth about the axis on [0, 2 pi).  A point that no draw finds sits on the axis
    at h/2; that happens with probability (1 - p)^64, p the accepted fraction of the cube."""
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(9)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    H = 1000
    h2 = H * H
    m = 20000
    pts = np.array([oracle.virtual_offset(77, 5, 3, 1 + f, h2, d, n_tc) for f in range(m)])
    fallback = np.rint(d * (0.5 * H)).astype(np.int64)
    on_axis = np.all(pts == fallback, axis=1)
    p = (4 / 3 * math.pi / n_tc) / 8.0
    q = (1 - p) ** 64
    assert abs(on_axis.mean() - q) < 5 * math.sqrt(q * (1 - q) / m) + 2e-4
    x = pts[~on_axis].astype(np.float64)
    r = np.linalg.norm(x, axis=1)
    assert np.all((r > 0) & (r * r <= h2))
    c = x @ d / r
    cmin = 1 - 2 / n_tc
    assert np.all(c >= cmin - 1e-12)
    e1 = np.cross(d, [1.0, 0.0, 0.0] if abs(d[0]) < 0.9 else [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    phi = np.arctan2(x @ e2, x @ e1) % (2 * math.pi)
    for sample, cdf in (((r / H) ** 3, stats.uniform(0, 1).cdf),
                        (c, stats.uniform(cmin, 1 - cmin).cdf),
                        (phi, stats.uniform(0, 2 * math.pi).cdf)):
        assert stats.kstest(sample, cdf).pvalue > 1e-3
    # the draws depend on every counter field
    base = oracle.virtual_offset(77, 5, 3, 1, h2, d, n_tc)
    for args in ((78, 5, 3, 1), (77, 6, 3, 1), (77, 5, 4, 1), (77, 5, 3, 1 + (1 << 32))):
        assert not np.array_equal(oracle.virtual_offset(*args, h2, d, n_tc), base)


def _m4(x):
    """M4 cubic spline of support 1 without its normalisation (Monaghan & Lattanzio 1985)."""
    return np.where(x <= 0.5, 1 - 6 * x ** 2 + 6 * x ** 3, np.where(x <= 1, 2 * (1 - x) ** 3, 0.0))


def _virtual_chain_against_brute_force(seed, near):
    """One packet into an empty cone; returns the number of virtual particles it made."""
    rng = np.random.default_rng(seed)
    L = 1.0 * KPC
    c0 = np.full(3, 0.5)
    d = np.array([1.0, 0.0, 0.0])

    def dirs(m, lo, hi):
        ct = rng.uniform(lo, hi, m)
        ph = rng.uniform(0.0, 2 * np.pi, m)
        st = np.sqrt(1 - ct ** 2)
        return np.stack([ct, st * np.cos(ph), st * np.sin(ph)], 1)

    # the sender's k neighbours all lie behind it; a group just beyond its smoothing radius,
    # near the axis, puts gas close to where the virtual particle lands (small r / h_v);
    # without it the first virtual particle's cone is often empty too (a chain)
    k = 16
    groups = [[c0], c0 + rng.uniform(0.04, 0.05, (k, 1)) * dirs(k, -1.0, -0.1)]
    if near:
        groups.append(c0 + rng.uniform(0.051, 0.065, (8, 1)) * dirs(8, 0.8, 1.0))
    groups += [c0 + rng.uniform(0.07, 0.2, (16, 1)) * dirs(16, 0.5, 1.0),
               c0 + rng.uniform(0.08, 0.15, (10, 1)) * dirs(10, -0.6, 0.6)]
    pos = np.concatenate(groups) * L
    n = len(pos)
    wl = W.tiny(n=n, seed=seed, n_ngb=k, L=L, n_tc=8)
    nH = np.exp(rng.normal(math.log(1e-3), 0.7, n))
    wl.update(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(), n_H=nH,
              N_H=nH * (0.05 * L) ** 3 * rng.uniform(0.5, 2.0, n), x_HI=rng.uniform(0.01, 0.2, n),
              T=np.full(n, 1e4), src_box=np.zeros(0, np.int32), src_x=np.zeros(0),
              src_y=np.zeros(0), src_z=np.zeros(0), src_ndot=np.zeros(0))
    wl["params"]["dt"] = wl["params"]["dt_em"] = 1.0
    s = oracle.Sim(wl)
    s.build_neighbours()
    qi = s.quantised()
    q = qi.astype(np.float64)
    nbr, h2s = s.neighbours()[:2]
    assert all((q[j] - q[0]) @ d < 0 for j in nbr[0])
    s.rotate(0)
    s.emit(0)
    N0 = 1e50
    _put_packet(s, 0, N0, d)
    b0 = int(np.nonzero(s.slots()[0][0])[0][0])
    assert s.transport(0) == 0

    u = L / (1 << 20)
    sigma = wl["sigma"][0]
    nHI = wl["x_HI"] * nH
    V = wl["N_H"] / nH
    cmin = 1.0 - 2.0 / 8
    idx = np.arange(n)
    dep = np.zeros(n)
    arrived = np.zeros(n)
    fid, hop, qs, h2, N = b0 + 1, 0, qi[0], int(h2s[0]), N0
    escaped = 0.0
    for _ in range(8):
        qv = qs + oracle.virtual_offset(wl["params"]["seed"], 0, hop, fid, h2, d, 8)
        if not np.all((qv >= 0) & (qv < (1 << 20))):
            escaped = N                 # a point outside the box: the photons leave it
            break
        d2 = ((qi - qv) ** 2).sum(1)
        near = np.lexsort((idx, d2))[:k]
        h2v = int(d2[near[-1]])
        om = V[near] * _m4(np.sqrt(d2[near] / h2v))
        l = ((qv - qs) @ d) * u
        A = N * -math.expm1(-sigma * (om @ nHI[near] / om.sum()) * l)
        dep[near] += A * om * nHI[near] / (om @ nHI[near])
        N -= A
        rel = q[near] - qv
        cosang = rel @ d / np.maximum(np.linalg.norm(rel, axis=1), 1e-300)
        assert np.all(np.abs(cosang - cmin) > 1e-9)
        members = near[cosang > cmin]
        if len(members):
            for j in members:
                lj = ((q[j] - qv) @ d) * u
                a = (N / len(members)) * -math.expm1(-sigma * nHI[j] * lj)
                dep[j] += a
                arrived[j] += N / len(members) - a
            break
        qs, h2, hop, fid = qv, h2v, hop + 1, oracle.mix64(fid)
    else:
        raise AssertionError("virtual chain longer than 8 hops")
    assert s.stats()["virtual"] == hop + 1
    got = s.deposits()[0][:, 0]
    assert np.allclose(got, dep, rtol=1e-11, atol=1e-13 * N0)
    assert np.allclose(s.slots()[0].sum(1), arrived, rtol=1e-11, atol=1e-13 * N0)
    assert abs(s.budget()[0][2] - escaped) <= 1e-12 * N0
    return hop + 1


def test_virtual_particle_shares_absorptions_by_sph_weight_and_neutral_density():
    """Brute force of a virtual-particle chain in a non-uniform medium (Sec. 2.1, reading 11):
    the point comes from the pinned placement draw; its neighbours are the n_ngb nearest gas
    particles (ties to the lower index); n_HI there is the Shepard-normalised SPH estimate with
    weights V_k W(r_k / h_v), V = N_H / n_H; the photons absorbed on the projected way to it are
    shared in proportion to V_k W_k n_HI,k; what is left goes to its cone members in equal
    shares (or to the next virtual particle, one hop later, with the mixed packet identity)."""
    chains = [_virtual_chain_against_brute_force(seed, near)
              for seed, near in zip(range(31, 39), [True] * 4 + [False] * 4)]
    assert max(chains) >= 2, chains     # a chain of virtual particles is exercised


@pytest.mark.parametrize("n_rc,shared", [(8, 0), (32, 0), (8, 1)])
def test_rebin_moves_each_held_packet_to_the_new_cone_of_its_direction(n_rc, shared):
    """At the start of a step the reception cones are rotated anew (Sec. 2.1) and every packet a
    particle holds moves, with its photons, momentum and energy, into the cone of the new set
    nearest its direction; packets landing in one cone merge, and every clock restarts.  In a
    shared bin the photon-weighted cross-section sum travels with its packet.  Brute force on
    random packets, the new cone taken as argmax over the rotated axes."""
    rng = np.random.default_rng(40 + n_rc + shared)
    wl = W.tiny(n=60, n_ngb=8, n_rc=n_rc, rec_shared_bin=shared)
    s = oracle.Sim(wl)
    s.build_neighbours()
    s.rotate(0)
    f = np.zeros((6, s.n, s.S))
    occ = rng.random((s.n, s.S)) < 0.3
    N = rng.uniform(1e40, 1e42, (s.n, s.S)) * occ
    d = rng.normal(size=(s.n, s.S, 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    f[0] = N
    f[1:4] = np.moveaxis(N[..., None] * d * rng.uniform(0.3, 1.0, (s.n, s.S, 1)), 2, 0)
    f[4] = N * rng.uniform(0.0, 1e13, (s.n, s.S))
    f[5] = N * rng.uniform(1.0, 5.0, (s.n, s.S)) * EV
    s.set_slots(f)
    G = None
    if shared:
        G = N[:, :n_rc] * rng.uniform(1e-18, 6e-18, (s.n, n_rc))
        s.set_shared_sigma(G)
    s.rotate(1)
    s.rebin()
    A = oracle.axis_set(n_rc)
    R = s.rotations()[0]
    want = np.zeros_like(f)
    wantG = np.zeros((s.n, n_rc))
    for i in range(s.n):
        Ri = R[i].reshape(3, 3)
        for sl in np.nonzero(occ[i])[0]:
            nu = sl // n_rc
            b = int(np.argmax((Ri @ A.T).T @ f[1:4, i, sl]))
            want[[0, 1, 2, 3, 5], i, nu * n_rc + b] += f[[0, 1, 2, 3, 5], i, sl]
            if shared and nu == 0:
                wantG[i, b] += G[i, sl]
    got = s.slots()
    for k in range(6):
        assert np.allclose(got[k], want[k], rtol=1e-13, atol=1e-13 * np.abs(want[k]).max())
    assert np.all(got[4] == 0.0)
    if shared:
        assert np.allclose(s.shared_sigma(), wantG, rtol=1e-13, atol=0)


@pytest.mark.parametrize("n_ec,k_em", [(8, 1), (32, 2), (8, 4)])
def test_source_emission_is_complete_and_isotropic(n_ec, k_em):
    """A source emits ndot dt photons per step (Sec. 2.1): K = dt / dt_em emissions, each split
    equally over N_EC packets along its emission axes, rotated at random before each emission.
    The axes of each emission sum to zero, so in an optically thin box, with every packet
    stopping at the first gas it reaches, the photons held afterwards total ndot dt and their
    momenta cancel."""
    wl = W.cfg1(n_side=12)
    n = len(wl["x"])
    dt = 1.0
    wl.update(x_HI=np.zeros(n))
    wl["params"].update(n_ec=n_ec, dt=dt, dt_em=dt / k_em)
    s = oracle.Sim(wl)
    s.build_neighbours()
    s.rotate(0)
    s.rebin()
    s.emit(0)
    ndot_dt = wl["src_ndot"].sum() * dt
    assert abs(s.budget()[0][0] - ndot_dt) <= 1e-14 * ndot_dt
    assert s.transport(0) == 0
    e, ab, esc, fl = s.budget()[0]
    assert ab == 0.0 and esc == 0.0
    f = s.slots()
    N = f[0].sum()
    assert abs(N - ndot_dt) <= 1e-13 * ndot_dt
    assert np.linalg.norm(f[1:4].sum(axis=(1, 2))) <= 1e-12 * ndot_dt
    Rs = s.rotations()[1]
    assert len(Rs) == k_em
    if k_em > 1:
        assert not np.allclose(Rs[0], Rs[1])     # a fresh rotation before each emission


def test_cost_does_not_grow_with_the_number_of_sources():
    """Packets merge per reception cone at every particle, so the work of a step is bounded by
    the particles and their cones, not by the sources (Sec. 2.1): in each hop at most
    n S gas slots send, plus each free packet (a source's first-hop packets and the virtual
    particles) once.  The same luminosity split over 64 sources clustered where one source
    sat costs well under twice as many sends, where a method tracing rays per source would
    cost about 64 times as many."""
    base = W.cfg1(n_side=16)
    L = base["box_L"][0]
    tot = base["src_ndot"].sum()
    rng = np.random.default_rng(1)
    p = base["params"]
    sends = {}
    for ns in (1, 64):
        pos = np.array([[0.5, 0.5, 0.5]]) * L if ns == 1 else (0.5 + rng.uniform(-0.02, 0.02, (ns, 3))) * L
        wl = dict(base, src_box=np.zeros(ns, np.int32), src_x=pos[:, 0].copy(),
                  src_y=pos[:, 1].copy(), src_z=pos[:, 2].copy(), src_ndot=np.full(ns, tot / ns))
        s = oracle.Sim(wl)
        s.build_neighbours()
        sends[ns] = 0
        for step in range(4):
            s.step(step)
            st = s.stats()
            bound = st["hops"] * s.n * s.S + ns * p["n_ec"] * p["n_freq_src"] + st["virtual"]
            assert 0 < st["sends"] <= bound
            sends[ns] += st["sends"]
        e, ab, esc, fl = s.budget()[0]
        assert abs(e - ab - esc - fl) <= 1e-12 * e
    assert sends[64] < 2 * sends[1], sends


def _front_radius(s, wl):
    L = wl["box_L"][0]
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    r = np.linalg.norm(pos - 0.5 * L, axis=1)
    x = s.state()["x_HI"]
    edges = np.linspace(0, 0.5 * L, 17)
    prof = [x[(r >= a) & (r < b)].mean() for a, b in zip(edges[:-1], edges[1:])]
    mid = 0.5 * (edges[:-1] + edges[1:])
    for k in range(1, len(prof)):
        if prof[k - 1] < 0.5 <= prof[k]:
            t = (0.5 - prof[k - 1]) / (prof[k] - prof[k - 1])
            return mid[k - 1] + t * (mid[k] - mid[k - 1]), np.array(prof), mid
    return np.nan, np.array(prof), mid


@pytest.mark.slow
def test_stromgren_sphere_and_case_a_b_limits():
    """Sec. 3 (Iliev Test 1 geometry): on-the-spot case B grows to the case-B Stromgren radius;
    with transport of recombination radiation the front lies between the case-A and case-B
    fronts and the inner neutral fraction is near the case-A value (Fig. 1 discussion)."""
    steps = 120   # 300 Myr ~ 2.5 t_rec
    res = {}
    for mode in (W.REC_OTS_CASE_B, W.REC_CASE_A, W.REC_TRANSPORT):
        wl = W.cfg1(rec_mode=mode)
        s = _run(wl, steps)
        rI, prof, mid = _front_radius(s, wl)
        res[mode] = (rI, prof)
        e, a, esc, fl = s.budget()[0]
        assert abs(e - a - esc - fl) <= 1e-12 * e
    aB = oracle.rates(1e4)["alpha_B"]
    R_S = (3 * 5e48 / (4 * math.pi * aB * 1e-6)) ** (1 / 3)
    t = steps * 2.5 * MYR
    r_expect = R_S * (1 - math.exp(-t * aB * 1e-3)) ** (1 / 3)
    h_mean = 13.2 * KPC / 16 * (32 * 3 / (4 * math.pi)) ** (1 / 3)
    rB, rA, rRT = res[W.REC_OTS_CASE_B][0], res[W.REC_CASE_A][0], res[W.REC_TRANSPORT][0]
    assert abs(rB - r_expect) < h_mean
    assert rA < rB - 0.25 * h_mean                # case A: smaller front (Sec. 3)
    assert abs(rRT - rB) < 0.25 * h_mean          # RT approaches case B at the front (Sec. 3)
    # near the source (r < 0.23 R_S): RT close to case A, case B lower by alpha_B/alpha_A ~ 0.6
    inner = slice(0, 3)
    pB, pA, pRT = (res[m][1][inner] for m in (W.REC_OTS_CASE_B, W.REC_CASE_A, W.REC_TRANSPORT))
    assert np.all(np.abs(pRT / pA - 1) < 0.15)
    r = oracle.rates(1e4)
    assert np.all(np.abs(pB / pA / (r["alpha_B"] / r["alpha_A"]) - 1) < 0.03)


def _shell_gamma_over_exact(n_side, x_val, reps=4):
    """Per radial shell around the source (shells of L/16 from 1.5/16 L out to 7.5/16 L), the
    photoionisation rate per neutral atom of one transport over uniform gas of neutral fraction
    x_val, averaged over `reps` steps' random rotations, over the exact rate of the attenuated
    point source, sigma Ndot exp(-sigma n_H x r) / (4 pi r^2)."""
    G = None
    for rep in range(reps):
        wl = W.cfg1(n_side=n_side, rec_mode=W.REC_OTS_CASE_B)
        wl["x_HI"][:] = x_val
        s = oracle.Sim(wl)
        s.build_neighbours()
        s.rotate(rep)
        s.rebin()
        s.emit(rep)
        assert s.transport(rep) == 0
        a, _, _ = s.deposits()
        g = a.sum(1) / (x_val * wl["N_H"] * wl["params"]["dt"])
        G = g if G is None else G + g
    G /= reps
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    r = np.linalg.norm(pos - np.array([wl["src_x"][0], wl["src_y"][0], wl["src_z"][0]]), axis=1)
    exact = 6.3e-18 * 5e48 * np.exp(-6.3e-18 * 1e-3 * x_val * r) / (4 * math.pi * r * r)
    L = float(wl["box_L"][0])
    out = []
    for k in range(2, 8):
        m = (r >= (k - 0.5) / 16 * L) & (r < (k + 0.5) / 16 * L)
        out.append(G[m].mean() / exact[m].mean())
    return np.array(out)


def test_interior_field_is_the_attenuated_point_source_field():
    """Sec. 2.1 transport in 3D: over uniform partly neutral gas the photoionisation rate of each
    radial shell follows the attenuated point-source field sigma Ndot e^-tau / (4 pi r^2) (the
    1/r^2 dilution and the Beer-Lambert attenuation through the shells inside), beyond the
    source's own smoothing scale: within 5% where the optical depth per particle spacing is
    0.01 and 15% where it is 0.1 (24^3 particles, the HII region's box and source).  A
    transport that kept the front but bent the interior field fails this."""
    thin = _shell_gamma_over_exact(24, 1e-3)
    assert np.all(np.abs(thin - 1) < 0.05), thin
    mid = _shell_gamma_over_exact(24, 1e-2)
    assert np.all(np.abs(mid - 1) < 0.15), mid


def test_absorbed_photons_ionise_at_first_order_in_the_time_step():
    """Sec. 2.1 chemistry: the step's absorptions give the photoionisation rate per neutral atom
    at the start of the step, which the subcycles apply to the evolving neutral fraction, so
    ionisations plus recombinations fall short of the absorbed photons where the gas ionises
    within the step.  The shortfall vanishes at first order as the step shrinks towards the
    0.1 Myr of Sec. 3 (App. A: converged at that step): during the expansion of the HII region
    (case B on the spot, 25-50 Myr) it falls at least 2.5-fold per 5-fold shorter step and is
    below 4% at 0.1 Myr."""
    aB = oracle.rates(1e4)["alpha_B"]
    deficit = []
    for dt in (2.5, 0.5, 0.1):
        wl = W.cfg1(rec_mode=W.REC_OTS_CASE_B, dt=dt * MYR, dt_em=dt * MYR)
        s = oracle.Sim(wl)
        s.build_neighbours()
        V = wl["N_H"] / wl["n_H"]
        steps = int(round(50 / dt))
        use = []
        for k in range(steps):
            x0, b0 = s.state()["x_HI"].copy(), s.budget()[0].copy()
            assert s.step(k) == 0
            x1, b1 = s.state()["x_HI"], s.budget()[0]
            if k >= steps // 2:
                xm = 0.5 * (x0 + x1)
                rec = np.sum(aB * wl["n_H"] ** 2 * (1 - xm) ** 2 * V) * dt * MYR
                use.append((rec + np.sum((x0 - x1) * wl["N_H"])) / (b1[1] - b0[1]))
        deficit.append(1.0 - np.mean(use))
    d25, d05, d01 = deficit
    assert d25 > d05 > d01 > 0
    assert d05 < d25 / 2.5 and d01 < d05 / 2.5
    assert d01 < 0.04


def test_original_emission_cone_recombination_conserves_photons():
    """The original implementation (Sec. 2.2): every recombining particle emits N_EC separate
    packets of its own, which leave through its neighbours; photons are still conserved."""
    wl = W.cfg1(rec_mode=W.REC_EMISSION_CONES)
    wl["x_HI"][:] = 0.05            # recombining gas from the first step on
    s = _run(wl, 4)
    e, a, esc, fl = s.budget()[0]
    assert s.stats()["virtual"] > 0
    assert abs(e - a - esc - fl) <= 1e-12 * e
    # the recombination photons are emitted: more photons than the source alone
    src = 5e48 * 4 * 2.5 * MYR
    assert e > 1.05 * src


def test_original_and_new_recombination_implementations_agree():
    """Sec. 2.2: the new implementation (recombination photons merged into the reception
    cones) and the original one (separate packets in per-particle emission cones) give nearly
    identical results.  After 20 steps of the Stromgren workload the radial median of x_HI of
    the two agrees to 3 % in every shell, while case A differs by more than 10 % somewhere."""
    res = {}
    for mode in (W.REC_TRANSPORT, W.REC_EMISSION_CONES, W.REC_CASE_A):
        wl = W.cfg1(rec_mode=mode)
        res[mode] = _run(wl, 20).state()["x_HI"]
    wl = W.cfg1()
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    r = np.linalg.norm(pos - 0.5 * wl["box_L"][0], axis=1) / KPC
    shells = [(0, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
    med = {m: np.array([np.median(x[(r >= a) & (r < b)]) for a, b in shells]) for m, x in res.items()}
    assert np.all(np.abs(med[W.REC_EMISSION_CONES] / med[W.REC_TRANSPORT] - 1) < 0.03)
    assert np.max(np.abs(med[W.REC_CASE_A] / med[W.REC_TRANSPORT] - 1)) > 0.10


def test_barrier_test_is_exact_against_rational_arithmetic():
    """The barrier disk test (Sec. 4) against exact rational arithmetic on random segments,
    including long ones and ones that graze the rim."""
    from fractions import Fraction
    rng = np.random.default_rng(3)
    Q = 1 << 20
    n_hit = 0
    for trial in range(3000):
        axis = int(rng.integers(3))
        p2 = 2 * int(rng.integers(Q)) + 1
        c1, c2 = 2 * int(rng.integers(Q)), 2 * int(rng.integers(Q))
        r2 = int(rng.integers(1, 1 << 21))
        a = rng.integers(0, Q, 3)
        b = rng.integers(0, Q, 3) if trial % 3 else a + rng.integers(-40, 41, 3)
        if trial % 5 == 0:           # put the ends on both sides of the plane, near the rim
            a[axis], b[axis] = (p2 - 1) // 2, (p2 + 1) // 2
            a[(axis + 1) % 3] = (c1 + r2) // 2
        i1, i2 = (axis + 1) % 3, (axis + 2) % 3
        sa, sb = 2 * int(a[axis]) - p2, 2 * int(b[axis]) - p2
        want = False
        if (sa < 0) != (sb < 0):
            t = Fraction(sa, sa - sb)
            y = 2 * int(a[i1]) + t * 2 * (int(b[i1]) - int(a[i1])) - c1
            z = 2 * int(a[i2]) + t * 2 * (int(b[i2]) - int(a[i2])) - c2
            want = y * y + z * z <= r2 * r2
        n_hit += want
        assert oracle.barrier_test(a, b, axis, p2, c1, c2, r2) == want, (a, b, axis)
    assert n_hit > 30


def test_plane_parallel_front_advances_at_F_over_nH():
    """The directed emitters of the plane-parallel front (Sec. 4): before recombinations
    matter (t << t_rec) every photon ionises one atom, so the front of an initially neutral
    slab of density n_H stands at x = F t / n_H.  With steps short enough for the front to
    cross less than a particle spacing per step, the front lies within one spacing of it."""
    wl = W.shadow(n_side=16, n_front=20, n_bnd=10, barrier=False, boundary=False,
                  rec_mode=W.REC_OTS_CASE_B, dt=0.01 * MYR, dt_em=0.01 * MYR)
    s = _run(wl, 40)
    e, a, esc, fl = s.budget()[0]
    assert abs(e - a - esc - fl) <= 1e-12 * e
    L = wl["box_L"][0]
    x = s.state()["x_HI"]
    px = wl["x"] / L
    edges = np.linspace(0, 1, 17)
    prof = np.array([x[(px >= lo) & (px < hi)].mean() for lo, hi in zip(edges[:-1], edges[1:])])
    k = int(np.argmax((prof[:-1] < 0.5) & (prof[1:] >= 0.5)))
    mid = 0.5 * (edges[:-1] + edges[1:]) * L
    xf = mid[k] + (0.5 - prof[k]) / (prof[k + 1] - prof[k]) * (mid[k + 1] - mid[k])
    expect = 1e6 * 40 * 0.01 * MYR / 1e-3
    assert abs(xf - expect) < L / 16


def _shadow_regions(wl):
    L = wl["box_L"][0]
    p = np.stack([wl["x"], wl["y"], wl["z"]], 1) / L
    r = np.hypot(p[:, 1] - 0.5, p[:, 2] - 0.5)
    behind = (p[:, 0] > 0.40) & (p[:, 0] < 0.9)
    return behind & (r < 0.12), behind & (r > 0.30)


@pytest.mark.slow
def test_barrier_shadow_is_ionised_and_heated_by_recombination_radiation():
    """Sec. 4: a disk barrier in a plane-parallel front casts a shadow.  On the spot (case B,
    no diffuse radiation) the shadow stays neutral and cold while the gas beside it is ionised
    and hot.  With recombination radiation transported, including the boundary emitters of
    App. B, the shadow becomes highly ionised, and is heated less than the directly lit gas
    (recombination photons carry less excess energy).  Photons are conserved with the barrier
    removing packets."""
    res = {}
    for name, kw in (("B", dict(rec_mode=W.REC_OTS_CASE_B, boundary=False)),
                     ("RT", dict(rec_mode=W.REC_TRANSPORT, boundary=True))):
        wl = W.shadow(n_side=16, n_front=20, n_bnd=10, **kw)
        s = _run(wl, 30)
        e, a, esc, fl = s.budget()[0]
        assert abs(e - a - esc - fl) <= 1e-12 * e
        st = s.state()
        sh, op = _shadow_regions(wl)
        res[name] = (np.median(st["x_HI"][sh]), np.median(st["x_HI"][op]),
                     np.median(st["T"][sh]), np.median(st["T"][op]))
    xs, xo, Ts, To = res["B"]
    assert xs > 0.9 and xo < 1e-3 and Ts < 1000 and To > 1.5e4
    xs, xo, Ts, To = res["RT"]
    assert xs < 1e-2 and xo < 1e-3
    assert 5e3 < Ts < 0.7 * To


# --- shared frequency bin (Sec. 2.2, last paragraph) -----------------------------------------
def _shared_chain(**kw):
    wl = _chain(**kw)
    wl["params"]["rec_shared_bin"] = 1
    return wl


def test_shared_bin_mixed_packet_follows_beer_lambert_with_its_mean_cross_section():
    """A packet of the shared bin holding photons of two cross-sections is attenuated with the
    photon-weighted mean N_abs = N (1 - exp(-sigma_mean n_HI l)) on every hop, and keeps that
    mean as it moves on: along the chain the photon count falls as exp(-sigma_mean sum n l).
    The bin's own cross-section, or a mean lost after the first hop, fails."""
    wl = _shared_chain()
    s = oracle.Sim(wl)
    assert s.nf == 1 and s.S == s.params["n_rc"]       # no bin of their own
    s.build_neighbours()
    s.rotate(0)
    s.emit(0)
    N0, sig0 = 1e50, wl["sigma"][0]
    Na, Nb, sb = 0.25 * N0, 0.75 * N0, 2.0 * sig0
    _put_packet(s, 1, N0, [1.0, 0.0, 0.0])
    G = np.zeros((s.n, s.params["n_rc"]))
    b = int(np.nonzero(s.slots()[0][1])[0][0])
    G[1, b] = Na * sig0 + Nb * sb
    s.set_shared_sigma(G)
    assert s.transport(0) == 0
    a = s.deposits()[0][:, 0]
    sig_mean = (Na * sig0 + Nb * sb) / N0                 # 1.75 sigma_0
    q = s.quantised()
    u = wl["box_L"][0] / (1 << 20)
    l = np.diff(q[1:, 0]) * u
    tau = sig_mean * wl["x_HI"][2:] * wl["n_H"][2:] * l
    N = N0 * np.exp(-np.concatenate([[0.0], np.cumsum(tau)]))
    assert np.allclose(a[2:-2], N[:-3] - N[1:-2], rtol=1e-12, atol=0)
    tau0 = sig0 * wl["x_HI"][2:] * wl["n_H"][2:] * l       # with the bin's own sigma: far off
    N_wrong = N0 * np.exp(-np.concatenate([[0.0], np.cumsum(tau0)]))
    assert not np.allclose(a[2:-2], N_wrong[:-3] - N_wrong[1:-2], rtol=1e-3)
    e, ab, esc, fl = s.budget()[0]
    assert abs(ab + esc - N0) <= 1e-12 * N0


def test_shared_bin_recombination_photons_merge_into_bin_0_with_their_cross_section():
    """With a shared bin the recombination photons of a particle go into its reception cones of
    source bin 0: per particle the bin gains N_rec photons and N_rec sigma_rec of cross-section
    sum, on top of the packet already there (photon-weighted merge)."""
    wl = W.cfg2(n_side=8, rec_shared_bin=1, ionised=False)
    s = oracle.Sim(wl)
    s.build_neighbours()
    nrc = s.params["n_rc"]
    assert s.nf == wl["params"]["n_freq_src"] and s.S == s.nf * nrc
    n = s.n
    nrec = np.zeros(n)
    nrec[[5, 77, 300]] = [1e55, 3e54, 7e53]
    s.set_state(N_rec=nrec, eps_rec=np.full(n, 2 * EV))
    s.rotate(3)
    _put_packet(s, 77, 2e54, [0.0, 1.0, 0.0])          # a stellar packet already in bin 0
    b77 = int(np.nonzero(s.slots()[0][77])[0][0])
    assert b77 < nrc
    G = np.zeros((n, nrc))
    G[77, b77] = 2e54 * wl["sigma"][0]
    s.set_shared_sigma(G)
    s.emit(3)
    f, G = s.slots(), s.shared_sigma()
    sr, s0 = wl["params"]["sigma_rec"], wl["sigma"][0]
    for i, extra in ((5, 0.0), (77, 2e54), (300, 0.0)):
        assert np.allclose(f[0][i, :nrc].sum(), nrec[i] + extra, rtol=1e-14)
        assert np.all(f[0][i, nrc:] == 0.0)             # the other source bins stay empty
        assert np.allclose(G[i].sum(), nrec[i] * sr + extra * s0, rtol=1e-14)
    # the cone holding the stellar packet: the photon-weighted mean of the two cross-sections
    e = nrec[77] / nrc
    assert np.isclose(G[77, b77] / f[0][77, b77], (2e54 * s0 + e * sr) / (2e54 + e), rtol=1e-14)


def test_shared_bin_conserves_photons_and_keeps_means_between_the_inputs():
    """Clock-limited steps (c dt < box side) leave packets held at the step end: photons are
    conserved to 1e-12 and every held packet of the shared bin has a mean cross-section between
    the bin's own and the recombination photons', some strictly between (merged)."""
    wl = W.cfg2(n_side=12, rec_shared_bin=1, dt=0.01 * MYR, dt_em=0.01 * MYR)
    s = _run(wl, 6)
    e, a, esc, fl = s.budget()[0]
    assert fl > 0.01 * e
    assert abs(e - a - esc - fl) <= 1e-12 * e
    nrc = s.params["n_rc"]
    N, G = s.slots()[0][:, :nrc], s.shared_sigma()
    m = N > 0
    sig = G[m] / N[m]
    lo, hi = sorted([wl["sigma"][0], wl["params"]["sigma_rec"]])
    assert np.all(sig >= lo * (1 - 1e-13)) and np.all(sig <= hi * (1 + 1e-13))
    assert np.any((sig > lo * 1.01) & (sig < hi * 0.99))
    assert np.all(G[~m] == 0.0)


def test_shared_and_separate_bins_agree_when_the_spectra_match():
    """Sec. 2.2: one bin for stellar and recombination photons is appropriate when the two
    spectra in it are alike.  In the Stromgren workload (13.6 eV source, sigma equal to the
    recombination photons') the shared and the separate bin give radial medians of x_HI within
    3 % of each other after 20 steps, while case A differs by more than 10 % somewhere."""
    res = {}
    for name, kw in (("sep", {}), ("shared", dict(rec_shared_bin=1)),
                     ("A", dict(rec_mode=W.REC_CASE_A))):
        res[name] = _run(W.cfg1(**kw), 20).state()["x_HI"]
    wl = W.cfg1()
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    r = np.linalg.norm(pos - 0.5 * wl["box_L"][0], axis=1) / KPC
    shells = [(0, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
    med = {m: np.array([np.median(x[(r >= a) & (r < b)]) for a, b in shells]) for m, x in res.items()}
    assert np.all(np.abs(med["shared"] / med["sep"] - 1) < 0.03)
    assert np.max(np.abs(med["A"] / med["sep"] - 1)) > 0.10


def test_chemistry_converges_to_its_rate_equations():
    """Sec. 2.1 chemistry: with the step cut into many short calls at a fixed photoionisation and
    photoheating rate per neutral atom, the oracle's update (electron density frozen within a
    subcycle, exact exponential for x_HI, explicit step for u) converges at first order to a
    stiff integration (scipy Radau) of the rate equations
        dx/dt = alpha_A n_e (1 - x) - (Gamma + beta n_e) x,
        du/dt = x n_H H - n_e n_HII L_rec,A - n_e n_HI L_cex,   u = 1.5 k T n_H (1 + x_HII),
    and its recombination photons to the integral of (alpha_A - alpha_B) n_e n_HII V.  A neutral
    cold particle is ionised and heated through the step.  A dropped term, a wrong sign, a case-B
    coefficient or a wrong normalisation converges elsewhere and fails."""
    from scipy.integrate import solve_ivp
    nH, L = 1e-3, 0.2 * KPC
    NH = nH * L ** 3
    x0, T0 = 0.9, 100.0
    Gam = 2e-12
    H = Gam * 3.0 * EV
    dt = 0.5 * MYR

    def rhs(t, y):
        x, u, _ = y
        xII = 1.0 - x
        r = oracle.rates(u / (1.5 * K_B * nH * (1.0 + xII)))
        ne = xII * nH
        return [r["alpha_A"] * ne * xII - (Gam + r["beta"] * ne) * x,
                x * nH * H - ne * xII * nH * r["Lrec_A"] - ne * x * nH * r["L_cex"],
                (r["alpha_A"] - r["alpha_B"]) * ne * xII * NH]

    u0 = 1.5 * K_B * T0 * nH * (2.0 - x0)
    sol = solve_ivp(rhs, (0.0, dt), [x0, u0, 0.0], method="Radau", rtol=1e-10,
                    atol=[1e-14, 1e-12 * u0, 1.0])
    xr, ur, nr_ref = sol.y[:, -1]
    Tr = ur / (1.5 * K_B * nH * (2.0 - xr))
    assert xr < 1e-3 and Tr > 5e3                     # ionised and heated within the step
    errs = []
    for n_calls in (1000, 4000):
        p = _params(dt=dt / n_calls, evolve_T=1, rec_mode=W.REC_TRANSPORT, sub_cap=100000)
        x, T, nrec = x0, T0, 0.0
        for _ in range(n_calls):
            h = dt / n_calls
            x, T, n, _, _ = oracle.chem_particle(p, nH, NH, Gam * x * NH * h, H * x * NH * h, x, T)
            nrec += n
        errs.append(max(abs(x / xr - 1), abs(T / Tr - 1), abs(nrec / nr_ref - 1)))
    assert errs[1] < 5e-3
    assert 2.5 < errs[0] / errs[1] < 6.0               # first order in the call length
