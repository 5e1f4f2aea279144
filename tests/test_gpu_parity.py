"""Parity of the CUDA library (through the C ABI) with the CPU oracle on identical seeded inputs.

Bars: integer and index work (quantised positions, neighbour lists, rotations, cone masks)
bit-exact; x_HI within 1e-3 relative (1e-7 absolute where x_HI < 1e-4), T within 1e-3
relative, photon budget within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1311_0182_gb300 import accuracy as ACC
from paper_1311_0182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_0182_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _pair(wl, **over):
    from paper_1311_0182_gb300 import rt
    if over:
        wl = dict(wl, params=dict(wl["params"], **over))
    g = rt.context_for(wl)
    o = oracle.Sim(wl)
    o.build_neighbours()
    return g, o


def _xhi_ok(xg, xo):
    rel = np.abs(xg - xo) / np.maximum(np.abs(xo), 1e-300)
    small = xo < 1e-4
    return np.where(small, np.abs(xg - xo) <= 1e-7, rel <= 1e-3)


# Routing flips of the FP32 transport, and the bars: paper_1311_0182_gb300/accuracy.py.  The FP32
# path takes every discrete decision exactly on its FP32 packet direction; a decision whose
# margin is below the FP32-FP64 direction difference goes the other way and that packet share
# takes another route.  Particles whose absorptions stay within ROUTE_TOL of the oracle's in every
# step are held to the bars; the others are counted against FLIP_BUDGET.


def _route_affected(g, o, NH, affected):
    """Mark the particles whose absorbed photons or energy of the last step differ from the
    oracle's by more than ROUTE_TOL (relative, plus the absolute floors)."""
    ag, eg, _ = g.deposits()
    ao, eo, _ = o.deposits()
    return ACC.mark_routing_affected(ag.sum(1), ao.sum(1), eg.sum(1),
                                     eo if eo.ndim == 1 else eo.sum(1), NH, affected)


def _assert_fp32_bars(sg, so, affected, steps, what=""):
    """Every particle not routing-affected within the x_HI and T bars; routing-affected
    particles within the flip budget of `steps` compared steps."""
    ok = ACC.state_ok(sg, so)
    bad = ~ok & ~affected
    n = len(ok)
    assert not bad.any(), (f"{what}: {bad.sum()} particles off the bars without a routing "
                           f"change (max x_HI rel {np.max(np.abs(sg['x_HI'] / so['x_HI'] - 1)[bad]):.2e})")
    assert affected.sum() <= ACC.flip_budget(n, steps), \
        f"{what}: {affected.sum()} of {n} routing-affected in {steps} steps"


def _clustered_boxes(n_boxes=5, seed=11):
    """Several independent boxes with clumps, duplicates and a near-minimal box."""
    rng = np.random.default_rng(seed)
    pos, nH, box_off, box_L = [], [], [0], []
    for b in range(n_boxes):
        L = (1 + b) * W.KPC
        n = 33 if b == 0 else int(rng.integers(300, 1500))
        c = rng.uniform(0.2, 0.8, size=(3, 3)) * L
        p = c[rng.integers(0, 3, n)] + rng.normal(0, 0.05 * L, size=(n, 3))
        p = np.clip(p, 0, np.nextafter(L, 0))
        if n > 40:
            p[10:20] = p[9]
        pos.append(p)
        nH.append(np.full(n, 1e-3))
        box_off.append(box_off[-1] + n)
        box_L.append(L)
    pos = np.concatenate(pos)
    n = len(pos)
    nHa = np.concatenate(nH)
    NH = np.concatenate([np.full(box_off[b + 1] - box_off[b], 1e-3 * box_L[b] ** 3 /
                                 (box_off[b + 1] - box_off[b])) for b in range(n_boxes)])
    params = W.default_params(seed=seed, dt=0.05 * W.MYR, dt_em=0.05 * W.MYR)
    src = np.array([[0.5 * L] * 3 for L in box_L])
    return W._pack(params, box_L, box_off, pos, nHa, NH, np.full(n, 0.3), np.full(n, 1e4),
                   np.arange(n_boxes), src, np.full((n_boxes, 1), 1e48), [6.3e-18], [0.0])


# --- integer work: bit-exact -------------------------------------------------------------------
@pytest.mark.parametrize("name", ["cfg1", "tiny", "clustered", "cfg2_small"])
def test_quantisation_and_neighbours_bit_exact(name):
    wl = {"cfg1": lambda: W.cfg1(), "tiny": lambda: W.tiny(n=300, n_ngb=16),
          "clustered": _clustered_boxes, "cfg2_small": lambda: W.cfg2(n_side=20)}[name]()
    g, o = _pair(wl)
    assert np.array_equal(g.quantised(), o.quantised())
    for a, b in zip(g.neighbours(), o.neighbours()):
        assert np.array_equal(a, b)


def _lattice_box(n_side=12):
    """One box of particles on a cubic lattice: many exactly equal distances."""
    L = W.KPC
    g = (np.arange(n_side) + 0.5) * L / n_side
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(pos)
    params = W.default_params(seed=5, dt=0.05 * W.MYR, dt_em=0.05 * W.MYR)
    return W._pack(params, [L], [0, n], pos, np.full(n, 1e-3), np.full(n, 1e-3 * L ** 3 / n),
                   np.full(n, 0.3), np.full(n, 1e4), [0], np.array([[0.5 * L] * 3]),
                   np.full((1, 1), 1e48), [6.3e-18], [0.0])


def _void_box(n_dense=20000, n_sparse=24, seed=13, src_at=0.15):
    """One box whose particles fill a corner cube of 0.3 of the side, with a few scattered over
    the rest: cells far from the cube have no candidate list (their n_ngb nearest lie far
    away), and queries there take the grid walk.  The source sits at src_at of the side on the
    diagonal."""
    rng = np.random.default_rng(seed)
    L = W.KPC
    pos = np.concatenate([rng.uniform(0.0, 0.3 * L, size=(n_dense, 3)),
                          rng.uniform(0.0, np.nextafter(L, 0.0), size=(n_sparse, 3))])
    n = len(pos)
    params = W.default_params(seed=seed, dt=0.05 * W.MYR, dt_em=0.05 * W.MYR)
    return W._pack(params, [L], [0, n], pos, np.full(n, 1e-3), np.full(n, 1e-3 * L ** 3 / n),
                   np.full(n, 0.3), np.full(n, 1e4), [0], np.array([[src_at * L] * 3]),
                   np.full((1, 1), 1e48), [6.3e-18], [0.0])


@pytest.mark.parametrize("name,occ", [("cfg2_small", 0), ("cfg2_small", 1), ("cfg2_small", 6),
                                      ("lattice", 0), ("lattice", 2), ("clustered", 0),
                                      ("clustered", 1), ("void", 0), ("void", 1)])
def test_virtual_particle_search_against_brute_force(name, occ):
    """The virtual particles' exact kNN from the per-cell candidate lists (Sec. 2.1: a virtual
    particle's neighbours are the n_ngb particles nearest to it) equals a brute-force search,
    ties to the lower index, for points like virtual particles (within a smoothing length of a
    particle), points on particles, cell corners and the edges and corners of the box, on
    uniform, lattice (exact ties) and clustered boxes with duplicate positions, at several
    grid occupancies; in a box that is mostly void, the cells without a list answer by the
    grid walk, with the same result."""
    from paper_1311_0182_gb300 import rt
    wl = {"cfg2_small": lambda: W.cfg2(n_side=20), "lattice": _lattice_box,
          "clustered": _clustered_boxes, "void": _void_box}[name]()
    g = rt.context_for(dict(wl, params=dict(wl["params"], cell_occupancy=occ)))
    if name == "void":
        assert g.stats()["candidate_fallback_cells"] > 0
    elif name in ("cfg2_small", "lattice"):
        assert g.stats()["candidate_fallback_cells"] == 0
    q = g.quantised()
    nbr, h2 = g.neighbours()[:2]
    k = wl["params"]["n_ngb"]
    rng = np.random.default_rng(3)
    off = wl["box_off"]
    Q = 1 << 20
    for b in range(len(off) - 1):
        lo, hi = int(off[b]), int(off[b + 1])
        qb = q[lo:hi]
        m = 200
        pi = rng.integers(0, hi - lo, m)
        d = rng.normal(size=(m, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        r = np.sqrt(h2[lo + pi]) * rng.uniform(0, 1, m) ** (1 / 3)
        pts = [np.clip(np.rint(qb[pi] + d * r[:, None]), 0, Q - 1).astype(np.int64),
               qb[rng.integers(0, hi - lo, 20)],
               np.array([[x, y, z] for x in (0, Q - 1) for y in (0, Q - 1) for z in (0, Q - 1)]),
               np.stack([rng.integers(0, Q, 20), np.zeros(20, np.int64),
                         np.full(20, Q - 1)], 1),
               (rng.integers(0, 8, (20, 3)) * (Q // 8)).astype(np.int64)]
        pts = np.concatenate(pts)
        got, gd2 = g.query_neighbours(b, pts)
        idx = np.arange(lo, hi)
        for p, nb, dd in zip(pts, got, gd2):
            d2 = ((qb - p) ** 2).sum(1)
            order = np.lexsort((idx, d2))[:k]
            assert np.array_equal(nb, idx[order]), (name, occ, b, p)
            assert np.array_equal(dd, d2[order])
    with pytest.raises(rt.RTError):
        g.query_neighbours(0, np.array([[0, 0, Q]]))
    g.close()


@pytest.mark.parametrize("fp32", [0, 1])
def test_steps_with_virtual_particles_in_cells_without_a_list(fp32):
    """Virtual particles placed in cells without a candidate list take the grid walk inside the
    step (the virtual-particle kernel's instance with the fallback).  The source sits deep in
    the void of a box whose particles fill a corner cube, so its empty cones place virtual
    particles far from the cube.  Three steps against the oracle: FP64 within 1e-7 in the
    absorptions and the state (a wrong neighbour set would move them by order one); FP32
    conserves photons and stays within the bars, with the routing-flip allowance of the other
    FP32 tests."""
    wl = _void_box(n_dense=6000, n_sparse=16, src_at=0.8)
    g, o = _pair(wl, transport_fp32=fp32, cell_occupancy=1)
    assert g.stats()["candidate_fallback_cells"] > 0
    affected = np.zeros(g.n, dtype=bool)
    for step in range(3):
        g.step(step)
        assert o.step(step) == 0
        if fp32:
            _route_affected(g, o, wl["N_H"], affected)
    assert g.stats()["virtual"] > 0
    if fp32 == 0:
        ag, eg, pg = g.deposits()
        ao, eo, po = o.deposits()
        assert np.allclose(ag, ao, rtol=1e-7, atol=1e-12 * max(ao.max(), 1e-300))
        sg, so = g.state(), o.state()
        assert np.allclose(sg["x_HI"], so["x_HI"], rtol=1e-7, atol=1e-15)
        assert np.allclose(sg["T"], so["T"], rtol=1e-7)
    else:
        _assert_fp32_bars(g.state(), o.state(), affected, 3, "void box")
    b = g.budget()[0]
    assert abs(b[0] - b[1:].sum()) <= (1e-9 if fp32 == 0 else 1e-6) * b[0]
    g.close()


def test_neighbours_full_size_sampled():
    """The timed 64^3 workload: sampled particles against a brute-force search."""
    wl = W.cfg2()
    from paper_1311_0182_gb300 import rt
    g = rt.context_for(wl)
    nbr, h2, snbr, sh2 = g.neighbours()
    q = g.quantised()
    k = wl["params"]["n_ngb"]
    rng = np.random.default_rng(0)
    idx = np.arange(g.n)
    for i in rng.choice(g.n, 64, replace=False):
        d2 = ((q - q[i]) ** 2).sum(1)
        keep = idx != i
        order = np.lexsort((idx[keep], d2[keep]))[:k]
        assert np.array_equal(nbr[i], idx[keep][order])
        assert h2[i] == d2[keep][order][-1]


@pytest.mark.parametrize("fp32", [0, 1])
def test_rotations_bit_exact(fp32):
    wl = W.cfg1()
    g, o = _pair(wl, transport_fp32=fp32)
    for step in (0, 7, 123456789012):
        g.assign_cones(step)
        o.rotate(step)
        Rg, Rsg = g.rotations()
        Ro, Rso = o.rotations()
        assert np.array_equal(Rg, Ro) and np.array_equal(Rsg, Rso)


def _random_slots(n, S, seed, frac=0.3, lo=40, hi=50):
    rng = np.random.default_rng(seed)
    f = np.zeros((6, n, S))
    on = rng.random((n, S)) < frac
    N = np.where(on, 10 ** rng.uniform(lo, hi, (n, S)), 0.0)
    d = rng.normal(size=(3, n, S))
    d /= np.linalg.norm(d, axis=0)
    f[0] = N
    f[1:4] = N * d
    f[4] = 0.0
    f[5] = N * 2.0 * W.EV
    return f


def test_cone_masks_bit_exact_fp64():
    for wl in (W.cfg1(), W.cfg2(n_side=16), W.tiny(n=500, n_ngb=24, n_tc=3)):
        g, o = _pair(wl, transport_fp32=0)
        f = _random_slots(g.n, g.S, 5)
        g.assign_cones(3)
        o.rotate(3)
        g.set_slots(f)
        o.set_slots(f)
        g.assign_cones(3)
        mg, mo = g.cone_masks(), o.cone_masks()
        assert np.array_equal(mg, mo)
        assert (mo != 0).mean() > 0.1


def _fp32_directions(M32):
    """The FP32 path's packet direction from its stored FP32 momentum ([3, ...] float32), in
    correctly rounded single-precision operations in the library's order: scale by the
    reciprocal of the largest component, (a^2 + b^2) + c^2, square root, reciprocal."""
    one = np.float32(1.0)
    s = np.maximum(np.abs(M32[0]), np.maximum(np.abs(M32[1]), np.abs(M32[2])))
    nz = s > 0
    is_ = np.where(nz, one / np.where(nz, s, one), np.float32(0.0)).astype(np.float32)
    a, b, c = (M32[0] * is_).astype(np.float32), (M32[1] * is_).astype(np.float32), \
        (M32[2] * is_).astype(np.float32)
    q = ((a * a).astype(np.float32) + (b * b).astype(np.float32)).astype(np.float32)
    q = (q + (c * c).astype(np.float32)).astype(np.float32)
    rn = (one / np.sqrt(np.where(nz, q, one)).astype(np.float32)).astype(np.float32)
    d = np.stack([(a * rn).astype(np.float32), (b * rn).astype(np.float32),
                  (c * rn).astype(np.float32)], -1).astype(np.float64)
    d[~nz] = (1.0, 0.0, 0.0)
    return d


def _edge_slots(g, wl, seed, frac=0.5):
    """Random packets, half of them aimed so that one neighbour lies within 1e-6 (relative, in
    angle) of the transmission cone's edge: the membership is then decided inside the FP32
    guard band, by the exact test."""
    rng = np.random.default_rng(seed)
    f = _random_slots(g.n, g.S, seed)
    q = g.quantised().astype(np.float64)
    nbr = g.neighbours()[0]
    cos_t = 1.0 - 2.0 / wl["params"]["n_tc"]
    th = np.arccos(cos_t)
    on = (f[0] > 0) & (rng.random((g.n, g.S)) < frac)
    ii, ss = np.nonzero(on)
    k = rng.integers(0, nbr.shape[1], len(ii))
    dl = q[nbr[ii, k]] - q[ii]
    u = dl / np.linalg.norm(dl, axis=1, keepdims=True)
    r = rng.normal(size=u.shape)
    w = r - (r * u).sum(1, keepdims=True) * u
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    ang = th * (1.0 + rng.uniform(-1e-6, 1e-6, len(ii)))
    d = np.cos(ang)[:, None] * u + np.sin(ang)[:, None] * w
    N = f[0][ii, ss]
    for a in range(3):
        f[1 + a][ii, ss] = N * d[:, a]
    return f


@pytest.mark.parametrize("name", ["cfg1", "cfg2_16", "tiny_ntc3"])
def test_cone_masks_fp32_bit_exact_on_the_float_directions(name):
    """FP32 path: the masks are the exact cone test (FP64) evaluated on the packet's FP32
    direction, a correctly rounded function of the stored FP32 momentum.  The oracle, given that
    direction (reproduced here from the stored momentum), gives the same masks bit for bit,
    with half the packets aimed at a cone edge."""
    wl = {"cfg1": lambda: W.cfg1(), "cfg2_16": lambda: W.cfg2(n_side=16),
          "tiny_ntc3": lambda: W.tiny(n=500, n_ngb=24, n_tc=3)}[name]()
    g, o = _pair(wl, transport_fp32=1)
    f = _edge_slots(g, wl, 6)
    g.assign_cones(1)
    o.rotate(1)
    g.set_slots(f)
    g.assign_cones(1)
    fg = g.slots()          # the FP32-stored packets, in physical units
    o.set_slots(fg)
    # the slot unit of the FP32 path is the box's source photons per step; dividing by it and
    # rounding to FP32 recovers the stored FP32 momentum exactly
    p = wl["params"]
    K = max(1, int(round(p["dt"] / p["dt_em"])))
    norm = float(np.sum(wl["src_ndot"]) * p["dt_em"] * K)
    M32 = (fg[1:4] / norm).astype(np.float32)
    assert np.allclose(M32.astype(np.float64) * norm, fg[1:4], rtol=1e-12, atol=0.0)
    mo = o.cone_masks_given_directions(_fp32_directions(M32))
    mg = g.cone_masks()
    assert np.array_equal(mg, mo)
    assert (mo != 0).mean() > 0.1


# --- floating-point work ------------------------------------------------------------------------
@pytest.mark.parametrize("fp32", [0, 1])
def test_step_parity_cfg1(fp32):
    """Strömgren workload (16^3, 8 cones): 12 steps of the whole step against the oracle."""
    wl = W.cfg1()
    g, o = _pair(wl, transport_fp32=fp32)
    affected = np.zeros(g.n, bool)
    for step in range(12):
        g.step(step)
        assert o.step(step) == 0
        if fp32 == 0:
            ok = _xhi_ok(g.state()["x_HI"], o.state()["x_HI"])
            assert ok.all(), f"step {step}: {np.count_nonzero(~ok)} particles off"
        else:
            _route_affected(g, o, wl["N_H"], affected)
            _assert_fp32_bars(g.state(), o.state(), affected, step + 1, f"step {step}")
    bg, bo = g.budget()[0], o.budget()[0]
    assert np.allclose(bg[:3], bo[:3], rtol=1e-6, atol=1e-6 * bo[0])
    assert abs(bg[0] - bg[1] - bg[2] - bg[3]) <= (1e-9 if fp32 == 0 else 1e-6) * bg[0]
    sg, so = g.stats(), o.stats()
    if fp32 == 0:
        # the last hops carry packets of ~1e-300 photons whose fate depends on the last bits
        # of exp(): hop and virtual counts agree closely but need not be equal
        assert abs(sg["hops"] - so["hops"]) <= 3
        assert abs(sg["virtual"] / so["virtual"] - 1) < 0.01


@pytest.mark.parametrize("fp32", [0, 1])
def test_step_parity_evolving_temperature(fp32):
    """The 1e5 K blackbody HII region with T evolving, 8 source bins, 32 cones, at 20^3."""
    wl = W.cfg2(n_side=20)
    g, o = _pair(wl, transport_fp32=fp32)
    affected = np.zeros(g.n, bool)
    for step in range(3):
        g.step(step)
        assert o.step(step) == 0
        _route_affected(g, o, wl["N_H"], affected)
    sg, so = g.state(), o.state()
    ok = _xhi_ok(sg["x_HI"], so["x_HI"])
    relT = np.abs(sg["T"] / so["T"] - 1)
    if fp32 == 0:
        assert ok.all()
        assert (relT < 1e-3).all()
        assert not affected.any()
    else:
        _assert_fp32_bars(sg, so, affected, 3)
    bg, bo = g.budget()[0], o.budget()[0]
    assert np.allclose(bg[:3], bo[:3], rtol=1e-6, atol=1e-6 * bo[0])


@pytest.fixture(scope="module")
def timed_config_oracle():
    """The oracle's run of the timed configuration at 32^3: the HII region from its seeded
    mid-expansion start, 1e5 K blackbody in 8 bins plus the recombination bin, 32 cones, T
    evolving, 3 steps; per step the absorbed photons and energy, the state and the budget."""
    wl = W.cfg2(n_side=32)
    o = oracle.Sim(wl)
    o.build_neighbours()
    steps = []
    for step in range(3):
        assert o.step(step) == 0
        a, e, _ = o.deposits()
        st = o.state()
        steps.append({"A": a.sum(1), "E": e if e.ndim == 1 else e.sum(1),
                      "x_HI": st["x_HI"].copy(), "T": st["T"].copy(), "N_rec": st["N_rec"].copy(),
                      "budget": o.budget().copy()})
    return wl, steps


@pytest.mark.parametrize("fp32", [0, 1])
def test_timed_configuration_against_the_oracle(fp32, timed_config_oracle):
    """The configuration the benchmark times (HII region, 32 cones, 9 bins, T evolving, from the
    mid-expansion start) at 32^3 for 3 steps, element by element against the oracle.  FP64:
    every particle's x_HI and T to 1e-7 and recombination photons to 1e-9, budget to 1e-9 (the
    explicit energy subcycles of particles heated from 100 K magnify last-bit differences of
    the rate fits to a few 1e-9).  FP32 transport
    / FP64 chemistry: every particle not routing-affected within the x_HI and T bars, the
    routing-affected ones within the flip budget, budget within 1e-6."""
    from paper_1311_0182_gb300 import rt
    wl, ref = timed_config_oracle
    g = rt.context_for(wl, transport_fp32=fp32)
    affected = np.zeros(g.n, bool)
    for step, r in enumerate(ref):
        g.step(step)
        ag, eg, _ = g.deposits()
        ACC.mark_routing_affected(ag.sum(1), r["A"], eg.sum(1), r["E"], wl["N_H"], affected)
        sg = g.state()
        bg, bo = g.budget()[0], r["budget"][0]
        if fp32 == 0:
            assert not affected.any(), f"step {step}"
            for k in ("x_HI", "T"):
                rel = np.abs(sg[k] / r[k] - 1)
                assert rel.max() < 1e-7, f"step {step} {k}: {rel.max():.2e}"
            # N_rec scales with 1 - x_HI, which magnifies the last bits of x_HI in nearly
            # neutral gas: compared relative to the largest emitter there
            assert np.allclose(sg["N_rec"], r["N_rec"], rtol=1e-7, atol=1e-9 * r["N_rec"].max())
            assert np.allclose(bg, bo, rtol=1e-9, atol=1e-9 * bo[0])
        else:
            _assert_fp32_bars(sg, r, affected, step + 1, f"step {step}")
            assert np.allclose(bg[:3], bo[:3], rtol=1e-6, atol=1e-6 * bo[0])
        assert abs(bg[0] - bg[1:].sum()) <= (1e-9 if fp32 == 0 else 1e-6) * bg[0]
    print(f"fp32={fp32}: {affected.sum()} of {g.n} particles routing-affected in 3 steps")


@pytest.mark.parametrize("fp32", [0, 1])
def test_subcycle_floor_reports_its_status(fp32):
    """A subcycle floor (dt/sub_cap, sub_cap = 4) too coarse for the heating at the front: the
    step completes and returns RT_ERR_SUBCYCLE_LIMIT, as the oracle's step does, on the step
    graph, on the host-driven loop and from rt_chemistry alone; the state is written (FP64: as
    the oracle's to 1e-9) and the floor hits are counted (FP64: as many as the oracle's).  With
    the default sub_cap the same step reports nothing."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg2(n_side=12, sub_cap=4)
    g, o = _pair(wl, transport_fp32=fp32)
    h = rt.context_for(wl, transport_fp32=fp32)
    h.set_graph(False)
    p = rt.context_for(wl, transport_fp32=fp32)
    assert o.step(0) == rt.RT_ERR_SUBCYCLE_LIMIT
    assert g.step(0, allow_subcycle_limit=True) == rt.RT_ERR_SUBCYCLE_LIMIT
    assert h.step(0, allow_subcycle_limit=True) == rt.RT_ERR_SUBCYCLE_LIMIT
    p.assign_cones(0)
    p.merge()
    p.emit(0)
    p.transport(0)
    assert p.chemistry(allow_subcycle_limit=True) == rt.RT_ERR_SUBCYCLE_LIMIT
    with pytest.raises(rt.RTError):
        h.step(1)
    fo = o.stats()["floor_hits"]
    assert fo > 0 and g.stats()["floor_hits"] > 0
    if fp32 == 0:
        # the subcycles held at the floor take explicit energy steps far beyond the 10% limit,
        # which magnify last-bit differences of the rate fits: 1e-6 here
        assert g.stats()["floor_hits"] == fo
        sg, so = g.state(), o.state()
        for k in ("x_HI", "T"):
            assert np.max(np.abs(sg[k] / so[k] - 1)) < 1e-6
    for c in (g, h, p):
        b = c.budget()[0]
        assert abs(b[0] - b[1:].sum()) <= 1e-6 * b[0]
    q = rt.context_for(W.cfg2(n_side=12), transport_fp32=fp32)
    assert q.step(0) == 0 and q.stats()["floor_hits"] == 0


@pytest.mark.parametrize("fp32", [0, 1])
def test_boxes_cut_out_of_a_batch_repeat_their_results(fp32):
    """The boxes of workload 4 split in two, each part run on its own context with the
    identities its particles and sources have in the whole batch (rt_set_identities): every
    box's particles end with the x_HI and T, and every box with the photon budget, of the
    unsplit run, bit for bit.  This is how the boxes are shared among GPUs."""
    from paper_1311_0182_gb300 import distributed as D, rt
    wl = W.cfg4(n_boxes=24, n_min=300, n_max=3000, transport_fp32=fp32)
    full = rt.context_for(wl)
    for step in range(3):
        full.step(step)
    sf, bf = full.state(), full.budget()
    for part in D.partition_boxes(np.diff(wl["box_off"]), 2):
        sub = D.local_workload(wl, part)
        g = rt.context_for(sub)
        for step in range(3):
            g.step(step)
        idx = np.concatenate([np.arange(wl["box_off"][b], wl["box_off"][b + 1]) for b in part])
        sg = g.state()
        assert np.array_equal(sg["x_HI"], sf["x_HI"][idx])
        assert np.array_equal(sg["T"], sf["T"][idx])
        assert np.array_equal(g.budget(), bf[part])


def test_cost_does_not_grow_with_the_number_of_sources():
    """Sec. 2.1 on the GPU: the HII region's luminosity split over 64 sources clustered where
    one sat moves well under twice the packets of the single source per step, and sends from no
    more particles than hops x particles, where tracing every source's rays would cost about
    64 times as much."""
    from paper_1311_0182_gb300 import rt
    moved = {}
    for ns in (1, 64):
        wl = W.split_sources(W.cfg2(n_side=24), ns)
        g = rt.context_for(wl)
        moved[ns] = 0
        for step in range(3):
            g.step(step)
            st = g.stats()
            assert 0 < st["senders"] <= st["hops"] * g.n
            moved[ns] += st["moving_packets"]
        b = g.budget()[0]
        assert abs(b[0] - b[1:].sum()) <= 1e-6 * b[0]
    assert moved[64] < 2 * moved[1], moved


def test_multi_box_parity_and_conservation():
    wl = _clustered_boxes()
    g, o = _pair(wl, transport_fp32=0)
    for step in range(3):
        g.step(step)
        assert o.step(step) == 0
    assert _xhi_ok(g.state()["x_HI"], o.state()["x_HI"]).all()
    bg, bo = g.budget(), o.budget()
    assert np.allclose(bg[:, :3], bo[:, :3], rtol=1e-6, atol=1e-6 * bo[:, :1])
    assert np.all(np.abs(bg[:, 0] - bg[:, 1:].sum(1)) <= 1e-9 * bg[:, 0])


def test_deposits_single_step():
    wl = W.cfg1()
    g, o = _pair(wl, transport_fp32=0)
    for step in range(4):
        g.step(step)
        o.step(step)
    ag, eg, pg = g.deposits()
    ao, eo, po = o.deposits()
    scale = ao.max()
    assert np.allclose(ag, ao, rtol=1e-6, atol=1e-9 * scale)
    assert np.allclose(pg, po, rtol=1e-6, atol=1e-9 * po.max())


def test_optically_thin_all_escape():
    wl = W.cfg1()
    wl["x_HI"][:] = 0.0
    g, o = _pair(wl, transport_fp32=1)
    g.step(0)
    b = g.budget()[0]
    assert b[1] == 0.0 and b[3] == 0.0
    assert abs(b[2] / b[0] - 1) < 1e-6


def test_no_sources_and_minimal_box():
    rng = np.random.default_rng(3)
    n = 33
    L = W.KPC
    pos = rng.uniform(0, L, (n, 3))
    params = W.default_params(seed=5, dt=0.05 * W.MYR, dt_em=0.05 * W.MYR)
    wl = W._pack(params, [L], [0, n], pos, np.full(n, 1e-3), np.full(n, 1e-3 * L ** 3 / n),
                 np.full(n, 0.5), np.full(n, 1e4), np.zeros(0, np.int32), np.zeros((0, 3)),
                 np.zeros((0, 1)), [6.3e-18], [0.0])
    g, o = _pair(wl)
    for step in range(3):
        g.step(step)
        o.step(step)
    assert _xhi_ok(g.state()["x_HI"], o.state()["x_HI"]).all()
    b = g.budget()[0]
    assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-9 * max(b[0], 1.0)


# --- regimes and options ------------------------------------------------------------------------
@pytest.mark.parametrize("fp32", [0, 1])
def test_clock_limited_steps_park_and_rebin(fp32):
    """c dt (3 kpc) shorter than the box: packets wait at particles, restart next step and are
    re-sorted into the new reception cones (rt_merge)."""
    wl = W.cfg1(dt=0.01 * W.MYR, dt_em=0.01 * W.MYR)
    wl["x_HI"][:] = 0.2
    g, o = _pair(wl, transport_fp32=fp32)
    affected = np.zeros(g.n, bool)
    for step in range(6):
        g.step(step)
        assert o.step(step) == 0
        _route_affected(g, o, wl["N_H"], affected)
    fg, fo = g.slots(), o.slots()
    assert (fo[0] > 0).sum() > 100                 # packets are waiting
    ok = _xhi_ok(g.state()["x_HI"], o.state()["x_HI"])
    bg, bo = g.budget()[0], o.budget()[0]
    if fp32 == 0:
        assert ok.all()
        assert np.array_equal(fg[0] > 0, fo[0] > 0)
        assert np.allclose(fg[0], fo[0], rtol=1e-9, atol=1e-12 * fo[0].max())
    else:
        _assert_fp32_bars(g.state(), o.state(), affected, 6)
    assert np.allclose(bg, bo, rtol=1e-6, atol=1e-6 * bo[0])
    assert abs(bg[0] - bg[1:].sum()) <= 1e-6 * bg[0]


@pytest.mark.parametrize("mode", [W.REC_OTS_CASE_B, W.REC_CASE_A])
def test_on_the_spot_and_case_a_modes(mode):
    wl = W.cfg1(rec_mode=mode)
    g, o = _pair(wl, transport_fp32=0)
    for step in range(8):
        g.step(step)
        assert o.step(step) == 0
    assert _xhi_ok(g.state()["x_HI"], o.state()["x_HI"]).all()
    assert np.all(g.state()["N_rec"] == 0.0)


@pytest.mark.parametrize("fp32", [0, 1])
def test_original_emission_cone_recombination_mode(fp32):
    """Recombination radiation through per-particle emission cones (Sec. 2.2, the original
    implementation): free packets from every recombining particle in the first hop.  FP64: the
    same numbers as the oracle to rounding; FP32: within the x_HI bar; budgets within 1e-6."""
    wl = W.cfg1(rec_mode=W.REC_EMISSION_CONES, n_ec=8)
    wl["x_HI"][:] = 0.05
    g, o = _pair(wl, transport_fp32=fp32)
    for step in range(6):
        g.step(step)
        assert o.step(step) == 0
    xg, xo = g.state()["x_HI"], o.state()["x_HI"]
    assert _xhi_ok(xg, xo).all()
    if not fp32:
        assert np.max(np.abs(xg / xo - 1)) < 1e-10
    assert g.state()["N_rec"].max() > 0
    bg, bo = g.budget()[0], o.budget()[0]
    assert np.allclose(bg, bo, rtol=1e-6, atol=1e-6 * bo[0])
    assert abs(bg[0] - bg[1:].sum()) <= 1e-6 * bg[0]


@pytest.mark.parametrize("n_ngb,n_tc,n_rc,n_ec", [(16, 2, 8, 32), (24, 64, 32, 8), (12, 3, 8, 8)])
def test_other_neighbour_and_cone_counts(n_ngb, n_tc, n_rc, n_ec):
    wl = W.cfg1(n_side=12, n_ngb=n_ngb, n_tc=n_tc, n_rc=n_rc, n_ec=n_ec)
    wl["x_HI"][:] = 0.05
    g, o = _pair(wl, transport_fp32=0)
    for a, b in zip(g.neighbours(), o.neighbours()):
        assert np.array_equal(a, b)
    for step in range(3):
        g.step(step)
        assert o.step(step) == 0
    assert _xhi_ok(g.state()["x_HI"], o.state()["x_HI"]).all()
    bg, bo = g.budget()[0], o.budget()[0]
    assert np.allclose(bg, bo, rtol=1e-6, atol=1e-6 * bo[0])


def test_fixed_recombination_energy_and_evolving_temperature():
    wl = W.cfg2(n_side=14, eps_rr_fixed=2.3 * W.EV)
    g, o = _pair(wl, transport_fp32=0)
    for step in range(3):
        g.step(step)
        o.step(step)
    sg, so = g.state(), o.state()
    assert np.all(sg["eps_rec"] == 2.3 * W.EV)
    assert _xhi_ok(sg["x_HI"], so["x_HI"]).all()
    assert (np.abs(sg["T"] / so["T"] - 1) < 1e-3).all()


def test_parts_equal_the_whole_step():
    """rt_assign_cones + rt_merge + rt_emit + rt_transport + rt_chemistry == rt_step."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg1()
    a = rt.context_for(wl)
    b = rt.context_for(wl)
    for step in range(4):
        a.step(step)
        b.assign_cones(step)
        b.merge()
        b.emit(step)
        b.transport(step)
        b.chemistry()
    assert np.array_equal(a.state()["x_HI"], b.state()["x_HI"])
    assert np.array_equal(a.budget(), b.budget())


def test_hop_cap_reports_and_conserves():
    wl = W.cfg1(hop_cap=5)
    wl["x_HI"][:] = 1e-3
    g, o = _pair(wl, transport_fp32=0)
    from paper_1311_0182_gb300 import rt
    g.assign_cones(0); g.merge(); g.emit(0)
    st = g.transport(0, allow_hop_limit=True)
    assert st == 4                                  # RT_ERR_HOP_LIMIT
    g.chemistry()
    o.rotate(0); o.rebin(); o.emit(0)
    assert o.transport(0) == 4
    o.chemistry()
    bg, bo = g.budget()[0], o.budget()[0]
    assert np.allclose(bg, bo, rtol=1e-9, atol=1e-9 * bo[0])
    assert abs(bg[0] - bg[1:].sum()) <= 1e-9 * bg[0]


def _graph_pair(wl):
    from paper_1311_0182_gb300 import rt
    a = rt.context_for(wl)
    b = rt.context_for(wl)
    b.set_graph(False)
    return a, b


def _same_results(a, b):
    sa, sb = a.state(), b.state()
    for k in ("x_HI", "T", "N_rec", "eps_rec"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a.budget(), b.budget())
    for x, y in zip(a.deposits(), b.deposits()):
        assert np.array_equal(x, y)
    # (the kNN grid occupancy, with the size of its candidate lists, and the launch sizes are
    # chosen by timing and may differ; results do not depend on them)
    sta, stb = a.stats(), b.stats()
    for k in ("cell_occupancy", "grid_send", "grid_virtual", "grid_receive", "candidate_entries"):
        sta.pop(k)
        stb.pop(k)
    assert sta == stb


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("name", ["cfg2_24", "shadow", "original", "shared"])
def test_step_graph_equals_hop_by_hop_loop(name, fp32):
    """rt_step as one captured CUDA graph (a conditional while node around the hop, a switch
    node over the four buffer pairs) gives the same bits as the host-driven hop loop, with the
    same kernel launch counts (the graph launches the hop-cap drop every step; the loop only
    at the cap): the HII region at 24^3 (32 cones, 8 frequency bins), the shadow workload
    (barrier, directed and gated emitters), the original recombination implementation and the
    shared frequency bin."""
    wl = {"cfg2_24": lambda: W.cfg2(n_side=24, transport_fp32=fp32),
          "shadow": lambda: W.shadow(n_side=16, n_front=20, n_bnd=10, transport_fp32=fp32),
          "original": lambda: W.cfg1(rec_mode=W.REC_EMISSION_CONES, transport_fp32=fp32),
          "shared": lambda: W.cfg2(n_side=16, rec_shared_bin=1, transport_fp32=fp32)}[name]()
    a, b = _graph_pair(wl)
    for step in range(5):
        a.step(step)
        b.step(step)
        assert a.stats()["hops"] > 0
        _same_results(a, b)
    ka, kb = a.kernel_times(), b.kernel_times()
    ka.pop("drop_free", None)
    kb.pop("drop_free", None)
    assert {k: v["launches"] for k, v in ka.items()} == {k: v["launches"] for k, v in kb.items()}


def test_step_graph_at_the_hop_cap_and_after_a_barrier_change():
    """The graph stops at the hop cap with the same status, drop and budget as the host loop;
    a barrier removed between steps (a changed kernel choice) makes the graph capture again."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg1(hop_cap=5)
    wl["x_HI"][:] = 1e-3
    a, b = _graph_pair(wl)
    for step in range(2):
        assert a.step(step, allow_hop_limit=True) == 4
        assert b.step(step, allow_hop_limit=True) == 4
        _same_results(a, b)
    bg = a.budget()[0]
    assert bg[2] > 0 and abs(bg[0] - bg[1:].sum()) <= 1e-9 * bg[0]
    wl = W.shadow(n_side=16, n_front=20, n_bnd=10)
    a, b = _graph_pair(wl)
    for step in range(6):
        if step == 3:
            for c in (a, b):
                c.set_barrier(0, 0, [0.0, 0.0, 0.0], 0.0)
        a.step(step)
        b.step(step)
        _same_results(a, b)


def test_launch_size_tuning_changes_nothing_but_time():
    """With tune_launch the first steps run as the step graph, each with one triple of grid
    sizes (152 x {8, 16, 32, 64} blocks for the sender and the receiver side, 152 x {2, 3, 4, 5}
    for the virtual particles; the candidate steps alternate with steps of the best so far),
    timed whole;
    the winner is kept and reused by a later context of the same configuration and size, which
    does not tune.  Sizes given in the configuration switch the tuning off.  The results agree
    bit for bit whatever the sizes."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg2(n_side=20)
    a = rt.context_for(wl, tune_launch=1)
    b = rt.context_for(wl, tune_launch=0, launch_grid=(152, 304, 456))
    seen = set()
    for step in range(20):          # 9 candidates, each after a step of the best: 18 steps
        a.step(step)
        b.step(step)
        _same_results(a, b)
        sa = a.stats()
        seen.add((sa["grid_send"], sa["grid_virtual"], sa["grid_receive"]))
    assert len(seen) >= 9            # every candidate ran
    final = (sa["grid_send"], sa["grid_virtual"], sa["grid_receive"])
    assert final[0] in (1216, 2432, 4864, 9728) and final[2] in (1216, 2432, 4864, 9728)
    assert final[1] in (304, 456, 608, 760)
    sb = b.stats()
    assert (sb["grid_send"], sb["grid_virtual"], sb["grid_receive"]) == (152, 304, 456)
    c = rt.context_for(wl, tune_launch=1)
    c.step(0)
    sc = c.stats()
    assert (sc["grid_send"], sc["grid_virtual"], sc["grid_receive"]) == final


@pytest.mark.parametrize("case", ["fp64", "fp32", "shared_clock_limited"])
def test_checkpoint_resume_repeats_the_run_bit_for_bit(case):
    """rt_save_state after two steps, rt_load_state into a fresh context built from the same
    inputs, two more steps: the same bits as four uninterrupted steps (state, budget,
    deposits, held packets).  With clock-limited steps packets are held across the checkpoint.
    A checkpoint of another configuration is refused."""
    from paper_1311_0182_gb300 import rt
    kw = {"fp64": dict(transport_fp32=0), "fp32": dict(transport_fp32=1),
          "shared_clock_limited": dict(transport_fp32=1, rec_shared_bin=1, dt=0.01 * W.MYR,
                                       dt_em=0.01 * W.MYR)}[case]
    wl = W.cfg2(n_side=16, **kw)
    a = rt.context_for(wl)
    b = rt.context_for(wl)
    for step in range(2):
        a.step(step)
        b.step(step)
    ck = b.save_state()
    b.close()
    c = rt.context_for(wl)
    c.load_state(ck)
    if case == "shared_clock_limited":
        assert np.count_nonzero(c.slots()[0]) > 1000 and np.count_nonzero(c.shared_sigma()) > 1000
    for step in range(2, 4):
        a.step(step)
        c.step(step)
    _same_results(a, c)
    assert np.array_equal(a.slots(), c.slots())
    other = rt.context_for(W.cfg2(n_side=16, transport_fp32=1 - kw["transport_fp32"]))
    with pytest.raises(rt.RTError):
        other.load_state(ck)


def test_free_packet_capacity_is_an_error_not_a_fault():
    from paper_1311_0182_gb300 import rt
    wl = W.cfg1(free_cap=300)
    wl["x_HI"][:] = 1e-3
    g = rt.context_for(wl)
    with pytest.raises(rt.RTError) as e:
        for step in range(3):
            g.step(step)
    assert e.value.status == 6                      # RT_ERR_CAPACITY
    # the context still works for inspection after the error
    assert g.state()["x_HI"].shape == (g.n,)


def test_state_round_trip_host_and_device():
    import torch
    from paper_1311_0182_gb300 import rt
    g = rt.context_for(W.cfg1())
    g.step(0)
    s = g.state()
    x = torch.tensor(s["x_HI"] * 0.5, device="cuda")
    g.set_state(x_HI=x)
    assert np.allclose(g.state()["x_HI"], s["x_HI"] * 0.5, rtol=0, atol=0)
    g.set_state(x_HI=s["x_HI"])
    assert np.array_equal(g.state()["x_HI"], s["x_HI"])


def test_query_neighbours_with_device_buffers():
    """rt_query_neighbours with device pointers gives what it gives with host arrays."""
    import ctypes
    import torch
    from paper_1311_0182_gb300 import rt
    g = rt.context_for(W.cfg2(n_side=16))
    q = g.quantised()
    rng = np.random.default_rng(4)
    pts = np.clip(q[rng.integers(0, g.n, 64)] + rng.integers(-5000, 5000, (64, 3)), 0,
                  (1 << 20) - 1).astype(np.int32)
    nh, dh = g.query_neighbours(0, pts)
    k = nh.shape[1]
    qd = torch.tensor(pts, device="cuda")
    nd = torch.empty((64, k), dtype=torch.int32, device="cuda")
    dd = torch.empty((64, k), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    st = g.L.rt_query_neighbours(g.h, 0, 64, ctypes.c_void_p(qd.data_ptr()),
                                 ctypes.c_void_p(nd.data_ptr()), ctypes.c_void_p(dd.data_ptr()),
                                 rt.RT_DEVICE, None)
    torch.cuda.synchronize()
    assert st == 0
    assert np.array_equal(nd.cpu().numpy(), nh) and np.array_equal(dd.cpu().numpy(), dh)
    g.close()


def test_profiling_mask_times_only_the_chosen_kernels():
    """Kernels outside the mask are counted but not timed; the mask leaves results unchanged."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg1()
    a = rt.context_for(wl)
    b = rt.context_for(wl)
    a.profile(["virtual_particles", "phase_a_send"])
    for step in range(2):
        a.step(step)
        b.step(step)
    kt = a.kernel_times()
    assert kt["virtual_particles"]["ms"] > 0 and kt["phase_a_send"]["ms"] > 0
    assert kt["phase_b_merge"]["launches"] > 0 and kt["phase_b_merge"]["ms"] == 0
    a.profile(False)
    assert np.array_equal(a.state()["x_HI"], b.state()["x_HI"])


@pytest.mark.parametrize("fp32", [0, 1])
def test_runs_are_bitwise_reproducible(fp32):
    """The hop loop runs on two streams with integer atomics; every floating-point sum has one
    fixed order, so two runs of the same input agree bit for bit (the HII region at 24^3)."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg2(n_side=24, transport_fp32=fp32)
    a = rt.context_for(wl)
    b = rt.context_for(wl)
    for step in range(3):
        a.step(step)
        b.step(step)
    sa, sb = a.state(), b.state()
    assert np.array_equal(sa["x_HI"], sb["x_HI"])
    assert np.array_equal(sa["T"], sb["T"])
    assert np.array_equal(a.budget(), b.budget())
    assert np.array_equal(a.deposits()[0], b.deposits()[0])


def test_workload1_all_200_steps_against_the_oracle():
    """Workload 1 (16^3 Stromgren sphere, 8 cones) for all of its 200 steps of 2.5 Myr: both GPU
    paths against the oracle at steps 50, 100 and 200 (x_HI bar and budget within 1e-6)."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg1()
    o = oracle.Sim(wl)
    o.build_neighbours()
    gs = {fp: rt.context_for(dict(wl, params=dict(wl["params"], transport_fp32=fp))) for fp in (0, 1)}
    for st in range(200):
        assert o.step(st) == 0
        for g in gs.values():
            g.step(st)
        if st in (49, 99, 199):
            xo, bo = o.state()["x_HI"], o.budget()[0]
            for fp, g in gs.items():
                assert _xhi_ok(g.state()["x_HI"], xo).all(), (st, fp)
                bg = g.budget()[0]
                assert np.allclose(bg[:3], bo[:3], rtol=1e-6, atol=1e-6 * bo[0]), (st, fp)
                assert abs(bg[0] - bg[1:].sum()) <= 1e-6 * bg[0]
    # the FP64 path follows the oracle to rounding
    xg = gs[0].state()["x_HI"]
    assert np.max(np.abs(xg / o.state()["x_HI"] - 1)) < 1e-10


def test_full_size_batched_and_clump_workloads_conserve_photons():
    """Workload 4 (512 boxes, 7.1M particles) and workload 3 (2.1M particles with a 200x clump,
    the three recombination modes) at full size: every box closes its photon budget to 1e-6."""
    from paper_1311_0182_gb300 import rt
    g = rt.context_for(W.cfg4())
    for st in range(2):
        g.step(st)
    b = g.budget()
    assert (np.abs(b[:, 0] - b[:, 1:].sum(1)) <= 1e-6 * b[:, 0]).all()
    assert g.stats()["virtual"] > 0
    g.close()
    wl3 = W.cfg3()
    for mode in (W.REC_TRANSPORT, W.REC_OTS_CASE_B, W.REC_CASE_A):
        g = rt.context_for(dict(wl3, params=dict(wl3["params"], rec_mode=mode)))
        g.step(0)
        b = g.budget()[0]
        assert abs(b[0] - b[1:].sum()) <= 1e-6 * b[0]
        g.close()


def test_grid_occupancy_search_changes_nothing_but_time():
    """The kNN grid occupancy is picked by timing the virtual particles' search from the
    per-cell candidate lists (cell_occupancy 0); any grid gives the same exact neighbours, and
    the steps agree bit for bit."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg2(n_side=20)
    ctxs = {occ: rt.context_for(dict(wl, params=dict(wl["params"], cell_occupancy=occ)))
            for occ in (0, 1, 2, 5, 16)}
    assert ctxs[0].stats()["cell_occupancy"] in (1, 2, 3, 4, 6)
    assert ctxs[5].stats()["cell_occupancy"] == 5
    assert all(g.stats()["candidate_entries"] > 0 for g in ctxs.values())
    ref = ctxs[5].neighbours()
    for occ in (0, 1, 2, 16):
        for a, b in zip(ctxs[occ].neighbours(), ref):
            assert np.array_equal(a, b)
    for g in ctxs.values():
        for step in range(2):
            g.step(step)
    x = ctxs[5].state()["x_HI"]
    assert all(np.array_equal(g.state()["x_HI"], x) for g in ctxs.values())


@pytest.mark.parametrize("fp32", [0, 1])
def test_shadow_workload_against_the_oracle(fp32):
    """The shadow test of Sec. 4 at 16^3 (directed front emitters, gated boundary emitters,
    the disk barrier): 14 steps, by which the front has passed the barrier and the boundary
    emitters have switched on.  FP64 follows the oracle to rounding; FP32 within the bars."""
    wl = W.shadow(n_side=16, n_front=20, n_bnd=10)
    g, o = _pair(wl, transport_fp32=fp32)
    for step in range(14):
        g.step(step)
        assert o.step(step) == 0
    xg, xo = g.state()["x_HI"], o.state()["x_HI"]
    assert _xhi_ok(xg, xo).all()
    if not fp32:
        assert np.max(np.abs(xg / xo - 1)) < 1e-9
    assert np.allclose(g.state()["T"], o.state()["T"], rtol=1e-3)
    bg, bo = g.budget()[0], o.budget()[0]
    assert bo[2] > 0.01 * bo[0]                      # the barrier removed photons
    assert np.allclose(bg, bo, rtol=1e-6, atol=1e-6 * bo[0])
    assert abs(bg[0] - bg[1:].sum()) <= 1e-6 * bg[0]


def test_full_size_on_a_non_blocking_stream():
    """The timed 64^3 workload on a non-blocking stream (as the bench runs it): the neighbour
    lists (built, then the grid occupancy searched) match brute force at sampled particles, and
    two steps agree bit for bit with the same steps on the default stream."""
    import torch
    from paper_1311_0182_gb300 import rt
    wl = W.cfg2()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = rt.context_for(wl, stream=s)
    nbr, h2, _, _ = g.neighbours()
    q = g.quantised()
    k = wl["params"]["n_ngb"]
    rng = np.random.default_rng(1)
    idx = np.arange(g.n)
    for i in rng.choice(g.n, 48, replace=False):
        d2 = ((q - q[i]) ** 2).sum(1)
        keep = idx != i
        order = np.lexsort((idx[keep], d2[keep]))[:k]
        assert np.array_equal(nbr[i], idx[keep][order])
    d = rt.context_for(wl)
    with torch.cuda.stream(s):
        for step in range(2):
            g.step(step)
    for step in range(2):
        d.step(step)
    assert np.array_equal(g.state()["x_HI"], d.state()["x_HI"])


@pytest.mark.parametrize("fp32", [1, 0])
def test_full_size_chemistry_sampled_against_the_oracle(fp32):
    """The timed 64^3 workload in the bench's launch sizes: after a step's transport, the
    chemistry of 300 sampled particles (200 at random, 100 with the most absorptions), computed
    one by one by the oracle from the same absorbed photons and energy and the same x_HI and T,
    matches the GPU's.  FP64 path: to 1e-9.  Mixed path, whose rate fits run in FP32: x_HI
    and T to 1e-4; the recombination photons to emit (an integral of the difference
    alpha_A - alpha_B of two FP32 fits times the electron density) to 1e-3, the bar of the fields
    they feed.  Both paths compare those photons per particle where the gas is at least 1 %
    ionised, and summed over the sample: in nearly neutral gas they scale with 1 - x_HI, which
    x_HI to a relative tolerance does not fix (the summed inputs already differ in their last
    bits)."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg2(transport_fp32=fp32)
    g = rt.context_for(wl)
    g.step(0)                        # recombination photons to emit in the next step
    g.assign_cones(1)
    g.merge()
    g.emit(1)
    g.transport(1)
    before = g.state()
    a, e, _ = g.deposits()
    g.chemistry()
    after = g.state()
    phot, heat = a.sum(1), e.sum(1)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(g.n, 200, replace=False), np.argsort(phot)[-100:]])
    assert phot[idx].max() > 0
    tol = 1e-4 if fp32 else 1e-9
    tol_rec = 1e-3 if fp32 else 1e-9
    sum_g = sum_o = 0.0
    for i in idx:
        x, T, nrec, _, _ = oracle.chem_particle(wl["params"], wl["n_H"][i], wl["N_H"][i],
                                                phot[i], heat[i], before["x_HI"][i],
                                                before["T"][i])
        xg, Tg, ng = after["x_HI"][i], after["T"][i], after["N_rec"][i]
        assert abs(xg - x) <= max(tol * x, 1e-7 if x < 1e-4 else 0.0), (i, xg, x)
        assert abs(Tg - T) <= tol * T, (i, Tg, T)
        if 1.0 - x > 0.01:
            assert abs(ng - nrec) <= tol_rec * max(nrec, 1e-300) + 1e-300, (i, ng, nrec)
        sum_g += ng
        sum_o += nrec
    assert sum_o > 0 and abs(sum_g - sum_o) <= tol_rec * sum_o


def test_app_a_convergence_with_resolution_and_time_step():
    """App. A: the Stromgren sphere with transported recombination radiation converges with
    particle number, RT time step and angular resolution.  After one t_rec, the I-fronts of
    32^3 and 64^3 runs, of runs with dt = 1 and 0.1 Myr (dt_em = 0.1 dt) and of runs with 8 and
    64 transmission cones lie within one smoothing length of each other, and the recombination
    intensity inside R_S/2 agrees to 25 % between the resolutions (narrow cones send more
    photons through virtual particles, which pass no gas particle, so that count is not
    compared across cone numbers)."""
    from paper_1311_0182_gb300 import convergence as CV
    a = CV.run(n_side=32, dt_myr=1.0, t_rec=1.0)
    b = CV.run(n_side=64, dt_myr=1.0, t_rec=1.0)
    c = CV.run(n_side=32, dt_myr=0.1, t_rec=1.0)
    d = CV.run(n_side=32, dt_myr=1.0, n_tc=64, t_rec=1.0)
    h = a["mean_h_over_RS"]
    assert abs(a["front_over_RS"] - b["front_over_RS"]) < h
    assert abs(a["front_over_RS"] - c["front_over_RS"]) < h
    assert abs(a["front_over_RS"] - d["front_over_RS"]) < h
    ia = np.array([p["intensity"] for p in a["profile"][:4]])
    ib = np.array([p["intensity"] for p in b["profile"][:4]])
    assert np.all(np.abs(ia / ib - 1) < 0.25)


# --- shared frequency bin (Sec. 2.2, last paragraph) ---------------------------------------------
def _shared_chain(n_part=40, spacing=0.1 * W.KPC):
    """Particles on a line with two neighbours each, one shared frequency bin: a packet sent
    along +x reaches only the next particle."""
    L = (n_part + 1) * spacing
    wl = W.tiny(n=n_part, n_ngb=2, L=L, n_tc=64, rec_shared_bin=1)
    yz = np.full(n_part, 0.5 * L)
    wl.update(x=(np.arange(n_part) + 0.5) * spacing, y=yz.copy(), z=yz.copy(),
              n_H=np.full(n_part, 1e-3), N_H=np.full(n_part, 1e-3 * spacing ** 3),
              x_HI=np.full(n_part, 1e-2), T=np.full(n_part, 1e4), src_box=np.zeros(0, np.int32),
              src_x=np.zeros(0), src_y=np.zeros(0), src_z=np.zeros(0), src_ndot=np.zeros(0))
    return wl


@pytest.mark.parametrize("fp32", [0, 1])
def test_shared_bin_mixed_packet_against_the_oracle(fp32):
    """A packet of the shared bin holding photons of two cross-sections (the bin's own and twice
    it) moves down a chain: every deposit, the cross-section field and the budget match the
    oracle (FP64 to rounding, FP32 within 1e-5)."""
    wl = _shared_chain()
    g, o = _pair(wl, transport_fp32=fp32)
    assert g.nf == 1 and g.S == wl["params"]["n_rc"]
    g.assign_cones(0)
    g.emit(0)
    o.rotate(0)
    o.emit(0)
    N0, s0 = 1e50, wl["sigma"][0]
    d = np.array([1.0, 0.0, 0.0])
    b = oracle.recv_bin(o.rotations()[0][1].reshape(3, 3), oracle.axis_set(wl["params"]["n_rc"]), d)
    f = np.zeros((6, g.n, g.S))
    f[0, 1, b] = N0
    f[1:4, 1, b] = N0 * d
    G = np.zeros((g.n, wl["params"]["n_rc"]))
    G[1, b] = 0.25 * N0 * s0 + 0.75 * N0 * 2 * s0
    for c in (g, o):
        c.set_slots(f)
        c.set_shared_sigma(G)
    assert np.allclose(g.shared_sigma(), G, rtol=1e-6 if fp32 else 0, atol=0)
    g.transport(0)
    assert o.transport(0) == 0
    ag, ao = g.deposits()[0][:, 0], o.deposits()[0][:, 0]
    assert ao[2:-2].min() > 0
    assert np.allclose(ag, ao, rtol=1e-12 if not fp32 else 1e-5, atol=1e-6 * ao.max() if fp32 else 0)
    for c in (g, o):                 # the library folds the step's absorptions into the budget here
        c.chemistry()
    bg, bo = g.budget()[0], o.budget()[0]
    assert np.allclose(bg, bo, rtol=1e-6, atol=1e-6 * N0)


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("clock_limited", [False, True])
def test_shared_frequency_bin_against_the_oracle(fp32, clock_limited):
    """The HII region (1e5 K blackbody in 8 bins, 32 cones, T evolving) with the recombination
    photons in source bin 0, their cross-sections averaged on merge.  With clock-limited steps
    (c dt < box side) packets are held across steps and re-binned with their cross-section
    sums.  FP64: x_HI, T and the cross-section field of the held packets as the oracle's to
    rounding; FP32: x_HI and T within the bars; budgets within 1e-6."""
    kw = dict(dt=0.01 * W.MYR, dt_em=0.01 * W.MYR) if clock_limited else {}
    wl = W.cfg2(n_side=16, rec_shared_bin=1, **kw)
    g, o = _pair(wl, transport_fp32=fp32)
    affected = np.zeros(g.n, bool)
    for step in range(4):
        g.step(step)
        assert o.step(step) == 0
        _route_affected(g, o, wl["N_H"], affected)
    sg, so = g.state(), o.state()
    ok = _xhi_ok(sg["x_HI"], so["x_HI"])
    relT = np.abs(sg["T"] / so["T"] - 1)
    assert so["N_rec"].max() > 0
    if fp32 == 0:
        assert ok.all() and (relT < 1e-3).all()
        assert np.max(np.abs(sg["x_HI"] / so["x_HI"] - 1)) < 1e-9
        Gg, Go = g.shared_sigma(), o.shared_sigma()
        if clock_limited:
            assert np.count_nonzero(Go) > 1000
        assert np.allclose(Gg, Go, rtol=1e-9, atol=1e-9 * np.abs(Go).max())
    else:
        _assert_fp32_bars(sg, so, affected, 4)
    bg, bo = g.budget()[0], o.budget()[0]
    assert np.allclose(bg, bo, rtol=1e-6, atol=1e-6 * bo[0])
    assert abs(bg[0] - bg[1:].sum()) <= 1e-6 * bg[0]


def test_box_above_2_22_particles_uses_24_bit_keys():
    """A box of 2^22 + 1000 particles takes the kNN instances with 24 index bits: sampled
    neighbour lists equal brute force and a step conserves photons.  In a box that size, a
    particle whose 32nd neighbour lies across the box cannot be ordered by the keys and the
    neighbour build says so (RT_ERR_KNN); the same geometry in a small box, with 22 index bits,
    builds."""
    from paper_1311_0182_gb300 import rt
    n = (1 << 22) + 1000
    L = 13.2 * W.KPC
    rng = np.random.default_rng(9)
    pos = rng.uniform(0.0, L, size=(n, 3))
    params = W.default_params(seed=9, n_ec=8, n_tc=8, n_rc=8, dt=0.05 * W.MYR, dt_em=0.05 * W.MYR,
                              transport_fp32=1)
    wl = W._pack(params, [L], [0, n], pos, np.full(n, 1e-3), np.full(n, 1e-3 * L ** 3 / n),
                 np.full(n, 0.5), np.full(n, 1e4), [0], np.array([[0.5 * L] * 3]), [[1e50]],
                 [6.3e-18], [0.0])
    g = rt.context_for(wl)
    nbr, h2, _, _ = g.neighbours()
    q = g.quantised()
    idx = np.arange(n)
    for i in rng.choice(n, 12, replace=False):
        d2 = ((q - q[i]) ** 2).sum(1)
        d2[i] = np.iinfo(np.int64).max
        cand = np.nonzero(d2 <= np.partition(d2, 31)[31])[0]      # ties at the 32nd kept
        order = cand[np.lexsort((cand, d2[cand]))][:32]
        assert np.array_equal(nbr[i], order)
        assert h2[i] == d2[order[-1]]
    # the virtual particles' search with 24-bit keys, at points near particles
    pts = np.clip(q[rng.choice(n, 6, replace=False)] + rng.integers(-2000, 2000, (6, 3)), 0,
                  (1 << 20) - 1)
    got, gd2 = g.query_neighbours(0, pts)
    for p_, nb_ in zip(pts, got):
        d2 = ((q - p_) ** 2).sum(1)
        cand = np.nonzero(d2 <= np.partition(d2, 31)[31])[0]
        assert np.array_equal(nb_, cand[np.lexsort((cand, d2[cand]))][:32])
    g.step(0)
    b = g.budget()[0]
    assert g.stats()["virtual"] > 0 and abs(b[0] - b[1:].sum()) <= 1e-6 * b[0]
    g.close()
    # one particle alone in the far corner, the rest spread over the octant [0, 0.4 L)^3 (about
    # 15 times the mean density, so the cell grid stays usable): the far particle's 32nd
    # neighbour is more than a box side away
    far = np.full((1, 3), np.nextafter(L, 0.0))
    for m, expect_error in ((n, True), (2000, False)):
        p = np.concatenate([rng.uniform(0.0, 0.4 * L, size=(m - 1, 3)), far])
        w2 = W._pack(params, [L], [0, m], p, np.full(m, 1e-3), np.full(m, 1e-3 * L ** 3 / m),
                     np.full(m, 0.5), np.full(m, 1e4), [0], np.array([[0.2 * L] * 3]), [[1e50]],
                     [6.3e-18], [0.0])
        c = rt.Context(w2)
        c.load_workload(w2)
        if expect_error:
            with pytest.raises(rt.RTError) as e:
                c.build_neighbours()
            assert e.value.status == 5
        else:
            c.build_neighbours()
            assert c.neighbours()[1][-1] > (1 << 40)      # its 32nd neighbour is across the box
        c.close()


def test_invalid_inputs_are_refused_with_a_status():
    """Host-side fault injection: a NaN density, a negative atom count, x_HI above 1, a zero
    temperature, a NaN position, a negative photon rate or a zero cross-section is refused with
    RT_ERR_INVALID before any step uses it; the context then needs valid inputs again and works
    with them."""
    from paper_1311_0182_gb300 import rt
    wl = W.cfg1(n_side=12)
    g = rt.Context(wl)
    f = lambda k: np.ascontiguousarray(wl[k], dtype=np.float64)
    good = [f(k) for k in ("x", "y", "z", "n_H", "N_H", "x_HI", "T")]
    for k, val in ((3, np.nan), (4, -1.0), (5, 1.5), (6, 0.0), (0, np.nan)):
        bad = [a.copy() for a in good]
        bad[k][7] = val
        with pytest.raises(rt.RTError) as e:
            g.set_particles(*bad)
        assert e.value.status == 1, (k, val)
        with pytest.raises(rt.RTError) as e:        # no particles until a valid call
            g.build_neighbours()
        assert e.value.status == 7
    g.set_particles(*good)
    src = [np.ascontiguousarray(wl["src_box"], dtype=np.int32), f("src_x"), f("src_y"),
           f("src_z"), f("src_ndot"), f("sigma"), f("eps")]
    for k, val in ((4, -5e48), (5, 0.0)):
        bad = [a.copy() for a in src]
        bad[k][0] = val
        with pytest.raises(rt.RTError) as e:
            g.set_sources(*bad)
        assert e.value.status == 1, (k, val)
    g.set_sources(*src)
    g.build_neighbours()
    g.step(0)
    x = g.state()["x_HI"].copy()
    x[3] = -0.1
    with pytest.raises(rt.RTError) as e:
        g.set_state(x_HI=x)
    assert e.value.status == 1
    x[3] = 0.5
    g.set_state(x_HI=x)
    g.step(1)
    b = g.budget()[0]
    assert abs(b[0] - b[1:].sum()) <= 1e-9 * b[0]
