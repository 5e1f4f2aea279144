"""The per-cell candidate lists of the virtual particles' neighbour search, as a CPU model.

Sec. 2.1 gives a virtual particle the n_ngb gas particles nearest to it.  The library finds
them from a list built once per cell of its kNN grid; this model builds the same lists in plain
numpy (exact integers, quantised positions) and runs the same early-exit scan, and the tests
check it against brute force.  What the model pins is the argument, not the CUDA code:
- U, the largest distance from any point of the cell to any of the n_ngb nearest particles of
  the cell's centre point, bounds the n_ngb-th neighbour distance of every point of the cell;
- so every particle that can be among the n_ngb nearest of a point of the cell lies within U
  of the cell;
- a particle p whose ring r = floor(|p - m| / w) is at least r w - |q - m| from a query q, so
  once that exceeds the running n_ngb-th distance the rest of the ring-ordered list can be
  skipped.
(The library also gives cells deep in voids no list and answers there by its grid walk; the
GPU tests cover that.)
"""
import math

import numpy as np
import pytest

Q = 1 << 20


def brute(q, p, k):
    """(d2, index) of the k nearest points of q, ties to the lower index."""
    d2 = ((q - p[None, :]) ** 2).sum(1) if p.ndim == 1 else ((q - p) ** 2).sum(1)
    order = np.lexsort((np.arange(len(q)), d2))[:k]
    return d2[order], order


def build_lists(q, G, kn):
    cs = -(-Q // G)
    w = cs >> 4 if cs >= 32 else 1
    lists = {}
    for cx in range(G):
        for cy in range(G):
            for cz in range(G):
                lo = np.array([cx, cy, cz], dtype=np.int64) * cs
                hi = lo + cs - 1
                m = np.minimum(lo + cs // 2, Q - 1)
                _, nn = brute(q, m, kn)
                far = np.maximum(q[nn] - lo, hi - q[nn])
                u2 = int((far ** 2).sum(1).max())
                gap = np.where(q < lo, lo - q, np.where(q > hi, q - hi, 0))
                cand = np.nonzero((gap ** 2).sum(1) <= u2)[0]
                dm2 = ((q[cand] - m) ** 2).sum(1)
                ring = np.minimum(np.floor(np.sqrt(dm2.astype(float)) / w).astype(np.int64), 255)
                while True:   # ring * w <= |p - m| exactly
                    over = (ring * w) ** 2 > dm2
                    if not over.any():
                        break
                    ring[over] -= 1
                order = np.argsort(ring, kind="stable")
                lists[(cx, cy, cz)] = (cand[order], ring[order], m)
    return lists, cs, w


def query(x, q, lists, cs, w, G, kn):
    """The ring-ordered scan of the query's cell, 32 entries at a time; returns the (d2,
    index) keys of the result and the number of entries scanned."""
    c = tuple(int(v) for v in np.minimum(x // cs, G - 1))
    cand, ring, m = lists[c]
    rq = math.sqrt(float(((x - m) ** 2).sum()))
    best = []
    scanned = 0
    for b in range(0, len(cand), 32):
        if len(best) >= kn:
            if ring[b] * w - rq > math.sqrt(best[kn - 1][0]):
                break
        ids = cand[b:b + 32]
        d2 = ((q[ids] - x) ** 2).sum(1)
        best = sorted(best + list(zip(d2.tolist(), ids.tolist())))[:kn]
        scanned += len(ids)
    return best, scanned


def uniform(n, rng):
    return rng.integers(0, Q, size=(n, 3))


def lattice(side):
    g = (np.arange(side) * (Q // side) + Q // (2 * side)).astype(np.int64)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


def clustered(n, rng):
    c = rng.integers(Q // 5, 4 * Q // 5, size=(3, 3))
    p = c[rng.integers(0, 3, n)] + rng.normal(0, Q / 20, size=(n, 3)).astype(np.int64)
    p = np.clip(p, 0, Q - 1)
    p[10:30] = p[9]                 # duplicate positions
    return p


@pytest.mark.parametrize("name,occ", [("uniform", 1), ("uniform", 3), ("lattice", 2),
                                      ("clustered", 2)])
def test_candidate_lists_give_the_exact_nearest_neighbours(name, occ):
    rng = np.random.default_rng(7)
    q = {"uniform": lambda: uniform(2000, rng), "lattice": lambda: lattice(12),
         "clustered": lambda: clustered(2000, rng)}[name]()
    kn = 32
    G = max(1, int(round((len(q) / occ) ** (1 / 3))))
    lists, cs, w = build_lists(q, G, kn)
    pts = np.concatenate([
        np.clip(q[rng.integers(0, len(q), 150)] + rng.integers(-cs, cs, (150, 3)), 0, Q - 1),
        q[rng.integers(0, len(q), 20)],                                   # on particles
        np.array([[a, b, c] for a in (0, Q - 1) for b in (0, Q - 1) for c in (0, Q - 1)]),
        (rng.integers(0, G, (20, 3)) * cs).astype(np.int64)])            # cell corners
    scanned, lengths = [], []
    for x in pts:
        got, n_scan = query(x, q, lists, cs, w, G, kn)
        d2, order = brute(q, x, kn)
        assert [i for _, i in got] == order.tolist(), (name, occ, x)
        assert [d for d, _ in got] == d2.tolist()
        c = tuple(int(v) for v in np.minimum(x // cs, G - 1))
        scanned.append(n_scan)
        lengths.append(len(lists[c][0]))
    if name == "uniform":
        # the early exit skips part of the lists
        assert np.mean(scanned) < 0.8 * np.mean(lengths)


def test_the_bound_holds_for_any_n_ngb_particles():
    """Any n_ngb particles bound a cell, not only the nearest of its centre: lists built from a
    worse set are longer but still hold every query's n_ngb nearest."""
    rng = np.random.default_rng(3)
    q = uniform(1500, rng)
    kn, G = 16, 8
    cs = -(-Q // G)
    for _ in range(40):
        cx, cy, cz = rng.integers(0, G, 3)
        lo = np.array([cx, cy, cz], dtype=np.int64) * cs
        hi = lo + cs - 1
        some = rng.choice(len(q), kn, replace=False)             # not the nearest
        far = np.maximum(q[some] - lo, hi - q[some])
        u2 = int((far ** 2).sum(1).max())
        gap = np.where(q < lo, lo - q, np.where(q > hi, q - hi, 0))
        inside = set(np.nonzero((gap ** 2).sum(1) <= u2)[0].tolist())
        for x in lo + rng.integers(0, cs, (5, 3)):
            _, order = brute(q, np.minimum(x, Q - 1), kn)
            assert set(order.tolist()) <= inside
