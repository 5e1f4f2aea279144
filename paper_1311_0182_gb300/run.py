"""Run a workload for a number of RT steps and log one JSON line per step.

    python -m paper_1311_0182_gb300.run cfg2 --steps 20 [--n-side 32] [--fp64] [--profile-every 10]
                                        [--checkpoint-every 10 --checkpoint-dir DIR] [--resume FILE]
                                        [--host-loop]

Each line holds the step, the simulated time, the wall time of the step, the hop and virtual-
particle counts, the photon budget (emitted, absorbed, escaped, in flight; Sec. 2.1: photon
conservation) with its closure, the ionised volume fraction and the I-front radius around the
first source (Sec. 3 follows the front of the HII region), and every --profile-every steps the
radial profiles of x_HI and T in shells of 1/32 of the box side.  Checkpoints go through
rt_save_state; --resume restores one and continues from the step it was taken after.
--host-loop drives the hop loop from the host (rt_set_graph off), so that every kernel of a step
is a launch of its own (a profiler sees kernel nodes under the step graph's conditional node
only as the graph launch).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import workloads as W


def ionised_fraction(x_HI, n_H, N_H) -> float:
    """Volume-weighted fraction of the gas with x_HI < 0.5 (particle volume N_H / n_H)."""
    v = np.asarray(N_H) / np.asarray(n_H)
    return float(v[np.asarray(x_HI) < 0.5].sum() / v.sum())


def radial_profile(r, values, r_max, n_shells=32):
    """Mean of `values` in n_shells equal shells of [0, r_max); empty shells give None."""
    edges = np.linspace(0.0, r_max, n_shells + 1)
    idx = np.searchsorted(edges, r, side="right") - 1
    out = []
    for k in range(n_shells):
        m = idx == k
        out.append(float(np.mean(values[m])) if m.any() else None)
    return edges, out


def cylindrical_profiles(pos, axis_point, axis: int, height, r_max: float, n_shells: int,
                         fields: dict) -> dict:
    """Means of each field in `fields` (per-particle arrays) over concentric cylindrical shells
    around the line through axis_point along coordinate `axis`, out to r_max, for particles
    whose coordinate along the axis lies in height = (lo, hi): the shells in which Sec. 4
    averages the intensities, neutral fractions and temperatures of the shadow region behind
    the barrier.  Returns the shell edges, the particle counts and, per field, the shell means
    (None for empty shells)."""
    pos = np.asarray(pos, dtype=np.float64)
    c = np.asarray(axis_point, dtype=np.float64)
    perp = [a for a in range(3) if a != axis]
    rc = np.sqrt(((pos[:, perp] - c[perp]) ** 2).sum(1))
    inside = (pos[:, axis] >= height[0]) & (pos[:, axis] < height[1])
    edges = np.linspace(0.0, r_max, n_shells + 1)
    idx = np.searchsorted(edges, rc, side="right") - 1
    out = {"edges": edges.tolist(), "count": [], **{k: [] for k in fields}}
    for k in range(n_shells):
        m = inside & (idx == k)
        out["count"].append(int(m.sum()))
        for name, v in fields.items():
            out[name].append(float(np.mean(np.asarray(v)[m])) if m.any() else None)
    return out


def shadow_profiles(wl: dict, state: dict, passing, dt: float, n_shells=10) -> dict:
    """The diagnostic of Sec. 4 for the shadow workload: cylindrical shells around the shadow's
    major axis (the line through the barrier's centre along x) out to half the box side, over
    the part of the box behind the barrier from 0.35 to 0.75 of the side; per shell the mean
    x_HI, T and intensity of the source photons (bin 0) and of the diffuse photons (every other
    bin: the boundary emitters and the transported recombination photons), each intensity in
    units of the source intensity of the outermost shell (photons passing a particle per
    step, Sec. 3 and Sec. 4)."""
    L = float(wl["box_L"][0])
    b, axis, centre, radius = wl["barriers"][0]
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    box0 = slice(int(wl["box_off"][0]), int(wl["box_off"][1]))
    pas = np.asarray(passing)[box0] / dt
    prof = cylindrical_profiles(pos[box0], centre, axis, (0.35 * L, 0.75 * L), 0.5 * L, n_shells,
                                {"x_HI": state["x_HI"][box0], "T": state["T"][box0],
                                 "I_source": pas[:, 0], "I_diffuse": pas[:, 1:].sum(1)})
    ref = prof["I_source"][-1]
    for k in ("I_source", "I_diffuse"):
        prof[k] = [None if v is None or not ref else v / ref for v in prof[k]]
    prof["barrier_radius"] = float(radius)
    return prof


def front_radius(r, x_HI, r_max, n_shells=32):
    """Radius where the shell-mean x_HI first crosses 0.5 going outwards (linear between shell
    centres); None when no shell crosses."""
    edges, prof = radial_profile(r, np.asarray(x_HI), r_max, n_shells)
    centres = 0.5 * (edges[:-1] + edges[1:])
    pts = [(c, p) for c, p in zip(centres, prof) if p is not None]
    for (ra, xa), (rb, xb) in zip(pts[:-1], pts[1:]):
        if xa < 0.5 <= xb:
            return float(ra + (0.5 - xa) / (xb - xa) * (rb - ra))
    return None


def _workload(name, args):
    make = {"cfg1": W.cfg1, "cfg2": W.cfg2, "cfg3": W.cfg3, "cfg4": W.cfg4, "cfg5": W.cfg5,
            "shadow": W.shadow}[name]
    kw = {"transport_fp32": 0 if args.fp64 else 1}
    if args.n_side and name in ("cfg1", "cfg2", "cfg3", "cfg5", "shadow"):
        kw["n_side"] = args.n_side
    return make(**kw)


def run(wl, steps, start=0, ctx=None, profile_every=0, checkpoint_every=0, checkpoint_dir=None,
        out=sys.stdout):
    """Advance the workload `steps` steps from step `start`, printing one JSON line per step;
    returns the context."""
    from . import rt
    if ctx is None:
        ctx = rt.context_for(wl)
    L = float(wl["box_L"][0])
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    box0 = slice(int(wl["box_off"][0]), int(wl["box_off"][1]))
    src = (np.array([wl["src_x"][0], wl["src_y"][0], wl["src_z"][0]])
           if len(wl["src_box"]) else np.full(3, 0.5 * L))
    r = np.linalg.norm(pos[box0] - src, axis=1)
    dt_myr = wl["params"]["dt"] / W.MYR
    for s in range(start, start + steps):
        t0 = time.perf_counter()
        ctx.step(s)
        st = ctx.state()
        ms = (time.perf_counter() - t0) * 1e3
        b = ctx.budget()
        stats = ctx.stats()
        x = st["x_HI"]
        line = {"step": s, "t_myr": (s + 1) * dt_myr, "ms": ms, "hops": stats["hops"],
                "virtual": stats["virtual"],
                "budget": {"emitted": float(b[:, 0].sum()), "absorbed": float(b[:, 1].sum()),
                           "escaped": float(b[:, 2].sum()), "in_flight": float(b[:, 3].sum())},
                "closure": float(np.max(np.abs(b[:, 0] - b[:, 1:].sum(1)) /
                                        np.maximum(b[:, 0], 1e-300))),
                "ionised_volume_fraction": ionised_fraction(x, wl["n_H"], wl["N_H"]),
                "front_kpc": (lambda f: None if f is None else f / W.KPC)(
                    front_radius(r, x[box0], 0.5 * L))}
        if profile_every and (s + 1) % profile_every == 0:
            edges, px = radial_profile(r, x[box0], 0.5 * L)
            _, pT = radial_profile(r, st["T"][box0], 0.5 * L)
            line["profile"] = {"r_kpc": (edges / W.KPC).tolist(), "x_HI": px, "T": pT}
            if wl.get("barriers"):
                line["shadow"] = shadow_profiles(wl, st, ctx.deposits()[2], wl["params"]["dt"])
        if checkpoint_every and checkpoint_dir and (s + 1) % checkpoint_every == 0:
            path = os.path.join(checkpoint_dir, f"step{s:06d}.ckpt")
            with open(path, "wb") as f:
                f.write(ctx.save_state())
            line["checkpoint"] = path
        print(json.dumps(line), file=out, flush=True)
    return ctx


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("workload", choices=["cfg1", "cfg2", "cfg3", "cfg4", "cfg5", "shadow"])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--n-side", type=int, default=0)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--profile-every", type=int, default=0)
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--checkpoint-dir", default=None)
    ap.add_argument("--resume", default=None, help="checkpoint file step<N>.ckpt to continue from")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the hop loop from the host: one launch per kernel and hop")
    args = ap.parse_args(argv)
    wl = _workload(args.workload, args)
    from . import rt
    ctx = rt.context_for(wl)
    if args.host_loop:
        ctx.set_graph(False)
    start = 0
    if args.resume:
        with open(args.resume, "rb") as f:
            ctx.load_state(f.read())
        start = int(os.path.basename(args.resume)[4:10]) + 1
    if args.checkpoint_dir:
        os.makedirs(args.checkpoint_dir, exist_ok=True)
    run(wl, args.steps, start=start, ctx=ctx, profile_every=args.profile_every,
        checkpoint_every=args.checkpoint_every, checkpoint_dir=args.checkpoint_dir)


if __name__ == "__main__":
    main()
