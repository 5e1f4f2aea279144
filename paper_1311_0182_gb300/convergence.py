"""App. A convergence runs: the Stromgren sphere with transported recombination radiation.

The HII region of Sec. 3 (workload 1 geometry: 13.2 kpc box, n_H = 1e-3, T = 1e4 K, a 5e48
s^-1 source at 13.6 eV) is run on the GPU to a given multiple of t_rec with a chosen particle
count, RT time step (emission step 0.1 dt, as in App. A) and number of transmission cones
(N_EC = N_RC = 8).  The result is the radial profile, in shells of R_S/8, of the neutral
fraction, of the recombination-radiation intensity (the photons of the recombination bin
passing each gas particle per step over its smoothing area: a per-area form of the paper's
diagnostic, which records the photons passing each SPH particle per step, Sec. 3) and of the
diffuse-to-source ratio of those counts.  Photons carried by virtual particles pass no gas
particle and are not counted, so the intensity drops as narrow cones (large N_TC) send more
photons through virtual particles.

    python -m paper_1311_0182_gb300.convergence [t/t_rec] [--quick]   # one JSON line per run
"""
from __future__ import annotations

import json
import math
import sys

import numpy as np

from . import workloads as W

T_REC_MYR = 122.4            # Sec. 3: t_rec = 1 / (alpha_B n_H) at n_H = 1e-3, T = 1e4 K
R_S_KPC = 5.4                 # the case-B Stromgren radius of the set-up


def run(n_side: int = 32, dt_myr: float = 1.0, n_tc: int = 8, t_rec: float = 4.0,
        transport_fp32: int = 1, stream=None) -> dict:
    from . import rt
    dt = dt_myr * W.MYR
    # narrow transmission cones leave most cones empty: room for one virtual particle per
    # (particle, reception cone) and per extra factor of 8 in the cone count
    free_cap = n_side ** 3 * 8 * max(1, n_tc // 8)
    wl = W.cfg1(n_side=n_side, dt=dt, dt_em=0.1 * dt, n_tc=n_tc, rec_mode=W.REC_TRANSPORT,
                transport_fp32=transport_fp32, free_cap=free_cap)
    ctx = rt.context_for(wl, stream=stream)
    steps = int(round(t_rec * T_REC_MYR / dt_myr))
    for s in range(steps):
        ctx.step(s)
    L = float(wl["box_L"][0])
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    r = np.linalg.norm(pos - 0.5 * L, axis=1) / (R_S_KPC * W.KPC)
    x = ctx.state()["x_HI"]
    _, _, pas = ctx.deposits()
    _, h2, _, _ = ctx.neighbours()
    h = np.sqrt(h2.astype(np.float64)) * L / (1 << 20)
    inten = pas[:, -1] / (dt * math.pi * h ** 2)      # recombination bin, per area and time
    edges = np.arange(0.0, 1.6001, 0.125)
    prof = []
    for a, b in zip(edges[:-1], edges[1:]):
        m = (r >= a) & (r < b)
        if m.any():
            # diffuse-to-source ratio: photons of the recombination bin over those of the
            # source bins passing the shell's particles (Sec. 3)
            src = float(pas[m, :-1].sum())
            prof.append({"r_over_RS": [float(a), float(b)], "x_HI": float(x[m].mean()),
                         "intensity": float(inten[m].mean()),
                         "diffuse_to_source": float(pas[m, -1].sum()) / src if src > 0 else None})
    # front: where the shell-averaged x_HI crosses 0.5
    front = None
    for p, q in zip(prof[:-1], prof[1:]):
        if p["x_HI"] < 0.5 <= q["x_HI"]:
            ra, rb = 0.5 * sum(p["r_over_RS"]), 0.5 * sum(q["r_over_RS"])
            front = ra + (0.5 - p["x_HI"]) / (q["x_HI"] - p["x_HI"]) * (rb - ra)
            break
    ctx.close()
    return {"n_side": n_side, "dt_myr": dt_myr, "n_tc": n_tc, "t_over_trec": t_rec,
            "steps": steps, "front_over_RS": front,
            "mean_h_over_RS": float(h.mean() / (R_S_KPC * W.KPC)), "profile": prof}


# the App. A sweeps: resolution at dt = 0.1 Myr, time step at 64^3, cones at 64^3
SWEEPS = ([dict(n_side=n, dt_myr=0.1) for n in (32, 64, 128)] +
          [dict(n_side=64, dt_myr=d) for d in (0.01, 1.0)] +
          [dict(n_side=64, dt_myr=0.1, n_tc=c) for c in (64, 128)])
# the same three questions at a cost of minutes: resolution at dt = 1 Myr, time step and cones
# at 32^3
SWEEPS_QUICK = ([dict(n_side=n, dt_myr=1.0) for n in (32, 64, 128)] +
                [dict(n_side=32, dt_myr=d) for d in (0.01, 0.1)] +
                [dict(n_side=32, dt_myr=1.0, n_tc=c) for c in (64, 128)])


def main(argv=None):
    """python -m paper_1311_0182_gb300.convergence [t / t_rec] [--quick]"""
    argv = sys.argv[1:] if argv is None else argv
    quick = "--quick" in argv
    nums = [a for a in argv if not a.startswith("--")]
    t_rec = float(nums[0]) if nums else 4.0
    for kw in (SWEEPS_QUICK if quick else SWEEPS):
        print(json.dumps(run(t_rec=t_rec, **kw)), flush=True)


if __name__ == "__main__":
    main()
