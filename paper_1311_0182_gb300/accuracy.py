"""Accuracy bars of the transport sweep against an FP64 reference, and the routing-flip count of
the FP32 transport.

Bars (per particle): x_HI within 1e-3 relative, or 1e-7 absolute where the reference x_HI is
below 1e-4; T within 1e-3 relative.

Routing flips.  The FP32 transport takes every discrete decision of Sec. 2.1 (is a neighbour in
the transmission cone, which reception cone receives a packet, where a virtual particle lands)
exactly, on its FP32 packet direction.  That direction differs from the FP64 one in the last
bits, so a decision whose margin is smaller than that difference goes the other way, and the
share of the packet concerned takes another route from then on.  FP32 arithmetic moves a
particle's absorbed photons by about 1e-6 of themselves; a change above ROUTE_TOL within one step
needs such a changed decision upstream.  A particle whose absorbed photons and energy stay within
ROUTE_TOL of the reference's in every step is held to the bars; the others are counted as
routing-affected, against FLIP_BUDGET per compared step (a fraction of all particles; the count
is the union over the steps compared, so it grows with them).  Two absolute floors keep
differences that cannot move the state out of the count: 1e-12 photons per atom, and 1e-8 eV per
atom (a temperature change below 1e-4 K; the fixed-point energy words count in units of 2^-36 eV
per neutral atom, whose rounding over many deposits reaches ~1e-9 eV per atom).
"""
from __future__ import annotations

import numpy as np

X_REL, X_ABS, X_SMALL, T_REL = 1e-3, 1e-7, 1e-4, 1e-3
ROUTE_TOL = 1e-3
FLIP_BUDGET = 0.0025          # routing-affected particles per compared step, fraction of all
FLOOR_PHOTONS_PER_ATOM = 1e-12
FLOOR_EV_PER_ATOM = 1e-8
EV = 1.602176634e-12


def xhi_ok(x, x_ref):
    """Per particle: x_HI within the bar of the reference value."""
    x, x_ref = np.asarray(x), np.asarray(x_ref)
    rel = np.abs(x - x_ref) / np.maximum(np.abs(x_ref), 1e-300)
    return np.where(x_ref < X_SMALL, np.abs(x - x_ref) <= X_ABS, rel <= X_REL)


def state_ok(s, s_ref):
    """Per particle: x_HI and T both within their bars."""
    return xhi_ok(s["x_HI"], s_ref["x_HI"]) & (np.abs(s["T"] / s_ref["T"] - 1) < T_REL)


def mark_routing_affected(A, A_ref, E, E_ref, NH, affected):
    """Mark (in place, and return) the particles whose absorbed photons A or energy E (erg) of
    one step differ from the reference's by more than ROUTE_TOL relative plus the floors."""
    A, A_ref, E, E_ref, NH = (np.asarray(v, dtype=np.float64) for v in (A, A_ref, E, E_ref, NH))
    affected |= np.abs(A - A_ref) > ROUTE_TOL * np.abs(A_ref) + FLOOR_PHOTONS_PER_ATOM * NH
    affected |= np.abs(E - E_ref) > ROUTE_TOL * np.abs(E_ref) + FLOOR_EV_PER_ATOM * EV * NH
    return affected


def flip_budget(n: int, steps: int) -> float:
    """Routing-affected particles allowed after `steps` compared steps of n particles."""
    return FLIP_BUDGET * n * steps


def summary(s, s_ref, affected, steps=1) -> dict:
    """Counts and largest relative errors, for all particles and for those not
    routing-affected."""
    relx = np.abs(np.asarray(s["x_HI"]) / np.asarray(s_ref["x_HI"]) - 1)
    relT = np.abs(np.asarray(s["T"]) / np.asarray(s_ref["T"]) - 1)
    ok = state_ok(s, s_ref)
    keep = ~affected
    n = len(ok)
    return {"particles": n, "routing_affected": int(affected.sum()),
            "routing_affected_frac": float(affected.sum()) / max(n, 1),
            "flip_budget_frac_per_step": FLIP_BUDGET,
            "within_flip_budget": bool(affected.sum() <= flip_budget(n, steps)),
            "off_bars": int((~ok).sum()), "off_bars_not_affected": int((~ok & keep).sum()),
            "max_rel_all": {"x_HI": float(relx.max(initial=0.0)), "T": float(relT.max(initial=0.0))},
            "max_rel_not_affected": {"x_HI": float(relx[keep].max(initial=0.0)),
                                     "T": float(relT[keep].max(initial=0.0))}}
