"""Plain FP64 CPU oracle of one TRAPHIC step (Raicevic et al., Sec. 2) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It wraps ``traphic_oracle.c`` (plain C, compiled with ``-ffp-contract=off``) through
ctypes; it shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtraphic_oracle.so")
_SRC = os.path.join(_HERE, "traphic_oracle.c")
_lock = threading.Lock()
_lib = None

REC_TRANSPORT, REC_OTS_CASE_B, REC_CASE_A = 0, 1, 2
COOL_REC, COOL_CEX, COOL_CION, COOL_FF = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "traphic_oracle.h"))
    ):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Config(C.Structure):
    _fields_ = [
        ("n_ngb", C.c_int), ("n_ec", C.c_int), ("n_tc", C.c_int), ("n_rc", C.c_int),
        ("n_freq_src", C.c_int), ("dt", C.c_double), ("dt_em", C.c_double),
        ("rec_mode", C.c_int), ("evolve_T", C.c_int), ("seed", C.c_uint64),
        ("hop_cap", C.c_int), ("sub_cap", C.c_int), ("cool_flags", C.c_int),
        ("T_floor", C.c_double), ("eps_rr_fixed", C.c_double), ("sigma_rec", C.c_double),
        ("rec_shared_bin", C.c_int),
    ]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i32, i64, u32 = C.c_double, C.c_int32, C.c_int64, C.c_uint32
            P = C.POINTER
            L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            L.orc_mix64.argtypes = [C.c_uint64]
            L.orc_mix64.restype = C.c_uint64
            L.orc_axis_set.argtypes = [C.c_int, P(d)]
            L.orc_rotation.argtypes = [C.c_uint64, u32, u32, u32, u32, P(d)]
            L.orc_in_cone.argtypes = [P(i64), P(d), C.c_int]
            L.orc_virtual_offset.argtypes = [C.c_uint64, C.c_longlong, C.c_int, C.c_uint64, i64,
                                             P(d), C.c_int, P(i64)]
            L.orc_virtual_offset.restype = None
            L.orc_bin.argtypes = [P(d), P(d), C.c_int, P(d)]
            L.orc_rates.argtypes = [d, P(d)]
            L.orc_chem_particle.argtypes = [P(Config), d, d, d, d, P(d), P(d), P(d)]
            L.orc_knn.argtypes = [C.c_longlong, P(i64), C.c_longlong, P(i64), C.c_longlong,
                                  C.c_int, C.c_int, P(i32), P(i64)]
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [P(Config), C.c_int, P(C.c_longlong), P(d), P(d), P(d), P(d),
                                     P(d), P(d), P(d), P(d), C.c_int, P(C.c_int), P(d), P(d),
                                     P(d), P(d), P(d), P(d)]
            vp = C.c_void_p
            L.orc_destroy.argtypes = [vp]
            L.orc_build_neighbours.argtypes = [vp]
            L.orc_get_neighbours.argtypes = [vp, P(i32), P(i64), P(i32), P(i64)]
            L.orc_get_quantised.argtypes = [vp, P(i64)]
            L.orc_rotate.argtypes = [vp, C.c_longlong]
            L.orc_get_rotations.argtypes = [vp, P(d), P(d)]
            L.orc_rebin.argtypes = [vp]
            L.orc_emit.argtypes = [vp, C.c_longlong]
            L.orc_transport.argtypes = [vp, C.c_longlong]
            L.orc_chemistry.argtypes = [vp]
            L.orc_step.argtypes = [vp, C.c_longlong]
            L.orc_cone_masks.argtypes = [vp, P(u32)]
            L.orc_set_identities.argtypes = [vp, P(C.c_longlong), P(C.c_longlong)]
            L.orc_cone_masks_dir.argtypes = [vp, P(d), P(u32)]
            L.orc_get_slots.argtypes = [vp, P(d)]
            L.orc_set_slots.argtypes = [vp, P(d)]
            L.orc_get_shared_sigma.argtypes = [vp, P(d)]
            L.orc_set_shared_sigma.argtypes = [vp, P(d)]
            L.orc_get_state.argtypes = [vp, P(d), P(d), P(d), P(d)]
            L.orc_set_state.argtypes = [vp, P(d), P(d), P(d), P(d)]
            L.orc_get_deposits.argtypes = [vp, P(d), P(d), P(d)]
            L.orc_get_budget.argtypes = [vp, P(d)]
            L.orc_get_stats.argtypes = [vp, P(C.c_longlong)]
            L.orc_set_source_options.argtypes = [vp, P(d), P(C.c_int)]
            L.orc_set_barrier.argtypes = [vp, C.c_int, C.c_int, P(d), d]
            L.orc_barrier_test.argtypes = [P(i64), P(i64), C.c_int, i64, i64, i64, i64]
            _lib = L
    return _lib


def make_config(p: dict) -> Config:
    """Oracle configuration from the workload parameter dictionary."""
    return Config(
        n_ngb=p["n_ngb"], n_ec=p["n_ec"], n_tc=p["n_tc"], n_rc=p["n_rc"],
        n_freq_src=p["n_freq_src"], dt=p["dt"], dt_em=p["dt_em"], rec_mode=p["rec_mode"],
        evolve_T=p["evolve_T"], seed=p["seed"], hop_cap=p["hop_cap"], sub_cap=p["sub_cap"],
        cool_flags=p["cool_flags"], T_floor=p["T_floor"], eps_rr_fixed=p["eps_rr_fixed"],
        sigma_rec=p["sigma_rec"], rec_shared_bin=p.get("rec_shared_bin", 0))


# --- building blocks ----------------------------------------------------------------------
def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def mix64(z: int) -> int:
    return int(lib().orc_mix64(C.c_uint64(z)))


def axis_set(n: int) -> np.ndarray:
    out = np.zeros((n, 3))
    if lib().orc_axis_set(n, _p(out, C.c_double)) != 0:
        raise ValueError(f"no axis set with {n} directions")
    return out


def rotation(seed, purpose, c0, c1, c2) -> np.ndarray:
    R = np.zeros(9)
    lib().orc_rotation(seed, purpose, c0, c1, c2, _p(R, C.c_double))
    return R.reshape(3, 3)


def in_cone(delta, d, n_tc) -> bool:
    dl = np.ascontiguousarray(delta, dtype=np.int64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    return bool(lib().orc_in_cone(_p(dl, C.c_int64), _p(dd, C.c_double), n_tc))


def virtual_offset(seed, step, hop, fid, h2, d, n_tc) -> np.ndarray:
    """Integer offset of a virtual particle from its sender."""
    out = np.zeros(3, np.int64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    lib().orc_virtual_offset(seed, step, hop, fid, h2, _p(dd, C.c_double), n_tc,
                             _p(out, C.c_int64))
    return out


def recv_bin(R, axes, d) -> int:
    Rr = np.ascontiguousarray(R, dtype=np.float64).reshape(9)
    ax = np.ascontiguousarray(axes, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    return int(lib().orc_bin(_p(Rr, C.c_double), _p(ax, C.c_double), ax.shape[0],
                             _p(dd, C.c_double)))


def rates(T: float) -> dict:
    out = np.zeros(8)
    lib().orc_rates(float(T), _p(out, C.c_double))
    keys = ["alpha_A", "alpha_B", "beta", "Lrec_A", "Lrec_B", "L_cex", "L_cion", "L_ff"]
    return dict(zip(keys, out.tolist()))


def chem_particle(params: dict, nH, NH, phot, heat, x, T):
    cfg = make_config(params)
    xx = np.array([x], float)
    TT = np.array([T], float)
    out = np.zeros(3)
    lib().orc_chem_particle(C.byref(cfg), nH, NH, phot, heat, _p(xx, C.c_double),
                            _p(TT, C.c_double), _p(out, C.c_double))
    return float(xx[0]), float(TT[0]), float(out[0]), int(out[1]), int(out[2])


def knn(pts, qpts, k, self_offset=-1, use_grid=True):
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    qpts = np.ascontiguousarray(qpts, dtype=np.int64)
    nq = qpts.shape[0]
    idx = np.zeros((nq, k), np.int32)
    d2 = np.zeros((nq, k), np.int64)
    rc = lib().orc_knn(pts.shape[0], _p(pts, C.c_int64), nq, _p(qpts, C.c_int64), self_offset,
                       k, int(use_grid), _p(idx, C.c_int32), _p(d2, C.c_int64))
    if rc != 0:
        raise ValueError("orc_knn failed")
    return idx, d2


def barrier_test(a, b, axis, p2, c1, c2, r2) -> bool:
    aa = np.ascontiguousarray(a, dtype=np.int64)
    bb = np.ascontiguousarray(b, dtype=np.int64)
    return bool(lib().orc_barrier_test(_p(aa, C.c_int64), _p(bb, C.c_int64), axis, p2, c1, c2, r2))


# --- the simulation --------------------------------------------------------------------------
class Sim:
    """One oracle simulation over the particles and sources of a workload dictionary."""

    def __init__(self, wl: dict):
        self.L = lib()
        p = wl["params"]
        self.params = p
        self.cfg = make_config(p)
        self.n = int(wl["box_off"][-1])
        self.nb = len(wl["box_L"])
        # a shared bin (Sec. 2.2) carries the recombination photons in source bin 0
        self.nf = p["n_freq_src"] + (0 if p.get("rec_shared_bin", 0) else 1)
        self.S = self.nf * p["n_rc"]
        self.K = max(1, int(round(p["dt"] / p["dt_em"])))
        self.ns = len(wl["src_box"])
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a

        box_off = arr(wl["box_off"], np.int64)
        box_L = arr(wl["box_L"], np.float64)
        x, y, z = (arr(wl[k], np.float64) for k in ("x", "y", "z"))
        nH, NH, xHI, T = (arr(wl[k], np.float64) for k in ("n_H", "N_H", "x_HI", "T"))
        sbox = arr(wl["src_box"], np.int32)
        sx, sy, sz = (arr(wl[k], np.float64) for k in ("src_x", "src_y", "src_z"))
        ndot = arr(wl["src_ndot"], np.float64)
        sig = arr(wl["sigma"], np.float64)
        eps = arr(wl["eps"], np.float64)
        d = C.c_double
        self.h = self.L.orc_create(
            C.byref(self.cfg), self.nb, _p(box_off, C.c_longlong), _p(box_L, d), _p(x, d),
            _p(y, d), _p(z, d), _p(nH, d), _p(NH, d), _p(xHI, d), _p(T, d), self.ns,
            _p(sbox, C.c_int), _p(sx, d), _p(sy, d), _p(sz, d), _p(ndot, d), _p(sig, d),
            _p(eps, d))
        if not self.h:
            raise ValueError("orc_create rejected the configuration")
        # optional: directed / gated sources and photon barriers (Sec. 4 set-up)
        if "src_dir" in wl or "src_gate" in wl:
            sd = arr(wl.get("src_dir", np.zeros((self.ns, 3))), np.float64)
            sg = arr(wl.get("src_gate", np.zeros(self.ns)), np.int32)
            self.L.orc_set_source_options(self.h, _p(sd, d), _p(sg, C.c_int))
        for (b, axis, centre, radius) in wl.get("barriers", []):
            c = arr(centre, np.float64)
            self.L.orc_set_barrier(self.h, int(b), int(axis), _p(c, d), float(radius))
        # optional: the identities of boxes and sources cut out of a larger workload
        if "box_first_id" in wl or "src_id" in wl:
            bf = arr(wl["box_first_id"], np.int64) if "box_first_id" in wl else None
            si = arr(wl["src_id"], np.int64) if "src_id" in wl else None
            self.L.orc_set_identities(self.h, None if bf is None else _p(bf, C.c_longlong),
                                      None if si is None else _p(si, C.c_longlong))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    def build_neighbours(self):
        rc = self.L.orc_build_neighbours(self.h)
        if rc != 0:
            raise ValueError(f"orc_build_neighbours status {rc}")

    def neighbours(self):
        k = self.params["n_ngb"]
        nbr = np.zeros((self.n, k), np.int32)
        h2 = np.zeros(self.n, np.int64)
        snbr = np.zeros((max(self.ns, 1), k), np.int32)
        sh2 = np.zeros(max(self.ns, 1), np.int64)
        self.L.orc_get_neighbours(self.h, _p(nbr, C.c_int32), _p(h2, C.c_int64),
                                  _p(snbr, C.c_int32), _p(sh2, C.c_int64))
        return nbr, h2, snbr[: self.ns], sh2[: self.ns]

    def quantised(self):
        q = np.zeros((self.n, 3), np.int64)
        self.L.orc_get_quantised(self.h, _p(q, C.c_int64))
        return q

    def rotate(self, step):
        self.L.orc_rotate(self.h, step)

    def rotations(self):
        R = np.zeros((self.n, 9))
        Rs = np.zeros((max(self.ns * self.K, 1), 9))
        self.L.orc_get_rotations(self.h, _p(R, C.c_double), _p(Rs, C.c_double))
        return R, Rs[: self.ns * self.K]

    def rebin(self):
        self.L.orc_rebin(self.h)

    def emit(self, step):
        self.L.orc_emit(self.h, step)

    def transport(self, step) -> int:
        return int(self.L.orc_transport(self.h, step))

    def chemistry(self) -> int:
        return int(self.L.orc_chemistry(self.h))

    def step(self, step) -> int:
        return int(self.L.orc_step(self.h, step))

    def cone_masks_given_directions(self, dirs):
        """Masks of the held packets with their directions given ([n, S, 3])."""
        dd = np.ascontiguousarray(dirs, dtype=np.float64).reshape(self.n * self.S * 3)
        m = np.zeros((self.n, self.S), np.uint32)
        self.L.orc_cone_masks_dir(self.h, _p(dd, C.c_double), _p(m, C.c_uint32))
        return m

    def cone_masks(self):
        m = np.zeros((self.n, self.S), np.uint32)
        self.L.orc_cone_masks(self.h, _p(m, C.c_uint32))
        return m

    def slots(self):
        f = np.zeros((6, self.n, self.S))
        self.L.orc_get_slots(self.h, _p(f, C.c_double))
        return f

    def set_slots(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self.L.orc_set_slots(self.h, _p(f, C.c_double))

    def shared_sigma(self):
        """Shared bin: G = sum N sigma of each slot of bin 0, [n, n_rc]."""
        G = np.zeros((self.n, self.params["n_rc"]))
        self.L.orc_get_shared_sigma(self.h, _p(G, C.c_double))
        return G

    def set_shared_sigma(self, G):
        G = np.ascontiguousarray(G, dtype=np.float64)
        self.L.orc_set_shared_sigma(self.h, _p(G, C.c_double))

    def state(self):
        out = [np.zeros(self.n) for _ in range(4)]
        self.L.orc_get_state(self.h, *[_p(a, C.c_double) for a in out])
        return dict(zip(["x_HI", "T", "N_rec", "eps_rec"], out))

    def set_state(self, x_HI=None, T=None, N_rec=None, eps_rec=None):
        vals = []
        keep = []
        for a in (x_HI, T, N_rec, eps_rec):
            if a is None:
                vals.append(None)
            else:
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                vals.append(_p(a, C.c_double))
        self.L.orc_set_state(self.h, *vals)

    def deposits(self):
        a = np.zeros((self.n, self.nf))
        e = np.zeros(self.n)
        ps = np.zeros((self.n, self.nf))
        self.L.orc_get_deposits(self.h, _p(a, C.c_double), _p(e, C.c_double), _p(ps, C.c_double))
        return a, e, ps

    def budget(self):
        out = np.zeros((self.nb, 4))
        self.L.orc_get_budget(self.h, _p(out, C.c_double))
        return out

    def stats(self):
        out = (C.c_longlong * 6)()
        self.L.orc_get_stats(self.h, out)
        return dict(zip(["hops", "virtual", "escaped_virtual", "subcycles", "sends", "floor_hits"],
                        list(out)))
