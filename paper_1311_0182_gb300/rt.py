"""Thin ctypes binding of the C ABI in include/traphic_rt.h (argument marshalling only).

Every step of the transport sweep runs in the CUDA library; this module only converts Python
arguments.  It raises if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RT_HOST, RT_DEVICE = 0, 1
STATUS = {0: "RT_OK", 1: "RT_ERR_INVALID", 2: "RT_ERR_OOM", 3: "RT_ERR_CUDA",
          4: "RT_ERR_HOP_LIMIT", 5: "RT_ERR_KNN", 6: "RT_ERR_CAPACITY", 7: "RT_ERR_STATE",
          8: "RT_ERR_RANGE", 9: "RT_ERR_SUBCYCLE_LIMIT"}
RT_ERR_HOP_LIMIT, RT_ERR_SUBCYCLE_LIMIT = 4, 9
SYMBOLS = ["rt_create", "rt_destroy", "rt_set_particles", "rt_set_sources", "rt_build_neighbours",
           "rt_assign_cones", "rt_merge", "rt_emit", "rt_transport", "rt_chemistry", "rt_step",
           "rt_get_state", "rt_set_state", "rt_get_budget", "rt_get_neighbours", "rt_get_quantised",
           "rt_get_rotations", "rt_get_cone_masks", "rt_get_cone_masks_noalloc", "rt_get_slots",
           "rt_set_slots",
           "rt_get_deposits", "rt_get_stats", "rt_axis_set", "rt_set_profiling",
           "rt_get_profile", "rt_last_error", "rt_set_source_options", "rt_set_barrier",
           "rt_set_graph", "rt_get_shared_sigma", "rt_set_shared_sigma", "rt_save_state",
           "rt_set_identities", "rt_query_neighbours",
           "rt_load_state"]


class RTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [
        ("n_ngb", C.c_int), ("n_ec", C.c_int), ("n_tc", C.c_int), ("n_rc", C.c_int),
        ("n_freq_src", C.c_int), ("dt", C.c_double), ("dt_em", C.c_double),
        ("rec_mode", C.c_int), ("evolve_T", C.c_int), ("transport_fp32", C.c_int),
        ("seed", C.c_ulonglong), ("hop_cap", C.c_int), ("sub_cap", C.c_int),
        ("cool_flags", C.c_int), ("T_floor", C.c_double), ("eps_rr_fixed", C.c_double),
        ("sigma_rec", C.c_double), ("free_cap", C.c_longlong), ("cell_occupancy", C.c_int),
        ("tune_launch", C.c_int), ("launch_grid", C.c_int * 3), ("rec_shared_bin", C.c_int),
    ]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the in-tree CUDA library; with build_if_missing compile it first."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
        _build.build()
    L = C.CDLL(_build.LIB)
    vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.c_double
    L.rt_create.argtypes = [C.POINTER(Config), i, C.POINTER(ll), C.POINTER(d), i, C.POINTER(vp)]
    L.rt_destroy.argtypes = [vp]
    L.rt_set_particles.argtypes = [vp] + [vp] * 7 + [i, vp]
    L.rt_set_sources.argtypes = [vp] + [vp] * 7 + [i, vp]
    L.rt_set_source_options.argtypes = [vp, vp, vp, i, vp]
    L.rt_set_barrier.argtypes = [vp, i, i, vp, d]
    L.rt_build_neighbours.argtypes = [vp, vp]
    L.rt_assign_cones.argtypes = [vp, ll, vp]
    L.rt_merge.argtypes = [vp, vp]
    L.rt_emit.argtypes = [vp, ll, vp]
    L.rt_transport.argtypes = [vp, ll, vp]
    L.rt_chemistry.argtypes = [vp, vp]
    L.rt_step.argtypes = [vp, ll, vp]
    L.rt_get_state.argtypes = [vp, vp, vp, vp, vp, i, vp]
    L.rt_set_state.argtypes = [vp, vp, vp, vp, vp, i, vp]
    L.rt_get_budget.argtypes = [vp, vp, vp]
    L.rt_get_neighbours.argtypes = [vp, vp, vp, vp, vp, i, vp]
    L.rt_get_quantised.argtypes = [vp, vp, i, vp]
    L.rt_get_rotations.argtypes = [vp, vp, vp, i, vp]
    L.rt_get_cone_masks.argtypes = [vp, vp, i, vp]
    L.rt_get_cone_masks_noalloc.argtypes = [vp, vp, i, vp]
    L.rt_get_slots.argtypes = [vp, vp, i, vp]
    L.rt_set_slots.argtypes = [vp, vp, i, vp]
    L.rt_get_shared_sigma.argtypes = [vp, vp, i, vp]
    L.rt_save_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.rt_load_state.argtypes = [vp, vp, C.c_size_t]
    L.rt_set_shared_sigma.argtypes = [vp, vp, i, vp]
    L.rt_get_deposits.argtypes = [vp, vp, vp, vp, i, vp]
    L.rt_get_stats.argtypes = [vp, vp]
    L.rt_axis_set.argtypes = [i, vp]
    L.rt_set_profiling.argtypes = [vp, i]
    L.rt_set_graph.argtypes = [vp, i]
    L.rt_set_identities.argtypes = [vp, vp, vp]
    L.rt_query_neighbours.argtypes = [vp, i, ll, vp, vp, vp, i, vp]
    L.rt_get_profile.argtypes = [vp, vp, i, vp, vp, vp, vp]
    L.rt_last_error.argtypes = [vp]
    L.rt_last_error.restype = C.c_char_p
    for s in SYMBOLS:
        if s != "rt_last_error":
            getattr(L, s).restype = C.c_int
    _lib = L
    return L


def make_config(p: dict) -> Config:
    return Config(
        n_ngb=p["n_ngb"], n_ec=p["n_ec"], n_tc=p["n_tc"], n_rc=p["n_rc"],
        n_freq_src=p["n_freq_src"], dt=p["dt"], dt_em=p["dt_em"], rec_mode=p["rec_mode"],
        evolve_T=p["evolve_T"], transport_fp32=p.get("transport_fp32", 0), seed=p["seed"],
        hop_cap=p["hop_cap"], sub_cap=p["sub_cap"], cool_flags=p["cool_flags"],
        T_floor=p["T_floor"], eps_rr_fixed=p["eps_rr_fixed"], sigma_rec=p["sigma_rec"],
        free_cap=p.get("free_cap", 0), cell_occupancy=p.get("cell_occupancy", 0),
        tune_launch=p.get("tune_launch", 0),
        launch_grid=(C.c_int * 3)(*p.get("launch_grid", (0, 0, 0))),
        rec_shared_bin=p.get("rec_shared_bin", 0))


def _ptr(a):
    """(pointer, where) of a numpy array (host) or a torch tensor (its device)."""
    if a is None:
        return None, RT_HOST
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data, RT_HOST
    assert a.is_contiguous()
    return a.data_ptr(), (RT_DEVICE if a.is_cuda else RT_HOST)


def axis_set(n: int) -> np.ndarray:
    out = np.zeros((n, 3))
    st = load().rt_axis_set(n, out.ctypes.data)
    if st:
        raise RTError(st, f"no axis set with {n} directions")
    return out


class Context:
    """One rt_ctx: the particles and sources of a workload dictionary, on the current device."""

    def __init__(self, wl: dict, stream=None, **overrides):
        self.L = load()
        p = dict(wl["params"])
        p.update(overrides)
        self.params = p
        self.cfg = make_config(p)
        self.box_off = np.ascontiguousarray(wl["box_off"], dtype=np.int64)
        self.box_L = np.ascontiguousarray(wl["box_L"], dtype=np.float64)
        self.n = int(self.box_off[-1])
        self.nb = len(self.box_L)
        self.ns = len(wl["src_box"])
        self.nf = p["n_freq_src"] + (0 if p.get("rec_shared_bin", 0) else 1)
        self.S = self.nf * p["n_rc"]
        self.K = max(1, int(round(p["dt"] / p["dt_em"])))
        self.stream = stream
        h = C.c_void_p()
        st = self.L.rt_create(C.byref(self.cfg), self.nb,
                              self.box_off.ctypes.data_as(C.POINTER(C.c_longlong)),
                              self.box_L.ctypes.data_as(C.POINTER(C.c_double)), self.ns,
                              C.byref(h))
        if st:
            raise RTError(st, "rt_create")
        self.h = h.value

    # -- plumbing ------------------------------------------------------------------------
    def _s(self):
        if self.stream is None:
            return None
        return getattr(self.stream, "cuda_stream", self.stream)

    def _check(self, st, what):
        if st:
            msg = self.L.rt_last_error(self.h)
            raise RTError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.L.rt_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    # -- set-up ----------------------------------------------------------------------------
    def set_particles(self, x, y, z, n_H, N_H, x_HI, T):
        ptrs = [_ptr(a) for a in (x, y, z, n_H, N_H, x_HI, T)]
        where = ptrs[0][1]
        self._check(self.L.rt_set_particles(self.h, *[p for p, _ in ptrs], where, self._s()),
                    "rt_set_particles")

    def set_sources(self, box, x, y, z, ndot, sigma, eps):
        ptrs = [_ptr(a) for a in (box, x, y, z, ndot, sigma, eps)]
        where = ptrs[1][1] if self.ns else ptrs[5][1]
        self._check(self.L.rt_set_sources(self.h, *[p for p, _ in ptrs], where, self._s()),
                    "rt_set_sources")

    def set_source_options(self, direction=None, gate=None):
        """Per source: fixed emission direction [ns, 3] (zero rows: isotropic) and gate [ns]."""
        dp = _ptr(direction) if direction is not None else (None, RT_HOST)
        gp = _ptr(gate) if gate is not None else (None, RT_HOST)
        where = dp[1] if direction is not None else gp[1]
        self._check(self.L.rt_set_source_options(self.h, dp[0], gp[0], where, self._s()),
                    "rt_set_source_options")

    def set_barrier(self, box, axis, centre, radius):
        c = np.ascontiguousarray(centre, dtype=np.float64)
        self._check(self.L.rt_set_barrier(self.h, int(box), int(axis), c.ctypes.data,
                                          float(radius)), "rt_set_barrier")

    def load_workload(self, wl):
        f = lambda k, dt=np.float64: np.ascontiguousarray(wl[k], dtype=dt)
        self.set_particles(f("x"), f("y"), f("z"), f("n_H"), f("N_H"), f("x_HI"), f("T"))
        self.set_sources(f("src_box", np.int32), f("src_x"), f("src_y"), f("src_z"),
                         f("src_ndot"), f("sigma"), f("eps"))
        if "src_dir" in wl or "src_gate" in wl:
            self.set_source_options(f("src_dir") if "src_dir" in wl else None,
                                    f("src_gate", np.int32) if "src_gate" in wl else None)
        for (b, axis, centre, radius) in wl.get("barriers", []):
            self.set_barrier(b, axis, centre, radius)
        if "box_first_id" in wl or "src_id" in wl:
            self.set_identities(wl.get("box_first_id"), wl.get("src_id"))

    def set_identities(self, box_first_id=None, src_id=None):
        """Random-stream identities of the boxes' particles and of the sources (None: their own
        indices); a sub-workload with its identities repeats the full workload's results."""
        bf = None if box_first_id is None else np.ascontiguousarray(box_first_id, np.int64)
        si = None if src_id is None else np.ascontiguousarray(src_id, np.int64)
        self._check(self.L.rt_set_identities(self.h, None if bf is None else bf.ctypes.data,
                                             None if si is None else si.ctypes.data),
                    "rt_set_identities")

    def build_neighbours(self):
        self._check(self.L.rt_build_neighbours(self.h, self._s()), "rt_build_neighbours")

    # -- the step and its parts ---------------------------------------------------------------
    def assign_cones(self, step):
        self._check(self.L.rt_assign_cones(self.h, step, self._s()), "rt_assign_cones")

    def merge(self):
        self._check(self.L.rt_merge(self.h, self._s()), "rt_merge")

    def emit(self, step):
        self._check(self.L.rt_emit(self.h, step, self._s()), "rt_emit")

    def transport(self, step, allow_hop_limit=False):
        st = self.L.rt_transport(self.h, step, self._s())
        if st == 4 and allow_hop_limit:
            return st
        self._check(st, "rt_transport")
        return st

    def chemistry(self, allow_subcycle_limit=False):
        st = self.L.rt_chemistry(self.h, self._s())
        if st == RT_ERR_SUBCYCLE_LIMIT and allow_subcycle_limit:
            return st
        self._check(st, "rt_chemistry")
        return st

    def step(self, step, allow_hop_limit=False, allow_subcycle_limit=False):
        st = self.L.rt_step(self.h, step, self._s())
        if (st == RT_ERR_HOP_LIMIT and allow_hop_limit) or \
                (st == RT_ERR_SUBCYCLE_LIMIT and allow_subcycle_limit):
            return st
        self._check(st, "rt_step")
        return st

    # -- state ---------------------------------------------------------------------------------
    def state(self):
        out = [np.zeros(self.n) for _ in range(4)]
        self._check(self.L.rt_get_state(self.h, *[a.ctypes.data for a in out], RT_HOST,
                                        self._s()), "rt_get_state")
        return dict(zip(["x_HI", "T", "N_rec", "eps_rec"], out))

    def get_state_into(self, x_HI=None, T=None, N_rec=None, eps_rec=None):
        ptrs = [_ptr(a) for a in (x_HI, T, N_rec, eps_rec)]
        where = next((w for p, w in ptrs if p is not None), RT_HOST)
        self._check(self.L.rt_get_state(self.h, *[p for p, _ in ptrs], where, self._s()),
                    "rt_get_state")

    def set_state(self, x_HI=None, T=None, N_rec=None, eps_rec=None):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) if isinstance(a, np.ndarray) else a
                for a in (x_HI, T, N_rec, eps_rec)]
        ptrs = [_ptr(a) for a in arrs]
        where = next((w for p, w in ptrs if p is not None), RT_HOST)
        self._check(self.L.rt_set_state(self.h, *[p for p, _ in ptrs], where, self._s()),
                    "rt_set_state")

    def budget(self):
        out = np.zeros((self.nb, 4))
        self._check(self.L.rt_get_budget(self.h, out.ctypes.data, self._s()), "rt_get_budget")
        return out

    def neighbours(self):
        k = self.params["n_ngb"]
        nbr = np.zeros((self.n, k), np.int32)
        h2 = np.zeros(self.n, np.int64)
        snbr = np.zeros((max(self.ns, 1), k), np.int32)
        sh2 = np.zeros(max(self.ns, 1), np.int64)
        self._check(self.L.rt_get_neighbours(self.h, nbr.ctypes.data, h2.ctypes.data,
                                             snbr.ctypes.data, sh2.ctypes.data, RT_HOST,
                                             self._s()), "rt_get_neighbours")
        return nbr, h2, snbr[: self.ns], sh2[: self.ns]

    def quantised(self):
        q = np.zeros((self.n, 3), np.int64)
        self._check(self.L.rt_get_quantised(self.h, q.ctypes.data, RT_HOST, self._s()),
                    "rt_get_quantised")
        return q

    def query_neighbours(self, box: int, q):
        """The exact n_ngb nearest particles (global indices) and their squared quantised
        distances for quantised points q [m, 3] of box `box`, by the virtual particles' search."""
        k = self.params["n_ngb"]
        q = np.ascontiguousarray(np.asarray(q, dtype=np.int32).reshape(-1, 3))
        nbr = np.zeros((len(q), k), np.int32)
        d2 = np.zeros((len(q), k), np.int64)
        self._check(self.L.rt_query_neighbours(self.h, box, len(q), q.ctypes.data,
                                               nbr.ctypes.data, d2.ctypes.data, RT_HOST,
                                               self._s()), "rt_query_neighbours")
        return nbr, d2

    def rotations(self):
        R = np.zeros((self.n, 9))
        Rs = np.zeros((max(self.ns * self.K, 1), 9))
        self._check(self.L.rt_get_rotations(self.h, R.ctypes.data, Rs.ctypes.data, RT_HOST,
                                            self._s()), "rt_get_rotations")
        return R, Rs[: self.ns * self.K]

    def cone_masks(self):
        m = np.zeros((self.n, self.S), np.uint32)
        self._check(self.L.rt_get_cone_masks(self.h, m.ctypes.data, RT_HOST, self._s()),
                    "rt_get_cone_masks")
        return m

    def cone_masks_noalloc(self, out=None):
        """Cone masks through the entry point that allocates nothing (static device scratch)."""
        m = np.zeros((self.n, self.S), np.uint32) if out is None else out
        p, where = _ptr(m)
        self._check(self.L.rt_get_cone_masks_noalloc(self.h, p, where, self._s()),
                    "rt_get_cone_masks_noalloc")
        return m

    def slots(self):
        f = np.zeros((6, self.n, self.S))
        self._check(self.L.rt_get_slots(self.h, f.ctypes.data, RT_HOST, self._s()),
                    "rt_get_slots")
        return f

    def set_slots(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(self.L.rt_set_slots(self.h, f.ctypes.data, RT_HOST, self._s()),
                    "rt_set_slots")

    def save_state(self) -> bytes:
        """Checkpoint between steps (rt_save_state): the held packets, particle state and budget."""
        n = C.c_size_t(0)
        self._check(self.L.rt_save_state(self.h, None, C.byref(n)), "rt_save_state")
        buf = (C.c_char * n.value)()
        self._check(self.L.rt_save_state(self.h, C.cast(buf, C.c_void_p), C.byref(n)),
                    "rt_save_state")
        return bytes(buf)

    def load_state(self, data: bytes):
        """Restore a checkpoint of a context with the same configuration and particles."""
        buf = C.create_string_buffer(data, len(data))
        self._check(self.L.rt_load_state(self.h, C.cast(buf, C.c_void_p), len(data)),
                    "rt_load_state")

    def shared_sigma(self):
        """Shared frequency bin: the cross-section sums N sigma of bin 0's packets, [n, n_rc]."""
        G = np.zeros((self.n, self.params["n_rc"]))
        self._check(self.L.rt_get_shared_sigma(self.h, G.ctypes.data, RT_HOST, self._s()),
                    "rt_get_shared_sigma")
        return G

    def set_shared_sigma(self, G):
        G = np.ascontiguousarray(G, dtype=np.float64)
        self._check(self.L.rt_set_shared_sigma(self.h, G.ctypes.data, RT_HOST, self._s()),
                    "rt_set_shared_sigma")

    def deposits(self):
        a = np.zeros((self.n, self.nf))
        e = np.zeros((self.n, self.nf))
        ps = np.zeros((self.n, self.nf))
        self._check(self.L.rt_get_deposits(self.h, a.ctypes.data, e.ctypes.data, ps.ctypes.data,
                                           RT_HOST, self._s()), "rt_get_deposits")
        return a, e, ps

    def set_graph(self, on=True):
        """step() as one captured CUDA graph (True, the default) or hop by hop from the host."""
        self._check(self.L.rt_set_graph(self.h, 1 if on else 0), "rt_set_graph")

    def profile(self, on=True):
        """Time kernels with CUDA events: True every kernel, False none, or an iterable of
        kernel names (as kernel_times() reports them)."""
        if on is True or on is False:
            mask = -1 if on else 0
        else:
            names = self.kernel_names()
            mask = 0
            for nm in on:
                mask |= 1 << names.index(nm)
        self._check(self.L.rt_set_profiling(self.h, mask), "rt_set_profiling")

    def kernel_names(self) -> list:
        names = self._profile()[1]
        return [names[k].decode() if names[k] else "" for k in range(32)]

    def _profile(self):
        nk = 32
        tot = C.c_longlong()
        names = (C.c_char_p * nk)()
        la = (C.c_longlong * nk)()
        ms = (C.c_double * nk)()
        by = (C.c_double * nk)()
        self._check(self.L.rt_get_profile(self.h, C.byref(tot), nk, names, la, ms, by),
                    "rt_get_profile")
        return tot.value, names, la, ms, by

    def launches(self) -> int:
        return self._profile()[0]

    def kernel_times(self) -> dict:
        tot, names, la, ms, by = self._profile()
        return {names[k].decode(): {"launches": la[k], "ms": ms[k], "bytes": by[k]}
                for k in range(32) if names[k] and la[k] > 0}

    def stats(self):
        out = (C.c_longlong * 20)()
        self._check(self.L.rt_get_stats(self.h, out), "rt_get_stats")
        keys = ["hops", "virtual", "escaped_virtual", "subcycles", "floor_hits", "peak_free",
                "peak_active", "gas_contrib", "senders", "moving_packets", "staged_contrib",
                "receiver_groups", "receiver_outputs", "cell_occupancy", "grid_send",
                "grid_virtual", "grid_receive", "candidate_entries", "candidate_fallback_cells"]
        return dict(zip(keys, list(out)))


def context_for(wl: dict, stream=None, **overrides) -> Context:
    """Create a context, upload the workload from host memory and build the neighbour lists."""
    c = Context(wl, stream=stream, **overrides)
    c.load_workload(wl)
    c.build_neighbours()
    return c
