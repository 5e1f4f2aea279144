"""Benchmark of the TRAPHIC transport sweep (transport + chemistry) on GB300.

One step = one RT step of the whole hot path (rotations, re-binning, emission, the hop loop with
virtual particles, chemistry, photon budget) over the workload.  Default workload: the 64^3
HII region (1e5 K blackbody in 8 grey bins + the recombination bin, 32 cones, T evolving,
FP32 transport / FP64 chemistry), started from a seeded mid-expansion state.

The timed steps run the product path, rt_step as one captured CUDA graph (the hop loop a
conditional while node).  The roofline's kernel duration comes from CUDA events around every
launch of the dominant kernel in the same steps run hop by hop on a second context.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-sweeps/s (transport+chemistry)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--n-side", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--original", action="store_true",
                    help="also time the original (emission-cone) recombination implementation")
    ap.add_argument("--shared", action="store_true",
                    help="also time one frequency bin shared by stellar and recombination photons")
    ap.add_argument("--batched", action="store_true",
                    help="also time workload 4: 512 independent boxes of uneven size in the same "
                         "launches, FP32 transport and all FP64")
    ap.add_argument("--paper-workloads", action="store_true",
                    help="also time workload 3 (128^3 with a dense clump) and workload 5 (256^3 "
                         "clustered volume, 256 sources), FP32 transport")
    ap.add_argument("--tuned", action="store_true",
                    help="also time the workload with the launch sizes of the hop kernels chosen "
                         "by the step-graph tuner (tune_launch) after its tuning steps")
    ap.add_argument("--source-count", action="store_true",
                    help="also time the same workload with its luminosity split over 1, 8 and 64 "
                         "sources clustered where the one source sits (Sec. 2.1: the cost does "
                         "not depend on the number of sources)")
    ap.add_argument("--on-the-spot", action="store_true",
                    help="also time the same workload without recombination transport (case B "
                         "on the spot), and with it in a shared bin against on the spot with one "
                         "bin fewer")
    return ap.parse_args()


def workload(args):
    from paper_1311_0182_gb300 import workloads as W
    return W.cfg2(n_side=args.n_side, transport_fp32=1 if args.precision == "fp32" else 0)


def workload_name(n_side: int) -> str:
    return f"hii_region_{n_side}^3_bb1e5K_8bins_32cones_Tevolving"


def workload_config(args, wl):
    p = wl["params"]
    n_side = round(int(wl["box_off"][-1]) ** (1 / 3))
    return {"workload": workload_name(n_side),
            "particles": int(wl["box_off"][-1]), "n_ngb": p["n_ngb"], "cones": p["n_tc"],
            "freq_bins": p["n_freq_src"] + 1, "dt_myr": p["dt"] / 3.15576e13,
            "start": "seeded mid-expansion HII region (front at 0.8 R_S)",
            "transport": args.precision, "chemistry": "fp64",
            "l2": "inputs larger than L2 (slot arrays > 1 GB)"}


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self):
        self.rows, self.proc = [], None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def stop(self, dev=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for r in self.rows if r and r[0] == str(dev)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _advance(ctx, stream, steps, start=0):
    import torch
    with torch.cuda.stream(stream):
        for s in range(start, start + steps):
            ctx.step(s)


def run_ours(args):
    import torch
    from paper_1311_0182_gb300 import rt

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wl = workload(args)
    n = int(wl["box_off"][-1])
    stream = torch.cuda.Stream()
    ctx = rt.Context(wl, stream=stream)
    with torch.cuda.stream(stream):
        ctx.load_workload(wl)
        ctx.build_neighbours()
    _advance(ctx, stream, args.warmup)      # the first step tunes the hop kernels' launch sizes
    # a second context on the same input runs the same steps hop by hop from the host: the
    # only way to bracket single kernels with CUDA events (the step graph's conditional hop
    # loop can hold no event nodes).  It takes the kNN grid and launch sizes the first one
    # chose, so its launches of the dominant kernel are the same launches, on the same data,
    # as those inside the timed graph steps
    st0 = ctx.stats()
    ctx_h = rt.Context(wl, stream=stream, cell_occupancy=st0["cell_occupancy"], tune_launch=0,
                       launch_grid=(st0["grid_send"], st0["grid_virtual"], st0["grid_receive"]))
    ctx_h.set_graph(False)
    with torch.cuda.stream(stream):
        ctx_h.load_workload(wl)
        ctx_h.build_neighbours()
    _advance(ctx_h, stream, args.warmup)
    step = args.warmup
    with torch.cuda.stream(stream):
        # one more (untimed) step with every kernel timed: the per-kernel shares of a step,
        # and the dominant modelled kernel
        for c in (ctx, ctx_h):
            c.profile(True)
            c.step(step)
        kt_all = ctx.kernel_times()
        shares = kernel_shares(kt_all)
        dominant = max(MODELLED, key=lambda k: kt_all.get(k, {"ms": 0.0})["ms"])
        ctx.profile(False)                 # the timed region: the step graph, nothing timed inside
        ctx_h.profile([dominant])
        step += 1
        stream.synchronize()
        if dist:
            tdist.barrier()
        clk = Clocks()
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        launches0 = ctx.launches()
        for s in range(step, step + args.steps):
            ctx.step(s)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = ctx.launches() - launches0
        clocks = clk.stop(local)
        st = ctx.stats()
        b = ctx.budget()
        # the same steps hop by hop, the dominant kernel bracketed with events
        clk_h = Clocks()
        clk_h.start()
        torch.cuda.synchronize()
        e0.record(stream)
        hops = []                       # per timed step (the same steps as the graph's)
        for s in range(step, step + args.steps):
            ctx_h.step(s)
            hops.append(ctx_h.stats()["hops"])     # a host-side read after the step's own sync
        e1.record(stream)
        torch.cuda.synchronize()
        ms_h = e0.elapsed_time(e1)
        clocks_h = clk_h.stop(local)
        kt = ctx_h.kernel_times()
        same = bool(np.array_equal(ctx.state()["x_HI"], ctx_h.state()["x_HI"]))
        ctx_h.profile(False)
        step += args.steps
    if dist:
        from paper_1311_0182_gb300.distributed import max_over_ranks
        ms = max_over_ranks(ms, device="cuda")      # one replica per rank: the slowest decides
    value = world * n * args.steps / (ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "particle-sweeps/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 transport / f64 chemistry" if args.precision == "fp32" else "f64",
           "data": "synthetic", "config": workload_config(args, wl), "gpu_launches": launches,
           "clocks": clocks,
           # a particle-hop is one gas particle taking part in one hop
           "hops_per_step": sum(hops) / len(hops),
           "particle_hops_per_s": world * n * sum(hops) / (ms / 1e3)}
    # roofline of the dominant kernel, timed over the same steps run hop by hop
    out["roofline"] = roofline(ctx_h, kt, ms_h, args)
    out["roofline"]["timing"] = ("CUDA events on the launching stream around every launch of "
                                 "the kernel, over the timed steps repeated hop by hop on a "
                                 "second context (identical launches and data)")
    out["hop_by_hop"] = {"value": n * args.steps / (ms_h / 1e3), "ms_per_step": ms_h / args.steps,
                         "same_result_bits": same, "clocks": clocks_h,
                         "note": "host-driven hop loop, one synchronisation per hop; the "
                                 "dominant kernel bracketed with events"}
    out["roofline"]["hop_loop_model"] = hop_loop_model(st, wl, ms / args.steps)
    out["roofline_issue"] = roofline_issue(out["roofline"], clocks_h)
    out["kernel_shares"] = shares
    out["stats_last_step"] = st
    out["floor_hits_last_step"] = st["floor_hits"]
    from paper_1311_0182_gb300.run import ionised_fraction
    out["ionised_volume_fraction"] = ionised_fraction(ctx.state()["x_HI"], wl["n_H"], wl["N_H"])
    out["budget_closure"] = float(abs(b[0, 0] - b[0, 1:].sum()) / b[0, 0])
    ctx_h.close()
    if not args.no_e2e:
        out["e2e"] = e2e(args, wl, stream, step - args.steps, st0, ctx.state()["x_HI"])
    ctx.close()
    if not args.no_fp64 and args.precision == "fp32":
        out["fp64_path"] = fp64_path(args, stream)
        out["fp32_over_fp64"] = out["value"] / out["fp64_path"]["value"]
        out["fp32_vs_fp64"] = precision_check(args, stream)
    if args.original:
        # the original implementation of recombination radiation (Sec. 2.2): per-particle
        # emission cones, on the same workload and precision
        out["original_recombination"] = fp64_path(
            args, stream, transport_fp32=int(args.precision == "fp32"), rec_mode=3)
    if args.shared:
        # stellar and recombination photons in one frequency bin (Sec. 2.2, last paragraph),
        # on the same workload and precision
        out["shared_frequency_bin"] = fp64_path(
            args, stream, transport_fp32=int(args.precision == "fp32"), rec_shared_bin=1)
    if args.on_the_spot:
        # the cost of transporting recombination radiation (Sec. 1, Sec. 2.2): on the spot,
        # with the same slots (a recombination bin that stays empty) and with the shared-bin
        # layout (no recombination bin)
        fp = int(args.precision == "fp32")
        out["on_the_spot"] = fp64_path(args, stream, transport_fp32=fp, rec_mode=1)
        out["on_the_spot_shared_layout"] = fp64_path(args, stream, transport_fp32=fp, rec_mode=1,
                                                     rec_shared_bin=1)
    if args.tuned:
        out["tuned_launch_sizes"] = tuned(args, stream)
    if args.source_count:
        out["source_count"] = source_count(args, stream)
    if args.batched:
        out["batched_boxes"] = batched(args, stream, world=world, rank=rank)
    if args.paper_workloads:
        out["paper_workloads"] = paper_workloads(stream)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
        out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores()
    if dist:
        tdist.destroy_process_group()
    return out if rank == 0 else None


MODELLED = ("phase_b_merge", "virtual_particles", "phase_a_send")


def kernel_shares(kt: dict) -> dict:
    """Per kernel of one profiled step: launches, ms and share of the summed kernel time."""
    tot = sum(v["ms"] for v in kt.values()) or 1.0
    return {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                "share": round(v["ms"] / tot, 4)}
            for k, v in sorted(kt.items(), key=lambda kv: -kv[1]["ms"]) if v["ms"] > 0}


def source_hash() -> str:
    """Hash of the CUDA sources: a committed ncu traffic figure is valid only for this source."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1311_0182_gb300", "csrc")
    for fn in ("rt_transport.cu", "rt_internal.cuh", "rt_knn.cuh"):   # where the hop kernels live
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


PER_UNIT_TABLE = ("profiles", "k_virtual_per_unit_hii_48cubed.md")


def committed_per_unit(kernel: str):
    """(DRAM bytes, warp instructions) per unit of work of `kernel` from the committed ncu
    summary, or None when the summary belongs to other CUDA sources."""
    path = os.path.join(ROOT, *PER_UNIT_TABLE)
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for line in lines:
        parts = [p.strip() for p in line.strip().strip("|").split("|")]
        if len(parts) >= 6 and parts[0] == kernel:
            try:
                dram, inst, src = float(parts[1]), float(parts[2]), parts[5]
            except ValueError:
                continue
            return (dram, inst) if src == source_hash() else None
    return None


def vp_model_bytes(params: dict) -> float:
    """Algorithmic bytes per virtual particle of k_virtual (the library's model): request and
    packet, per neighbour its position, four properties, two deposit words and the forwarded
    list entry, and the forwarded packet."""
    R = 4 if params["transport_fp32"] else 8
    kn = params["n_ngb"]
    return 8 + 6 * R + 40 + kn * (16 + 4 * R + 16 + 4) + 6 * R + 40


def issue_peak(sm_mhz) -> float:
    """Warp instructions per second the GPU can issue: 152 SMs x 4 schedulers x 1 per cycle."""
    return 152 * 4 * (sm_mhz or 2070.0) * 1e6


def roofline(ctx, kt, ms_step_total, args):
    peak, kind = peaks()
    if not kt:
        return None
    name = max(kt, key=lambda k: kt[k]["ms"])
    if name not in MODELLED:
        name = max(MODELLED, key=lambda k: kt.get(k, {"ms": 0})["ms"])
    k = kt[name]
    ms = k["ms"] / max(k["launches"], 1)
    B = k["bytes"] / max(k["launches"], 1)
    ach = B / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    # DRAM traffic per launch: the committed per-virtual-particle figure times this launch's
    # virtual particles (its algorithmic bytes over the model's bytes per virtual particle)
    pu = committed_per_unit(name) if name == "virtual_particles" else None
    units = B / vp_model_bytes(ctx.params) if pu else None
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_kind": f"{kind} (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else kind,
            "traffic": pu[0] * units if pu else None,
            "units_per_launch": units,
            "algorithmic_bytes_per_launch": B, "ms_per_launch": ms, "launches": k["launches"],
            "share_of_step": k["ms"] / ms_step_total if ms_step_total else None,
            "all_kernels": {n: {"launches": v["launches"], "ms": round(v["ms"], 3),
                                "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] and v["bytes"] else None}
                            for n, v in kt.items() if v["ms"] > 0}}


def roofline_issue(rf: dict, clocks: dict):
    """The bound the dominant kernel actually meets: instruction issue.  Warp instructions per
    launch (the committed ncu count per virtual particle times the launch's virtual particles)
    over the launch's event-timed duration, against 152 SMs x 4 schedulers x 1 instruction per
    cycle at the SM clock sampled during those launches."""
    if not rf or rf.get("kernel") != "virtual_particles":
        return None
    pu = committed_per_unit("virtual_particles")
    if not pu or not rf.get("units_per_launch"):
        return None
    inst = pu[1] * rf["units_per_launch"]
    ach = inst / (rf["ms_per_launch"] / 1e3)
    peak = issue_peak(clocks.get("sm_mhz"))
    return {"bound": "issue", "kernel": "virtual_particles", "achieved": ach, "peak": peak,
            "unit": "warp-instructions/s", "frac": ach / peak,
            "warp_instructions_per_launch": inst, "sm_mhz": clocks.get("sm_mhz"),
            "peak_kind": "152 SMs x 4 schedulers x 1 warp instruction per cycle at the sampled SM clock"}


def hop_loop_model(st: dict, wl: dict, ms_step: float) -> dict:
    """The per-particle-hop byte model of the whole sweep: per hop and active particle
    2 S_act 20 B of slots read and written, n_ngb (4 + 4) B of reverse and forward lists, 12 B of
    position, 8 B of x_HI and n_H, 16 N_f B of tallies; plus about 100 + 8 N_f B per particle of
    chemistry per step.  The active counts are the device counters of the last timed step
    (packets able to move and particles holding one, summed over its hops).  Virtual particles
    are outside this model; the per-kernel models count them."""
    peak, kind = peaks()
    p = wl["params"]
    kn, nf = p["n_ngb"], p["n_freq_src"] + (0 if p.get("rec_shared_bin", 0) else 1)
    n = int(wl["box_off"][-1])
    B = (2 * 20 * st["moving_packets"] + (8 * kn + 12 + 8 + 16 * nf) * st["senders"] +
         (100 + 8 * nf) * n)
    ach = B / (ms_step / 1e3) / 1e9
    return {"bytes_per_step": B, "ms_per_step": ms_step, "achieved": ach, "unit": "GB/s",
            "peak": peak, "frac": ach / peak, "packets_moved": st["moving_packets"],
            "particle_hops": st["senders"], "peak_kind": kind}


def fp64_path(args, stream, **over):
    """The all-FP64 GPU path on the same workload and start state (the comparison path); with
    `over`, the same timing for other parameters."""
    import torch
    from paper_1311_0182_gb300 import rt, workloads as W
    wl = W.cfg2(n_side=args.n_side, **dict(dict(transport_fp32=0), **over))
    ctx = rt.Context(wl, stream=stream)
    steps = max(1, args.steps)
    with torch.cuda.stream(stream):
        ctx.load_workload(wl)
        ctx.build_neighbours()
        for s in range(args.warmup + 1):    # the main run's warm-up and its profiled step
            ctx.step(s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for s in range(steps):
            ctx.step(args.warmup + 1 + s)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    n = int(wl["box_off"][-1])
    ctx.close()
    pr = wl["params"]
    R = 4 if pr["transport_fp32"] else 8
    nrc = pr["n_rc"]
    S = (pr["n_freq_src"] + (0 if pr.get("rec_shared_bin", 0) else 1)) * nrc
    # packet storage: two slot buffers of 6 fields, the sender records (8 values a slot) and,
    # with a shared bin, two buffers of bin-0 cross-section sums
    slot_bytes = n * R * (2 * 6 * S + 8 * S + (2 * nrc if pr.get("rec_shared_bin", 0) else 0))
    return {"value": n * steps / (ms / 1e3), "unit": "particle-sweeps/s",
            "ms_per_step": ms / steps, "steps": steps, "packet_storage_bytes": slot_bytes,
            "dtype": "f64" if not wl["params"]["transport_fp32"] else "f32 transport / f64 chemistry"}


def tuned(args, stream, tuning_steps=18):
    """The timed workload with tune_launch: 18 tuning steps (whole step-graph launches, each a
    candidate triple of grid sizes or the best so far), then the main run's warm-up and timed
    steps with the sizes it chose, against the same steps with the built-in sizes."""
    import torch
    from paper_1311_0182_gb300 import rt
    wl = workload(args)
    out = {}
    for name, over in (("tuned", dict(tune_launch=1)), ("built_in", dict(tune_launch=0))):
        ctx = rt.Context(wl, stream=stream, **over)
        with torch.cuda.stream(stream):
            ctx.load_workload(wl)
            ctx.build_neighbours()
            for s in range(tuning_steps + args.warmup):
                ctx.step(s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            s0 = tuning_steps + args.warmup
            for s in range(s0, s0 + args.steps):
                ctx.step(s)
            e1.record(stream)
            torch.cuda.synchronize()
        st = ctx.stats()
        out[name] = {"ms_per_step": e0.elapsed_time(e1) / args.steps,
                     "grids": [st["grid_send"], st["grid_virtual"], st["grid_receive"]]}
        ctx.close()
    out["tuned_over_built_in"] = out["tuned"]["ms_per_step"] / out["built_in"]["ms_per_step"]
    return out


def source_count(args, stream, counts=(1, 8, 64), warmup=3, steps=3):
    """Sec. 2.1: packets merge per reception cone at every particle, so the work of a step is
    bounded by the particles and their cones, not by the number of sources.  The timed workload
    with its luminosity split over 1, 8 and 64 sources clustered within 2% of the box side
    around the centre: ms per step and the per-step work counters (particles sending, packets
    moved, virtual particles, hops) of the last timed step, same precision and start state."""
    import torch
    from paper_1311_0182_gb300 import rt, workloads as W
    out = {"spread_of_box": 0.02, "warmup": warmup, "steps": steps, "runs": {}}
    for ns in counts:
        wl = W.split_sources(W.cfg2(n_side=args.n_side,
                                    transport_fp32=int(args.precision == "fp32")), ns)
        ctx = rt.Context(wl, stream=stream)
        with torch.cuda.stream(stream):
            ctx.load_workload(wl)
            ctx.build_neighbours()
            for s in range(warmup):
                ctx.step(s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for s in range(warmup, warmup + steps):
                ctx.step(s)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
        st = ctx.stats()
        b = ctx.budget()
        out["runs"][str(ns)] = {"ms_per_step": ms, "senders": st["senders"],
                                "moving_packets": st["moving_packets"], "virtual": st["virtual"],
                                "hops": st["hops"],
                                "budget_closure": float(abs(b[0, 0] - b[0, 1:].sum()) / b[0, 0])}
        ctx.close()
    r1 = out["runs"][str(counts[0])]
    for ns in counts[1:]:
        r = out["runs"][str(ns)]
        r["ms_over_one_source"] = r["ms_per_step"] / r1["ms_per_step"]
        r["moving_packets_over_one_source"] = r["moving_packets"] / r1["moving_packets"]
    return out


def batched(args, stream, warmup=2, steps=3, world=1, rank=0):
    """Workload 4: 512 independent boxes of 8^3 to 40^3 particles (log-uniform count),
    lognormal densities, one central source each, T evolving, 8 cones, advanced together in
    the same launches (the step graph), FP32 transport and all FP64.  With several ranks the
    boxes are split between them (longest-processing-time greedy on particle count), each rank
    runs its boxes with no collective in the timed region, the time is the slowest rank's and
    the per-box photon budgets are summed over ranks afterwards."""
    import torch
    from paper_1311_0182_gb300 import distributed as D, rt, workloads as W
    wl_all = W.cfg4()
    n = int(wl_all["box_off"][-1])
    nb = len(wl_all["box_L"])
    mine = np.arange(nb)
    wl = wl_all
    if world > 1:
        mine = D.partition_boxes(np.diff(wl_all["box_off"]), world)[rank]
        wl = D.local_workload(wl_all, mine)
    out = {"workload": "512 boxes, 8^3-40^3 particles each (log-uniform), lognormal density, "
                       "central source, 8 cones, 2 frequency bins, T evolving",
           "particles": n, "boxes": nb, "warmup": warmup, "steps": steps, "ranks": world,
           "scaling": "strong" if world > 1 else None,
           "partition": "LPT on particle count; no collective inside the timed steps"}
    for fp in (1, 0):
        ctx = rt.Context(wl, stream=stream, transport_fp32=fp)
        with torch.cuda.stream(stream):
            ctx.load_workload(wl)
            ctx.build_neighbours()
            for s in range(warmup):
                ctx.step(s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for s in range(warmup, warmup + steps):
                ctx.step(s)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        st = ctx.stats()
        b = np.zeros((nb, 4))
        b[mine] = ctx.budget()
        if world > 1:
            ms = D.max_over_ranks(ms, device="cuda")
            b = D.sum_over_ranks(b, device="cuda")
        out["fp32" if fp else "fp64"] = {
            "value": n * steps / (ms / 1e3), "unit": "particle-sweeps/s",
            "ms_per_step": ms / steps, "hops_last_step_rank0": st["hops"],
            "virtual_last_step_rank0": st["virtual"],
            "worst_box_budget_closure": float(np.max(np.abs(b[:, 0] - b[:, 1:].sum(1)) / b[:, 0]))}
        ctx.close()
    out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def paper_workloads(stream, warmup=1, steps=2):
    """Workload 3 (128^3 equal-mass particles with a clump 200x denser, 5 kpc from a
    3e51 s^-1 source; 8 cones, grey bin, 0.1 Myr steps) and workload 5 (256^3 particles sampled
    from a lognormal field, 256 sources in its densest 1 %; 8 cones, 1 Myr steps), FP32
    transport, from their initial states."""
    import torch
    from paper_1311_0182_gb300 import rt, workloads as W
    out = {}
    for name, make in (("workload3_clump_128^3", W.cfg3), ("workload5_clustered_256^3", W.cfg5)):
        wl = make(transport_fp32=1)
        n = int(wl["box_off"][-1])
        ctx = rt.Context(wl, stream=stream)
        with torch.cuda.stream(stream):
            ctx.load_workload(wl)
            ctx.build_neighbours()
            for s in range(warmup):
                ctx.step(s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for s in range(warmup, warmup + steps):
                ctx.step(s)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        st = ctx.stats()
        b = ctx.budget()
        out[name] = {"particles": n, "sources": len(wl["src_box"]), "warmup": warmup,
                     "steps": steps, "value": n * steps / (ms / 1e3), "unit": "particle-sweeps/s",
                     "ms_per_step": ms / steps, "hops_last_step": st["hops"],
                     "virtual_last_step": st["virtual"], "cell_occupancy": st["cell_occupancy"],
                     "budget_closure": float(abs(b[0, 0] - b[0, 1:].sum()) / b[0, 0])}
        ctx.close()
        del wl
    return out


def precision_check(args, stream, steps=10):
    """FP32-transport path against the all-FP64 path (which follows the oracle to rounding in
    the parity tests), same workload and start, run side by side for `steps` steps: the
    routing-affected particles (absorptions of some step off by more than ROUTE_TOL, see
    paper_1311_0182_gb300/accuracy.py), the largest relative errors of x_HI and T among all
    particles and among the others, and per radial shell around the source (shells of 1/16 of
    the box side) the largest errors and affected counts."""
    import torch
    from paper_1311_0182_gb300 import accuracy as ACC, rt, workloads as W
    wl = W.cfg2(n_side=args.n_side)
    ctx = {fp: rt.Context(wl, stream=stream, transport_fp32=fp) for fp in (1, 0)}
    affected = np.zeros(int(wl["box_off"][-1]), bool)
    with torch.cuda.stream(stream):
        for c in ctx.values():
            c.load_workload(wl)
            c.build_neighbours()
        for s in range(steps):
            dep = {}
            for fp, c in ctx.items():
                c.step(s)
                a, e, _ = c.deposits()
                dep[fp] = (a.sum(1), e.sum(1))
            ACC.mark_routing_affected(dep[1][0], dep[0][0], dep[1][1], dep[0][1], wl["N_H"],
                                      affected)
    st = {fp: c.state() for fp, c in ctx.items()}
    for c in ctx.values():
        c.close()
    out = {"steps": steps, "reference": "all-FP64 GPU path",
           **ACC.summary(st[1], st[0], affected, steps)}
    pos = np.stack([wl["x"], wl["y"], wl["z"]], 1)
    src = np.array([wl["src_x"][0], wl["src_y"][0], wl["src_z"][0]])
    r = np.linalg.norm(pos - src, axis=1) / float(wl["box_L"][0])
    relx = np.abs(st[1]["x_HI"] / st[0]["x_HI"] - 1)
    relT = np.abs(st[1]["T"] / st[0]["T"] - 1)
    shells = []
    for k in range(9):
        m = (r >= k / 16) & (r < (k + 1) / 16)
        if m.any():
            shells.append([round(k / 16, 4), int(m.sum()), int(affected[m].sum()),
                           float(f"{relx[m].max():.3g}"), float(f"{relT[m].max():.3g}")])
    out["shells"] = {"columns": ["r_over_L_from", "particles", "routing_affected",
                                 "x_HI_max_rel", "T_max_rel"], "rows": shells}
    return out


def e2e(args, wl, stream, first, st0, x_ref):
    """Same metric through the C ABI with host buffers: per step the state arrays go host ->
    device, the step runs, and the state and photon budget come back.  A fresh context with
    the main run's grid and launch sizes is brought to the first timed step untimed, so the
    timed steps are the same steps, with the same work, as `value`'s; its state after them is
    compared with the main run's."""
    import torch
    from paper_1311_0182_gb300 import rt
    ctx = rt.Context(wl, stream=stream, cell_occupancy=st0["cell_occupancy"], tune_launch=0,
                     launch_grid=(st0["grid_send"], st0["grid_virtual"], st0["grid_receive"]))
    with torch.cuda.stream(stream):
        ctx.load_workload(wl)
        ctx.build_neighbours()
    _advance(ctx, stream, first)
    n = ctx.n
    hx = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    hT = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    ctx.get_state_into(x_HI=hx, T=hT)      # the host holds the state of the first timed step
    steps = args.steps
    step = first
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            ctx.set_state(x_HI=hx, T=hT)
            ctx.step(step)
            step += 1
            ctx.get_state_into(x_HI=hx, T=hT)
            ctx.budget()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    out = {"value": n * steps / dt, "unit": "particle-sweeps/s", "h2d_bytes_per_step": 16 * n,
           "d2h_bytes_per_step": 16 * n + 32 * ctx.nb, "steps": steps,
           "timed_steps": [first, first + steps - 1],
           "same_result_bits": bool(np.array_equal(hx, x_ref))}
    ctx.close()
    return out


def _oracle_sample(n_side, steps):
    """One process's share of the all-cores CPU baseline: `steps` whole RT steps of the HII-region
    recipe at n_side^3 after one untimed step; returns (particle-sweeps, seconds)."""
    import oracle
    from paper_1311_0182_gb300 import workloads as W
    s = oracle.Sim(W.cfg2(n_side=n_side))
    s.build_neighbours()
    s.step(0)
    t0 = time.perf_counter()
    for k in range(steps):
        s.step(1 + k)
    return n_side ** 3 * steps, time.perf_counter() - t0


def cpu_baseline_all_cores(n_side=24, steps=3):
    """The oracle as it stands, one independent copy of the same sample per host core (a process
    pool started with spawn, as the process has already used the GPU): total particle-sweeps over
    the wall time of the whole pool."""
    import multiprocessing as mp
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.starmap(_oracle_sample, [(n_side, steps)] * cores)
    wall = time.perf_counter() - t0
    work = sum(r[0] for r in res)
    timed = max(r[1] for r in res)
    return {"value": work / timed, "unit": "particle-sweeps/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent copies, one per core, each {steps} whole RT steps "
                      f"(after one untimed) of the HII-region recipe at {n_side}^3; rate over the "
                      f"slowest copy's timed steps ({timed:.1f} s; pool wall time {wall:.1f} s)"}


def cpu_baseline(args, budget_s=20.0):
    """The oracle as it stands on the host cores (1 thread) on a bounded sample: whole steps
    of the same workload at a reduced particle count, scaled per particle-sweep."""
    import oracle
    from paper_1311_0182_gb300 import workloads as W
    n_side = 24
    wl = W.cfg2(n_side=n_side)
    s = oracle.Sim(wl)
    s.build_neighbours()
    s.step(0)            # the first step carries no recombination photons yet: not timed
    t0 = time.perf_counter()
    steps = 0
    while steps < 4 and time.perf_counter() - t0 < budget_s:
        s.step(1 + steps)
        steps += 1
    dt = time.perf_counter() - t0
    n = n_side ** 3
    return {"value": n * steps / dt, "unit": "particle-sweeps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} whole RT steps (after one untimed) of the same HII-region recipe "
                      f"at {n_side}^3 particles instead of 64^3 (32 cones, 9 bins, T evolving), "
                      f"{dt:.1f} s single-threaded; per-particle cost grows with the box (more hops)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    wl_args = argparse.Namespace(**vars(args))
    from paper_1311_0182_gb300 import workloads as W
    n_side = 24
    wl = W.cfg2(n_side=n_side)
    s = oracle.Sim(wl)
    s.build_neighbours()
    step = 0
    for _ in range(args.warmup):
        s.step(step)
        step += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(step)
        step += 1
    dt = time.perf_counter() - t0
    n = n_side ** 3
    v = n * args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-sweeps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(wl_args, wl), transport="fp64 (oracle)",
                           sample_of=workload_name(args.n_side),
                           note=f"the oracle times whole steps of the same recipe at {n_side}^3 "
                                f"particles, a bounded sample of the {args.n_side}^3 workload; "
                                f"per-particle cost grows with the box (more hops)"),
            "cpu_baseline": {"value": v, "unit": "particle-sweeps/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step a whole RT step of the workload at {n_side}^3"},
            "e2e": {"value": v, "unit": "particle-sweeps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def relaunch_on_ranks(n: int) -> int:
    """`--gpus N` without a launcher: run this same command as N ranks under
    torch.distributed.run on this node (rendezvous on 127.0.0.1); returns its exit code."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_on_ranks(args.gpus))
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
