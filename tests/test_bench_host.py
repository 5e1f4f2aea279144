"""Host logic of the benchmark (no GPU): the roofline arithmetic, the committed DRAM traffic
(taken only when the CUDA sources match the profiled ones, scaled by particle count), the
per-kernel shares of a step, the clock samples' summary, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys
import types

import numpy as np

import bench


def test_roofline_is_algorithmic_bytes_over_event_time(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (6684.1, "measured"))
    monkeypatch.setattr(bench, "committed_per_unit", lambda k: None)
    kt = {"virtual_particles": {"ms": 10.0, "launches": 10, "bytes": 6.6841e9},
          "phase_a_send": {"ms": 2.0, "launches": 10, "bytes": 1e9},
          "hop_lens": {"ms": 20.0, "launches": 30, "bytes": 0.0}}
    r = bench.roofline(types.SimpleNamespace(params={"transport_fp32": 1, "n_ngb": 32}), kt, 50.0,
                       types.SimpleNamespace(n_side=64))
    # the dominant modelled kernel, not the slowest kernel without a bytes model
    assert r["kernel"] == "virtual_particles"
    assert np.isclose(r["ms_per_launch"], 1.0)
    assert np.isclose(r["achieved"], 668.41)              # 6.6841e8 bytes in 1 ms
    assert np.isclose(r["frac"], 0.1)
    assert np.isclose(r["share_of_step"], 0.2)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None


def _fake_tree(tmp_path, table_hash):
    csrc = tmp_path / "paper_1311_0182_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in ("rt_transport.cu", "rt_internal.cuh", "rt_knn.cuh"):
        (csrc / fn).write_text("// " + fn + "\n")
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / bench.PER_UNIT_TABLE[1]).write_text(
        "| kernel | DRAM bytes per unit | warp instructions per unit | unit | units in capture | source hash |\n"
        "|---|---|---|---|---|---|\n"
        f"| virtual_particles | 700.0 | 2500.0 | virtual particle | 1000 | {table_hash} |\n")


def test_per_unit_figures_are_taken_only_for_the_profiled_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _fake_tree(tmp_path, "0" * 16)
    h = bench.source_hash()
    assert bench.committed_per_unit("virtual_particles") is None        # other sources
    import shutil
    shutil.rmtree(tmp_path / "profiles")
    shutil.rmtree(tmp_path / "paper_1311_0182_gb300")
    _fake_tree(tmp_path, h)
    assert bench.committed_per_unit("virtual_particles") == (700.0, 2500.0)
    assert bench.committed_per_unit("phase_b_merge") is None


def test_traffic_and_issue_rooflines_scale_by_the_launch_units(tmp_path, monkeypatch):
    """Traffic and instructions per launch: the committed per-virtual-particle figures times the
    launch's virtual particles (its algorithmic bytes over the model's bytes per particle)."""
    monkeypatch.setattr(bench, "peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "committed_per_unit", lambda k: (700.0, 2500.0))
    params = {"transport_fp32": 1, "n_ngb": 32}
    per = bench.vp_model_bytes(params)
    assert per == 8 + 24 + 40 + 32 * (16 + 16 + 16 + 4) + 24 + 40
    kt = {"virtual_particles": {"ms": 2.0, "launches": 2, "bytes": 2 * 1000 * per}}
    ctx = types.SimpleNamespace(params=params)
    r = bench.roofline(ctx, kt, 10.0, types.SimpleNamespace(n_side=64))
    assert np.isclose(r["units_per_launch"], 1000) and np.isclose(r["traffic"], 700.0 * 1000)
    ri = bench.roofline_issue(r, {"sm_mhz": 2000.0})
    assert np.isclose(ri["achieved"], 2500.0 * 1000 / 1e-3)
    assert np.isclose(ri["peak"], 152 * 4 * 2000e6) and ri["bound"] == "issue"


def test_kernel_shares_sum_to_one():
    kt = {"a": {"ms": 3.0, "launches": 1}, "b": {"ms": 1.0, "launches": 2},
          "c": {"ms": 0.0, "launches": 5}}
    sh = bench.kernel_shares(kt)
    assert list(sh) == ["a", "b"]                       # sorted by time, idle kernels left out
    assert np.isclose(sum(v["share"] for v in sh.values()), 1.0)


def test_clock_summary_reports_throttle_reasons():
    c = bench.Clocks()
    c.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0)
    row = lambda sm, *flags: ["0", str(sm), "2070", "900.5", "0x0"] + list(flags)
    c.rows = [row(2070, "Not Active", "Not Active", "Not Active", "Not Active"),
              row(1995, "Not Active", "Not Active", "Not Active", "Active"),
              row(2070, "Not Active", "Not Active", "Not Active", "Not Active"),
              ["1", "300", "2070", "10", "0x0", "Active", "Active", "Active", "Active"]]
    out = c.stop(dev=0)
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]           # the other GPU's row is not counted


def _reference_arm(env_extra):
    from conftest import ROOT
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                          cwd=ROOT, env=env, timeout=600)


def test_reference_arm_prints_one_contract_line_on_rank_0_only():
    """The reference arm times the CPU oracle: one JSON line with the contract's keys, its
    cpu_baseline and e2e describing the same run; the other ranks of a torchrun print nothing."""
    r = _reference_arm({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in out, key
    assert out["impl"] == "reference" and out["value"] > 0 and out["steps"] == 1
    assert out["metric"] == bench.METRIC and out["higher_is_better"] is True
    assert "workload" in out["config"]
    # the config names the size the oracle actually timed, and what it samples
    assert out["config"]["particles"] == 24 ** 3 and "24^3" in out["config"]["workload"]
    assert out["config"]["sample_of"] == bench.workload_name(64)
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == out["value"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    r1 = _reference_arm({"RANK": "1"})
    assert r1.returncode == 0 and r1.stdout.strip() == ""


def test_hop_loop_model_counts_the_per_particle_hop_bytes(monkeypatch):
    """Per hop and active particle 2 S_act 20 B of slots, n_ngb (4 + 4) B of lists, 12 + 8 B of
    position and density, 16 N_f B of tallies; 100 + 8 N_f B of chemistry per particle."""
    monkeypatch.setattr(bench, "peaks", lambda: (8000.0, "measured"))
    wl = {"params": {"n_ngb": 32, "n_freq_src": 8, "rec_shared_bin": 0}, "box_off": [0, 1000]}
    st = {"moving_packets": 5000, "senders": 300}
    m = bench.hop_loop_model(st, wl, 2.0)
    B = 40 * 5000 + (256 + 20 + 144) * 300 + (100 + 72) * 1000
    assert m["bytes_per_step"] == B
    assert np.isclose(m["achieved"], B / 2e-3 / 1e9) and np.isclose(m["frac"], m["achieved"] / 8000)


def test_accuracy_bars_and_routing_count():
    from paper_1311_0182_gb300 import accuracy as A
    ref = {"x_HI": np.array([0.5, 5e-5, 0.9, 0.2]), "T": np.array([1e4, 1e4, 100.0, 300.0])}
    got = {"x_HI": np.array([0.5004, 5e-5 + 2e-7, 0.9, 0.2]), "T": np.array([1e4, 1e4, 100.2, 300.0])}
    assert A.xhi_ok(got["x_HI"], ref["x_HI"]).tolist() == [True, False, True, True]
    assert A.state_ok(got, ref).tolist() == [True, False, False, True]
    NH = np.full(4, 1e55)                  # floors: 1e43 photons, 1e47 eV
    Ao = np.array([1e50, 1e50, 1e50, 0.0])
    Eo = Ao * 5 * A.EV
    # photons 0.2% off; 0.01% off; nothing off; energy off by half the energy floor
    Ag = np.array([1.002e50, 1e50 + 1e46, 1e50, 0.0])
    Eg = Eo + np.array([0.0, 0.0, 0.0, 0.5e-8 * A.EV * 1e55])
    aff = A.mark_routing_affected(Ag, Ao, Eg, Eo, NH, np.zeros(4, bool))
    assert aff.tolist() == [True, False, False, False]
    s = A.summary(got, ref, aff)
    assert s["routing_affected"] == 1 and s["off_bars"] == 2 and s["off_bars_not_affected"] == 2
