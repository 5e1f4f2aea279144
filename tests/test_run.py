"""The JSON-lines run driver: its host diagnostics on CPU, and a short logged run with a
checkpoint and a resume on the GPU."""
import io
import json

import numpy as np
import pytest

from paper_1311_0182_gb300 import run as R
from paper_1311_0182_gb300 import workloads as W


def test_front_and_ionised_fraction_of_a_sharp_sphere():
    """A sphere of radius 0.3 fully ionised inside a neutral box: the front lies within one
    shell of 0.3, and the ionised volume fraction is the sphere's share of the volume."""
    rng = np.random.default_rng(2)
    pos = rng.uniform(-0.5, 0.5, size=(200000, 3))
    r = np.linalg.norm(pos, axis=1)
    x = np.where(r < 0.3, 1e-4, 1.0)
    f = R.front_radius(r, x, 0.5)
    assert f is not None and abs(f - 0.3) < 0.5 / 32
    ones = np.ones_like(r)
    assert abs(R.ionised_fraction(x, ones, ones) - 4 / 3 * np.pi * 0.3 ** 3) < 0.005
    # volume weights: particles of twice the volume inside count twice
    assert abs(R.ionised_fraction(x, ones, np.where(r < 0.3, 2.0, 1.0)) -
               2 * 0.1131 / (1 + 0.1131)) < 0.01
    assert R.front_radius(r, np.ones_like(r), 0.5) is None


@pytest.mark.gpu
def test_logged_run_with_checkpoint_and_resume(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    wl = W.cfg1(n_side=12)
    out = io.StringIO()
    R.run(wl, 4, profile_every=2, checkpoint_every=2, checkpoint_dir=str(tmp_path), out=out)
    lines = [json.loads(s) for s in out.getvalue().splitlines()]
    assert [d["step"] for d in lines] == [0, 1, 2, 3]
    assert all(d["closure"] < 1e-9 for d in lines)
    assert lines[-1]["ionised_volume_fraction"] > lines[0]["ionised_volume_fraction"] > 0
    assert "profile" in lines[1] and len(lines[1]["profile"]["x_HI"]) == 32
    # resume from the checkpoint after step 1: steps 2 and 3 repeat the uninterrupted run
    out2 = io.StringIO()
    from paper_1311_0182_gb300 import rt
    ctx = rt.context_for(wl)
    ctx.load_state(open(lines[1]["checkpoint"], "rb").read())
    R.run(wl, 2, start=2, ctx=ctx, out=out2)
    again = [json.loads(s) for s in out2.getvalue().splitlines()]
    for a, b in zip(again, lines[2:]):
        for k in ("hops", "virtual", "budget", "ionised_volume_fraction", "front_kpc"):
            assert a[k] == b[k], k


def test_shadow_profiles_in_cylindrical_shells():
    """Sec. 4 diagnostic on the oracle's shadow run (16^3, 14 steps: the front has passed the
    barrier): in cylindrical shells around the shadow's axis, behind the barrier, no source
    photons reach the shells inside the barrier's radius, where the gas stays neutral and cold,
    while outside it the source intensity is that of the outer shell and the gas is ionised
    and hot."""
    import oracle
    wl = W.shadow(n_side=16, n_front=20, n_bnd=10)
    s = oracle.Sim(wl)
    s.build_neighbours()
    for k in range(14):
        assert s.step(k) == 0
    _, _, ps = s.deposits()
    pr = R.shadow_profiles(wl, s.state(), ps, wl["params"]["dt"], n_shells=8)
    e = np.array(pr["edges"])
    rb = pr["barrier_radius"]
    # shells more than a smoothing length (~0.1 of the side at 16^3) inside or outside the
    # shadow's edge
    shadow = e[1:] <= 0.65 * rb
    lit = e[:-1] >= 1.2 * rb
    assert shadow.sum() >= 2 and lit.sum() >= 3
    Is, x, T = (np.array(pr[k], dtype=float) for k in ("I_source", "x_HI", "T"))
    assert np.all(Is[shadow] < 0.05) and np.all(Is[lit] > 0.5)
    assert np.all(x[shadow] > 0.9) and np.all(x[lit] < 0.5)
    assert T[shadow].max() < 0.1 * T[lit].min()
    assert sum(pr["count"]) > 0 and pr["I_source"][-1] == 1.0
