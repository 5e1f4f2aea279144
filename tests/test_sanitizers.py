"""Host-side ASan/UBSan runs (no GPU needed).

The oracle, and the host code of the C-ABI library's entry file (configuration and option
validation, the direction sets), are rebuilt with -fsanitize=address,undefined and driven in a
child process with the ASan runtime preloaded; any report ends that process with an error.  A
copy of the oracle with one out-of-bounds store planted in it checks that the harness does
report, so a clean run means something.
"""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

from conftest import ROOT

SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _runtime():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                           text=True).stdout.strip()
    except OSError:
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


ASAN = _runtime()
pytestmark = pytest.mark.skipif(ASAN is None, reason="no gcc ASan runtime")


def _run(script, tmp_path, *args):
    path = tmp_path / "drive.py"
    path.write_text(textwrap.dedent(script))
    env = dict(os.environ, LD_PRELOAD=ASAN, PYTHONMALLOC="malloc",
               ASAN_OPTIONS="detect_leaks=0,protect_shadow_gap=0,abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1", PYTHONPATH=ROOT)
    return subprocess.run([sys.executable, str(path), *args], capture_output=True, text=True,
                          env=env, timeout=600)


def _build_oracle(src, out):
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", *SAN, "-o", str(out), str(src), "-lm"])


ORACLE_RUN = """
    import sys
    import oracle
    oracle.build = lambda force=False: sys.argv[1]
    from paper_1311_0182_gb300 import workloads as W
    cases = [(W.cfg1(n_side=10), 3),
             (W.shadow(n_side=12, n_front=10, n_bnd=6), 3),
             (W.cfg1(n_side=10, rec_mode=W.REC_EMISSION_CONES), 3),
             (W.cfg2(n_side=8, rec_shared_bin=1), 2)]
    for wl, steps in cases:
        s = oracle.Sim(wl)
        s.build_neighbours()
        for st in range(steps):
            s.step(st)
        s.budget()
    print("clean")
"""


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    so = tmp_path / "liborc_san.so"
    _build_oracle(os.path.join(ROOT, "oracle", "traphic_oracle.c"), so)
    r = _run(ORACLE_RUN, tmp_path, str(so))
    assert r.returncode == 0 and "clean" in r.stdout, r.stderr[-4000:]


def test_the_harness_reports_a_planted_overflow(tmp_path):
    """One past the end of the rotation array, written in a copy of the oracle on the CPU."""
    src = open(os.path.join(ROOT, "oracle", "traphic_oracle.c")).read()
    good = "for (long long i = 0; i < n; ++i) s->R[9 * i] ="
    assert src.count(good) == 1
    bad = tmp_path / "traphic_oracle.c"
    bad.write_text(src.replace(good, "for (long long i = 0; i <= n; ++i) s->R[9 * i] ="))
    shutil.copy(os.path.join(ROOT, "oracle", "traphic_oracle.h"), tmp_path / "traphic_oracle.h")
    so = tmp_path / "liborc_bad.so"
    _build_oracle(bad, so)
    r = _run(ORACLE_RUN, tmp_path, str(so))
    assert r.returncode != 0
    assert "heap-buffer-overflow" in r.stderr


ABI_RUN = """
    import sys
    import numpy as np
    from paper_1311_0182_gb300 import build as _build, rt, workloads as W
    import oracle
    _build.LIB = sys.argv[1]
    for n in (8, 32):
        assert np.array_equal(rt.axis_set(n), oracle.axis_set(n))
    wl = W.cfg1()

    def status(w):
        try:
            rt.Context(w)
        except rt.RTError as e:
            return e.status
        return 0

    bad = [dict(n_rc=7), dict(n_ngb=33), dict(rec_shared_bin=1, n_freq_src=0),
           dict(rec_shared_bin=2), dict(launch_grid=(0, -1, 0)), dict(cell_occupancy=-3),
           dict(rec_mode=4)]
    assert [status(dict(wl, params=dict(wl["params"], **b))) for b in bad] == [1] * len(bad)
    assert status(dict(wl, box_off=np.array([0, 20]), box_L=np.array([1.0]))) == 5
    assert status(dict(wl, box_off=np.array([0, (1 << 24) + 1]), box_L=np.array([1.0]))) == 1
    print("clean")
"""


def test_abi_host_code_is_clean_under_asan_and_ubsan(tmp_path):
    """The entry file is recompiled with the sanitizers (its host code only: device code is
    unaffected) and linked with the other translation units of the normal build."""
    from paper_1311_0182_gb300 import build
    build.build()
    obj = tmp_path / "rt_api.o"
    flags = [f for f in build.FLAGS if f not in ("-O3", "-Xptxas", "-warn-spills")]
    host = [f for f in flags if f.startswith("-fPIC")]
    assert host, flags
    # nvcc splits -Xcompiler arguments at commas: one flag per sanitizer
    nv_san = ["-fsanitize=address", "-fsanitize=undefined"] + SAN[1:]
    flags[flags.index(host[0])] = host[0] + "," + ",".join(nv_san)
    subprocess.check_call([build.NVCC, *flags, "-O1", "-c",
                           os.path.join(build.CSRC, "rt_api.cu"), "-o", str(obj)])
    others = [os.path.join(build.OUT, s.replace(".cu", ".o")) for s in build.SOURCES
              if s != "rt_api.cu"]
    so = tmp_path / "librt_san.so"
    subprocess.check_call([build.NVCC, *build.ARCH, "-shared", "-Xcompiler",
                           "-fsanitize=address,-fsanitize=undefined", "-o", str(so), str(obj),
                           *others])
    r = _run(ABI_RUN, tmp_path, str(so))
    assert r.returncode == 0 and "clean" in r.stdout, r.stderr[-4000:]
