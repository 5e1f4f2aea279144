"""rt_get_cone_masks_noalloc: the cone masks without any device allocation.

Callers that must not allocate device memory -- code that runs under a memory budget or pool
owned by someone else, or a host thread that may not call cudaMalloc/cudaFree while other GPU
work is in flight -- get the masks assembled in a fixed file-scope device array instead of a
temporary buffer.  This checks, through the C ABI, that two calls in a row return exactly what
the allocating rt_get_cone_masks returns (masks are integers: exact equality), on a larger and
then a smaller context (the shared array keeps the previous call's contents), into host and
into device memory, and that a size beyond the array's capacity is refused.
"""
import numpy as np
import pytest

from paper_1311_0182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_0182_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _context_with_packets(wl, seed, fp32):
    from paper_1311_0182_gb300 import rt
    wl = dict(wl, params=dict(wl["params"], transport_fp32=fp32))
    g = rt.context_for(wl)
    rng = np.random.default_rng(seed)
    f = np.zeros((6, g.n, g.S))
    on = rng.random((g.n, g.S)) < 0.3
    N = np.where(on, 10 ** rng.uniform(44, 50, (g.n, g.S)), 0.0)
    d = rng.normal(size=(3, g.n, g.S))
    d /= np.linalg.norm(d, axis=0)
    f[0] = N
    f[1:4] = N * d
    g.assign_cones(seed)
    g.set_slots(f)
    g.assign_cones(seed)
    return g


@pytest.mark.parametrize("fp32", [1, 0])
def test_noalloc_masks_equal_the_allocating_entry_point(fp32):
    import torch
    for seed, wl in ((3, W.cfg2(n_side=20)), (4, W.cfg1())):
        g = _context_with_packets(wl, seed, fp32)
        ref = g.cone_masks()
        assert (ref != 0).mean() > 0.05
        first = g.cone_masks_noalloc()
        second = g.cone_masks_noalloc()
        assert np.array_equal(first, ref)
        assert np.array_equal(second, ref)
        dev = torch.zeros((g.n, g.S), dtype=torch.int32, device="cuda")
        g.cone_masks_noalloc(out=dev)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy().view(np.uint32), ref)
        g.close()


def test_noalloc_refuses_sizes_beyond_its_array():
    from paper_1311_0182_gb300 import rt
    g = rt.context_for(W.cfg2(n_side=28))      # 21952 particles x 288 slots > 4194304
    with pytest.raises(rt.RTError) as e:
        g.cone_masks_noalloc()
    assert e.value.status == 1
    assert "static scratch" in str(e.value)
