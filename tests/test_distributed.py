"""The N > 1 path on CPU: world size 2 over gloo (no GPU)."""
import os
import socket

import numpy as np

from paper_1311_0182_gb300 import distributed as D
from paper_1311_0182_gb300 import workloads as W


def test_partition_is_complete_balanced_and_deterministic():
    rng = np.random.default_rng(0)
    counts = np.exp(rng.uniform(np.log(512), np.log(64000), 512)).astype(int)
    for world in (1, 2, 3, 8):
        parts = D.partition_boxes(counts, world)
        allb = np.sort(np.concatenate(parts))
        assert np.array_equal(allb, np.arange(len(counts)))
        loads = [counts[p].sum() for p in parts]
        assert max(loads) - min(loads) <= counts.max()        # LPT bound
        assert all(np.array_equal(a, b) for a, b in zip(parts, D.partition_boxes(counts, world)))


def test_local_workload_keeps_boxes_and_their_sources():
    wl = W.cfg4(n_boxes=6, n_min=40, n_max=200)
    parts = D.partition_boxes(np.diff(wl["box_off"]), 2)
    tot = 0
    for p in parts:
        sub = D.local_workload(wl, p)
        assert len(sub["box_L"]) == len(p) == len(sub["src_box"])
        assert sub["box_off"][-1] == sum(wl["box_off"][b + 1] - wl["box_off"][b] for b in p)
        tot += sub["box_off"][-1]
        b0 = p[0]
        assert np.array_equal(sub["x"][: wl["box_off"][b0 + 1] - wl["box_off"][b0]],
                              wl["x"][wl["box_off"][b0]: wl["box_off"][b0 + 1]])
    assert tot == wl["box_off"][-1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counts = np.arange(10, 30)
    parts = D.partition_boxes(counts, world)
    mine = parts[rank]
    # each rank "runs" its boxes: a per-box budget row, then the cross-rank reductions
    tally = np.zeros((len(counts), 4))
    tally[mine, 0] = counts[mine]
    total = D.sum_over_ranks(tally)
    t = D.max_over_ranks(float(rank + 1) * 10.0)
    q.put((rank, total.tolist(), t))
    dist.destroy_process_group()


def test_two_rank_gloo_reductions():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    counts = np.arange(10, 30)
    for rank, total, t in out:
        assert np.array_equal(np.array(total)[:, 0], counts)   # every box counted exactly once
        assert t == 20.0                                        # slowest rank


def _oracle_worker(rank, world, port, q):
    """One rank of the partitioned batched run on the CPU: its share of the boxes (LPT) through
    the oracle, 3 steps, then the per-box budgets and the neutral fractions summed over ranks."""
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.cfg4(n_boxes=6, n_min=300, n_max=1200)
    mine = D.partition_boxes(np.diff(wl["box_off"]), world)[rank]
    s = oracle.Sim(D.local_workload(wl, mine))
    s.build_neighbours()
    for k in range(3):
        assert s.step(k) == 0
    budget = np.zeros((len(wl["box_L"]), 4))
    budget[mine] = s.budget()
    x = np.zeros(int(wl["box_off"][-1]))
    idx = np.concatenate([np.arange(wl["box_off"][b], wl["box_off"][b + 1]) for b in mine])
    x[idx] = s.state()["x_HI"]
    q.put((rank, D.sum_over_ranks(budget).tolist(), D.sum_over_ranks(x).tolist()))
    dist.destroy_process_group()


def test_partitioned_boxes_repeat_the_unsplit_run():
    """Workload 4's boxes split over two gloo ranks: each rank runs its boxes (with the
    identities they have in the whole workload) through the oracle; the per-box photon budgets
    and every particle's x_HI, summed over the ranks, equal those of one unsplit run exactly."""
    import torch.multiprocessing as mp
    import oracle
    wl = W.cfg4(n_boxes=6, n_min=300, n_max=1200)
    full = oracle.Sim(wl)
    full.build_neighbours()
    for k in range(3):
        assert full.step(k) == 0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, budget, x in out:
        assert np.array_equal(np.array(budget), full.budget())
        assert np.array_equal(np.array(x), full.state()["x_HI"])
