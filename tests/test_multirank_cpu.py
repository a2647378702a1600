"""The N > 1 path of bench.py on the CPU: two gloo ranks.

Every rank contracts its own problem (same structure, its own seeds: weak
scaling, no data-path collective); the only collective is the MAX of the step
time, and the whole-job value is world x per-rank FLOPs / slowest time.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_2405_12196_gb300 import ytn
    dist.init_process_group("gloo", init_method="env://")
    w, r, lr = bench.rank_env()
    assert (w, r, lr) == (world, rank, rank)
    cfg = bench.make_workload("cfg3", r)
    ctx = ytn.ytn_ctx_create(-1)
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    flops = plan.info["useful_flops"]
    mine = torch.tensor([flops, float(np.sum(cfg["A"]["data"][:1000]))], dtype=torch.float64)
    allv = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allv, mine)
    t = 0.010 * (1 + r)                       # rank-dependent step time
    tmax = bench.max_over_ranks(t, torch.device("cpu"))
    value = bench.weak_value(flops, 5, w, tmax)
    out.put((r, [v.tolist() for v in allv], tmax, value, flops))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_weak_scaling():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (_, allv0, tmax0, value0, flops0), (_, allv1, tmax1, value1, flops1) = res
    # same structure (same useful FLOPs), different data (own seeds)
    assert allv0 == allv1
    assert allv0[0][0] == allv0[1][0] == flops0 == flops1
    assert allv0[0][1] != allv0[1][1]
    # the slowest rank's time, and the whole-job value from it
    assert tmax0 == tmax1 == pytest.approx(0.020)
    assert value0 == value1 == pytest.approx(2 * flops0 * 5 / 0.020 / 1e12)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload, warmup, steps, ref_budget, gpus = "cfg3", 0, 1, 0.1, 2
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
