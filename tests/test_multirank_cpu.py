"""The N > 1 path on the CPU: two gloo ranks with host-only contexts.

One contraction is shared out over the ranks by charge sectors (ytn_plan_shard):
every rank plans its part from the same structure, with no data-path collective.
The union of the parts' output blocks must be the single-rank plan's output, bit for
bit, with no block twice; the useful FLOPs must add up and be balanced within 5%.
The only collective of the timed path is the MAX of the step time; the whole-job
value is the whole contraction's FLOPs / the slowest rank's time (strong scaling).
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


def _shard_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_2405_12196_gb300 import ytn
    dist.init_process_group("gloo", init_method="env://")
    w, r, _ = bench.rank_env()
    cfg = bench.make_workload("cfg3", 0)          # the same problem on every rank
    ctx = ytn.ytn_ctx_create(-1)
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"], shard=(r, w))
    mine = {"rank": r, "flops": plan.info["useful_flops"], "nsectors": plan.info["nsectors"],
            "t": plan.out["t"].tolist(), "D": plan.out["D"].tolist()}
    parts = [None] * w
    dist.all_gather_object(parts, mine)
    total = bench.sum_over_ranks(plan.info["useful_flops"], torch.device("cpu"))
    t = 0.010 * (1 + r)                       # rank-dependent step time
    tmax = bench.max_over_ranks(t, torch.device("cpu"))
    out.put((r, parts, total, tmax, bench.strong_value(total, 5, tmax)))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_share_one_contraction_by_sectors():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    from paper_2405_12196_gb300 import ytn
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    parts = res[0][1]
    assert parts == res[1][1]
    cfg = bench.make_workload("cfg3", 0)
    full = ytn.ytn_plan(ytn.ytn_ctx_create(-1), ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    F = full.info["useful_flops"]
    # every output block exactly once, with its dimensions
    got = {}
    for pt in parts:
        for t, d in zip(pt["t"], pt["D"]):
            key = tuple(map(tuple, t))
            assert key not in got
            got[key] = tuple(d)
    want = {tuple(map(tuple, t)): tuple(d) for t, d in zip(full.out["t"].tolist(), full.out["D"].tolist())}
    assert got == want
    # each part's blocks in canonical (ascending) order
    for pt in parts:
        keys = [tuple(np.ravel(t)) for t in pt["t"]]
        assert keys == sorted(keys)
    flops = [pt["flops"] for pt in parts]
    assert sum(flops) == pytest.approx(F, rel=1e-12)
    assert max(flops) <= 1.05 * F / 2
    for r, _, total, tmax, value in res:
        assert total == pytest.approx(F, rel=1e-12)
        assert tmax == pytest.approx(0.020)
        assert value == pytest.approx(F * 5 / 0.020 / 1e12)


def test_shards_of_one_rank_are_the_whole_plan():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2405_12196_gb300 import ytn
    cfg = bench.make_workload("cfg3", 0)
    ctx = ytn.ytn_ctx_create(-1)
    full = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    one = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"], shard=(0, 1))
    assert one.handle == full.handle
    np.testing.assert_array_equal(one.out["t"], full.out["t"])
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"], shard=(2, 2))
    assert e.value.name == "YTN_E_INVALID"
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(ctx, ytn.YTN_OP_FUSE, cfg["A"], groups=((0, 1), (2,), (3,)), shard=(0, 2))
    assert e.value.name == "YTN_E_INVALID"


@pytest.mark.parametrize("world", [3, 8])
def test_partition_of_the_d20_contraction(world):
    """The D = 20 environment contraction over 3 and 8 ranks: every block once, the
    FLOPs balanced within 5% (its largest sector alone is 11% of the whole)."""
    sys.path.insert(0, ROOT)
    import workloads as W
    from paper_2405_12196_gb300 import ytn
    cfg = W.config5()
    ctx = ytn.ytn_ctx_create(-1)
    full = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    F = full.info["useful_flops"]
    blocks, flops, nsec = [], [], 0
    for r in range(world):
        p = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"], shard=(r, world))
        blocks += [tuple(x.ravel()) for x in p.out["t"]]
        flops.append(p.info["useful_flops"])
        nsec += p.info["nsectors"]
        p.release()
    assert len(blocks) == len(set(blocks)) == full.out["t"].shape[0]
    assert set(blocks) == {tuple(x.ravel()) for x in full.out["t"]}
    assert sum(flops) == pytest.approx(F, rel=1e-12)
    assert max(flops) <= 1.05 * F / world
    if world == 8:   # sectors above a quarter of a rank's share, cut by rows, land on several ranks
        assert nsec > full.info["nsectors"]


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload, warmup, steps, ref_budget, gpus = "cfg3", 0, 1, 0.1, 2
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
