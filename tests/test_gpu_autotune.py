"""YTN_AUTO: per-plan choice between the FP64 and split paths (ytn_tensordot).

Whatever it picks, the result must meet rtol against the oracle; the choice is
cached on the plan; with rtol below what the split path guarantees it is FP64;
on a large contraction the split path wins; under graph capture the cost
model decides and the replay is correct.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import FP64_RTOL, device, rel_frobenius, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _setup(ctx, cfg, rtol):
    import torch
    from paper_2405_12196_gb300 import ytn
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    n = plan.out["size"]
    da, db = to_dev(A["data"]), to_dev(B["data"])
    dc = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device=device())
    ws = torch.empty(max(ytn.ytn_workspace_size(plan, ytn.YTN_AUTO, rtol), 1), dtype=torch.uint8, device=device())
    return plan, da, db, dc, ws, n


def _cfg1():
    c = W.config1()
    return {"A": c["A"], "B": c["B"], "axa": c["axa"], "axb": c["axb"]}


def test_auto_small_plan_meets_rtol_and_caches(ctx):
    from paper_2405_12196_gb300 import ytn
    cfg = _cfg1()
    ref = O.to_record(O.tensordot(O.from_record(cfg["A"]), O.from_record(cfg["B"]), cfg["axa"], cfg["axb"]))
    plan, da, db, dc, ws, n = _setup(ctx, cfg, 1e-10)
    first = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_AUTO, rtol=1e-10, workspace=ws)
    ytn.ytn_sync(ctx)
    assert first["precision"] == ytn.YTN_SPLIT_BF16        # the timing call leaves the split result
    assert rel_frobenius(dc[:n].cpu().numpy(), ref["data"]) <= 1e-10
    picks = set()
    for _ in range(3):
        dc.fill_(float("nan"))
        r = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_AUTO, rtol=1e-10, workspace=ws)
        ytn.ytn_sync(ctx)
        picks.add(r["precision"])
        assert rel_frobenius(dc[:n].cpu().numpy(), ref["data"]) <= 1e-10
    assert len(picks) == 1                                  # cached


def test_auto_below_split_guarantee_is_fp64(ctx):
    from paper_2405_12196_gb300 import ytn
    cfg = _cfg1()
    ref = O.to_record(O.tensordot(O.from_record(cfg["A"]), O.from_record(cfg["B"]), cfg["axa"], cfg["axb"]))
    plan, da, db, dc, ws, n = _setup(ctx, cfg, 1e-16)
    r = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_AUTO, rtol=1e-16, workspace=ws)
    ytn.ytn_sync(ctx)
    assert r["precision"] == ytn.YTN_FP64 and r["slices"] == 0
    assert rel_frobenius(dc[:n].cpu().numpy(), ref["data"]) <= FP64_RTOL


def test_auto_picks_split_on_a_large_contraction(ctx):
    from paper_2405_12196_gb300 import ytn
    cfg = W.config5(D=14)
    plan, da, db, dc, ws, n = _setup(ctx, cfg, 1e-10)
    ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_AUTO, rtol=1e-10, workspace=ws)
    r = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_AUTO, rtol=1e-10, workspace=ws)
    ytn.ytn_sync(ctx)
    assert r["precision"] == ytn.YTN_SPLIT_BF16 and r["slices"] == 5   # the forecast 128 eta(s) <= 1e-10 first holds at s = 5
    # the first call timed both paths and kept the faster
    t = ytn.ytn_plan_tuning(plan, 5)
    assert t["auto_choice"] == 1 and 0 < t["split_ms"] < t["fp64_ms"]


def test_auto_under_graph_capture_uses_the_model(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    # a context of its own: plans are cached per context, and this plan's choices
    # must still be undecided when the capture starts
    ctx = ytn.ytn_ctx_create(0)
    cfg = W.config3()
    X2 = cfg["X2"]
    dl = cfg["dleg"]
    a = W.random_tensor((0, 0), [W.Leg(-1, dl.t, dl.D), W.Leg(1, dl.t, dl.D), W.Leg(1, dl.t, dl.D),
                                 W.Leg(-1, dl.t, dl.D)], (0, 0), 3002)
    c = {"A": X2, "B": a, "axa": (1, 2), "axb": (0, 1)}
    plan, da, db, dc, ws, n = _setup(ctx, c, 1e-10)
    stream = torch.cuda.Stream(device=device())
    torch.cuda.synchronize()
    ytn.ytn_graph_begin(ctx, stream)
    ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_AUTO, rtol=1e-10, workspace=ws, stream=stream)
    g = ytn.ytn_graph_end(ctx, stream)
    g.launch(stream)
    ytn.ytn_sync(ctx, stream)
    ref = O.to_record(O.tensordot(O.from_record(X2), O.from_record(a), (1, 2), (0, 1)))
    assert rel_frobenius(dc[:n].cpu().numpy(), ref["data"]) <= 1e-10
    # the cost model decided: a choice, no timings
    t = ytn.ytn_plan_tuning(plan, 5)
    assert t["auto_choice"] in (0, 1) and t["fp64_ms"] == 0.0 and t["split_ms"] == 0.0
    g.close()
