"""Continuous-batching server (ytn_server_*), through the C ABI.

Each request's result must be the same alone and in the mix; admission must keep
the workspaces of concurrently running requests inside the arena (the HBM
budget); requests that can never fit are rejected.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import rel_frobenius

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _requests(ctx, nruns=6):
    """Independent U(1) environment contractions X2_r . a_r of several sizes."""
    import torch
    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    out = []
    for run in W.serving_runs(nruns=nruns, seed=777, Ds=(4, 6, 8)):
        X2, a = W.serving_request(run)
        plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, X2, a, (1, 2), (0, 1))
        out.append({"plan": plan, "a": torch.from_numpy(X2["data"]).to(dev),
                    "b": torch.from_numpy(a["data"]).to(dev), "n": plan.out["size"]})
    return out


def _alone(ctx, r, prec, rtol):
    import torch
    from paper_2405_12196_gb300 import ytn
    c = torch.full((max(r["n"], 1),), float("nan"), dtype=torch.float64, device=r["a"].device)
    ws = torch.empty(max(ytn.ytn_workspace_size(r["plan"], prec, rtol), 1), dtype=torch.uint8,
                     device=r["a"].device)
    ytn.ytn_tensordot(r["plan"], r["a"], r["b"], c, prec=prec, rtol=rtol, workspace=ws)
    ytn.ytn_sync(ctx)
    return c[:r["n"]].cpu().numpy()


def test_results_same_alone_and_in_the_mix(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    reqs = _requests(ctx)
    precs = [(ytn.YTN_FP64, 0.0), (ytn.YTN_SPLIT_BF16, 1e-10)]
    alone = {(i, k): _alone(ctx, r, p, t) for i, r in enumerate(reqs) for k, (p, t) in enumerate(precs)}
    # arena for about two requests at a time
    need = max(ytn.ytn_workspace_size(r["plan"], p, t) for r in reqs for p, t in precs)
    arena = torch.empty(2 * need + (1 << 20), dtype=torch.uint8, device=reqs[0]["a"].device)
    srv = ytn.Server(ctx, 4, arena)
    outs = {}
    rid = 0
    for rep in range(2):
        for i, r in enumerate(reqs):
            for k, (p, t) in enumerate(precs):
                c = torch.full((max(r["n"], 1),), float("nan"), dtype=torch.float64, device=r["a"].device)
                outs[rid] = (i, k, c)
                srv.submit(rid, r["plan"], r["a"], r["b"], c, prec=p, rtol=t)
                rid += 1
    srv.drain(timeout_ms=120000)
    infos = srv.poll()
    srv.close()
    assert len(infos) == rid
    assert all(x["status"] == 0 for x in infos)
    for rid_, (i, k, c) in outs.items():
        got = c[:reqs[i]["n"]].cpu().numpy()
        tol = 1e-12 if k == 0 else 1e-10
        assert rel_frobenius(got, alone[(i, k)]) <= tol
        np.testing.assert_array_equal(got, alone[(i, k)])   # deterministic kernels: identical bits
    # admission kept the running workspaces inside the arena
    events = sorted([(x["t_admit"], x["workspace"]) for x in infos] + [(x["t_done"], -x["workspace"]) for x in infos],
                    key=lambda e: (e[0], e[1]))
    used = peak = 0
    for _, w in events:
        used += w
        peak = max(peak, used)
    assert peak <= arena.numel()
    assert max(x["slot"] for x in infos) <= 3
    # with two slots' worth of arena and four slots, some requests had to wait
    assert any(x["t_admit"] > x["t_arrive"] + 1e-3 for x in infos)


def test_request_larger_than_the_arena_is_rejected(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    reqs = _requests(ctx, nruns=2)
    r = reqs[0]
    arena = torch.empty(1 << 16, dtype=torch.uint8, device=r["a"].device)
    srv = ytn.Server(ctx, 2, arena)
    c = torch.empty(max(r["n"], 1), dtype=torch.float64, device=r["a"].device)
    assert ytn.ytn_workspace_size(r["plan"], ytn.YTN_FP64) > (1 << 16)
    srv.submit(7, r["plan"], r["a"], r["b"], c)
    srv.drain(timeout_ms=10000)
    infos = srv.poll()
    srv.close()
    assert len(infos) == 1 and infos[0]["id"] == 7
    assert ytn.STATUS[infos[0]["status"]] == "YTN_E_WORKSPACE"
