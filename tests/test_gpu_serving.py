"""Continuous-batching server (ytn_server_*), through the C ABI.

Every request's result is checked against the CPU oracle (block structure bit for
bit, values within 1e-12 on the FP64 path and 1e-10 on the split path), and must be
the same alone and in the mix; admission must keep the workspaces of concurrently
running requests inside the arena (the HBM budget); requests that can never fit are
rejected.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import check_against_oracle, oracle_tensordot, rel_frobenius

pytestmark = pytest.mark.gpu

SPLIT_RTOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _runs(per_d=2):
    """Independent U(1) runs of the serving stream's recipe, ``per_d`` of each of
    D = 4, 6 and 8 (three bond dimensions in one mix)."""
    runs = []
    for i, D in enumerate((4, 6, 8)):
        runs += W.serving_runs(nruns=per_d, seed=777 + i, Ds=(D,))
    return runs


def _requests(ctx, runs):
    """One environment contraction X2_r . a_r per run, with its oracle result."""
    import torch
    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    out = []
    for run in runs:
        X2, a = W.serving_request(run)
        plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, X2, a, (1, 2), (0, 1))
        out.append({"plan": plan, "D": run["D"], "X2": X2, "a_rec": a,
                    "a": torch.from_numpy(X2["data"]).to(dev),
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


def _serve(ctx, reqs, precs, arena_bytes, nslots, reps):
    """Submit every (request, precision) ``reps`` times at once and drain."""
    import torch
    from paper_2405_12196_gb300 import ytn
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device=reqs[0]["a"].device)
    srv = ytn.Server(ctx, nslots, arena)
    outs = {}
    rid = 0
    for _ in range(reps):
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
    return outs, infos, arena.numel()


def test_results_match_the_oracle_alone_and_in_the_mix(ctx):
    from paper_2405_12196_gb300 import ytn
    reqs = _requests(ctx, _runs())
    assert len({r["D"] for r in reqs}) == 3
    precs = [(ytn.YTN_FP64, 0.0), (ytn.YTN_SPLIT_BF16, SPLIT_RTOL)]
    alone = {}
    for i, r in enumerate(reqs):
        ref = oracle_tensordot(r["X2"], r["a_rec"], (1, 2), (0, 1))
        for k, (p, t) in enumerate(precs):
            got = _alone(ctx, r, p, t)
            rec = dict(r["plan"].out)
            rec["data"] = got
            check_against_oracle(rec, ref, rtol=1e-12 if k == 0 else SPLIT_RTOL)
            alone[(i, k)] = got
    # arena for about two requests at a time, four slots: requests queue for memory
    need = max(ytn.ytn_workspace_size(r["plan"], p, t) for r in reqs for p, t in precs)
    outs, infos, arena_bytes = _serve(ctx, reqs, precs, 2 * need + (1 << 20), 4, 2)
    for rid_, (i, k, c) in outs.items():
        got = c[:reqs[i]["n"]].cpu().numpy()
        tol = 1e-12 if k == 0 else SPLIT_RTOL
        assert rel_frobenius(got, alone[(i, k)]) <= tol
        np.testing.assert_array_equal(got, alone[(i, k)])   # deterministic kernels: identical bits
    # admission kept the running workspaces inside the arena
    events = sorted([(x["t_admit"], x["workspace"]) for x in infos] + [(x["t_done"], -x["workspace"]) for x in infos],
                    key=lambda e: (e[0], e[1]))
    used = peak = 0
    for _, w in events:
        used += w
        peak = max(peak, used)
    assert peak <= arena_bytes
    assert max(x["slot"] for x in infos) <= 3
    # with two slots' worth of arena and four slots, some requests had to wait
    assert any(x["t_admit"] > x["t_arrive"] + 1e-3 for x in infos)


def test_mixed_bond_dimensions_and_precisions_in_flight(ctx):
    """Both precisions and three bond dimensions submitted together into a roomy
    arena: results equal the alone runs bit for bit, and requests overlapped."""
    from paper_2405_12196_gb300 import ytn
    reqs = _requests(ctx, _runs(per_d=1))
    precs = [(ytn.YTN_FP64, 0.0), (ytn.YTN_SPLIT_BF16, SPLIT_RTOL)]
    alone = {(i, k): _alone(ctx, r, p, t) for i, r in enumerate(reqs) for k, (p, t) in enumerate(precs)}
    total = sum(ytn.ytn_workspace_size(r["plan"], p, t) for r in reqs for p, t in precs)
    outs, infos, _ = _serve(ctx, reqs, precs, total + (1 << 20), 6, 3)
    for rid_, (i, k, c) in outs.items():
        np.testing.assert_array_equal(c[:reqs[i]["n"]].cpu().numpy(), alone[(i, k)])
    by_id = {x["id"]: x for x in infos}
    kinds = {(reqs[i]["D"], k) for (i, k, _) in outs.values()}
    assert len({d for d, _ in kinds}) == 3 and len({k for _, k in kinds}) == 2
    spans = sorted((by_id[r]["t_admit"], by_id[r]["t_done"]) for r in outs)
    assert any(spans[j + 1][0] < spans[j][1] for j in range(len(spans) - 1)), "no two requests overlapped"


def test_request_larger_than_the_arena_is_rejected(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    reqs = _requests(ctx, W.serving_runs(nruns=2, seed=777, Ds=(4, 6, 8)))
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
