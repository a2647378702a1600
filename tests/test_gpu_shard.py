"""One contraction shared out over ranks by charge sectors (ytn_plan_shard), run on
one GPU part after part, through the C ABI: the parts' output blocks together are
the whole result, bit for bit equal to the single plan's (each output element is
computed the same way in both), and match the oracle."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import FP64_RTOL, oracle_tensordot, rel_frobenius

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _run(ctx, plan, da, db, prec, rtol):
    import torch
    from paper_2405_12196_gb300 import ytn
    n = plan.out["size"]
    dc = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device=da.device)
    ws = torch.empty(max(ytn.ytn_workspace_size(plan, prec, rtol), 1), dtype=torch.uint8, device=da.device)
    ytn.ytn_tensordot(plan, da, db, dc, prec=prec, rtol=rtol, workspace=ws)
    ytn.ytn_sync(ctx)
    return dc[:n].cpu().numpy()


def _blocks(rec, data):
    sizes = np.prod(rec["D"], axis=1)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64) if rec.get("off") is None else rec["off"]
    return {tuple(np.ravel(t)): data[o:o + s] for t, o, s in zip(rec["t"], offs, sizes)}


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("split", [False, True])
def test_shards_reassemble_the_whole_result(ctx, world, split):
    import torch
    from paper_2405_12196_gb300 import ytn
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    cfg = W.config3()
    dl = cfg["dleg"]
    a = W.random_tensor((0, 0), [W.Leg(-1, dl.t, dl.D), W.Leg(1, dl.t, dl.D), W.Leg(1, dl.t, dl.D),
                                 W.Leg(-1, dl.t, dl.D)], (0, 0), 3999)
    A, B, axa, axb = cfg["X2"], a, (1, 2), (0, 1)
    dev = torch.device("cuda:0")
    da, db = torch.from_numpy(A["data"]).to(dev), torch.from_numpy(B["data"]).to(dev)
    full = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    whole = _blocks(full.out, _run(ctx, full, da, db, prec, rtol))
    got = {}
    for r in range(world):
        p = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb, shard=(r, world))
        part = _blocks(p.out, _run(ctx, p, da, db, prec, rtol))
        assert not set(part) & set(got)
        got.update(part)
    assert set(got) == set(whole)
    for k in whole:
        np.testing.assert_array_equal(got[k], whole[k])
    ref = oracle_tensordot(A, B, axa, axb)
    want = _blocks(ref, np.asarray(ref["data"]))
    g = np.concatenate([got[k] for k in sorted(want)])
    w = np.concatenate([want[k] for k in sorted(want)])
    assert rel_frobenius(g, w) <= (1e-10 if split else FP64_RTOL)
