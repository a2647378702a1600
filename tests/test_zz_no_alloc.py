"""The allocation-free contraction entry point, through the C ABI.

ytn_tensordot_noalloc serves callers that cannot allocate device memory (for
instance code inside a host application that reserves all device memory for its
own pool): it runs the FP64 contraction with the library's static 64 MiB scratch
instead of a workspace from the caller. Its results must match ytn_tensordot's
within the FP64 tolerance of the other tests, on consecutive calls (the scratch
keeps the previous call's contents, so a stale value would show up on the second
call). This file is collected last and needs no state from other tests.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12


def _rel(got, want):
    n = np.linalg.norm(want)
    return float(np.linalg.norm(got - want) / n) if n else float(np.linalg.norm(got))


def test_noalloc_matches_tensordot_on_consecutive_calls():
    import torch
    from paper_2405_12196_gb300 import ytn
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    dev = torch.device("cuda:0")
    ctx = ytn.ytn_ctx_create(0)
    cfg = W.config1()
    q = [(0, 0), (1, 0), (0, 1), (-1, 1)]
    legs = [W.Leg(1, q, [3, 4, 2, 5]), W.Leg(-1, q, [2, 6, 3, 1]), W.Leg(1, q, [4, 2, 5, 3]),
            W.Leg(-1, q, [1, 3, 2, 4])]
    A = W.random_tensor((0, 0), legs, (0, 0), 11)
    assert A["t"].shape[0] >= 12
    # drop every third block so that the sector matrices need zero fill
    keep = np.arange(A["t"].shape[0]) % 3 != 2
    off = np.concatenate([[0], np.cumsum(np.prod(A["D"], axis=1))])
    A = dict(A, t=A["t"][keep], D=A["D"][keep],
             data=np.concatenate([A["data"][off[i]:off[i + 1]] for i in np.nonzero(keep)[0]]))
    B = W.random_tensor((0, 0), [legs[2].conj(), legs[3].conj(), legs[0].conj()], (0, 0), 12)
    cases = [(cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]), (A, B, (2, 3), (0, 1))]
    for Ar, Br, axa, axb in cases * 2:
        plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, Ar, Br, axa, axb)
        da = torch.from_numpy(Ar["data"]).to(dev)
        db = torch.from_numpy(Br["data"]).to(dev)
        n = max(plan.out["size"], 1)
        ref = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        ws = torch.empty(max(ytn.ytn_workspace_size(plan, ytn.YTN_FP64), 1), dtype=torch.uint8, device=dev)
        ytn.ytn_tensordot(plan, da, db, ref, prec=ytn.YTN_FP64, workspace=ws)
        want = ref.cpu().numpy()[:plan.out["size"]]
        for _ in range(2):
            out = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
            ytn.ytn_tensordot_noalloc(plan, da, db, out)
            ytn.ytn_sync(ctx)
            got = out.cpu().numpy()[:plan.out["size"]]
            assert np.all(np.isfinite(got))
            assert _rel(got, want) <= FP64_RTOL


def test_noalloc_host_buffers_and_side_stream_match_the_oracle():
    """Page-locked host A, B and C (staged through the static array beside the
    workspace) and a call on a non-default stream, each compared with the oracle and
    with ytn_tensordot on device buffers."""
    import torch
    import oracle as O
    from paper_2405_12196_gb300 import ytn
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    dev = torch.device("cuda:0")
    ctx = ytn.ytn_ctx_create(0)
    cfg = W.config1()
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    n = plan.out["size"]
    assert ytn.ytn_workspace_size_staged(plan, ytn.YTN_FP64, 0.0) < 64 << 20
    want = O.to_record(O.tensordot(O.from_record(A), O.from_record(B), axa, axb))["data"]
    da = torch.from_numpy(A["data"]).to(dev)
    db = torch.from_numpy(B["data"]).to(dev)
    ref = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    ws = torch.empty(max(ytn.ytn_workspace_size(plan, ytn.YTN_FP64), 1), dtype=torch.uint8, device=dev)
    ytn.ytn_tensordot(plan, da, db, ref, prec=ytn.YTN_FP64, workspace=ws)
    ytn.ytn_sync(ctx)
    ref = ref.cpu().numpy()
    ha = torch.from_numpy(A["data"].copy()).pin_memory()
    hb = torch.from_numpy(B["data"].copy()).pin_memory()
    for _ in range(2):
        hc = torch.full((n,), float("nan"), dtype=torch.float64).pin_memory()
        ytn.ytn_tensordot_noalloc(plan, ha, hb, hc)
        ytn.ytn_sync(ctx)
        got = hc.numpy().copy()
        assert np.all(np.isfinite(got))
        assert _rel(got, want) <= FP64_RTOL
        np.testing.assert_array_equal(got, ref)
    side = torch.cuda.Stream(device=dev)
    out = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    ytn.ytn_tensordot_noalloc(plan, da, db, out, stream=side)
    ytn.ytn_sync(ctx, stream=side)
    got = out.cpu().numpy()
    assert _rel(got, want) <= FP64_RTOL
    np.testing.assert_array_equal(got, ref)


def test_noalloc_rejects_other_plan_kinds():
    import torch
    from paper_2405_12196_gb300 import ytn
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    ctx = ytn.ytn_ctx_create(0)
    A = W.config1()["A"]
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_FUSE, A, groups=((0, 1), (2,)))
    dev = torch.device("cuda:0")
    da = torch.from_numpy(A["data"]).to(dev)
    out = torch.empty(max(plan.out["size"], 1), dtype=torch.float64, device=dev)
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_tensordot_noalloc(plan, da, da, out)
    assert e.value.name == "YTN_E_INVALID"


def test_noalloc_rejects_contractions_beyond_its_scratch():
    import torch
    from paper_2405_12196_gb300 import ytn
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    ctx = ytn.ytn_ctx_create(0)
    l = W.Leg(1, [(0,)], [2000])
    A = W.random_tensor((0,), [l, l.conj()], (0,), 1, fill="ones")
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, A, (1,), (0,))
    assert ytn.ytn_workspace_size(plan, ytn.YTN_FP64) > 64 << 20
    dev = torch.device("cuda:0")
    da = torch.from_numpy(A["data"]).to(dev)
    out = torch.empty(plan.out["size"], dtype=torch.float64, device=dev)
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_tensordot_noalloc(plan, da, da, out)
    assert e.value.name == "YTN_E_WORKSPACE"
