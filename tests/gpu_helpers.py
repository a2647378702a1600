"""Helpers of the GPU parity tests: run the library through its C ABI on device
buffers, compare with the oracle. Imports torch and the binding lazily."""
import numpy as np

import oracle as O
import workloads as W

# FP64 path tolerance (relative Frobenius error against the oracle).
FP64_RTOL = 1e-12


def device():
    import torch
    return torch.device("cuda:0")


def to_dev(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)).to(device())


def run_tensordot(ctx, A, B, axa, axb, prec=None, rtol=0.0):
    """C = tensordot(A, B) on the GPU; returns (plan, C record with data, result)."""
    import torch
    from paper_2405_12196_gb300 import ytn
    prec = ytn.YTN_FP64 if prec is None else prec
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    da, db = to_dev(A["data"]), to_dev(B["data"])
    out = plan.out
    dc = torch.full((max(out["size"], 1),), float("nan"), dtype=torch.float64, device=device())
    nbytes = ytn.ytn_workspace_size(plan, prec, rtol)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device())
    res = ytn.ytn_tensordot(plan, da, db, dc, prec=prec, rtol=rtol, workspace=ws)
    ytn.ytn_sync(ctx)
    if res["precision"] == ytn.YTN_SPLIT_BF16:
        res["report"] = ytn.ytn_tensordot_report(plan, ws)   # the device's data-aware estimate
    rec = dict(out)
    rec["data"] = dc[:out["size"]].cpu().numpy()
    return plan, rec, res


def run_move(ctx, kind, A, **kw):
    import torch
    from paper_2405_12196_gb300 import ytn
    plan = ytn.ytn_plan(ctx, kind, A, **kw)
    da = to_dev(A["data"])
    out = plan.out
    dc = torch.full((max(out["size"], 1),), float("nan"), dtype=torch.float64, device=device())
    fn = {ytn.YTN_OP_FUSE: ytn.ytn_fuse, ytn.YTN_OP_UNFUSE: ytn.ytn_unfuse,
          ytn.YTN_OP_TRACE: ytn.ytn_trace}[kind]
    fn(plan, da, dc)
    ytn.ytn_sync(ctx)
    rec = dict(out)
    rec["data"] = dc[:out["size"]].cpu().numpy()
    return plan, rec


def same_structure(rec, ref):
    assert rec.get("dtype", "f64") == ref.get("dtype", "f64")
    assert tuple(rec["sig"]) == tuple(ref["sig"])
    assert tuple(rec["n"]) == tuple(ref["n"])
    np.testing.assert_array_equal(rec["t"], np.asarray(ref["t"]).reshape(rec["t"].shape))
    np.testing.assert_array_equal(rec["D"], np.asarray(ref["D"]).reshape(rec["D"].shape))
    assert rec["size"] == np.asarray(ref["data"]).size


def rel_frobenius(got, want):
    got = np.asarray(got)     # real or complex
    want = np.asarray(want)
    nw = np.linalg.norm(want)
    if nw == 0.0:
        return float(np.linalg.norm(got))
    return float(np.linalg.norm(got - want) / nw)


def check_against_oracle(rec, ref, rtol=FP64_RTOL, exact=False):
    same_structure(rec, ref)
    assert np.all(np.isfinite(rec["data"])), "unwritten output elements"
    if exact:
        np.testing.assert_array_equal(rec["data"], ref["data"])
    else:
        err = rel_frobenius(rec["data"], ref["data"])
        assert err <= rtol, f"relative Frobenius error {err:.3e} > {rtol:.1e}"
        return err


def oracle_tensordot(A, B, axa, axb):
    return O.to_record(O.tensordot(O.from_record(A), O.from_record(B), axa, axb))
