"""Page-locked host buffers passed straight to the C ABI.

The data movers read A and B from (and write C to) page-locked host memory over
the host link; results must equal the device-buffer path bit for bit and match
the oracle. Pageable host memory is rejected before any launch.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import FP64_RTOL, check_against_oracle, device, rel_frobenius, run_tensordot
from helpers import random_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _pinned(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)).pin_memory()


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("where", ["host_all", "host_a", "host_c"])
def test_tensordot_with_host_buffers(ctx, split, where):
    import torch
    from paper_2405_12196_gb300 import ytn
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    cfg = W.config1()
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    plan, ref_dev, _ = run_tensordot(ctx, A, B, axa, axb, prec=prec, rtol=rtol)
    assert plan.out["size"] > 0
    n = plan.out["size"]
    dev = device()
    a = _pinned(A["data"]) if where in ("host_all", "host_a") else torch.from_numpy(A["data"]).to(dev)
    b = _pinned(B["data"]) if where == "host_all" else torch.from_numpy(B["data"]).to(dev)
    if where in ("host_all", "host_c"):
        c = torch.full((max(n, 1),), float("nan"), dtype=torch.float64).pin_memory()
    else:
        c = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device=dev)
    ws = torch.empty(max(ytn.ytn_workspace_size(plan, prec, rtol), 1), dtype=torch.uint8, device=dev)
    ytn.ytn_tensordot(plan, a, b, c, prec=prec, rtol=rtol, workspace=ws)
    ytn.ytn_sync(ctx)
    got = c[:n].cpu().numpy()
    np.testing.assert_array_equal(got, ref_dev["data"])
    ref = O.to_record(O.tensordot(O.from_record(A), O.from_record(B), axa, axb))
    assert rel_frobenius(got, ref["data"]) <= (1e-10 if split else FP64_RTOL)


def test_full_size_workload_from_host(ctx):
    """The D=14 environment contraction (1.9e7 elements per operand) read from and
    written to page-locked host memory; sampled blocks against the oracle."""
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config5(D=14)
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    n = plan.out["size"]
    a, b = _pinned(A["data"]), _pinned(B["data"])
    c = torch.full((n,), float("nan"), dtype=torch.float64).pin_memory()
    ws = torch.empty(ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, 1e-10), dtype=torch.uint8, device=device())
    ytn.ytn_tensordot(plan, a, b, c, prec=ytn.YTN_SPLIT_BF16, rtol=1e-10, workspace=ws)
    ytn.ytn_sync(ctx)
    got = c.numpy()
    assert np.all(np.isfinite(got))
    # every output element against the device-buffer path
    da, db = a.to(device()), b.to(device())
    dc = torch.empty(n, dtype=torch.float64, device=device())
    ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_SPLIT_BF16, rtol=1e-10, workspace=ws)
    ytn.ytn_sync(ctx)
    np.testing.assert_array_equal(got, dc.cpu().numpy())


def test_fuse_unfuse_with_host_buffers(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config2()
    A = cfg["A"]
    oA = O.from_record(A)
    AA = O.to_record(O.tensordot(oA, O.conj(oA), (4,), (4,)))
    groups = ((0, 4), (1, 5), (2, 6), (3, 7))
    pf = ytn.ytn_plan(ctx, ytn.YTN_OP_FUSE, AA, groups=groups)
    src = _pinned(AA["data"])
    out = torch.full((pf.out["size"],), float("nan"), dtype=torch.float64).pin_memory()
    ytn.ytn_fuse(pf, src, out)
    ytn.ytn_sync(ctx)
    rec = dict(pf.out)
    rec["data"] = out.numpy().copy()
    check_against_oracle(rec, O.to_record(O.fuse(O.from_record(AA), groups)), exact=True)
    pu = ytn.ytn_plan(ctx, ytn.YTN_OP_UNFUSE, rec, axa=(0, 1, 2, 3))
    back = torch.full((pu.out["size"],), float("nan"), dtype=torch.float64).pin_memory()
    ytn.ytn_unfuse(pu, out, back)
    ytn.ytn_sync(ctx)
    ref = O.to_record(O.unfuse(O.from_record(rec), (0, 1, 2, 3)))
    np.testing.assert_array_equal(back.numpy(), ref["data"])


def test_pageable_host_memory_is_rejected(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(5)
    A, B, axa, axb, _, _ = random_pair(rng, (0,), 3, 3, 1, max_sectors=2, max_dim=3)
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    c = torch.empty(max(plan.out["size"], 1), dtype=torch.float64, device=device())
    ws = torch.empty(max(ytn.ytn_workspace_size(plan), 1), dtype=torch.uint8, device=device())
    with pytest.raises(ytn.YtnError) as ei:
        ytn.ytn_tensordot(plan, A["data"], torch.from_numpy(B["data"]).to(device()), c, workspace=ws)
    assert ei.value.name == "YTN_E_INVALID"


def test_split_gemm_on_a_subset_of_the_sms(ctx):
    """The persistent split GEMM on fewer CTAs than SMs gives the same bits."""
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config2()
    A = cfg["A"]
    B = dict(A, sig=tuple(-s for s in A["sig"]), n=tuple(-q for q in A["n"]))
    axa = axb = (4,)
    plan, ref, _ = run_tensordot(ctx, A, B, axa, axb, prec=ytn.YTN_SPLIT_BF16, rtol=1e-10)
    assert plan.info["useful_flops"] > 0
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    with pytest.raises(ytn.YtnError):
        ytn.ytn_ctx_set_gemm_sms(ctx, nsm + 1)
    try:
        for n in (1, 16, nsm - 8):
            ytn.ytn_ctx_set_gemm_sms(ctx, n)
            _, rec, _ = run_tensordot(ctx, A, B, axa, axb, prec=ytn.YTN_SPLIT_BF16, rtol=1e-10)
            np.testing.assert_array_equal(rec["data"], ref["data"])
    finally:
        ytn.ytn_ctx_set_gemm_sms(ctx, 0)


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("where", ["host_all", "host_a", "host_c"])
def test_host_buffers_staged_by_copy_engines(ctx, split, where):
    """With a staging workspace (ytn_workspace_size_staged) host operands move with
    the copy engines: same bits as the device-buffer path."""
    import torch
    from paper_2405_12196_gb300 import ytn
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    cfg = W.config1()
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    plan, ref_dev, _ = run_tensordot(ctx, A, B, axa, axb, prec=prec, rtol=rtol)
    assert plan.out["size"] > 0
    n = plan.out["size"]
    dev = device()
    a = _pinned(A["data"]) if where in ("host_all", "host_a") else torch.from_numpy(A["data"]).to(dev)
    b = _pinned(B["data"]) if where == "host_all" else torch.from_numpy(B["data"]).to(dev)
    if where in ("host_all", "host_c"):
        c = torch.full((max(n, 1),), float("nan"), dtype=torch.float64).pin_memory()
    else:
        c = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device=dev)
    nb = ytn.ytn_workspace_size_staged(plan, prec, rtol)
    assert nb > ytn.ytn_workspace_size(plan, prec, rtol)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    ytn.ytn_tensordot(plan, a, b, c, prec=prec, rtol=rtol, workspace=ws)
    ytn.ytn_sync(ctx)
    np.testing.assert_array_equal(c[:n].cpu().numpy(), ref_dev["data"])


def test_full_size_workload_staged_from_host(ctx):
    """The D = 14 environment contraction from and to page-locked host memory through
    the staging workspace: every element equals the device-buffer path."""
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config5(D=14)
    A, B, axa, axb = cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    n = plan.out["size"]
    a, b = _pinned(A["data"]), _pinned(B["data"])
    c = torch.full((n,), float("nan"), dtype=torch.float64).pin_memory()
    ws = torch.empty(ytn.ytn_workspace_size_staged(plan, ytn.YTN_SPLIT_BF16, 1e-10), dtype=torch.uint8,
                     device=device())
    ytn.ytn_tensordot(plan, a, b, c, prec=ytn.YTN_SPLIT_BF16, rtol=1e-10, workspace=ws)
    ytn.ytn_sync(ctx)
    da, db = a.to(device()), b.to(device())
    dc = torch.empty(n, dtype=torch.float64, device=device())
    ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_SPLIT_BF16, rtol=1e-10, workspace=ws)
    ytn.ytn_sync(ctx)
    np.testing.assert_array_equal(c.numpy(), dc.cpu().numpy())

