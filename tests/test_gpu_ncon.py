"""Networks through ytn_ncon (the C ABI), against the oracle's ncon.

Random chains, traces and outer products (U(1), Z2, U(1)xU(1)), and the
enlarged corner of a U(1)xU(1) CTMRG step (C.T.T.a, 2.96e10 useful FLOPs) in
FP64 and split precision; page-locked host inputs; label errors.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import FP64_RTOL, check_against_oracle, device, to_dev
from helpers import random_network

pytestmark = pytest.mark.gpu

SYMS = {"U1": (0,), "Z2": (2,), "U1xU1": (0, 0)}


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _run(ctx, ts, labels, prec, rtol, host=False):
    import torch
    from paper_2405_12196_gb300 import ytn
    nc = ytn.ytn_ncon_plan(ctx, ts, labels)
    if host:
        data = [torch.from_numpy(np.ascontiguousarray(t["data"])).pin_memory() for t in ts]
    else:
        data = [to_dev(t["data"]) for t in ts]
    n = nc.out["size"]
    out = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device=device())
    ws = torch.empty(max(ytn.ytn_ncon_workspace_size(nc, prec, rtol), 1), dtype=torch.uint8, device=device())
    ytn.ytn_ncon(nc, data, out, prec=prec, rtol=rtol, workspace=ws)
    ytn.ytn_sync(ctx)
    rec = dict(nc.out)
    rec["data"] = out[:n].cpu().numpy()
    return nc, rec


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("kind", ["chain", "trace", "outer"])
def test_random_networks(ctx, sym, kind):
    from paper_2405_12196_gb300 import ytn
    done = 0
    for case in range(40):
        rng = np.random.default_rng(8700 + 31 * case + len(sym) + len(kind))
        _, ts, labels = random_network(rng, SYMS[sym], kind)
        want = O.to_record(O.ncon([O.from_record(t) for t in ts], labels))
        if want["data"].size == 0 or not np.any(want["data"]):
            continue
        nc, rec = _run(ctx, ts, labels, ytn.YTN_FP64, 0.0)
        check_against_oracle(rec, want)
        done += 1
        if done == 3:
            break
    assert done == 3


@pytest.fixture(scope="module")
def corner():
    ts, labels = W.ctm_corner_network(W.config3())
    return ts, labels, O.to_record(O.ncon([O.from_record(t) for t in ts], labels))


@pytest.mark.parametrize("split", [False, True])
def test_ctm_enlarged_corner(ctx, corner, split):
    from paper_2405_12196_gb300 import ytn
    ts, labels, want = corner
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    nc, rec = _run(ctx, ts, labels, prec, rtol)
    assert nc.info["ncalls"] == 4 and nc.info["useful_flops"] > 2e10
    check_against_oracle(rec, want, rtol=1e-10 if split else FP64_RTOL)


def test_host_inputs_and_label_errors(ctx, corner):
    from paper_2405_12196_gb300 import ytn
    ts, labels, want = corner
    _, rec = _run(ctx, ts, labels, ytn.YTN_FP64, 0.0, host=True)
    check_against_oracle(rec, want)
    for bad in ([[1, 2], [2, 3, -1], [-2, 4, 1], [3, -3, -5, 4]],     # gap in the negative labels
                [[1, 2], [2, 3, -1], [-2, 4, 1], [3, -3, -4, 3]]):    # a label three times
        with pytest.raises(ytn.YtnError) as ei:
            ytn.ytn_ncon_plan(ctx, ts, bad)
        assert ei.value.name == "YTN_E_INVALID"


def test_einsum_front_end_gives_the_ncon_bits(ctx, corner):
    """The enlarged corner from einsum subscripts: the same calls as the ncon labels
    (summed letters numbered by first appearance), so the same bits."""
    import torch
    from paper_2405_12196_gb300 import ytn
    ts, labels, want = corner
    nc = ytn.ytn_einsum_plan(ctx, "pq,qrw,xsp,ryzs->wxyz", ts)
    assert nc.info["ncalls"] == 4
    data = [to_dev(t["data"]) for t in ts]
    out = torch.full((nc.out["size"],), float("nan"), dtype=torch.float64, device=device())
    ws = torch.empty(max(ytn.ytn_ncon_workspace_size(nc), 1), dtype=torch.uint8, device=device())
    ytn.ytn_ncon(nc, data, out, workspace=ws)
    ytn.ytn_sync(ctx)
    rec = dict(nc.out)
    rec["data"] = out.cpu().numpy()
    _, ref = _run(ctx, ts, labels, ytn.YTN_FP64, 0.0)
    np.testing.assert_array_equal(rec["data"], ref["data"])
    check_against_oracle(rec, want)
