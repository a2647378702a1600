"""Graph capture of a chain of calls (ytn_graph_*), through the C ABI.

A recorded chain A.A* -> fuse -> T.a (the Z2 double-layer step) must give the
same bits as the eager calls, follow new input data written into the same
buffers, and keep working after the caller released its plans.
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


def _chain(ctx, prec, rtol):
    """Plans and device buffers of the chain; returns (run(stream), buffers, plans)."""
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config2()
    A, T = cfg["A"], dict(cfg["T"])
    Ac = dict(A)
    Ac["sig"] = tuple(-s for s in A["sig"])
    p1 = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, Ac, (4,), (4,))
    AA = dict(p1.out)
    groups = ((0, 4), (1, 5), (2, 6), (3, 7))
    p2 = ytn.ytn_plan(ctx, ytn.YTN_OP_FUSE, AA, groups=groups)
    a = dict(p2.out)
    T["fus"] = [None, dict(a["fus"][0], sig=tuple(-s for s in a["fus"][0]["sig"])), None]
    p3 = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, T, a, (1,), (0,))
    dev = device()
    buf = {"A": to_dev(A["data"]), "T": to_dev(T["data"]),
           "AA": torch.empty(max(AA["size"], 1), dtype=torch.float64, device=dev),
           "a": torch.empty(max(a["size"], 1), dtype=torch.float64, device=dev),
           "Ta": torch.empty(max(p3.out["size"], 1), dtype=torch.float64, device=dev)}
    ws1 = torch.empty(ytn.ytn_workspace_size(p1, prec, rtol), dtype=torch.uint8, device=dev)
    ws3 = torch.empty(ytn.ytn_workspace_size(p3, prec, rtol), dtype=torch.uint8, device=dev)
    buf["ws1"], buf["ws3"] = ws1, ws3

    def run(stream):
        ytn.ytn_tensordot(p1, buf["A"], buf["A"], buf["AA"], prec=prec, rtol=rtol, workspace=ws1, stream=stream)
        ytn.ytn_fuse(p2, buf["AA"], buf["a"], stream=stream)
        ytn.ytn_tensordot(p3, buf["T"], buf["a"], buf["Ta"], prec=prec, rtol=rtol, workspace=ws3, stream=stream)

    recs = {"A": A, "Ac": Ac, "T": T, "groups": groups, "out": dict(p3.out)}
    return run, buf, [p1, p2, p3], recs


def _oracle_chain(recs, A_data):
    A = dict(recs["A"], data=A_data)
    oA = O.from_record(A)
    oAA = O.tensordot(oA, O.conj(oA), (4,), (4,))
    oa = O.fuse(oAA, recs["groups"])
    return O.tensordot(O.from_record(recs["T"]), oa, (1,), (0,))


@pytest.mark.parametrize("split", [False, True])
def test_graph_replay_matches_eager_and_oracle(ctx, split):
    import torch
    from paper_2405_12196_gb300 import ytn
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    run, buf, plans, recs = _chain(ctx, prec, rtol)
    n = recs["out"]["size"]
    stream = torch.cuda.Stream(device=device())
    run(stream)
    ytn.ytn_sync(ctx, stream)
    eager = buf["Ta"][:n].cpu().numpy().copy()

    ytn.ytn_graph_begin(ctx, stream)
    run(stream)
    graph = ytn.ytn_graph_end(ctx, stream)
    for p in plans:     # the graph keeps its own references
        p.release()
    buf["Ta"].fill_(float("nan"))
    torch.cuda.synchronize()
    graph.launch(stream)
    ytn.ytn_sync(ctx, stream)
    np.testing.assert_array_equal(buf["Ta"][:n].cpu().numpy(), eager)

    # new data in the same input buffer: the replay follows it
    rng = np.random.default_rng(99)
    A2 = rng.standard_normal(recs["A"]["data"].size)
    buf["A"].copy_(torch.from_numpy(A2))
    torch.cuda.synchronize()
    for _ in range(3):
        graph.launch(stream)
    ytn.ytn_sync(ctx, stream)
    got = buf["Ta"][:n].cpu().numpy()
    want = O.to_record(_oracle_chain(recs, A2))["data"]
    tol = 1e-10 if split else FP64_RTOL
    assert rel_frobenius(got, want) <= tol
    graph.close()


def test_graph_capture_errors(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    stream = torch.cuda.Stream(device=device())
    with pytest.raises(ytn.YtnError):
        ytn.ytn_graph_begin(ctx, None)          # the default stream cannot be captured
    ytn.ytn_graph_begin(ctx, stream)
    with pytest.raises(ytn.YtnError):
        ytn.ytn_graph_begin(ctx, stream)        # one capture per context
    g = ytn.ytn_graph_end(ctx, stream)          # an empty graph is valid
    g.launch(stream)
    ytn.ytn_sync(ctx, stream)
    g.close()
    with pytest.raises(ytn.YtnError):
        ytn.ytn_graph_end(ctx, stream)          # not capturing any more


def test_ctm_step_chain_as_one_graph(ctx):
    """The contractions of one U(1)xU(1) CTMRG step (A.A*, fuse, C.T, CT.T, X2.a;
    the bench's --chain workload) with YTN_AUTO: one graph launch gives the bits of
    the eager calls, and X2.a matches the oracle within the split tolerance."""
    import os
    import sys

    import torch
    from paper_2405_12196_gb300 import ytn
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    stream = torch.cuda.Stream(device=device())
    run, plans, out, n, flops = bench.ctm_chain(ytn, ctx, device(), ytn.YTN_AUTO, 1e-10)
    assert flops > 3e10
    run(stream)                      # eager: YTN_AUTO decides (and caches) each path
    run(stream)
    ytn.ytn_sync(ctx, stream)
    eager = out[:n].cpu().numpy().copy()
    ytn.ytn_graph_begin(ctx, stream)
    run(stream)
    g = ytn.ytn_graph_end(ctx, stream)
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    g.launch(stream)
    ytn.ytn_sync(ctx, stream)
    np.testing.assert_array_equal(out[:n].cpu().numpy(), eager)
    g.close()
    # X2.a against the oracle: a = fuse(A.A*), X2 with a's conjugate fusion records
    cfg = W.config3()
    A, X2 = cfg["A"], dict(cfg["X2"])
    oA = O.from_record(A)
    oa = O.fuse(O.tensordot(oA, O.conj(oA), (4,), (4,)), ((0, 4), (1, 5), (2, 6), (3, 7)))
    ra = O.to_record(oa)
    conj = lambda f: dict(f, sig=tuple(-x for x in f["sig"]))   # noqa: E731
    X2["fus"] = [None, conj(ra["fus"][0]), conj(ra["fus"][1]), None]
    want = O.to_record(O.tensordot(O.from_record(X2), oa, (1, 2), (0, 1)))["data"]
    assert rel_frobenius(eager, want) <= 1e-10
