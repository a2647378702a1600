"""Complex128 tensors through the C ABI, against the oracle.

Contractions of complex (and mixed real/complex) operands on both paths, the
moves that are bit-exact (fuse, unfuse, conj in and out of place, swap gate),
the trace, and the complex scalar product <A, B> = sum conj(a) b.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import FP64_RTOL, check_against_oracle, device, rel_frobenius
from helpers import random_legs, random_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _dev(rec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(rec["data"])).to(device())


def _empty(out):
    import torch
    dt = torch.complex128 if out.get("dtype") == "c128" else torch.float64
    return torch.full((max(out["size"], 1),), float("nan"), dtype=dt, device=device())


def _rec(plan_out, buf):
    rec = dict(plan_out)
    rec["data"] = buf[:plan_out["size"]].cpu().numpy()
    return rec


def _tensordot(ctx, A, B, axa, axb, prec, rtol):
    import torch
    from paper_2405_12196_gb300 import ytn
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    c = _empty(plan.out)
    ws = torch.empty(max(ytn.ytn_workspace_size(plan, prec, rtol), 1), dtype=torch.uint8, device=device())
    ytn.ytn_tensordot(plan, _dev(A), _dev(B), c, prec=prec, rtol=rtol, workspace=ws)
    ytn.ytn_sync(ctx)
    return plan, _rec(plan.out, c)


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("dts", [("c128", "c128"), ("c128", "f64"), ("f64", "c128")])
@pytest.mark.parametrize("case", range(4))
def test_complex_tensordot(ctx, dts, case, split):
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(12500 + 11 * case + len(dts[1]))
    mods = [(0,), (2,), (0, 0), (3,)][case]
    A, _, axa, axb, legsA, legsB = random_pair(rng, mods, 3, 3, 1 + case % 2, dtype=dts[0], max_dim=12)
    B = W.random_tensor(mods, legsB, (0,) * len(mods), 90 + case, dtype=dts[1])
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    _, rec = _tensordot(ctx, A, B, axa, axb, prec, rtol)
    want = O.to_record(O.tensordot(O.from_record(A), O.from_record(B), axa, axb))
    check_against_oracle(rec, want, rtol=1e-10 if split else FP64_RTOL)


@pytest.mark.parametrize("split", [False, True])
def test_complex_double_layer_chain(ctx, split):
    """The Z2 double-layer step with a complex site tensor: A.conj(A) over the
    physical leg, then T.a over the fused ket/bra leg (T complex too)."""
    from paper_2405_12196_gb300 import ytn
    cfg = W.config2()
    A = dict(cfg["A"])
    rngA = np.random.default_rng(7)
    A["data"] = (rngA.standard_normal(A["data"].size) + 1j * rngA.standard_normal(A["data"].size))
    A["dtype"] = "c128"
    oA = O.from_record(A)
    Ac = O.to_record(O.conj(oA))
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    _, AA = _tensordot(ctx, A, Ac, (4,), (4,), prec, rtol)
    want = O.to_record(O.tensordot(oA, O.conj(oA), (4,), (4,)))
    check_against_oracle(AA, want, rtol=1e-10 if split else FP64_RTOL)


def test_complex_moves_are_exact(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(51)
    legs = random_legs(rng, (0, 0), 4, max_sectors=3, max_dim=5)
    A = W.random_tensor((0, 0), legs, (0, 0), 3, dtype="c128")
    assert A["data"].size > 0
    oA = O.from_record(A)
    pf = ytn.ytn_plan(ctx, ytn.YTN_OP_FUSE, A, groups=((0, 2), (1, 3)))
    f = _empty(pf.out)
    ytn.ytn_fuse(pf, _dev(A), f)
    ytn.ytn_sync(ctx)
    F = _rec(pf.out, f)
    check_against_oracle(F, O.to_record(O.fuse(oA, ((0, 2), (1, 3)))), exact=True)
    pu = ytn.ytn_plan(ctx, ytn.YTN_OP_UNFUSE, F, axa=(0, 1))
    u = _empty(pu.out)
    ytn.ytn_unfuse(pu, f, u)
    ytn.ytn_sync(ctx)
    check_against_oracle(_rec(pu.out, u), O.to_record(O.unfuse(O.from_record(F), (0, 1))), exact=True)
    pc = ytn.ytn_plan(ctx, ytn.YTN_OP_CONJ, A)
    want = O.to_record(O.conj(oA))
    c = _empty(pc.out)
    ytn.ytn_conj(pc, _dev(A), c)
    ytn.ytn_sync(ctx)
    check_against_oracle(_rec(pc.out, c), want, exact=True)
    a = _dev(A)
    ytn.ytn_conj(pc, a, a)              # in place
    ytn.ytn_sync(ctx)
    check_against_oracle(_rec(pc.out, a), want, exact=True)
    ps = ytn.ytn_plan(ctx, ytn.YTN_OP_SWAP_GATE, A, groups=((0,), (1, 3)))
    s = _empty(ps.out)
    ytn.ytn_swap_gate(ps, _dev(A), s)
    ytn.ytn_sync(ctx)
    check_against_oracle(_rec(ps.out, s), O.to_record(O.swap_gate(oA, (0,), (1, 3))), exact=True)
    del torch


def test_complex_trace_and_vdot(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    l = W.Leg(1, [(0,), (1,), (2,)], [3, 5, 2])
    m = W.Leg(1, [(-1,), (0,), (1,)], [40, 70, 30])
    A = W.random_tensor((0,), [l, m, l.conj()], (0,), 1, dtype="c128")
    pt = ytn.ytn_plan(ctx, ytn.YTN_OP_TRACE, A, axa=(0,), axb=(2,))
    t = _empty(pt.out)
    ytn.ytn_trace(pt, _dev(A), t)
    ytn.ytn_sync(ctx)
    check_against_oracle(_rec(pt.out, t), O.to_record(O.trace(O.from_record(A), (0,), (2,))))
    B = W.random_tensor((0,), [l, m, l.conj()], (0,), 2, dtype="c128")
    pv = ytn.ytn_plan(ctx, ytn.YTN_OP_VDOT, A, B)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=device())
    ws = torch.empty(max(ytn.ytn_workspace_size(pv), 1), dtype=torch.uint8, device=device())
    vals = []
    for _ in range(2):
        ytn.ytn_vdot(pv, _dev(A), _dev(B), out, workspace=ws)
        ytn.ytn_sync(ctx)
        vals.append(complex(out[0].item(), out[1].item()))
    assert vals[0] == vals[1]
    want = O.vdot(O.from_record(A), O.from_record(B))
    scale = float(np.sum(np.abs(A["data"]) * np.abs(B["data"])))
    assert abs(vals[0] - want) <= 1e-13 * scale
    assert rel_frobenius([vals[0]], [want]) < 1e-12
