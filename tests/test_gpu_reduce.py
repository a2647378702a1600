"""FP64 scalar products (ytn_vdot) through the C ABI, against the oracle.

The kernel sums in a different order than the oracle, so the bound is on the
error relative to sum |a b| (what a different summation order can change), at
1e-13; repeated calls must give identical bits.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import device, to_dev
from helpers import random_legs

pytestmark = pytest.mark.gpu

SYMS = {"U1": (0,), "Z2": (2,), "Z3": (3,), "U1xU1": (0, 0)}


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _vdot(ctx, A, B, host=False):
    import torch
    from paper_2405_12196_gb300 import ytn
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_VDOT, A, B)
    if host:
        a = torch.from_numpy(np.ascontiguousarray(A["data"])).pin_memory()
        b = torch.from_numpy(np.ascontiguousarray(B["data"])).pin_memory()
        out = torch.full((1,), float("nan"), dtype=torch.float64).pin_memory()
    else:
        a, b = to_dev(A["data"]), to_dev(B["data"])
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=device())
    ws = torch.empty(max(ytn.ytn_workspace_size(plan), 1), dtype=torch.uint8, device=device())
    vals = []
    for _ in range(2):
        ytn.ytn_vdot(plan, a, b, out, workspace=ws)
        ytn.ytn_sync(ctx)
        vals.append(float(out.cpu()[0]))
    assert vals[0] == vals[1] or (np.isnan(vals[0]) and np.isnan(vals[1]))
    return vals[0], plan


def _abs(rec):
    return dict(rec, data=np.abs(rec["data"]))


def _check(got, A, B):
    oA, oB = O.from_record(A), O.from_record(B)
    want = O.vdot(oA, oB)
    scale = O.vdot(O.from_record(_abs(A)), O.from_record(_abs(B)))
    assert abs(got - want) <= 1e-13 * max(scale, 1e-300), (got, want, scale)


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(5))
def test_vdot_random(ctx, sym, case):
    mods = SYMS[sym]
    rng = np.random.default_rng(9100 + 17 * case + len(sym))
    legs = random_legs(rng, mods, int(rng.integers(1, 5)), max_dim=9)
    n = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    A = W.random_tensor(mods, legs, n, 3 * case + 1)
    B = W.random_tensor(mods, legs, n, 3 * case + 2)
    got, _ = _vdot(ctx, A, B)
    _check(got, A, B)
    # the squared norm
    got, _ = _vdot(ctx, A, A)
    assert got == pytest.approx(float(np.sum(A["data"] ** 2)), rel=1e-13, abs=1e-300)


def test_vdot_partial_overlap_and_disjoint(ctx):
    q, d = [(0, 0), (1, 0), (0, 1), (-1, 0)], [2, 3, 2, 1]
    legs = [W.Leg(s, q, d) for s in (1, 1, -1, -1)]
    A = W.random_tensor((0, 0), legs, (0, 0), 1)
    B = W.random_tensor((0, 0), legs, (0, 0), 2)
    keep = np.arange(B["t"].shape[0]) % 3 != 1
    off = np.concatenate([[0], np.cumsum(np.prod(B["D"], axis=1))])
    B = dict(B, t=B["t"][keep], D=B["D"][keep],
             data=np.concatenate([B["data"][off[i]:off[i + 1]] for i in np.nonzero(keep)[0]]))
    got, _ = _vdot(ctx, A, B)
    _check(got, A, B)
    # no common block: a different total charge
    C = W.random_tensor((0, 0), legs, (1, 0), 3)
    got, plan = _vdot(ctx, A, C)
    assert got == 0.0 and plan.info["moved_elems"] == 0


def test_vdot_large_blocks_and_host_buffers(ctx):
    """Blocks of 5000 and 9000 elements (several pieces each), from host memory too."""
    legs = [W.Leg(1, [(0,), (1,)], [50, 90]), W.Leg(-1, [(0,), (1,)], [100, 100])]
    A = W.random_tensor((0,), legs, (0,), 7)
    B = W.random_tensor((0,), legs, (0,), 8)
    got, _ = _vdot(ctx, A, B)
    _check(got, A, B)
    got_h, _ = _vdot(ctx, A, B, host=True)
    assert got_h == got


def test_vdot_full_size_environment_tensors(ctx):
    """Two D=20 environment tensors X2 on the same legs (3.36e8 elements each)."""
    A = W.config5(seed=5001)["A"]
    B = W.config5(seed=6001)["A"]
    got, plan = _vdot(ctx, A, B)
    assert plan.info["moved_elems"] == A["data"].size
    _check(got, A, B)
