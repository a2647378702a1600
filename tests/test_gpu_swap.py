"""Fermionic swap gates (ytn_swap_gate) through the C ABI, against the oracle.

Sign changes are exact, so the GPU result must equal the oracle bit for bit:
random U(1), Z2, U(1)xU(1) and U(1)xZ2 tensors (fused legs included), in place,
from page-locked host memory, with explicit fermionic components, and on a
D = 20 environment tensor.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import check_against_oracle, to_dev
from helpers import random_legs

pytestmark = pytest.mark.gpu

SYMS = {"U1": (0,), "Z2": (2,), "U1xU1": (0, 0), "U1xZ2": (0, 2)}


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _swap(ctx, A, g1, g2, fermionic=None, in_place=False, host=False):
    import torch
    from paper_2405_12196_gb300 import ytn
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_SWAP_GATE, A, groups=(tuple(g1), tuple(g2)), fermionic=fermionic)
    if host:
        a = torch.from_numpy(np.ascontiguousarray(A["data"])).pin_memory()
        out = a if in_place else torch.full_like(a, float("nan")).pin_memory()
    else:
        a = to_dev(A["data"])
        out = a if in_place else torch.full_like(a, float("nan"))
    ytn.ytn_swap_gate(plan, a, out)
    ytn.ytn_sync(ctx)
    rec = dict(plan.out)
    rec["data"] = out.cpu().numpy()
    return rec


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(5))
def test_swap_gate_random(ctx, sym, case):
    mods = SYMS[sym]
    rng = np.random.default_rng(9300 + 7 * case + len(sym))
    rank = int(rng.integers(2, 6))
    A = W.random_tensor(mods, random_legs(rng, mods, rank, max_dim=9), (0,) * len(mods), case + 11)
    perm = [int(x) for x in rng.permutation(rank)]
    k1 = int(rng.integers(1, rank))
    g1, g2 = perm[:k1], perm[k1:]
    want = O.to_record(O.swap_gate(O.from_record(A), g1, g2))
    check_against_oracle(_swap(ctx, A, g1, g2), want, exact=True)
    check_against_oracle(_swap(ctx, A, g1, g2, in_place=True), want, exact=True)


def test_swap_gate_fused_legs_host_memory_and_explicit_components(ctx):
    q, d = [(0, 0), (1, 1), (-1, 1), (0, 1), (1, 0)], [2, 1, 2, 1, 3]
    A = W.random_tensor((0, 2), [W.Leg(s, q, d) for s in (1, 1, -1, -1)], (0, 0), 5)
    assert A["data"].size > 0
    oA = O.from_record(A)
    F = O.to_record(O.fuse(oA, ((0, 1), (2,), (3,))))
    want = O.to_record(O.swap_gate(O.from_record(F), (0,), (2,)))
    check_against_oracle(_swap(ctx, F, (0,), (2,)), want, exact=True)
    check_against_oracle(_swap(ctx, F, (0,), (2,), host=True), want, exact=True)
    check_against_oracle(_swap(ctx, F, (0,), (2,), host=True, in_place=True), want, exact=True)
    for fm in [(False, True), (True, False), (False, False)]:
        want = O.to_record(O.swap_gate(oA, (0, 1), (3,), fermionic=fm))
        check_against_oracle(_swap(ctx, A, (0, 1), (3,), fermionic=fm), want, exact=True)


def test_swap_gate_of_an_empty_fused_tensor(ctx):
    """A tensor without blocks (its fused leg has an empty record) plans and runs."""
    rng = np.random.default_rng(31)
    A = W.random_tensor((0, 2), random_legs(rng, (0, 2), 4, max_dim=6), (0, 0), 5)
    assert A["data"].size == 0
    F = O.to_record(O.fuse(O.from_record(A), ((0, 1), (2,), (3,))))
    rec = _swap(ctx, F, (0,), (1, 2))
    assert rec["size"] == 0 and rec["t"].shape[0] == 0


def test_swap_gate_full_size_environment_tensor(ctx):
    """A D=20 environment tensor X2 (3.36e8 elements, 103725 blocks), lines 0 and 1
    against 2 and 3, every element against the oracle."""
    A = W.config5(seed=5001)["A"]
    want = O.to_record(O.swap_gate(O.from_record(A), (0, 1), (2, 3)))
    got = _swap(ctx, A, (0, 1), (2, 3))
    np.testing.assert_array_equal(got["data"], want["data"])
    assert np.any(got["data"] != A["data"])
