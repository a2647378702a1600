"""CPU checks of the C ABI: the library loads and exports every entry point declared
in include/ytn.h, and the host planner's structures (output blocks, offsets, fusion
records, sizes) equal the oracle's bit for bit. No device work: a host-only context
(device < 0) plans without uploading."""
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import fusion_mismatch_pair, random_legs, random_pair
from paper_2405_12196_gb300 import ytn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ytn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ytn_[a-z_]+)\s*\(", src)))


def test_library_exports_every_header_function():
    names = header_functions()
    assert "ytn_tensordot" in names and "ytn_plan" in names
    lib = ytn.load_library()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ytn.SYMBOLS), "binding and header declare different entry points"
    assert "sm_103a" in ytn.ytn_version()


@pytest.fixture(scope="module")
def hctx():
    return ytn.ytn_ctx_create(-1)


def same_structure(rec, ref):
    """Compare a library output record with an oracle record, bit for bit."""
    assert rec.get("dtype", "f64") == ref.get("dtype", "f64")
    assert tuple(rec["mods"]) == tuple(ref["mods"])
    assert tuple(rec["sig"]) == tuple(ref["sig"])
    assert tuple(rec["n"]) == tuple(ref["n"])
    np.testing.assert_array_equal(rec["t"], ref["t"].reshape(rec["t"].shape))
    np.testing.assert_array_equal(rec["D"], ref["D"].reshape(rec["D"].shape))
    np.testing.assert_array_equal(rec["off"], W.block_offsets(ref["D"]))
    assert rec["size"] == ref["data"].size
    rf, ff = ref.get("fus"), rec.get("fus")
    if rf is None:
        assert ff is None
    else:
        for a, b in zip(ff, rf):
            assert (a is None) == (b is None)
            if a is not None:
                assert tuple(a["sig"]) == tuple(b["sig"])
                for k in ("nu", "t", "D"):
                    np.testing.assert_array_equal(a[k], b[k])


SYMS = {"U1": (0,), "Z2": (2,), "Z3": (3,), "U1xU1": (0, 0)}


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(10))
def test_tensordot_structure_matches_oracle(hctx, sym, case):
    mods = SYMS[sym]
    rng = np.random.default_rng(7000 + 31 * case + len(sym))
    rankA, rankB = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    ncon = int(rng.integers(0, min(rankA, rankB) + 1))
    A, B, axa, axb, _, _ = random_pair(rng, mods, rankA, rankB, ncon)
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    oA, oB = O.from_record(A), O.from_record(B)
    ref = O.to_record(O.tensordot(oA, oB, axa, axb))
    same_structure(plan.out, ref)
    assert plan.info["useful_flops"] == O.useful_flops(oA, oB, axa, axb)
    # moved elements: the A and B blocks with a partner on the contracted legs, and C
    ka = [tuple(map(tuple, t[list(axa)])) for t in A["t"]]
    kb = [tuple(map(tuple, t[list(axb)])) for t in B["t"]]
    cov_a = sum(int(np.prod(d)) for k, d in zip(ka, A["D"]) if k in set(kb))
    cov_b = sum(int(np.prod(d)) for k, d in zip(kb, B["D"]) if k in set(ka))
    assert plan.info["moved_elems"] == cov_a + cov_b + ref["data"].size


def test_config1_plan_counts(hctx):
    cfg = W.config1()
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    assert plan.info["nsectors"] == 5
    assert plan.out["t"].shape[0] == 14 and plan.out["size"] == 458
    assert plan.info["useful_flops"] == 5640
    assert (plan.info["max_m"], plan.info["max_n"], plan.info["max_k"]) == (12, 12, 8)


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(6))
def test_fuse_unfuse_structure_matches_oracle(hctx, sym, case):
    mods = SYMS[sym]
    rng = np.random.default_rng(8100 + case)
    rank = int(rng.integers(2, 6))
    legs = random_legs(rng, mods, rank)
    rec = W.random_tensor(mods, legs, tuple([0] * len(mods)), 300 + case)
    if rec["t"].shape[0] == 0:
        return
    perm = [int(a) for a in rng.permutation(rank)]
    cut = int(rng.integers(1, rank))
    groups = (tuple(perm[:cut]), tuple(perm[cut:]))
    T = O.from_record(rec)
    F = O.fuse(T, groups)
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_FUSE, rec, groups=groups)
    same_structure(plan.out, O.to_record(F))
    fused_legs = [i for i, g in enumerate(groups) if len(g) > 1]
    if not fused_legs:
        return
    U = O.unfuse(F, fused_legs)
    uplan = ytn.ytn_plan(hctx, ytn.YTN_OP_UNFUSE, plan.out, axa=fused_legs)
    same_structure(uplan.out, O.to_record(U))


@pytest.mark.parametrize("case", range(8))
def test_trace_structure_matches_oracle(hctx, case):
    rng = np.random.default_rng(9100 + case)
    mods = [(0,), (2,), (0, 0), (3,)][case % 4]
    base = random_legs(rng, mods, 2)
    other = random_legs(rng, mods, int(rng.integers(0, 3)))
    legs = [base[0], base[1], base[0].conj(), base[1].conj()] + other
    npair = int(rng.integers(1, 3))
    ax1, ax2 = (0, 1)[:npair], (2, 3)[:npair]
    rec = W.random_tensor(mods, legs, tuple([0] * len(mods)), 60 + case)
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TRACE, rec, axa=ax1, axb=ax2)
    same_structure(plan.out, O.to_record(O.trace(O.from_record(rec), ax1, ax2)))


def test_errors_are_status_codes(hctx):
    l = W.Leg(1, [(0,), (1,)], [2, 3])
    A = W.random_tensor((0,), [l, l.conj()], (0,), 1)
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, A, A, (0,), (0,))
    assert e.value.name == "YTN_E_SIGNATURE"
    lb = W.Leg(-1, [(0,), (1,)], [2, 4])
    B = W.random_tensor((0,), [lb, W.Leg(1, [(0,), (1,)], [2, 4])], (0,), 2)
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, A, B, (1,), (1,))
    assert e.value.name == "YTN_E_DIM_MISMATCH"
    bad = dict(A)
    bad["t"] = A["t"].copy()
    bad["t"][0, 0, 0] = 5
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, bad, A, (1,), (0,))
    assert e.value.name in ("YTN_E_CHARGE", "YTN_E_INVALID")
    unsorted = dict(A)
    unsorted["t"] = A["t"][::-1].copy()
    unsorted["D"] = A["D"][::-1].copy()
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, unsorted, A, (1,), (0,))
    assert e.value.name == "YTN_E_INVALID"
    fused = ytn.ytn_plan(hctx, ytn.YTN_OP_FUSE, A, groups=((0, 1),)).out
    plain = W.random_tensor((0,), [W.Leg(-1, [(0,)], [13])], (0,), 3)
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, fused, plain, (0,), (0,))
    assert e.value.name == "YTN_E_FUSION_MISMATCH"
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, A, A, (0, 0), (1, 1))
    assert e.value.name == "YTN_E_INVALID"


def test_plan_cache_returns_same_plan(hctx):
    cfg = W.config1()
    p1 = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    p2 = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    assert p1.handle == p2.handle
    p3 = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], (0,), (2,))
    assert p3.handle != p1.handle


def test_execution_needs_a_device_context(hctx):
    cfg = W.config1()
    p = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_tensordot(p, 1 << 20, 1 << 20, 1 << 20, workspace=1 << 20, workspace_bytes=1 << 30)
    assert e.value.name == "YTN_E_INVALID"


def test_auto_workspace_covers_the_admissible_paths(hctx):
    """YTN_AUTO needs the split layout when the split path meets rtol (it may run
    both paths), else the FP64 layout."""
    cfg = W.config1()
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    f64 = ytn.ytn_workspace_size(plan, ytn.YTN_FP64)
    split = ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, 1e-10)
    assert split > f64 > 0
    assert ytn.ytn_workspace_size(plan, ytn.YTN_AUTO, 1e-10) == split
    assert ytn.ytn_workspace_size(plan, ytn.YTN_AUTO, 1e-16) == f64
    with pytest.raises(ytn.YtnError):
        ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, 1e-16)


def test_gemm_sms_needs_a_device_context(hctx):
    with pytest.raises(ytn.YtnError):
        ytn.ytn_ctx_set_gemm_sms(hctx, 8)


def test_vdot_planning_matches_the_oracle_rules(hctx):
    """VDOT plans: common elements counted as the oracle's common blocks; the same
    errors as the oracle for tensors that do not lie on the same legs."""
    rng = np.random.default_rng(21)
    for mods in [(0,), (2,), (0, 0)]:
        legs = random_legs(rng, mods, 3)
        A = W.random_tensor(mods, legs, (0,) * len(mods), 1)
        B = W.random_tensor(mods, legs, (0,) * len(mods), 2)
        plan = ytn.ytn_plan(hctx, ytn.YTN_OP_VDOT, A, B)
        oA, oB = O.from_record(A), O.from_record(B)
        common = sum(oA.blocks[k].size for k in oA.blocks if k in oB.blocks)
        assert plan.info["moved_elems"] == common
        assert plan.info["useful_flops"] == 2 * common
        assert plan.out["size"] == 1
        assert ytn.ytn_workspace_size(plan) == (0 if common == 0 else 256 * (-(-8 * -(-common // 8192) // 256)))
    l = W.Leg(1, [(-1,), (1,)], [2, 3])
    A = W.random_tensor((0,), [l, l.conj()], (0,), 1)
    bad = {
        "YTN_E_SIGNATURE": W.random_tensor((0,), [l.conj(), l], (0,), 2),
        "YTN_E_DIM_MISMATCH": W.random_tensor((0,), [W.Leg(1, [(-1,), (1,)], [2, 4]),
                                                     W.Leg(-1, [(-1,), (1,)], [2, 4])], (0,), 3),
        "YTN_E_INVALID": W.random_tensor((2,), [W.Leg(1, [(0,), (1,)], [2, 3])] * 2, (0,), 4),
    }
    for name, B in bad.items():
        with pytest.raises(ytn.YtnError) as ei:
            ytn.ytn_plan(hctx, ytn.YTN_OP_VDOT, A, B)
        assert ei.value.name == name


def test_swap_gate_planning(hctx):
    """SWAP_GATE plans keep the structure of a, move every element once and reject
    what the oracle rejects (overlapping groups, a Z3 component as fermionic)."""
    rng = np.random.default_rng(23)
    for mods in [(0,), (2,), (0, 0)]:
        legs = random_legs(rng, mods, 4)
        A = W.random_tensor(mods, legs, (0,) * len(mods), 1)
        plan = ytn.ytn_plan(hctx, ytn.YTN_OP_SWAP_GATE, A, groups=((0, 2), (3,)))
        same_structure(plan.out, O.to_record(O.swap_gate(O.from_record(A), (0, 2), (3,))))
        assert plan.info["moved_elems"] == A["data"].size
        ytn.ytn_plan(hctx, ytn.YTN_OP_SWAP_GATE, A, groups=((1,), (0,)), fermionic=(False,) * len(mods))
    A = W.random_tensor((0,), random_legs(rng, (0,), 3), (0,), 2)
    for groups in [((0, 1), (1,)), ((0,),), ((0,), (3,)), ((), (1,))]:
        with pytest.raises(ytn.YtnError) as ei:
            ytn.ytn_plan(hctx, ytn.YTN_OP_SWAP_GATE, A, groups=groups)
        assert ei.value.name == "YTN_E_INVALID"
    Z3 = W.random_tensor((3,), random_legs(rng, (3,), 2), (0,), 3)
    with pytest.raises(ytn.YtnError):
        ytn.ytn_plan(hctx, ytn.YTN_OP_SWAP_GATE, Z3, groups=((0,), (1,)))
    U1Z3 = W.random_tensor((0, 3), random_legs(rng, (0, 3), 2), (0, 0), 4)
    ytn.ytn_plan(hctx, ytn.YTN_OP_SWAP_GATE, U1Z3, groups=((0,), (1,)), fermionic=(True, False))


def test_empty_fusion_record_round_trip(hctx):
    """Fusing a tensor without blocks gives a fused leg with an empty record; that
    record comes back through the ABI and plans like any other."""
    rng = np.random.default_rng(31)
    A = W.random_tensor((0, 2), random_legs(rng, (0, 2), 4, max_dim=6), (0, 0), 5)
    assert A["data"].size == 0
    pf = ytn.ytn_plan(hctx, ytn.YTN_OP_FUSE, A, groups=((0, 1), (2,), (3,)))
    F = O.to_record(O.fuse(O.from_record(A), ((0, 1), (2,), (3,))))
    same_structure(pf.out, F)
    assert pf.out["fus"][0]["nu"].shape[0] == 0
    for rec in (F, dict(pf.out)):
        ytn.ytn_plan(hctx, ytn.YTN_OP_SWAP_GATE, rec, groups=((0,), (2,)))
        pu = ytn.ytn_plan(hctx, ytn.YTN_OP_UNFUSE, rec, axa=(0,))
        assert pu.out["size"] == 0


@pytest.mark.parametrize("drops", [(1, None), (None, -1), (1, -1), (0, 1)])
def test_fusion_mismatch_resolution_structure(hctx, drops):
    """Contracted fused legs with different fusion histories plan (Sec. II.B footnote):
    C's structure and useful FLOPs equal the oracle's resolved contraction."""
    A, B, _, _, _, _ = fusion_mismatch_pair(*drops)
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, O.to_record(A), O.to_record(B), (0,), (0,))
    ref = O.tensordot(A, B, (0,), (0,))
    same_structure(plan.out, O.to_record(ref))
    assert plan.info["useful_flops"] == O.useful_flops(O.unfuse(A, [0]), O.unfuse(B, [0]), (0, 1), (0, 1))


def test_fusion_mismatch_errors_as_status_codes(hctx):
    A, _, _, _, _, _ = fusion_mismatch_pair(1, None)
    l0 = W.Leg(-1, [(-1,), (0,), (1,)], [2, 3, 1])
    l1 = W.Leg(-1, [(0,), (1,)], [2, 2])
    l1b = W.Leg(-1, [(0,), (1,)], [2, 5])
    lx = W.Leg(-1, [(0,)], [1])
    l3 = W.Leg(1, [(-1,), (0,), (1,)], [1, 1, 1])
    three = O.fuse(O.from_record(W.random_tensor((0,), [l0, l1, lx, l3], (0,), 5)), ((0, 1, 2), (3,)))
    wrong = O.fuse(O.from_record(W.random_tensor((0,), [l0, l1b, l3], (0,), 6)), ((0, 1), (2,)))
    for other, name in ((three, "YTN_E_FUSION_MISMATCH"), (wrong, "YTN_E_DIM_MISMATCH")):
        with pytest.raises(ytn.YtnError) as ei:
            ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, O.to_record(A), O.to_record(other), (0,), (0,))
        assert ei.value.name == name


@pytest.mark.parametrize("dts", [("c128", "c128"), ("c128", "f64"), ("f64", "c128")])
@pytest.mark.parametrize("case", range(6))
def test_complex_plans_match_the_oracle(hctx, dts, case):
    """Complex operands (real and complex mixed too): tensordot's structure and
    element type equal the oracle's; its FLOPs count the real products of the
    doubled sector matrices; fuse, unfuse, trace, swap gate and conj keep the
    complex element type."""
    rng = np.random.default_rng(12000 + 17 * case + len(dts[0]) + 3 * len(dts[1]))
    mods = [(0,), (2,), (0, 0)][case % 3]
    A, _, axa, axb, legsA, legsB = random_pair(rng, mods, 3, 3, 1 + case % 2, dtype=dts[0])
    B = W.random_tensor(mods, legsB, (0,) * len(mods), 77 + case, dtype=dts[1])
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    oA, oB = O.from_record(A), O.from_record(B)
    same_structure(plan.out, O.to_record(O.tensordot(oA, oB, axa, axb)))
    mult = (2 if dts[0] == "c128" else 1) * (2 if dts[1] == "c128" else 1)
    assert plan.info["useful_flops"] == mult * O.useful_flops(oA, oB, axa, axb)
    if dts[0] == "c128":
        same_structure(ytn.ytn_plan(hctx, ytn.YTN_OP_FUSE, A, groups=((0, 1), (2,))).out,
                       O.to_record(O.fuse(oA, ((0, 1), (2,)))))
        same_structure(ytn.ytn_plan(hctx, ytn.YTN_OP_CONJ, A).out, O.to_record(O.conj(oA)))
        same_structure(ytn.ytn_plan(hctx, ytn.YTN_OP_SWAP_GATE, A, groups=((0,), (1, 2))).out,
                       O.to_record(O.swap_gate(oA, (0,), (1, 2))))


def test_complex_vdot_and_trace_planning(hctx):
    l = W.Leg(1, [(0,), (1,)], [2, 3])
    A = W.random_tensor((0,), [l, l.conj(), l], (1,), 1, dtype="c128")
    B = W.random_tensor((0,), [l, l.conj(), l], (1,), 2, dtype="c128")
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_VDOT, A, B)
    assert plan.out.get("dtype") == "c128" and plan.info["moved_elems"] == A["data"].size
    assert ytn.ytn_workspace_size(plan) == 256
    with pytest.raises(ytn.YtnError) as ei:
        ytn.ytn_plan(hctx, ytn.YTN_OP_VDOT, A, W.random_tensor((0,), [l, l.conj(), l], (1,), 3))
    assert ei.value.name == "YTN_E_UNSUPPORTED"
    tr = ytn.ytn_plan(hctx, ytn.YTN_OP_TRACE, A, axa=(0,), axb=(1,))
    same_structure(tr.out, O.to_record(O.trace(O.from_record(A), (0,), (1,))))


def test_einsum_plans_equal_the_oracle(hctx):
    from helpers import random_network
    rng = np.random.default_rng(61)
    for spec, kind in (("abc,bde,cef->adf", "chain"), ("abbc,cd->da", "trace"), ("ab,bc,de", "outer")):
        _, ts, _ = random_network(rng, (0,), kind)
        nc = ytn.ytn_einsum_plan(hctx, spec, ts)
        same_structure(nc.out, O.to_record(O.einsum(spec, *[O.from_record(t) for t in ts])))
    _, ts, _ = random_network(rng, (0,), "chain")
    for bad in ("abc,bde->adf", "abc,bde,cee->a", "abc,bde,cef->ad", "abc,bde,c1f->adf"):
        with pytest.raises(ytn.YtnError) as ei:
            ytn.ytn_einsum_plan(hctx, bad, ts)
        assert ei.value.name == "YTN_E_INVALID"


@pytest.mark.parametrize("seed", range(4))
def test_svd_and_slice_planning(hctx, seed):
    """SVD plans: U, S and V have the oracle's structures (sectors, new-leg charges
    and dimensions, signatures); a SLICE plan keeps the oracle's truncated blocks."""
    rng = np.random.default_rng(300 + seed)
    mods = (0,) if seed % 2 == 0 else (0, 0)
    pool = [(0,), (1,), (-1,)] if mods == (0,) else [(0, 0), (1, 0), (0, 1)]
    legs = [W.Leg(s, pool, [int(d) for d in rng.integers(1, 5, 3)]) for s in (1, 1, -1, -1)]
    A = W.random_tensor(mods, legs, (0,) * len(mods), seed)
    rows, cols = (0, 2), (1, 3)
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_SVD, A, groups=(rows, cols))
    U, S, V = O.svd(O.from_record(A), rows, cols)
    for got, want in zip(plan.outs, (U, S, V)):
        same_structure(got, O.to_record(want))
    keep = O.truncation(S, max(1, sum(S.blocks[k].shape[0] for k in S.blocks) // 2))
    ps = ytn.ytn_plan(hctx, ytn.YTN_OP_SLICE, plan.outs[0], axa=(2,), keep=keep)
    same_structure(ps.out, O.to_record(O.slice_leg(U, (2,), keep)))
    ps2 = ytn.ytn_plan(hctx, ytn.YTN_OP_SLICE, plan.outs[1], axa=(0, 1), keep=keep)
    same_structure(ps2.out, O.to_record(O.slice_leg(S, (0, 1), keep)))
    with pytest.raises(ytn.YtnError):
        ytn.ytn_plan(hctx, ytn.YTN_OP_SVD, A, groups=((0, 1), (1, 2, 3)))
    Ac = W.random_tensor(mods, legs, (0,) * len(mods), 1, dtype="c128")
    pc = ytn.ytn_plan(hctx, ytn.YTN_OP_SVD, Ac, groups=(rows, cols))
    for got, want in zip(pc.outs, O.svd(O.from_record(Ac), rows, cols)):
        same_structure(got, O.to_record(want))


@pytest.mark.parametrize("dtype", ["f64", "c128"])
def test_eigh_planning(hctx, dtype):
    """EIGH plans: U and S have the oracle's structures; non-dual legs or n != 0 are
    rejected."""
    rng = np.random.default_rng(77)
    pool = [(0,), (1,), (-1,)]
    r = [W.Leg(s, pool, [int(d) for d in rng.integers(1, 5, 3)]) for s in (1, -1)]
    H = W.random_tensor((0,), r + [l.conj() for l in r], (0,), 3, dtype=dtype)
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_EIGH, H, groups=((0, 1), (2, 3)))
    U, S = O.eigh(O.from_record(H), (0, 1), (2, 3))
    assert len(plan.outs) == 2
    same_structure(plan.outs[0], O.to_record(U))
    same_structure(plan.outs[1], O.to_record(S))
    with pytest.raises(ytn.YtnError) as ei:
        ytn.ytn_plan(hctx, ytn.YTN_OP_EIGH, H, groups=((0, 1), (3, 2)))
    assert ei.value.name == "YTN_E_SIGNATURE"


@pytest.mark.parametrize("sym", ["U1", "Z2", "Z3", "U1xU1"])
@pytest.mark.parametrize("case", range(4))
def test_blocks_from_legs_match_the_generator(hctx, sym, case):
    """ytn_plan_blocks (the paper's rand(legs, n) structure) == every block the input
    generator allows (an independent enumeration), canonical and packed."""
    mods = SYMS[sym]
    rng = np.random.default_rng(900 + 7 * case + len(sym))
    legs = random_legs(rng, mods, int(rng.integers(1, 5)), max_sectors=4, max_dim=4)
    n = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    plan = ytn.ytn_plan_blocks(hctx, mods, legs, n)
    want = W.random_tensor(mods, legs, n, 1)
    same_structure(plan.out, dict(want, data=np.zeros(want["data"].size)))
    O.from_record(dict(want, t=plan.out["t"], D=plan.out["D"]))   # validates conservation


def test_blocks_from_legs_errors(hctx):
    from types import SimpleNamespace
    for bad in (SimpleNamespace(s=1, t=[(1,), (0,)], D=[2, 3]),     # charges not ascending
                SimpleNamespace(s=2, t=[(0,)], D=[2]),              # signature
                SimpleNamespace(s=1, t=[(0,)], D=[0])):             # dimension
        with pytest.raises(ytn.YtnError) as ei:
            ytn.ytn_plan_blocks(hctx, (0,), [bad], (0,))
        assert ei.value.name == "YTN_E_INVALID"


def test_host_only_plans_have_no_pipeline_groups(hctx):
    """The pipelined fused split needs the device's SM count and streams: a plan of a
    host-only context reports no pipeline groups, even one large enough to have
    them on a GPU."""
    q = [(c,) for c in range(10)]
    A = W.random_tensor((0,), [W.Leg(1, q, [1024] * 10), W.Leg(-1, q, [256] * 10)], (0,), 1, fill="ones")
    B = W.random_tensor((0,), [W.Leg(1, q, [256] * 10), W.Leg(-1, q, [1024] * 10)], (0,), 2, fill="ones")
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, A, B, (1,), (0,))
    assert plan.info["split_fused"] == 1 and plan.info["split_pipe_groups"] == 0


def test_tuning_of_a_new_plan_is_undecided(hctx):
    """A plan that has run no split call has no cached choice and no timings; slice
    counts outside 1..6 are rejected."""
    cfg = W.config1()
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    for s in range(1, 7):
        t = ytn.ytn_plan_tuning(plan, s)
        assert t["slices"] == s
        assert (t["auto_choice"], t["split_variant"], t["tile_policy"]) == (-1, -1, -1)
        assert all(t[k] == 0.0 for k in ("fp64_ms", "split_ms", "staged_ms", "fused_ms", "wide_ms", "narrow_ms",
                                         "pipelined_ms"))
    for s in (0, 7):
        with pytest.raises(ytn.YtnError) as e:
            ytn.ytn_plan_tuning(plan, s)
        assert e.value.name == "YTN_E_INVALID"


def test_sector_subset_workload_keeps_whole_sectors():
    """The profiling-size workload is every block of a subset of the full contraction's
    sectors: its blocks and their data are the full tensors', and each kept sector keeps
    all of its blocks on both sides."""
    full = W.config5(seed=5001, D=14)
    part = W.config5_sectors(seed=5001, D=14)
    for name, legs in (("A", (1, 2)), ("B", (0, 1))):
        F, P = full[name], part[name]
        size = np.prod(F["D"], axis=1)
        off = np.concatenate([[0], np.cumsum(size)])
        index = {tuple(map(tuple, t)): i for i, t in enumerate(F["t"])}
        key = lambda t: tuple(t[legs[0]] - t[legs[1]])
        kept = {key(t) for t in P["t"]}
        assert 0 < len(kept) < len({key(t) for t in F["t"]})
        pos = 0
        for t, d in zip(P["t"], P["D"]):
            i = index[tuple(map(tuple, t))]
            np.testing.assert_array_equal(d, F["D"][i])
            n = int(np.prod(d))
            np.testing.assert_array_equal(P["data"][pos:pos + n], F["data"][off[i]:off[i + 1]])
            pos += n
        assert pos == P["data"].size
        assert len(P["t"]) == sum(1 for t in F["t"] if key(t) in kept)


def test_piece_dims_of_interleaved_and_merged_contractions(hctx):
    """The copy pieces of a contraction over every other leg of a rank-8 tensor keep
    eight dims (nothing merges); a contraction of trailing legs merges to at most four."""
    legs = [W.Leg(s, [(0,), (1,)], [2, 3]) for s in (1, -1, 1, -1, 1, -1, 1, -1)]
    A = W.random_tensor((0,), legs, (0,), 81)
    legsB = [legs[1].conj(), legs[3].conj(), legs[5].conj(), legs[7].conj(), W.Leg(1, [(0,)], [3])]
    B = W.random_tensor((0,), legsB, (2,), 82)
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, A, B, (1, 3, 5, 7), (0, 1, 2, 3))
    assert plan.info["max_copy_dims"] == 8
    cfg = W.config1()
    plan = ytn.ytn_plan(hctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    assert 1 <= plan.info["max_copy_dims"] <= 4
