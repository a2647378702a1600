"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test names the passage it pins. A plausible mistake in the oracle (a dropped
pair, a wrong sign in charge matching, a transposed operand, a misplaced fused
sub-block, a wrong trace pairing) fails at least one of these.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import fusion_mismatch_pair, leg_map, random_legs, random_network, random_pair

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _tensor_from_golden(g, key="blocks"):
    blocks = {}
    for charges, val in g[key]:
        k = tuple(tuple(c) for c in charges)
        blocks[k] = np.array(val, dtype=np.float64).reshape([1] * len(k))
    return O.OTensor(tuple(g["mods"]), tuple(g["sig"]), tuple(g["n"]), blocks).validate()


# ---------------------------------------------------------------- the paper's example

def test_heisenberg_structure_and_closed_form():
    """Sec. II.A/II.B example: H = S1.S2 on legs [l, l, lc, lc]; (S1.S2)^2 = 3/16 - H/2."""
    g = _golden("heisenberg_two_site.json")
    H = _tensor_from_golden(g)
    assert len(H.blocks) == 6
    # the generator's allowed blocks for these legs are exactly the 6 of the example
    l = W.Leg(1, [(-1,), (1,)], [1, 1])
    rec = W.random_tensor((0,), [l, l, l.conj(), l.conj()], (0,), 0)
    assert sorted(O.from_record(rec).blocks) == sorted(H.blocks)
    H2 = O.tensordot(H, H, (2, 3), (0, 1))
    want = _tensor_from_golden(g, "H2_blocks")
    assert sorted(H2.blocks) == sorted(want.blocks)
    for k in want.blocks:
        assert H2.blocks[k].shape == (1, 1, 1, 1)
        assert H2.blocks[k][0, 0, 0, 0] == pytest.approx(want.blocks[k][0, 0, 0, 0], abs=1e-15)


def test_heisenberg_traces():
    g = _golden("heisenberg_two_site.json")
    H = _tensor_from_golden(g)
    trH = O.trace(H, (0, 1), (2, 3))
    assert trH.rank == 0 and list(trH.blocks) == [()]
    assert float(trH.blocks[()]) == pytest.approx(g["trace_H"], abs=1e-15)
    H2 = O.tensordot(H, H, (2, 3), (0, 1))
    assert float(O.trace(H2, (0, 1), (2, 3)).blocks[()]) == pytest.approx(g["trace_H2"], abs=1e-15)


def test_heisenberg_fused_matrix_and_two_routes():
    """Sec. II.B: H_mat sectors nu in {-2,0,2} with dims {1,2,1}; tensordot(H,H) equals
    (H_mat @ H_mat).unfuse_legs((0,1)) in structure and values."""
    g = _golden("heisenberg_two_site.json")
    H = _tensor_from_golden(g)
    Hm = O.fuse(H, ((0, 1), (2, 3)))
    assert Hm.sig == (1, -1)
    for leg, key in ((0, "H_mat_leg0_sectors"), (1, "H_mat_leg1_sectors")):
        want = {tuple(q): d for q, d in g[key]}
        assert O.leg_sectors(Hm, leg) == want
    want_blocks = {tuple(tuple(c) for c in k): np.array(v) for k, v in g["H_mat_blocks"]}
    assert sorted(Hm.blocks) == sorted(want_blocks)
    for k, v in want_blocks.items():
        np.testing.assert_array_equal(Hm.blocks[k], v)
    route1 = O.tensordot(H, H, (2, 3), (0, 1))
    route2 = O.unfuse(O.tensordot(Hm, Hm, (1,), (0,)), (0, 1))
    assert sorted(route1.blocks) == sorted(route2.blocks)
    for k in route1.blocks:
        np.testing.assert_allclose(route2.blocks[k], route1.blocks[k], atol=1e-15)


# ---------------------------------------------------------------- hand-derived counts

def test_config1_structure_counts():
    """Hand-derived block/element/sector counts of the U(1) rank-3 workload."""
    g = _golden("config1_structure.json")
    cfg = W.config1()
    A, B = O.from_record(cfg["A"]), O.from_record(cfg["B"])
    assert len(A.blocks) == g["A_blocks"]
    assert sum(b.size for b in A.blocks.values()) == g["A_elements"]
    C = O.tensordot(A, B, cfg["axa"], cfg["axb"])
    assert len(C.blocks) == g["C_blocks"]
    assert sum(b.size for b in C.blocks.values()) == g["C_elements"]
    assert O.useful_flops(A, B, cfg["axa"], cfg["axb"]) == g["useful_flops"]
    # sector view: rows/cols of each contracted charge x
    for x, M, N, K in g["sectors"]:
        rows = {k[:2] for k in A.blocks if k[2] == (x,)}
        cols = {k[1:] for k in B.blocks if k[0] == (x,)}
        assert sum(A.blocks[next(k for k in A.blocks if k[:2] == r)].shape[0] for r in rows) == M
        assert sum(B.blocks[next(k for k in B.blocks if k[1:] == c)].shape[2] for c in cols) == N
        assert cfg["A"]["D"][[i for i, k in enumerate(sorted(A.blocks)) if k[2] == (x,)][0], 2] == K


# ---------------------------------------------------------------- brute force

SYMS = {"U1": (0,), "Z2": (2,), "Z3": (3,), "U1xU1": (0, 0)}


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(12))
def test_tensordot_equals_dense_brute_force(sym, case):
    """Symmetric contraction == dense contraction of the block-embedded tensors, and the
    dense result vanishes outside C's blocks (Sec. II.A block form, Sec. II.B contraction)."""
    mods = SYMS[sym]
    rng = np.random.default_rng(1000 * case + len(sym))
    rankA = int(rng.integers(1, 5))
    rankB = int(rng.integers(1, 5))
    ncon = int(rng.integers(0, min(rankA, rankB) + 1))
    A, B, axa, axb, legsA, legsB = random_pair(rng, mods, rankA, rankB, ncon)
    oA, oB = O.from_record(A), O.from_record(B)
    C = O.tensordot(oA, oB, axa, axb)
    dA = O.to_dense(oA, [leg_map(l) for l in legsA])
    dB = O.to_dense(oB, [leg_map(l) for l in legsB])
    want = np.tensordot(dA, dB, axes=(axa, axb))
    freeA = [i for i in range(rankA) if i not in axa]
    freeB = [i for i in range(rankB) if i not in axb]
    legsC = [leg_map(legsA[i]) for i in freeA] + [leg_map(legsB[i]) for i in freeB]
    got = O.to_dense(C, legsC)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    # every C block conserves charge n_A + n_B
    C.validate()
    assert C.n == tuple((a + b) % m if m else a + b for a, b, m in zip(A["n"], B["n"], mods))


def test_trivial_symmetry_is_dense_tensordot():
    """All charges zero: one block per tensor, the result is numpy.tensordot itself."""
    rng = np.random.default_rng(7)
    legs = [W.Leg(1, [(0,)], [d]) for d in (3, 4, 5)]
    legsB = [W.Leg(-1, [(0,)], [5]), W.Leg(1, [(0,)], [2])]
    A = O.from_record(W.random_tensor((0,), legs, (0,), 11))
    B = O.from_record(W.random_tensor((0,), legsB, (0,), 12))
    C = O.tensordot(A, B, (2,), (0,))
    assert list(C.blocks) == [((0,), (0,), (0,))]
    want = np.tensordot(A.blocks[((0,), (0,), (0,))], B.blocks[((0,), (0,))], axes=((2,), (0,)))
    np.testing.assert_array_equal(C.blocks[((0,), (0,), (0,))], want)
    del rng


def test_full_contraction_is_rank0_dot_product():
    """Contracting every leg gives a rank-0 tensor holding the dense inner product."""
    rng = np.random.default_rng(3)
    legs = random_legs(rng, (0,), 3)
    A = O.from_record(W.random_tensor((0,), legs, (0,), 21))
    B = O.from_record(W.random_tensor((0,), [l.conj() for l in legs], (0,), 22))
    C = O.tensordot(A, B, (0, 1, 2), (0, 1, 2))
    dA = O.to_dense(A, [leg_map(l) for l in legs])
    dB = O.to_dense(B, [leg_map(l) for l in legs])
    if A.blocks:
        assert C.rank == 0 and list(C.blocks) == [()]
        assert float(C.blocks[()]) == pytest.approx(float(np.sum(dA * dB)), rel=1e-13)


def test_no_matching_pair_gives_empty_result():
    """Contracted charges present on one side only contribute nothing (not an error)."""
    la = W.Leg(1, [(0,), (1,)], [2, 2])
    A = O.from_record(W.random_tensor((0,), [la, W.Leg(-1, [(0,), (1,)], [2, 2])], (0,), 1))
    lb = W.Leg(1, [(5,)], [3])
    B = O.from_record(W.random_tensor((0,), [lb, W.Leg(-1, [(5,)], [1])], (0,), 2))
    assert len(B.blocks) == 1
    C = O.tensordot(A, B, (1,), (0,))
    assert C.blocks == {}


# ---------------------------------------------------------------- errors (compatibility)

def test_incompatible_legs_raise():
    l = W.Leg(1, [(0,), (1,)], [2, 3])
    A = O.from_record(W.random_tensor((0,), [l, l.conj()], (0,), 1))
    with pytest.raises(O.SignatureError):
        O.tensordot(A, A, (0,), (0,))
    lb = W.Leg(-1, [(0,), (1,)], [2, 4])
    B = O.from_record(W.random_tensor((0,), [lb, W.Leg(1, [(0,), (1,)], [2, 4])], (0,), 2))
    with pytest.raises(O.DimMismatchError):
        O.tensordot(A, B, (1,), (1,))
    F = O.fuse(A, ((0, 1),))
    with pytest.raises(O.FusionMismatchError):
        O.tensordot(F, O.from_record(W.random_tensor((0,), [W.Leg(-1, [(0,)], [13])], (0,), 3)), (0,), (0,))
    with pytest.raises(O.InvalidError):
        O.tensordot(A, A, (0, 0), (1, 1))


def test_charge_conservation_is_checked():
    rec = W.random_tensor((0,), [W.Leg(1, [(0,), (1,)], [1, 1]), W.Leg(-1, [(0,), (1,)], [1, 1])], (0,), 5)
    rec = dict(rec)
    rec["t"] = rec["t"].copy()
    rec["t"][0, 0, 0] = 7
    with pytest.raises(O.ChargeError):
        O.from_record(rec)


# ---------------------------------------------------------------- fusion

@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(6))
def test_fuse_unfuse_roundtrip_and_sizes(sym, case):
    """unfuse(fuse(T)) == T for fully populated T; sum_nu D_nu <= prod D with equality
    when every charge combination occurs (Sec. II.B, fused dimension)."""
    mods = SYMS[sym]
    rng = np.random.default_rng(77 + case)
    rank = int(rng.integers(2, 6))
    legs = random_legs(rng, mods, rank)
    T = O.from_record(W.random_tensor(mods, legs, tuple([0] * len(mods)), 100 + case))
    if not T.blocks:
        return
    perm = [int(a) for a in rng.permutation(rank)]
    cut = int(rng.integers(1, rank))
    groups = (tuple(perm[:cut]), tuple(perm[cut:]))
    F = O.fuse(T, groups)
    F.validate()
    assert sum(b.size for b in F.blocks.values()) >= sum(b.size for b in T.blocks.values())
    for gi, g in enumerate(groups):
        if len(g) > 1:
            dsum = sum(O.leg_sectors(F, gi).values())
            assert dsum <= int(np.prod([legs[a].dim for a in g]))
    U = O.unfuse(F, [i for i, g in enumerate(groups) if len(g) > 1])
    # unfuse restores the legs in group order: permute T's keys the same way
    order = [a for g in groups for a in g]
    want = {tuple(k[a] for a in order): np.transpose(v, order) for k, v in T.blocks.items()}
    for k, v in want.items():
        np.testing.assert_array_equal(U.blocks[k], v)
    # extra blocks of U (zero-filled sub-blocks) must be exactly zero
    for k in set(U.blocks) - set(want):
        assert not np.any(U.blocks[k])


def test_full_product_leg_dimension_equality():
    """Every charge combination present: sum_nu D_nu = prod D exactly."""
    l1 = W.Leg(1, [(-1,), (0,), (1,)], [2, 1, 3])
    l2 = W.Leg(1, [(0,), (2,)], [2, 2])
    # a third dummy leg absorbs any total charge, so every (rho1, rho2) pair is stored
    l3 = W.Leg(-1, [(q,) for q in range(-1, 4)], [1] * 5)
    T = O.from_record(W.random_tensor((0,), [l1, l2, l3], (0,), 4))
    F = O.fuse(T, ((0, 1), (2,)))
    assert sum(O.leg_sectors(F, 0).values()) == l1.dim * l2.dim
    assert O.leg_sectors(F, 0) == {(-1,): 4, (0,): 2, (1,): 10, (2,): 2, (3,): 6}


@pytest.mark.parametrize("case", range(6))
def test_fused_matrix_has_same_singular_values(case):
    """Fusion only reorders rows and columns of the matricised dense tensor: the dense
    embedding of fuse(T, ((0,1),(2,3))) has the singular values of dense(T) reshaped."""
    rng = np.random.default_rng(500 + case)
    mods = [(0,), (2,), (0, 0)][case % 3]
    legs = random_legs(rng, mods, 4)
    T = O.from_record(W.random_tensor(mods, legs, tuple([0] * len(mods)), 900 + case))
    if not T.blocks:
        return
    dense = O.to_dense(T, [leg_map(l) for l in legs])
    F = O.fuse(T, ((0, 1), (2, 3)))
    dF = O.to_dense(F)
    sv1 = np.linalg.svd(dense.reshape(dense.shape[0] * dense.shape[1], -1), compute_uv=False)
    sv2 = np.linalg.svd(dF, compute_uv=False)
    k = min(len(sv1), len(sv2))
    np.testing.assert_allclose(sv2[:k], sv1[:k], rtol=1e-12, atol=1e-12)
    assert np.all(np.abs(sv1[k:]) < 1e-12) and np.all(np.abs(sv2[k:]) < 1e-12)


def test_fused_charge_rule():
    """nu = s_r (s_i rho + s_j rho') with s_r the first leg's signature (Sec. II.B)."""
    l1 = W.Leg(-1, [(0,), (1,), (2,)], [1, 1, 1])
    l2 = W.Leg(1, [(0,), (3,)], [1, 2])
    l3 = W.Leg(1, [(q,) for q in range(-6, 7)], [1] * 13)
    T = O.from_record(W.random_tensor((0,), [l1, l2, l3], (0,), 9))
    F = O.fuse(T, ((0, 1), (2,)))
    # s_r = -1: nu = -(-rho + rho') = rho - rho'
    want = {}
    for q1, d1 in zip(l1.t, l1.D):
        for q2, d2 in zip(l2.t, l2.D):
            nu = (q1[0] - q2[0],)
            want[nu] = want.get(nu, 0) + d1 * d2
    assert O.leg_sectors(F, 0) == want


def test_fused_contraction_matches_unfused():
    """Contracting fused legs gives the unfused contraction after unfusing (Sec. II.B)."""
    rng = np.random.default_rng(42)
    legs = random_legs(rng, (0,), 4, max_sectors=3, max_dim=3)
    A = O.from_record(W.random_tensor((0,), legs, (0,), 1))
    # B's legs (l2*, l3*, l0*, l1*) allow exactly the (rho2, rho3) combinations that A
    # allows, so the lazy fusion records of the contracted fused legs are conjugate.
    B = O.from_record(W.random_tensor((0,), [legs[2].conj(), legs[3].conj(), legs[0].conj(), legs[1].conj()], (0,), 2))
    direct = O.tensordot(A, B, (2, 3), (0, 1))
    Am = O.fuse(A, ((0, 1), (2, 3)))
    Bm = O.fuse(B, ((0, 1), (2, 3)))
    via = O.unfuse(O.tensordot(Am, Bm, (1,), (0,)), (0, 1))
    dl = [leg_map(legs[0]), leg_map(legs[1]), leg_map(legs[0]), leg_map(legs[1])]
    np.testing.assert_allclose(O.to_dense(via, dl), O.to_dense(direct, dl), rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- trace

@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(5))
def test_trace_equals_dense_trace(sym, case):
    mods = SYMS[sym]
    rng = np.random.default_rng(300 + case)
    base = random_legs(rng, mods, 2)
    other = random_legs(rng, mods, int(rng.integers(0, 3)))
    legs = [base[0], base[1], base[0].conj(), base[1].conj()] + other
    npair = int(rng.integers(1, 3))
    ax1, ax2 = (0, 1)[:npair], (2, 3)[:npair]
    T = O.from_record(W.random_tensor(mods, legs, tuple([0] * len(mods)), 40 + case))
    R = O.trace(T, ax1, ax2)
    dense = O.to_dense(T, [leg_map(l) for l in legs])
    sub = "abcdefgh"[:len(legs)]
    sub_l = list(sub)
    for a, b in zip(ax1, ax2):
        sub_l[b] = sub_l[a]
    out = "".join(c for i, c in enumerate(sub_l) if i not in ax1 + ax2)
    want = np.einsum("".join(sub_l) + "->" + out, dense)
    rest = [i for i in range(len(legs)) if i not in ax1 + ax2]
    got = O.to_dense(R, [leg_map(legs[i]) for i in rest])
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_trace_signature_rule():
    l = W.Leg(1, [(0,), (1,)], [2, 2])
    T = O.from_record(W.random_tensor((0,), [l, l, W.Leg(-1, [(q,) for q in range(3)], [1, 1, 1])], (0,), 3))
    with pytest.raises(O.SignatureError):
        O.trace(T, (0,), (1,))


def test_fuse_sub_block_order_convention():
    """Hand-worked fusion with unequal sub-block sizes: fixes the sub-block order
    (ascending constituent charges) and the row-major placement inside a sector."""
    g = _golden("fuse_order_example.json")
    legs = [W.Leg(s, [tuple(q) for q in t], D) for s, t, D in g["legs"]]
    rec = W.random_tensor((0,), legs, (0,), 0, fill="ones")
    rec["data"] = np.array(g["data"], dtype=np.float64)
    T = O.from_record(rec)
    F = O.fuse(T, ((0, 1), (2,)))
    want = {tuple(tuple(c) for c in k): np.array(v, dtype=np.float64) for k, v in g["fused_blocks"]}
    assert sorted(F.blocks) == sorted(want)
    for k, v in want.items():
        np.testing.assert_array_equal(F.blocks[k], v)


@pytest.mark.parametrize("mods,n,want", [((0,), (1,), (-1,)), ((3,), (1,), (2,)), ((0, 2), (2, 1), (-2, 1))])
def test_conj_flips_signatures_and_charge(mods, n, want):
    """Conjugation flips every signature (Sec. II.A footnote); the blocks then conserve
    -n, so the total charge of the conjugate is -n."""
    rng = np.random.default_rng(sum(n) + len(mods))
    legs = random_legs(rng, mods, 3)
    T = O.from_record(W.random_tensor(mods, legs, n, 8))
    Tc = O.conj(T)
    Tc.validate()
    assert Tc.sig == tuple(-s for s in T.sig)
    assert Tc.n == want


@pytest.mark.parametrize("case", range(4))
def test_tensordot_block_matches_tensordot(case):
    """The single-block evaluation used for sampled checks of large contractions gives
    the same blocks as the full contraction."""
    rng = np.random.default_rng(4242 + case)
    mods = [(0,), (2,), (0, 0), (3,)][case]
    A, B, axa, axb, _, _ = random_pair(rng, mods, 3, 3, 2)
    oA, oB = O.from_record(A), O.from_record(B)
    C = O.tensordot(oA, oB, axa, axb)
    for k, v in C.blocks.items():
        np.testing.assert_allclose(O.tensordot_block(oA, oB, axa, axb, k), v, rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- scalar products

@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(8))
def test_vdot_equals_dense_scalar_product(sym, case):
    """<A, B> of two tensors on the same legs == numpy.vdot of their dense embeddings,
    also when B lacks some of A's blocks; <A, A> is the squared Frobenius norm."""
    mods = SYMS[sym]
    rng = np.random.default_rng(7000 + 31 * case + len(sym))
    legs = random_legs(rng, mods, int(rng.integers(1, 5)))
    n = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    A = O.from_record(W.random_tensor(mods, legs, n, 2 * case + 1))
    B = O.from_record(W.random_tensor(mods, legs, n, 2 * case + 2))
    for k in list(B.blocks)[::3]:
        del B.blocks[k]
    lm = [leg_map(l) for l in legs]
    dA, dB = O.to_dense(A, lm), O.to_dense(B, lm)
    assert O.vdot(A, B) == pytest.approx(float(np.vdot(dA, dB)), rel=1e-12, abs=1e-12)
    assert O.vdot(A, A) == pytest.approx(float(np.sum(dA * dA)), rel=1e-12, abs=1e-300)
    assert O.vdot(A, A) >= 0.0


def test_vdot_is_the_full_contraction_with_the_dual_tensor():
    """<A, B> == tensordot over every leg of A with B on dual legs (flipped signatures
    and total charge), a different route through the oracle."""
    rng = np.random.default_rng(11)
    legs = random_legs(rng, (0, 0), 3)
    A = O.from_record(W.random_tensor((0, 0), legs, (0, 0), 5))
    B = O.from_record(W.random_tensor((0, 0), legs, (0, 0), 6))
    Bd = O.OTensor(B.mods, tuple(-s for s in B.sig), tuple(-q for q in B.n), dict(B.blocks))
    C = O.tensordot(A, Bd, (0, 1, 2), (0, 1, 2))
    want = float(C.blocks[()]) if C.blocks else 0.0
    assert O.vdot(A, B) == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_vdot_is_invariant_under_fusion():
    """Fusion only relabels and regroups elements (Sec. II.B): <fuse A, fuse B> == <A, B>."""
    rng = np.random.default_rng(13)
    legs = random_legs(rng, (0,), 4)
    A = O.from_record(W.random_tensor((0,), legs, (0,), 7))
    B = O.from_record(W.random_tensor((0,), legs, (0,), 8))
    g = ((0, 2), (1, 3))
    assert O.vdot(O.fuse(A, g), O.fuse(B, g)) == pytest.approx(O.vdot(A, B), rel=1e-12, abs=1e-12)


def test_heisenberg_norm():
    """The paper's two-spin example: ||H||^2 = Tr H^2 = 3/4 (H is symmetric)."""
    g = _golden("heisenberg_two_site.json")
    H = _tensor_from_golden(g)
    assert O.vdot(H, H) == pytest.approx(g["trace_H2"], abs=1e-15)


def test_vdot_rejects_incomparable_tensors():
    l = W.Leg(1, [(-1,), (1,)], [2, 3])
    A = O.from_record(W.random_tensor((0,), [l, l.conj()], (0,), 1))
    with pytest.raises(O.SignatureError):
        O.vdot(A, O.from_record(W.random_tensor((0,), [l.conj(), l], (0,), 2)))
    l2 = W.Leg(1, [(-1,), (1,)], [2, 4])
    with pytest.raises(O.DimMismatchError):
        O.vdot(A, O.from_record(W.random_tensor((0,), [l2, l2.conj()], (0,), 3)))
    with pytest.raises(O.InvalidError):
        O.vdot(A, O.from_record(W.random_tensor((2,), [W.Leg(1, [(0,), (1,)], [2, 3])] * 2, (0,), 4)))


# ---------------------------------------------------------------- fermionic swap gates

FERMI_SYMS = {"U1": (0,), "Z2": (2,), "U1xU1": (0, 0)}


def _dense_parities(legs):
    """Per leg, the parity of every dense index: the parity of its sector's charge
    (sum of the components, all fermionic), sectors in ascending charge order."""
    out = []
    for lg in legs:
        lm = leg_map(lg)
        out.append(np.concatenate([np.full(lm[q], sum(q) % 2) for q in sorted(lm)]))
    return out


def _dense_sign(par, g1, g2):
    """(-1)^(P1 P2) on the dense index grid, P_g = sum of the group's index parities."""
    grids = np.meshgrid(*par, indexing="ij")
    p1 = sum(grids[a] for a in g1) % 2 if g1 else 0
    p2 = sum(grids[b] for b in g2) % 2 if g2 else 0
    return np.where((p1 * p2) % 2 == 1, -1.0, 1.0)


@pytest.mark.parametrize("sym", list(FERMI_SYMS))
@pytest.mark.parametrize("case", range(8))
def test_swap_gate_equals_dense_parity_sign(sym, case):
    """Sec. IV: a swap gate changes the sign where both crossing lines are odd. On the
    dense embedding this is the element-wise product with (-1)^(P1 P2), P the parity
    of a group's indices -- checked element by element."""
    mods = FERMI_SYMS[sym]
    rng = np.random.default_rng(8100 + 13 * case + len(sym))
    rank = int(rng.integers(2, 5))
    legs = random_legs(rng, mods, rank)
    n = tuple(int(rng.integers(0, m)) if m else int(rng.integers(-1, 2)) for m in mods)
    A = O.from_record(W.random_tensor(mods, legs, n, case + 1))
    perm = [int(x) for x in rng.permutation(rank)]
    k1 = int(rng.integers(1, rank))
    k2 = int(rng.integers(1, rank - k1 + 1))
    g1, g2 = perm[:k1], perm[k1:k1 + k2]
    lm = [leg_map(lg) for lg in legs]
    got = O.to_dense(O.swap_gate(A, g1, g2), lm)
    want = O.to_dense(A, lm) * _dense_sign(_dense_parities(legs), g1, g2)
    np.testing.assert_array_equal(got, want)


def test_swap_gate_is_an_involution_and_bilinear():
    """Applying a swap gate twice is the identity; a gate against a union of two groups
    is the product of the two gates (the parity of a union is the sum of parities)."""
    rng = np.random.default_rng(17)
    legs = random_legs(rng, (0, 0), 4)
    A = O.from_record(W.random_tensor((0, 0), legs, (1, 0), 3))
    S = O.swap_gate(O.swap_gate(A, (0,), (2, 3)), (0,), (2, 3))
    assert all(np.array_equal(S.blocks[k], A.blocks[k]) for k in A.blocks)
    one = O.swap_gate(A, (0, 1), (2, 3))
    two = O.swap_gate(O.swap_gate(A, (0, 1), (2,)), (0, 1), (3,))
    assert all(np.array_equal(one.blocks[k], two.blocks[k]) for k in A.blocks)


def test_swap_gate_fermionic_swap_of_two_modes():
    """Closed form: the swap gate applied to the permutation P[o1, o2, i1, i2] =
    delta(o1, i2) delta(o2, i1) of two spinless fermionic modes (Z2, |0>, |1>) gives
    the fermionic SWAP, diag(1, 1, 1, -1) times the swap of the occupations."""
    l = W.Leg(1, [(0,), (1,)], [1, 1])
    blocks = {}
    for a in (0, 1):
        for b in (0, 1):
            blocks[((a,), (b,), (b,), (a,))] = np.ones((1, 1, 1, 1))
    P = O.OTensor((2,), (1, 1, -1, -1), (0,), blocks).validate()
    F = O.swap_gate(P, (2,), (3,))
    lm = [leg_map(l)] * 4
    mat = O.to_dense(F, lm).reshape(4, 4)
    want = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, -1]], dtype=np.float64)
    np.testing.assert_array_equal(mat, want)


def test_swap_gate_special_cases():
    """Bosonic components (no fermionic flag) and even groups leave every block as it
    is; a Z3 component cannot carry a parity."""
    rng = np.random.default_rng(19)
    legs = random_legs(rng, (2,), 3)
    A = O.from_record(W.random_tensor((2,), legs, (0,), 5))
    B = O.swap_gate(A, (0,), (1,), fermionic=(False,))
    assert all(np.array_equal(B.blocks[k], A.blocks[k]) for k in A.blocks)
    ev = W.Leg(1, [(0,), (2,)], [2, 3])
    od = W.Leg(1, [(-1,), (1,)], [1, 2])
    T = O.from_record(W.random_tensor((0,), [ev, od, od.conj()], (0,), 6))
    S = O.swap_gate(T, (0,), (1, 2))
    assert all(np.array_equal(S.blocks[k], T.blocks[k]) for k in T.blocks)
    U = O.swap_gate(T, (1,), (2,))
    assert any(not np.array_equal(U.blocks[k], T.blocks[k]) for k in T.blocks)
    with pytest.raises(O.InvalidError):
        O.swap_gate(O.from_record(W.random_tensor((3,), random_legs(rng, (3,), 2), (0,), 7)), (0,), (1,))
    with pytest.raises(O.InvalidError):
        O.swap_gate(A, (0, 1), (1,))


# ---------------------------------------------------------------- fusion-history mismatch

@pytest.mark.parametrize("drops", [(1, None), (None, -1), (1, -1), (0, 1)])
def test_fusion_mismatch_is_zero_padding(drops):
    """Sec. II.B footnote: a charge of the fusion history missing on one contracted
    fused leg but present on its partner is resolved. The result equals the ordinary
    contraction of the zero-padded tensors, whose records agree."""
    A, B, A_pad, B_pad, _, _ = fusion_mismatch_pair(*drops)
    assert A.fus[0].key() != B.fus[0].conj().key()
    assert A_pad.fus[0].key() == B_pad.fus[0].conj().key()
    got = O.tensordot(A, B, (0,), (0,))
    want = O.tensordot(A_pad, B_pad, (0,), (0,))
    assert set(got.blocks) <= set(want.blocks)
    for k in want.blocks:
        ref = want.blocks[k]
        np.testing.assert_allclose(got.blocks.get(k, np.zeros_like(ref)), ref, rtol=1e-13, atol=1e-13)


def test_fusion_mismatch_matches_the_dense_constituent_contraction():
    """The resolved contraction over the fused leg is the contraction over its
    constituent legs, checked on dense embeddings with numpy."""
    A, B, _, _, a, b = fusion_mismatch_pair(1, -1)
    C = O.tensordot(A, B, (0,), (0,))
    la = [O.leg_sectors(a, i) for i in range(3)]
    lb = [O.leg_sectors(b, i) for i in range(3)]
    for i in range(2):          # common basis of the contracted constituent legs
        merged = dict(la[i])
        merged.update(lb[i])
        la[i] = lb[i] = merged
    want = np.tensordot(O.to_dense(a, la), O.to_dense(b, lb), axes=((0, 1), (0, 1)))
    lc = [la[2], lb[2]]
    np.testing.assert_allclose(O.to_dense(C, lc), want, rtol=1e-13, atol=1e-13)


def test_fusion_mismatch_errors():
    """Fused legs from a different number of constituents, or disagreeing on the
    dimension of a common constituent charge, are not resolvable."""
    A, B, _, _, a, _ = fusion_mismatch_pair(1, None)
    l0 = W.Leg(-1, [(-1,), (0,), (1,)], [2, 3, 1])
    l1 = W.Leg(-1, [(0,), (1,)], [2, 2])
    l1b = W.Leg(-1, [(0,), (1,)], [2, 5])
    lx = W.Leg(-1, [(0,)], [1])
    l3 = W.Leg(1, [(-1,), (0,), (1,)], [1, 1, 1])
    three = O.fuse(O.from_record(W.random_tensor((0,), [l0, l1, lx, l3], (0,), 5)), ((0, 1, 2), (3,)))
    with pytest.raises(O.FusionMismatchError):
        O.tensordot(A, three, (0,), (0,))
    wrong = O.fuse(O.from_record(W.random_tensor((0,), [l0, l1b, l3], (0,), 6)), ((0, 1), (2,)))
    with pytest.raises(O.DimMismatchError):
        O.tensordot(A, wrong, (0,), (0,))


# ---------------------------------------------------------------- networks (ncon)

@pytest.mark.parametrize("sym", ["U1", "Z2", "U1xU1"])
@pytest.mark.parametrize("kind", ["chain", "trace", "outer"])
@pytest.mark.parametrize("case", range(3))
def test_ncon_equals_dense_einsum(sym, kind, case):
    """ncon of a network == numpy.einsum of the dense embeddings with the same labels
    (a library routine as the independent route; output legs -1, -2, ... in order)."""
    mods = SYMS[sym]
    rng = np.random.default_rng(8700 + 31 * case + len(sym) + len(kind))
    legs, ts, labels = random_network(rng, mods, kind)
    C = O.ncon([O.from_record(t) for t in ts], labels)
    letters = {}
    def sub(lab):
        return "".join(letters.setdefault(x, "abcdefghijklmnop"[len(letters)]) for x in lab)
    dense = [O.to_dense(O.from_record(t), [leg_map(l) for l in lg]) for t, lg in zip(ts, legs)]
    outl = sorted({x for lab in labels for x in lab if x < 0}, reverse=True)
    spec = ",".join(sub(lab) for lab in labels) + "->" + sub(outl)
    want = np.einsum(spec, *dense)
    out_legs = {x: leg_map(l) for lg, lab in zip(legs, labels) for l, x in zip(lg, lab) if x < 0}
    got = O.to_dense(C, [out_legs[x] for x in outl])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_ncon_two_spin_example():
    """The paper's example H2 = tensordot(H, H, axes=((2, 3), (0, 1))) as a network:
    ncon([H, H], [[-1, -2, 1, 2], [1, 2, -3, -4]]) gives (S1.S2)^2 = 3/16 - H/2."""
    g = _golden("heisenberg_two_site.json")
    H = _tensor_from_golden(g)
    H2 = O.ncon([H, H], [[-1, -2, 1, 2], [1, 2, -3, -4]])
    ref = O.tensordot(H, H, (2, 3), (0, 1))
    for k in set(H2.blocks) | set(ref.blocks):
        np.testing.assert_allclose(H2.blocks[k], ref.blocks[k], atol=1e-15)
        want = 3.0 / 16 * (1.0 if k[:2] == k[2:] else 0.0) - 0.5 * (H.blocks[k] if k in H.blocks else 0.0)
        np.testing.assert_allclose(H2.blocks[k], np.full_like(H2.blocks[k], want), atol=1e-15)


def test_ncon_label_errors():
    l = W.Leg(1, [(0,), (1,)], [2, 3])
    A = O.from_record(W.random_tensor((0,), [l, l.conj()], (0,), 1))
    for labels in ([[1, 1, 2]], [[1, -1]], [[-1, -3]], [[0, -1]], [[1, 2]]):
        with pytest.raises(O.InvalidError):
            O.ncon([A], labels)


# ---------------------------------------------------------------- complex128

def _parts(T):
    """Real and imaginary parts of a complex OTensor as real OTensors."""
    re = O.OTensor(T.mods, T.sig, T.n, {k: v.real.copy() for k, v in T.blocks.items()}, list(T.fus), np.float64)
    im = O.OTensor(T.mods, T.sig, T.n, {k: v.imag.copy() for k, v in T.blocks.items()}, list(T.fus), np.float64)
    return re, im


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(6))
def test_complex_tensordot_equals_dense(sym, case):
    """Complex data (Sec. II.A footnote): tensordot == numpy.tensordot of the complex
    dense embeddings, and == the four real products (re re - im im) + i (re im + im re)
    of the real oracle."""
    mods = SYMS[sym]
    rng = np.random.default_rng(9900 + 13 * case + len(sym))
    rankA, rankB = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    ncon = int(rng.integers(0, min(rankA, rankB) + 1))
    A, B, axa, axb, legsA, legsB = random_pair(rng, mods, rankA, rankB, ncon, dtype="c128")
    oA, oB = O.from_record(A), O.from_record(B)
    assert oA.dtype == np.complex128 and oB.dtype == np.complex128
    C = O.tensordot(oA, oB, axa, axb)
    lmA, lmB = [leg_map(l) for l in legsA], [leg_map(l) for l in legsB]
    want = np.tensordot(O.to_dense(oA, lmA), O.to_dense(oB, lmB), axes=(axa, axb))
    freeA = [lmA[i] for i in range(rankA) if i not in axa]
    freeB = [lmB[i] for i in range(rankB) if i not in axb]
    np.testing.assert_allclose(O.to_dense(C, freeA + freeB), want, rtol=1e-12, atol=1e-12)
    (ar, ai), (br, bi) = _parts(oA), _parts(oB)
    rr, ii = O.tensordot(ar, br, axa, axb), O.tensordot(ai, bi, axa, axb)
    ri, ir = O.tensordot(ar, bi, axa, axb), O.tensordot(ai, br, axa, axb)
    for k in C.blocks:
        np.testing.assert_allclose(C.blocks[k].real, rr.blocks[k] - ii.blocks[k], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(C.blocks[k].imag, ri.blocks[k] + ir.blocks[k], rtol=1e-12, atol=1e-12)


def test_complex_conj_vdot_fuse_trace_swap():
    """conj conjugates the elements (and flips the structure); <A, B> = sum conj(a) b
    (numpy.vdot of the dense embeddings), <A, B> = conj(<B, A>), <A, A> = ||A||^2 > 0;
    fuse/unfuse round trip, trace and swap gate keep the complex values."""
    rng = np.random.default_rng(41)
    legs = random_legs(rng, (0,), 4, max_sectors=3, max_dim=3)
    A = O.from_record(W.random_tensor((0,), legs, (0,), 1, dtype="c128"))
    B = O.from_record(W.random_tensor((0,), legs, (0,), 2, dtype="c128"))
    lm = [leg_map(l) for l in legs]
    dA, dB = O.to_dense(A, lm), O.to_dense(B, lm)
    Ac = O.conj(A)
    np.testing.assert_array_equal(O.to_dense(Ac, lm), np.conj(dA))
    assert Ac.sig == tuple(-s for s in A.sig)
    assert O.vdot(A, B) == pytest.approx(np.vdot(dA, dB), rel=1e-12, abs=1e-12)
    assert O.vdot(A, B) == pytest.approx(np.conj(O.vdot(B, A)), rel=1e-13, abs=1e-13)
    nrm = O.vdot(A, A)
    assert abs(nrm.imag) < 1e-12 and nrm.real == pytest.approx(float(np.sum(np.abs(dA) ** 2)), rel=1e-12)
    F = O.fuse(A, ((0, 2), (1, 3)))
    assert F.dtype == np.complex128
    U = O.unfuse(F, (0, 1))     # legs now in the order 0, 2, 1, 3
    for k, v in A.blocks.items():
        np.testing.assert_array_equal(U.blocks[(k[0], k[2], k[1], k[3])], np.transpose(v, (0, 2, 1, 3)))
    S = O.swap_gate(A, (0,), (1, 2))
    par = [np.concatenate([np.full(lm[a][q], q[0] % 2) for q in sorted(lm[a])]) for a in range(4)]
    g = np.meshgrid(*par, indexing="ij")
    sign = np.where((g[0] * ((g[1] + g[2]) % 2)) % 2 == 1, -1.0, 1.0)
    np.testing.assert_array_equal(O.to_dense(S, lm), dA * sign)
    l = W.Leg(1, [(0,), (1,)], [2, 3])
    T = O.from_record(W.random_tensor((0,), [l, l.conj(), legs[0]], (0,), 3, dtype="c128"))
    tr = O.trace(T, (0,), (1,))
    dT = O.to_dense(T, [leg_map(l), leg_map(l), lm[0]])
    np.testing.assert_allclose(O.to_dense(tr, [lm[0]]), np.einsum("iik->k", dT), rtol=1e-13, atol=1e-13)


def test_einsum_equals_numpy_einsum():
    """einsum subscripts (Sec. II.B: einsum and ncon differ only by syntax) against
    numpy.einsum of the dense embeddings: a chain, a trace, implicit output order."""
    rng = np.random.default_rng(61)
    for spec, kind in (("abc,bde,cef->adf", "chain"), ("abbc,cd->da", "trace"), ("ab,bc,de", "outer")):
        legs, ts, labels = random_network(rng, (0,), kind)
        C = O.einsum(spec, *[O.from_record(t) for t in ts])
        dense = [O.to_dense(O.from_record(t), [leg_map(l) for l in lg]) for t, lg in zip(ts, legs)]
        want = np.einsum(spec, *dense)
        lhs = spec.split("->")[0].split(",")
        where = {c: leg_map(legs[i][k]) for i, grp in enumerate(lhs) for k, c in enumerate(grp)}
        out = spec.split("->")[1] if "->" in spec else "".join(sorted(c for c in where if "".join(lhs).count(c) == 1))
        np.testing.assert_allclose(O.to_dense(C, [where[c] for c in out]), want, rtol=1e-12, atol=1e-12)
    l = W.Leg(1, [(0,), (1,)], [2, 3])
    A = O.from_record(W.random_tensor((0,), [l, l.conj()], (0,), 1))
    for bad in ("aa->a", "ab,ab,ab->", "ab->abc", "a1,b"):
        with pytest.raises(O.InvalidError):
            O.einsum(bad, A, A) if bad.count(",") == 1 else O.einsum(bad, A)


# ---------------------------------------------------------------- block-diagonal SVD

def _svd_case(seed, mods=(0,), dtype="f64"):
    rng = np.random.default_rng(seed)
    pool = [(0,), (1,), (-1,)] if mods == (0,) else [(0, 0), (1, 0), (0, 1), (-1, 0)]
    legs = [W.Leg(s, pool[:3], [int(d) for d in rng.integers(1, 5, 3)]) for s in (1, 1, -1, -1)]
    return legs, O.from_record(W.random_tensor(mods, legs, (0,) * len(mods), seed, dtype=dtype))


def _dense_matrix(A, legs, rows, cols):
    d = O.to_dense(A, [leg_map(l) for l in legs])
    d = np.transpose(d, rows + cols)
    r = int(np.prod([d.shape[i] for i in range(len(rows))]))
    return d.reshape(r, -1)


@pytest.mark.parametrize("dtype", ["f64", "c128"])
@pytest.mark.parametrize("seed", range(4))
def test_svd_reconstructs_and_is_orthonormal(seed, dtype):
    """CTM's SVD (Sec. III) block by block: U S V == A, U^H U = 1 and V V^H = 1 per
    sector, S real, non-negative and descending."""
    legs, A = _svd_case(100 + seed, (0,) if seed % 2 == 0 else (0, 0), dtype)
    rows, cols = (0, 2), (1, 3)
    U, S, V = O.svd(A, rows, cols)
    R = O.tensordot(O.tensordot(U, S, (2,), (0,)), V, (2,), (0,))
    R = O.fuse(R, ((0,), (2,), (1,), (3,)))
    for k in A.blocks:
        np.testing.assert_allclose(R.blocks[k], A.blocks[k], rtol=1e-12, atol=1e-12)
    UU = O.tensordot(O.conj(U), U, (0, 1), (0, 1))
    VV = O.tensordot(V, O.conj(V), (1, 2), (1, 2))
    for (c, _), blk in S.blocks.items():
        sv = np.diag(blk)
        assert np.all(sv >= 0) and np.all(np.diff(sv) <= 0)
        np.testing.assert_allclose(UU.blocks[(c, c)], np.eye(sv.size), atol=1e-12)
        np.testing.assert_allclose(VV.blocks[(c, c)], np.eye(sv.size), atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_svd_values_and_truncation_match_the_dense_svd(seed):
    """The singular values of all sectors are those of the dense matrix (rows = row
    legs); truncating to the D largest leaves the Frobenius error sqrt(sum of the
    discarded s^2) (Eckart-Young), equal to the dense rank-D error."""
    legs, A = _svd_case(200 + seed)
    rows, cols = (0, 3), (1, 2)
    U, S, V = O.svd(A, rows, cols)
    ours = np.sort(np.concatenate([np.diag(b) for b in S.blocks.values()]))[::-1]
    dense = np.linalg.svd(_dense_matrix(A, legs, rows, cols), compute_uv=False)
    nz = ours[ours > 1e-10]
    np.testing.assert_allclose(nz, dense[:nz.size], rtol=1e-12)
    assert np.all(dense[nz.size:] < 1e-10)
    D = max(1, nz.size // 2)
    keep = O.truncation(S, D)
    assert sum(keep.values()) == D
    Ut, St, Vt = O.slice_leg(U, (2,), keep), O.slice_leg(S, (0, 1), keep), O.slice_leg(V, (0,), keep)
    R = O.fuse(O.tensordot(O.tensordot(Ut, St, (2,), (0,)), Vt, (2,), (0,)), ((0,), (2,), (3,), (1,)))
    err = np.linalg.norm(O.to_dense(R, [leg_map(l) for l in legs]) - O.to_dense(A, [leg_map(l) for l in legs]))
    assert err == pytest.approx(float(np.sqrt(np.sum(dense[D:] ** 2))), rel=1e-9, abs=1e-12)
    keep_tol = O.truncation(S, 10 ** 6, tol=0.5)
    assert sum(keep_tol.values()) == int(np.sum(dense >= 0.5 * dense[0]))


@pytest.mark.parametrize("dtype", ["f64", "c128"])
@pytest.mark.parametrize("seed", range(3))
def test_eigh_of_a_hermitian_tensor(seed, dtype):
    """H = B + B^H on legs (r, r*): U diag(w) U^H == H, U^H U = 1, w ascending and
    equal to the dense matrix's eigenvalues (numpy.linalg.eigvalsh)."""
    rng = np.random.default_rng(500 + seed)
    pool = [(0,), (1,), (-1,)]
    r = [W.Leg(s, pool, [int(d) for d in rng.integers(1, 5, 3)]) for s in (1, -1)]
    legs = r + [l.conj() for l in r]
    B = O.from_record(W.random_tensor((0,), legs, (0,), seed, dtype=dtype))
    Bh = O.fuse(O.conj(B), ((2,), (3,), (0,), (1,)))   # conj(B) with rows and columns swapped
    H = O.OTensor(B.mods, B.sig, B.n, {k: B.blocks[k] + Bh.blocks[k] for k in B.blocks}, dtype=B.dtype)
    U, S = O.eigh(H, (0, 1), (2, 3))
    R = O.tensordot(O.tensordot(U, S, (2,), (0,)), O.fuse(O.conj(U), ((2,), (0,), (1,))), (2,), (0,))
    for k in H.blocks:
        np.testing.assert_allclose(R.blocks[k], H.blocks[k], rtol=1e-12, atol=1e-12)
    UU = O.tensordot(O.conj(U), U, (0, 1), (0, 1))
    for (c, _), blk in S.blocks.items():
        w = np.diag(blk)
        assert np.all(np.diff(w) >= 0)
        np.testing.assert_allclose(UU.blocks[(c, c)], np.eye(w.size), atol=1e-12)
    ours = np.sort(np.concatenate([np.diag(b) for b in S.blocks.values()]))
    d = _dense_matrix(H, legs, (0, 1), (2, 3))
    np.testing.assert_allclose(ours, np.linalg.eigvalsh(d), rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- random data

def test_philox_known_answers():
    """Philox4x32-10 against the known-answer vectors published with the generator
    (Salmon et al., SC'11, Random123): zero counter and key, all-ones, and the pi
    digits."""
    assert O.philox4x32((0, 0, 0, 0), (0, 0)) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert O.philox4x32((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert O.philox4x32((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0)) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_normal_fill_is_box_muller_of_philox():
    """Each pair is sqrt(-2 ln u) (cos, sin)(2 pi v) of one pair of Philox words, so
    z0^2 + z1^2 = -2 ln u exactly in the words; over 4e4 numbers the mean and
    variance are those of N(0, 1) within 5 standard errors."""
    z = O.normal_fill(12345, 40000)
    w = O.philox4x32((0, 0, 0, 0), (12345, 0))
    np.testing.assert_allclose(z[0] ** 2 + z[1] ** 2, -2 * np.log((w[0] + 1.0) * 2.0 ** -32), rtol=1e-14)
    np.testing.assert_allclose(z[2] ** 2 + z[3] ** 2, -2 * np.log((w[2] + 1.0) * 2.0 ** -32), rtol=1e-14)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    np.testing.assert_array_equal(O.normal_fill(12345, 7), z[:7])
