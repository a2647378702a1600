"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Structure (blocks, charges, dimensions, offsets) must be bit-exact; pure data
movement (fuse, unfuse) must be bit-exact; FP64 contractions must agree within a
relative Frobenius error of 1e-12 (the bound the FP64 path is held to).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import (FP64_RTOL, check_against_oracle, oracle_tensordot, rel_frobenius,
                         run_move, run_tensordot, same_structure)
from helpers import random_legs, random_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


SYMS = {"U1": (0,), "Z2": (2,), "Z3": (3,), "U1xU1": (0, 0)}


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(10))
def test_random_tensordot_fp64(ctx, sym, case):
    mods = SYMS[sym]
    rng = np.random.default_rng(12000 + 17 * case + len(sym))
    rankA, rankB = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    ncon = int(rng.integers(0, min(rankA, rankB) + 1))
    A, B, axa, axb, _, _ = random_pair(rng, mods, rankA, rankB, ncon, max_sectors=4, max_dim=5)
    _, rec, res = run_tensordot(ctx, A, B, axa, axb)
    check_against_oracle(rec, oracle_tensordot(A, B, axa, axb))


def test_config1(ctx):
    cfg = W.config1()
    plan, rec, res = run_tensordot(ctx, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    check_against_oracle(rec, oracle_tensordot(cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]))
    assert res["useful_flops"] == 5640


@pytest.mark.parametrize("dims", [(1, 1, 1), (64, 64, 16), (65, 63, 17), (200, 130, 77), (3, 300, 5),
                                  (257, 1, 129), (32, 32, 16), (33, 31, 17), (20, 100, 40), (31, 65, 3)])
def test_single_sector_tiles_and_ragged_tails(ctx, dims):
    """One dense sector spanning several tiles with ragged M, N and K tails; the
    planner picks 64x64 tiles for the larger sectors here and 32x32 tiles for the
    small or thin ones ((1,1), (3,300), (257,1), (32,32), (33,31), (20,100), (31,65))."""
    M, N, K = dims
    l_m = W.Leg(1, [(0,)], [M])
    l_k = W.Leg(1, [(0,)], [K])
    l_n = W.Leg(1, [(0,)], [N])
    A = W.random_tensor((0,), [l_m, l_k], (0,), M * 7 + K)
    B = W.random_tensor((0,), [l_k.conj(), l_n], (0,), N * 3 + K)
    _, rec, _ = run_tensordot(ctx, A, B, (1,), (0,))
    want = A["data"].reshape(M, K) @ B["data"].reshape(K, N)
    assert rel_frobenius(rec["data"], want.ravel()) <= FP64_RTOL


def test_multi_leg_permutations(ctx):
    """Contract middle legs in a permuted order: gathers need transposes."""
    rng = np.random.default_rng(5)
    legs = random_legs(rng, (0,), 5, max_sectors=3, max_dim=9)
    A = W.random_tensor((0,), legs, (0,), 1)
    legsB = [legs[3].conj(), W.Leg(1, [(0,), (1,)], [7, 11]), legs[1].conj()]
    B = W.random_tensor((0,), legsB, (1,), 2)
    _, rec, _ = run_tensordot(ctx, A, B, (3, 1), (0, 2))
    check_against_oracle(rec, oracle_tensordot(A, B, (3, 1), (0, 2)))


def test_large_blocks_transpose_paths(ctx):
    """Blocks big enough for the shared-memory transpose path of the data movers."""
    l0 = W.Leg(1, [(0,), (1,)], [40, 33])
    l1 = W.Leg(1, [(0,), (1,)], [48, 37])
    l2 = W.Leg(-1, [(0,), (1,), (2,)], [35, 41, 20])
    A = W.random_tensor((0,), [l0, l1, l2], (0,), 3)
    B = W.random_tensor((0,), [l0.conj(), W.Leg(1, [(0,), (1,)], [50, 45])], (0,), 4)
    for axa, axb in (((0,), (0,)),):
        _, rec, _ = run_tensordot(ctx, A, B, axa, axb)
        check_against_oracle(rec, oracle_tensordot(A, B, axa, axb))
    C = W.random_tensor((0,), [l2.conj(), l1.conj()], (-1,), 5)
    _, rec, _ = run_tensordot(ctx, A, C, (2, 1), (0, 1))
    check_against_oracle(rec, oracle_tensordot(A, C, (2, 1), (0, 1)))


def test_edge_cases(ctx):
    # outer product (no contracted leg)
    l = W.Leg(1, [(0,), (1,)], [2, 3])
    A = W.random_tensor((0,), [l, l.conj()], (0,), 1)
    _, rec, _ = run_tensordot(ctx, A, A, (), ())
    check_against_oracle(rec, oracle_tensordot(A, A, (), ()))
    # full contraction to rank 0
    B = W.random_tensor((0,), [l.conj(), l], (0,), 2)
    _, rec, _ = run_tensordot(ctx, A, B, (0, 1), (0, 1))
    check_against_oracle(rec, oracle_tensordot(A, B, (0, 1), (0, 1)))
    # no matching charges: empty output
    E = W.random_tensor((0,), [W.Leg(1, [(7,)], [2]), W.Leg(-1, [(7,)], [2])], (0,), 3)
    assert E["t"].shape[0] == 1
    _, rec, _ = run_tensordot(ctx, A, E, (1,), (0,))
    assert rec["t"].shape[0] == 0 and rec["size"] == 0
    # empty input tensor
    Z = W.random_tensor((0,), [l, W.Leg(-1, [(5,)], [1])], (0,), 4)
    assert Z["t"].shape[0] == 0
    _, rec, _ = run_tensordot(ctx, A, Z, (1,), (0,))
    assert rec["t"].shape[0] == 0 and rec["size"] == 0
    # 1x1x1 blocks only
    one = W.Leg(1, [(q,) for q in range(-3, 4)], [1] * 7)
    S = W.random_tensor((0,), [one, one, one.conj()], (0,), 9)
    _, rec, _ = run_tensordot(ctx, S, S, (2,), (0,))
    check_against_oracle(rec, oracle_tensordot(S, S, (2,), (0,)))


def test_partially_populated_needs_zero_fill(ctx):
    """Blocks missing from an allowed set: sector matrices get zero-filled gaps."""
    rng = np.random.default_rng(11)
    legs = random_legs(rng, (0,), 4, max_sectors=3, max_dim=4)
    A = W.random_tensor((0,), legs, (0,), 5)
    keep = np.arange(A["t"].shape[0]) % 3 != 1
    sizes = np.prod(A["D"], axis=1)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    A2 = dict(A)
    A2["t"], A2["D"] = A["t"][keep], A["D"][keep]
    A2["data"] = np.concatenate([A["data"][offs[i]:offs[i + 1]] for i in np.nonzero(keep)[0]])
    B = W.random_tensor((0,), [legs[2].conj(), legs[3].conj()], (0,), 6)
    _, rec, _ = run_tensordot(ctx, A2, B, (2, 3), (0, 1))
    check_against_oracle(rec, oracle_tensordot(A2, B, (2, 3), (0, 1)))


def test_heisenberg_example_closed_form(ctx):
    """The two-spin example of Sec. II: tensordot(H, H) = 3/16 - H/2 on the GPU."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "heisenberg_two_site.json")))
    l = W.Leg(1, [(-1,), (1,)], [1, 1])
    H = W.random_tensor((0,), [l, l, l.conj(), l.conj()], (0,), 0)
    vals = {tuple(tuple(c) for c in k): v for k, v in g["blocks"]}
    H["data"] = np.array([vals[tuple(tuple(int(c) for c in H["t"][b, a]) for a in range(4))]
                          for b in range(H["t"].shape[0])], dtype=np.float64)
    _, rec, _ = run_tensordot(ctx, H, H, (2, 3), (0, 1))
    want = {tuple(tuple(c) for c in k): v for k, v in g["H2_blocks"]}
    got = {tuple(tuple(int(c) for c in rec["t"][b, a]) for a in range(4)): rec["data"][b]
           for b in range(rec["t"].shape[0])}
    assert got.keys() == want.keys()
    for k in want:
        assert abs(got[k] - want[k]) <= 1e-15


# ------------------------------------------------------------------ fuse / unfuse / trace

@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(5))
def test_fuse_unfuse_bit_exact(ctx, sym, case):
    from paper_2405_12196_gb300 import ytn
    mods = SYMS[sym]
    rng = np.random.default_rng(33000 + case)
    rank = int(rng.integers(2, 6))
    legs = random_legs(rng, mods, rank, max_sectors=3, max_dim=6)
    rec = W.random_tensor(mods, legs, tuple([0] * len(mods)), 700 + case)
    if rec["t"].shape[0] == 0:
        return
    perm = [int(a) for a in rng.permutation(rank)]
    cut = int(rng.integers(1, rank))
    groups = (tuple(perm[:cut]), tuple(perm[cut:]))
    F = O.fuse(O.from_record(rec), groups)
    fplan, frec = run_move(ctx, ytn.YTN_OP_FUSE, rec, groups=groups)
    check_against_oracle(frec, O.to_record(F), exact=True)
    fused = [i for i, g in enumerate(groups) if len(g) > 1]
    if not fused:
        return
    uplan, urec = run_move(ctx, ytn.YTN_OP_UNFUSE, frec, axa=fused)
    check_against_oracle(urec, O.to_record(O.unfuse(F, fused)), exact=True)


@pytest.mark.parametrize("case", range(6))
def test_trace(ctx, case):
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(44000 + case)
    mods = [(0,), (2,), (0, 0)][case % 3]
    base = random_legs(rng, mods, 2, max_sectors=3, max_dim=5)
    other = random_legs(rng, mods, int(rng.integers(0, 3)))
    legs = [base[0], base[1], base[0].conj(), base[1].conj()] + other
    npair = int(rng.integers(1, 3))
    ax1, ax2 = (0, 1)[:npair], (2, 3)[:npair]
    rec = W.random_tensor(mods, legs, tuple([0] * len(mods)), 80 + case)
    _, trec = run_move(ctx, ytn.YTN_OP_TRACE, rec, axa=ax1, axb=ax2)
    check_against_oracle(trec, O.to_record(O.trace(O.from_record(rec), ax1, ax2)))


# ------------------------------------------------------------------ workload chains

def test_config2_double_layer_chain(ctx):
    """Z2 double layer: A . A* over the physical leg, fuse ket/bra pairs into D^2 legs,
    then T . a over a D^2 leg; every step against the oracle."""
    from paper_2405_12196_gb300 import ytn
    cfg = W.config2()
    A = cfg["A"]
    Ac = dict(A)
    Ac["sig"] = tuple(-s for s in A["sig"])
    _, AA, _ = run_tensordot(ctx, A, Ac, (4,), (4,))
    oAA = O.tensordot(O.from_record(A), O.conj(O.from_record(A)), (4,), (4,))
    check_against_oracle(AA, O.to_record(oAA))
    groups = ((0, 4), (1, 5), (2, 6), (3, 7))
    _, a = run_move(ctx, ytn.YTN_OP_FUSE, AA, groups=groups)
    oa = O.fuse(oAA, groups)
    check_against_oracle(a, O.to_record(oa), rtol=FP64_RTOL)
    # the edge tensor's D^2 leg is plain, the double layer's is fused: contract against
    # an edge tensor carrying the conjugate fusion record of a's t leg
    T = dict(cfg["T"])
    T["fus"] = [None, dict(a["fus"][0], sig=tuple(-s for s in a["fus"][0]["sig"])), None]
    _, Ta, _ = run_tensordot(ctx, T, a, (1,), (0,))
    oTa = O.tensordot(O.from_record(T), O.from_record(a), (1,), (0,))
    check_against_oracle(Ta, O.to_record(oTa))


def test_config3_environment_contraction(ctx):
    """U(1)xU(1) CTM step, dominant contraction X2 . a over two D^2 legs (7225 + 7225
    blocks, 81 sectors)."""
    cfg = W.config3()
    X2 = cfg["X2"]
    dl = cfg["dleg"]
    a = W.random_tensor((0, 0), [W.Leg(-1, dl.t, dl.D), W.Leg(1, dl.t, dl.D), W.Leg(1, dl.t, dl.D),
                                 W.Leg(-1, dl.t, dl.D)], (0, 0), 3999)
    plan, rec, _ = run_tensordot(ctx, X2, a, (1, 2), (0, 1))
    assert plan.info["nsectors"] == 81
    check_against_oracle(rec, oracle_tensordot(X2, a, (1, 2), (0, 1)))


@pytest.mark.slow
def test_config5_full_size_sampled(ctx):
    """Full-size U(1)xU(1) X2 . a (D=20, chi=400: 103,725 + 103,725 blocks, 225 sectors)
    in the benchmark's configuration; sampled output blocks against the oracle."""
    cfg = W.config5()
    A, B = cfg["A"], cfg["B"]
    plan, rec, res = run_tensordot(ctx, A, B, cfg["axa"], cfg["axb"])
    assert plan.info["nsectors"] == 225
    assert A["t"].shape[0] == 103725 and rec["t"].shape[0] == 103725
    oA, oB = O.from_record(A), O.from_record(B)
    rng = np.random.default_rng(0)
    nb = rec["t"].shape[0]
    sizes = np.prod(rec["D"], axis=1)
    pick = list(rng.choice(nb, 24, replace=False)) + [int(np.argmax(sizes)), 0, nb - 1]
    for b in pick:
        key = tuple(tuple(int(c) for c in rec["t"][b, a]) for a in range(rec["t"].shape[1]))
        want = O.tensordot_block(oA, oB, cfg["axa"], cfg["axb"], key)
        got = rec["data"][rec["off"][b]:rec["off"][b] + sizes[b]].reshape(want.shape)
        assert rel_frobenius(got, want) <= FP64_RTOL
    # charge conservation of every output block (any size)
    t = rec["t"].astype(np.int64)
    tot = np.einsum("bac,a->bc", t, np.array(rec["sig"]))
    assert np.all(tot == 0)
    assert np.all(np.isfinite(rec["data"]))


# ------------------------------------------------------------------ split precision (BF16 slices on tcgen05)

SPLIT_RTOL = 1e-10


def _split(ctx, A, B, axa, axb, rtol=SPLIT_RTOL):
    from paper_2405_12196_gb300 import ytn
    return run_tensordot(ctx, A, B, axa, axb, prec=ytn.YTN_SPLIT_BF16, rtol=rtol)


@pytest.mark.parametrize("sym", list(SYMS))
@pytest.mark.parametrize("case", range(6))
def test_random_tensordot_split(ctx, sym, case):
    mods = SYMS[sym]
    rng = np.random.default_rng(52000 + 13 * case + len(sym))
    rankA, rankB = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    ncon = int(rng.integers(0, min(rankA, rankB) + 1))
    A, B, axa, axb, _, _ = random_pair(rng, mods, rankA, rankB, ncon, max_sectors=4, max_dim=7)
    _, rec, res = _split(ctx, A, B, axa, axb)
    err = check_against_oracle(rec, oracle_tensordot(A, B, axa, axb), rtol=SPLIT_RTOL)
    assert res["slices"] >= 4 and err <= max(res["report"]["err_est"], 1e-15)


@pytest.mark.parametrize("dims", [(1, 1, 1), (128, 128, 32), (129, 127, 33), (300, 260, 500), (40, 700, 129),
                                  (257, 3, 1000), (65, 64, 64), (64, 130, 65), (3, 5, 63), (130, 128, 256),
                                  (128, 129, 257), (64, 64, 512), (5, 7, 255)])
def test_split_tiles_chunks_and_ragged_tails(ctx, dims):
    """Tiles of 128 x 128, K stages of 32 and exact-accumulation chunks of 256, all
    with ragged tails."""
    M, N, K = dims
    l_m, l_k, l_n = W.Leg(1, [(0,)], [M]), W.Leg(1, [(0,)], [K]), W.Leg(1, [(0,)], [N])
    A = W.random_tensor((0,), [l_m, l_k], (0,), M + 3 * K)
    B = W.random_tensor((0,), [l_k.conj(), l_n], (0,), N + 5 * K)
    _, rec, res = _split(ctx, A, B, (1,), (0,))
    want = A["data"].reshape(M, K) @ B["data"].reshape(K, N)
    err = rel_frobenius(rec["data"], want.ravel())
    assert err <= SPLIT_RTOL, err


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("K", [512, 1024, 2048])
def test_split_extreme_digits_fill_the_exact_accumulators(ctx, sign, K):
    """Every element just below a power of two has leading digit +-128, so every
    order-0 digit product is 2^14: over each chunk of 256 of K the order-0
    accumulator reaches exactly +-2^22, the end of the range its drain reads from
    the bit pattern; over several chunks (K = 1024, 2048) the drains add up exactly.
    The result must still be right."""
    x = 2.0 - 2.0 ** -40
    l_m, l_k, l_n = W.Leg(1, [(0,)], [130]), W.Leg(1, [(0,)], [K]), W.Leg(1, [(0,)], [129])
    A = W.random_tensor((0,), [l_m, l_k], (0,), 1)
    B = W.random_tensor((0,), [l_k.conj(), l_n], (0,), 2)
    A["data"] = np.full_like(A["data"], sign * x)
    B["data"] = np.full_like(B["data"], x)
    # rtol 3e-11 asks for six slices, which hold x's 41 significant bits exactly
    _, rec, res = _split(ctx, A, B, (1,), (0,), rtol=3e-11)
    assert res["slices"] == 6
    want = np.full(130 * 129, sign * K * x * x)
    assert rel_frobenius(rec["data"], want) <= 1e-15


def test_split_is_exact_on_small_integers(ctx):
    """Integer operands with few significant bits are represented exactly by the
    slices and every product sum is exact: the split path must reproduce the exact
    result bit for bit."""
    l_m, l_k, l_n = W.Leg(1, [(0,), (1,)], [150, 70]), W.Leg(1, [(0,), (1,)], [400, 333]), W.Leg(1, [(0,), (1,)], [90, 140])
    A = W.random_tensor((0,), [l_m, l_k.conj()], (0,), 1, fill="integer")
    B = W.random_tensor((0,), [l_k, l_n.conj()], (0,), 2, fill="integer")
    _, rec, _ = _split(ctx, A, B, (1,), (0,))
    ref = oracle_tensordot(A, B, (1,), (0,))
    check_against_oracle(rec, ref, exact=True)


def test_split_wide_dynamic_range(ctx):
    """Rows and columns scaled over many orders of magnitude (per-row exponents)."""
    rng = np.random.default_rng(77)
    l_m, l_k, l_n = W.Leg(1, [(0,)], [96]), W.Leg(1, [(0,)], [300]), W.Leg(1, [(0,)], [80])
    A = W.random_tensor((0,), [l_m, l_k], (0,), 3)
    B = W.random_tensor((0,), [l_k.conj(), l_n], (0,), 4)
    A["data"] = (A["data"].reshape(96, 300) * (10.0 ** rng.uniform(-30, 30, size=(96, 1)))).ravel()
    B["data"] = (B["data"].reshape(300, 80) * (10.0 ** rng.uniform(-30, 30, size=(1, 80)))).ravel()
    _, rec, _ = _split(ctx, A, B, (1,), (0,))
    want = A["data"].reshape(96, 300) @ B["data"].reshape(300, 80)
    # error of each element relative to its row and column scale |a_i| |b_j|
    got = rec["data"].reshape(96, 80)
    na = np.linalg.norm(A["data"].reshape(96, 300), axis=1)[:, None]
    nb = np.linalg.norm(B["data"].reshape(300, 80), axis=0)[None, :]
    assert np.max(np.abs(got - want) / (na * nb)) <= 1e-12
    assert rel_frobenius(got / np.abs(want).max(axis=1, keepdims=True), want / np.abs(want).max(axis=1, keepdims=True)) <= SPLIT_RTOL


@pytest.mark.parametrize("axes", [((1,), (0,)), ((0,), (1,))])
def test_split_row_maximum_in_a_late_chunk(ctx, axes):
    """In each row of A_q one K chunk of 256 is scaled by 2^8 (in each column of B_q
    one by 2^6), the chunk depending on the row: the row exponent must be the maximum
    over every chunk, whichever holds it, in both operand orientations (K contiguous,
    or the rows contiguous). An exponent taken from fewer chunks would push digits
    far outside their range. (Whole chunks are scaled, not single elements, so that
    |c_ij| stays within a small factor of the scale 2^(e_i + f_j) that the slice
    arithmetic works at.)"""
    M, K, N = 140, 1000, 70
    axa, axb = axes
    rng = np.random.default_rng(5)
    a_mat = rng.standard_normal((M, K))
    b_mat = rng.standard_normal((K, N))
    for i in range(M):
        c = (i * 7) % 4
        a_mat[i, c * 256:(c + 1) * 256] *= 2.0 ** 8
    for j in range(N):
        c = (j * 5 + 1) % 4
        b_mat[c * 256:(c + 1) * 256, j] *= 2.0 ** 6
    l_m, l_k, l_n = W.Leg(1, [(0,)], [M]), W.Leg(1, [(0,)], [K]), W.Leg(1, [(0,)], [N])
    if axa == (1,):
        A = W.random_tensor((0,), [l_m, l_k], (0,), 1)
        A["data"] = a_mat.ravel().copy()
    else:
        A = W.random_tensor((0,), [l_k, l_m], (0,), 1)
        A["data"] = a_mat.T.ravel().copy()
    if axb == (0,):
        B = W.random_tensor((0,), [l_k.conj(), l_n], (0,), 2)
        B["data"] = b_mat.ravel().copy()
    else:
        B = W.random_tensor((0,), [l_n, l_k.conj()], (0,), 2)
        B["data"] = b_mat.T.ravel().copy()
    _, rec, _ = _split(ctx, A, B, axa, axb)
    err = rel_frobenius(rec["data"], (a_mat @ b_mat).ravel())
    assert err <= SPLIT_RTOL, err


def test_split_slice_count_follows_tolerance(ctx):
    from paper_2405_12196_gb300 import ytn
    cfg = W.config1()
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    counts = {}
    for rtol in (1e-4, 1e-7, 1e-10):
        _, rec, res = _split(ctx, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"], rtol=rtol)
        counts[rtol] = res["slices"]
        err = check_against_oracle(rec, oracle_tensordot(cfg["A"], cfg["B"], cfg["axa"], cfg["axb"]), rtol=rtol)
        assert err <= res["report"]["err_est"]
    assert counts[1e-4] <= counts[1e-7] <= counts[1e-10]
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, 1e-16)
    assert e.value.name == "YTN_E_TOLERANCE"


def test_split_config3(ctx):
    cfg = W.config3()
    dl = cfg["dleg"]
    a = W.random_tensor((0, 0), [W.Leg(-1, dl.t, dl.D), W.Leg(1, dl.t, dl.D), W.Leg(1, dl.t, dl.D),
                                 W.Leg(-1, dl.t, dl.D)], (0, 0), 3999)
    _, rec, res = _split(ctx, cfg["X2"], a, (1, 2), (0, 1))
    check_against_oracle(rec, oracle_tensordot(cfg["X2"], a, (1, 2), (0, 1)), rtol=SPLIT_RTOL)


def test_split_reports_no_device_timeout(ctx):
    from paper_2405_12196_gb300 import ytn
    cfg = W.config1()
    _split(ctx, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    ytn.ytn_sync(ctx, timeout_ms=10000)


@pytest.mark.slow
def test_config5_full_size_split_vs_fp64(ctx):
    """Full-size U(1)xU(1) X2 . a in the benchmark's configuration: the split path
    against the FP64 path on every element, and sampled blocks against the oracle."""
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config5()
    A, B = cfg["A"], cfg["B"]
    _, r64, _ = run_tensordot(ctx, A, B, cfg["axa"], cfg["axb"])
    plan, rsp, res = _split(ctx, A, B, cfg["axa"], cfg["axb"])
    assert res["slices"] >= 3
    err = rel_frobenius(rsp["data"], r64["data"])
    assert err <= SPLIT_RTOL, err
    oA, oB = O.from_record(A), O.from_record(B)
    rng = np.random.default_rng(1)
    sizes = np.prod(rsp["D"], axis=1)
    for b in list(rng.choice(rsp["t"].shape[0], 8, replace=False)) + [int(np.argmax(sizes))]:
        key = tuple(tuple(int(c) for c in rsp["t"][b, x]) for x in range(rsp["t"].shape[1]))
        want = O.tensordot_block(oA, oB, cfg["axa"], cfg["axb"], key)
        got = rsp["data"][rsp["off"][b]:rsp["off"][b] + sizes[b]].reshape(want.shape)
        assert rel_frobenius(got, want) <= SPLIT_RTOL
    del torch


def _u1u1_pair(seed, ncon):
    """A, B on U(1)xU(1) legs over {(0,0), (+-1,0), (0,+-1)} with total charge 0, so
    that many blocks meet (random legs of a product group rarely do)."""
    rng = np.random.default_rng(seed)
    pool = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1)]

    def leg():
        return W.Leg(int(rng.choice([-1, 1])), pool, [int(d) for d in rng.integers(1, 7, len(pool))])
    la = [leg() for _ in range(3)]
    lb = [la[i].conj() for i in range(ncon)] + [leg() for _ in range(3 - ncon)]
    A = W.random_tensor((0, 0), la, (0, 0), seed + 1)
    B = W.random_tensor((0, 0), lb, (0, 0), seed + 2)
    return A, B, tuple(range(ncon)), tuple(range(ncon))


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("case", range(4))
def test_u1u1_tensordot(ctx, case, split):
    A, B, axa, axb = _u1u1_pair(71000 + case, 1 + case % 2)
    if split:
        _, rec, res = _split(ctx, A, B, axa, axb)
    else:
        _, rec, res = run_tensordot(ctx, A, B, axa, axb)
    assert res["useful_flops"] > 0
    check_against_oracle(rec, oracle_tensordot(A, B, axa, axb), rtol=SPLIT_RTOL if split else FP64_RTOL)


@pytest.mark.parametrize("split", [False, True])
def test_interleaved_legs_need_eight_dim_pieces(ctx, split):
    """Contracting every other leg of a rank-8 tensor (dims 2 or 3 per charge, so no
    unit dim disappears): in A's gather no two neighbouring dims merge, so its pieces
    keep eight dims (the copy kernel's instantiation for up to eight dims; the split
    path takes its staged slicing, the fused tables allowing three dims per side)."""
    from paper_2405_12196_gb300 import ytn
    legs = [W.Leg(s, [(0,), (1,)], [2, 3]) for s in (1, -1, 1, -1, 1, -1, 1, -1)]
    A = W.random_tensor((0,), legs, (0,), 81)
    legsB = [legs[1].conj(), legs[3].conj(), legs[5].conj(), legs[7].conj(), W.Leg(1, [(0,)], [3])]
    B = W.random_tensor((0,), legsB, (2,), 82)
    axa, axb = (1, 3, 5, 7), (0, 1, 2, 3)
    prec = ytn.YTN_SPLIT_BF16 if split else ytn.YTN_FP64
    plan, rec, _ = run_tensordot(ctx, A, B, axa, axb, prec=prec, rtol=SPLIT_RTOL if split else 0.0)
    if split:
        assert plan.info["split_fused"] == 0
    check_against_oracle(rec, oracle_tensordot(A, B, axa, axb), rtol=SPLIT_RTOL if split else FP64_RTOL)
