"""Accuracy of the split-precision path on data that defeats a data-blind bound,
through the C ABI.

The split products are off, per element, by a small multiple of the product of the
row and column scales 2^(e_i + f_j). When most of a row lies far below its largest
element, or when the products cancel, the result is small against those scales and
the relative error grows with the ratio. The call estimates that error per charge
sector from its own exponents and result, recomputes the sectors above rtol on the
FP64 path, and reports the estimate (ytn_tensordot_report); when even the FP64
products cannot reach rtol, ytn_sync returns YTN_E_TOLERANCE. Every case here
compares with the oracle (or an FP64 reference computed independently) element by
element through the relative Frobenius error.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import rel_frobenius

pytestmark = pytest.mark.gpu

SPLIT_RTOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _dense_pair(a_mat, b_mat, a_kmajor=True, b_kmajor=False):
    """Records of one dense U(1) sector: A (M x K) and B (K x N) with the contracted
    leg first or last (both operand orientations of the sector matrices)."""
    M, K = a_mat.shape
    N = b_mat.shape[1]
    l_m, l_k, l_n = W.Leg(1, [(0,)], [M]), W.Leg(1, [(0,)], [K]), W.Leg(1, [(0,)], [N])
    if a_kmajor:
        A = W.random_tensor((0,), [l_m, l_k], (0,), 1)
        A["data"] = a_mat.ravel().copy()
        axa = (1,)
    else:
        A = W.random_tensor((0,), [l_k, l_m], (0,), 1)
        A["data"] = a_mat.T.ravel().copy()
        axa = (0,)
    if not b_kmajor:
        B = W.random_tensor((0,), [l_k.conj(), l_n], (0,), 2)
        B["data"] = b_mat.ravel().copy()
        axb = (0,)
    else:
        B = W.random_tensor((0,), [l_n, l_k.conj()], (0,), 2)
        B["data"] = b_mat.T.ravel().copy()
        axb = (1,)
    return A, B, axa, axb


def _split_run(ctx, A, B, axa, axb, rtol=SPLIT_RTOL):
    """One split-precision call; returns (C data, ytn_result, report, ytn_sync status)."""
    import torch
    from paper_2405_12196_gb300 import ytn
    dev = torch.device("cuda:0")
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    da = torch.from_numpy(np.ascontiguousarray(A["data"])).to(dev)
    db = torch.from_numpy(np.ascontiguousarray(B["data"])).to(dev)
    n = plan.out["size"]
    dc = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device=dev)
    ws = torch.empty(max(ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, rtol), 1), dtype=torch.uint8, device=dev)
    res = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_SPLIT_BF16, rtol=rtol, workspace=ws)
    rep = ytn.ytn_tensordot_report(plan, ws)
    try:
        ytn.ytn_sync(ctx)
        status = "YTN_OK"
    except ytn.YtnError as e:
        status = e.name
    return dc[:n].cpu().numpy(), res, rep, status


def _dominant(rng, M, K, N, ratio):
    """One element per row of A and per column of B (random positions) at magnitude
    1..2, every other element N(0, 1) times 2^-ratio."""
    a = rng.standard_normal((M, K)) * 2.0 ** -ratio
    b = rng.standard_normal((K, N)) * 2.0 ** -ratio
    a[np.arange(M), rng.integers(0, K, M)] = rng.choice([-1.0, 1.0], M) * rng.uniform(1, 2, M)
    b[rng.integers(0, K, N), np.arange(N)] = rng.choice([-1.0, 1.0], N) * rng.uniform(1, 2, N)
    return a, b


@pytest.mark.parametrize("orient", [(True, False), (False, True)])
def test_one_dominant_element_per_row_and_column(ctx, orient):
    """One large element per row of A_q and per column of B_q, the rest 2^8 below it,
    K = 1000: element-wise, not whole chunks. The result must meet rtol against the
    oracle and the reported estimate must bound the measured error."""
    rng = np.random.default_rng(2024)
    a, b = _dominant(rng, 140, 1000, 70, 8)
    A, B, axa, axb = _dense_pair(a, b, *orient)
    got, res, rep, status = _split_run(ctx, A, B, axa, axb)
    want = O.to_record(O.tensordot(O.from_record(A), O.from_record(B), axa, axb))["data"]
    err = rel_frobenius(got, want)
    assert status == "YTN_OK"
    assert rep["within"] == 1
    assert err <= SPLIT_RTOL, err
    assert err <= rep["err_est"], (err, rep)
    assert rep["err_est"] <= SPLIT_RTOL


@pytest.mark.parametrize("ratio", [0, 4, 8, 12, 16, 20])
def test_dominance_ratio_sweep(ctx, ratio):
    """The same shape over ratios 2^0 .. 2^20: always within rtol, the estimate
    bounds the error, and at large ratios the sector is recomputed in FP64."""
    rng = np.random.default_rng(300 + ratio)
    a, b = _dominant(rng, 130, 1000, 129, ratio)
    A, B, axa, axb = _dense_pair(a, b)
    got, res, rep, status = _split_run(ctx, A, B, axa, axb)
    err = rel_frobenius(got.reshape(130, 129), a @ b)
    assert status == "YTN_OK"
    assert err <= SPLIT_RTOL, (ratio, err, rep)
    assert err <= rep["err_est"], (ratio, err, rep)
    if rep["nfallback"] == 0:
        assert err <= rep["split_err_est"]
    if ratio >= 16:
        assert rep["nfallback"] == 1 and rep["split_err_est"] > SPLIT_RTOL


@pytest.mark.parametrize("dist", ["normal", "uniform", "near_powers_of_two", "log_range"])
def test_estimate_bounds_the_error_without_fallback(ctx, dist):
    """Ordinary data: no sector is recomputed, and the estimate bounds the split
    error without being far above it."""
    rng = np.random.default_rng({"normal": 1, "uniform": 2, "near_powers_of_two": 3, "log_range": 4}[dist])
    M, K, N = 200, 3000, 150

    def draw(shape):
        if dist == "normal":
            return rng.standard_normal(shape)
        if dist == "uniform":
            return rng.uniform(-1, 1, shape)
        if dist == "near_powers_of_two":
            return rng.choice([-1.0, 1.0], shape) * rng.uniform(0.95, 0.999, shape)
        return rng.choice([-1.0, 1.0], shape) * 2.0 ** rng.uniform(-30, 0, shape)
    a, b = draw((M, K)), draw((K, N))
    A, B, axa, axb = _dense_pair(a, b)
    got, res, rep, status = _split_run(ctx, A, B, axa, axb)
    err = rel_frobenius(got.reshape(M, N), a @ b)
    assert status == "YTN_OK"
    assert rep["nfallback"] == 0
    assert err <= rep["split_err_est"] <= SPLIT_RTOL, (err, rep)
    assert rep["split_err_est"] <= 1000 * max(err, 1e-15), (err, rep)


def test_only_the_cancelling_sector_is_recomputed(ctx):
    """Two sectors (charges 0 and 1 of a U(1) leg): sector 0 ordinary, sector 1 with
    one dominant element per row and column at 2^20. Only sector 1 goes to FP64; the
    whole result matches the oracle within rtol."""
    rng = np.random.default_rng(7)
    M, K, N = 90, 700, 80
    a1, b1 = _dominant(rng, M, K, N, 20)
    l_m = W.Leg(1, [(0,), (1,)], [M, M])
    l_k = W.Leg(1, [(0,), (1,)], [K, K])
    l_n = W.Leg(1, [(0,), (1,)], [N, N])
    A = W.random_tensor((0,), [l_m, l_k.conj()], (0,), 11)
    B = W.random_tensor((0,), [l_k, l_n.conj()], (0,), 12)
    # blocks in canonical order: charge 0 then charge 1 (M x K, then K x N)
    A["data"][M * K:] = a1.ravel()
    B["data"][K * N:] = b1.ravel()
    got, res, rep, status = _split_run(ctx, A, B, (1,), (0,))
    want = O.to_record(O.tensordot(O.from_record(A), O.from_record(B), (1,), (0,)))["data"]
    assert status == "YTN_OK"
    assert rep["nsectors"] == 2 and rep["nfallback"] == 1
    assert rep["fallback_flops"] == 2.0 * M * N * K
    err = rel_frobenius(got, want)
    assert err <= SPLIT_RTOL and err <= rep["err_est"], (err, rep)


def test_cancellation_beyond_fp64_is_reported(ctx):
    """B's columns almost orthogonal to A's rows, so that C is about 2^-45 of the
    scales: no FP64 product reaches 1e-10 relative to such a result either. The call
    must say so: the record is not within rtol, and ytn_sync returns YTN_E_TOLERANCE
    once (the status word is then clear)."""
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(8)
    M, K, N = 64, 512, 64
    a = rng.standard_normal((M, K))
    x = rng.standard_normal((K, N))
    q, _ = np.linalg.qr(a.T)
    b = x - q @ (q.T @ x) + 2.0 ** -45 * x
    A, B, axa, axb = _dense_pair(a, b)
    got, res, rep, status = _split_run(ctx, A, B, axa, axb)
    assert rep["nfallback"] == 1
    assert rep["within"] == 0 and rep["err_est"] > SPLIT_RTOL
    assert status == "YTN_E_TOLERANCE"
    ytn.ytn_sync(ctx)   # cleared


def test_report_needs_a_completed_split_call(ctx):
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config1()
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"])
    ws = torch.zeros(ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, SPLIT_RTOL), dtype=torch.uint8,
                     device=torch.device("cuda:0"))
    with pytest.raises(ytn.YtnError) as e:
        ytn.ytn_tensordot_report(plan, ws)
    assert e.value.name == "YTN_E_INVALID"


def test_staged_split_path_for_blocks_with_many_dims(ctx):
    """Blocks with four free dims that cannot merge (legs free, contracted, free, ...
    interleaved) are beyond the fused split (three per side): the staged path (FP64
    sector matrices first) runs, and must meet the tolerance against the oracle."""
    from gpu_helpers import check_against_oracle, oracle_tensordot
    l = W.Leg(1, [(0,), (1,)], [2, 2])
    A = W.random_tensor((0,), [l] * 7, (2,), 21)
    B = W.random_tensor((0,), [l.conj()] * 3 + [l] * 2, (-1,), 22)
    axa, axb = (1, 3, 5), (0, 1, 2)
    got, res, rep, status = _split_run(ctx, A, B, axa, axb)
    from paper_2405_12196_gb300 import ytn
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    assert plan.info["split_fused"] == 0
    rec = dict(plan.out)
    rec["data"] = got
    check_against_oracle(rec, oracle_tensordot(A, B, axa, axb), rtol=SPLIT_RTOL)
    assert status == "YTN_OK" and rep["within"] == 1


def test_fused_split_path_on_the_environment_contraction(ctx):
    """The CTM environment contraction X2 . a (U(1)xU(1), D = 12) takes the fused
    path, and meets the tolerance against the oracle."""
    from gpu_helpers import check_against_oracle, oracle_tensordot
    from paper_2405_12196_gb300 import ytn
    cfg = W.config3()
    dl = cfg["dleg"]
    a = W.random_tensor((0, 0), [W.Leg(-1, dl.t, dl.D), W.Leg(1, dl.t, dl.D), W.Leg(1, dl.t, dl.D),
                                 W.Leg(-1, dl.t, dl.D)], (0, 0), 3999)
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, cfg["X2"], a, (1, 2), (0, 1))
    assert plan.info["split_fused"] == 1
    got, res, rep, status = _split_run(ctx, cfg["X2"], a, (1, 2), (0, 1))
    rec = dict(plan.out)
    rec["data"] = got
    check_against_oracle(rec, oracle_tensordot(cfg["X2"], a, (1, 2), (0, 1)), rtol=SPLIT_RTOL)
    assert status == "YTN_OK" and rep["nfallback"] == 0


def _interleaved_pair(pattern, seed):
    """U(1) tensors whose contracted legs ('k') and free legs ('f') alternate as in
    `pattern`, in both operands: no two neighbouring legs of a side merge, so each
    side keeps two or three dims per block."""
    lk = W.Leg(1, [(-1,), (0,), (1,)], [2, 3, 2])
    lf = W.Leg(1, [(-1,), (0,), (1,)], [3, 2, 3])
    A = W.random_tensor((0,), [lk if ch == "k" else lf for ch in pattern], (0,), seed)
    B = W.random_tensor((0,), [lk.conj() if ch == "k" else W.Leg(-1, lf.t, [2, 2, 2]) for ch in pattern],
                        (0,), seed + 1)
    ax = tuple(i for i, ch in enumerate(pattern) if ch == "k")
    return A, B, ax, ax


@pytest.mark.parametrize("pattern", ["kfkf", "kfkfkf", "fkfk", "fkfkfk"])
def test_fused_split_walks_unmerged_dims(pattern):
    """The fused slicing walks a block side of two or three dims with its stepped
    index: K when the block's rows are its contiguous direction (free leg last),
    else the rows (contracted leg last). The first split call on a plan leaves the
    fused candidate's result in C; it must meet the tolerance against the oracle,
    and a later call (the autotuner's choice) must give the same bits."""
    import torch
    from gpu_helpers import check_against_oracle, oracle_tensordot
    from paper_2405_12196_gb300 import ytn
    A, B, axa, axb = _interleaved_pair(pattern, 31 + len(pattern))
    fresh = ytn.ytn_ctx_create(0)   # the first call on this structure must be the timing one
    plan = ytn.ytn_plan(fresh, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    assert plan.info["split_fused"] == 1
    dev = torch.device("cuda:0")
    da, db = torch.from_numpy(A["data"]).to(dev), torch.from_numpy(B["data"]).to(dev)
    ws = torch.empty(ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, SPLIT_RTOL), dtype=torch.uint8, device=dev)
    ref = oracle_tensordot(A, B, axa, axb)
    outs = []
    for call in range(2):
        dc = torch.full((plan.out["size"],), float("nan"), dtype=torch.float64, device=dev)
        res = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_SPLIT_BF16, rtol=SPLIT_RTOL, workspace=ws)
        ytn.ytn_sync(fresh)
        if call == 0:
            assert res["split_variant"] == 1
        rec = dict(plan.out)
        rec["data"] = dc.cpu().numpy()
        check_against_oracle(rec, ref, rtol=SPLIT_RTOL)
        outs.append(rec["data"])
    np.testing.assert_array_equal(outs[0], outs[1])


def _many_sector_pair(nsec=10, m=1024, k=256, n=1024, seed=77):
    """U(1) matrices with `nsec` charge sectors of m x k times k x n each."""
    q = [(c,) for c in range(nsec)]
    A = W.random_tensor((0,), [W.Leg(1, q, [m] * nsec), W.Leg(-1, q, [k] * nsec)], (0,), seed)
    B = W.random_tensor((0,), [W.Leg(1, q, [k] * nsec), W.Leg(-1, q, [n] * nsec)], (0,), seed + 1)
    return A, B, (1,), (0,)


def test_pipelined_fused_split():
    """Ten sectors of 1024 x 256 x 1024 (640 tiles of 128 x 128) make two pipeline
    groups. The first split call times the staged, fused and pipelined variants in
    that order and leaves the pipelined run's result in C (no sector has a 64-wide
    tail to try): it must meet the tolerance against the oracle, and a later call
    (the autotuner's choice, whichever it is) must give the same bits."""
    import torch
    from gpu_helpers import check_against_oracle, oracle_tensordot
    from paper_2405_12196_gb300 import ytn
    A, B, axa, axb = _many_sector_pair()
    fresh = ytn.ytn_ctx_create(0)
    plan = ytn.ytn_plan(fresh, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    assert plan.info["split_fused"] == 1 and plan.info["split_pipe_groups"] == 2
    dev = torch.device("cuda:0")
    da, db = torch.from_numpy(A["data"]).to(dev), torch.from_numpy(B["data"]).to(dev)
    ws = torch.empty(ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, SPLIT_RTOL), dtype=torch.uint8, device=dev)
    ref = oracle_tensordot(A, B, axa, axb)
    outs, variants = [], []
    for call in range(2):
        dc = torch.full((plan.out["size"],), float("nan"), dtype=torch.float64, device=dev)
        res = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_SPLIT_BF16, rtol=SPLIT_RTOL, workspace=ws)
        ytn.ytn_sync(fresh)
        variants.append(res["split_variant"])
        rec = dict(plan.out)
        rec["data"] = dc.cpu().numpy()
        check_against_oracle(rec, ref, rtol=SPLIT_RTOL)
        outs.append(rec["data"])
    assert variants[0] == 2
    t = ytn.ytn_plan_tuning(plan, res["slices"])
    assert t["pipelined_ms"] > 0 and t["fused_ms"] > 0 and t["staged_ms"] > 0
    assert t["split_variant"] == variants[1]
    assert (t["split_variant"] == 2) == (t["pipelined_ms"] < min(t["fused_ms"], t["staged_ms"]))
    np.testing.assert_array_equal(outs[0], outs[1])


def test_split_variants_give_identical_bits(ctx):
    """A plan with fused tables: the first split call times the staged and the fused
    variant (leaving the fused result) and caches the faster; later calls use the
    cached one. Both variants build the same slices, so every call gives the same
    bits."""
    import torch
    from paper_2405_12196_gb300 import ytn
    cfg = W.config3()
    dl = cfg["dleg"]
    a = W.random_tensor((0, 0), [W.Leg(-1, dl.t, dl.D), W.Leg(1, dl.t, dl.D), W.Leg(1, dl.t, dl.D),
                                 W.Leg(-1, dl.t, dl.D)], (0, 0), 4001)
    # a context of its own: plans are cached per context by structure, and this one's
    # first call must be the one that times the variants
    fresh = ytn.ytn_ctx_create(0)
    plan = ytn.ytn_plan(fresh, ytn.YTN_OP_TENSORDOT, cfg["X2"], a, (1, 2), (0, 1))
    assert plan.info["split_fused"] == 1
    dev = torch.device("cuda:0")
    da, db = torch.from_numpy(cfg["X2"]["data"]).to(dev), torch.from_numpy(a["data"]).to(dev)
    ws = torch.empty(ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, SPLIT_RTOL), dtype=torch.uint8, device=dev)
    outs, variants = [], []
    for _ in range(3):
        dc = torch.full((plan.out["size"],), float("nan"), dtype=torch.float64, device=dev)
        res = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_SPLIT_BF16, rtol=SPLIT_RTOL, workspace=ws)
        ytn.ytn_sync(fresh)
        outs.append(dc.cpu().numpy())
        variants.append(res["split_variant"])
    assert variants[0] == 1 and variants[1] == variants[2] and variants[1] in (0, 1)
    # the cached choice is the faster of the two timed runs
    t = ytn.ytn_plan_tuning(plan, res["slices"])
    assert t["split_variant"] == variants[1] and t["staged_ms"] > 0 and t["fused_ms"] > 0
    assert (t["fused_ms"] < t["staged_ms"]) == (variants[1] == 1)
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[1], outs[2])


@pytest.mark.parametrize("dims", [(200, 300, 60), (130, 1000, 190), (64, 96, 1), (257, 513, 129)])
def test_narrow_sector_tails(ctx, dims):
    """Sectors whose N ends in the first half of a 128-wide tile get a 128 x 64 last
    column tile in the second tile list. The first split call runs every candidate
    and leaves the last one's result, the one with the narrow tails, in C: it must
    meet the tolerance against the oracle; later calls (the cached choice) too."""
    import torch
    from gpu_helpers import check_against_oracle, oracle_tensordot
    from paper_2405_12196_gb300 import ytn
    M, K, N = dims
    rng = np.random.default_rng(M + K + N)
    A, B, axa, axb = _dense_pair(rng.standard_normal((M, K)), rng.standard_normal((K, N)))
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_TENSORDOT, A, B, axa, axb)
    ref = oracle_tensordot(A, B, axa, axb)
    dev = torch.device("cuda:0")
    da, db = torch.from_numpy(A["data"]).to(dev), torch.from_numpy(B["data"]).to(dev)
    ws = torch.empty(ytn.ytn_workspace_size(plan, ytn.YTN_SPLIT_BF16, SPLIT_RTOL), dtype=torch.uint8, device=dev)
    for call in range(2):
        dc = torch.full((plan.out["size"],), float("nan"), dtype=torch.float64, device=dev)
        res = ytn.ytn_tensordot(plan, da, db, dc, prec=ytn.YTN_SPLIT_BF16, rtol=SPLIT_RTOL, workspace=ws)
        ytn.ytn_sync(ctx)
        rec = dict(plan.out)
        rec["data"] = dc.cpu().numpy()
        check_against_oracle(rec, ref, rtol=SPLIT_RTOL)
        if call == 0:
            assert res["narrow_tiles"] == (1 if 0 < N % 128 <= 64 else 0)
