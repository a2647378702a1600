"""Block-diagonal SVD (ytn_svd) and its truncation (ytn_slice) through the C ABI.

Singular vectors are unique only up to sign (and rotations within repeated
values), so the checks are on what is unique: the singular values against the
oracle's, U S V == A, U^T U = 1 and V V^T = 1 per sector, and the truncated
reconstruction error against the Eckart-Young value; the slices are bit-exact.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import device, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


def _svd(ctx, A, rows, cols):
    import torch
    from paper_2405_12196_gb300 import ytn
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_SVD, A, groups=(rows, cols))
    bufs = [torch.full((max(o["size"], 1),), float("nan"), dtype=torch.float64, device=device()) for o in plan.outs]
    ws = torch.empty(ytn.ytn_workspace_size(plan), dtype=torch.uint8, device=device())
    ytn.ytn_svd(plan, to_dev(A["data"]), *bufs, workspace=ws)
    ytn.ytn_sync(ctx)
    recs = []
    for o, b in zip(plan.outs, bufs):
        r = dict(o)
        r["data"] = b[:o["size"]].cpu().numpy()
        recs.append(r)
    return plan, [O.from_record(r) for r in recs]


def _check(A, rows, cols, U, S, V, ref_S):
    oA = O.from_record(A)
    for k, blk in ref_S.blocks.items():
        np.testing.assert_allclose(np.diag(S.blocks[k]), np.diag(blk), rtol=1e-10, atol=1e-12 * np.max(blk))
        assert np.count_nonzero(S.blocks[k] - np.diag(np.diag(S.blocks[k]))) == 0
    R = O.tensordot(O.tensordot(U, S, (len(rows),), (0,)), V, (len(rows),), (0,))
    perm = [0] * A["D"].shape[1]
    for i, a in enumerate(list(rows) + list(cols)):
        perm[a] = i
    R = O.fuse(R, [(p,) for p in perm])
    scale = max(np.max(np.abs(b)) for b in oA.blocks.values())
    for k in oA.blocks:
        np.testing.assert_allclose(R.blocks[k], oA.blocks[k], rtol=0, atol=1e-11 * scale)
    UU = O.tensordot(O.conj(U), U, tuple(range(len(rows))), tuple(range(len(rows))))
    VV = O.tensordot(V, O.conj(V), tuple(range(1, len(cols) + 1)), tuple(range(1, len(cols) + 1)))
    for (c, _), blk in S.blocks.items():
        np.testing.assert_allclose(UU.blocks[(c, c)], np.eye(blk.shape[0]), atol=1e-11)
        np.testing.assert_allclose(VV.blocks[(c, c)], np.eye(blk.shape[0]), atol=1e-11)


@pytest.mark.parametrize("seed", range(4))
def test_svd_random(ctx, seed):
    rng = np.random.default_rng(400 + seed)
    mods = (0,) if seed % 2 == 0 else (0, 0)
    pool = [(0,), (1,), (-1,)] if mods == (0,) else [(0, 0), (1, 0), (0, 1)]
    legs = [W.Leg(s, pool, [int(d) for d in rng.integers(1, 9, 3)]) for s in (1, 1, -1, -1)]
    A = W.random_tensor(mods, legs, (0,) * len(mods), seed)
    rows, cols = ((0, 2), (1, 3)) if seed < 2 else ((0,), (1, 2, 3))
    _, (U, S, V) = _svd(ctx, A, rows, cols)
    _, ref_S, _ = O.svd(O.from_record(A), rows, cols)
    _check(A, rows, cols, U, S, V, ref_S)


def test_svd_truncation_with_slices(ctx):
    """Keep the D largest singular values over all sectors: slices of U, S, V on
    the GPU equal the oracle's slices of the same factors, and the reconstruction
    error is sqrt(sum of the discarded s^2)."""
    import torch
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(17)
    pool = [(0,), (1,), (-1,), (2,)]
    legs = [W.Leg(s, pool, [int(d) for d in rng.integers(2, 7, 4)]) for s in (1, 1, -1, -1)]
    A = W.random_tensor((0,), legs, (0,), 5)
    rows, cols = (0, 1), (2, 3)
    plan, (U, S, V) = _svd(ctx, A, rows, cols)
    allsv = np.sort(np.concatenate([np.diag(b) for b in S.blocks.values()]))[::-1]
    D = allsv.size // 3
    keep = O.truncation(S, D)
    outs = []
    for T, rec, axes in ((U, plan.outs[0], (2,)), (S, plan.outs[1], (0, 1)), (V, plan.outs[2], (0,))):
        full = dict(rec)
        full["data"] = O.to_record(T)["data"]
        ps = ytn.ytn_plan(ctx, ytn.YTN_OP_SLICE, full, axa=axes, keep=keep)
        out = torch.full((max(ps.out["size"], 1),), float("nan"), dtype=torch.float64, device=device())
        ytn.ytn_slice(ps, to_dev(full["data"]), out)
        ytn.ytn_sync(ctx)
        got = dict(ps.out)
        got["data"] = out[:ps.out["size"]].cpu().numpy()
        want = O.to_record(O.slice_leg(T, axes, keep))
        np.testing.assert_array_equal(got["data"], want["data"])
        outs.append(O.from_record(got))
    Ut, St, Vt = outs
    R = O.fuse(O.tensordot(O.tensordot(Ut, St, (2,), (0,)), Vt, (2,), (0,)), ((0,), (1,), (2,), (3,)))
    oA = O.from_record(A)
    err2 = sum(np.sum((R.blocks.get(k, 0) - oA.blocks[k]) ** 2) for k in oA.blocks)
    assert np.sqrt(err2) == pytest.approx(float(np.sqrt(np.sum(allsv[D:] ** 2))), rel=1e-8)


def test_svd_of_the_ctm_enlarged_corner(ctx):
    """The SVD of a CTMRG enlarged corner (Sec. III, Fig. 3(d)): the U(1)xU(1)
    D=12 corner C.T.T.a (from the oracle's ncon) as a matrix (chi D^2) x (chi D^2)."""
    ts, labels = W.ctm_corner_network(W.config3())
    corner = O.to_record(O.ncon([O.from_record(t) for t in ts], labels))
    rows, cols = (0, 2), (1, 3)
    plan, (U, S, V) = _svd(ctx, corner, rows, cols)
    _, ref_S, _ = O.svd(O.from_record(corner), rows, cols)
    _check(corner, rows, cols, U, S, V, ref_S)
    assert max(b.shape[0] for b in S.blocks.values()) > 500


@pytest.mark.parametrize("seed", range(2))
def test_complex_svd(ctx, seed):
    """Complex tensors: complex U and V, real S; the same checks with conjugate
    transposes."""
    import torch
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(450 + seed)
    pool = [(0,), (1,), (-1,)]
    legs = [W.Leg(s, pool, [int(d) for d in rng.integers(1, 9, 3)]) for s in (1, 1, -1, -1)]
    A = W.random_tensor((0,), legs, (0,), seed, dtype="c128")
    rows, cols = ((0, 2), (1, 3)) if seed == 0 else ((0,), (1, 2, 3))
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_SVD, A, groups=(rows, cols))
    dts = [torch.complex128, torch.float64, torch.complex128]
    bufs = [torch.full((max(o["size"], 1),), float("nan"), dtype=dt, device=device()) for o, dt in zip(plan.outs, dts)]
    ws = torch.empty(ytn.ytn_workspace_size(plan), dtype=torch.uint8, device=device())
    ytn.ytn_svd(plan, torch.from_numpy(A["data"]).to(device()), *bufs, workspace=ws)
    ytn.ytn_sync(ctx)
    recs = []
    for o, b in zip(plan.outs, bufs):
        r = dict(o)
        r["data"] = b[:o["size"]].cpu().numpy()
        recs.append(O.from_record(r))
    U, S, V = recs
    _, ref_S, _ = O.svd(O.from_record(A), rows, cols)
    _check(A, rows, cols, U, S, V, ref_S)



@pytest.mark.parametrize("dtype", ["f64", "c128"])
def test_eigh_of_a_hermitian_tensor(ctx, dtype):
    """H = B + B^H on legs (r, r*): eigenvalues against the oracle's, U S U^H == H and
    U^H U = 1 per sector."""
    import torch
    from paper_2405_12196_gb300 import ytn
    rng = np.random.default_rng(610)
    pool = [(0,), (1,), (-1,)]
    r = [W.Leg(s, pool, [int(d) for d in rng.integers(2, 12, 3)]) for s in (1, -1)]
    B = O.from_record(W.random_tensor((0,), r + [l.conj() for l in r], (0,), 5, dtype=dtype))
    Bh = O.fuse(O.conj(B), ((2,), (3,), (0,), (1,)))
    Ho = O.OTensor(B.mods, B.sig, B.n, {k: B.blocks[k] + Bh.blocks[k] for k in B.blocks}, dtype=B.dtype)
    H = O.to_record(Ho)
    plan = ytn.ytn_plan(ctx, ytn.YTN_OP_EIGH, H, groups=((0, 1), (2, 3)))
    dts = [torch.complex128 if dtype == "c128" else torch.float64, torch.float64]
    bufs = [torch.full((max(o["size"], 1),), float("nan"), dtype=dt, device=device()) for o, dt in zip(plan.outs, dts)]
    ws = torch.empty(ytn.ytn_workspace_size(plan), dtype=torch.uint8, device=device())
    ytn.ytn_eigh(plan, torch.from_numpy(H["data"]).to(device()), *bufs, workspace=ws)
    ytn.ytn_sync(ctx)
    U, S = [O.from_record(dict(o, data=b[:o["size"]].cpu().numpy())) for o, b in zip(plan.outs, bufs)]
    _, ref_S = O.eigh(Ho, (0, 1), (2, 3))
    scale = max(np.max(np.abs(b)) for b in Ho.blocks.values())
    for k, blk in ref_S.blocks.items():
        np.testing.assert_allclose(np.diag(S.blocks[k]), np.diag(blk), rtol=1e-10, atol=1e-12 * scale)
    R = O.tensordot(O.tensordot(U, S, (2,), (0,)), O.fuse(O.conj(U), ((2,), (0,), (1,))), (2,), (0,))
    for k in Ho.blocks:
        np.testing.assert_allclose(R.blocks[k], Ho.blocks[k], rtol=0, atol=1e-11 * scale)
    UU = O.tensordot(O.conj(U), U, (0, 1), (0, 1))
    for (c, _), blk in S.blocks.items():
        np.testing.assert_allclose(UU.blocks[(c, c)], np.eye(blk.shape[0]), atol=1e-11)
