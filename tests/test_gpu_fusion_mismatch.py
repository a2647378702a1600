"""Contractions over fused legs with different fusion histories (Sec. II.B
footnote), through the C ABI, against the oracle's resolved contraction.

The planner contracts over the constituents of unfused views of both operands
(strided sub-blocks of the fused blocks); missing constituent charges count as
zero. FP64 within 1e-12, split within 1e-10.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import FP64_RTOL, check_against_oracle, run_tensordot
from helpers import fusion_mismatch_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    return ytn.ytn_ctx_create(0)


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("drops", [(1, None), (None, -1), (1, -1), (0, 1)])
def test_small_mismatched_histories(ctx, drops, split):
    from paper_2405_12196_gb300 import ytn
    A, B, _, _, _, _ = fusion_mismatch_pair(*drops)
    ra, rb = O.to_record(A), O.to_record(B)
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    _, rec, _ = run_tensordot(ctx, ra, rb, (0,), (0,), prec=prec, rtol=rtol)
    check_against_oracle(rec, O.to_record(O.tensordot(A, B, (0,), (0,))), rtol=1e-10 if split else FP64_RTOL)


@pytest.fixture(scope="module")
def ctm_case():
    """U(1)xU(1) CTM step: X2 carries the fusion records of the full double layer a;
    a' is built from a site tensor without the blocks of one virtual charge on its
    top and left legs, so a's fused legs miss those constituent charges."""
    cfg = W.config3()
    oA = O.from_record(cfg["A"])
    groups = ((0, 4), (1, 5), (2, 6), (3, 7))
    a_full = O.fuse(O.tensordot(oA, O.conj(oA), (4,), (4,)), groups)
    thin = O.OTensor(oA.mods, oA.sig, oA.n,
                     {k: v for k, v in oA.blocks.items() if k[0] != (1, 1) and k[1] != (-1, 0)})
    a_thin = O.fuse(O.tensordot(thin, O.conj(thin), (4,), (4,)), groups)
    assert a_thin.fus[0].key() != a_full.fus[0].key()
    X2 = O.from_record(dict(cfg["X2"]))
    X2.fus = [None, a_full.fus[0].conj(), a_full.fus[1].conj(), None]
    want = O.to_record(O.tensordot(X2, a_thin, (1, 2), (0, 1)))
    return X2, a_thin, want


@pytest.mark.parametrize("split", [False, True])
def test_ctm_environment_with_a_thinner_double_layer(ctx, ctm_case, split):
    """X2.a' over two fused legs with different histories is resolved and matches the
    oracle."""
    from paper_2405_12196_gb300 import ytn
    X2, a_thin, want = ctm_case
    prec, rtol = (ytn.YTN_SPLIT_BF16, 1e-10) if split else (ytn.YTN_FP64, 0.0)
    _, rec, _ = run_tensordot(ctx, O.to_record(X2), O.to_record(a_thin), (1, 2), (0, 1), prec=prec, rtol=rtol)
    check_against_oracle(rec, want, rtol=1e-10 if split else FP64_RTOL)
    assert np.any(rec["data"] != 0)
