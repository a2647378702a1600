"""The device failure path, without faulting or hanging the GPU.

A kernel waits (bounded) for a flag that nothing sets; it must record its code in
the context's status word, ytn_sync must report YTN_E_TIMEOUT once and clear it,
and the context must still run contractions correctly afterwards.
"""
import pytest

import workloads as W
from gpu_helpers import FP64_RTOL, check_against_oracle, run_tensordot

import oracle as O

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    ctx = ytn.ytn_ctx_create(0)
    ytn.ytn_sync(ctx)
    ytn.ytn_selftest_timeout(ctx)
    with pytest.raises(ytn.YtnError) as ei:
        ytn.ytn_sync(ctx, timeout_ms=10000)
    assert ei.value.name == "YTN_E_TIMEOUT"
    ytn.ytn_sync(ctx, timeout_ms=10000)           # the word was cleared
    cfg = W.config1()
    for prec in (ytn.YTN_FP64, ytn.YTN_SPLIT_BF16):
        _, rec, _ = run_tensordot(ctx, cfg["A"], cfg["B"], cfg["axa"], cfg["axb"], prec=prec,
                                  rtol=1e-10 if prec else 0.0)
        want = O.to_record(O.tensordot(O.from_record(cfg["A"]), O.from_record(cfg["B"]), cfg["axa"], cfg["axb"]))
        check_against_oracle(rec, want, rtol=FP64_RTOL if prec == ytn.YTN_FP64 else 1e-10)
    ytn.ytn_sync(ctx, timeout_ms=10000)


def test_selftest_needs_a_device_context():
    from paper_2405_12196_gb300 import ytn
    with pytest.raises(ytn.YtnError):
        ytn.ytn_selftest_timeout(ytn.ytn_ctx_create(-1))
