"""Random tensors from legs (ytn_plan_blocks, ytn_fill_normal) against the oracle's
Philox4x32-10 / Box-Muller fill: same numbers up to the last bits of the math
functions, and deterministic."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import device

pytestmark = pytest.mark.gpu


def test_normal_fill_matches_the_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_2405_12196_gb300 import ytn
    ctx = ytn.ytn_ctx_create(0)
    l = W.Leg(1, [(-1,), (0,), (1,)], [30, 50, 20])
    plan = ytn.ytn_plan_blocks(ctx, (0,), [l, l, l.conj()], (0,))
    n = plan.out["size"]
    assert n > 10000
    outs = []
    for _ in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device=device())
        ytn.ytn_fill_normal(plan, 2**40 + 7, out)
        ytn.ytn_sync(ctx)
        outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    want = O.normal_fill(2**40 + 7, n)
    np.testing.assert_allclose(outs[0], want, rtol=1e-12, atol=1e-14)
    assert abs(outs[0].mean()) < 5 / np.sqrt(n)
