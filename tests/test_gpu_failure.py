"""Failure detection without a GPU fault (needs a GPU).

The cost kernels' staging waits are bounded. With the test hook that withholds the staging thread's
mbarrier arrivals (a completion that nothing signals), every wait runs out after about a second; the
kernel latches BSM_ERR_TIMEOUT in the context's status word and returns. The host reads the status,
and the same context then runs a normal call correctly. Covered: the one-column popcount kernel
(cost_variant 0 with the hook) and the tensor-core kernel (cost_variant 3), whose producer then issues
no copies, so its operand builders, MMA issuer and epilogue all give up. The two-column kernel
completes its copies by cp.async groups and has no wait to withhold.
"""
import time

import numpy as np
import pytest

from paper_1402_2020_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2020_gb300 import build

    build.build()
    from paper_1402_2020_gb300 import bsm

    return bsm


@pytest.mark.parametrize("variant,kernel,shape", [(0, 1, (40, 12, 32)), (3, 3, (300, 24, 32))])
def test_bounded_wait_reports_timeout_and_context_recovers(B, orc, variant, kernel, shape):
    pairs = synth.pair_table(256, 31, seed=3000)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=5, dmax=32))
    try:
        w, h, dmax = shape  # one wave of CTAs
        B.bsm_set_tuning(ctx, 0, 0, 0, variant, 0)
        B.bsm_debug_set(ctx, B.BSM_DEBUG_WITHHOLD_ARRIVALS, 1)
        assert B.bsm_cost_plan(ctx, w, h, dmax)["kernel"] == kernel  # the kernel the hook reaches
        B.bsm_debug_set(ctx, B.BSM_DEBUG_WITHHOLD_ARRIVALS, 0)
        l, r, _ = synth.stereo_pair(w, h, dmax, seed=3001)
        dl, dr = torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()
        P = [torch.empty((h, w, 8), dtype=torch.int32, device="cuda") for _ in range(4)]
        dL = torch.full((h, w), -9, dtype=torch.int32, device="cuda")
        dR = torch.full((h, w), -9, dtype=torch.int32, device="cuda")
        B.bsm_describe(ctx, dl, w, h, 3 * w, P[0], P[1])
        B.bsm_describe(ctx, dr, w, h, 3 * w, P[2], P[3])
        B.bsm_debug_set(ctx, B.BSM_DEBUG_WITHHOLD_ARRIVALS, 1)
        t0 = time.time()
        B.bsm_cost_aggregate_wta(ctx, P[0], P[1], P[2], P[3], w, h, dmax, dL, dR)
        assert B.bsm_last_error(ctx) == B.BSM_ERR_TIMEOUT
        assert 0.5 < time.time() - t0 < 30
        assert (dL.cpu().numpy() == -9).all()  # nothing was written past the failed wait
        assert (dR.cpu().numpy() == -9).all()
        # the status is read-and-clear, and the context keeps working
        assert B.bsm_last_error(ctx) == B.BSM_OK
        B.bsm_debug_set(ctx, B.BSM_DEBUG_WITHHOLD_ARRIVALS, 0)
        B.bsm_cost_aggregate_wta(ctx, P[0], P[1], P[2], P[3], w, h, dmax, dL, dR)
        assert B.bsm_last_error(ctx) == B.BSM_OK
        oBL, oPL = orc.describe(l, pairs)
        oBR, _ = orc.describe(r, pairs)
        assert (dL.cpu().numpy() == orc.wta(oBL, oPL, oBR, dmax, 5, 0)).all()
        oBR, oPR = orc.describe(r, pairs)
        assert (dR.cpu().numpy() == orc.wta(oBR, oPR, oBL, dmax, 5, 1)).all()
    finally:
        B.bsm_destroy(ctx)


def test_debug_hook_rejects_unknown_keys(B):
    ctx = B.bsm_create(B.make_params(synth.pair_table(64, 31, seed=3002), dmax=8))
    try:
        with pytest.raises(B.BsmError):
            B.bsm_debug_set(ctx, 99, 1)
        with pytest.raises(B.BsmError):
            B.bsm_debug_set(ctx, B.BSM_DEBUG_WITHHOLD_ARRIVALS, 2)
    finally:
        B.bsm_destroy(ctx)
