"""Long descriptors (n = 512 ... 4096 bits, the paper's n = 4096 of Sec. 4.1) vs the oracle, bit-exact.

These run the long-descriptor kernels (warp-per-pixel describe, chunked cost) through the same C ABI
calls as the short descriptors; the oracle is the same code for every n.
"""
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


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def _describe(B, ctx, img, nw, pad=0, noalloc=False):
    h, w, _ = img.shape
    pitch = 3 * w + pad
    buf = np.zeros((h, pitch), np.uint8)
    buf[:, : 3 * w] = img.reshape(h, 3 * w)
    d = torch.from_numpy(buf).cuda()
    Bp = torch.full((h, w, nw), -1, dtype=torch.int32, device="cuda")
    Pp = torch.full((h, w, nw), -1, dtype=torch.int32, device="cuda")
    (B.bsm_describe_noalloc if noalloc else B.bsm_describe)(ctx, d, w, h, pitch, Bp, Pp)
    return Bp, Pp, d, pitch


@pytest.mark.parametrize("w,h,n,S,sigma,k,pad", [
    (37, 23, 512, 31, None, 0, 5),      # ragged tiles, pitch > 3w
    (40, 9, 1024, 31, None, 300, 0),
    (70, 13, 2048, 31, None, 2048, 0),  # k = n: every pair kept
    (45, 17, 4096, 26, 4.0, 0, 1),      # the paper's n = 4096, S = 26, sigma = 4
    (1, 1, 4096, 26, 4.0, 1, 0),        # one pixel, k = 1
])
def test_long_describe_bit_exact(B, orc, w, h, n, S, sigma, k, pad):
    l, _, _ = synth.stereo_pair(w, h, 16, seed=500 + w)
    pairs = synth.pair_table(n, S, sigma=sigma, seed=n + w)
    p = B.make_params(pairs, window_S=S + (S % 2 == 0), mask_rank=k, dmax=16, agg_window=1)
    ctx = B.bsm_create(p)
    Bp, Pp, _, _ = _describe(B, ctx, l, n // 32, pad)
    torch.cuda.synchronize()
    oB, oP = orc.describe(l, pairs, k if k else None)
    assert (u32(Bp) == oB).all()
    assert (u32(Pp) == oP).all()
    # the mask really keeps k pairs (Eq. 6/7): at least k ones, as in the oracle
    assert (np.unpackbits(oP.view(np.uint8), axis=-1).reshape(h, w, -1).sum(-1) >= (k if k else n // 4)).all()
    B.bsm_destroy(ctx)


@pytest.mark.parametrize("n,win,dmax,w,h", [
    (512, 5, 24, 61, 29),
    (1024, 7, 40, 50, 21),
    (2048, 3, 137, 70, 15),   # dmax not a multiple of 8, most matches outside the image
    (4096, 3, 64, 61, 29),
    (4096, 1, 256, 40, 9),    # the largest dmax on a narrow image, no aggregation
])
def test_long_cost_volume_bit_exact(B, orc, n, win, dmax, w, h):
    l, r, _ = synth.stereo_pair(w, h, min(dmax, w), seed=600 + n)
    pairs = synth.pair_table(n, 26, sigma=4.0, seed=601)
    p = B.make_params(pairs, window_S=27, agg_window=win, dmax=dmax)
    ctx = B.bsm_create(p)
    nw = n // 32
    BL, PL, _, _ = _describe(B, ctx, l, nw)
    BR, PR, _, _ = _describe(B, ctx, r, nw)
    dL = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
    dR = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
    cost = torch.zeros((h, w, dmax), dtype=torch.int16, device="cuda")
    B.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, cost)
    torch.cuda.synchronize()
    oBL, oPL = orc.describe(l, pairs)
    oBR, oPR = orc.describe(r, pairs)
    assert (u32(BL) == oBL).all() and (u32(PR) == oPR).all()
    A = orc.aggregate(oBL, oPL, oBR, dmax, win, 0)
    assert (cost.cpu().numpy().view(np.uint16).astype(np.uint32) == A).all()
    assert (dL.cpu().numpy() == np.argmin(A, axis=2)).all()
    AR = orc.aggregate(oBR, oPR, oBL, dmax, win, 1)
    assert (dR.cpu().numpy() == np.argmin(AR, axis=2)).all()
    B.bsm_destroy(ctx)


@pytest.mark.parametrize("rows", [8, 16, 512])
def test_long_row_band_does_not_change_bits(B, orc, rows):
    w, h, dmax, n = 53, 37, 48, 1024
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=650)
    pairs = synth.pair_table(n, 31, seed=651)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=5, dmax=dmax))
    B.bsm_set_tuning(ctx, rows, 0, 0, 1)
    BL, PL, _, _ = _describe(B, ctx, l, n // 32)
    BR, PR, _, _ = _describe(B, ctx, r, n // 32)
    dL = torch.empty((h, w), dtype=torch.int32, device="cuda")
    dR = torch.empty_like(dL)
    B.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR)
    torch.cuda.synchronize()
    oBL, oPL = orc.describe(l, pairs)
    oBR, oPR = orc.describe(r, pairs)
    assert (dL.cpu().numpy() == orc.wta(oBL, oPL, oBR, dmax, 5, 0)).all()
    assert (dR.cpu().numpy() == orc.wta(oBR, oPR, oBL, dmax, 5, 1)).all()
    B.bsm_destroy(ctx)


def test_long_full_chain_paper_setting(B, orc):
    # the paper's descriptor (n = 4096, S = 26, sigma = 4, k = n/4) with a 3x3 box, through refinement
    w, h, dmax = 120, 70, 40
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=700)
    pairs = synth.pair_table(4096, 26, sigma=4.0, seed=701)
    ctx = B.bsm_create(B.make_params(pairs, window_S=27, agg_window=3, dmax=dmax, vote_radius=6))
    BL, PL, dl, pitch = _describe(B, ctx, l, 128)
    BR, PR, _, _ = _describe(B, ctx, r, 128)
    dL = torch.empty((h, w), dtype=torch.int32, device="cuda")
    dR = torch.empty_like(dL)
    B.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR)
    out = torch.empty_like(dL)
    B.bsm_refine(ctx, dl, pitch, dL, dR, w, h, dmax, out)
    torch.cuda.synchronize()
    ref = orc.pipeline(l, r, pairs, dmax, win=3, R=6)
    assert (dL.cpu().numpy() == ref["dL"]).all()
    assert (dR.cpu().numpy() == ref["dR"]).all()
    assert (out.cpu().numpy() == ref["disp"]).all()
    # the host entry point runs the same kernels
    host = np.zeros((h, w), np.int32)
    B.bsm_match_host(ctx, l, r, w, h, 3 * w, dmax, host)
    assert (host == ref["disp"]).all()
    B.bsm_destroy(ctx)


def test_long_noalloc_describe_equals_describe(B):
    w, h, n = 64, 20, 2048
    l, _, _ = synth.stereo_pair(w, h, 16, seed=710)
    ctx = B.bsm_create(B.make_params(synth.pair_table(n, 31, seed=711), dmax=16, agg_window=3))
    B0, P0, _, _ = _describe(B, ctx, l, n // 32)
    B1, P1, _, _ = _describe(B, ctx, l, n // 32, noalloc=True)
    torch.cuda.synchronize()
    assert torch.equal(B0, B1) and torch.equal(P0, P1)
    B.bsm_destroy(ctx)


def test_long_descriptors_refused_where_not_built(B):
    w, h, dmax, n = 32, 8, 16, 512
    ctx = B.bsm_create(B.make_params(synth.pair_table(n, 31, seed=720), dmax=dmax))
    with pytest.raises(B.BsmError) as e:
        B.bsm_set_tuning(ctx, 0, 0, 0, 2)  # the two-column cost kernel is for n = 128 and 256
    assert e.value.status == B.BSM_ERR_UNSUPPORTED
    t = lambda *s: torch.zeros(s, dtype=torch.int32, device="cuda")
    img = torch.zeros((h, 3 * w), dtype=torch.uint8, device="cuda")
    d = B.pair_desc(img, img, w, h, 3 * w, dmax, t(h, w, 16), t(h, w, 16), t(h, w, 16), t(h, w, 16), t(h, w),
                    t(h, w), t(h, w))
    with pytest.raises(B.BsmError) as e:
        B.bsm_batch_run(ctx, [d])
    assert e.value.status == B.BSM_ERR_UNSUPPORTED
    B.bsm_destroy(ctx)


# ---------------------------------------------------------------- mask ablations

@pytest.mark.parametrize("mode,n,win,dmax", [(1, 256, 5, 40), (1, 64, 1, 24), (2, 256, 5, 40), (2, 256, 1, 137),
                                             (2, 512, 3, 24)])
def test_mask_modes_full_chain(B, orc, mode, n, win, dmax):
    w, h = 83, 31
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=800 + n + mode)
    pairs = synth.pair_table(n, 31, seed=801)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=win, dmax=dmax, vote_radius=5, mask_mode=mode))
    nw = n // 32
    BL, PL, dl, pitch = _describe(B, ctx, l, nw)
    BR, PR, _, _ = _describe(B, ctx, r, nw)
    dL = torch.empty((h, w), dtype=torch.int32, device="cuda")
    dR = torch.empty_like(dL)
    cost = torch.zeros((h, w, dmax), dtype=torch.int16, device="cuda")
    B.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, cost)
    out = torch.empty_like(dL)
    B.bsm_refine(ctx, dl, pitch, dL, dR, w, h, dmax, out)
    torch.cuda.synchronize()
    ref = orc.pipeline(l, r, pairs, dmax, win=win, R=5, mask_mode=mode)
    assert (u32(PL) == ref["PhiL"]).all() and (u32(PR) == ref["PhiR"]).all()
    A = orc.aggregate(ref["BL"], ref["PhiL"], ref["BR"], dmax, win, 0, Phioth=ref["PhiR"] if mode == 2 else None)
    assert (cost.cpu().numpy().view(np.uint16).astype(np.uint32) == A).all()
    assert (dL.cpu().numpy() == ref["dL"]).all()
    assert (dR.cpu().numpy() == ref["dR"]).all()
    assert (out.cpu().numpy() == ref["disp"]).all()
    B.bsm_destroy(ctx)


def test_both_masks_refused_where_not_built(B):
    ctx = B.bsm_create(B.make_params(synth.pair_table(256, 31, seed=810), dmax=16, mask_mode=2))
    with pytest.raises(B.BsmError) as e:
        B.bsm_set_tuning(ctx, 0, 0, 0, 2)
    assert e.value.status == B.BSM_ERR_UNSUPPORTED
    w, h = 32, 8
    t = lambda *s: torch.zeros(s, dtype=torch.int32, device="cuda")
    img = torch.zeros((h, 3 * w), dtype=torch.uint8, device="cuda")
    d = B.pair_desc(img, img, w, h, 3 * w, 16, t(h, w, 8), t(h, w, 8), t(h, w, 8), t(h, w, 8), t(h, w), t(h, w),
                    t(h, w))
    with pytest.raises(B.BsmError) as e:
        B.bsm_batch_run(ctx, [d])
    assert e.value.status == B.BSM_ERR_UNSUPPORTED
    B.bsm_destroy(ctx)
