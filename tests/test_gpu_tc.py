"""The tensor-core cost kernel (cost_variant 3: Eq. 8 as an exact E4M3 product on tcgen05) against the
oracle, bit-exact: both aggregated cost volumes, both WTA maps, the refined map (needs a GPU)."""
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


def _planes(B, ctx, img, nw):
    h, w, _ = img.shape
    d = torch.from_numpy(img).cuda()
    Bp = torch.full((h, w, nw), -1, dtype=torch.int32, device="cuda")
    Pp = torch.full((h, w, nw), -1, dtype=torch.int32, device="cuda")
    B.bsm_describe(ctx, d, w, h, 3 * w, Bp, Pp)
    return Bp, Pp, d


@pytest.mark.parametrize("w,h,dmax,win,rows", [
    (61, 29, 24, 5, 0),      # one tile, dmax below one 32-column group
    (300, 40, 256, 5, 0),    # the largest dmax: two N-blocks, tiles with and without border matches
    (300, 40, 256, 5, 8),    # short bands: the window's first rows in every band
    (257, 33, 137, 3, 0),    # dmax not a multiple of 32
    (130, 21, 64, 7, 16),
    (200, 19, 100, 1, 0),    # no aggregation
    (17, 50, 40, 5, 0),      # narrower than the disparity range
    (1, 9, 8, 3, 0),         # one column
    (126, 3, 200, 7, 0),     # fewer rows than the window
    (4100, 9, 256, 5, 0),    # long rows: 34 column tiles, a few rows
    (1500, 64, 200, 7, 32),  # window 7 (the popcount ring's deepest lead), bands of 32 rows
])
def test_tc_cost_volumes_bit_exact(B, orc, w, h, dmax, win, rows):
    l, r, _ = synth.stereo_pair(w, h, min(dmax, max(w - 1, 1)), seed=1000 + w + h)
    pairs = synth.pair_table(256, 31, seed=1001)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=win, dmax=dmax))
    B.bsm_set_tuning(ctx, rows, 0, 0, 3)
    BL, PL, _ = _planes(B, ctx, l, 8)
    BR, PR, _ = _planes(B, ctx, r, 8)
    dL = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
    dR = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
    cL = torch.zeros((h, w, dmax), dtype=torch.int16, device="cuda")
    cR = torch.zeros((h, w, dmax), dtype=torch.int16, device="cuda")
    B.bsm_cost_volumes(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, cL, cR)
    torch.cuda.synchronize()
    assert B.bsm_last_error(ctx) == B.BSM_OK
    oBL, oPL = orc.describe(l, pairs)
    oBR, oPR = orc.describe(r, pairs)
    AL = orc.aggregate(oBL, oPL, oBR, dmax, win, 0)
    AR = orc.aggregate(oBR, oPR, oBL, dmax, win, 1)
    gl = cL.cpu().numpy().view(np.uint16)
    gr = cR.cpu().numpy().view(np.uint16)
    bad = np.argwhere(gl != AL)
    assert bad.size == 0, f"left cost differs at {bad[:5].tolist()} ({gl[tuple(bad[0])]} vs {AL[tuple(bad[0])]})"
    bad = np.argwhere(gr != AR)
    assert bad.size == 0, f"right cost differs at {bad[:5].tolist()} ({gr[tuple(bad[0])]} vs {AR[tuple(bad[0])]})"
    assert (dL.cpu().numpy() == np.argmin(AL, axis=2)).all()
    assert (dR.cpu().numpy() == np.argmin(AR, axis=2)).all()
    B.bsm_destroy(ctx)


@pytest.mark.parametrize("mode", [0, 1])
def test_tc_full_chain(B, orc, mode):
    w, h, dmax = 450, 120, 60
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=1010 + mode)
    pairs = synth.pair_table(256, 31, seed=1011)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=5, dmax=dmax, mask_mode=mode))
    B.bsm_set_tuning(ctx, 0, 0, 0, 3)
    BL, PL, dl = _planes(B, ctx, l, 8)
    BR, PR, _ = _planes(B, ctx, r, 8)
    dL = torch.empty((h, w), dtype=torch.int32, device="cuda")
    dR = torch.empty_like(dL)
    B.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR)
    out = torch.empty_like(dL)
    B.bsm_refine(ctx, dl, 3 * w, dL, dR, w, h, dmax, out)
    torch.cuda.synchronize()
    ref = orc.pipeline(l, r, pairs, dmax, win=5, mask_mode=mode)
    assert (dL.cpu().numpy() == ref["dL"]).all()
    assert (dR.cpu().numpy() == ref["dR"]).all()
    assert (out.cpu().numpy() == ref["disp"]).all()
    B.bsm_destroy(ctx)


def test_tc_matches_the_popcount_kernels_at_full_size(B):
    # 1390 x 1110, dmax 256: the tensor-core kernel and the two-column popcount kernel agree everywhere
    w, h, dmax = 1390, 1110, 256
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=2, radiometric_change=True)
    ctx = B.bsm_create(B.make_params(synth.pair_table(256, 31, seed=11), agg_window=5, dmax=dmax))
    BL, PL, _ = _planes(B, ctx, l, 8)
    BR, PR, _ = _planes(B, ctx, r, 8)
    maps = []
    for variant in (2, 3):
        B.bsm_set_tuning(ctx, 0, 0, 0, variant)
        dL = torch.empty((h, w), dtype=torch.int32, device="cuda")
        dR = torch.empty_like(dL)
        B.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR)
        maps.append((dL, dR))
    torch.cuda.synchronize()
    assert B.bsm_last_error(ctx) == B.BSM_OK
    assert torch.equal(maps[0][0], maps[1][0]) and torch.equal(maps[0][1], maps[1][1])
    B.bsm_destroy(ctx)


def test_tc_refused_where_not_built(B):
    ctx = B.bsm_create(B.make_params(synth.pair_table(128, 31, seed=1020), dmax=32))
    with pytest.raises(B.BsmError) as e:
        B.bsm_set_tuning(ctx, 0, 0, 0, 3)
    assert e.value.status == B.BSM_ERR_UNSUPPORTED
    B.bsm_destroy(ctx)
