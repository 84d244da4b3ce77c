"""CUDA path vs the oracle, element by element, through the C ABI (needs a GPU).

Everything here is integer or bit work, so the bar is bit-exact equality: colour table, descriptor
and mask planes, aggregated cost volume, both WTA maps and the refined map.
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


class Ctx:
    def __init__(self, bsm, pairs, **kw):
        self.bsm = bsm
        self.params = bsm.make_params(pairs, **kw)
        self.ctx = bsm.bsm_create(self.params)
        self.nw = pairs.shape[0] // 32

    def close(self):
        self.bsm.bsm_destroy(self.ctx)

    def describe(self, img, pitch_pad=0):
        h, w, _ = img.shape
        pitch = 3 * w + pitch_pad
        buf = np.zeros((h, pitch), np.uint8)
        buf[:, : 3 * w] = img.reshape(h, 3 * w)
        d = torch.from_numpy(buf).cuda()
        Bp = torch.full((h, w, self.nw), -1, dtype=torch.int32, device="cuda")
        Pp = torch.full((h, w, self.nw), -1, dtype=torch.int32, device="cuda")
        self.bsm.bsm_describe(self.ctx, d, w, h, pitch, Bp, Pp)
        return Bp, Pp, d, pitch

    def cost_wta(self, BL, PhiL, BR, PhiR, dmax, want_cost=False):
        h, w, _ = BL.shape
        dL = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
        dR = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
        cost = torch.zeros((h, w, dmax), dtype=torch.int16, device="cuda") if want_cost else None
        self.bsm.bsm_cost_aggregate_wta(self.ctx, BL, PhiL, BR, PhiR, w, h, dmax, dL, dR, cost)
        return dL, dR, cost

    def refine(self, dimg, pitch, dL, dR, dmax):
        h, w = dL.shape
        out = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
        self.bsm.bsm_refine(self.ctx, dimg, pitch, dL, dR, w, h, dmax, out)
        return out


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_color_table_exhaustive(B, orc):
    pairs = synth.pair_table(256, 31, seed=1)
    c = Ctx(B, pairs)
    tab = torch.zeros(1 << 24, dtype=torch.int32, device="cuda")
    B.bsm_copy_color_table(c.ctx, tab)
    torch.cuda.synchronize()
    t = u32(tab)
    L, A, Bc, I = orc.lab_all()
    assert ((t & 0xFF).astype(np.int64) == L.astype(np.int64)).all()
    assert (((t >> 8) & 0xFF).astype(np.int64) - 128 == A.astype(np.int64)).all()
    assert (((t >> 16) & 0xFF).astype(np.int64) - 128 == Bc.astype(np.int64)).all()
    assert ((t >> 24).astype(np.int64) == I.astype(np.int64)).all()
    c.close()


@pytest.mark.parametrize("w,h,n,k,pad", [
    (450, 375, 256, 0, 0),   # Teddy-shaped, the paper's mask rank n/4
    (37, 23, 256, 100, 5),   # ragged tiles, pitch > 3w, another rank
    (1, 1, 64, 0, 0),
    (5, 7, 128, 1, 3),
    (33, 2, 32, 32, 0),
    (70, 40, 64, 64, 0),
])
def test_describe_bit_exact(B, orc, w, h, n, k, pad):
    l, _, _ = synth.stereo_pair(w, h, 16, seed=100 + w)
    pairs = synth.pair_table(n, 31, seed=w + h)
    c = Ctx(B, pairs, mask_rank=k, dmax=16)
    Bp, Pp, _, _ = c.describe(l, pad)
    torch.cuda.synchronize()
    oB, oP = orc.describe(l, pairs, k if k else None)
    assert (u32(Bp) == oB).all()
    assert (u32(Pp) == oP).all()
    c.close()


# k picks the bracket of T's search: k <= 32 (the lanes' smallest weights), 33..64 at n = 256 (their second
# smallest; 64 is the default n/4), any other rank (the smallest and the largest weight)
@pytest.mark.parametrize("w,h,n,k", [(450, 375, 256, 0), (37, 23, 256, 100), (33, 2, 64, 64), (5, 7, 128, 1),
                                     (61, 9, 256, 32), (61, 9, 256, 33), (40, 11, 64, 16), (29, 13, 128, 64),
                                     (70, 5, 256, 256)])
def test_describe_warp_per_pixel_bit_exact(B, orc, w, h, n, k):
    l, _, _ = synth.stereo_pair(w, h, 16, seed=120 + w)
    pairs = synth.pair_table(n, 31, seed=w + h + 1)
    c = Ctx(B, pairs, mask_rank=k, dmax=16)
    B.bsm_set_tuning(c.ctx, 0, 0, 0, 0, 2)
    Bp, Pp, _, _ = c.describe(l, 3)
    torch.cuda.synchronize()
    oB, oP = orc.describe(l, pairs, k if k else None)
    assert (u32(Bp) == oB).all()
    assert (u32(Pp) == oP).all()
    c.close()


# The warp-per-pixel kernel with 2..4 copies of its tile, each sample read from the copy its gather plan
# assigns (a tuning; the default is one copy); S = 9 makes a small halo, S = 63 takes fewer copies.
@pytest.mark.parametrize("w,h,n,S,copies", [(450, 375, 256, 31, 4), (37, 23, 256, 31, 2), (61, 9, 128, 31, 3),
                                            (40, 11, 64, 9, 4), (29, 13, 256, 63, 4)])
def test_describe_tile_copies_bit_exact(B, orc, w, h, n, S, copies):
    l, _, _ = synth.stereo_pair(w, h, 16, seed=130 + w)
    pairs = synth.pair_table(n, S, seed=w + h + 2)
    c = Ctx(B, pairs, dmax=16, window_S=S)
    B.bsm_set_tuning(c.ctx, 0, 0, 0, 0, 2, copies)
    assert B.bsm_get_tuning(c.ctx)["describe_copies"] == copies
    Bp, Pp, _, _ = c.describe(l, 3)
    torch.cuda.synchronize()
    oB, oP = orc.describe(l, pairs, None)
    assert (u32(Bp) == oB).all()
    assert (u32(Pp) == oP).all()
    c.close()


@pytest.mark.parametrize("win,n,dmax", [(1, 256, 24), (3, 64, 24), (5, 256, 24), (7, 128, 24), (5, 32, 24),
                                        (3, 256, 150), (7, 256, 137), (1, 128, 140)])
def test_cost_volume_bit_exact(B, orc, win, n, dmax):
    w, h = 61, 29
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=200 + win)
    pairs = synth.pair_table(n, 31, seed=201)
    c = Ctx(B, pairs, agg_window=win, dmax=dmax)
    BL, PL, _, _ = c.describe(l)
    BR, PR, _, _ = c.describe(r)
    dL, dR, cost = c.cost_wta(BL, PL, BR, PR, dmax, want_cost=True)
    torch.cuda.synchronize()
    oBL, oPL = orc.describe(l, pairs)
    oBR, oPR = orc.describe(r, pairs)
    A = orc.aggregate(oBL, oPL, oBR, dmax, win, 0)
    got = cost.cpu().numpy().view(np.uint16).astype(np.uint32)
    assert (got == A).all()
    assert (dL.cpu().numpy() == np.argmin(A, axis=2)).all()
    AR = orc.aggregate(oBR, oPR, oBL, dmax, win, 1)
    assert (dR.cpu().numpy() == np.argmin(AR, axis=2)).all()
    c.close()


@pytest.mark.parametrize("rows,plain,variant,dmax", [(8, 0, 1, 40), (8, 1, 1, 40), (16, 1, 2, 40), (128, 0, 2, 40),
                                                    (512, 1, 1, 40), (8, 0, 2, 200), (32, 1, 2, 129),
                                                    (16, 0, 1, 200), (32, 2, 2, 200), (64, 2, 2, 40)])
def test_tuning_does_not_change_bits(B, orc, rows, plain, variant, dmax):
    w, h = 77, 41
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=250)
    pairs = synth.pair_table(256, 31, seed=251)
    c = Ctx(B, pairs, agg_window=5, dmax=dmax)
    B.bsm_set_tuning(c.ctx, rows, plain, 0, variant)
    assert B.bsm_get_tuning(c.ctx) == {"cost_rows": rows, "cost_popc_plain": plain, "batch_rows": 0,
                                       "cost_variant": variant, "describe_variant": 0, "describe_copies": 0}
    BL, PL, _, _ = c.describe(l)
    BR, PR, _, _ = c.describe(r)
    dL, dR, cost = c.cost_wta(BL, PL, BR, PR, dmax, want_cost=True)
    torch.cuda.synchronize()
    oBL, oPL = orc.describe(l, pairs)
    oBR, oPR = orc.describe(r, pairs)
    A = orc.aggregate(oBL, oPL, oBR, dmax, 5, 0)
    assert (cost.cpu().numpy().view(np.uint16).astype(np.uint32) == A).all()
    assert (dL.cpu().numpy() == np.argmin(A, axis=2)).all()
    assert (dR.cpu().numpy() == orc.wta(oBR, oPR, oBL, dmax, 5, 1)).all()
    c.close()


@pytest.mark.parametrize("win", [1, 5])
def test_wta_and_refine_teddy_shape(B, orc, win):
    w, h, dmax = 450, 375, 60
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=1)
    pairs = synth.pair_table(256, 31, seed=11)
    c = Ctx(B, pairs, agg_window=win, dmax=dmax)
    BL, PL, dl, pitch = c.describe(l)
    BR, PR, _, _ = c.describe(r)
    dL, dR, _ = c.cost_wta(BL, PL, BR, PR, dmax)
    torch.cuda.synchronize()
    ref = orc.pipeline(l, r, pairs, dmax, win=win)
    assert (u32(BL) == ref["BL"]).all() and (u32(PR) == ref["PhiR"]).all()
    assert (dL.cpu().numpy() == ref["dL"]).all()
    assert (dR.cpu().numpy() == ref["dR"]).all()
    # refinement from the oracle's own WTA maps, then the GPU's full chain
    out_o = c.refine(dl, pitch, torch.from_numpy(ref["dL"]).cuda(), torch.from_numpy(ref["dR"]).cuda(), dmax)
    out = c.refine(dl, pitch, dL, dR, dmax)
    torch.cuda.synchronize()
    assert (out_o.cpu().numpy() == ref["disp"]).all()
    assert (out.cpu().numpy() == ref["disp"]).all()
    assert 0.02 < 1 - ref["valid"].mean() < 0.6  # the refinement really ran on many pixels
    c.close()


@pytest.mark.parametrize("n", [64, 256])
@pytest.mark.parametrize("w,h,dmax,win", [
    (20, 9, 40, 5),    # dmax > width: most matches fall outside the image
    (3, 3, 1, 1),      # dmax = 1
    (1, 12, 8, 3),
    (130, 17, 256, 5), # the largest dmax on a narrow image
    (95, 33, 13, 7),   # dmax not a multiple of 8
    (70, 9, 64, 3),    # 64 columns plus a ragged tail
])
def test_edge_shapes_full_chain(B, orc, w, h, dmax, win, n):
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=300 + w)
    pairs = synth.pair_table(n, 31, seed=301)
    c = Ctx(B, pairs, agg_window=win, dmax=dmax, vote_radius=4)
    BL, PL, dl, pitch = c.describe(l, 1)
    BR, PR, _, _ = c.describe(r, 1)
    dL, dR, _ = c.cost_wta(BL, PL, BR, PR, dmax)
    out = c.refine(dl, pitch, dL, dR, dmax)
    torch.cuda.synchronize()
    ref = orc.pipeline(l, r, pairs, dmax, win=win, R=4)
    assert (dL.cpu().numpy() == ref["dL"]).all()
    assert (dR.cpu().numpy() == ref["dR"]).all()
    assert (out.cpu().numpy() == ref["disp"]).all()
    c.close()


def test_refine_fallback_and_tolerance(B, orc):
    # Hand-made maps: a band with no valid pixel within R forces the row fallback.
    w, h, dmax = 90, 12, 32
    l, _, _ = synth.stereo_pair(w, h, dmax, seed=400)
    rng = np.random.default_rng(401)
    dL = rng.integers(0, dmax, size=(h, w)).astype(np.int32)
    dR = rng.integers(0, dmax, size=(h, w)).astype(np.int32)
    for tol in (0, 1, 3):
        c = Ctx(B, synth.pair_table(32, 31, seed=402), dmax=dmax, vote_radius=2, lr_tol=tol)
        img = torch.from_numpy(np.ascontiguousarray(l.reshape(h, 3 * w))).cuda()
        out = c.refine(img, 3 * w, torch.from_numpy(dL).cuda(), torch.from_numpy(dR).cuda(), dmax)
        torch.cuda.synchronize()
        valid = orc.lr_check(dL, dR, tol)
        ref = orc.refine(l, dL, valid, dmax, R=2)
        assert (out.cpu().numpy() == ref).all()
        c.close()


# An image with at least 4 x 152 blocks of 32 x 32 takes the refinement's 32-row blocks in decreasing order
# of their invalid pixels (counted by the pre-pass). Hand-made maps: disparities below 24 constant over
# 96 x 96 blocks with dR = dL (invalid only where the match crosses a block edge), and a few large rectangles where
# dR disagrees, so a handful of blocks carry most of the invalid pixels. R = 7 runs the general-radius
# kernel, R = 15 the unrolled one.
@pytest.mark.parametrize("R,w,h", [(7, 1280, 512), (15, 1280, 512), (15, 1290, 500)])  # the last: ragged blocks
def test_refine_ordered_blocks_bit_exact(B, orc, R, w, h):
    dmax = 64
    l, _, _ = synth.stereo_pair(w, h, dmax, seed=450)
    rng = np.random.default_rng(451 + R + w)
    blocks = rng.integers(0, 24, size=((h + 95) // 96, (w + 95) // 96))
    dL = np.kron(blocks, np.ones((96, 96), np.int64))[:h, :w].astype(np.int32)
    dR = dL.copy()
    for _ in range(6):
        y0, x0 = int(rng.integers(0, h - 100)), int(rng.integers(0, w - 160))
        dR[y0:y0 + int(rng.integers(40, 100)), x0:x0 + int(rng.integers(60, 160))] = rng.integers(0, dmax)
    c = Ctx(B, synth.pair_table(64, 31, seed=452), dmax=dmax, vote_radius=R)
    img = torch.from_numpy(np.ascontiguousarray(l.reshape(h, 3 * w))).cuda()
    out = c.refine(img, 3 * w, torch.from_numpy(dL).cuda(), torch.from_numpy(dR).cuda(), dmax)
    torch.cuda.synchronize()
    valid = orc.lr_check(dL, dR, 1)
    assert 0.02 < 1.0 - valid.mean() < 0.6  # some invalid pixels, clustered in the rectangles
    ref = orc.refine(l, dL, valid, dmax, R=R)
    assert (out.cpu().numpy() == ref).all()
    c.close()


def test_match_host_equals_device_chain(B, orc):
    w, h, dmax = 200, 90, 48
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=500)
    pairs = synth.pair_table(256, 31, seed=501)
    c = Ctx(B, pairs, dmax=dmax)
    out = np.zeros((h, w), np.int32)
    B.bsm_match_host(c.ctx, l, r, w, h, 3 * w, dmax, out)
    ref = orc.pipeline(l, r, pairs, dmax, win=5)
    assert (out == ref["disp"]).all()
    c.close()


def test_constant_shift_on_gpu(B):
    w, h, dmax, s = 160, 60, 32, 9
    l, r = synth.shifted_pair(w, h, s, seed=600)
    c = Ctx(B, synth.pair_table(256, 31, seed=601), dmax=dmax)
    BL, PL, _, _ = c.describe(l)
    BR, PR, _, _ = c.describe(r)
    dL, dR, _ = c.cost_wta(BL, PL, BR, PR, dmax)
    m = 17
    assert (dL.cpu().numpy()[m:-m, m + s : w - m] == s).all()
    assert (dR.cpu().numpy()[m:-m, m : w - m - s] == s).all()
    c.close()


def test_argument_errors_are_synchronous(B):
    c = Ctx(B, synth.pair_table(64, 31, seed=700), dmax=16)
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BsmError) as e:
        B.bsm_cost_aggregate_wta(c.ctx, x, x, x, x, 4, 4, 17, x, x)  # dmax above the context's
    assert e.value.status == B.BSM_ERR_INVALID_ARG
    with pytest.raises(B.BsmError):
        B.bsm_describe(c.ctx, x, 4, 4, 11, x, x)  # pitch < 3 w
    with pytest.raises(B.BsmError):
        B.bsm_describe(c.ctx, x, 0, 4, 12, x, x)
    with pytest.raises(B.BsmError):
        B.bsm_describe(c.ctx, x, 4, 4, 12, x.data_ptr() + 4, x)  # misaligned plane
    assert B.bsm_last_error(c.ctx) == B.BSM_OK
    c.close()


def test_autotuner_applies_a_candidate_and_bits_stay(B, orc):
    from paper_1402_2020_gb300 import autotune

    w, h, dmax = 150, 70, 48
    pairs = synth.pair_table(256, 31, seed=260)
    c = Ctx(B, pairs, agg_window=5, dmax=dmax)
    t = autotune.tune_cost(c.ctx, 256, 5, w, h, dmax, reps=1, use_cache=False)
    assert t["cost_rows"] in autotune.COST_ROWS + (0,) and t["cost_popc_plain"] in (0, 1, 2)
    assert t["cost_variant"] in autotune.VARIANTS
    assert B.bsm_get_tuning(c.ctx)["cost_rows"] == t["cost_rows"]
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=261)
    BL, PL, _, _ = c.describe(l)
    BR, PR, _, _ = c.describe(r)
    dL, _, _ = c.cost_wta(BL, PL, BR, PR, dmax)
    oBL, oPL = orc.describe(l, pairs)
    oBR, _ = orc.describe(r, pairs)
    assert (dL.cpu().numpy() == orc.wta(oBL, oPL, oBR, dmax, 5, 0)).all()
    c.close()
