"""bsm_batch_run against the per-pair C-ABI path and the oracle (needs a GPU)."""
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


def make_pair(w, h, dmax, seed, nw):
    l, r, _ = synth.stereo_pair(w, h, dmax, seed)
    dev = "cuda"
    t = {"w": w, "h": h, "dmax": dmax, "l": l, "r": r,
         "rgbL": torch.from_numpy(l).to(dev), "rgbR": torch.from_numpy(r).to(dev)}
    for k in ("BL", "PhiL", "BR", "PhiR"):
        t[k] = torch.full((h, w, nw), -1, dtype=torch.int32, device=dev)
    for k in ("dispL", "dispR", "out"):
        t[k] = torch.full((h, w), -5, dtype=torch.int32, device=dev)
    return t


def desc(B, t):
    return B.pair_desc(t["rgbL"], t["rgbR"], t["w"], t["h"], 3 * t["w"], t["dmax"], t["BL"], t["PhiL"], t["BR"],
                       t["PhiR"], t["dispL"], t["dispR"], t["out"])


def per_pair(B, ctx, t, nw):
    w, h, dmax = t["w"], t["h"], t["dmax"]
    o = {k: torch.empty_like(t[k]) for k in ("BL", "PhiL", "BR", "PhiR", "dispL", "dispR", "out")}
    B.bsm_describe(ctx, t["rgbL"], w, h, 3 * w, o["BL"], o["PhiL"])
    B.bsm_describe(ctx, t["rgbR"], w, h, 3 * w, o["BR"], o["PhiR"])
    B.bsm_cost_aggregate_wta(ctx, o["BL"], o["PhiL"], o["BR"], o["PhiR"], w, h, dmax, o["dispL"], o["dispR"])
    B.bsm_refine(ctx, t["rgbL"], 3 * w, o["dispL"], o["dispR"], w, h, dmax, o["out"])
    return o


SHAPES_A = [(320, 240, 64), (97, 61, 13), (200, 33, 192), (150, 90, 256), (41, 300, 128), (5, 3, 1), (64, 64, 60)]
SHAPES_B = [(130, 70, 256), (333, 51, 64), (17, 200, 100)]


@pytest.mark.parametrize("win,n", [(5, 256), (3, 64)])
def test_batch_equals_per_pair(B, win, n):
    pairs = synth.pair_table(n, 31, seed=1000 + n)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=win, dmax=256))
    nw = n // 32
    try:
        for rnd, shapes in enumerate((SHAPES_A, SHAPES_B, SHAPES_A)):  # graph replays with new shapes
            ts = [make_pair(w, h, d, seed=1100 + 10 * rnd + i, nw=nw) for i, (w, h, d) in enumerate(shapes)]
            B.bsm_batch_run(ctx, [desc(B, t) for t in ts])
            torch.cuda.synchronize()
            for t in ts:
                ref = per_pair(B, ctx, t, nw)
                torch.cuda.synchronize()
                for k in ("BL", "PhiL", "BR", "PhiR", "dispL", "dispR", "out"):
                    assert torch.equal(t[k], ref[k]), (k, t["w"], t["h"], t["dmax"], rnd)
        assert B.bsm_last_error(ctx) == B.BSM_OK
    finally:
        B.bsm_destroy(ctx)


# describe variants: 0 picks warp per pixel at n = 256 and thread per pixel below; 1 and 2 force one
@pytest.mark.parametrize("n,variants", [(256, (0, 1)), (128, (2, 1)), (64, (0, 2))])
def test_batch_matches_oracle(B, orc, n, variants):
    pairs = synth.pair_table(n, 31, seed=1200 + n)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=5, dmax=64, vote_radius=6))
    try:
        for rnd, variant in enumerate(variants):  # the second variant needs a new graph
            B.bsm_set_tuning(ctx, 0, 0, 0, 0, variant)
            shapes = [(90, 40, 32), (47, 29, 64), (33, 7, 20)]
            ts = [make_pair(w, h, d, seed=1300 + 10 * rnd + i, nw=n // 32) for i, (w, h, d) in enumerate(shapes)]
            B.bsm_batch_run(ctx, [desc(B, t) for t in ts])
            torch.cuda.synchronize()
            for t in ts:
                ref = orc.pipeline(t["l"], t["r"], pairs, t["dmax"], win=5, R=6)
                assert (t["BL"].cpu().numpy().view(np.uint32) == ref["BL"]).all(), (n, variant)
                assert (t["PhiR"].cpu().numpy().view(np.uint32) == ref["PhiR"]).all(), (n, variant)
                assert (t["dispL"].cpu().numpy() == ref["dL"]).all()
                assert (t["dispR"].cpu().numpy() == ref["dR"]).all()
                assert (t["out"].cpu().numpy() == ref["disp"]).all()
        assert B.bsm_last_error(ctx) == B.BSM_OK
    finally:
        B.bsm_destroy(ctx)


def test_batch_argument_errors(B):
    pairs = synth.pair_table(64, 31, seed=1400)
    ctx = B.bsm_create(B.make_params(pairs, dmax=32))
    try:
        t = make_pair(40, 20, 32, seed=1401, nw=2)
        d = desc(B, t)
        d.dmax = 33  # above the context's dmax
        with pytest.raises(B.BsmError):
            B.bsm_batch_run(ctx, [d])
        with pytest.raises(B.BsmError):
            B.bsm_batch_run(ctx, [])
        d = desc(B, t)
        d.out = None
        with pytest.raises(B.BsmError):
            B.bsm_batch_run(ctx, [d])
    finally:
        B.bsm_destroy(ctx)


def test_batch_with_tensor_core_pairs(B):
    # pairs of at least 1280 x 720 x 128 pixel-disparities run the tensor-core cost kernel inside the batch;
    # every output equals the per-pair calls' (popcount cost kernel) bit for bit
    pairs = synth.pair_table(256, 31, seed=1500)
    ctx = B.bsm_create(B.make_params(pairs, agg_window=5, dmax=256))
    try:
        shapes = [(1280, 720, 128), (200, 90, 64), (1300, 740, 256), (97, 61, 13)]
        ts = [make_pair(w, h, d, seed=1510 + i, nw=8) for i, (w, h, d) in enumerate(shapes)]
        B.bsm_batch_run(ctx, [desc(B, t) for t in ts])
        torch.cuda.synchronize()
        B.bsm_set_tuning(ctx, 0, 0, 0, 2)  # the per-pair reference takes the two-column popcount kernel
        for t in ts:
            ref = per_pair(B, ctx, t, 8)
            torch.cuda.synchronize()
            for k in ("BL", "PhiL", "BR", "PhiR", "dispL", "dispR", "out"):
                assert torch.equal(t[k], ref[k]), (k, t["w"], t["h"], t["dmax"])
        assert B.bsm_last_error(ctx) == B.BSM_OK
    finally:
        B.bsm_destroy(ctx)
