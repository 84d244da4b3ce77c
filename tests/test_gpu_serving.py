"""The serving engine (continuous batching) against the per-pair path (needs a GPU)."""
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


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def reference_map(B, ctx, l, r, dmax):
    h, w, _ = l.shape
    out = np.zeros((h, w), np.int32)
    B.bsm_match_host(ctx, np.ascontiguousarray(l), np.ascontiguousarray(r), w, h, 3 * w, dmax, out)
    return out


def wait_all(B, srv, ids, timeout_s=60):
    got = {}
    t0 = time.time()
    while len(got) < len(ids):
        for cid, st, lat in B.bsm_server_poll(srv, 256, 10000):
            got[cid] = st
        assert time.time() - t0 < timeout_s, "requests did not complete"
    return got


SHAPES = [(640, 480, 64), (320, 240, 128), (200, 150, 256), (500, 90, 64), (97, 41, 13), (640, 480, 256)]


def test_alone_and_in_the_mix(B):
    pairs = synth.pair_table(256, 31, seed=2000)
    params = B.make_params(pairs, agg_window=5, dmax=256)
    ctx = B.bsm_create(params)
    srv = B.bsm_server_create(params, lanes=2, max_batch=8)
    try:
        reqs = []
        for i, (w, h, d) in enumerate(SHAPES * 3):
            l, r, _ = synth.stereo_pair(w, h, d, seed=2100 + i % len(SHAPES))
            reqs.append({"w": w, "h": h, "d": d, "l": pinned(l), "r": pinned(r), "l_np": l, "r_np": r,
                         "out": torch.full((h, w), -3, dtype=torch.int32).pin_memory()})
        # the first request alone
        a = reqs[0]
        assert B.bsm_server_submit(srv, 0, a["l"], a["r"], a["w"], a["h"], 3 * a["w"], a["d"], a["out"]) == B.BSM_OK
        assert wait_all(B, srv, [0]) == {0: B.BSM_OK}
        alone = a["out"].numpy().copy()
        # everything at once, the first request included again
        a["out"].fill_(-3)
        for i, q in enumerate(reqs):
            assert B.bsm_server_submit(srv, 100 + i, q["l"], q["r"], q["w"], q["h"], 3 * q["w"], q["d"],
                                       q["out"]) == B.BSM_OK
        got = wait_all(B, srv, list(range(100, 100 + len(reqs))))
        assert all(st == B.BSM_OK for st in got.values())
        assert (a["out"].numpy() == alone).all()
        for q in reqs[: len(SHAPES)]:
            assert (q["out"].numpy() == reference_map(B, ctx, q["l_np"], q["r_np"], q["d"])).all()
        for i, q in enumerate(reqs[len(SHAPES):]):
            assert (q["out"].numpy() == reqs[i % len(SHAPES)]["out"].numpy()).all()
        st = B.bsm_server_get_stats(srv)
        assert st["completed"] == len(reqs) + 1 and st["failed"] == 0 and st["bytes_in_use"] == 0
        assert st["max_batch_seen"] > 1  # requests were batched together
    finally:
        B.bsm_server_destroy(srv)
        B.bsm_destroy(ctx)


def test_rejects_and_small_budget(B):
    pairs = synth.pair_table(64, 31, seed=2200)
    params = B.make_params(pairs, agg_window=3, dmax=64)
    ctx = B.bsm_create(params)
    # room for about one 400x300 request at a time: admission must wait for memory, not fail
    budget = 400 * 300 * (2 * 3 + 4 * 8 + 3 * 4 + 4) + 8 * 4096  # views, planes, maps, lane scratch
    srv = B.bsm_server_create(params, lanes=3, max_batch=4, device_budget=budget)
    try:
        l, r, _ = synth.stereo_pair(400, 300, 64, seed=2201)
        L, R = pinned(l), pinned(r)
        outs = [torch.zeros((300, 400), dtype=torch.int32).pin_memory() for _ in range(5)]
        for i in range(5):
            assert B.bsm_server_submit(srv, i, L, R, 400, 300, 1200, 64, outs[i]) == B.BSM_OK
        # malformed (dmax above the engine's) and larger than the whole budget
        assert B.bsm_server_submit(srv, 50, L, R, 400, 300, 1200, 65, outs[0]) == B.BSM_ERR_INVALID_ARG
        big = torch.zeros((1000, 1000), dtype=torch.int32).pin_memory()
        assert B.bsm_server_submit(srv, 51, L, R, 1000, 1000, 3000, 64, big) == B.BSM_ERR_INVALID_ARG
        got = wait_all(B, srv, [0, 1, 2, 3, 4, 50, 51])
        assert got[50] == B.BSM_ERR_INVALID_ARG and got[51] == B.BSM_ERR_INVALID_ARG
        assert all(got[i] == B.BSM_OK for i in range(5))
        ref = reference_map(B, ctx, l, r, 64)
        for o in outs:
            assert (o.numpy() == ref).all()
        B.bsm_server_drain(srv, 10000)
        st = B.bsm_server_get_stats(srv)
        assert st["failed"] == 2 and st["completed"] == 5 and st["max_batch_seen"] == 1
        assert 0 < st["scratch_bytes"] <= 3 * 4 * 400 * 300  # one colour plane per lane at most, charged
    finally:
        B.bsm_server_destroy(srv)
        B.bsm_destroy(ctx)


def test_large_request_alone_in_the_mix_and_against_the_oracle(B, orc):
    """A request of 1280 x 720 x 128 pixel-disparities takes the engine's per-pair branch (two describes,
    the tensor-core cost kernel, refine on the lane's stream) while small requests are batched beside it:
    its map is the same alone and in the mix, and equals the oracle on a band of rows."""
    pairs = synth.pair_table(256, 31, seed=2300)
    params = B.make_params(pairs, agg_window=5, dmax=256)
    ctx = B.bsm_create(params)
    srv = B.bsm_server_create(params, lanes=2, max_batch=8)
    try:
        W, H, D = 1280, 720, 128
        assert B.bsm_cost_plan(ctx, W, H, D)["kernel"] == 3  # the automatic choice at this size
        big_l, big_r, _ = synth.stereo_pair(W, H, D, seed=2301)
        big = {"l": pinned(big_l), "r": pinned(big_r)}
        outs = [torch.full((H, W), -3, dtype=torch.int32).pin_memory() for _ in range(2)]
        assert B.bsm_server_submit(srv, 0, big["l"], big["r"], W, H, 3 * W, D, outs[0]) == B.BSM_OK
        assert wait_all(B, srv, [0], timeout_s=120) == {0: B.BSM_OK}
        small = []
        for i, (w, h, d) in enumerate([(640, 480, 64), (320, 240, 128), (640, 480, 256), (200, 150, 64)] * 2):
            l, r, _ = synth.stereo_pair(w, h, d, seed=2310 + i)
            small.append({"w": w, "h": h, "d": d, "l": pinned(l), "r": pinned(r),
                          "out": torch.full((h, w), -3, dtype=torch.int32).pin_memory()})
        # the large request in the middle of the small ones, all submitted at once
        for i, q in enumerate(small[:4]):
            assert B.bsm_server_submit(srv, 10 + i, q["l"], q["r"], q["w"], q["h"], 3 * q["w"], q["d"],
                                       q["out"]) == B.BSM_OK
        assert B.bsm_server_submit(srv, 1, big["l"], big["r"], W, H, 3 * W, D, outs[1]) == B.BSM_OK
        for i, q in enumerate(small[4:]):
            assert B.bsm_server_submit(srv, 14 + i, q["l"], q["r"], q["w"], q["h"], 3 * q["w"], q["d"],
                                       q["out"]) == B.BSM_OK
        got = wait_all(B, srv, [1] + list(range(10, 18)), timeout_s=120)
        assert all(st == B.BSM_OK for st in got.values())
        assert (outs[1].numpy() == outs[0].numpy()).all()  # alone == in the mix
        for q in small[:2]:
            assert (q["out"].numpy() == reference_map(B, ctx, q["l"].numpy(), q["r"].numpy(), q["d"])).all()
        # the oracle on rows 300 .. 303: both WTA maps over the rows their vote windows reach
        y0, y1, R, win = 300, 304, 15, 5
        a, b = y0 - R - win // 2, y1 + R + win // 2
        h, w = H, W
        planes = [np.zeros((h, w, 8), np.uint32) for _ in range(4)]
        orc.describe(big_l, pairs, None, a, b, out=(planes[0], planes[1]))
        orc.describe(big_r, pairs, None, a, b, out=(planes[2], planes[3]))
        far = 10 ** 6
        dL = np.full((h, w), far, np.int32)
        dR = np.zeros((h, w), np.int32)
        dL[y0 - R:y1 + R] = orc.wta(planes[0], planes[1], planes[2], D, win, 0, 0, w, y0 - R, y1 + R)
        dR[y0 - R:y1 + R] = orc.wta(planes[2], planes[3], planes[0], D, win, 1, 0, w, y0 - R, y1 + R)
        valid = orc.lr_check(dL, dR, 1)
        expect = orc.refine_region(big_l, dL, valid, D, 0, w, y0, y1, R=R)
        assert (outs[1].numpy()[y0:y1] == expect).all()
        st = B.bsm_server_get_stats(srv)
        assert st["failed"] == 0
    finally:
        B.bsm_server_destroy(srv)
        B.bsm_destroy(ctx)
