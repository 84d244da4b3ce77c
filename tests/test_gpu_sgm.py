"""Semi-global aggregation (the global optimisation of the paper's future work) and the two-view cost
volumes, against the oracle, bit-exact (needs a GPU)."""
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


@pytest.fixture(scope="module")
def ctx(B):
    c = B.bsm_create(B.make_params(synth.pair_table(256, 31, seed=900), dmax=256))
    yield c
    B.bsm_destroy(c)


def _run_sgm(B, ctx, C, P1, P2, paths):
    h, w, dmax = C.shape
    dC = torch.from_numpy(C.view(np.int16)).cuda()
    S = torch.full((h, w, dmax), -1, dtype=torch.int32, device="cuda")
    disp = torch.full((h, w), -1, dtype=torch.int32, device="cuda")
    B.bsm_sgm(ctx, dC, w, h, dmax, P1, P2, paths, S, disp)
    torch.cuda.synchronize()
    return S.cpu().numpy().view(np.uint32), disp.cpu().numpy()


@pytest.mark.parametrize("h,w,dmax,P1,P2,cmax", [
    (1, 1, 5, 3, 9, 100),
    (1, 17, 1, 0, 0, 50),
    (13, 1, 7, 2, 2, 30),
    (29, 37, 24, 8, 32, 200),
    (23, 41, 33, 5, 40, 90),     # dmax just above one lane's worth
    (31, 19, 100, 4, 64, 400),
    (17, 45, 137, 10, 100, 6400),
    (12, 20, 256, 7, 65535, 65535),  # the largest values: the packed keys must not overflow
])
@pytest.mark.parametrize("paths", [4, 8])
def test_sgm_bit_exact(B, orc, ctx, h, w, dmax, P1, P2, cmax, paths):
    rng = np.random.default_rng(h * 1000 + w + dmax)
    C = rng.integers(0, cmax + 1, size=(h, w, dmax)).astype(np.uint16)
    S, disp = _run_sgm(B, ctx, C, P1, P2, paths)
    oS, odisp = orc.sgm(C, P1, P2, orc.SGM_DIRS4 if paths == 4 else orc.SGM_DIRS8)
    assert (S == oS).all()
    assert (disp == odisp).all()


def test_cost_volumes_both_views(B, orc):
    w, h, dmax = 67, 29, 40
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=910)
    pairs = synth.pair_table(256, 31, seed=911)
    c = B.bsm_create(B.make_params(pairs, agg_window=3, dmax=dmax))
    BL, PL, BR, PR = (torch.empty((h, w, 8), dtype=torch.int32, device="cuda") for _ in range(4))
    dl, dr = torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()
    B.bsm_describe(c, dl, w, h, 3 * w, BL, PL)
    B.bsm_describe(c, dr, w, h, 3 * w, BR, PR)
    dL, dR = torch.empty((h, w), dtype=torch.int32, device="cuda"), torch.empty((h, w), dtype=torch.int32,
                                                                                 device="cuda")
    cL = torch.zeros((h, w, dmax), dtype=torch.int16, device="cuda")
    cR = torch.zeros((h, w, dmax), dtype=torch.int16, device="cuda")
    B.bsm_cost_volumes(c, BL, PL, BR, PR, w, h, dmax, dL, dR, cL, cR)
    torch.cuda.synchronize()
    oBL, oPL = orc.describe(l, pairs)
    oBR, oPR = orc.describe(r, pairs)
    AL = orc.aggregate(oBL, oPL, oBR, dmax, 3, 0)
    AR = orc.aggregate(oBR, oPR, oBL, dmax, 3, 1)
    assert (cL.cpu().numpy().view(np.uint16) == AL).all()
    assert (cR.cpu().numpy().view(np.uint16) == AR).all()
    assert (dL.cpu().numpy() == np.argmin(AL, axis=2)).all()
    assert (dR.cpu().numpy() == np.argmin(AR, axis=2)).all()
    B.bsm_destroy(c)


@pytest.mark.parametrize("n,win,paths,variant", [(256, 1, 8, 0), (256, 5, 4, 1), (64, 3, 8, 0), (512, 3, 4, 0)])
def test_sgm_full_chain(B, orc, n, win, paths, variant):
    w, h, dmax = 90, 40, 48
    l, r, _ = synth.stereo_pair(w, h, dmax, seed=920 + n + win)
    pairs = synth.pair_table(n, 31, seed=921)
    P1, P2 = 2 * win * win, 8 * win * win
    c = B.bsm_create(B.make_params(pairs, agg_window=win, dmax=dmax, vote_radius=6))
    if variant:
        B.bsm_set_tuning(c, 0, 0, 0, variant)
    nw = n // 32
    BL, PL, BR, PR = (torch.empty((h, w, nw), dtype=torch.int32, device="cuda") for _ in range(4))
    dl, dr = torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()
    B.bsm_describe(c, dl, w, h, 3 * w, BL, PL)
    B.bsm_describe(c, dr, w, h, 3 * w, BR, PR)
    wL, wR, sL, sR, out = (torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(5))
    cL = torch.empty((h, w, dmax), dtype=torch.int16, device="cuda")
    cR = torch.empty_like(cL)
    S = torch.empty((h, w, dmax), dtype=torch.int32, device="cuda")
    B.bsm_cost_volumes(c, BL, PL, BR, PR, w, h, dmax, wL, wR, cL, cR)
    B.bsm_sgm(c, cL, w, h, dmax, P1, P2, paths, S, sL)
    B.bsm_sgm(c, cR, w, h, dmax, P1, P2, paths, S, sR)
    B.bsm_refine(c, dl, 3 * w, sL, sR, w, h, dmax, out)
    torch.cuda.synchronize()
    dirs = orc.SGM_DIRS4 if paths == 4 else orc.SGM_DIRS8
    ref = orc.pipeline(l, r, pairs, dmax, win=win, R=6, sgm_params=(P1, P2, dirs))
    assert (sL.cpu().numpy() == ref["dL"]).all()
    assert (sR.cpu().numpy() == ref["dR"]).all()
    assert (out.cpu().numpy() == ref["disp"]).all()
    B.bsm_destroy(c)


def test_sgm_argument_errors(B, ctx):
    C = torch.zeros((4, 4, 8), dtype=torch.int16, device="cuda")
    S = torch.zeros((4, 4, 8), dtype=torch.int32, device="cuda")
    d = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    for P1, P2, paths in ((5, 4, 4), (-1, 4, 4), (1, 70000, 4), (1, 4, 6), (1, 4, 0)):
        with pytest.raises(B.BsmError) as e:
            B.bsm_sgm(ctx, C, 4, 4, 8, P1, P2, paths, S, d)
        assert e.value.status == B.BSM_ERR_INVALID_ARG
    with pytest.raises(B.BsmError):
        B.bsm_sgm(ctx, C, 4, 4, 300, 1, 4, 4, S, d)  # dmax above the context's
    with pytest.raises(B.BsmError):
        B.bsm_sgm(ctx, None, 4, 4, 8, 1, 4, 4, S, d)
