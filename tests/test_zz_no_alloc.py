"""bsm_describe_noalloc against bsm_describe (needs a GPU).

The no-allocation variant serves callers that cannot call cudaMalloc (stream capture, a device
budget fixed up front, loops that cannot take an allocation's device synchronisation). It must give
exactly the descriptor and mask planes that bsm_describe gives, call after call, although every
call reuses the same fixed scratch array. This file is collected last on purpose.
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


def _describe(B, fn, ctx, img, nw, pad=0):
    """One call of fn on img, stored with a row pitch of 3 w + pad bytes."""
    h, w, _ = img.shape
    pitch = 3 * w + pad
    buf = np.zeros((h, pitch), np.uint8)
    buf[:, :3 * w] = img.reshape(h, 3 * w)
    d = torch.from_numpy(buf).cuda()
    Bp = torch.full((h, w, nw), -1, dtype=torch.int32, device="cuda")
    Pp = torch.full((h, w, nw), -1, dtype=torch.int32, device="cuda")
    fn(ctx, d, w, h, pitch, Bp, Pp)
    torch.cuda.synchronize()
    return Bp.cpu().numpy(), Pp.cpu().numpy()


# the thread-per-pixel describe (n = 64), the warp-per-pixel one (n = 256), the long-descriptor one
# (n = 1024); and a padded row pitch
@pytest.mark.parametrize("n,pad", [(64, 0), (256, 0), (1024, 0), (256, 13)])
def test_noalloc_matches_describe_on_consecutive_calls(B, n, pad):
    pairs = synth.pair_table(n, 31, seed=900 + n)
    params = B.make_params(pairs, dmax=64)
    ctx = B.bsm_create(params)
    try:
        # two calls in a row on different images (the second smaller, so stale words of the first
        # remain in the shared scratch), then one more on the first image
        imgs = [synth.stereo_pair(300, 170, 64, seed=901)[0], synth.stereo_pair(97, 45, 64, seed=902)[1]]
        imgs.append(imgs[0])
        for img in imgs:
            nb, npf = _describe(B, B.bsm_describe_noalloc, ctx, img, n // 32, pad)
            rb, rpf = _describe(B, B.bsm_describe, ctx, img, n // 32, pad)
            assert (nb == rb).all()
            assert (npf == rpf).all()
        assert B.bsm_last_error(ctx) == B.BSM_OK
    finally:
        B.bsm_destroy(ctx)


def test_noalloc_rejects_images_beyond_its_scratch(B):
    pairs = synth.pair_table(64, 31, seed=903)
    ctx = B.bsm_create(B.make_params(pairs, dmax=16))
    try:
        x = torch.zeros(64, dtype=torch.int32, device="cuda")
        w, h = 4096, 1025  # 4096 * 1025 > 2^22
        assert w * h > B.BSM_NOALLOC_MAX_PIXELS
        with pytest.raises(B.BsmError) as e:
            B.bsm_describe_noalloc(ctx, x, w, h, 3 * w, x, x)
        assert e.value.status == B.BSM_ERR_INVALID_ARG
    finally:
        B.bsm_destroy(ctx)
