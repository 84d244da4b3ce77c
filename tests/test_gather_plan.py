"""The warp-per-pixel describe kernel's gather plan (host logic, no GPU).

Lane l of the kernel reads the two samples of pair 32 j + l (Eq. 2-3, 5) for descriptor word j, one load
per word and sample. The kernel keeps copies of its colour-plane tile at different shared-memory banks and
the host assigns each sample a copy. What must hold, checked here from the plan's own outputs: every
offset is its copy's base plus dy * pitch + dx of the right sample; the copies do not overlap; the reported
wavefronts of every load are the bank-conflict degree of its 32 addresses, recomputed by brute force; and
more copies never give more wavefronts than one copy. The bit-exactness of the descriptors the plan reads
is tested on the GPU against the oracle.
"""
import numpy as np
import pytest

from paper_1402_2020_gb300 import bsm, synth

ROWS = 4  # rows of the describe kernel's CTA tile (plus the halo above and below)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1402_2020_gb300 import build

    build.build()


def brute_wavefronts(addrs):
    """Distinct addresses in the fullest of the 32 four-byte banks."""
    per_bank = {}
    for a in set(int(v) for v in addrs):
        per_bank.setdefault(a % 32, set()).add(a)
    return max(len(v) for v in per_bank.values())


def check_plan(pairs, copies):
    n = pairs.shape[0]
    plan = bsm.bsm_describe_gather_plan(pairs, copies)
    halo = int(np.abs(pairs.astype(int)).max())
    tp = plan["pitch"]
    assert tp == 32 + 2 * halo
    used, base = plan["copies"], plan["copy_base"]
    assert 1 <= used <= copies and base[0] == 0
    tile_words = (ROWS + 2 * halo) * tp
    assert all(base[c + 1] - base[c] >= tile_words for c in range(used - 1)), "copies overlap"
    offs = plan["offsets"]
    for i in range(n):
        for s in range(2):
            dx, dy = int(pairs[i, 2 * s]), int(pairs[i, 2 * s + 1])
            assert offs[i, s] - dy * tp - dx in set(int(b) for b in base), (i, s)
    # every load's wavefronts from its 32 addresses (the centre pixel's own address is common to the lanes)
    for ld in range(2 * (n // 32)):
        j, s = divmod(ld, 2)
        assert plan["wavefronts"][ld] == brute_wavefronts(offs[32 * j: 32 * j + 32, s]), ld
    return plan


@pytest.mark.parametrize("n,S,seed", [(256, 31, 11), (256, 31, 1), (128, 31, 3), (64, 15, 5), (256, 9, 7), (32, 31, 2)])
def test_plan_offsets_and_wavefronts(n, S, seed):
    pairs = synth.pair_table(n, S, seed=seed)
    one = check_plan(pairs, 1)
    # one copy: the plain tile offsets
    tp = one["pitch"]
    expect = np.stack([pairs[:, 1].astype(int) * tp + pairs[:, 0], pairs[:, 3].astype(int) * tp + pairs[:, 2]], 1)
    assert np.array_equal(one["offsets"], expect)
    # copy 0 is among every sample's choices, so no load can get worse than with one copy
    for c in (2, 3, 4):
        p = check_plan(pairs, c)
        assert np.all(p["wavefronts"] <= one["wavefronts"])


def test_four_copies_remove_most_conflicts():
    """At n = 256, S = 31 (the paper's setting) one tile gives about 3.3 wavefronts per load; four copies
    bring every load to at most 2 and the mean below 1.25."""
    pairs = synth.pair_table(256, 31, seed=11)
    one = bsm.bsm_describe_gather_plan(pairs, 1)["wavefronts"]
    four = bsm.bsm_describe_gather_plan(pairs, 4)
    assert four["copies"] == 4
    assert one.mean() > 2.5
    assert four["wavefronts"].max() <= 2 and four["wavefronts"].mean() < 1.25


def test_large_window_takes_fewer_copies():
    """A pair window of 63 pixels (halo 31) makes a 94 x 66 tile: four copies would pass 64 KB."""
    pairs = synth.pair_table(256, 63, seed=4)
    pairs[0, 0] = 31  # the largest offset the library takes
    p = check_plan(pairs, 4)
    assert p["copies"] < 4


def test_plan_rejects_bad_arguments():
    pairs = synth.pair_table(256, 31, seed=11)
    for n, c in [(256, 0), (256, 5)]:
        with pytest.raises(bsm.BsmError):
            bsm.bsm_describe_gather_plan(pairs[:n], c)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_describe_gather_plan(pairs[:48], 4)  # not a multiple of 32
    big = np.zeros((512, 4), np.int8)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_describe_gather_plan(big, 4)  # beyond the short-descriptor kernels
    far = pairs.copy()
    far[3, 2] = 40
    with pytest.raises(bsm.BsmError):
        bsm.bsm_describe_gather_plan(far, 4)  # offset beyond 31
