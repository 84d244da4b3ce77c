"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Every check here is independent of the oracle's own code path: published colour anchors, closed
forms, invariants, special cases that reduce to a library routine (numpy bit counts, scipy box
sums, numpy argmin) and hand-built cases whose answer follows from the equation by hand.
"""
import math
import sys
import os

import numpy as np
import pytest

from paper_1402_2020_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gray_image(values):
    v = np.asarray(values, dtype=np.uint8)
    return np.repeat(v[:, :, None], 3, axis=2)


def bitcount(a):
    return np.bitwise_count(np.asarray(a, dtype=np.uint32)).astype(np.int64)


# ---------------------------------------------------------------- intensity and colour (Eq. 3, Eq. 5)

def test_intensity_gray_identity_and_weights(orc):
    for v in range(256):
        assert orc.intensity(v, v, v) == v
    # luma weights 77/256, 150/256, 29/256 with rounding
    assert orc.intensity(255, 0, 0) == 77
    assert orc.intensity(0, 255, 0) == 149
    assert orc.intensity(0, 0, 255) == 29
    assert orc.intensity(255, 255, 255) == 255


def test_lab_published_anchors(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lab_anchors.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 9
    for r in rows:
        R, G, B, L, a, b = map(int, r)
        assert orc.lab(R, G, B) == (L, a, b), (R, G, B)


def test_lab_gray_axis(orc):
    prev = -1
    for v in range(256):
        L, a, b = orc.lab(v, v, v)
        assert a == 0 and b == 0
        assert L >= prev
        prev = L
    assert orc.lab(255, 255, 255)[0] == 100


def test_lab_ranges(orc):
    rng = np.random.default_rng(0)
    for R, G, B in rng.integers(0, 256, size=(2000, 3)):
        L, a, b = orc.lab(R, G, B)
        assert 0 <= L <= 100 and -128 <= a <= 127 and -128 <= b <= 127


# ---------------------------------------------------------------- descriptor B (Eq. 2-3)

def test_flat_image_descriptor_and_mask(orc):
    img = np.full((9, 11, 3), 77, np.uint8)
    pairs = synth.pair_table(64, 31, seed=1)
    B, Phi = orc.describe(img, pairs)
    assert not B.any()  # Eq. 3: I(p) > I(q) never holds
    assert (Phi == 0xFFFFFFFF).all()  # all w = 0 = T, so every delta is 1


def test_bit_order_is_pair_index(orc):
    # pair i compares (x+1, y) with (x, y) on a left-to-right ramp, every other pair is (x, x)
    n = 64
    img = gray_image(np.tile(np.arange(0, 200, 10), (5, 1)))
    for i in (0, 5, 31, 32, 63):
        pairs = np.zeros((n, 4), np.int8)
        pairs[i] = (1, 0, 0, 0)
        B, _ = orc.describe(img, pairs, k=16)
        x = 5
        expect = np.zeros(2, np.uint32)
        expect[i // 32] = np.uint32(1) << np.uint32(i % 32)  # weight 2^(i-1) for the 1-based pair i+1
        assert (B[2, x] == expect).all(), i
        # at the right border p is clamped onto x itself: I(p) = I(q), so tau = 0
        assert not B[2, img.shape[1] - 1].any()


def test_descriptor_monotone_invariance(orc):
    # Eq. 3 only compares intensities, so a strictly increasing map of a gray image keeps B.
    rng = np.random.default_rng(3)
    v = rng.integers(0, 256, size=(16, 20))
    pairs = synth.pair_table(128, 15, seed=4)
    B1, _ = orc.describe(gray_image(v), pairs)
    uniq = np.unique(v)
    new_vals = np.linspace(3, 250, len(uniq)).round().astype(np.int64)
    assert (np.diff(new_vals) > 0).all()
    mapped = new_vals[np.searchsorted(uniq, v)]
    B2, _ = orc.describe(gray_image(mapped), pairs)
    assert (B1 == B2).all()


def test_swapping_pair_inverts_bits(orc):
    rng = np.random.default_rng(5)
    v = rng.integers(0, 256, size=(12, 14))
    img = gray_image(v)
    pairs = synth.pair_table(32, 9, seed=6)
    swapped = pairs[:, [2, 3, 0, 1]].copy()
    B1, _ = orc.describe(img, pairs)
    B2, _ = orc.describe(img, swapped)
    h, w = v.shape
    for y in range(h):
        for x in range(w):
            for i in range(32):
                px = min(max(x + pairs[i, 0], 0), w - 1)
                py = min(max(y + pairs[i, 1], 0), h - 1)
                qx = min(max(x + pairs[i, 2], 0), w - 1)
                qy = min(max(y + pairs[i, 3], 0), h - 1)
                b1 = (int(B1[y, x, 0]) >> i) & 1
                b2 = (int(B2[y, x, 0]) >> i) & 1
                if v[py, px] == v[qy, qx]:
                    assert b1 == 0 and b2 == 0
                else:
                    assert b1 + b2 == 1


# ---------------------------------------------------------------- mask Phi (Eq. 5-7)

def test_mask_keeps_exactly_the_k_nearest_colours(orc):
    # q_i is the centre itself, so w_i = SAD(x, p_i); p_i walks along a gray ramp whose CIELAB
    # lightness strictly increases, so the k pairs with the smallest |offset| win (no ties).
    ramp = np.arange(0, 31 * 8, 8)
    img = gray_image(np.tile(ramp, (3, 1)))
    x = 15
    offsets = [o for o in range(-15, 16) if o != 0][:30] + [0, 0]
    pairs = np.array([(o, 0, 0, 0) for o in offsets], np.int8)
    Ls = [orc.lab(int(v), int(v), int(v))[0] for v in ramp]
    w_i = [abs(Ls[x + o] - Ls[x]) for o in offsets]
    k = 9
    T = sorted(w_i)[k - 1]
    _, Phi = orc.describe(img, pairs, k=k)
    got = [(int(Phi[1, x, 0]) >> i) & 1 for i in range(32)]
    assert got == [int(wv <= T) for wv in w_i]
    assert sum(got) >= k


def test_mask_weight_uses_both_pair_points(orc):
    # p_i is the centre and q_i walks the ramp: w_i = max(SAD(x, x), SAD(x, q_i)) = SAD(x, q_i) (Eq. 5),
    # so the mask keeps the k pairs whose q lies nearest in lightness.
    ramp = np.arange(0, 31 * 8, 8)
    img = gray_image(np.tile(ramp, (3, 1)))
    x = 15
    offsets = list(range(1, 16)) + list(range(-15, 0)) + [0, 0]
    pairs = np.array([(0, 0, o, 0) for o in offsets], np.int8)
    Ls = [orc.lab(int(v), int(v), int(v))[0] for v in ramp]
    w_i = [abs(Ls[x + o] - Ls[x]) for o in offsets]
    k = 11
    T = sorted(w_i)[k - 1]
    _, Phi = orc.describe(img, pairs, k=k)
    assert [(int(Phi[1, x, 0]) >> i) & 1 for i in range(32)] == [int(wv <= T) for wv in w_i]


def test_mask_exactly_k_bits_when_weights_are_distinct(orc):
    # weights strictly increase with the offset (one-sided ramp, q at the centre): T is the k-th
    # smallest of distinct values, so exactly k bits are set and they are the first k pairs.
    ramp = np.arange(0, 64 * 4, 4)[:64]
    img = gray_image(np.tile(ramp, (3, 1)))
    x = 1
    pairs = np.array([(min(1 + i, 31), 0, 0, 0) for i in range(32)], np.int8)
    w_i = [orc.lab(*(3 * [int(ramp[x + 1 + i])]))[0] - orc.lab(*(3 * [int(ramp[x])]))[0] for i in range(31)]
    assert all(b > a for a, b in zip(w_i, w_i[1:]))
    for k in (1, 8, 20):
        _, Phi = orc.describe(img, pairs, k=k)
        word = int(Phi[1, x, 0])
        assert bin(word).count("1") == k
        assert word == (1 << k) - 1


def test_mask_popcount_at_least_k(orc):
    l, _, _ = synth.stereo_pair(40, 30, 16, seed=7)
    pairs = synth.pair_table(256, 31, seed=8)
    for k in (1, 17, 64, 200, 256):
        _, Phi = orc.describe(l, pairs, k=k)
        pc = bitcount(Phi).sum(axis=2)
        assert (pc >= k).all()
        if k == 256:
            assert (pc == 256).all()


def test_mask_quarter_rank_definition(orc):
    # T is the k-th smallest weight: count(w <= T) >= k and count(w < T) < k. With pairs whose
    # q is the centre, w_i = SAD(x, p_i) can be listed by hand from the pinned colour conversion.
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, size=(9, 9, 3)).astype(np.uint8)
    offs = rng.integers(-4, 5, size=(64, 2))
    pairs = np.zeros((64, 4), np.int8)
    pairs[:, 0:2] = offs
    x = y = 4
    lab = {}
    for yy in range(9):
        for xx in range(9):
            lab[(xx, yy)] = orc.lab(*img[yy, xx])
    c = lab[(x, y)]
    w_i = [sum(abs(a - b) for a, b in zip(lab[(x + int(dx), y + int(dy))], c)) for dx, dy in offs]
    _, Phi = orc.describe(img, pairs)  # k = n/4 = 16
    bits = [(int(Phi[y, x, i // 32]) >> (i % 32)) & 1 for i in range(64)]
    T = max(wv for wv, bt in zip(w_i, bits) if bt)
    assert all((wv <= T) == bool(bt) for wv, bt in zip(w_i, bits))
    assert sum(wv <= T for wv in w_i) >= 16
    assert sum(wv < T for wv in w_i) < 16


# ---------------------------------------------------------------- cost (Eq. 4, Eq. 8)

def test_cost_precedence_and_reference_mask(orc):
    # one-word planes, 2 x 1 pixels: (B XOR B') AND Phi, with Phi from the reference pixel only
    Bref = np.array([[[0b1011], [0b0001]]], np.uint32)
    Phiref = np.array([[[0b0110], [0b1111]]], np.uint32)
    Both = np.array([[[0b0000], [0b1110]]], np.uint32)
    # x=1, d=1, left reference: match x-d=0 -> (0001 ^ 0000) & 1111 = 1 -> 1
    assert orc.cost_at(Bref, Phiref, Both, 1, 0, 1, 0) == 1
    # x=0, d=0: (1011 ^ 0000) & 0110 = 0010 -> 1 (B ^ (B' & Phi) would give 3)
    assert orc.cost_at(Bref, Phiref, Both, 0, 0, 0, 0) == 1
    # x=0, d=1, right reference: match x+d=1 -> (1011 ^ 1110) & 0110 = 0100 -> 1
    assert orc.cost_at(Bref, Phiref, Both, 0, 0, 1, 1) == 1
    # match outside the image costs n = 32
    assert orc.cost_at(Bref, Phiref, Both, 0, 0, 1, 0) == 32
    assert orc.cost_at(Bref, Phiref, Both, 1, 0, 1, 1) == 32


def test_cost_is_hamming_with_full_mask(orc):
    rng = np.random.default_rng(11)
    h, w, nw, dmax = 6, 13, 8, 9
    Bref = rng.integers(0, 2**32, size=(h, w, nw), dtype=np.uint32)
    Both = rng.integers(0, 2**32, size=(h, w, nw), dtype=np.uint32)
    Phi = np.full((h, w, nw), 0xFFFFFFFF, np.uint32)
    A = orc.aggregate(Bref, Phi, Both, dmax, 1, 0)
    for d in range(dmax):
        for x in range(w):
            if x - d >= 0:
                ham = bitcount(Bref[:, x] ^ Both[:, x - d]).sum(axis=1)  # Eq. 4
                assert (A[:, x, d] == ham).all()
            else:
                assert (A[:, x, d] == 256).all()


def test_cost_bounds_and_zero_for_identical(orc):
    l, r, _ = synth.stereo_pair(48, 20, 12, seed=12)
    pairs = synth.pair_table(64, 31, seed=13)
    BL, PhiL = orc.describe(l, pairs)
    BR, _ = orc.describe(r, pairs)
    A = orc.aggregate(BL, PhiL, BR, 12, 1, 0)
    pc = bitcount(PhiL).sum(axis=2)
    for d in range(12):
        inimg = np.arange(48) >= d
        assert (A[:, inimg, d] <= pc[:, inimg]).all()
        assert (A[:, ~inimg, d] == 64).all()
    A0 = orc.aggregate(BL, PhiL, BL, 12, 1, 0)
    assert (A0[:, :, 0] == 0).all()


def test_aggregation_is_zero_padded_box_sum(orc):
    from scipy.signal import convolve2d

    l, r, _ = synth.stereo_pair(30, 17, 10, seed=14)
    pairs = synth.pair_table(64, 31, seed=15)
    BL, PhiL = orc.describe(l, pairs)
    BR, PhiR = orc.describe(r, pairs)
    for direction, (Br, Pr, Bo) in enumerate(((BL, PhiL, BR), (BR, PhiR, BL))):
        C = orc.aggregate(Br, Pr, Bo, 10, 1, direction)
        for win in (3, 5):
            A = orc.aggregate(Br, Pr, Bo, 10, win, direction)
            for d in range(10):
                ref = convolve2d(C[:, :, d].astype(np.float64), np.ones((win, win)), mode="same",
                                 boundary="fill", fillvalue=0)
                assert (A[:, :, d] == ref.astype(np.int64)).all()


# ---------------------------------------------------------------- mask ablations (Eq. 4; both views' masks)

def test_both_masks_brute_force_and_symmetry(orc):
    # popcount((b ^ o) & m & mo) written bit by bit on tiny planes, the matched pixel's mask taken at x_d
    rng = np.random.default_rng(41)
    h, w, nw = 3, 7, 1
    BL, BR, PL, PR = (rng.integers(0, 2**32, size=(h, w, nw), dtype=np.uint32) for _ in range(4))
    for y in range(h):
        for x in range(w):
            for d in range(4):
                xd = x - d
                if xd < 0:
                    assert orc.cost_at(BL, PL, BR, x, y, d, 0, Phioth=PR) == 32
                    continue
                want = sum(1 for i in range(32)
                           if ((int(BL[y, x, 0]) >> i) & 1) != ((int(BR[y, xd, 0]) >> i) & 1)
                           and (int(PL[y, x, 0]) >> i) & 1 and (int(PR[y, xd, 0]) >> i) & 1)
                assert orc.cost_at(BL, PL, BR, x, y, d, 0, Phioth=PR) == want
                # with both masks the cost no longer depends on which view is the reference
                assert orc.cost_at(BR, PR, BL, xd, y, d, 1, Phioth=PL) == want


def test_both_masks_reduce_to_eq8_and_bound_it(orc):
    l, r, _ = synth.stereo_pair(40, 12, 10, seed=42)
    pairs = synth.pair_table(64, 31, seed=43)
    BL, PhiL = orc.describe(l, pairs)
    BR, PhiR = orc.describe(r, pairs)
    ones = np.full_like(PhiR, 0xFFFFFFFF)
    A8 = orc.aggregate(BL, PhiL, BR, 10, 3, 0)
    assert (orc.aggregate(BL, PhiL, BR, 10, 3, 0, Phioth=ones) == A8).all()
    A2 = orc.aggregate(BL, PhiL, BR, 10, 3, 0, Phioth=PhiR)
    assert (A2 <= A8).all() and (A2 < A8).any()


def test_no_mask_pipeline_is_eq4(orc):
    # MASK_NONE: Phi is all ones, so the WTA runs on the plain Hamming distance of Eq. 4
    l, r, _ = synth.stereo_pair(36, 14, 9, seed=44)
    pairs = synth.pair_table(64, 31, seed=45)
    ref = orc.pipeline(l, r, pairs, 9, win=1, R=3, mask_mode=orc.MASK_NONE)
    assert (ref["PhiL"] == 0xFFFFFFFF).all() and (ref["PhiR"] == 0xFFFFFFFF).all()
    BL, BR = ref["BL"], ref["BR"]
    for x in range(36):
        ham = np.stack([bitcount(BL[:, x] ^ BR[:, x - d]).sum(axis=1) if x - d >= 0 else np.full(14, 64)
                        for d in range(9)], axis=1)
        assert (ref["dL"][:, x] == np.argmin(ham, axis=1)).all()
    # describe with k = n sets every mask bit: the same maps
    kn = orc.pipeline(l, r, pairs, 9, win=1, R=3, k=64)
    assert (kn["PhiL"] == 0xFFFFFFFF).all()
    assert (kn["dL"] == ref["dL"]).all() and (kn["disp"] == ref["disp"]).all()


# ---------------------------------------------------------------- WTA (Eq. 1)

def test_wta_is_first_argmin(orc):
    l, r, _ = synth.stereo_pair(26, 14, 11, seed=16)
    pairs = synth.pair_table(64, 31, seed=17)
    BL, PhiL = orc.describe(l, pairs)
    BR, PhiR = orc.describe(r, pairs)
    for direction, (Br, Pr, Bo) in enumerate(((BL, PhiL, BR), (BR, PhiR, BL))):
        for win in (1, 3):
            A = orc.aggregate(Br, Pr, Bo, 11, win, direction)
            disp = orc.wta(Br, Pr, Bo, 11, win, direction)
            assert (disp == np.argmin(A, axis=2)).all()


@pytest.mark.parametrize("shift", [0, 3, 7])
def test_constant_shift_recovered(orc, shift):
    w, h, dmax = 60, 24, 10
    l, r = synth.shifted_pair(w, h, shift, seed=18 + shift)
    pairs = synth.pair_table(256, 31, seed=19)
    BL, PhiL = orc.describe(l, pairs)
    BR, PhiR = orc.describe(r, pairs)
    for win in (1, 5):
        dL = orc.wta(BL, PhiL, BR, dmax, win, 0)
        dR = orc.wta(BR, PhiR, BL, dmax, win, 1)
        m = 15 + win // 2  # sampling half-window plus aggregation radius
        ys = slice(m, h - m)
        # left reference: x - shift must keep the right window away from the border clamp
        assert (dL[ys, m + shift : w - m] == shift).all()
        assert (dR[ys, m : w - m - shift] == shift).all()
        valid = orc.lr_check(dL, dR, 1)
        assert valid[ys, m + shift : w - m].all()


# ---------------------------------------------------------------- left/right check

def test_lr_check_hand_cases(orc):
    dL = np.array([[0, 1, 2, 5, 1]], np.int32)
    dR = np.array([[0, 3, 2, 0, 0]], np.int32)
    # x=0: d=0 -> dR[0]=0 ok; x=1: d=1 -> dR[0]=0, |1-0|=1 ok; x=2: d=2 -> dR[0]=0, |2|>1 no;
    # x=3: d=5 -> x-d<0 no; x=4: d=1 -> dR[3]=0, ok
    assert orc.lr_check(dL, dR, 1).tolist() == [[1, 1, 0, 0, 1]]
    assert orc.lr_check(dL, dR, 0).tolist() == [[1, 0, 0, 0, 0]]


# ---------------------------------------------------------------- refinement (Eq. 9-10)

def test_vote_tables_closed_form(orc):
    Ec, Es = orc.vote_tables(9.0, 16.0, 15)
    assert Ec[0] == 32768 and Es[0] == 32768
    assert Ec[9] == round(32768 / math.e) == 12055  # exp(-9/9)
    assert Es[256] == 12055  # exp(-sqrt(256)/16)
    assert Ec[18] == round(32768 / math.e ** 2)
    assert (np.diff(Ec.astype(np.int64)) <= 0).all() and (np.diff(Es.astype(np.int64)) <= 0).all()
    assert Ec[-1] == 0


def test_refine_all_valid_is_identity(orc):
    l, _, _ = synth.stereo_pair(20, 12, 8, seed=20)
    dL = np.random.default_rng(21).integers(0, 8, size=(12, 20)).astype(np.int32)
    out = orc.refine(l, dL, np.ones((12, 20), np.uint8), 8)
    assert (out == dL).all()


def test_refine_single_voter(orc):
    img = np.full((21, 21, 3), 90, np.uint8)
    dL = np.zeros((21, 21), np.int32)
    valid = np.zeros((21, 21), np.uint8)
    valid[12, 13] = 1
    dL[12, 13] = 6
    out = orc.refine(img, dL, valid, 8, R=15)
    # every pixel sees the one valid pixel within R=15 except where the window misses it
    assert (out[valid == 0] == 6).all()


def test_refine_weighted_vote_hand_case(orc):
    # invalid centre (2,2) in a 5x5 gray image; voters: one at distance 1 with colour difference
    # c, disparity 3; two at distance 2 (same colour), disparity 5.
    img = np.full((5, 5, 3), 100, np.uint8)
    img[2, 3] = (110, 110, 110)
    L0 = orc.lab(100, 100, 100)[0]
    L1 = orc.lab(110, 110, 110)[0]
    c = abs(L1 - L0)
    dL = np.zeros((5, 5), np.int32)
    valid = np.zeros((5, 5), np.uint8)
    valid[2, 3] = 1
    dL[2, 3] = 3
    valid[2, 0] = 1
    dL[2, 0] = 5
    valid[0, 2] = 1
    dL[0, 2] = 5
    Ec, Es = orc.vote_tables(9.0, 16.0, 15)
    w3 = (int(Ec[c]) * int(Es[1])) >> 15
    w5 = 2 * ((int(Ec[0]) * int(Es[4])) >> 15)
    out = orc.refine(img, dL, valid, 8, R=15)
    assert out[2, 2] == (3 if w3 > w5 else 5)
    assert w3 != w5


def test_refine_distance_term_decides(orc):
    # Eq. 10's spatial term: a voter one pixel away with a slightly different colour (disparity 3)
    # against a voter ten pixels away with the same colour (disparity 5). Only the bilateral weight
    # with both terms makes the near voter win.
    img = np.full((1, 21, 3), 100, np.uint8)
    img[0, 11] = (110, 110, 110)
    dL = np.zeros((1, 21), np.int32)
    valid = np.zeros((1, 21), np.uint8)
    valid[0, 11], dL[0, 11] = 1, 3
    valid[0, 20], dL[0, 20] = 1, 5
    Ec, Es = orc.vote_tables(9.0, 16.0, 15)
    c = abs(orc.lab(110, 110, 110)[0] - orc.lab(100, 100, 100)[0])
    near = (int(Ec[c]) * int(Es[1])) >> 15
    far = (int(Ec[0]) * int(Es[100])) >> 15
    assert near > far and int(Ec[c]) < int(Ec[0])  # the case separates the two readings
    out = orc.refine(img, dL, valid, 8, R=15)
    assert out[0, 10] == 3


def test_refine_tie_goes_to_smallest_disparity(orc):
    # two voters with identical colour and distance vote for disparities 6 and 2 with equal weight
    img = np.full((1, 11, 3), 80, np.uint8)
    dL = np.zeros((1, 11), np.int32)
    valid = np.zeros((1, 11), np.uint8)
    valid[0, 3], dL[0, 3] = 1, 6
    valid[0, 7], dL[0, 7] = 1, 2
    out = orc.refine(img, dL, valid, 8, R=5)
    assert out[0, 5] == 2


def test_refine_fallback_on_the_row(orc):
    img = np.full((1, 60, 3), 50, np.uint8)
    dL = np.zeros((1, 60), np.int32)
    valid = np.zeros((1, 60), np.uint8)
    valid[0, 0] = 1
    dL[0, 0] = 4
    valid[0, 59] = 1
    dL[0, 59] = 2
    out = orc.refine(img, dL, valid, 8, R=3)
    assert out[0, 1] == 4  # window reaches x=0 only
    assert out[0, 58] == 2
    assert out[0, 30] == 2  # no voter within R: min of the nearest valid left (4) and right (2)
    valid[0, 59] = 0
    out = orc.refine(img, dL, valid, 8, R=3)
    assert out[0, 30] == 4
    out = orc.refine(img, dL, np.zeros_like(valid), 8, R=3)
    assert (out == 0).all()


def test_pipeline_tracks_ground_truth(orc):
    l, r, gt = synth.stereo_pair(96, 64, 16, seed=22)
    pairs = synth.pair_table(256, 31, seed=23)
    res = orc.pipeline(l, r, pairs, 16, win=5)
    inner = (slice(16, -16), slice(32, -16))
    bad = np.abs(res["disp"][inner] - gt[inner]) > 1
    assert bad.mean() < 0.35, bad.mean()


# ---------------------------------------------------------------- semi-global aggregation (reading R10)

def test_sgm_without_penalties_is_a_sum_of_costs(orc):
    C = np.random.default_rng(51).integers(0, 60, size=(6, 9, 7)).astype(np.uint16)
    for dirs in (orc.SGM_DIRS4, orc.SGM_DIRS8):
        S, disp = orc.sgm(C, 0, 0, dirs)
        assert (S == len(dirs) * C.astype(np.uint32)).all()
        assert (disp == np.argmin(C, axis=2)).all()


def _viterbi_brute_force(C, chain, P1, P2):
    """Minimum over every labelling of the chain of sum C + penalties, per label of the last pixel."""
    import itertools

    dmax = C.shape[2]
    best = np.full(dmax, np.iinfo(np.int64).max)
    for labels in itertools.product(range(dmax), repeat=len(chain)):
        cost = sum(int(C[y, x, d]) for (x, y), d in zip(chain, labels))
        for a, b in zip(labels, labels[1:]):
            cost += 0 if a == b else (P1 if abs(a - b) == 1 else P2)
        best[labels[-1]] = min(best[labels[-1]], cost)
    return best


@pytest.mark.parametrize("direction", [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_sgm_path_cost_is_the_best_labelling(orc, direction):
    # One direction: L(p, .) is, up to a constant, the cheapest labelling of the path that ends at p.
    rng = np.random.default_rng(52)
    h, w, dmax, P1, P2 = 4, 5, 3, 2, 5
    C = rng.integers(0, 9, size=(h, w, dmax)).astype(np.uint16)
    S, _ = orc.sgm(C, P1, P2, (direction,))
    dx, dy = direction
    for y in range(h):
        for x in range(w):
            chain = [(x, y)]
            while 0 <= chain[0][0] - dx < w and 0 <= chain[0][1] - dy < h:
                chain.insert(0, (chain[0][0] - dx, chain[0][1] - dy))
            V = _viterbi_brute_force(C, chain, P1, P2)
            L = S[y, x].astype(np.int64)
            assert (L - L.min() == V - V.min()).all(), (x, y)


def test_sgm_transpose_and_mirror(orc):
    C = np.random.default_rng(53).integers(0, 40, size=(7, 10, 6)).astype(np.uint16)
    for dirs in (orc.SGM_DIRS4, orc.SGM_DIRS8):
        S, d = orc.sgm(C, 3, 11, dirs)
        St, dt = orc.sgm(np.ascontiguousarray(C.transpose(1, 0, 2)), 3, 11, dirs)
        assert (St.transpose(1, 0, 2) == S).all() and (dt.T == d).all()
        Sm, dm = orc.sgm(np.ascontiguousarray(C[:, ::-1]), 3, 11, dirs)
        assert (Sm[:, ::-1] == S).all() and (dm[:, ::-1] == d).all()


def test_sgm_smooths_an_outlier(orc):
    # a constant disparity 2 everywhere except one pixel whose cost prefers 5: the penalties pull it back
    h, w, dmax = 9, 9, 8
    C = np.full((h, w, dmax), 20, np.uint16)
    C[:, :, 2] = 10
    C[4, 4, :] = 20
    C[4, 4, 5] = 8
    _, d0 = orc.sgm(C, 0, 0)
    assert d0[4, 4] == 5
    _, d1 = orc.sgm(C, 4, 30, orc.SGM_DIRS8)
    assert (d1 == 2).all()
