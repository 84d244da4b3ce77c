"""The integer and fp16 identities the describe kernels rely on, checked exhaustively on the host (no GPU).

These are facts about the encodings, not about the oracle: the fp16 form of the Eq. 5 weights, the
per-step count of the T bisection (Eq. 6) from saturating fp16 subtracts, and the order-statistic bracket
that starts the bisection."""
import numpy as np
import pytest

M32 = (1 << 32) - 1


def half_bits(x):
    return int(np.array(x, dtype=np.float16).view(np.uint16))


def test_biased_weight_is_the_fp16_of_1024_plus_w():
    # every weight is a 3-channel SAD of 8-bit values (<= 765); 0x6400 + w must be the fp16 pattern of
    # 1024 + w, exactly, and the pattern order must be the order of w
    for w in range(0, 1024):
        assert 0x6400 + w == half_bits(1024.0 + w)
    pats = np.arange(0x6400, 0x6400 + 1024, dtype=np.uint16).view(np.float16).astype(np.float64)
    assert (np.diff(pats) == 1.0).all()


@pytest.mark.parametrize("nh", [1, 2, 4])
def test_saturating_count(nh):
    # One step of the T bisection. Per fp16x2 register of weights (1024 + w), a saturating subtract from
    # 1024 + t + 1 gives 1 in each half where w <= t and 0 elsewhere; the lane adds its nh results to a
    # bias of 1024, so each half's bits are 0x6400 + that half's count; the warp's 32 lane sums added as
    # 32-bit integers, minus 32 * 0x6400 * (1 + 2^16) mod 2^32, leave the low halves' count in the low 16
    # bits and the high halves' count above. Every value is an integer below 2048: exact in fp16.
    assert (32 * 0x6400 * (1 + (1 << 16))) & M32 == 0x800C8000
    rng = np.random.default_rng(nh)
    for _ in range(300):
        t = int(rng.integers(0, 766))
        w = rng.integers(0, 766, size=(32, nh, 2))  # lanes x registers x halves
        c = np.clip(np.float16(1024 + t + 1) - (1024 + w).astype(np.float16), np.float16(0), np.float16(1))
        assert (c == (w <= t)).all()
        s = np.full((32, 2), 1024, dtype=np.float16)
        for m in range(nh):
            s = (s + c[:, m, :]).astype(np.float16)
        bits = s.view(np.uint16).astype(np.uint64)
        assert (bits - 0x6400 == (w <= t).sum(axis=1)).all()
        words = bits[:, 0] | (bits[:, 1] << 16)
        tot = (int(words.sum()) - 0x800C8000) & M32
        assert tot & 0xFFFF == int((w[:, :, 0] <= t).sum())
        assert tot >> 16 == int((w[:, :, 1] <= t).sum())


@pytest.mark.parametrize("nw,k", [(2, 16), (4, 32), (8, 64), (8, 33), (8, 32), (4, 1), (8, 256)])
def test_order_statistic_bracket(nw, k):
    # lane l holds the weights of pairs l, l + 32, ...; with a = ceil(k / 32) - 1 and s_a(l) the lane's
    # a-th smallest (0-based), the k-th smallest weight T lies in [min_l s_a(l), max_l s_a(l)]
    rng = np.random.default_rng(nw * 1000 + k)
    a = (k + 31) // 32 - 1
    for trial in range(300):
        hi = [4, 30, 765][trial % 3]
        w = rng.integers(0, hi + 1, size=32 * nw)
        T = np.sort(w)[k - 1]
        lanes = w.reshape(nw, 32).T  # [lane][j] = pair 32 j + lane
        s = np.sort(lanes, axis=1)[:, min(a, nw - 1)]
        assert s.min() <= T <= s.max()


def test_bracket_statistic_from_half_pairs():
    # at nw = 8 the lane's eight weights sit in four fp16x2 registers; the kernel takes the smallest and
    # the second smallest per half with a min/max network, then the lane's smallest and second smallest
    # from the two halves (and their swapped copies)
    rng = np.random.default_rng(7)
    for _ in range(2000):
        w = rng.integers(0, 766, size=8)
        lo_half, hi_half = w[0::2], w[1::2]  # pairs 2 m (low) and 2 m + 1 (high) of register m
        def m12(v):
            a, A = min(v[0], v[1]), max(v[0], v[1])
            b, B = min(v[2], v[3]), max(v[2], v[3])
            return min(a, b), min(max(a, b), min(A, B))
        l1, l2 = m12(lo_half)
        h1, h2 = m12(hi_half)
        s0 = min(l1, h1)
        s1 = min(max(l1, h1), min(l2, h2))
        srt = np.sort(w)
        assert s0 == srt[0] and s1 == srt[1]


# ---------------------------------------------------------------- the tensor-core cost kernel's operands
# Eq. 8 as a product: with s_i = Phi_i (1 - 2 B_i) and o_i the other view's bit, the masked Hamming cost
# is popcount(Phi & B) + sum_i s_i o_i. The kernel stores o_i and s_i as E4M3 bytes; byte k of operand
# word q carries bit 8k + q of a descriptor word. The checks below restate the kernel's byte formulas
# and decode them as E4M3 values.

def e4m3(byte):
    """Value of an E4M3 byte (sign, 4 exponent bits with bias 7, 3 mantissa bits; subnormals below 2^-6)."""
    sign = -1.0 if byte & 0x80 else 1.0
    e, m = (byte >> 3) & 15, byte & 7
    assert not (e == 15 and m == 7), "NaN"
    return sign * (m / 8.0 * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7))


def b_words(o):
    """The kernel's B operand words 0..7 of one other-view word o."""
    return [o & 0x01010101, o & 0x02020202, o & 0x04040404, o & 0x08080808, o & 0x10101010, o & 0x20202020,
            o & 0x40404040, (o >> 1) & 0x40404040]


def a_words(b, m):
    """The kernel's A operand words 0..7 of one descriptor word b and mask word m."""
    sb = m & b
    P = (0x70, 0x68, 0x60, 0x58, 0x50, 0x40)
    out = [(((m & (0x01010101 << q)) * (P[q] >> q)) + ((sb & (0x01010101 << q)) * (0x80 >> q))) & M32
           for q in range(6)]
    out.append(((m >> 1) & 0x20202020) | ((sb << 1) & 0x80808080))
    out.append(((m >> 2) & 0x20202020) | (sb & 0x80808080))
    return out


def test_tc_operand_bytes_decode_to_s_and_o():
    rng = np.random.default_rng(5)
    for _ in range(300):
        b, m, o = (int(v) for v in rng.integers(0, 1 << 32, size=3, dtype=np.uint64))
        A, Bw = a_words(b, m), b_words(o)
        for q in range(8):
            for k in range(4):
                bit = 8 * k + q
                s = ((m >> bit) & 1) * (1 - 2 * ((b >> bit) & 1))
                ov = (o >> bit) & 1
                ab, bb = (A[q] >> 8 * k) & 0xFF, (Bw[q] >> 8 * k) & 0xFF
                assert e4m3(ab) * e4m3(bb) == s * ov * 0.25, (q, k, hex(ab), hex(bb))
                if ov == 0:
                    assert bb == 0
                if s == 0:
                    assert ab == 0


def test_tc_product_equals_masked_hamming_cost():
    # the 256-bit cost of Eq. 8 (reference mask) from the operand bytes: 4 * sum(a * o) + popcount(Phi & B)
    rng = np.random.default_rng(6)
    for _ in range(200):
        B = [int(v) for v in rng.integers(0, 1 << 32, size=8, dtype=np.uint64)]
        P = [int(v) for v in rng.integers(0, 1 << 32, size=8, dtype=np.uint64)]
        O = [int(v) for v in rng.integers(0, 1 << 32, size=8, dtype=np.uint64)]
        acc = 0.0
        for j in range(8):
            A, Bw = a_words(B[j], P[j]), b_words(O[j])
            for q in range(8):
                for k in range(4):
                    acc += e4m3((A[q] >> 8 * k) & 0xFF) * e4m3((Bw[q] >> 8 * k) & 0xFF)
        want = sum(bin((B[j] ^ O[j]) & P[j]).count("1") for j in range(8))
        assert 4 * acc + sum(bin(P[j] & B[j]).count("1") for j in range(8)) == want
