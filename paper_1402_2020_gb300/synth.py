"""Seeded synthetic stereo inputs shaped like the paper's workloads.

This module holds none of the matching method's arithmetic: it only draws images, ground-truth
disparities, sampling-pair tables, batch shapes and request traces from a seed. Both the CUDA path
and the oracle are fed from it.

Recipe (the paper's Middlebury and radiometric datasets are not available; these stand in for them):
- left view: three octaves of smooth value noise, low-amplitude per-pixel noise, 10-30 uniform
  rectangles and 5-15 strongly textured patches;
- ground-truth disparity: 3-6 random planes d = round(a x + b y + c) over Voronoi regions,
  clamped to [0, dmax-1];
- right view: the left view forward-warped by that disparity (x_R = x_L - d; the larger d wins a
  collision), holes (occlusions) filled from noise;
- optional radiometric change of the right view: v' = clamp(round(255 (g v / 255)^gamma + o_c)),
  g in [0.5, 2], gamma in [0.7, 1.5], o_c in [-20, 20] per channel;
- sampling pairs: i.i.d. isotropic Gaussian offsets (sigma = S / 5 unless given), rounded, drawn
  again when outside the S x S window (|offset| <= S // 2).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def pair_table(n: int = 256, S: int = 31, sigma: float | None = None, seed: int = 0) -> np.ndarray:
    """n sampling pairs (px, py, qx, qy) as int8 offsets from the centre pixel (Sec. 3, Eq. 2)."""
    rng = _rng(seed)
    half = S // 2
    sigma = S / 5.0 if sigma is None else float(sigma)
    out = np.empty((n, 4), np.int8)
    filled = 0
    while filled < n:
        v = np.rint(rng.normal(0.0, sigma, size=(n, 4)))
        v = v[np.all(np.abs(v) <= half, axis=1)][: n - filled]
        out[filled : filled + len(v)] = v.astype(np.int8)
        filled += len(v)
    return out


def _value_noise(rng: np.random.Generator, h: int, w: int, cell: int) -> np.ndarray:
    gh, gw = h // cell + 2, w // cell + 2
    g = rng.random((gh, gw, 3), dtype=np.float32)
    ys = np.arange(h, dtype=np.float32) / cell
    xs = np.arange(w, dtype=np.float32) / cell
    y0 = ys.astype(np.int64)
    x0 = xs.astype(np.int64)
    fy = (ys - y0)[:, None, None]
    fx = (xs - x0)[None, :, None]
    fy = fy * fy * (3 - 2 * fy)
    fx = fx * fx * (3 - 2 * fx)
    top = g[y0][:, x0] * (1 - fx) + g[y0][:, x0 + 1] * fx
    bot = g[y0 + 1][:, x0] * (1 - fx) + g[y0 + 1][:, x0 + 1] * fx
    return top * (1 - fy) + bot * fy


def left_view(w: int, h: int, rng: np.random.Generator) -> np.ndarray:
    base = np.zeros((h, w, 3), np.float32)
    scale = max(w, h)
    for cell, amp in ((max(8, scale // 8), 150.0), (max(4, scale // 40), 70.0), (4, 35.0)):
        base += amp * _value_noise(rng, h, w, cell)
    base += rng.normal(0.0, 3.0, size=(h, w, 3)).astype(np.float32)
    img = base
    for _ in range(int(rng.integers(10, 31))):
        rw = int(rng.integers(max(2, w // 20), max(3, w // 4)))
        rh = int(rng.integers(max(2, h // 20), max(3, h // 4)))
        x0 = int(rng.integers(0, max(1, w - rw)))
        y0 = int(rng.integers(0, max(1, h - rh)))
        img[y0 : y0 + rh, x0 : x0 + rw] = rng.integers(0, 256, size=3).astype(np.float32)
    for _ in range(int(rng.integers(5, 16))):
        rw = int(rng.integers(max(2, w // 30), max(3, w // 6)))
        rh = int(rng.integers(max(2, h // 30), max(3, h // 6)))
        x0 = int(rng.integers(0, max(1, w - rw)))
        y0 = int(rng.integers(0, max(1, h - rh)))
        rw, rh = min(rw, w - x0), min(rh, h - y0)
        tone = rng.integers(30, 226, size=3).astype(np.float32)
        img[y0 : y0 + rh, x0 : x0 + rw] = tone + rng.normal(0.0, 40.0, size=(rh, rw, 3)).astype(np.float32)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def disparity_planes(w: int, h: int, dmax: int, rng: np.random.Generator) -> np.ndarray:
    m = int(rng.integers(3, 7))
    sx = rng.integers(0, w, size=m)
    sy = rng.integers(0, h, size=m)
    c = rng.uniform(0, dmax - 1, size=m)
    slope = 0.25 * dmax / max(w, h)
    a = rng.uniform(-slope, slope, size=m)
    b = rng.uniform(-slope, slope, size=m)
    ys, xs = np.mgrid[0:h, 0:w]
    best = np.full((h, w), np.inf)
    label = np.zeros((h, w), np.int64)
    for i in range(m):
        dist = (xs - sx[i]) ** 2 + (ys - sy[i]) ** 2
        closer = dist < best
        best[closer] = dist[closer]
        label[closer] = i
    d = np.rint(a[label] * (xs - sx[label]) + b[label] * (ys - sy[label]) + c[label])
    return np.clip(d, 0, dmax - 1).astype(np.int32)


def forward_warp(left: np.ndarray, disp: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    h, w, _ = left.shape
    ys, xs = np.mgrid[0:h, 0:w]
    xr = xs - disp
    ok = xr >= 0
    key = np.full(h * w, -1, np.int64)
    target = (ys * w + xr)[ok]
    np.maximum.at(key, target, (disp.astype(np.int64) * w + xs)[ok])
    right = rng.integers(0, 256, size=(h * w, 3)).astype(np.uint8)
    hit = key >= 0
    src_x = key[hit] % w
    src_y = np.nonzero(hit)[0] // w
    right[hit] = left[src_y, src_x]
    return right.reshape(h, w, 3)


def radiometric_fixed(img: np.ndarray, gain: float, gamma: float, off=(0.0, 0.0, 0.0)) -> np.ndarray:
    """v' = clamp(round(255 (gain v / 255)^gamma + off_c)): one exposure/illumination setting."""
    v = 255.0 * np.power(gain * img.astype(np.float64) / 255.0, gamma) + np.asarray(off, np.float64)
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def radiometric(img: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    gain = rng.uniform(0.5, 2.0)
    gamma = rng.uniform(0.7, 1.5)
    off = rng.uniform(-20.0, 20.0, size=3)
    return radiometric_fixed(img, gain, gamma, off)


def stereo_pair(w: int, h: int, dmax: int, seed: int, radiometric_change: bool = False):
    """(left, right, ground-truth left disparity): uint8 [h][w][3] twice and int32 [h][w]."""
    rng = _rng(seed)
    left = left_view(w, h, rng)
    gt = disparity_planes(w, h, dmax, rng)
    right = forward_warp(left, gt, rng)
    if radiometric_change:
        right = radiometric(right, rng)
    return np.ascontiguousarray(left), np.ascontiguousarray(right), gt


def shifted_pair(w: int, h: int, shift: int, seed: int):
    """A textured pair with right(x - shift) == left(x): a constant integer disparity ``shift``."""
    rng = _rng(seed)
    left = rng.integers(0, 256, size=(h, w + shift, 3)).astype(np.uint8)
    left[:, :, 1] = np.clip(left[:, :, 1].astype(np.int32) // 2 + 64, 0, 255)
    right = np.ascontiguousarray(left[:, shift : shift + w])
    left = np.ascontiguousarray(left[:, :w])
    return left, right


def batch_shapes(count: int = 64, seed: int = 3, dmaxes=(64, 128, 192, 256)):
    """Uneven batch: widths U[320, 1920], heights U[240, 1080], dmax from ``dmaxes``."""
    rng = _rng(seed)
    out = []
    for i in range(count):
        w = int(rng.integers(320, 1921))
        h = int(rng.integers(240, 1081))
        d = int(dmaxes[int(rng.integers(0, len(dmaxes)))])
        out.append((w, h, d, int(seed) * 1000 + i))
    return out


SERVE_SIZES = ((640, 480), (1280, 720), (1920, 1080), (3840, 2160))
SERVE_DMAX = (64, 128, 256)


def request_trace(count: int, rate_per_s: float, seed: int = 5):
    """Poisson arrivals: list of (arrival_s, w, h, dmax) with sizes and dmax drawn uniformly."""
    rng = _rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    sizes = rng.integers(0, len(SERVE_SIZES), size=count)
    dm = rng.integers(0, len(SERVE_DMAX), size=count)
    return [(float(t[i]), SERVE_SIZES[sizes[i]][0], SERVE_SIZES[sizes[i]][1], SERVE_DMAX[dm[i]])
            for i in range(count)]
