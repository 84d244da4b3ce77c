"""NumPy front end of the Binary Stereo Matching oracle (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may import this
module. It loads ``liboracle.so`` (built from ``bsm_oracle.cpp`` by ``oracle/build.py``), which is a
plain single-threaded statement of Sec. 3 of "Binary Stereo Matching" (Zhang et al.). It never
touches the CUDA library.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(_build.build()))
    return _lib


def bind(L):
    """Declare the C signatures of an oracle library handle (the built one, or a test's variant)."""
    if True:
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        L.oracle_intensity.argtypes = [I, I, I]
        L.oracle_intensity.restype = I
        L.oracle_lab.argtypes = [I, I, I, P]
        L.oracle_lab.restype = None
        L.oracle_lab_all.argtypes = [P, P, P, P]
        L.oracle_lab_all.restype = None
        L.oracle_describe.argtypes = [P, I, I, I, P, I, I, I, I, P, P]
        L.oracle_describe.restype = I
        L.oracle_cost_at.argtypes = [P, P, P, I, I, I, I, I, I, I, P]
        L.oracle_cost_at.restype = ctypes.c_uint32
        L.oracle_aggregate.argtypes = [P, P, P, I, I, I, I, I, I, I, I, I, I, P, P]
        L.oracle_aggregate.restype = I
        L.oracle_wta.argtypes = [P, P, P, I, I, I, I, I, I, I, I, I, I, P, P]
        L.oracle_wta.restype = I
        L.oracle_lr_check.argtypes = [P, P, I, I, I, P]
        L.oracle_lr_check.restype = I
        L.oracle_vote_tables.argtypes = [D, D, I, I, P, P]
        L.oracle_vote_tables.restype = None
        L.oracle_refine.argtypes = [P, I, P, P, I, I, I, I, D, D, P]
        L.oracle_refine.restype = I
        L.oracle_refine_region.argtypes = [P, I, P, P, I, I, I, I, D, D, I, I, I, I, P]
        L.oracle_refine_region.restype = I
        L.oracle_sgm.argtypes = [P, I, I, I, I, I, P, I, P, P]
        L.oracle_sgm.restype = I
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _rgb(img):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    assert img.ndim == 3 and img.shape[2] == 3
    return img


def intensity(R, G, B):
    """I(x) of Eq. 3 for one RGB pixel."""
    return lib().oracle_intensity(int(R), int(G), int(B))


def lab(R, G, B):
    """Integer CIELAB (L, a, b) of one RGB pixel, as used by the SAD of Eq. 5."""
    out = np.zeros(3, np.int32)
    lib().oracle_lab(int(R), int(G), int(B), _p(out))
    return tuple(int(v) for v in out)


def lab_all():
    """(L, a, b, I) of all 2^24 colours, index (R << 16) | (G << 8) | B (int8, int8, int8, uint8)."""
    n = 1 << 24
    L = np.zeros(n, np.int8)
    A = np.zeros(n, np.int8)
    Bc = np.zeros(n, np.int8)
    I = np.zeros(n, np.uint8)
    lib().oracle_lab_all(_p(L), _p(A), _p(Bc), _p(I))
    return L, A, Bc, I


def describe(img, pairs, k=None, y0=0, y1=None, out=None):
    """B (Eq. 2-3) and Phi (Eq. 5-7) planes [h][w][n/32] (uint32) of one RGB view.

    Only rows [y0, y1) are computed; the rest of the planes are zero (or left as in ``out``).
    """
    img = _rgb(img)
    h, w, _ = img.shape
    pairs = np.ascontiguousarray(pairs, dtype=np.int8)
    n = pairs.shape[0]
    k = n // 4 if k is None else int(k)
    y1 = h if y1 is None else int(y1)
    if out is None:
        B = np.zeros((h, w, n // 32), np.uint32)
        Phi = np.zeros((h, w, n // 32), np.uint32)
    else:
        B, Phi = out
    rc = lib().oracle_describe(_p(img), w, h, w * 3, _p(pairs), n, k, int(y0), y1, _p(B), _p(Phi))
    if rc != 0:
        raise ValueError("oracle_describe rejected its arguments")
    return B, Phi


def _opt(p):
    """The optional other-view mask plane as a C pointer (None: Eq. 8's reference mask only)."""
    return None if p is None else _p(p)


def cost_at(Bref, Phiref, Both, x, y, d, direction, Phioth=None):
    """C(x, d) of Eq. 8 at one pixel (direction 0: left reference, 1: right reference).

    With Phioth (the other view's mask plane) the matched pixel's mask is ANDed as well: the mask
    ablation, not the paper's Eq. 8."""
    h, w, nw = Bref.shape
    if Phioth is not None:
        Phioth = np.ascontiguousarray(Phioth, dtype=np.uint32)
    return int(lib().oracle_cost_at(_p(Bref), _p(Phiref), _p(Both), w, h, 32 * nw, int(x), int(y), int(d),
                                    int(direction), _opt(Phioth)))


def _planes(*ps):
    return [None if p is None else np.ascontiguousarray(p, dtype=np.uint32) for p in ps]


def aggregate(Bref, Phiref, Both, dmax, win, direction, x0=0, x1=None, y0=0, y1=None, Phioth=None):
    """Window-aggregated cost A[y][x][d] (uint32) over the region; win = 1 gives Eq. 8 itself."""
    Bref, Phiref, Both, Phioth = _planes(Bref, Phiref, Both, Phioth)
    h, w, nw = Bref.shape
    x1 = w if x1 is None else x1
    y1 = h if y1 is None else y1
    A = np.zeros((y1 - y0, x1 - x0, dmax), np.uint32)
    rc = lib().oracle_aggregate(_p(Bref), _p(Phiref), _p(Both), w, h, 32 * nw, dmax, win, direction,
                                x0, x1, y0, y1, _p(A), _opt(Phioth))
    if rc != 0:
        raise ValueError("oracle_aggregate rejected its arguments")
    return A


def wta(Bref, Phiref, Both, dmax, win, direction, x0=0, x1=None, y0=0, y1=None, Phioth=None):
    """Eq. 1 on the aggregated cost: int32 disparities [y1-y0][x1-x0]."""
    Bref, Phiref, Both, Phioth = _planes(Bref, Phiref, Both, Phioth)
    h, w, nw = Bref.shape
    x1 = w if x1 is None else x1
    y1 = h if y1 is None else y1
    disp = np.zeros((y1 - y0, x1 - x0), np.int32)
    rc = lib().oracle_wta(_p(Bref), _p(Phiref), _p(Both), w, h, 32 * nw, dmax, win, direction,
                          x0, x1, y0, y1, _p(disp), _opt(Phioth))
    if rc != 0:
        raise ValueError("oracle_wta rejected its arguments")
    return disp


def lr_check(dL, dR, tol=1):
    """Left/right consistency of the left map: uint8 valid mask."""
    dL = np.ascontiguousarray(dL, dtype=np.int32)
    dR = np.ascontiguousarray(dR, dtype=np.int32)
    h, w = dL.shape
    valid = np.zeros((h, w), np.uint8)
    if lib().oracle_lr_check(_p(dL), _p(dR), w, h, int(tol), _p(valid)) != 0:
        raise ValueError("oracle_lr_check rejected its arguments")
    return valid


def vote_tables(lambda_c=9.0, lambda_e=16.0, R=15):
    """Integer vote tables (Ec over colour SAD 0..765, Es over squared distance 0..2R^2)."""
    nc, ne = 766, 2 * R * R + 1
    Ec = np.zeros(nc, np.uint32)
    Es = np.zeros(ne, np.uint32)
    lib().oracle_vote_tables(float(lambda_c), float(lambda_e), nc, ne, _p(Ec), _p(Es))
    return Ec, Es


def refine(imgL, dL, valid, dmax, R=15, lambda_c=9.0, lambda_e=16.0):
    """Eq. 9-10 voting refinement of the invalid pixels of the left map."""
    imgL = _rgb(imgL)
    h, w, _ = imgL.shape
    dL = np.ascontiguousarray(dL, dtype=np.int32)
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    out = np.zeros((h, w), np.int32)
    rc = lib().oracle_refine(_p(imgL), w * 3, _p(dL), _p(valid), w, h, dmax, int(R), float(lambda_c),
                             float(lambda_e), _p(out))
    if rc != 0:
        raise ValueError("oracle_refine rejected its arguments")
    return out


def refine_region(imgL, dL, valid, dmax, x0, x1, y0, y1, R=15, lambda_c=9.0, lambda_e=16.0):
    """Eq. 9-10 for the output region [x0, x1) x [y0, y1) (inputs are full-image maps)."""
    imgL = _rgb(imgL)
    h, w, _ = imgL.shape
    dL = np.ascontiguousarray(dL, dtype=np.int32)
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    out = np.zeros((y1 - y0, x1 - x0), np.int32)
    rc = lib().oracle_refine_region(_p(imgL), w * 3, _p(dL), _p(valid), w, h, dmax, int(R), float(lambda_c),
                                    float(lambda_e), x0, x1, y0, y1, _p(out))
    if rc != 0:
        raise ValueError("oracle_refine_region rejected its arguments")
    return out


SGM_DIRS4 = ((1, 0), (-1, 0), (0, 1), (0, -1))
SGM_DIRS8 = SGM_DIRS4 + ((1, 1), (-1, 1), (1, -1), (-1, -1))


def sgm(C, P1, P2, dirs=SGM_DIRS4):
    """Semi-global aggregation (reading R10) of a cost volume C[h][w][dmax]: returns (S uint32, disp int32)."""
    C = np.ascontiguousarray(C, dtype=np.uint16)
    h, w, dmax = C.shape
    d = np.ascontiguousarray(np.asarray(dirs, np.int32).reshape(-1))
    S = np.zeros((h, w, dmax), np.uint32)
    disp = np.zeros((h, w), np.int32)
    if lib().oracle_sgm(_p(C), w, h, dmax, int(P1), int(P2), _p(d), len(d) // 2, _p(S), _p(disp)) != 0:
        raise ValueError("oracle_sgm rejected its arguments")
    return S, disp


MASK_REFERENCE, MASK_NONE, MASK_BOTH = 0, 1, 2


def pipeline(imgL, imgR, pairs, dmax, win=5, k=None, tol=1, R=15, lambda_c=9.0, lambda_e=16.0,
             mask_mode=MASK_REFERENCE, sgm_params=None):
    """The whole method of Sec. 3 on one pair: returns dict of every intermediate and the final map.

    mask_mode: MASK_REFERENCE is Eq. 8 as printed; MASK_NONE drops the mask (Eq. 4, every Phi bit set);
    MASK_BOTH also ANDs the matched pixel's Phi (the mask ablation). sgm_params = (P1, P2, dirs) replaces
    Eq. 1 on the aggregated cost by semi-global aggregation followed by Eq. 1 (reading R10)."""
    BL, PhiL = describe(imgL, pairs, k)
    BR, PhiR = describe(imgR, pairs, k)
    if mask_mode == MASK_NONE:
        PhiL = np.full_like(PhiL, 0xFFFFFFFF)
        PhiR = np.full_like(PhiR, 0xFFFFFFFF)
    both = mask_mode == MASK_BOTH
    if sgm_params is None:
        dL = wta(BL, PhiL, BR, dmax, win, 0, Phioth=PhiR if both else None)
        dR = wta(BR, PhiR, BL, dmax, win, 1, Phioth=PhiL if both else None)
    else:  # reading R10 on the aggregated cost volumes of both reference views
        P1, P2, dirs = sgm_params
        dL = sgm(aggregate(BL, PhiL, BR, dmax, win, 0, Phioth=PhiR if both else None), P1, P2, dirs)[1]
        dR = sgm(aggregate(BR, PhiR, BL, dmax, win, 1, Phioth=PhiL if both else None), P1, P2, dirs)[1]
    valid = lr_check(dL, dR, tol)
    out = refine(imgL, dL, valid, dmax, R, lambda_c, lambda_e)
    return {"BL": BL, "PhiL": PhiL, "BR": BR, "PhiR": PhiR, "dL": dL, "dR": dR, "valid": valid, "disp": out}
