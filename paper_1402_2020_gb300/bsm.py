"""Thin Python binding of libbsm.so (include/bsm.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. Functions take PyTorch CUDA tensors (device
memory and streams come from PyTorch) or raw integer addresses, and raise ``BsmError`` on any
non-OK status. If the compiled library is missing this module raises at load time: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbsm.so")

BSM_OK = 0
BSM_ERR_INVALID_ARG = 1
BSM_ERR_OUT_OF_MEMORY = 2
BSM_ERR_CUDA = 3
BSM_ERR_TIMEOUT = 4
BSM_ERR_UNSUPPORTED = 5

# Every symbol include/bsm.h declares.
EXPORTED = (
    "bsm_create", "bsm_destroy", "bsm_describe", "bsm_cost_aggregate_wta", "bsm_refine", "bsm_match_host",
    "bsm_last_error", "bsm_status_string", "bsm_copy_color_table", "bsm_vote_tables", "bsm_validate_params",
    "bsm_abi_version", "bsm_set_tuning", "bsm_get_tuning", "bsm_reserve", "bsm_describe_noalloc",
    "bsm_batch_run", "bsm_reserve_batch", "bsm_last_cuda_error", "bsm_server_create", "bsm_server_submit",
    "bsm_server_poll", "bsm_server_drain", "bsm_server_get_stats", "bsm_server_destroy", "bsm_debug_set",
    "bsm_cost_volumes", "bsm_sgm", "bsm_cost_plan", "bsm_describe_gather_plan",
)
BSM_DEBUG_WITHHOLD_ARRIVALS = 1
BSM_MAX_BATCH = 1024

BSM_NOALLOC_MAX_PIXELS = 4194304


class BsmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {status_name(status)} ({status})")


class bsm_params(ctypes.Structure):
    _fields_ = [
        ("n_bits", ctypes.c_int32),
        ("window_S", ctypes.c_int32),
        ("pairs", ctypes.POINTER(ctypes.c_int8)),
        ("agg_window", ctypes.c_int32),
        ("mask_rank", ctypes.c_int32),
        ("dmax", ctypes.c_int32),
        ("lr_tol", ctypes.c_int32),
        ("vote_radius", ctypes.c_int32),
        ("lambda_c", ctypes.c_int32),
        ("lambda_e", ctypes.c_int32),
        ("mask_mode", ctypes.c_int32),
    ]


BSM_MASK_REFERENCE, BSM_MASK_NONE, BSM_MASK_BOTH = 0, 1, 2


class bsm_tuning(ctypes.Structure):
    _fields_ = [("cost_rows", ctypes.c_int32), ("cost_popc_plain", ctypes.c_int32), ("batch_rows", ctypes.c_int32),
                ("cost_variant", ctypes.c_int32), ("describe_variant", ctypes.c_int32),
                ("describe_copies", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class bsm_cost_plan_info(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("rows_per_band", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


COST_KERNELS = {1: ("cost_wta_kernel", "bsm_cost.cu"), 2: ("cost2_kernel", "bsm_cost2.cu"),
                3: ("cost_tc_kernel", "bsm_cost_tc.cu"), 4: ("cost_long_kernel", "bsm_long.cu")}


class bsm_pair_desc(ctypes.Structure):
    _fields_ = [("rgbL", ctypes.c_void_p), ("rgbR", ctypes.c_void_p), ("w", ctypes.c_int32), ("h", ctypes.c_int32),
                ("pitch_bytes", ctypes.c_int32), ("dmax", ctypes.c_int32), ("BL", ctypes.c_void_p),
                ("PhiL", ctypes.c_void_p), ("BR", ctypes.c_void_p), ("PhiR", ctypes.c_void_p),
                ("dispL", ctypes.c_void_p), ("dispR", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class bsm_server_config(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("device_budget", ctypes.c_int64),
                ("max_batch_work", ctypes.c_int64)]


class bsm_request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("rgbL", ctypes.c_void_p), ("rgbR", ctypes.c_void_p), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("pitch_bytes", ctypes.c_int32), ("dmax", ctypes.c_int32),
                ("out", ctypes.c_void_p)]


class bsm_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("latency_us", ctypes.c_double)]


class bsm_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "batches", "max_batch_seen",
                                              "queued", "bytes_in_use", "budget", "scratch_bytes")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libbsm.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, I, S = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
        L.bsm_create.argtypes = [ctypes.POINTER(bsm_params), ctypes.POINTER(P)]
        L.bsm_create.restype = S
        L.bsm_destroy.argtypes = [P]
        L.bsm_destroy.restype = None
        L.bsm_describe.argtypes = [P, P, I, I, I, P, P, P]
        L.bsm_describe.restype = S
        L.bsm_cost_aggregate_wta.argtypes = [P, P, P, P, P, I, I, I, P, P, P, P]
        L.bsm_cost_aggregate_wta.restype = S
        L.bsm_cost_volumes.argtypes = [P, P, P, P, P, I, I, I, P, P, P, P, P]
        L.bsm_cost_volumes.restype = S
        L.bsm_sgm.argtypes = [P, P, I, I, I, I, I, I, P, P, P]
        L.bsm_sgm.restype = S
        L.bsm_refine.argtypes = [P, P, I, P, P, I, I, I, P, P]
        L.bsm_refine.restype = S
        L.bsm_match_host.argtypes = [P, P, P, I, I, I, I, P, P]
        L.bsm_match_host.restype = S
        L.bsm_last_error.argtypes = [P]
        L.bsm_last_error.restype = S
        L.bsm_status_string.argtypes = [S]
        L.bsm_status_string.restype = ctypes.c_char_p
        L.bsm_copy_color_table.argtypes = [P, P, P]
        L.bsm_copy_color_table.restype = S
        L.bsm_vote_tables.argtypes = [I, I, I, I, P, P]
        L.bsm_vote_tables.restype = S
        L.bsm_validate_params.argtypes = [ctypes.POINTER(bsm_params)]
        L.bsm_validate_params.restype = S
        L.bsm_set_tuning.argtypes = [P, ctypes.POINTER(bsm_tuning)]
        L.bsm_set_tuning.restype = S
        L.bsm_get_tuning.argtypes = [P, ctypes.POINTER(bsm_tuning)]
        L.bsm_get_tuning.restype = S
        L.bsm_describe_noalloc.argtypes = [P, P, I, I, I, P, P, P]
        L.bsm_describe_noalloc.restype = S
        L.bsm_server_create.argtypes = [ctypes.POINTER(bsm_params), ctypes.POINTER(bsm_server_config),
                                        ctypes.POINTER(P)]
        L.bsm_server_create.restype = S
        L.bsm_server_submit.argtypes = [P, ctypes.POINTER(bsm_request)]
        L.bsm_server_submit.restype = S
        L.bsm_server_poll.argtypes = [P, ctypes.POINTER(bsm_completion), I, I]
        L.bsm_server_poll.restype = I
        L.bsm_server_drain.argtypes = [P, I]
        L.bsm_server_drain.restype = S
        L.bsm_server_get_stats.argtypes = [P, ctypes.POINTER(bsm_server_stats)]
        L.bsm_server_get_stats.restype = S
        L.bsm_server_destroy.argtypes = [P]
        L.bsm_server_destroy.restype = None
        L.bsm_debug_set.argtypes = [P, I, I]
        L.bsm_debug_set.restype = S
        L.bsm_cost_plan.argtypes = [P, I, I, I, ctypes.POINTER(bsm_cost_plan_info)]
        L.bsm_cost_plan.restype = S
        IP = ctypes.POINTER(ctypes.c_int32)
        L.bsm_describe_gather_plan.argtypes = [ctypes.c_void_p, I, I, IP, IP, IP, IP, IP]
        L.bsm_describe_gather_plan.restype = S
        L.bsm_last_cuda_error.argtypes = [P]
        L.bsm_last_cuda_error.restype = ctypes.c_char_p
        L.bsm_batch_run.argtypes = [P, ctypes.POINTER(bsm_pair_desc), I, P]
        L.bsm_batch_run.restype = S
        L.bsm_reserve_batch.argtypes = [P, ctypes.c_int64]
        L.bsm_reserve_batch.restype = S
        L.bsm_reserve.argtypes = [P, I, I]
        L.bsm_reserve.restype = S
        L.bsm_abi_version.argtypes = []
        L.bsm_abi_version.restype = I
        _lib = L
    return _lib


def status_name(s: int) -> str:
    return lib().bsm_status_string(int(s)).decode()


def _check(s: int, where: str, ctx: int = 0):
    if s != BSM_OK:
        detail = lib().bsm_last_cuda_error(ctx).decode() if ctx and s == BSM_ERR_CUDA else ""
        raise BsmError(s, where + (f" [{detail}]" if detail else ""))


def bsm_debug_set(ctx: int, key: int, value: int) -> None:
    _check(lib().bsm_debug_set(ctx, key, value), "bsm_debug_set")


def bsm_last_cuda_error(ctx: int) -> str:
    return lib().bsm_last_cuda_error(ctx).decode()


def _ptr(t) -> int:
    """Device/host address of a torch tensor, a numpy array, an int address, or None -> 0."""
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(pairs: np.ndarray, window_S: int = 31, agg_window: int = 5, mask_rank: int = 0, dmax: int = 256,
                lr_tol: int = 1, vote_radius: int = 15, lambda_c: int = 9, lambda_e: int = 16,
                mask_mode: int = BSM_MASK_REFERENCE):
    """bsm_params for a pair table (int8 [n][4]); keeps the table alive on the returned object."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int8)
    p = bsm_params()
    p.n_bits = pairs.shape[0]
    p.window_S = window_S
    p.pairs = pairs.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    p.agg_window = agg_window
    p.mask_rank = mask_rank
    p.dmax = dmax
    p.lr_tol = lr_tol
    p.vote_radius = vote_radius
    p.lambda_c = lambda_c
    p.lambda_e = lambda_e
    p.mask_mode = mask_mode
    p._keep = pairs
    return p


def bsm_abi_version() -> int:
    return lib().bsm_abi_version()


def bsm_validate_params(params: bsm_params) -> int:
    return lib().bsm_validate_params(ctypes.byref(params))


def bsm_vote_tables(lambda_c: int, lambda_e: int, nc: int, ne: int):
    Ec = np.zeros(nc, np.uint32)
    Es = np.zeros(ne, np.uint32)
    _check(lib().bsm_vote_tables(lambda_c, lambda_e, nc, ne, Ec.ctypes.data, Es.ctypes.data), "bsm_vote_tables")
    return Ec, Es


def bsm_create(params: bsm_params) -> int:
    h = ctypes.c_void_p()
    _check(lib().bsm_create(ctypes.byref(params), ctypes.byref(h)), "bsm_create")
    return h.value


def bsm_destroy(ctx: int) -> None:
    lib().bsm_destroy(ctx)


def bsm_describe(ctx: int, rgb, w: int, h: int, pitch: int, B, Phi, stream=None) -> None:
    _check(lib().bsm_describe(ctx, _ptr(rgb), w, h, pitch, _ptr(B), _ptr(Phi), _stream(stream)), "bsm_describe", ctx)


def bsm_describe_noalloc(ctx: int, rgb, w: int, h: int, pitch: int, B, Phi, stream=None) -> None:
    """bsm_describe with its scratch in a fixed device array: allocates nothing (see include/bsm.h)."""
    _check(lib().bsm_describe_noalloc(ctx, _ptr(rgb), w, h, pitch, _ptr(B), _ptr(Phi), _stream(stream)),
           "bsm_describe_noalloc", ctx)


def bsm_cost_aggregate_wta(ctx: int, BL, PhiL, BR, PhiR, w: int, h: int, dmax: int, dispL, dispR, cost=None,
                           stream=None) -> None:
    _check(lib().bsm_cost_aggregate_wta(ctx, _ptr(BL), _ptr(PhiL), _ptr(BR), _ptr(PhiR), w, h, dmax, _ptr(dispL),
                                        _ptr(dispR), _ptr(cost), _stream(stream)), "bsm_cost_aggregate_wta", ctx)


def bsm_cost_volumes(ctx: int, BL, PhiL, BR, PhiR, w: int, h: int, dmax: int, dispL, dispR, costL, costR,
                     stream=None) -> None:
    _check(lib().bsm_cost_volumes(ctx, _ptr(BL), _ptr(PhiL), _ptr(BR), _ptr(PhiR), w, h, dmax, _ptr(dispL),
                                  _ptr(dispR), _ptr(costL), _ptr(costR), _stream(stream)), "bsm_cost_volumes", ctx)


def bsm_sgm(ctx: int, cost, w: int, h: int, dmax: int, P1: int, P2: int, paths: int, S, disp, stream=None) -> None:
    _check(lib().bsm_sgm(ctx, _ptr(cost), w, h, dmax, P1, P2, paths, _ptr(S), _ptr(disp), _stream(stream)),
           "bsm_sgm", ctx)


def bsm_refine(ctx: int, rgbL, pitch: int, dispL, dispR, w: int, h: int, dmax: int, out, stream=None) -> None:
    _check(lib().bsm_refine(ctx, _ptr(rgbL), pitch, _ptr(dispL), _ptr(dispR), w, h, dmax, _ptr(out),
                            _stream(stream)), "bsm_refine", ctx)


def bsm_match_host(ctx: int, rgbL_host, rgbR_host, w: int, h: int, pitch: int, dmax: int, out_host,
                   stream=None) -> None:
    _check(lib().bsm_match_host(ctx, _ptr(rgbL_host), _ptr(rgbR_host), w, h, pitch, dmax, _ptr(out_host),
                                _stream(stream)), "bsm_match_host", ctx)


def bsm_last_error(ctx: int) -> int:
    return lib().bsm_last_error(ctx)


def bsm_status_string(s: int) -> str:
    return status_name(s)


def bsm_copy_color_table(ctx: int, dst, stream=None) -> None:
    _check(lib().bsm_copy_color_table(ctx, _ptr(dst), _stream(stream)), "bsm_copy_color_table")


def bsm_reserve(ctx: int, max_w: int, max_h: int) -> None:
    _check(lib().bsm_reserve(ctx, max_w, max_h), "bsm_reserve")


def bsm_set_tuning(ctx: int, cost_rows: int = 0, cost_popc_plain: int = 0, batch_rows: int = 0,
                   cost_variant: int = 0, describe_variant: int = 0, describe_copies: int = 0) -> None:
    t = bsm_tuning()
    t.cost_rows = cost_rows
    t.cost_popc_plain = cost_popc_plain
    t.batch_rows = batch_rows
    t.cost_variant = cost_variant
    t.describe_variant = describe_variant
    t.describe_copies = describe_copies
    _check(lib().bsm_set_tuning(ctx, ctypes.byref(t)), "bsm_set_tuning")


def bsm_cost_plan(ctx: int, w: int, h: int, dmax: int) -> dict:
    """The cost launch bsm_cost_aggregate_wta makes for this shape: kernel id (1..4), its name and source
    file, output rows per CTA band, launches per call."""
    p = bsm_cost_plan_info()
    _check(lib().bsm_cost_plan(ctx, w, h, dmax, ctypes.byref(p)), "bsm_cost_plan")
    name, src = COST_KERNELS[p.kernel]
    return {"kernel": p.kernel, "name": name, "source": src, "rows_per_band": p.rows_per_band,
            "launches": p.launches}


def bsm_describe_gather_plan(pairs: np.ndarray, copies: int = 4) -> dict:
    """The warp-per-pixel describe kernel's gather plan for a pair table (host only): tile pitch, copies
    used, copy bases, each sample's word offset from the pixel (n_bits x 2) and each load's wavefronts."""
    pr = np.ascontiguousarray(pairs, dtype=np.int8)
    n = int(pr.shape[0])
    nl = max(1, 2 * (n // 32))
    pitch, used = ctypes.c_int32(), ctypes.c_int32()
    base = np.zeros(4, np.int32)
    offs = np.zeros((max(n, 1), 2), np.int32)
    wf = np.zeros(nl, np.int32)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
    _check(lib().bsm_describe_gather_plan(pr.ctypes.data, n, copies, ctypes.byref(pitch), ctypes.byref(used),
                                          ip(base), ip(offs), ip(wf)), "bsm_describe_gather_plan")
    return {"pitch": pitch.value, "copies": used.value, "copy_base": base[: used.value].copy(), "offsets": offs[:n],
            "wavefronts": wf}


def bsm_get_tuning(ctx: int) -> dict:
    t = bsm_tuning()
    _check(lib().bsm_get_tuning(ctx, ctypes.byref(t)), "bsm_get_tuning")
    return {"cost_rows": t.cost_rows, "cost_popc_plain": t.cost_popc_plain, "batch_rows": t.batch_rows,
            "cost_variant": t.cost_variant, "describe_variant": t.describe_variant,
            "describe_copies": t.describe_copies}


def pair_desc(rgbL, rgbR, w, h, pitch, dmax, BL, PhiL, BR, PhiR, dispL, dispR, out) -> bsm_pair_desc:
    return bsm_pair_desc(_ptr(rgbL), _ptr(rgbR), w, h, pitch, dmax, _ptr(BL), _ptr(PhiL), _ptr(BR), _ptr(PhiR),
                         _ptr(dispL), _ptr(dispR), _ptr(out))


def bsm_batch_run(ctx: int, descs, stream=None) -> None:
    arr = (bsm_pair_desc * len(descs))(*descs)
    _check(lib().bsm_batch_run(ctx, arr, len(descs), _stream(stream)), "bsm_batch_run", ctx)


def bsm_reserve_batch(ctx: int, total_pixels: int) -> None:
    _check(lib().bsm_reserve_batch(ctx, int(total_pixels)), "bsm_reserve_batch", ctx)


class Matcher:
    """Convenience owner of one context plus torch-allocated outputs (still only marshalling)."""

    def __init__(self, pairs, **kw):
        import torch

        self.torch = torch
        self.params = make_params(pairs, **kw)
        self.n_bits = self.params.n_bits
        self.ctx = bsm_create(self.params)

    def close(self):
        if self.ctx:
            bsm_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def planes(self, h, w, device="cuda"):
        t = self.torch
        nw = self.n_bits // 32
        return (t.empty((h, w, nw), dtype=t.int32, device=device), t.empty((h, w, nw), dtype=t.int32, device=device))

    def describe(self, rgb, stream=None):
        h, w, _ = rgb.shape
        B, Phi = self.planes(h, w, rgb.device)
        bsm_describe(self.ctx, rgb, w, h, rgb.stride(0), B, Phi, stream)
        return B, Phi

    def cost_wta(self, BL, PhiL, BR, PhiR, dmax, want_cost=False, stream=None):
        t = self.torch
        h, w, _ = BL.shape
        dL = t.empty((h, w), dtype=t.int32, device=BL.device)
        dR = t.empty((h, w), dtype=t.int32, device=BL.device)
        cost = t.empty((h, w, dmax), dtype=t.int16, device=BL.device) if want_cost else None
        bsm_cost_aggregate_wta(self.ctx, BL, PhiL, BR, PhiR, w, h, dmax, dL, dR, cost, stream)
        return dL, dR, cost

    def refine(self, rgbL, dL, dR, dmax, stream=None):
        t = self.torch
        h, w, _ = rgbL.shape
        out = t.empty((h, w), dtype=t.int32, device=rgbL.device)
        bsm_refine(self.ctx, rgbL, rgbL.stride(0), dL, dR, w, h, dmax, out, stream)
        return out

    def match(self, rgbL, rgbR, dmax, stream=None):
        BL, PhiL = self.describe(rgbL, stream)
        BR, PhiR = self.describe(rgbR, stream)
        dL, dR, _ = self.cost_wta(BL, PhiL, BR, PhiR, dmax, stream=stream)
        return self.refine(rgbL, dL, dR, dmax, stream)

    def match_sgm(self, rgbL, rgbR, dmax, P1, P2, paths=8, stream=None):
        """The method with semi-global aggregation of both views' cost volumes before Eq. 1."""
        t = self.torch
        h, w, _ = rgbL.shape
        BL, PhiL = self.describe(rgbL, stream)
        BR, PhiR = self.describe(rgbR, stream)
        dL = t.empty((h, w), dtype=t.int32, device=rgbL.device)
        dR, sL, sR = t.empty_like(dL), t.empty_like(dL), t.empty_like(dL)
        cL = t.empty((h, w, dmax), dtype=t.int16, device=rgbL.device)
        cR = t.empty_like(cL)
        S = t.empty((h, w, dmax), dtype=t.int32, device=rgbL.device)
        bsm_cost_volumes(self.ctx, BL, PhiL, BR, PhiR, w, h, dmax, dL, dR, cL, cR, stream)
        bsm_sgm(self.ctx, cL, w, h, dmax, P1, P2, paths, S, sL, stream)
        bsm_sgm(self.ctx, cR, w, h, dmax, P1, P2, paths, S, sR, stream)
        return self.refine(rgbL, sL, sR, dmax, stream)


def bsm_server_create(params: bsm_params, lanes: int = 2, max_batch: int = 64, device_budget: int = 0,
                      max_batch_work: int = 0) -> int:
    cfg = bsm_server_config(lanes, max_batch, device_budget, max_batch_work)
    h = ctypes.c_void_p()
    _check(lib().bsm_server_create(ctypes.byref(params), ctypes.byref(cfg), ctypes.byref(h)), "bsm_server_create")
    return h.value


def bsm_server_submit(srv: int, req_id: int, rgbL, rgbR, w: int, h: int, pitch: int, dmax: int, out) -> int:
    """Queue one request (host buffers). Returns the status (a rejected request also completes)."""
    r = bsm_request(req_id, _ptr(rgbL), _ptr(rgbR), w, h, pitch, dmax, _ptr(out))
    return lib().bsm_server_submit(srv, ctypes.byref(r))


def bsm_server_poll(srv: int, max_out: int = 256, timeout_us: int = 1000):
    """List of (id, status, latency_us) completions."""
    arr = (bsm_completion * max_out)()
    n = lib().bsm_server_poll(srv, arr, max_out, timeout_us)
    if n < 0:
        raise BsmError(BSM_ERR_INVALID_ARG, "bsm_server_poll")
    return [(arr[i].id, arr[i].status, arr[i].latency_us) for i in range(n)]


def bsm_server_drain(srv: int, timeout_ms: int = -1) -> None:
    _check(lib().bsm_server_drain(srv, timeout_ms), "bsm_server_drain")


def bsm_server_get_stats(srv: int) -> dict:
    st = bsm_server_stats()
    _check(lib().bsm_server_get_stats(srv, ctypes.byref(st)), "bsm_server_get_stats")
    return {k: getattr(st, k) for k, _ in bsm_server_stats._fields_}


def bsm_server_destroy(srv: int) -> None:
    lib().bsm_server_destroy(srv)
