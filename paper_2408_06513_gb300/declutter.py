"""Thin ctypes binding of ``libdeclutter.so`` (C ABI in ``include/declutter.h``).

Argument marshalling only: every step of the method runs in the CUDA
library.  Tensors are PyTorch CUDA tensors used as device memory; their data
pointers go straight to the C calls.  There is no CPU fallback: if the
library is missing, importing this module's functions raises.

The function names are those of the C ABI:

    declutter_create, declutter_destroy, declutter_get_info,
    splat_density, integral_images, integral_images_u32,
    displacement_field, lens_field, contour_segments, advect_samples, regularize, regularize_host,
    quality_metrics, declutter_sync, declutter_profile_regularize,
    declutter_kernel_name, declutter_status_string, declutter_last_error
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "DeclutterError", "Context", "dc_params", "dc_info", "load_library", "exported_symbols",
    "declutter_create", "declutter_destroy", "declutter_get_info", "splat_density", "integral_images",
    "integral_images_u32", "splat_counts", "density_from_counts", "displacement_field", "lens_field", "contour_segments", "advect_samples", "regularize", "regularize_host",
    "quality_metrics", "declutter_counts", "declutter_sync", "regularize_adaptive", "transition_positions",
    "layout_metrics", "warp_texture", "transfer_function", "DC_WARP_VALUE", "DC_WARP_MASS", "declutter_profile_regularize", "declutter_kernel_name",
    "declutter_status_string", "declutter_last_error", "DC_CARRY_COMPENSATED", "DC_CARRY_F64",
    "DC_OPT_FUSED_BANDS", "DC_OPT_SEPARATE_SMOOTH", "DC_OPT_STAGE_HOST", "DC_OPT_BATCHED_LAUNCHES",
    "DC_OPT_TEST_UNREACHED_BARRIER", "DC_SG_MMA_SYNC", "DC_SG_TCGEN05", "DC_SG_AUTO",
    "integral_images_u32_noalloc", "DC_NOALLOC_MAX_LOG2_RES", "Batch", "declutter_batch_create",
    "declutter_batch_destroy", "declutter_batch_regularize", "declutter_batch_sync",
    "declutter_autotune_band_rows", "declutter_batch_autotune", "declutter_autotune", "declutter_autotune_save",
    "declutter_autotune_load", "declutter_autotune_clear", "regularize_tracers", "Surrogate",
    "surrogate_create", "surrogate_destroy", "surrogate_num_params", "surrogate_get_params", "surrogate_set_params",
    "surrogate_get_grads", "surrogate_set_skip", "surrogate_set_tensor_path", "surrogate_forward", "surrogate_loss_grad", "surrogate_train_step", "surrogate_apply",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdeclutter.so")
KERNEL_KINDS = 10

DC_CARRY_COMPENSATED = 0
DC_CARRY_F64 = 1
DC_NOALLOC_MAX_LOG2_RES = 10
# dc_params.options
DC_OPT_FUSED_BANDS = 1
DC_OPT_SEPARATE_SMOOTH = 2
DC_OPT_STAGE_HOST = 4
DC_OPT_BATCHED_LAUNCHES = 8
DC_OPT_TEST_UNREACHED_BARRIER = 1 << 30
# warp_texture modes
DC_WARP_VALUE = 0
DC_WARP_MASS = 1
# surrogate_set_tensor_path
DC_SG_MMA_SYNC = 0
DC_SG_TCGEN05 = 1
DC_SG_AUTO = 2


class DeclutterError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


class dc_params(ctypes.Structure):
    _fields_ = [
        ("log2_res", ctypes.c_uint32),
        ("kernel_r", ctypes.c_int32),
        ("sigma", ctypes.c_float),
        ("d0", ctypes.c_float),
        ("pixel_center", ctypes.c_int32),
        ("clamp_positions", ctypes.c_int32),
        ("carry_mode", ctypes.c_int32),
        ("band_rows", ctypes.c_int32),
        ("keep_order", ctypes.c_int32),
        ("options", ctypes.c_int32),
        ("wait_limit_us", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 1),
    ]


class dc_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("kernel_r", ctypes.c_int32),
        ("sigma", ctypes.c_float),
        ("band_rows", ctypes.c_int32),
        ("n_bands", ctypes.c_int32),
        ("band_threads", ctypes.c_int32),
        ("kernels_per_iter", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("scratch_bytes", ctypes.c_int64),
    ]


_lib = None

# (name, restype, argtypes) of every exported symbol
_P = ctypes.c_void_p
_SIGS = [
    ("declutter_create", ctypes.c_int, [ctypes.POINTER(dc_params), ctypes.c_int, _P, ctypes.POINTER(_P)]),
    ("declutter_destroy", ctypes.c_int, [_P]),
    ("declutter_get_info", ctypes.c_int, [_P, ctypes.POINTER(dc_info)]),
    ("splat_density", ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    ("splat_counts", ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    ("density_from_counts", ctypes.c_int, [_P, _P, ctypes.c_int64]),
    ("integral_images", ctypes.c_int, [_P, _P, _P]),
    ("integral_images_u32", ctypes.c_int, [_P, _P, _P, _P]),
    ("displacement_field", ctypes.c_int, [_P, _P]),
    ("lens_field", ctypes.c_int, [_P, _P, ctypes.c_float, _P]),
    ("contour_segments", ctypes.c_int, [_P, _P, ctypes.c_float, _P]),
    ("advect_samples", ctypes.c_int, [_P, _P, ctypes.c_int64]),
    ("regularize", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, _P]),
    ("regularize_host", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, _P]),
    ("quality_metrics", ctypes.c_int, [_P, _P]),
    ("declutter_counts", ctypes.c_int, [_P, _P]),
    ("regularize_adaptive", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    ("transition_positions", ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_float, _P]),
    ("layout_metrics", ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    ("warp_texture", ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    ("transfer_function", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, _P, _P]),
    ("declutter_sync", ctypes.c_int, [_P]),
    ("declutter_profile_regularize", ctypes.c_int,
     [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    ("integral_images_u32_noalloc", ctypes.c_int, [_P, ctypes.c_uint32, _P, _P, _P]),
    ("declutter_batch_create", ctypes.c_int,
     [ctypes.POINTER(dc_params), _P, _P, ctypes.c_int32, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    ("declutter_batch_destroy", ctypes.c_int, [_P]),
    ("declutter_batch_regularize", ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P]),
    ("declutter_batch_sync", ctypes.c_int, [_P]),
    ("declutter_autotune_band_rows", ctypes.c_int,
     [ctypes.POINTER(dc_params), ctypes.c_int, _P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P]),
    ("declutter_batch_autotune", ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P]),
    ("declutter_autotune", ctypes.c_int,
     [ctypes.POINTER(dc_params), ctypes.c_int, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(dc_params), _P]),
    ("declutter_autotune_save", ctypes.c_int, [ctypes.c_char_p]),
    ("declutter_autotune_load", ctypes.c_int, [ctypes.c_char_p]),
    ("declutter_autotune_clear", ctypes.c_int, []),
    ("regularize_tracers", ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32]),
    ("surrogate_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_uint64, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    ("surrogate_set_skip", ctypes.c_int, [_P, ctypes.c_float]),
    ("surrogate_set_tensor_path", ctypes.c_int, [_P, ctypes.c_int32]),
    ("surrogate_destroy", ctypes.c_int, [_P]),
    ("surrogate_num_params", ctypes.c_int, [_P, _P, _P]),
    ("surrogate_get_params", ctypes.c_int, [_P, _P, _P]),
    ("surrogate_set_params", ctypes.c_int, [_P, _P, _P]),
    ("surrogate_get_grads", ctypes.c_int, [_P, _P, _P]),
    ("surrogate_forward", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, _P]),
    ("surrogate_loss_grad", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    ("surrogate_train_step", ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_float, _P]),
    ("surrogate_apply", ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_int32, _P, _P]),
    ("declutter_kernel_name", ctypes.c_char_p, [ctypes.c_int32]),
    ("declutter_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("declutter_last_error", ctypes.c_char_p, []),
]


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return [s[0] for s in _SIGS]


def declutter_status_string(status: int) -> str:
    return load_library().declutter_status_string(int(status)).decode()


def declutter_last_error() -> str:
    return load_library().declutter_last_error().decode()


def declutter_kernel_name(k: int):
    r = load_library().declutter_kernel_name(int(k))
    return None if r is None else r.decode()


def _check(status: int, where: str):
    if status != 0:
        raise DeclutterError(status, where, f"{declutter_status_string(status)}: {declutter_last_error()}")


def _ptr(t, dtype=None, numel=None, name="tensor", device=None):
    """Device pointer of a CUDA tensor (or None -> NULL); with ``device``,
    the tensor must live on that CUDA device."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if device is not None and t.device.index != int(device):
        raise ValueError(f"{name} is on {t.device}, expected cuda:{int(device)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Context:
    """Owner of a ``dc_ctx*``; call :func:`declutter_destroy` (or use ``with``)."""
    handle: ctypes.c_void_p
    params: dc_params
    device: int

    @property
    def N(self) -> int:
        return 1 << int(self.params.log2_res)

    def info(self) -> dc_info:
        return declutter_get_info(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        declutter_destroy(self)


def make_params(log2_res: int, kernel_r: int = -1, sigma: float = 0.0, d0: float = -1.0,
                pixel_center: bool = False, clamp_positions: bool = True,
                carry_mode: int = DC_CARRY_COMPENSATED, band_rows: int = 0, keep_order: bool = False,
                options: int = 0, wait_limit_us: int = 0) -> dc_params:
    p = dc_params()
    p.log2_res = int(log2_res)
    p.kernel_r = int(kernel_r)
    p.sigma = float(sigma)
    p.d0 = float(d0)
    p.pixel_center = int(bool(pixel_center))
    p.clamp_positions = int(bool(clamp_positions))
    p.carry_mode = int(carry_mode)
    p.band_rows = int(band_rows)
    p.keep_order = int(bool(keep_order))
    p.options = int(options)
    p.wait_limit_us = int(wait_limit_us)
    return p


def _stream_ptr(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    sp = getattr(stream, "cuda_stream", stream) or 0
    return ctypes.c_void_p(sp) if sp else None


def declutter_create(log2_res: int, kernel_r: int = -1, sigma: float = 0.0, d0: float = -1.0,
                     pixel_center: bool = False, clamp_positions: bool = True,
                     carry_mode: int = DC_CARRY_COMPENSATED, band_rows: int = 0, keep_order: bool = False,
                     options: int = 0, wait_limit_us: int = 0, device: int | None = None, stream=None) -> Context:
    """Create a context.  ``stream``: a ``torch.cuda.Stream`` or None for the
    current torch stream (the library makes its own stream, ordered with the
    legacy default stream, when that is the default stream)."""
    import torch
    lib = load_library()
    if device is None:
        device = torch.cuda.current_device()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    sp = getattr(stream, "cuda_stream", stream) or 0
    p = make_params(log2_res, kernel_r, sigma, d0, pixel_center, clamp_positions, carry_mode, band_rows, keep_order,
                    options, wait_limit_us)
    h = ctypes.c_void_p()
    _check(lib.declutter_create(ctypes.byref(p), int(device), ctypes.c_void_p(sp) if sp else None,
                                ctypes.byref(h)), "declutter_create")
    return Context(h, p, int(device))


def declutter_destroy(ctx: Context) -> None:
    if ctx.handle:
        _check(load_library().declutter_destroy(ctx.handle), "declutter_destroy")
        ctx.handle = ctypes.c_void_p()


def declutter_get_info(ctx: Context) -> dc_info:
    out = dc_info()
    _check(load_library().declutter_get_info(ctx.handle, ctypes.byref(out)), "declutter_get_info")
    return out


def _pos_args(pos, device=None, name="pos"):
    import torch
    if pos.dim() != 2 or pos.shape[1] != 2:
        raise ValueError(f"{name} must have shape [n, 2]")
    return _ptr(pos, torch.float32, name=name, device=device), int(pos.shape[0])


def splat_density(ctx: Context, pos, counts_out=None, density_out=None) -> None:
    import torch
    pp, n = _pos_args(pos, ctx.device)
    NN = ctx.N * ctx.N
    _check(load_library().splat_density(ctx.handle, pp, n,
                                        _ptr(counts_out, torch.int32, NN, "counts_out", ctx.device),
                                        _ptr(density_out, torch.float32, NN, "density_out", ctx.device)), "splat_density")


def splat_counts(ctx: Context, pos, counts_out) -> None:
    """This shard's counts (uint32 bit patterns) into the CUDA int32 tensor
    ``counts_out`` of N*N elements."""
    import torch
    pp, n = _pos_args(pos, ctx.device)
    _check(load_library().splat_counts(ctx.handle, pp, n, _ptr(counts_out, torch.int32, ctx.N * ctx.N, "counts_out",
                                                               ctx.device)), "splat_counts")


def density_from_counts(ctx: Context, counts, n_total: int) -> None:
    """The summed count grid of all ``n_total`` samples (CUDA int32, N*N) as
    the context's density."""
    import torch
    _check(load_library().density_from_counts(ctx.handle, _ptr(counts, torch.int32, ctx.N * ctx.N, "counts",
                                                               ctx.device), int(n_total)), "density_from_counts")


def _u64(t, NN, name, device=None):
    import torch
    if t is None:
        return None
    if t.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise TypeError(f"{name} must be a 64-bit integer tensor")
    return _ptr(t, None, NN, name, device)


def integral_images(ctx: Context, alpha_out=None, alpha_t_out=None) -> None:
    """Exact mode: int64/uint64 outputs; float mode: float32 outputs."""
    import torch
    NN = ctx.N * ctx.N
    if int(ctx.params.kernel_r) == 0:
        a, b = _u64(alpha_out, NN, "alpha_out", ctx.device), _u64(alpha_t_out, NN, "alpha_t_out", ctx.device)
    else:
        a = _ptr(alpha_out, torch.float32, NN, "alpha_out", ctx.device)
        b = _ptr(alpha_t_out, torch.float32, NN, "alpha_t_out", ctx.device)
    _check(load_library().integral_images(ctx.handle, a, b), "integral_images")


def integral_images_u32(ctx: Context, grid, alpha_out=None, alpha_t_out=None) -> None:
    """``grid``: CUDA int32 tensor holding uint32 bit patterns, N*N."""
    import torch
    NN = ctx.N * ctx.N
    g = _ptr(grid, torch.int32, NN, "grid", ctx.device)
    _check(load_library().integral_images_u32(ctx.handle, g, _u64(alpha_out, NN, "alpha_out", ctx.device),
                                              _u64(alpha_t_out, NN, "alpha_t_out", ctx.device)), "integral_images_u32")


def displacement_field(ctx: Context, disp_out=None) -> None:
    import torch
    _check(load_library().displacement_field(ctx.handle, _ptr(disp_out, torch.float32, 2 * ctx.N * ctx.N,
                                                              "disp_out", ctx.device)), "displacement_field")


def lens_field(ctx: Context, density, density_mean: float = 0.0, disp_out=None) -> None:
    """The lens mapping t(x, y; d) - (x, y) of a CUDA float32 density [N, N]
    into the context's field (and ``disp_out``, float32 2*N*N, if given)."""
    import torch
    NN = ctx.N * ctx.N
    _check(load_library().lens_field(ctx.handle, _ptr(density, torch.float32, NN, "density", ctx.device), float(density_mean),
                                     _ptr(disp_out, torch.float32, 2 * NN, "disp_out", ctx.device)), "lens_field")


def contour_segments(ctx: Context, field, level: float, segs_out) -> None:
    """Marching squares of a CUDA float32 field [N, N] at ``level`` into
    ``segs_out`` (CUDA float32, 8 (N-1)^2 values: two (x0, y0, x1, y1) slots a
    cell, NaN when unused)."""
    import torch
    M = ctx.N - 1
    _check(load_library().contour_segments(ctx.handle, _ptr(field, torch.float32, ctx.N * ctx.N, "field", ctx.device),
                                           float(level), _ptr(segs_out, torch.float32, 8 * M * M, "segs_out", ctx.device)),
           "contour_segments")


def advect_samples(ctx: Context, pos) -> None:
    pp, n = _pos_args(pos, ctx.device)
    _check(load_library().advect_samples(ctx.handle, pp, n), "advect_samples")


def regularize(ctx: Context, pos, iters: int, uniformity: bool = False):
    pp, n = _pos_args(pos, ctx.device)
    out = (ctypes.c_double * max(int(iters), 1))() if uniformity else None
    _check(load_library().regularize(ctx.handle, pp, n, int(iters), out), "regularize")
    return list(out)[:iters] if uniformity else None


def regularize_host(ctx: Context, host_pos, iters: int, uniformity: bool = False):
    """``host_pos``: numpy float32 [n, 2] or a CPU torch tensor (pinned for
    asynchronous copies); updated in place."""
    if isinstance(host_pos, np.ndarray):
        if host_pos.dtype != np.float32 or not host_pos.flags["C_CONTIGUOUS"]:
            raise TypeError("host_pos must be C-contiguous float32")
        ptr, n = host_pos.ctypes.data, host_pos.shape[0]
    else:
        if host_pos.is_cuda or not host_pos.is_contiguous():
            raise TypeError("host_pos must be a contiguous CPU tensor")
        ptr, n = host_pos.data_ptr(), host_pos.shape[0]
    out = (ctypes.c_double * max(int(iters), 1))() if uniformity else None
    _check(load_library().regularize_host(ctx.handle, ctypes.c_void_p(ptr), int(n), int(iters), out),
           "regularize_host")
    return list(out)[:iters] if uniformity else None


def regularize_adaptive(ctx: Context, pos, max_iters: int, target_cv: float = 0.0, min_move_px: float = 0.0,
                        max_ms: float = 0.0) -> dict:
    """Iterate until a stopping criterion holds (see the C header); returns
    ``{"iters": k, "cv": [...], "move_px": [...]}`` for the k iterations done."""
    pp, n = _pos_args(pos, ctx.device)
    it = ctypes.c_int32()
    cv = (ctypes.c_double * max(int(max_iters), 1))()
    mv = (ctypes.c_double * max(int(max_iters), 1))()
    _check(load_library().regularize_adaptive(ctx.handle, pp, n, int(max_iters), float(target_cv),
                                              float(min_move_px), float(max_ms), ctypes.byref(it), cv, mv),
           "regularize_adaptive")
    k = int(it.value)
    return {"iters": k, "cv": list(cv)[:k], "move_px": list(mv)[:k]}


def transition_positions(ctx: Context, from_pos, to_pos, s: float, out) -> None:
    """out = (1 - s) from + s to for CUDA float32 [n, 2] tensors."""
    fp, n = _pos_args(from_pos, ctx.device, "from_pos")
    tp, n2 = _pos_args(to_pos, ctx.device, "to_pos")
    op, n3 = _pos_args(out, ctx.device, "out")
    if not (n == n2 == n3):
        raise ValueError("from_pos, to_pos and out must have the same shape")
    _check(load_library().transition_positions(ctx.handle, fp, tp, n, float(s), op), "transition_positions")


def layout_metrics(ctx: Context, orig, reg, k: int, queries=None, n_queries: int | None = None,
                   want_terms: bool = False) -> dict:
    """Trustworthiness and orthogonal ordering of ``reg`` against ``orig``
    (CUDA float32 [n, 2]) over the query samples: ``queries`` a CUDA int32
    tensor of indices, or None for the first ``n_queries`` samples (all when
    None).  Returns ``{"trustworthiness": T, "ordering": O}`` (+ ``"terms"``,
    int64 [m, 2], with ``want_terms``)."""
    import torch
    op, n = _pos_args(orig, ctx.device, "orig")
    rp, n2 = _pos_args(reg, ctx.device, "reg")
    if n != n2:
        raise ValueError("orig and reg must have the same shape")
    if queries is not None:
        m = int(queries.numel())
        qp = _ptr(queries, torch.int32, m, "queries", ctx.device)
    else:
        m = int(n if n_queries is None else n_queries)
        qp = None
    out = (ctypes.c_double * 2)()
    terms = np.zeros((m, 2), np.int64) if want_terms else None
    _check(load_library().layout_metrics(ctx.handle, op, rp, n, qp, m, int(k), out,
                                         terms.ctypes.data_as(ctypes.c_void_p) if want_terms else None),
           "layout_metrics")
    res = {"trustworthiness": out[0], "ordering": out[1]}
    if want_terms:
        res["terms"] = terms
    return res


def warp_texture(ctx: Context, nodes, texture, out_log2: int, out, mass: bool = False, tri_out=None) -> None:
    """Draw ``texture`` (CUDA float32, N*N values at the pixel nodes) on the
    mesh of the moved nodes ``nodes`` (CUDA float32 [N*N, 2]) into ``out``
    (CUDA float32, M*M, M = 2^out_log2); ``tri_out`` (CUDA int32 M*M) gets
    the winning triangle per pixel (-1: none)."""
    import torch
    NN = ctx.N * ctx.N
    MM = 1 << (2 * int(out_log2))
    np_, nn = _pos_args(nodes, ctx.device, "nodes")
    if nn != NN:
        raise ValueError(f"nodes must have {NN} rows")
    _check(load_library().warp_texture(ctx.handle, np_, _ptr(texture, torch.float32, NN, "texture", ctx.device),
                                       int(out_log2), DC_WARP_MASS if mass else DC_WARP_VALUE,
                                       _ptr(out, torch.float32, MM, "out", ctx.device),
                                       _ptr(tri_out, torch.int32, MM, "tri_out", ctx.device)), "warp_texture")


def transfer_function(ctx: Context, values, lo: float, hi: float, lut, rgba_out) -> None:
    """RGBA8 colours (CUDA int32 bit patterns) of CUDA float32 ``values``
    through the 256-entry table ``lut`` (CUDA int32)."""
    import torch
    n = int(values.numel())
    _check(load_library().transfer_function(ctx.handle, _ptr(values, torch.float32, None, "values", ctx.device), n,
                                            float(lo), float(hi), _ptr(lut, torch.int32, 256, "lut", ctx.device),
                                            _ptr(rgba_out, torch.int32, n, "rgba_out", ctx.device)),
           "transfer_function")


def declutter_counts(ctx: Context, counts_out) -> None:
    """Copy the context's current count grid (uint32 bit patterns) into the
    CUDA int32 tensor ``counts_out`` of N*N elements."""
    import torch
    _check(load_library().declutter_counts(ctx.handle, _ptr(counts_out, torch.int32, ctx.N * ctx.N, "counts_out",
                                                            ctx.device)), "declutter_counts")


def quality_metrics(ctx: Context) -> dict:
    out = (ctypes.c_double * 3)()
    _check(load_library().quality_metrics(ctx.handle, out), "quality_metrics")
    return {"bin_std": out[0], "bin_cv": out[1], "overplot": out[2]}


def declutter_sync(ctx: Context) -> None:
    _check(load_library().declutter_sync(ctx.handle), "declutter_sync")


def declutter_profile_regularize(ctx: Context, pos, iters: int, reps: int = 10, reset_src=None) -> dict:
    """In-graph device time of regularize(iters) and of each kernel kind in
    it (see the C header).  Returns ``{"step_ms": t, "kernels": {name:
    {"ms": per call, "launches": per call}}}``."""
    pp, n = _pos_args(pos, ctx.device)
    src = None
    if reset_src is not None:
        src, n2 = _pos_args(reset_src, ctx.device)
        if n2 != n:
            raise ValueError("reset_src must have the shape of pos")
    step = ctypes.c_float()
    ms = (ctypes.c_float * KERNEL_KINDS)()
    cnt = (ctypes.c_int32 * KERNEL_KINDS)()
    _check(load_library().declutter_profile_regularize(ctx.handle, pp, src, n, int(iters), int(reps),
                                                       ctypes.byref(step), ms, cnt),
           "declutter_profile_regularize")
    return {"step_ms": float(step.value),
            "kernels": {declutter_kernel_name(k): {"ms": float(ms[k]), "launches": int(cnt[k])}
                        for k in range(KERNEL_KINDS)}}


def integral_images_u32_noalloc(grid, log2_res: int, alpha_out=None, alpha_t_out=None, stream=None) -> None:
    """No-allocation integral images of a uint32 grid (int32 CUDA tensor
    holding the bit patterns); for callers that cannot allocate device
    memory at call time.  ``stream``: a ``torch.cuda.Stream`` or None for the
    current torch stream."""
    import torch
    NN = 1 << (2 * int(log2_res))
    g = _ptr(grid, torch.int32, NN, "grid")
    dev = grid.device.index
    a = _u64(alpha_out, NN, "alpha_out", dev)
    at = _u64(alpha_t_out, NN, "alpha_t_out", dev)
    # the C call runs on the calling thread's current device: make it the grid's
    with torch.cuda.device(grid.device):
        if stream is None:
            stream = torch.cuda.current_stream(grid.device)
        sp = getattr(stream, "cuda_stream", stream) or 0
        _check(load_library().integral_images_u32_noalloc(g, int(log2_res), a, at,
                                                          ctypes.c_void_p(sp) if sp else None),
               "integral_images_u32_noalloc")


@dataclass
class Batch:
    """Owner of a ``dc_batch*`` (panels of a scatterplot matrix)."""
    handle: ctypes.c_void_p
    log2_res: list
    max_samples: list
    device: int

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        declutter_batch_destroy(self)


def declutter_batch_create(log2_res, max_samples, device: int | None = None, stream=None, **params) -> Batch:
    """``log2_res``, ``max_samples``: per-panel lists; ``params``: as for
    :func:`declutter_create` (its log2_res is per panel here)."""
    import torch
    if device is None:
        device = torch.cuda.current_device()
    P = len(log2_res)
    if len(max_samples) != P:
        raise ValueError("log2_res and max_samples differ in length")
    p = make_params(0, **params)
    l2 = (ctypes.c_uint32 * P)(*[int(x) for x in log2_res])
    ms = (ctypes.c_int64 * P)(*[int(x) for x in max_samples])
    h = ctypes.c_void_p()
    _check(load_library().declutter_batch_create(ctypes.byref(p), l2, ms, P, int(device),
                                                 _stream_ptr(stream, device), ctypes.byref(h)),
           "declutter_batch_create")
    return Batch(h, list(log2_res), list(max_samples), int(device))


def declutter_batch_destroy(batch: Batch) -> None:
    if batch.handle:
        _check(load_library().declutter_batch_destroy(batch.handle), "declutter_batch_destroy")
        batch.handle = ctypes.c_void_p()


def _batch_arrays(positions):
    P = len(positions)
    ptrs = (ctypes.c_void_p * P)()
    ns = (ctypes.c_int64 * P)()
    for k, t in enumerate(positions):
        pp, n = _pos_args(t)
        ptrs[k] = pp
        ns[k] = n
    return ptrs, ns


def declutter_batch_regularize(batch: Batch, positions, iters: int, uniformity: bool = False):
    """``positions``: list of CUDA float32 [n_p, 2] tensors, one per panel."""
    P = len(positions)
    ptrs, ns = _batch_arrays(positions)
    out = (ctypes.c_double * max(P * int(iters), 1))() if uniformity else None
    _check(load_library().declutter_batch_regularize(batch.handle, ptrs, ns, int(iters), out),
           "declutter_batch_regularize")
    if not uniformity:
        return None
    return [list(out[p * iters:(p + 1) * iters]) for p in range(P)]


def declutter_batch_sync(batch: Batch) -> None:
    _check(load_library().declutter_batch_sync(batch.handle), "declutter_batch_sync")


def declutter_autotune_band_rows(pos, iters: int, log2_res: int, device: int | None = None, stream=None,
                                 **params):
    """Fastest band height for ``regularize(iters)`` on these samples:
    returns ``(band_rows, median_ms or -1 if cached)``."""
    import torch
    if device is None:
        device = torch.cuda.current_device()
    p = make_params(log2_res, **params)
    pp, n = _pos_args(pos)
    best = ctypes.c_int32()
    ms = ctypes.c_float()
    _check(load_library().declutter_autotune_band_rows(ctypes.byref(p), int(device), _stream_ptr(stream, device), pp,
                                                       n, int(iters), ctypes.byref(best), ctypes.byref(ms)),
           "declutter_autotune_band_rows")
    return int(best.value), float(ms.value)


def declutter_autotune(pos, iters: int, log2_res: int, device: int | None = None, stream=None, **params):
    """Tuned band height and launch options for these samples: returns
    ``(band_rows, options, median_ms)`` (median -1 when cached)."""
    import torch
    lib = load_library()
    if device is None:
        device = torch.cuda.current_device()
    pp, n = _pos_args(pos, device)
    p = make_params(log2_res, **params)
    best = dc_params()
    ms = ctypes.c_float()
    _check(lib.declutter_autotune(ctypes.byref(p), int(device), _stream_ptr(stream, device), pp, n, int(iters),
                                  ctypes.byref(best), ctypes.byref(ms)), "declutter_autotune")
    return int(best.band_rows), int(best.options), float(ms.value)


def declutter_autotune_save(path: str) -> None:
    _check(load_library().declutter_autotune_save(os.fsencode(path)), "declutter_autotune_save")


def declutter_autotune_load(path: str) -> None:
    _check(load_library().declutter_autotune_load(os.fsencode(path)), "declutter_autotune_load")


def declutter_autotune_clear() -> None:
    _check(load_library().declutter_autotune_clear(), "declutter_autotune_clear")


def declutter_batch_autotune(batch: Batch, positions, iters: int):
    P = len(positions)
    ptrs, ns = _batch_arrays(positions)
    out = (ctypes.c_int32 * P)()
    _check(load_library().declutter_batch_autotune(batch.handle, ptrs, ns, int(iters), out),
           "declutter_batch_autotune")
    return list(out)


def regularize_tracers(ctx: Context, pos, tracers, iters: int) -> None:
    """``regularize`` that also moves ``tracers`` (CUDA float32 [m, 2]) by each
    iteration's field without splatting them."""
    pp, n = _pos_args(pos, ctx.device)
    tp, nt = _pos_args(tracers, ctx.device)
    _check(load_library().regularize_tracers(ctx.handle, pp, n, tp, nt, int(iters)), "regularize_tracers")


@dataclass
class Surrogate:
    """Owner of a ``dc_surrogate*``."""
    handle: ctypes.c_void_p
    log2_res: int
    levels: int
    base_channels: int
    max_batch: int
    device: int
    in_channels: int = 1

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        surrogate_destroy(self)


def surrogate_create(log2_res: int, levels: int = 4, base_channels: int = 32, max_batch: int = 16, seed: int = 0,
                     device: int | None = None, stream=None, in_channels: int = 1) -> Surrogate:
    """``in_channels``: 1 (density) or 3 (density and one plain iteration's field)."""
    import torch
    if device is None:
        device = torch.cuda.current_device()
    h = ctypes.c_void_p()
    _check(load_library().surrogate_create(int(log2_res), int(levels), int(base_channels), int(in_channels),
                                           int(max_batch), int(seed), int(device), _stream_ptr(stream, device),
                                           ctypes.byref(h)), "surrogate_create")
    return Surrogate(h, int(log2_res), int(levels), int(base_channels), int(max_batch), int(device), int(in_channels))


def surrogate_set_skip(sg: Surrogate, kappa: float) -> None:
    _check(load_library().surrogate_set_skip(sg.handle, float(kappa)), "surrogate_set_skip")


def surrogate_set_tensor_path(sg: Surrogate, path: int) -> None:
    """``DC_SG_MMA_SYNC``, ``DC_SG_TCGEN05`` or ``DC_SG_AUTO`` (default: tcgen05
    for batches of two or more samples) for the forward convolutions of
    64..256 output channels."""
    _check(load_library().surrogate_set_tensor_path(sg.handle, int(path)), "surrogate_set_tensor_path")


def surrogate_destroy(sg: Surrogate) -> None:
    if sg.handle:
        _check(load_library().surrogate_destroy(sg.handle), "surrogate_destroy")
        sg.handle = ctypes.c_void_p()


def surrogate_num_params(sg: Surrogate):
    nw, nb = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().surrogate_num_params(sg.handle, ctypes.byref(nw), ctypes.byref(nb)), "surrogate_num_params")
    return int(nw.value), int(nb.value)


def surrogate_get_params(sg: Surrogate):
    nw, nb = surrogate_num_params(sg)
    w = np.empty(nw, np.float32)
    b = np.empty(nb, np.float32)
    _check(load_library().surrogate_get_params(sg.handle, w.ctypes.data, b.ctypes.data), "surrogate_get_params")
    return w, b


def surrogate_set_params(sg: Surrogate, w, b) -> None:
    w = np.ascontiguousarray(w, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    nw, nb = surrogate_num_params(sg)
    if w.size != nw or b.size != nb:
        raise ValueError("parameter sizes")
    _check(load_library().surrogate_set_params(sg.handle, w.ctypes.data, b.ctypes.data), "surrogate_set_params")


def surrogate_get_grads(sg: Surrogate):
    nw, nb = surrogate_num_params(sg)
    w = np.empty(nw, np.float32)
    b = np.empty(nb, np.float32)
    _check(load_library().surrogate_get_grads(sg.handle, w.ctypes.data, b.ctypes.data), "surrogate_get_grads")
    return w, b


def _grid_arg(t, batch, H, ch, name):
    import torch
    return _ptr(t, torch.float32, batch * H * H * ch, name)


def _scales_arg(scales, batch):
    import torch
    if scales is None:
        return None
    return _ptr(scales, torch.float32, batch, "scales")


def _field_arg(field, B, H):
    return _grid_arg(field, B, H, 2, "field") if field is not None else None


def surrogate_forward(sg: Surrogate, density, scales=None, out=None, field=None) -> None:
    """``density``: CUDA float32 [B, H, W]; ``scales``: CUDA float32 [B] or None;
    ``field``: CUDA float32 [B, H, W, 2] (pixels), required with in_channels = 3."""
    B = density.shape[0]
    H = 1 << sg.log2_res
    _check(load_library().surrogate_forward(sg.handle, _grid_arg(density, B, H, 1, "density"), _scales_arg(scales, B),
                                            _field_arg(field, B, H), B,
                                            _grid_arg(out, B, H, 2, "out") if out is not None else None),
           "surrogate_forward")


def surrogate_loss_grad(sg: Surrogate, density, scales, target, field=None) -> float:
    B = density.shape[0]
    H = 1 << sg.log2_res
    loss = ctypes.c_float()
    _check(load_library().surrogate_loss_grad(sg.handle, _grid_arg(density, B, H, 1, "density"),
                                              _scales_arg(scales, B), _field_arg(field, B, H),
                                              _grid_arg(target, B, H, 2, "target"), B, ctypes.byref(loss)),
           "surrogate_loss_grad")
    return float(loss.value)


def surrogate_train_step(sg: Surrogate, density, scales, target, lr: float, want_loss: bool = True, field=None):
    B = density.shape[0]
    H = 1 << sg.log2_res
    loss = ctypes.c_float()
    _check(load_library().surrogate_train_step(sg.handle, _grid_arg(density, B, H, 1, "density"),
                                               _scales_arg(scales, B), _field_arg(field, B, H),
                                               _grid_arg(target, B, H, 2, "target"), B, float(lr),
                                               ctypes.byref(loss) if want_loss else None), "surrogate_train_step")
    return float(loss.value) if want_loss else None


def surrogate_apply(ctx: Context, sg: Surrogate, pos, target_cv: float, max_plain_iters: int):
    pp, n = _pos_args(pos, ctx.device)
    used = ctypes.c_int32()
    cv = ctypes.c_double()
    _check(load_library().surrogate_apply(ctx.handle, sg.handle, pp, n, float(target_cv), int(max_plain_iters),
                                          ctypes.byref(used), ctypes.byref(cv)), "surrogate_apply")
    return int(used.value), float(cv.value)
