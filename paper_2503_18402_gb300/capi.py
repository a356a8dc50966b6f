"""ctypes binding of the C ABI in include/dashgs.h (argument marshalling only).

Every function has the C name and argument order; tensor arguments may be
torch tensors (their data_ptr is passed) or raw integer device addresses.
A non-zero status raises ``DashGSError`` with the library's message.  Import
fails loudly when the CUDA library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_LIB_PATH = _build.LIB
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"CUDA library {_LIB_PATH} is missing: run paper_2503_18402_gb300.build.build() "
                      "(there is no CPU fallback)")
_lib = ctypes.CDLL(_LIB_PATH)

NPARAM = 59
FEAT_FLOATS = 12
DG_OK, DG_ERR_ARG, DG_ERR_CAPACITY, DG_ERR_TIMEOUT, DG_ERR_CUDA = 0, -1, -2, -3, -4

MAX_VIEWS = 16
EXPORTS = ("dg_last_error", "dg_abi_version", "dg_kernel_launches", "dg_project", "dg_bin_workspace_size", "dg_bin_count",
           "dg_bin_sort", "dg_lookback_probe", "dg_render_workspace_size", "dg_render_fwd", "dg_render_bwd", "dg_pack_records", "dg_project_bwd", "dg_project_bwd_adam",
           "dg_project_bwd_adam_dev",
           "dg_loss_workspace_size", "dg_ssim_workspace_size", "dg_loss_l1_dssim",
           "dg_loss_l1", "dg_loss_l1_noalloc", "dg_adam_step", "dg_adam_hparams_fill", "dg_adam_step_dev",
           "dg_sparse_adam_step", "dg_visibility", "dg_spectrum_workspace_size",
           "dg_spectrum_accumulate", "dg_spectrum_finalize", "dg_downsample_area", "dg_schedule_init",
           "dg_schedule_step", "dg_schedule_densify", "dg_schedule_init_plain", "dg_densify_budget",
           "dg_camera_scale", "dg_batch_adam_scale", "dg_densify_stats", "dg_densify_workspace_size",
           "dg_densify_mark", "dg_densify_apply", "dg_mse", "dg_opacity_reset")
L1_NOALLOC_MAX_N = 1024 * 256 * 1024


class DashGSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dashgs status {status}: {msg}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class RasterOpts(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("near_plane", ctypes.c_float),
                ("eps2d", ctypes.c_float), ("bg", ctypes.c_float * 3), ("pixels_per_thread", ctypes.c_int32),
                ("split_len", ctypes.c_int32), ("record", ctypes.c_int32), ("mip2d", ctypes.c_float),
                ("tight_bins", ctypes.c_int32)]


SCHED_MAX_LEVELS = 64


class SchedParams(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int64), ("a", ctypes.c_double), ("m", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("eta", ctypes.c_double), ("P_init", ctypes.c_double),
                ("P_cap", ctypes.c_double), ("lr_pos_init", ctypes.c_double), ("lr_pos_final", ctypes.c_double)]


class Schedule(ctypes.Structure):
    _fields_ = [("p", SchedParams), ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("m", ctypes.c_int32),
                ("X0", ctypes.c_double), ("Xm", ctypes.c_double), ("r_m", ctypes.c_double),
                ("X", ctypes.c_double * (SCHED_MAX_LEVELS + 1)), ("r", ctypes.c_double * (SCHED_MAX_LEVELS + 1)),
                ("s", ctypes.c_double * (SCHED_MAX_LEVELS + 1)), ("k_full", ctypes.c_int64), ("P_fin", ctypes.c_double)]


class SchedOut(ctypes.Structure):
    _fields_ = [("r_cont", ctypes.c_double), ("r_mod", ctypes.c_int32), ("height", ctypes.c_int32),
                ("width", ctypes.c_int32), ("lr_pos", ctypes.c_double), ("P_target", ctypes.c_double)]


class DensifyOpts(ctypes.Structure):
    _fields_ = [("grad_thresh", ctypes.c_float), ("min_opacity", ctypes.c_float), ("percent_dense", ctypes.c_float),
                ("extent", ctypes.c_float), ("max_screen_radius", ctypes.c_float), ("max_world_scale", ctypes.c_float)]


def densify_opts(grad_thresh=0.0002, min_opacity=0.005, percent_dense=0.01, extent=1.0, max_screen_radius=0.0,
                 max_world_scale=0.0) -> DensifyOpts:
    return DensifyOpts(grad_thresh, min_opacity, percent_dense, extent, max_screen_radius, max_world_scale)


def sched_params(S, a=4.0, m=0, gamma=0.98, eta=1.0, P_init=1e5, P_cap=3e6, lr_pos_init=1.6e-4,
                 lr_pos_final=1.6e-6) -> SchedParams:
    return SchedParams(int(S), float(a), int(m), float(gamma), float(eta), float(P_init), float(P_cap),
                       float(lr_pos_init), float(lr_pos_final))


def camera(viewmat, fx, fy, cx, cy, width, height) -> Camera:
    c = Camera()
    vm = [float(x) for row in viewmat for x in row] if hasattr(viewmat[0], "__len__") else [float(x) for x in viewmat]
    assert len(vm) == 12
    c.viewmat[:] = vm
    c.fx, c.fy, c.cx, c.cy = float(fx), float(fy), float(cx), float(cy)
    c.width, c.height = int(width), int(height)
    return c


def raster_opts(tile=16, sh_degree=3, near_plane=0.2, eps2d=0.3, bg=(0.0, 0.0, 0.0),
                pixels_per_thread=0, split_len=0, record=0, mip2d=0.0, tight_bins=0) -> RasterOpts:
    o = RasterOpts()
    o.tile, o.sh_degree, o.near_plane, o.eps2d = int(tile), int(sh_degree), float(near_plane), float(eps2d)
    o.bg[:] = [float(b) for b in bg]
    o.pixels_per_thread = int(pixels_per_thread)
    o.split_len = int(split_len)
    o.record = int(record)
    o.mip2d = float(mip2d)
    o.tight_bins = int(tight_bins)
    return o


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_F = ctypes.c_float
_SZ = ctypes.c_size_t
_ST = ctypes.c_int32
_CAM = ctypes.POINTER(Camera)
_OPT = ctypes.POINTER(RasterOpts)

_SIGS = {
    "dg_last_error": ([], ctypes.c_char_p),
    "dg_abi_version": ([], _I32),
    "dg_kernel_launches": ([], _I64),
    "dg_project": ([_P, _I64, _I64, _CAM, _P, _I32, _OPT, _P, _P, _P, _P, _P, _P], _ST),
    "dg_bin_workspace_size": ([_I64, _I32, _I64], _SZ),
    "dg_bin_count": ([_P, _P, _I64, _I32, _P, _SZ, _I64, _P, _P], _ST),
    "dg_bin_sort": ([_P, _P, _I64, _CAM, _I32, _I32, _P, _SZ, _I64, _P, _P, _P, _P], _ST),
    "dg_lookback_probe": ([_P, _I64, _I32, _I32, _I32, _P, _P, _P], _ST),
    "dg_render_workspace_size": ([_CAM, _I32, _OPT, _I64], _SZ),
    "dg_pack_records": ([_P, _I64, _P, _P], _ST),
    "dg_render_fwd": ([_P, _P, _P, _CAM, _I32, _OPT, _P, _P, _P, _P, _P, _P, _SZ, _P], _ST),
    "dg_render_bwd": ([_P, _P, _P, _CAM, _I32, _OPT, _P, _P, _P, _I64, _P, _P, _SZ, _P], _ST),
    "dg_project_bwd": ([_P, _I64, _I64, _CAM, _P, _I32, _OPT, _P, _P, _P, _P, _P], _ST),
    "dg_project_bwd_adam": ([_P, _I64, _I64, _CAM, _P, _I32, _OPT, _P, _P, _P, _P, _P, _P, _P, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, _I64, _P], _ST),
    "dg_project_bwd_adam_dev": ([_P, _I64, _I64, _CAM, _P, _I32, _OPT, _P, _P, _P, _P, _P, _P, _P, _P, _P], _ST),
    "dg_ssim_workspace_size": ([_P, _I32], _SZ),
    "dg_loss_l1_dssim": ([_P, _P, _P, _I32, ctypes.c_float, _P, _P, _P, _SZ, _P], _ST),
    "dg_loss_workspace_size": ([_I64], _SZ),
    "dg_loss_l1": ([_P, _P, _I64, _P, _P, _P, _SZ, _P], _ST),
    "dg_loss_l1_noalloc": ([_P, _P, _I64, _P, _P, _P], _ST),
    "dg_adam_step": ([_P, _P, _P, _P, _I64, _I64, _P, _F, _F, _F, _I64, _P], _ST),
    "dg_sparse_adam_step": ([_P, _P, _P, _P, _I64, _I64, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I64,
                             _P, _P], _ST),
    "dg_visibility": ([_P, _I64, _I32, _P, _P], _ST),
    "dg_adam_hparams_fill": ([_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I64, _P], _ST),
    "dg_adam_step_dev": ([_P, _P, _P, _P, _I64, _I64, _P, _P, _P], _ST),
    "dg_spectrum_workspace_size": ([_I32, _I32], _SZ),
    "dg_spectrum_accumulate": ([_P, _I32, _I32, _P, _P, _SZ, _P], _ST),
    "dg_spectrum_finalize": ([_P, _I32, _I32, _I32, _P, _P, _P], _ST),
    "dg_downsample_area": ([_P, _I32, _I32, _I32, _P, _I32, _I32, _P], _ST),
    "dg_mse": ([_P, _P, _I64, _P, _P, _SZ, _P], _ST),
    "dg_opacity_reset": ([_P, _P, _P, _I64, _I64, _F, _P], _ST),
    "dg_densify_stats": ([_P, _P, _I64, _CAM, _I32, _P, _P, _P, _P], _ST),
    "dg_densify_workspace_size": ([_I64], _SZ),
    "dg_densify_mark": ([_P, _I64, _I64, _P, _P, _P, ctypes.POINTER(DensifyOpts), _P, _SZ, _P, _P], _ST),
    "dg_densify_apply": ([_P, _P, _P, _I64, _I64, _I64, _I64, _P, _P, _SZ, _P, _P, _P, _I64, _P, _P], _ST),
    "dg_schedule_init": ([_P, _I32, _I32, ctypes.POINTER(SchedParams), ctypes.POINTER(Schedule)], _ST),
    "dg_schedule_step": ([ctypes.POINTER(Schedule), _I64, ctypes.POINTER(SchedOut)], _ST),
    "dg_schedule_densify": ([ctypes.POINTER(Schedule), _I64, _I64, ctypes.POINTER(SchedOut)], _ST),
    "dg_schedule_init_plain": ([_I32, _I32, ctypes.POINTER(SchedParams), ctypes.POINTER(Schedule)], _ST),
    "dg_densify_budget": ([ctypes.POINTER(Schedule), _I64, _I64, _I64, _I64, ctypes.POINTER(_I64),
                           ctypes.POINTER(SchedOut)], _ST),
    "dg_camera_scale": ([_CAM, _I32, _I32, _CAM], _ST),
    "dg_batch_adam_scale": ([_I32, ctypes.POINTER(_F), ctypes.POINTER(_F), ctypes.POINTER(_F)], _ST),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def _a(x):
    """Device/host address of a tensor, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _s(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def cameras(cams) -> ctypes.Array:
    """A ctypes Camera array from one Camera or a sequence of them."""
    if isinstance(cams, ctypes.Array):
        return cams
    if isinstance(cams, Camera):
        cams = [cams]
    arr = (Camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = c
    return arr


def _c(cams):
    return ctypes.cast(cameras(cams), _CAM)


def _check(status):
    if status != DG_OK:
        raise DashGSError(status, _lib.dg_last_error().decode())


def library_path() -> str:
    return _LIB_PATH


def dg_last_error() -> str:
    return _lib.dg_last_error().decode()


def dg_abi_version() -> int:
    return _lib.dg_abi_version()


def dg_kernel_launches() -> int:
    return _lib.dg_kernel_launches()


def dg_project(params, stride, P, cams, n_views, opts, feat, depth, radius, tiles, clamp, stream=None,
               cams_dev=None):
    """cams: host cameras; cams_dev: optional device copy (read when the kernel runs)."""
    _check(_lib.dg_project(_a(params), stride, P, _c(cams), _a(cams_dev), n_views, ctypes.byref(opts), _a(feat),
                           _a(depth), _a(radius), _a(tiles), _a(clamp), _s(stream)))


def dg_bin_workspace_size(P, n_views, M_cap) -> int:
    return _lib.dg_bin_workspace_size(P, n_views, M_cap)


def dg_bin_count(depth, tiles, P, n_views, ws, ws_bytes, M_cap, M_out, stream=None):
    _check(_lib.dg_bin_count(_a(depth), _a(tiles), P, n_views, _a(ws), ws_bytes, M_cap, _a(M_out), _s(stream)))


def dg_lookback_probe(look, tile, stride, digit, max_polls, sum_out, err_out, stream=None):
    _check(_lib.dg_lookback_probe(_a(look), tile, stride, digit, max_polls, _a(sum_out), _a(err_out), _s(stream)))


LB_AGG, LB_INC = 1 << 62, 2 << 62  # look-back word states (count in the low 62 bits)


def dg_bin_sort(feat, radius, P, cams, n_views, tile, ws, ws_bytes, M_cap, gid, ranges, status, stream=None):
    _check(_lib.dg_bin_sort(_a(feat), _a(radius), P, _c(cams), n_views, tile, _a(ws), ws_bytes, M_cap, _a(gid),
                            _a(ranges), _a(status), _s(stream)))


def dg_render_workspace_size(cams, n_views, opts, M_cap=0) -> int:
    return _lib.dg_render_workspace_size(_c(cams), n_views, ctypes.byref(opts), M_cap)


PACKED_RECORD_BYTES = 24


def dg_pack_records(feat, n_records, packed, stream=None):
    _check(_lib.dg_pack_records(_a(feat), n_records, _a(packed), _s(stream)))


def dg_render_fwd(feat, gid, ranges, cams, n_views, opts, img, T_final, last, examined, blended, ws, ws_bytes,
                  stream=None):
    _check(_lib.dg_render_fwd(_a(feat), _a(gid), _a(ranges), _c(cams), n_views, ctypes.byref(opts), _a(img),
                              _a(T_final), _a(last), _a(examined), _a(blended), _a(ws), ws_bytes, _s(stream)))


def dg_render_bwd(feat, gid, ranges, cams, n_views, opts, T_final, last, dL_dimg, n_records, grad2d, ws, ws_bytes,
                  stream=None):
    _check(_lib.dg_render_bwd(_a(feat), _a(gid), _a(ranges), _c(cams), n_views, ctypes.byref(opts), _a(T_final),
                              _a(last), _a(dL_dimg), n_records, _a(grad2d), _a(ws), ws_bytes, _s(stream)))


def dg_project_bwd(params, stride, P, cams, n_views, opts, radius, clamp, grad2d, grads, stream=None, cams_dev=None):
    _check(_lib.dg_project_bwd(_a(params), stride, P, _c(cams), _a(cams_dev), n_views, ctypes.byref(opts), _a(radius),
                               _a(clamp), _a(grad2d), _a(grads), _s(stream)))


def dg_project_bwd_adam(params, stride, P, cams, n_views, opts, radius, clamp, grad2d, grads, m, v, lr, beta1,
                        beta2, eps, step, stream=None, cams_dev=None):
    lr_arr = (ctypes.c_float * NPARAM)(*[float(x) for x in lr])
    _check(_lib.dg_project_bwd_adam(_a(params), stride, P, _c(cams), _a(cams_dev), n_views, ctypes.byref(opts),
                                    _a(radius), _a(clamp), _a(grad2d), _a(grads), _a(m), _a(v),
                                    ctypes.cast(lr_arr, ctypes.c_void_p), beta1, beta2, eps, step, _s(stream)))


def dg_project_bwd_adam_dev(params, stride, P, cams, n_views, opts, radius, clamp, grad2d, grads, m, v, hp_dev,
                            skip_if=None, stream=None, cams_dev=None):
    _check(_lib.dg_project_bwd_adam_dev(_a(params), stride, P, _c(cams), _a(cams_dev), n_views, ctypes.byref(opts),
                                        _a(radius), _a(clamp), _a(grad2d), _a(grads), _a(m), _a(v), _a(hp_dev),
                                        _a(skip_if), _s(stream)))


def dg_loss_workspace_size(n) -> int:
    return _lib.dg_loss_workspace_size(n)


def dg_loss_l1(img, target, n, dL_dimg, loss, ws, ws_bytes, stream=None):
    _check(_lib.dg_loss_l1(_a(img), _a(target), n, _a(dL_dimg), _a(loss), _a(ws), ws_bytes, _s(stream)))


def _wh(sizes):
    """Host int32 [n][2] array of (W, H) pairs."""
    flat = [int(x) for wh in sizes for x in wh]
    return (ctypes.c_int32 * len(flat))(*flat)


def dg_ssim_workspace_size(sizes) -> int:
    return _lib.dg_ssim_workspace_size(_wh(sizes), len(sizes))


def dg_loss_l1_dssim(img, target, sizes, lam, dL_dimg, loss, ws, ws_bytes, stream=None):
    """(1 - lam) L1 + lam (1 - SSIM) per view; sizes: list of (W, H)."""
    _check(_lib.dg_loss_l1_dssim(_a(img), _a(target), _wh(sizes), len(sizes), float(lam), _a(dL_dimg), _a(loss),
                                 _a(ws), ws_bytes, _s(stream)))


def dg_loss_l1_noalloc(img, target, n, dL_dimg, loss, stream=None):
    """dg_loss_l1 without a workspace: for callers that cannot allocate device memory."""
    _check(_lib.dg_loss_l1_noalloc(_a(img), _a(target), n, _a(dL_dimg), _a(loss), _s(stream)))


def dg_sparse_adam_step(params, grads, m, v, stride, P, lr, beta1, beta2, eps, step, visible, stream=None):
    lr_arr = (ctypes.c_float * NPARAM)(*[float(x) for x in lr])
    _check(_lib.dg_sparse_adam_step(_a(params), _a(grads), _a(m), _a(v), stride, P,
                                    ctypes.cast(lr_arr, ctypes.c_void_p), beta1, beta2, eps, step, _a(visible),
                                    _s(stream)))


def dg_visibility(radius, P, n_views, visible, stream=None):
    _check(_lib.dg_visibility(_a(radius), P, n_views, _a(visible), _s(stream)))


class AdamHparams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * NPARAM), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("bc1", ctypes.c_float), ("bc2_sqrt", ctypes.c_float), ("eps", ctypes.c_float)]


def dg_adam_hparams_fill(lr, beta1, beta2, eps, step) -> AdamHparams:
    lr_arr = (ctypes.c_float * NPARAM)(*[float(x) for x in lr])
    out = AdamHparams()
    _check(_lib.dg_adam_hparams_fill(ctypes.cast(lr_arr, ctypes.c_void_p), beta1, beta2, eps, step,
                                     ctypes.byref(out)))
    return out


def dg_adam_step_dev(params, grads, m, v, stride, P, hp_dev, skip_if=None, stream=None):
    _check(_lib.dg_adam_step_dev(_a(params), _a(grads), _a(m), _a(v), stride, P, _a(hp_dev), _a(skip_if),
                                 _s(stream)))


def dg_adam_step(params, grads, m, v, stride, P, lr, beta1, beta2, eps, step, stream=None):
    """lr: sequence of 59 per-row learning rates (host)."""
    lr_arr = (ctypes.c_float * NPARAM)(*[float(x) for x in lr])
    _check(_lib.dg_adam_step(_a(params), _a(grads), _a(m), _a(v), stride, P,
                             ctypes.cast(lr_arr, ctypes.c_void_p), beta1, beta2, eps, step, _s(stream)))


def dg_spectrum_workspace_size(H, W) -> int:
    return _lib.dg_spectrum_workspace_size(H, W)


def dg_spectrum_accumulate(view, H, W, acc, ws, ws_bytes, stream=None):
    _check(_lib.dg_spectrum_accumulate(_a(view), H, W, _a(acc), _a(ws), ws_bytes, _s(stream)))


def dg_spectrum_finalize(acc, n_views, H, W, shifted, sat, stream=None):
    _check(_lib.dg_spectrum_finalize(_a(acc), n_views, H, W, _a(shifted), _a(sat), _s(stream)))


def dg_downsample_area(src, C, H, W, dst, h, w, stream=None):
    _check(_lib.dg_downsample_area(_a(src), C, H, W, _a(dst), h, w, _s(stream)))


def dg_schedule_init(sat_host, H, W, params: SchedParams) -> Schedule:
    """sat_host: host float64 array (H+1, W+1), C-contiguous (numpy)."""
    import numpy as np
    sat = np.ascontiguousarray(sat_host, dtype=np.float64)
    assert sat.shape == (H + 1, W + 1)
    out = Schedule()
    _check(_lib.dg_schedule_init(sat.ctypes.data_as(ctypes.c_void_p), H, W, ctypes.byref(params),
                                 ctypes.byref(out)))
    return out


def dg_schedule_step(sched: Schedule, it) -> SchedOut:
    out = SchedOut()
    _check(_lib.dg_schedule_step(ctypes.byref(sched), int(it), ctypes.byref(out)))
    return out


def dg_schedule_densify(sched: Schedule, it, P_add) -> SchedOut:
    out = SchedOut()
    _check(_lib.dg_schedule_densify(ctypes.byref(sched), int(it), int(P_add), ctypes.byref(out)))
    return out


def dg_schedule_init_plain(H, W, params: SchedParams) -> Schedule:
    out = Schedule()
    _check(_lib.dg_schedule_init_plain(H, W, ctypes.byref(params), ctypes.byref(out)))
    return out


def dg_densify_budget(sched, it, n_keep, n_cand, P_cap):
    """-> (budget, SchedOut or None); sched None = the backbone (every candidate)."""
    b = _I64(0)
    out = SchedOut()
    _check(_lib.dg_densify_budget(ctypes.byref(sched) if sched is not None else None, int(it), int(n_keep),
                                  int(n_cand), int(P_cap), ctypes.byref(b), ctypes.byref(out)))
    return int(b.value), (out if sched is not None else None)


def dg_camera_scale(full: Camera, width, height) -> Camera:
    out = Camera()
    _check(_lib.dg_camera_scale(ctypes.byref(full), int(width), int(height), ctypes.byref(out)))
    return out


def dg_batch_adam_scale(views_per_step, lr, beta1, beta2):
    """-> (lr list of 59, beta1, beta2) for views_per_step views per Adam step."""
    arr = (_F * NPARAM)(*[float(x) for x in lr])
    b1, b2 = _F(beta1), _F(beta2)
    _check(_lib.dg_batch_adam_scale(int(views_per_step), arr, ctypes.byref(b1), ctypes.byref(b2)))
    return list(arr), b1.value, b2.value


def dg_densify_stats(grad2d, radius, P, cams, n_views, grad_accum, denom, max_radius, stream=None):
    _check(_lib.dg_densify_stats(_a(grad2d), _a(radius), P, _c(cams), n_views, _a(grad_accum), _a(denom),
                                 _a(max_radius), _s(stream)))


def dg_densify_workspace_size(P) -> int:
    return _lib.dg_densify_workspace_size(P)


def dg_densify_mark(params, stride, P, grad_accum, denom, max_radius, opts: DensifyOpts, ws, ws_bytes, counts,
                    stream=None):
    _check(_lib.dg_densify_mark(_a(params), stride, P, _a(grad_accum), _a(denom), _a(max_radius),
                                ctypes.byref(opts), _a(ws), ws_bytes, _a(counts), _s(stream)))


def dg_densify_apply(params, m, v, stride, P, n_cand, budget, noise, ws, ws_bytes, dst_params, dst_m, dst_v,
                     dst_stride, P_out, stream=None):
    _check(_lib.dg_densify_apply(_a(params), _a(m), _a(v), stride, P, n_cand, budget, _a(noise), _a(ws), ws_bytes,
                                 _a(dst_params), _a(dst_m), _a(dst_v), dst_stride, _a(P_out), _s(stream)))


def dg_mse(a, b, n, mse, ws, ws_bytes, stream=None):
    _check(_lib.dg_mse(_a(a), _a(b), n, _a(mse), _a(ws), ws_bytes, _s(stream)))


def dg_opacity_reset(params, m, v, stride, P, max_opacity, stream=None):
    _check(_lib.dg_opacity_reset(_a(params), _a(m), _a(v), stride, P, max_opacity, _s(stream)))
