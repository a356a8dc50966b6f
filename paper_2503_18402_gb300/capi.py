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

EXPORTS = ("dg_last_error", "dg_abi_version", "dg_kernel_launches", "dg_project", "dg_bin_workspace_size", "dg_bin_count",
           "dg_bin_sort", "dg_render_fwd", "dg_render_bwd", "dg_project_bwd", "dg_loss_workspace_size",
           "dg_loss_l1", "dg_loss_l1_noalloc", "dg_adam_step")
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
                ("eps2d", ctypes.c_float), ("bg", ctypes.c_float * 3)]


def camera(viewmat, fx, fy, cx, cy, width, height) -> Camera:
    c = Camera()
    vm = [float(x) for row in viewmat for x in row] if hasattr(viewmat[0], "__len__") else [float(x) for x in viewmat]
    assert len(vm) == 12
    c.viewmat[:] = vm
    c.fx, c.fy, c.cx, c.cy = float(fx), float(fy), float(cx), float(cy)
    c.width, c.height = int(width), int(height)
    return c


def raster_opts(tile=16, sh_degree=3, near_plane=0.2, eps2d=0.3, bg=(0.0, 0.0, 0.0)) -> RasterOpts:
    o = RasterOpts()
    o.tile, o.sh_degree, o.near_plane, o.eps2d = int(tile), int(sh_degree), float(near_plane), float(eps2d)
    o.bg[:] = [float(b) for b in bg]
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
    "dg_project": ([_P, _I64, _I64, _CAM, _OPT, _P, _P, _P, _P, _P, _P], _ST),
    "dg_bin_workspace_size": ([_I64, _I64, _I32], _SZ),
    "dg_bin_count": ([_P, _P, _I64, _P, _SZ, _I64, _I32, _P, _P], _ST),
    "dg_bin_sort": ([_P, _P, _I64, _CAM, _I32, _P, _SZ, _I64, _P, _P, _P, _P], _ST),
    "dg_render_fwd": ([_P, _P, _P, _CAM, _OPT, _P, _P, _P, _P, _P], _ST),
    "dg_render_bwd": ([_P, _P, _P, _CAM, _OPT, _P, _P, _P, _I64, _P, _P], _ST),
    "dg_project_bwd": ([_P, _I64, _I64, _CAM, _OPT, _P, _P, _P, _P, _P], _ST),
    "dg_loss_workspace_size": ([_I64], _SZ),
    "dg_loss_l1": ([_P, _P, _I64, _P, _P, _P, _SZ, _P], _ST),
    "dg_loss_l1_noalloc": ([_P, _P, _I64, _P, _P, _P], _ST),
    "dg_adam_step": ([_P, _P, _P, _P, _I64, _I64, _P, _F, _F, _F, _I64, _P], _ST),
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


def dg_project(params, stride, P, cam, opts, feat, depth, radius, tiles, clamp, stream=None):
    _check(_lib.dg_project(_a(params), stride, P, ctypes.byref(cam), ctypes.byref(opts), _a(feat),
                           _a(depth), _a(radius), _a(tiles), _a(clamp), _s(stream)))


def dg_bin_workspace_size(P, M_cap, n_tiles) -> int:
    return _lib.dg_bin_workspace_size(P, M_cap, n_tiles)


def dg_bin_count(depth, tiles, P, ws, ws_bytes, M_cap, n_tiles, M_out, stream=None):
    _check(_lib.dg_bin_count(_a(depth), _a(tiles), P, _a(ws), ws_bytes, M_cap, n_tiles, _a(M_out), _s(stream)))


def dg_bin_sort(feat, radius, P, cam, tile, ws, ws_bytes, M_cap, gid, ranges, status, stream=None):
    _check(_lib.dg_bin_sort(_a(feat), _a(radius), P, ctypes.byref(cam), tile, _a(ws), ws_bytes, M_cap,
                            _a(gid), _a(ranges), _a(status), _s(stream)))


def dg_render_fwd(feat, gid, ranges, cam, opts, img, T_final, last, examined, stream=None):
    _check(_lib.dg_render_fwd(_a(feat), _a(gid), _a(ranges), ctypes.byref(cam), ctypes.byref(opts), _a(img),
                              _a(T_final), _a(last), _a(examined), _s(stream)))


def dg_render_bwd(feat, gid, ranges, cam, opts, T_final, last, dL_dimg, P, grad2d, stream=None):
    _check(_lib.dg_render_bwd(_a(feat), _a(gid), _a(ranges), ctypes.byref(cam), ctypes.byref(opts),
                              _a(T_final), _a(last), _a(dL_dimg), P, _a(grad2d), _s(stream)))


def dg_project_bwd(params, stride, P, cam, opts, radius, clamp, grad2d, grads, stream=None):
    _check(_lib.dg_project_bwd(_a(params), stride, P, ctypes.byref(cam), ctypes.byref(opts), _a(radius),
                               _a(clamp), _a(grad2d), _a(grads), _s(stream)))


def dg_loss_workspace_size(n) -> int:
    return _lib.dg_loss_workspace_size(n)


def dg_loss_l1(img, target, n, dL_dimg, loss, ws, ws_bytes, stream=None):
    _check(_lib.dg_loss_l1(_a(img), _a(target), n, _a(dL_dimg), _a(loss), _a(ws), ws_bytes, _s(stream)))


def dg_loss_l1_noalloc(img, target, n, dL_dimg, loss, stream=None):
    """dg_loss_l1 without a workspace: for callers that cannot allocate device memory."""
    _check(_lib.dg_loss_l1_noalloc(_a(img), _a(target), n, _a(dL_dimg), _a(loss), _s(stream)))


def dg_adam_step(params, grads, m, v, stride, P, lr, beta1, beta2, eps, step, stream=None):
    """lr: sequence of 59 per-row learning rates (host)."""
    lr_arr = (ctypes.c_float * NPARAM)(*[float(x) for x in lr])
    _check(_lib.dg_adam_step(_a(params), _a(grads), _a(m), _a(v), stride, P,
                             ctypes.cast(lr_arr, ctypes.c_void_p), beta1, beta2, eps, step, _s(stream)))

