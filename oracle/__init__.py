"""FP64 CPU oracle of the DashGaussian rasterizer path and schedule.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2503_18402_gb300``; it is the independent,
slow, obviously-correct definition that the CUDA path is checked against.

``dgo.c`` holds the rasterizer (projection, SH colour, binning, Eq. 1
compositing, their exact adjoint, L1 loss, Adam); ``schedule.py`` holds the
resolution and primitive schedules (Sec. 4.2, 4.3 and the supplementary
Eq. 6-8) in numpy FP64.

Parity pins: every function here is checked by ``tests/test_oracle_*.py``
against closed forms, brute force, finite differences or library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIBPATH = os.path.join(_LIBDIR, "libdgo.so")
_SRC = os.path.join(_HERE, "dgo.c")

NP = 59  # parameters per Gaussian
NF = 9   # feature record: u v A B C o r g b


def build(force: bool = False) -> str:
    """Compile dgo.c with gcc (plain C11, FP64, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC)):
        return _LIBPATH
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


class Consts(ctypes.Structure):
    _fields_ = [("near_plane", ctypes.c_double), ("eps2d", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("alpha_min", ctypes.c_double),
                ("t_min", ctypes.c_double), ("frustum_guard", ctypes.c_double),
                ("tile", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("mip2d", ctypes.c_double)]


class Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


def consts(tile=16, sh_degree=3, near_plane=0.2, eps2d=0.3, alpha_max=0.99,
           alpha_min=1.0 / 255.0, t_min=1e-4, frustum_guard=1.3, mip2d=0.0) -> Consts:
    """mip2d > 0: Mip-Splatting's 2D filter (variance mip2d, opacity compensated)
    in place of the eps2d dilation (the backbone variant of the supplementary)."""
    return Consts(near_plane, eps2d, alpha_max, alpha_min, t_min, frustum_guard,
                  tile, sh_degree, mip2d)


def camera(viewmat, fx, fy, cx, cy, width, height) -> Camera:
    vm = np.asarray(viewmat, dtype=np.float64).reshape(3, 4)
    c = Camera()
    c.R[:] = list(vm[:, :3].reshape(-1))
    c.t[:] = list(vm[:, 3])
    c.fx, c.fy, c.cx, c.cy = float(fx), float(fy), float(cx), float(cy)
    c.width, c.height = int(width), int(height)
    return c


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.dgo_sh_basis.argtypes = [_P, _I64, _P]
        L.dgo_project.argtypes = [_I64, _P, ctypes.POINTER(Camera), ctypes.POINTER(Consts),
                                  _P, _P, _P, _P, _P, _P, _P]
        L.dgo_bin.argtypes = [_I64, _P, _P, _P, _I32, _I32, _I32, _I64, _P, _P, _P]
        L.dgo_bin.restype = _I64
        L.dgo_render_fwd.argtypes = [_P, _I32, _I32, _I32, _P, _P, _P, ctypes.POINTER(Consts),
                                     _P, _P, _P, _P, _P]
        L.dgo_render_bwd.argtypes = [_P, _I32, _I32, _I32, _P, _P, _P, ctypes.POINTER(Consts),
                                     _P, _P]
        L.dgo_project_bwd.argtypes = [_I64, _P, ctypes.POINTER(Camera), ctypes.POINTER(Consts),
                                      _P, _P]
        L.dgo_tile_list.argtypes = [_I64, _P, _P, _P, _I32, _I32, _I32, _I64, _I64, _P]
        L.dgo_tile_list.restype = _I64
        L.dgo_render_pixels.argtypes = [_P, _I32, _I32, _P, _P, _P, ctypes.POINTER(Consts), _I64, _P, _P,
                                        _P, _P, _P, _P]
        L.dgo_loss_l1.argtypes = [_I64, _P, _P, _P]
        L.dgo_loss_l1.restype = _D
        L.dgo_adam.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _D, _D, _I64]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
def sh_basis(dirs) -> np.ndarray:
    """Real orthonormal SH basis (degree <= 3, 16 values) at unit directions."""
    d = _f64(dirs).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16))
    lib().dgo_sh_basis(_ptr(d), d.shape[0], _ptr(out))
    return out


def project(g, cam: Camera, k: Consts) -> dict:
    """Projection + colour of Gaussians g (P x 59, FP64)."""
    g = _f64(g)
    n = g.shape[0]
    out = dict(feat=np.zeros((n, NF)), depth=np.zeros(n), depth_key=np.zeros(n, np.uint32),
               radius=np.zeros(n, np.int32), tiles=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), clamp=np.zeros((n, 3), np.uint8))
    lib().dgo_project(n, _ptr(g), ctypes.byref(cam), ctypes.byref(k), _ptr(out["feat"]),
                      _ptr(out["depth"]), _ptr(out["depth_key"]), _ptr(out["radius"]),
                      _ptr(out["tiles"]), _ptr(out["rect"]), _ptr(out["clamp"]))
    return out


def bin_sort(uv, radius, depth_key, W, H, B) -> dict:
    """All (tile, Gaussian) pairs ordered by (tile, depth key, index) + ranges."""
    uv = _f64(uv).reshape(-1, 2)
    radius = np.ascontiguousarray(radius, dtype=np.int32)
    depth_key = np.ascontiguousarray(depth_key, dtype=np.uint32)
    n = uv.shape[0]
    TX, TY = (W + B - 1) // B, (H + B - 1) // B
    ranges = np.zeros((TX * TY, 2), np.uint32)
    cap = 0
    tiles = np.zeros(1, np.uint32)
    gids = np.zeros(1, np.uint32)
    M = lib().dgo_bin(n, _ptr(uv), _ptr(radius), _ptr(depth_key), W, H, B, cap,
                      _ptr(tiles), _ptr(gids), _ptr(ranges))
    tiles = np.zeros(max(M, 1), np.uint32)
    gids = np.zeros(max(M, 1), np.uint32)
    M2 = lib().dgo_bin(n, _ptr(uv), _ptr(radius), _ptr(depth_key), W, H, B, M,
                       _ptr(tiles), _ptr(gids), _ptr(ranges))
    assert M2 == M
    return dict(M=int(M), tile=tiles[:M], gid=gids[:M], ranges=ranges)


def tile_list(uv, radius, depth_key, W, H, B, tile_id) -> np.ndarray:
    """Gaussian indices of one tile's list, ordered by (depth key, index)."""
    uv = _f64(uv).reshape(-1, 2)
    radius = np.ascontiguousarray(radius, dtype=np.int32)
    depth_key = np.ascontiguousarray(depth_key, dtype=np.uint32)
    out = np.zeros(1, np.uint32)
    m = lib().dgo_tile_list(uv.shape[0], _ptr(uv), _ptr(radius), _ptr(depth_key), W, H, B, tile_id, 0, _ptr(out))
    out = np.zeros(max(m, 1), np.uint32)
    lib().dgo_tile_list(uv.shape[0], _ptr(uv), _ptr(radius), _ptr(depth_key), W, H, B, tile_id, m, _ptr(out))
    return out[:m]


def render_pixels(feat, W, B, gid, ranges, bg, k: Consts, px, py) -> dict:
    """Eq. 1 at sampled pixels (px, py) given a tile-sorted list."""
    feat = _f64(feat)
    gid = np.ascontiguousarray(gid, dtype=np.uint32)
    if gid.size == 0:
        gid = np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
    px = np.ascontiguousarray(px, dtype=np.int32)
    py = np.ascontiguousarray(py, dtype=np.int32)
    n = px.size
    rgb = np.zeros((n, 3)); T = np.zeros(n); last = np.zeros(n, np.int32); ex = np.zeros(n, np.int32)
    lib().dgo_render_pixels(_ptr(feat), W, B, _ptr(gid), _ptr(ranges), _ptr(_f64(bg)), ctypes.byref(k), n,
                            _ptr(px), _ptr(py), _ptr(rgb), _ptr(T), _ptr(last), _ptr(ex))
    return dict(rgb=rgb, T=T, last=last, examined=ex)


def render_fwd(feat, W, H, B, gid, ranges, bg, k: Consts) -> dict:
    feat = _f64(feat)
    gid = np.ascontiguousarray(gid, dtype=np.uint32)
    if gid.size == 0:
        gid = np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
    bg = _f64(bg)
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    last = np.zeros((H, W), np.int32)
    ex = np.zeros((H, W), np.int32)
    bl = np.zeros((H, W), np.int32)
    lib().dgo_render_fwd(_ptr(feat), W, H, B, _ptr(gid), _ptr(ranges), _ptr(bg),
                         ctypes.byref(k), _ptr(img), _ptr(T), _ptr(last), _ptr(ex), _ptr(bl))
    return dict(img=img, T=T, last=last, examined=ex, blended=bl)


def render_bwd(feat, W, H, B, gid, ranges, bg, k: Consts, dL_dimg) -> np.ndarray:
    feat = _f64(feat)
    gid = np.ascontiguousarray(gid, dtype=np.uint32)
    if gid.size == 0:
        gid = np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
    bg = _f64(bg)
    dL = _f64(dL_dimg).reshape(3, H, W)
    g2 = np.zeros((feat.shape[0], NF))
    lib().dgo_render_bwd(_ptr(feat), W, H, B, _ptr(gid), _ptr(ranges), _ptr(bg),
                         ctypes.byref(k), _ptr(dL), _ptr(g2))
    return g2


def project_bwd(g, cam: Camera, k: Consts, grad2d) -> np.ndarray:
    g = _f64(g)
    g2 = _f64(grad2d)
    out = np.zeros_like(g)
    lib().dgo_project_bwd(g.shape[0], _ptr(g), ctypes.byref(cam), ctypes.byref(k),
                          _ptr(g2), _ptr(out))
    return out


def loss_l1(img, target):
    img = _f64(img)
    target = _f64(target)
    grad = np.zeros_like(img)
    loss = lib().dgo_loss_l1(img.size, _ptr(img), _ptr(target), _ptr(grad))
    return loss, grad


def adam(param, grad, m, v, lr, beta1, beta2, eps, step):
    """In-place Adam on FP64 arrays (param, m, v); lr broadcast to param."""
    for a in (param, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    grad = _f64(grad)
    lr = _f64(np.broadcast_to(lr, param.shape))
    lib().dgo_adam(param.size, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), _ptr(lr),
                   beta1, beta2, eps, step)


def sparse_adam(param, grad, m, v, lr, beta1, beta2, eps, step, visible):
    """Sparse Adam of the Taming-3DGS backbone on planar [59][P] FP64 arrays:
    the Adam update of ``adam`` on the columns (Gaussians) with visible != 0;
    the other columns keep parameters and moments.  Global step count."""
    vis = np.flatnonzero(np.asarray(visible) != 0)
    if vis.size == 0:
        return
    lr = np.broadcast_to(np.asarray(lr, np.float64), param.shape)
    sub = [np.ascontiguousarray(a[:, vis]) for a in (param, m, v)]
    adam(sub[0], np.asarray(grad, np.float64)[:, vis], sub[1], sub[2], np.ascontiguousarray(lr[:, vis]),
         beta1, beta2, eps, step)
    for a, b in zip((param, m, v), sub):
        a[:, vis] = b


# --------------------------------------------------------------------------
def forward(g, cam: Camera, k: Consts, bg=(0.0, 0.0, 0.0)) -> dict:
    """Full FP64 forward: project -> bin/sort -> composite."""
    W, H, B = cam.width, cam.height, k.tile
    pr = project(g, cam, k)
    bs = bin_sort(pr["feat"][:, :2], pr["radius"], pr["depth_key"], W, H, B)
    rf = render_fwd(pr["feat"], W, H, B, bs["gid"], bs["ranges"], np.asarray(bg, float), k)
    return dict(proj=pr, bins=bs, **rf)


def backward(g, cam: Camera, k: Consts, fwd: dict, dL_dimg, bg=(0.0, 0.0, 0.0)) -> dict:
    """Full FP64 adjoint of ``forward``: returns grad2d and per-parameter grads."""
    W, H, B = cam.width, cam.height, k.tile
    g2 = render_bwd(fwd["proj"]["feat"], W, H, B, fwd["bins"]["gid"], fwd["bins"]["ranges"],
                    np.asarray(bg, float), k, dL_dimg)
    gp = project_bwd(g, cam, k, g2)
    return dict(grad2d=g2, grad=gp)
