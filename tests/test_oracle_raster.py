"""Pins of the FP64 oracle's rasterizer against facts fixed outside the oracle.

Each test checks the oracle against a closed form, a brute-force
re-derivation, a library routine or finite differences, chosen so that a
dropped term, a wrong sign/index or a transposed operand fails one of them.
Compositing follows Eq. 1 (Sec. 3); the projection, SH colour, binning and
thresholds follow the readings listed in the oracle's header.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2503_18402_gb300 import synth
from tests import _util as U

K = oracle.consts(tile=16, sh_degree=3)


# ---------------------------------------------------------------- SH basis
def _sphere_rule(n_theta=10, n_phi=20):
    x, w = np.polynomial.legendre.leggauss(n_theta)  # exact in cos(theta) up to degree 19
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi  # exact for |m| < n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(n_phi, 2 * math.pi / n_phi)[None, :]).reshape(-1)
    return dirs, wts


def test_sh_orthonormal_by_quadrature():
    dirs, wts = _sphere_rule()
    Y = oracle.sh_basis(dirs)
    gram = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_addition_theorem():
    # sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b): pins each degree block
    rng = np.random.default_rng(5)
    a = rng.normal(size=(50, 3)); a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = rng.normal(size=(50, 3)); b /= np.linalg.norm(b, axis=1, keepdims=True)
    Ya, Yb = oracle.sh_basis(a), oracle.sh_basis(b)
    cosg = np.sum(a * b, 1)
    for l in range(4):
        sl = slice(l * l, (l + 1) * (l + 1))
        lhs = np.sum(Ya[:, sl] * Yb[:, sl], 1)
        Pl = np.polynomial.legendre.legval(cosg, [0] * l + [1])
        np.testing.assert_allclose(lhs, (2 * l + 1) / (4 * math.pi) * Pl, atol=1e-12)


def test_sh_degree0_and_degree1_forms():
    d = np.array([[0.36, -0.48, 0.8]])
    Y = oracle.sh_basis(d)[0]
    assert Y[0] == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-15)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[1:4], c1 * np.array([-0.48, 0.8, 0.36]), atol=1e-15)


# ----------------------------------------------------- closed-form renders
def _render(g, cam, bg=(0.0, 0.0, 0.0), k=K):
    return oracle.forward(g, U.oracle_cam(oracle, cam), k, bg=bg)


def _iso_expected(W, H, u, v, s2, o, c, radius, B=16):
    """Closed form for one Gaussian: alpha = o exp(-d^2 / (2 s2)) on the
    pixels whose tile lies inside the rect, cut at 1/255, clamped at 0.99."""
    xs = np.arange(W) + 0.5
    ys = np.arange(H) + 0.5
    dx = u - xs[None, :]
    dy = v - ys[:, None]
    a = o * np.exp(-(dx ** 2 + dy ** 2) / (2 * s2))
    a = np.minimum(a, 0.99)
    a[a < 1 / 255] = 0
    TX, TY = (W + B - 1) // B, (H + B - 1) // B
    x0, x1 = max(0, math.floor((u - radius) / B)), min(TX, math.floor((u + radius) / B) + 1)
    y0, y1 = max(0, math.floor((v - radius) / B)), min(TY, math.floor((v + radius) / B) + 1)
    tx = (np.arange(W) // B)[None, :]
    ty = (np.arange(H) // B)[:, None]
    inside = (tx >= x0) & (tx < x1) & (ty >= y0) & (ty < y1)
    a = np.where(inside, a, 0.0)
    return a[None] * np.asarray(c, float)[:, None, None], 1 - a


@pytest.mark.parametrize("sigma,centre", [(0.05, (32.5, 32.5)), (0.3, (32.5, 32.5)),
                                          (0.3, (17.25, 40.75)), (0.6, (30.0, 20.0))])
def test_single_isotropic_gaussian_closed_form(sigma, centre):
    W = H = 64
    f, z, o = 60.0, 4.0, 0.7
    cam = U.identity_cam(W, H, f, cx=centre[0], cy=centre[1])
    g = U.single_gaussian((0, 0, z), [math.log(sigma)] * 3, opacity=o, dc=(0.8, 0.3, 0.55))
    out = _render(g, cam)
    s2 = (f * sigma / z) ** 2 + 0.3
    radius = math.ceil(3 * math.sqrt(s2))
    assert out["proj"]["radius"][0] == radius
    img, T = _iso_expected(W, H, centre[0], centre[1], s2, o, (0.8, 0.3, 0.55), radius)
    np.testing.assert_allclose(out["img"], img, atol=1e-12)
    np.testing.assert_allclose(out["T"], T, atol=1e-12)
    # the peak pixel, when the mean sits on a pixel centre, gets alpha = o exactly
    if centre == (32.5, 32.5):
        assert out["img"][0, 32, 32] == pytest.approx(o * 0.8, abs=1e-14)


def test_anisotropic_rotated_closed_form():
    # axis-aligned scales rotated about the optical axis by theta:
    # cov2D = R2 diag((f sx/z)^2, (f sy/z)^2) R2^T + 0.3 I
    W = H = 64
    f, z, o, th = 60.0, 5.0, 0.6, 0.4
    sx, sy, sz = 0.35, 0.12, 0.2
    quat = (math.cos(th / 2), 0.0, 0.0, math.sin(th / 2))
    cam = U.identity_cam(W, H, f, cx=32.5, cy=32.5)
    g = U.single_gaussian((0, 0, z), np.log([sx, sy, sz]), quat=quat, opacity=o, dc=(0.9, 0.9, 0.9))
    out = _render(g, cam)
    R2 = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    cov = R2 @ np.diag([(f * sx / z) ** 2, (f * sy / z) ** 2]) @ R2.T + 0.3 * np.eye(2)
    con = np.linalg.inv(cov)
    feat = out["proj"]["feat"][0]
    np.testing.assert_allclose(feat[2:5], [con[0, 0], con[0, 1], con[1, 1]], rtol=1e-12)
    lam = np.linalg.eigvalsh(cov).max()
    assert out["proj"]["radius"][0] == math.ceil(3 * math.sqrt(lam))


def test_background_only():
    W, H = 40, 24
    cam = U.identity_cam(W, H, 50.0)
    bg = (0.2, 0.5, 0.9)
    # empty scene
    out = _render(np.zeros((0, 59)), cam, bg=bg)
    assert out["bins"]["M"] == 0
    np.testing.assert_array_equal(out["img"], np.broadcast_to(np.array(bg)[:, None, None], (3, H, W)))
    np.testing.assert_array_equal(out["T"], 1.0)
    np.testing.assert_array_equal(out["last"], 0)
    # all culled: behind the near plane, behind the camera, far off-screen
    g = np.concatenate([U.single_gaussian((0, 0, 0.1), [-2] * 3),
                        U.single_gaussian((0, 0, -3.0), [-2] * 3),
                        U.single_gaussian((40.0, 0, 2.0), [-3] * 3)])
    out = _render(g, cam, bg=bg)
    assert out["bins"]["M"] == 0
    np.testing.assert_array_equal(out["proj"]["radius"][:2], 0)
    np.testing.assert_array_equal(out["img"], np.broadcast_to(np.array(bg)[:, None, None], (3, H, W)))


def _stack(Kn, o, colours, z0=3.0, dz=0.25, sigma=0.1, f=60.0):
    rows = []
    for i in range(Kn):
        z = z0 + dz * i
        rows.append(U.single_gaussian((0, 0, z), [math.log(sigma * z / z0)] * 3, opacity=o,
                                      dc=colours[i]))
    return np.concatenate(rows)


def test_transmittance_product_and_termination():
    # K coincident footprints, identical alpha: T = (1-a)^K, C = sum a (1-a)^i c_i;
    # termination at the first i with (1-a)^(i+1) < 1e-4, which is not blended.
    W = H = 32
    cam = U.identity_cam(W, H, 60.0, cx=16.5, cy=16.5)
    rng = np.random.default_rng(3)
    cols = rng.uniform(0.1, 0.9, size=(20, 3))
    # shuffle the rows: the order must come from depth, not from the index
    g = _stack(20, 0.5, cols)
    perm = rng.permutation(20)
    out = _render(g[perm], cam)
    a = 0.5
    n_blend = 13  # 0.5^13 = 1.22e-4 >= 1e-4 > 0.5^14
    expect = sum(a * (1 - a) ** i * cols[i] for i in range(n_blend))
    np.testing.assert_allclose(out["img"][:, 16, 16], expect, atol=1e-13)
    assert out["T"][16, 16] == pytest.approx(0.5 ** 13, rel=1e-13)
    assert out["last"][16, 16] == 13
    assert out["examined"][16, 16] == 14
    assert out["blended"][16, 16] == 13
    # a lighter stack: no termination, T = (1-a)^K
    g = _stack(6, 0.3, cols)
    out = _render(g, cam)
    assert out["T"][16, 16] == pytest.approx(0.7 ** 6, rel=1e-13)
    expect = sum(0.3 * 0.7 ** i * cols[i] for i in range(6))
    np.testing.assert_allclose(out["img"][:, 16, 16], expect, atol=1e-13)


def test_alpha_clamp_and_cutoff():
    W = H = 32
    f, z, sigma = 60.0, 4.0, 0.2
    cam = U.identity_cam(W, H, f, cx=16.5, cy=16.5)
    s2 = (f * sigma / z) ** 2 + 0.3
    # clamp: opacity -> 1 at the centre gives alpha = 0.99 exactly
    g = U.single_gaussian((0, 0, z), [math.log(sigma)] * 3, opacity=0.99995, dc=(1, 1, 1))
    out = _render(g, cam)
    assert out["img"][0, 16, 16] == pytest.approx(0.99, abs=1e-15)
    assert out["T"][16, 16] == pytest.approx(0.01, abs=1e-15)
    # cutoff: choose o so that the pixel 3 px right of the centre sits just
    # below / just above 1/255
    G3 = math.exp(-9 / (2 * s2))
    for factor, contributes in ((1 - 1e-9, False), (1 + 1e-9, True)):
        o = factor / 255 / G3
        g = U.single_gaussian((0, 0, z), [math.log(sigma)] * 3, opacity=o, dc=(1, 1, 1))
        out = _render(g, cam)
        assert (out["img"][0, 16, 19] > 0) == contributes
        assert out["img"][0, 16, 18] > 0


# ----------------------------------------------------- projection pins
def _proj_numeric(g, cam, eps2d=0.3):
    """Projection re-derived with library routines: scipy rotation, numeric
    Jacobian of the pinhole map, numpy inverse and eigenvalues."""
    vm = cam["viewmat"]; R, t = vm[:, :3], vm[:, 3]
    fx, fy, cx, cy = cam["intr"]
    W, H = cam["width"], cam["height"]
    p = g[0:3]
    tc = R @ p + t
    q = g[6:10]
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    S = np.diag(np.exp(g[3:6]))
    Sig = Rq @ S @ S @ Rq.T
    lx, ly = 1.3 * 0.5 * W / fx, 1.3 * 0.5 * H / fy
    tg = np.array([np.clip(tc[0] / tc[2], -lx, lx) * tc[2], np.clip(tc[1] / tc[2], -ly, ly) * tc[2], tc[2]])

    def pin(x):
        return np.array([fx * x[0] / x[2], fy * x[1] / x[2]])
    h = 1e-6
    J = np.stack([(pin(tg + h * e) - pin(tg - h * e)) / (2 * h) for e in np.eye(3)], 1)
    cov = J @ R @ Sig @ R.T @ J.T + eps2d * np.eye(2)
    u = fx * tc[0] / tc[2] + cx
    v = fy * tc[1] / tc[2] + cy
    return u, v, np.linalg.inv(cov), math.ceil(3 * math.sqrt(np.linalg.eigvalsh(cov).max())), tc[2]


def test_projection_against_library_rederivation():
    g = synth.random_gaussians(300, 11)
    cam = synth.camera_cfg0(64, 64, 4.0)
    pr = oracle.project(g, U.oracle_cam(oracle, cam), K)
    checked = 0
    for i in range(g.shape[0]):
        if pr["radius"][i] == 0:
            continue
        u, v, con, rad, z = _proj_numeric(g[i], cam)
        f = pr["feat"][i]
        assert f[0] == pytest.approx(u, rel=1e-12) and f[1] == pytest.approx(v, rel=1e-12)
        np.testing.assert_allclose(f[2:5], [con[0, 0], con[0, 1], con[1, 1]], rtol=1e-6)
        assert pr["radius"][i] == rad
        assert pr["depth"][i] == pytest.approx(z, rel=1e-14)
        assert pr["depth_key"][i] == np.float32(z).view(np.uint32)
        o = 1 / (1 + math.exp(-g[i, 10]))
        assert f[5] == pytest.approx(o, rel=1e-14)
        checked += 1
    assert checked > 200


def test_frustum_guard_on_jacobian_only():
    # far off-axis Gaussian: the mean projects unclamped, the Jacobian uses the
    # guarded t_x/t_z (1.3 x half-FOV tangent)
    W = H = 64
    f = 40.0
    cam = U.identity_cam(W, H, f)
    g = U.single_gaussian((3.2, 0.4, 2.0), [math.log(0.8)] * 3, opacity=0.9)
    pr = oracle.project(g, U.oracle_cam(oracle, cam), K)
    u, v, con, rad, z = _proj_numeric(g[0], cam)
    assert 3.2 / 2.0 > 1.3 * 0.5 * W / f  # guard active
    assert pr["radius"][0] > 0
    np.testing.assert_allclose(pr["feat"][0, 2:5], [con[0, 0], con[0, 1], con[1, 1]], rtol=1e-6)
    assert pr["feat"][0, 0] == pytest.approx(u, rel=1e-13)


def test_colour_is_sh_plus_half_clamped():
    g = synth.random_gaussians(200, 12)
    g[:, 11:59] *= 5.0  # large coefficients: many clamped channels
    cam = synth.camera_cfg0(64, 64, 4.0)
    pr = oracle.project(g, U.oracle_cam(oracle, cam), K)
    vm = cam["viewmat"]
    campos = -vm[:, :3].T @ vm[:, 3]
    vis = pr["radius"] > 0
    d = g[:, 0:3] - campos
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(d)
    raw = np.einsum("nk,nkc->nc", Y, g[:, 11:59].reshape(-1, 16, 3)) + 0.5
    np.testing.assert_allclose(pr["feat"][vis, 6:9], np.maximum(raw[vis], 0), atol=1e-13)
    np.testing.assert_array_equal(pr["clamp"][vis], (raw[vis] < 0).astype(np.uint8))
    assert pr["clamp"][vis].sum() > 50


# ----------------------------------------------------- brute force
def _brute_force(feat, radius, depth_key, W, H, B, bg):
    TX = (W + B - 1) // B
    n = feat.shape[0]
    rects = []
    for i in range(n):
        if radius[i] <= 0:
            rects.append(None); continue
        u, v, r = feat[i, 0], feat[i, 1], int(radius[i])
        x0 = max(0, math.floor((math.floor(u) - r) / B)); x1 = min(TX, math.floor((math.floor(u) + r) / B) + 1)
        y0 = max(0, math.floor((math.floor(v) - r) / B)); y1 = min((H + B - 1) // B, math.floor((math.floor(v) + r) / B) + 1)
        rects.append((x0, y0, x1, y1) if (x0 < x1 and y0 < y1) else None)
    img = np.zeros((3, H, W)); T_out = np.ones((H, W))
    for py in range(H):
        for px in range(W):
            tx, ty = px // B, py // B
            cand = [i for i in range(n) if rects[i] and rects[i][0] <= tx < rects[i][2] and rects[i][1] <= ty < rects[i][3]]
            cand.sort(key=lambda i: (int(depth_key[i]), i))
            T, C = 1.0, np.zeros(3)
            for i in cand:
                u, v, A, Bc, Cc, o = feat[i, :6]
                dx, dy = u - (px + 0.5), v - (py + 0.5)
                pw = -0.5 * (A * dx * dx + Cc * dy * dy) - Bc * dx * dy
                if pw > 0:
                    continue
                a = min(0.99, o * math.exp(pw))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                C += a * T * feat[i, 6:9]
                T *= 1 - a
            img[:, py, px] = C + T * np.asarray(bg)
            T_out[py, px] = T
    return img, T_out


def test_tile_pipeline_equals_brute_force():
    g = synth.random_gaussians(120, 21)
    g[:, 3:6] += 0.8  # bigger footprints: many multi-tile rects
    cam = synth.camera_cfg0(48, 40, 4.0)  # ragged: 3 x 3 tiles, partial last row/col
    bg = (0.1, 0.2, 0.3)
    out = _render(g, cam, bg=bg)
    pr = out["proj"]
    img, T = _brute_force(pr["feat"], pr["radius"], pr["depth_key"], 48, 40, 16, bg)
    np.testing.assert_allclose(out["img"], img, atol=1e-12)
    np.testing.assert_allclose(out["T"], T, atol=1e-12)
    assert out["bins"]["M"] > 150


def test_bin_lists_are_sorted_rect_members():
    g = synth.random_gaussians(400, 22)
    g[:, 3:6] += 0.5
    cam = synth.camera_cfg0(80, 72, 4.0)
    pr = oracle.project(g, U.oracle_cam(oracle, cam), K)
    bs = oracle.bin_sort(pr["feat"][:, :2], pr["radius"], pr["depth_key"], 80, 72, 16)
    TX = 5
    for t in range(TX * 5):
        s, e = bs["ranges"][t]
        got = list(bs["gid"][s:e])
        ty, tx = divmod(t, TX)
        members = [i for i in range(400) if pr["radius"][i] > 0 and pr["rect"][i, 0] <= tx < pr["rect"][i, 2]
                   and pr["rect"][i, 1] <= ty < pr["rect"][i, 3]]
        members.sort(key=lambda i: (int(pr["depth_key"][i]), i))
        assert got == members
        assert all(bs["tile"][s:e] == t)
    assert bs["M"] == int(pr["tiles"].sum())


# ----------------------------------------------------- loss, Adam
def test_l1_loss_and_grad():
    rng = np.random.default_rng(4)
    a, b = rng.uniform(size=(3, 8, 9)), rng.uniform(size=(3, 8, 9))
    b[0, 0, 0] = a[0, 0, 0]
    loss, grad = oracle.loss_l1(a, b)
    assert loss == pytest.approx(np.mean(np.abs(a - b)), rel=1e-15)
    np.testing.assert_array_equal(grad, np.sign(a - b) / a.size)
    assert grad[0, 0, 0] == 0.0


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    p = rng.normal(size=200)
    m = np.zeros(200); v = np.zeros(200)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 6):
        gr = rng.normal(size=200)
        oracle.adam(p, gr, m, v, 0.01, 0.9, 0.999, 1e-15, step)
        tp.grad = torch.tensor(gr)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_sparse_adam_matches_torch_sparse_adam():
    """The oracle's sparse Adam (planar [59][P], visibility mask) equals
    torch.optim.SparseAdam on the transposed [P][59] parameter with sparse
    gradients holding only the visible Gaussians' rows."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    P = 50
    p = rng.normal(size=(59, P))
    m = np.zeros((59, P)); v = np.zeros((59, P))
    tp = torch.tensor(p.T.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.SparseAdam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 7):
        vis = rng.random(P) < 0.6
        gr = rng.normal(size=(59, P)) * vis[None, :]
        before = p.copy()
        oracle.sparse_adam(p, gr, m, v, 0.01, 0.9, 0.999, 1e-15, step, vis)
        np.testing.assert_array_equal(p[:, ~vis], before[:, ~vis])  # invisible columns untouched
        idx = np.flatnonzero(vis)
        tp.grad = torch.sparse_coo_tensor(torch.tensor(idx[None, :]), torch.tensor(gr.T[idx]), size=(P, 59))
        opt.step()
        # torch folds the bias corrections into the step size (different rounding order)
        np.testing.assert_allclose(p, tp.detach().numpy().T, rtol=1e-10, atol=1e-13)


def test_mip_2d_filter_isotropic_closed_form():
    """Mip-Splatting's 2D filter on a single isotropic Gaussian on the optical
    axis: covariance (f sigma / z)^2 + s in place of the dilation, opacity
    scaled by (f sigma / z)^2 / ((f sigma / z)^2 + s) (the determinant ratio of
    2x2 isotropic matrices, square-rooted); the centre pixel gets that alpha."""
    W = H = 64
    f, z, o, sigma, s = 60.0, 4.0, 0.7, 0.02, 0.1
    cam = U.identity_cam(W, H, f, cx=32.5, cy=32.5)
    g = U.single_gaussian((0, 0, z), [math.log(sigma)] * 3, opacity=o, dc=(0.8, 0.3, 0.55))
    k = oracle.consts(mip2d=s)
    out = oracle.forward(g, U.oracle_cam(oracle, cam), k)
    v0 = (f * sigma / z) ** 2
    feat = out["proj"]["feat"][0]
    np.testing.assert_allclose(feat[2:5], [1.0 / (v0 + s), 0.0, 1.0 / (v0 + s)], rtol=1e-12, atol=1e-15)
    o_eff = o * v0 / (v0 + s)
    assert feat[5] == pytest.approx(o_eff, rel=1e-12)
    assert out["proj"]["radius"][0] == math.ceil(3 * math.sqrt(v0 + s))
    assert out["img"][0, 32, 32] == pytest.approx(o_eff * 0.8, rel=1e-12)
    # without the filter the same Gaussian keeps its opacity (dilation only)
    out0 = oracle.forward(g, U.oracle_cam(oracle, cam), oracle.consts())
    assert out0["proj"]["feat"][0][5] == pytest.approx(o, rel=1e-14)
