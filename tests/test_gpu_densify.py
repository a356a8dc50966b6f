"""GPU densification (dg_densify_*) against the oracle: statistics, prune /
candidate / split flags and counts (exact), top-k selection and compaction
(exact copies), split samples (FP32 tolerance)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import densify as D  # noqa: E402
from paper_2503_18402_gb300 import capi, synth  # noqa: E402

pytestmark = pytest.mark.gpu
OPTS = dict(grad_thresh=2e-4, min_opacity=0.005, percent_dense=0.01, extent=5.0)


def _state(n, seed):
    rng = np.random.default_rng(seed)
    g = synth.random_gaussians(n, seed).astype(np.float32)
    g[:, 10] = rng.normal(-3.0, 2.5, size=n)
    g[:, 3:6] = rng.normal(-3.9, 0.4, size=(n, 3))
    acc = (np.abs(rng.normal(0, 6e-4, size=n)) * 3).astype(np.float32)
    den = rng.integers(0, 4, size=n).astype(np.float32)
    acc[den == 0] = 0
    acc[::97] = acc[1::97][: len(acc[::97])]  # ties in the score
    den[::97] = den[1::97][: len(den[::97])]
    return g, acc, den


def _run(g, acc, den, budget_frac, seed):
    P = g.shape[0]
    dev = "cuda"
    prm = torch.from_numpy(np.ascontiguousarray(g.T)).to(dev)
    rng = np.random.default_rng(seed)
    m_np = rng.normal(size=g.shape).astype(np.float32)
    m = torch.from_numpy(np.ascontiguousarray(m_np.T)).to(dev)
    v = m.abs()
    ta, td = torch.from_numpy(acc).to(dev), torch.from_numpy(den).to(dev)
    mr = torch.zeros(P, device=dev)
    opts = capi.densify_opts(**OPTS)
    ws = torch.empty(capi.dg_densify_workspace_size(P), dtype=torch.uint8, device=dev)
    counts = torch.zeros(2, dtype=torch.int64, device=dev)
    capi.dg_densify_mark(prm, P, P, ta, td, mr, opts, ws, ws.numel(), counts)
    n_keep, n_cand = (int(x) for x in counts.cpu())
    budget = int(n_cand * budget_frac)
    n_sel = min(n_cand, budget)
    noise = rng.normal(size=(max(n_sel, 1), 2, 3)).astype(np.float32)
    cap = P + n_sel
    dp = torch.full((59, cap), np.nan, device=dev)
    dm = torch.full((59, cap), np.nan, device=dev)
    dv = torch.full((59, cap), np.nan, device=dev)
    Pout = torch.zeros(1, dtype=torch.int64, device=dev)
    capi.dg_densify_apply(prm, m, v, P, P, n_cand, budget, torch.from_numpy(noise).to(dev), ws, ws.numel(),
                          dp, dm, dv, cap, Pout)
    torch.cuda.synchronize()
    Pn = int(Pout.item())
    # oracle
    f = D.mark(g, acc, den, np.zeros(P, np.float32), OPTS)
    assert n_keep == int(f["keep0"].sum()) and n_cand == int(f["cand"].sum())
    sel = D.select(f["cand"], f["score"], budget)
    og, om, ov = D.apply(g.astype(np.float64), m_np.astype(np.float64), np.abs(m_np).astype(np.float64), f, sel,
                         noise.astype(np.float64))
    assert Pn == og.shape[0] == n_keep + n_sel
    gp = dp[:, :Pn].cpu().numpy().T
    keep = int((f["keep0"] & ~(sel & f["split"])).sum())
    np.testing.assert_array_equal(gp[:keep], og[:keep].astype(np.float32))
    np.testing.assert_array_equal(dm[:, :keep].cpu().numpy().T, om[:keep].astype(np.float32))
    np.testing.assert_array_equal(dv[:, :keep].cpu().numpy().T, ov[:keep].astype(np.float32))
    np.testing.assert_allclose(gp[keep:], og[keep:], rtol=2e-6, atol=2e-6)
    assert np.all(dm[:, keep:Pn].cpu().numpy() == 0) and np.all(dv[:, keep:Pn].cpu().numpy() == 0)
    return n_cand, n_sel


@pytest.mark.parametrize("P,frac", [(20000, 0.5), (20000, 2.0), (5003, 0.1), (100, 0.0)])
def test_densify_matches_oracle(P, frac):
    g, acc, den = _state(P, P)
    n_cand, n_sel = _run(g, acc, den, frac, 1)
    assert n_cand > 0


def test_densify_stats_matches_oracle():
    rng = np.random.default_rng(2)
    P, W, H = 10000, 1237, 822
    g2 = np.zeros((P, 12), np.float32)
    g2[:, :9] = rng.normal(0, 1e-5, size=(P, 9))
    rad = rng.integers(-1, 30, size=P).clip(0).astype(np.int32)
    acc = np.abs(rng.normal(size=P)).astype(np.float32)
    den = rng.integers(0, 5, size=P).astype(np.float32)
    mr = rng.integers(0, 20, size=P).astype(np.float32)
    t = [torch.from_numpy(x.copy()).cuda() for x in (g2, rad, acc, den, mr)]
    cam = capi.camera([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], 100, 100, W / 2, H / 2, W, H)
    capi.dg_densify_stats(t[0], t[1], P, cam, 1, t[2], t[3], t[4])
    torch.cuda.synchronize()
    oa, od, om = D.stats_update(acc.astype(np.float64), den.astype(np.float64), mr.astype(np.float64),
                                g2.astype(np.float64), rad, W, H)
    np.testing.assert_allclose(t[2].cpu().numpy(), oa, rtol=1e-6)
    np.testing.assert_array_equal(t[3].cpu().numpy(), od)
    np.testing.assert_array_equal(t[4].cpu().numpy(), om)
