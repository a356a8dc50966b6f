"""End-to-end optimisation through the library (plain and scheduled arms) on a
small seeded scene: the loss falls, held-out PSNR rises over the initial state,
densification respects the Eq. 4/5 budget and the cap, and the scheduled arm
renders its early iterations at reduced resolution."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import schedule as sch  # noqa: E402
from paper_2503_18402_gb300 import synth  # noqa: E402
from paper_2503_18402_gb300.train import Trainer, TrainConfig, make_dataset  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    dev = torch.device("cuda")
    gt, cams, imgs, train, test = make_dataset(60_000, 24, 192, 128, dev)
    init = synth.perturb(gt, 3001, n_keep=6000)
    return gt, cams, imgs, train, test, init


@pytest.mark.parametrize("scheduled", [False, True])
def test_training_improves_and_respects_budget(data, scheduled):
    gt, cams, imgs, train, test, init = data
    cfg = TrainConfig(iters=1200, scheduled=scheduled, densify_from=60, densify_until=900, densify_every=60,
                      opacity_reset_every=600, P_cap=40_000)
    tr = Trainer(cfg, init, [cams[i] for i in train], [imgs[i] for i in train])
    tv = [cams[i] for i in test]
    ti = [imgs[i] for i in test]
    psnr0 = tr.psnr(tv, ti)
    res = tr.run()
    psnr1 = tr.psnr(tv, ti)
    assert psnr1 > psnr0 + 3.0, (psnr0, psnr1)
    assert tr.P <= cfg.P_cap and tr.P > init.shape[0] // 2
    for h in tr.history:
        assert h["P"] == h["n_keep"] + min(h["budget"], h["n_cand"])
    if scheduled:
        assert tr.sched.m >= 1 and tr.sched.r_m >= 1.0
        assert res["iters_per_factor"].get("1", 0) < cfg.iters  # some iterations below full resolution
        # Eq. 5 state: P_fin(0) = 5 P_init, then one update per densification
        # step with P_add = that step's candidate count
        P_fin = 5.0 * init.shape[0]
        for h in tr.history:
            P_fin = sch.pfin_update(P_fin, h["n_cand"], cfg.gamma, cfg.eta)
        assert tr.sched.P_fin == pytest.approx(P_fin, rel=1e-12)
        assert tr.sched.P_fin >= 5.0 * init.shape[0]
