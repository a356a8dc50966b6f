"""The paper's printed constants (tests/golden/paper_printed_values.txt, each
line cited) against the defaults and behaviour of the library's host-side
schedule and of the schedule oracle.  CPU only."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from oracle import schedule as sch

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.txt")


def _golden() -> dict:
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, cite = line.split("|", 1)
        name, value = (t.strip() for t in lhs.split("="))
        assert cite.strip(), f"{name} has no citation"
        vals[name] = float(value)
    return vals


@pytest.fixture(scope="module")
def capi():
    from paper_2503_18402_gb300 import build
    build.build()
    from paper_2503_18402_gb300 import capi as c
    return c


def _sat(Mbar):
    H, W = Mbar.shape
    s = np.zeros((H + 1, W + 1))
    s[1:, 1:] = Mbar.cumsum(0).cumsum(1)
    return s


def _spectrum(H=48, W=64, seed=5):
    rng = np.random.default_rng(seed)
    img = rng.random((3, H, W))
    return sch.spectrum_mean(img[None])


def test_library_defaults_are_the_printed_values(capi):
    g = _golden()
    p = capi.sched_params(30000)
    assert p.a == g["a"] and p.gamma == pytest.approx(g["gamma"], abs=0) and p.eta == g["eta"]
    P_init = 12345.0
    s = capi.dg_schedule_init(_sat(_spectrum()), 48, 64, capi.sched_params(30000, P_init=P_init))
    assert s.P_fin == g["pfin0_over_pinit"] * P_init


def test_oracle_defaults_are_the_printed_values():
    g = _golden()
    # Eq. 5 defaults of the oracle: one update from P_fin = 0 with P_add = 1 gives eta
    assert sch.pfin_update(0.0, 1.0) == g["eta"]
    # and gamma: 100 gamma + 10 eta exceeds 100, so the max takes the momentum term
    assert sch.pfin_update(100.0, 10.0) == pytest.approx(100.0 * g["gamma"] + 10.0 * g["eta"], rel=1e-15)


def test_eq8_steady_state_library_and_oracle(capi):
    g = _golden()
    S, P_init, P_add = 30000, 1000.0, 1000.0
    s = capi.dg_schedule_init(_sat(_spectrum()), 48, 64, capi.sched_params(S, P_init=P_init, P_cap=1e12))
    P_fin = s.P_fin
    for _ in range(3000):  # gamma^3000 ~ 5e-27: converged to the fixed point
        capi.dg_schedule_densify(s, S // 2, int(P_add))
        P_fin = sch.pfin_update(P_fin, P_add)
    assert s.P_fin == pytest.approx(g["eq8_pfin_over_padd"] * P_add, rel=1e-9)
    assert P_fin == pytest.approx(g["eq8_pfin_over_padd"] * P_add, rel=1e-9)


def test_eq4_exponent_runs_from_2_to_1(capi):
    g = _golden()
    S, P_init, P_fin, r = 30000, 1e5, 2e6, 3
    for k, want in ((0, g["eq4_exponent_at_start"]), (S, g["eq4_exponent_at_end"])):
        P_k = sch.primitive_target(k, S, r, P_init, P_fin)
        assert math.log((P_fin - P_init) / (P_k - P_init)) / math.log(r) == pytest.approx(want, rel=1e-12)
    # the library's budget at a low-resolution iteration has the same exponent 2 - k/S
    s = capi.dg_schedule_init(_sat(_spectrum()), 48, 64, capi.sched_params(S, P_init=P_init, P_cap=1e12))
    k = 1000
    o = capi.dg_schedule_densify(s, k, 0)
    assert o.r_mod > 1
    expo = math.log((s.P_fin - P_init) / (o.P_target - P_init)) / math.log(o.r_mod)
    assert expo == pytest.approx(g["eq4_exponent_at_start"] - k / S, rel=1e-12)
