"""Host logic of the render launch-shape autotuner (no GPU: timing events are
fakes with the two methods the tuner calls)."""
from __future__ import annotations

import pytest

pytest.importorskip("torch")
autotune = pytest.importorskip("paper_2503_18402_gb300.autotune")
Shape, RenderTuner, bucket = autotune.Shape, autotune.RenderTuner, autotune.bucket


class FakeEvent:
    def __init__(self, t, done=True):
        self.t = t
        self.done = done

    def query(self):
        return self.done

    def elapsed_time(self, other):
        return other.t - self.t


def _tuner(cands, trials=2):
    tu = RenderTuner(device="cpu", candidates=cands, trials=trials)
    tu.rasterizer = lambda shape: None  # no buffers: only the selection logic runs
    return tu


def _time(tu, key, shape, ms, done=True):
    tu.pending.append((key, shape, FakeEvent(0.0), FakeEvent(ms, done)))


def test_bucket_is_half_octaves_of_pixels_and_octaves_of_P():
    assert bucket(1237 * 822, 2_000_000) == bucket(1237 * 822 + 1000, 1_100_000)
    assert bucket(1237 * 822, 2_000_000) != bucket(1237 * 822 // 2, 2_000_000)  # half the pixels: two buckets down
    assert bucket(64 * 64, 1000)[0] == 24 and bucket(64 * 64, 1000)[1] == (1000).bit_length()
    assert bucket(0, 0) == (0, 1)


def test_cycles_candidates_then_keeps_the_fastest_median():
    a, b, c = Shape(8, 1, 1, 0), Shape(8, 1, 1, -1), Shape(16, 1, 1, 0)
    tu = _tuner((a, b, c), trials=2)
    npix, P = 1237 * 822, 2_000_000
    key = bucket(npix, P)
    # while tuning, each pick takes the candidate with the fewest timings (done or in flight)
    seen = []
    for _ in range(3):
        s, _, k = tu.pick(npix, P)
        assert k == key
        seen.append(s)
        _time(tu, key, s, 1.0, done=False)
    assert sorted(seen, key=lambda s: s.label()) == sorted((a, b, c), key=lambda s: s.label())
    tu.pending.clear()
    # first timing of each shape is a warm-up and is dropped; then the median of the rest
    times = {a: [50.0, 3.0, 3.2, 9.0], b: [1.0, 2.9, 2.8, 3.1], c: [2.0, 4.0, 4.1, 3.9]}
    for s, ts in times.items():
        for t in ts[:3]:
            _time(tu, key, s, t)
    s, _, _ = tu.pick(npix, P)
    assert tu.best[key] == b  # medians of (3.0, 3.2) / (2.9, 2.8) / (4.0, 4.1): b
    assert s == b
    # a decided bucket keeps its shape; another bucket starts its own cycle
    s2, _, k2 = tu.pick(64 * 64, 1000)
    assert k2 != key and k2 not in tu.best
    assert tu.summary() == {f"{key[0]}:{key[1]}": b.label()}


def test_events_still_in_flight_are_not_read():
    a, b = Shape(8, 1, 1, 0), Shape(16, 1, 1, 0)
    tu = _tuner((a, b), trials=1)
    key = bucket(100 * 100, 5000)
    for s in (a, b):
        _time(tu, key, s, 9.0)
        _time(tu, key, s, 1.0 if s == a else 2.0)
    _time(tu, key, b, 0.1, done=False)  # would make b the fastest if it were read
    tu.pick(100 * 100, 5000)
    assert tu.best[key] == a
    assert len(tu.pending) == 1


def test_fixed_shape_bypasses_tuning():
    f = Shape(16, 2, 4, 0)
    tu = RenderTuner(device="cpu", fixed=f)
    tu.rasterizer = lambda shape: "rz"
    assert tu.pick(10, 10) == (f, "rz", None)
    tu.stop(None, f, FakeEvent(0.0))  # no key: nothing recorded
    assert tu.pending == []
