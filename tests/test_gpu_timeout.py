"""The bounded wait between thread blocks gives up and reports DG_ERR_TIMEOUT.

The depth-order passes of the binning sum the digit counts of earlier tiles
by walking back over their published look-back words (decoupled look-back);
a word that is never published would stall the walk, so every wait is
bounded and records DG_ERR_TIMEOUT.  dg_lookback_probe runs that same device
function on a caller-built word array: an unpublished predecessor with a
small poll limit makes the wait give up in microseconds and return, with the
GPU left usable (the next call works).  Nothing here starves a real pass.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_18402_gb300 import capi  # noqa: E402

pytestmark = pytest.mark.gpu


def _words(states_counts, stride=4, digit=1):
    """[tiles][stride] uint64 words; column `digit` from (state, count) pairs,
    the other columns hold junk that the walk must not read."""
    w = np.full((len(states_counts), stride), 0x7777, dtype=np.uint64)
    for t, (st, c) in enumerate(states_counts):
        w[t, digit] = np.uint64((st << 62) | c)
    return torch.from_numpy(w.view(np.int64)).cuda()


def _probe(look, tile, max_polls, stride=4, digit=1):
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    err = torch.full((1,), 123, dtype=torch.int32, device="cuda")
    capi.dg_lookback_probe(look, tile, stride, digit, max_polls, out, err)
    torch.cuda.synchronize()
    return int(out.item()), int(err.item())


def test_published_words_sum_exactly():
    counts = [5, 7, 11, 13, 17, 19, 23, 29, 31, 37]
    look = _words([(2, counts[0])] + [(1, c) for c in counts[1:]])
    assert _probe(look, 10, 0) == (sum(counts), 0)
    # an inclusive word stops the walk (its count already holds everything before it)
    look = _words([(1, 1000), (0, 0), (2, 50)] + [(1, c) for c in counts[3:]])
    assert _probe(look, 10, 0) == (50 + sum(counts[3:]), 0)
    # more than one window (16 words) of aggregates
    many = [(2, 3)] + [(1, i) for i in range(1, 40)]
    assert _probe(_words(many), 40, 0) == (3 + sum(range(1, 40)), 0)


@pytest.mark.parametrize("max_polls", [0, 1, 64])
def test_unpublished_predecessor_gives_up_with_timeout(max_polls):
    counts = [5, 7, 11, 13, 17, 19, 23, 29, 31, 37]
    # tile 3 never publishes; no inclusive word after it
    look = _words([(2, counts[0]), (1, counts[1]), (1, counts[2]), (0, 0)] + [(1, c) for c in counts[4:]])
    total, err = _probe(look, 10, max_polls)
    assert err == capi.DG_ERR_TIMEOUT
    assert total == sum(counts[4:])  # the words walked before the stall
    # the context is still usable: the next wait on published words succeeds
    look2 = _words([(2, 4), (1, 6)])
    assert _probe(look2, 2, max_polls) == (10, 0)


def test_probe_rejects_bad_arguments():
    t = torch.zeros(8, dtype=torch.int64, device="cuda")
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    for args in ((t, -1, 4, 0, 0), (t, 1, 0, 0, 0), (t, 1, 4, 4, 0), (t, 1, 4, 0, -1), (t, 1, 4, 0, (1 << 20) + 1)):
        with pytest.raises(capi.DashGSError) as ex:
            capi.dg_lookback_probe(*args, t, e)
        assert ex.value.status == capi.DG_ERR_ARG
