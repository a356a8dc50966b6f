"""dg_loss_l1_noalloc: the L1 loss for callers that cannot allocate device memory.

Callers such as plugins whose host application owns every device allocation,
or real-time loops that forbid allocator calls after start-up, cannot hand the
library a workspace.  This entry point keeps its partial sums in a fixed device
array inside the library instead.  The tests call it through the C ABI twice in
a row on different inputs (the shared array keeps the previous call's contents,
which must not leak into the next result), once with a synchronisation between
the calls and once queued back to back on one non-default stream, and compare
loss and gradient with dg_loss_l1, which takes a caller workspace.  The file
name sorts last so that a run stopping at the first failure has run every other
test.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_18402_gb300 import capi  # noqa: E402

pytestmark = pytest.mark.gpu


def _pair(seed, shape):
    rng = np.random.default_rng(seed)
    a = torch.from_numpy(rng.uniform(size=shape).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.uniform(size=shape).astype(np.float32)).cuda()
    return a, b


def test_noalloc_matches_workspace_entry_point_twice():
    # second call smaller than the first: stale partials of call 1 beyond
    # call 2's block count must not be read
    for seed, shape in ((11, (3, 822, 1237)), (12, (3, 97, 131))):
        img, tgt = _pair(seed, shape)
        n = img.numel()
        d_ref = torch.empty_like(img)
        l_ref = torch.zeros(1, device="cuda")
        ws = torch.empty(capi.dg_loss_workspace_size(n), dtype=torch.uint8, device="cuda")
        capi.dg_loss_l1(img, tgt, n, d_ref, l_ref, ws, ws.numel())
        d = torch.empty_like(img)
        l = torch.full((1,), -1.0, device="cuda")
        capi.dg_loss_l1_noalloc(img, tgt, n, d, l)
        torch.cuda.synchronize()
        assert abs(l.item() - l_ref.item()) <= 1e-6 * abs(l_ref.item())
        assert torch.equal(d, d_ref)
        exact = float(torch.mean(torch.abs(img.double() - tgt.double())))
        assert abs(l.item() - exact) <= 1e-6 * exact


def test_noalloc_two_calls_in_order_on_one_stream():
    # two calls queued on one non-default stream with no synchronisation
    # between them: the stream orders them, so each sees its own partials
    side = torch.cuda.Stream()
    cases = [_pair(21, (3, 411, 618)), _pair(22, (3, 205, 309))]
    refs = []
    for img, tgt in cases:
        n = img.numel()
        d_ref = torch.empty_like(img)
        l_ref = torch.zeros(1, device="cuda")
        ws = torch.empty(capi.dg_loss_workspace_size(n), dtype=torch.uint8, device="cuda")
        capi.dg_loss_l1(img, tgt, n, d_ref, l_ref, ws, ws.numel())
        refs.append((d_ref, l_ref))
    outs = [(torch.empty_like(img), torch.full((1,), -1.0, device="cuda")) for img, _ in cases]
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        for (img, tgt), (d, l) in zip(cases, outs):
            capi.dg_loss_l1_noalloc(img, tgt, img.numel(), d, l, side)
    side.synchronize()
    for (d, l), (d_ref, l_ref) in zip(outs, refs):
        assert abs(l.item() - l_ref.item()) <= 1e-6 * abs(l_ref.item())
        assert torch.equal(d, d_ref)


def test_noalloc_rejects_sizes_beyond_its_limit():
    t = torch.zeros(4, device="cuda")
    with pytest.raises(capi.DashGSError) as e:
        capi.dg_loss_l1_noalloc(t, t, capi.L1_NOALLOC_MAX_N + 1, t, t)
    assert e.value.status == capi.DG_ERR_ARG and "limit" in str(e.value)
    with pytest.raises(capi.DashGSError):
        capi.dg_loss_l1_noalloc(t, t, 0, t, t)
