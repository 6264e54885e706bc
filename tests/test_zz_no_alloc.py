"""nrv_l1_loss_noalloc: the L1 loss for callers that cannot allocate device memory (a host
application whose memory pool owns the device, a frame loop that must not stall on cudaMalloc,
a plug-in handed only its buffers).  Called through the C ABI and checked against nrv_l1_loss,
the allocating entry point, on two calls in a row; sizes beyond its fixed scratch are refused.
This file is collected last so a stop-at-first-failure run has run every other test first."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call(fn, y, t, n, loss, dy):
    from paper_2407_19097_gb300 import nrv
    return fn(ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(t.data_ptr()), n,
              ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(dy.data_ptr()) if dy is not None else None,
              nrv._stream())


def test_noalloc_matches_allocating_entry_point():
    import torch
    from paper_2407_19097_gb300 import nrv
    L = nrv.lib()
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(17)
    for n in (3 * 1920 * 1080 + 5, 1000):          # a large call, then a smaller one
        y = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
        t = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
        t[::7] = y[::7]                              # exact zeros of y - t
        l_ref, l_new = torch.zeros(1, device=dev), torch.zeros(1, device=dev)
        d_ref, d_new = torch.empty_like(y), torch.empty_like(y)
        assert _call(L.nrv_l1_loss, y, t, n, l_ref, d_ref) == nrv.NRV_OK
        assert _call(L.nrv_l1_loss_noalloc, y, t, n, l_new, d_new) == nrv.NRV_OK, L.nrv_last_error()
        torch.cuda.synchronize()
        assert abs(l_new.item() - l_ref.item()) <= 1e-6 * abs(l_ref.item())
        assert torch.equal(d_new, d_ref)


def test_noalloc_allocates_nothing_after_warm_up():
    """After one warm-up call (which may load the library's device code), calls leave the
    device's free memory unchanged."""
    import torch
    from paper_2407_19097_gb300 import nrv
    L = nrv.lib()
    dev = torch.device("cuda:0")
    n = 1 << 22
    y = torch.randn(n, device=dev)
    t = torch.randn(n, device=dev)
    loss, dy = torch.zeros(1, device=dev), torch.empty_like(y)
    assert _call(L.nrv_l1_loss_noalloc, y, t, n, loss, dy) == nrv.NRV_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(3):
        assert _call(L.nrv_l1_loss_noalloc, y, t, n, loss, dy) == nrv.NRV_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)


def test_noalloc_refuses_sizes_beyond_its_scratch():
    import torch
    from paper_2407_19097_gb300 import nrv
    L = nrv.lib()
    dev = torch.device("cuda:0")
    y = torch.zeros(16, device=dev)
    loss = torch.full((1,), 7.0, device=dev)
    limit = 134217728
    assert _call(L.nrv_l1_loss_noalloc, y, y, limit + 1, loss, None) == nrv.NRV_ERR_ARG
    assert b"at most" in L.nrv_last_error()
    torch.cuda.synchronize()
    assert loss.item() == 7.0                        # nothing was launched
