"""Network parameters in and out of a handle: the seeded Xavier-uniform draw of
nrv_net_init_params equals the host generator's (SplitMix64, the same published definition on both
sides) bit for bit; nrv_net_get_params returns what was loaded; nrv_net_save / nrv_net_load
round-trip the parameters and the FP8 scales, and a reloaded net shades identically."""
import numpy as np
import pytest

import nrv_inputs as I
from gpu_util import torch_dev

pytestmark = pytest.mark.gpu


def _host_xavier(c0, seed):
    from paper_2407_19097_gb300 import nrv
    flat = np.zeros(nrv.param_count(c0), np.float32)
    for t, (name, kind, ci, co, wo, bo) in enumerate(nrv.layer_table(c0)):
        k2 = {0: 9, 1: 4, 2: 1}[kind]
        shape = {0: (co, ci, 3, 3), 1: (ci, co, 2, 2), 2: (co, ci)}[kind]
        flat[wo:wo + int(np.prod(shape))] = I.xavier_uniform(seed, 1000 + t, shape, ci * k2,
                                                             co * k2).ravel()
    return flat


@pytest.mark.parametrize("c0,seed", [(5, 1), (7, 123456789)])
def test_init_params_matches_host_draw(c0, seed):
    import torch
    from paper_2407_19097_gb300 import nrv
    net = nrv.Net(c0)
    p = torch.full((nrv.param_count(c0),), float("nan"), device=torch_dev())
    net.init_params(seed, p)
    got = p.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), _host_xavier(c0, seed).view(np.uint32))
    back = torch.empty_like(p)
    net.get_params(back)
    assert torch.equal(back, p)


def test_save_load_round_trip(tmp_path):
    import torch
    from paper_2407_19097_gb300 import nrv
    dev = torch_dev()
    c0, H, W = 5, 64, 96
    a = nrv.Net(c0)
    p = torch.empty((nrv.param_count(c0),), device=dev)
    a.init_params(42, p)
    p += 0.01 * torch.randn_like(p)          # biases non-zero too
    a.set_params(p)
    scales = [0.01 * (1 + i) for i in range(21)]
    a.set_act_scales(scales)
    path = tmp_path / "net.bin"
    a.save(path)
    b = nrv.Net(c0)
    b.load(path)
    got = torch.empty_like(p)
    b.get_params(got)
    assert torch.equal(got, p)
    assert np.allclose(b.act_scales(), np.float32(scales), rtol=0, atol=0)
    x = torch.randn((1, H, W, 8), device=dev).to(torch.bfloat16)
    x[..., c0:] = 0
    ya = torch.empty((1, H, W, 3), device=dev)
    yb = torch.empty_like(ya)
    a.shade(x, 1, H, W, nrv.PREC_BF16, ya)
    b.shade(x, 1, H, W, nrv.PREC_BF16, yb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    # another input width, and a file that is not a network, are refused
    c = nrv.Net(6)
    assert nrv.lib().nrv_net_load(c.h, str(path).encode(), None) == nrv.NRV_ERR_ARG
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NRVNET01" + b"\0" * 7)
    assert nrv.lib().nrv_net_load(b.h, str(bad).encode(), None) == nrv.NRV_ERR_ARG
