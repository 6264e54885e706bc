"""Pins for the gated network oracle (Sec. 3.3's gated convolutions with ELU, 1x1 G-buffer
projection with multiscale injection): the whole forward against the same network written
with torch's float64 library routines (conv2d, conv_transpose2d, avg_pool2d, elu, sigmoid),
and closed forms of the gating."""
import numpy as np
import pytest

import nrv_inputs as I
from oracle import gated

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _params(c0, seed=3):
    flat = []
    for t, (name, kind, ci, co) in enumerate(gated.layers(c0)):
        for k, shp in enumerate(gated.shapes(kind, ci, co)):
            if len(shp) == 1:
                flat.append((0.1 * I.normal_array(seed, 3000 + 8 * t + k, shp[0])).astype(np.float32))
            else:
                k2 = 9 if kind == "gated" else (4 if kind == "convT2" else 1)
                flat.append(I.xavier_uniform(seed, 2000 + 8 * t + k, shp, ci * k2, co * k2).ravel())
    return np.concatenate(flat).astype(np.float32)


def _torch_forward(x, P):
    t = lambda a: torch.from_numpy(np.asarray(a, np.float64))
    X = t(x).permute(0, 3, 1, 2)
    gt = lambda z, wf, bf, wg, bg: F.elu(F.conv2d(z, t(wf), t(bf), padding=1)) * torch.sigmoid(
        F.conv2d(z, t(wg), t(bg), padding=1))
    w, b = P["inj"]
    g = [F.conv2d(X, t(w)[:, :, None, None], t(b))]
    for _ in range(3):
        g.append(F.avg_pool2d(g[-1], 2))
    e = [gt(g[0], *P["e0"])]
    for l in range(1, 4):
        e.append(gt(torch.cat([F.avg_pool2d(e[-1], 2), g[l]], 1), *P["e%d" % l]))
    d = e[3]
    for l in (2, 1, 0):
        w, b = P["up%d" % l]
        u = F.conv_transpose2d(d, t(w), t(b), stride=2)
        d = gt(torch.cat([u, e[l]], 1), *P["d%d" % l])
    w, b = P["head"]
    return F.conv2d(d, t(w)[:, :, None, None], t(b)).permute(0, 2, 3, 1).numpy()


@pytest.mark.parametrize("c0", [5, 8])
def test_forward_matches_torch_float64(c0):
    rng = np.random.default_rng(c0)
    x = rng.standard_normal((2, 16, 24, c0))
    flat = _params(c0)
    assert flat.size == gated.param_count(c0)
    P = gated.unflatten(flat, c0)
    np.testing.assert_allclose(gated.forward(x, P), _torch_forward(x, P), rtol=1e-11, atol=1e-12)


def test_gating_closed_forms():
    """A 1-channel gated conv with only centre taps: out = ELU(a x + b) * sigmoid(c x + d)."""
    x = np.linspace(-3, 3, 64).reshape(1, 8, 8, 1)
    wf = np.zeros((1, 1, 3, 3)); wf[0, 0, 1, 1] = 1.5
    wg = np.zeros((1, 1, 3, 3)); wg[0, 0, 1, 1] = -0.7
    y = gated.gated(x, wf, np.array([0.2]), wg, np.array([0.4]))
    f = 1.5 * x + 0.2
    want = np.where(f > 0, f, np.exp(f) - 1) / (1 + np.exp(-(-0.7 * x + 0.4)))
    np.testing.assert_allclose(y, want, rtol=1e-13)
    assert gated.elu(np.array([-1e-300]))[0] == -1e-300 and gated.elu(np.array([2.0]))[0] == 2.0
