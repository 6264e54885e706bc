"""FP8 (E4M3) network (App. B quantisation, taken to 8 bits): every conv and transposed conv
layer alone against the oracle on the same E4M3 inputs, with the weights quantised the same
way (per output column, scale = max|column| / 448, decided in FP32 on both sides); and the
whole calibrated FP8 network on a rendered frame against the float64 oracle."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import make_params, psnr_range, torch_dev, upload_scene
from oracle import unet

pytestmark = pytest.mark.gpu

f32 = np.float32
CODES = np.arange(256, dtype=np.uint8)
VALS = oracle.e4m3_value(CODES)
# every finite E4M3 value in increasing order, to measure distances in code steps
ORDER = np.unique(VALS[np.isfinite(VALS)])


def _steps(a_codes, b_codes):
    a = np.searchsorted(ORDER, oracle.e4m3_value(a_codes))
    b = np.searchsorted(ORDER, oracle.e4m3_value(b_codes))
    return np.abs(a - b)


# scale index of each layer's first input, second input, output (0 = network input)
ACTS = ["e0a", "e0b", "p0", "e1a", "e1b", "p1", "e2a", "e2b", "p2", "e3a", "e3b", "up3", "d2a",
        "d2b", "up2", "d1a", "d1b", "up1", "d0a", "d0b"]
IDX = {a: 1 + i for i, a in enumerate(ACTS)}
IDX["x"] = 0
LAYER_IO = {"e0a": ("x", None, "e0a"), "e0b": ("e0a", None, "e0b"), "e1a": ("p0", None, "e1a"),
            "e1b": ("e1a", None, "e1b"), "e2a": ("p1", None, "e2a"), "e2b": ("e2a", None, "e2b"),
            "e3a": ("p2", None, "e3a"), "e3b": ("e3a", None, "e3b"), "up3": ("e3b", None, "up3"),
            "d2a": ("up3", "e2b", "d2a"), "d2b": ("d2a", None, "d2b"), "up2": ("d2b", None, "up2"),
            "d1a": ("up2", "e1b", "d1a"), "d1b": ("d1a", None, "d1b"), "up1": ("d1b", None, "up1"),
            "d0a": ("up1", "e0b", "d0a"), "d0b": ("d0a", None, "d0b")}


def _scales():
    s = [f32(0.01 * (1.0 + 0.13 * k)) for k in range(21)]
    for p, e in (("p0", "e0b"), ("p1", "e1b"), ("p2", "e2b")):
        s[IDX[p]] = s[IDX[e]]
    return s


LAYERS = [(i, name, kind) for i, (name, kind, _, _) in enumerate(unet.layers(5)) if kind != "conv1"]


@pytest.mark.parametrize("layer,name,kind", LAYERS)
def test_fp8_layer(layer, name, kind):
    import torch
    from paper_2407_19097_gb300 import nrv
    c0 = 5
    flat = make_params(c0, seed=layer + 71, bias_sigma=0.1)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    sc = _scales()
    net.set_act_scales(sc)
    src1, src2, dst = LAYER_IO[name]
    s1, s_out = sc[IDX[src1]], sc[IDX[dst]]
    s2 = sc[IDX[src2]] if src2 else None
    _, _, ci, co = unet.layers(c0)[layer]
    cin = 16 if layer == 0 else ci
    c1 = cin // 2 if src2 else cin
    n, h, w = 2, 5, 300
    rng = np.random.default_rng(layer)
    v1 = rng.standard_normal((n, h, w, c1)) * 1.5
    if layer == 0:
        v1[..., c0:] = 0.0
    q1 = oracle.e4m3_bits((v1 / s1).astype(f32))
    q2 = oracle.e4m3_bits((rng.standard_normal((n, h, w, cin - c1)) * 1.5 / s2).astype(f32)) if src2 else None
    dev = torch_dev()
    x1 = torch.from_numpy(q1).to(dev)
    x2 = torch.from_numpy(q2).to(dev) if src2 else None
    oh, ow = (h, w) if kind == "conv3" else (2 * h, 2 * w)
    y = torch.empty((n, oh, ow, co), dtype=torch.uint8, device=dev)
    nrv.check(nrv.lib().nrv_net_run_layer(net.h, layer, nrv._ptr(x1), nrv._ptr(x2), n, h, w,
                                          nrv.PREC_FP8_E4M3, nrv._ptr(y), nrv._stream()))
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    # the oracle quantises the weights the same way, in FP32
    W, b = unet.unflatten(flat.astype(np.float64), c0)[name]
    W32 = W.astype(f32)
    fold = f32(s2) / f32(s1) if src2 else f32(1.0)
    if kind == "conv3":
        Wf = W32.copy()
        if src2:
            Wf[:, c1:] = (W32[:, c1:] * fold).astype(f32)
        amax = np.abs(Wf).reshape(co, -1).max(axis=1).astype(f32)
        sw = np.where(amax > 0, amax / f32(448.0), f32(1.0)).astype(f32)
        w8 = oracle.e4m3_value(oracle.e4m3_bits((Wf / sw[:, None, None, None]).astype(f32)))
        xv = oracle.e4m3_value(q1)
        if src2:
            xv = np.concatenate([xv, oracle.e4m3_value(q2)], axis=-1)
        acc = unet.conv3(xv[..., :ci], w8, np.zeros(co))
        colscale = (f32(s1) * sw).astype(f32)
        bias = b.astype(f32)
    else:
        # columns n = (2a + b) * co + o; scale per column over the c inputs
        amax = np.abs(W32).max(axis=0).astype(f32)               # [co, 2, 2]
        sw = np.where(amax > 0, amax / f32(448.0), f32(1.0)).astype(f32)
        w8 = oracle.e4m3_value(oracle.e4m3_bits((W32 / sw[None]).astype(f32)))
        acc = unet.convT2(oracle.e4m3_value(q1), w8, np.zeros(co))
        colscale = None
        bias = b.astype(f32)
    if kind == "conv3":
        v = (acc.astype(f32).astype(np.float64) * colscale + bias).astype(f32)
        v = np.maximum(v, 0)
    else:
        # the per-column scale depends on the output position (a, b)
        cs = (f32(s1) * sw).astype(f32)                          # [co, 2, 2]
        v = np.empty_like(acc, dtype=f32)
        for a in range(2):
            for c in range(2):
                v[:, a::2, c::2, :] = (acc[:, a::2, c::2, :].astype(f32).astype(np.float64)
                                       * cs[:, a, c] + bias).astype(f32)
    ref = oracle.e4m3_bits((v * (f32(1.0) / f32(s_out))).astype(f32))
    steps = _steps(got, ref)
    assert np.mean(steps == 0) >= 0.98 and steps.max() <= 1, (np.mean(steps == 0), steps.max())
    assert net.backends()[layer] == 1


def test_fp8_e4m3_network_frame():
    """NRV_PREC_FP8_E4M3 (every stored tensor E4M3), calibrated on the frame itself (BF16),
    against the float64 oracle.  This mode is documented as below the reduced-precision bar
    (max abs <= 2e-2): its 3-bit mantissas compound over the full-resolution layers.  The test
    holds it to the PSNR half of the bar and to a max-abs error that stays within 0.15."""
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.trajectory_scene(2000, 35, seed=2)
    c0 = len(sc.channels) + 2
    scene = upload_scene(sc)
    dev = torch_dev()
    H, W = 120, 200
    view = I.fitted_view(sc, W, H)
    ds, do = I.depth_normalisation(sc, view)
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    key = torch.empty((H, W), dtype=torch.int64, device=dev)
    depth = torch.empty((H, W), dtype=torch.int32, device=dev)
    mask = torch.empty((H, W), dtype=torch.uint8, device=dev)
    gattr = torch.empty((3, H, W), dtype=torch.int32, device=dev)
    nrv.rasterize(scene, [view], [key], [depth], [mask], [gattr])
    xb = torch.empty((H, W, 8), dtype=torch.bfloat16, device=dev)
    nrv.pack(depth, mask, gattr, H, W, desc, nrv.PREC_BF16, xb)
    flat = make_params(c0, seed=5, bias_sigma=0.05)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(flat).to(dev))
    net.calibrate(xb, 1, H, W)
    s_in = net.act_scales()[0]
    x8 = torch.empty((H, W, 16), dtype=torch.uint8, device=dev)
    nrv.pack(depth, mask, gattr, H, W, desc, nrv.PREC_FP8_E4M3, x8, 1.0 / s_in)
    out = torch.empty((H, W, 3), device=dev)
    net.shade(x8, 1, H, W, nrv.PREC_FP8_E4M3, out)
    torch.cuda.synchronize()
    _, d, m, g = oracle.rasterize(sc, view)
    x = oracle.pack(d, m, g, sc.channels, ds, do, H, W, 8, 0).astype(np.float64)
    ref = unet.forward(x[None, :, :, :c0], unet.unflatten(flat, c0))[0]
    got = out.cpu().numpy()
    p = psnr_range(got, ref)
    err = float(np.abs(got - ref).max())
    print(f"E4M3 frame vs float64: PSNR {p:.2f} dB, max abs {err:.4f}")
    assert all(b == 1 for b, k in zip(net.backends(), [l[1] for l in unet.layers(c0)]) if k != "conv1")
    assert p >= 40.0 and err <= 0.15, (p, err)


def test_fp8_network_frame_meets_target():
    """NRV_PREC_FP8, the FP8 network (E4M3 for levels 1-3, BF16 for level 0, from the BF16
    input), calibrated on the frame, against the float64 oracle: the accuracy bar of the
    method's reduced-precision pass, PSNR >= 45 dB over the oracle's output range and max abs
    <= 2e-2.  (All-E4M3 storage misses the max-abs bar: the errors of 3-bit mantissas compound
    over the full-resolution layers.)"""
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.trajectory_scene(2000, 35, seed=2)
    c0 = len(sc.channels) + 2
    scene = upload_scene(sc)
    dev = torch_dev()
    H, W = 120, 200
    view = I.fitted_view(sc, W, H)
    ds, do = I.depth_normalisation(sc, view)
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    key = torch.empty((H, W), dtype=torch.int64, device=dev)
    depth = torch.empty((H, W), dtype=torch.int32, device=dev)
    mask = torch.empty((H, W), dtype=torch.uint8, device=dev)
    gattr = torch.empty((3, H, W), dtype=torch.int32, device=dev)
    nrv.rasterize(scene, [view], [key], [depth], [mask], [gattr])
    hn, wn = (H + 7) // 8 * 8, (W + 7) // 8 * 8
    xb = torch.zeros((hn, wn, 8), dtype=torch.bfloat16, device=dev)
    nrv.pack(depth, mask, gattr, H, W, desc, nrv.PREC_FP8, xb)
    flat = make_params(c0, seed=5, bias_sigma=0.05)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(flat).to(dev))
    net.calibrate(xb, 1, H, W)
    out = torch.empty((H, W, 3), device=dev)
    net.shade(xb, 1, H, W, nrv.PREC_FP8, out)
    torch.cuda.synchronize()
    _, d, m, g = oracle.rasterize(sc, view)
    x = oracle.pack(d, m, g, sc.channels, ds, do, hn, wn, 8, 0).astype(np.float64)
    ref = unet.forward(x[None, :, :, :c0], unet.unflatten(flat, c0))[0][:H, :W]
    got = out.cpu().numpy()
    p = psnr_range(got, ref)
    err = float(np.abs(got - ref).max())
    assert all(b == 1 for b, k in zip(net.backends(), [l[1] for l in unet.layers(c0)]) if k != "conv1")
    assert p >= 45.0 and err <= 2e-2, (p, err)
