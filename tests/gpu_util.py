"""Helpers for the GPU parity tests: upload seeded inputs and call the library's C ABI."""
import numpy as np

import nrv_inputs as I
from oracle import unet


def torch_dev():
    import torch
    return torch.device("cuda:0")


def upload_scene(sc):
    import torch
    from paper_2407_19097_gb300 import nrv
    dev = torch_dev()
    xyz = torch.from_numpy(np.ascontiguousarray(sc.xyz)).to(dev)
    attr = torch.from_numpy(np.ascontiguousarray(sc.attr).view(np.int32)).to(dev)
    return nrv.Scene(xyz, attr, sc.n_words)


def gpu_raster(scene, views, planes=True, k=None):
    """Run nrv_rasterize; return per view (key u64, depth u32, mask u8, gattr u32 [K,H,W])."""
    import torch
    from paper_2407_19097_gb300 import nrv
    dev = torch_dev()
    k = scene.n_words if k is None else k
    keys = [torch.empty((v.height, v.width), dtype=torch.int64, device=dev) for v in views]
    if planes:
        depth = [torch.empty((v.height, v.width), dtype=torch.int32, device=dev) for v in views]
        mask = [torch.empty((v.height, v.width), dtype=torch.uint8, device=dev) for v in views]
        gattr = [torch.empty((k, v.height, v.width), dtype=torch.int32, device=dev) for v in views]
    else:
        depth = mask = gattr = None
    nrv.rasterize(scene, views, keys, depth, mask, gattr)
    torch.cuda.synchronize()
    out = []
    for i in range(len(views)):
        kk = keys[i].cpu().numpy().view(np.uint64)
        if planes:
            out.append((kk, depth[i].cpu().numpy().view(np.uint32), mask[i].cpu().numpy(),
                        gattr[i].cpu().numpy().view(np.uint32)))
        else:
            out.append((kk,))
    return out


def make_params(c0, seed=1, bias_sigma=0.0):
    flat = []
    for t, (name, kind, ci, co) in enumerate(unet.layers(c0)):
        fi, fo = unet.fans(kind, ci, co)
        flat.append(I.xavier_uniform(seed, 1000 + t, unet.weight_shape(kind, ci, co), fi, fo).ravel())
        if bias_sigma > 0:
            flat.append((bias_sigma * I.normal_array(seed, 2000 + t, co)).astype(np.float32))
        else:
            flat.append(np.zeros(co, np.float32))
    return np.concatenate(flat).astype(np.float32)


def psnr_range(a, ref):
    """PSNR with the peak set to the oracle output's dynamic range."""
    ref = np.asarray(ref, np.float64)
    r = float(ref.max() - ref.min())
    mse = float(np.mean((np.asarray(a, np.float64) - ref) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(r * r / mse)
