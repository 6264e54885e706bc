"""Points across GPUs (the multi-GPU split of the render pass), emulated on one GPU: shards of
a scene rendered with their global index bases, key images combined by a minimum in signed
order (the library's sign flip, then torch.minimum standing in for the MIN collective), resolved
by owner and added -- bit-exact against the whole scene rendered at once and the oracle."""
import os

import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import torch_dev

pytestmark = pytest.mark.gpu


def _scene(sc, lo, hi):
    import torch
    from paper_2407_19097_gb300 import nrv
    xyz = torch.from_numpy(np.ascontiguousarray(sc.xyz[lo:hi])).to(torch_dev())
    attr = torch.from_numpy(np.ascontiguousarray(sc.attr[lo:hi]).view(np.int32)).to(torch_dev())
    return nrv.Scene(xyz, attr, sc.n_words, index_base=lo)


@pytest.mark.parametrize("variant", [None, "0", "8"])
def test_shards_combine_to_the_whole_scene(variant):
    import torch
    from paper_2407_19097_gb300 import nrv, split
    sc = I.trajectory_scene(30011, 35, seed=2)              # 1.05M points, ragged shards
    view = I.fitted_view(sc, 640, 360)
    H, W = view.height, view.width
    world = 3
    if variant is not None:
        os.environ["NRV_VIS_VARIANT"] = variant
    try:
        shards = [_scene(sc, *split.shard_range(sc.n, r, world)) for r in range(world)]
        keys = []
        for s in shards:
            k = torch.empty((H, W), dtype=torch.int64, device=torch_dev())
            nrv.rasterize(s, [view], [k])
            nrv.keys_flip_sign(k)
            keys.append(k)
        comb = keys[0].clone()
        for k in keys[1:]:
            torch.minimum(comb, k, out=comb)
        nrv.keys_flip_sign(comb)
        depth = torch.zeros((H, W), dtype=torch.int64, device=torch_dev())
        mask = torch.zeros((H, W), dtype=torch.int64, device=torch_dev())
        gattr = torch.zeros((sc.n_words, H, W), dtype=torch.int64, device=torch_dev())
        for s in shards:
            d = torch.empty((H, W), dtype=torch.int32, device=torch_dev())
            m = torch.empty((H, W), dtype=torch.uint8, device=torch_dev())
            g = torch.empty((sc.n_words, H, W), dtype=torch.int32, device=torch_dev())
            nrv.resolve(s, view, comb, d, m, g)
            depth += d.to(torch.int64) & 0xFFFFFFFF
            mask += m.to(torch.int64)
            gattr += g.to(torch.int64) & 0xFFFFFFFF
        torch.cuda.synchronize()
    finally:
        if variant is not None:
            del os.environ["NRV_VIS_VARIANT"]
    rk, rd, rm, rg = oracle.rasterize(sc, view)
    assert np.array_equal(comb.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(depth.cpu().numpy().astype(np.uint32), rd)
    assert np.array_equal(mask.cpu().numpy().astype(np.uint8), rm)
    assert np.array_equal(gattr.cpu().numpy().astype(np.uint32), rg)
    assert (rm > 0).mean() > 0.05
