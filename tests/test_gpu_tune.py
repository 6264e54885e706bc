"""Tuned launch choices (render-pass variant; the tensor-core conv's read-ahead and CTAs per SM):
a process that tunes and saves its choices, and a second process that loads them through
NRV_TUNE_CACHE, makes no tuning run and renders the same frame bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

SCRIPT = r'''
import os, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import nrv_inputs as I
from paper_2407_19097_gb300 import nrv
from gpu_util import make_params, upload_scene
sc = I.trajectory_scene(30011, 35, seed=2)              # 1.05M points: the render pass tunes
scene = upload_scene(sc)
c0 = len(sc.channels) + 2
net = nrv.Net(c0)
net.set_params(torch.from_numpy(make_params(c0, seed=2)).to("cuda:0"))
views = [I.fitted_view(sc, 320, 200), I.fitted_view(sc, 320, 200, direction=(1, 0.3, 0.2))]
ds, do = I.depth_normalisation(sc, views[0])
desc = nrv.make_pack_desc(sc.channels, ds, do)
outs = [torch.empty((200, 320, 3), device="cuda:0") for _ in views]
for _ in range(3):
    nrv.render_batch(scene, net, desc, views, outs, nrv.PREC_BF16)
    nrv.render_batch(scene, net, desc, views[:1], outs[:1], nrv.PREC_BF16)
torch.cuda.synchronize()
np.save(sys.argv[1], np.stack([o.cpu().numpy() for o in outs]))
if len(sys.argv) > 2:
    nrv.tune_save(sys.argv[2])
print("timings", nrv.lib().nrv_tune_timings(), "count", nrv.lib().nrv_tune_count())
'''


def _run(tmp, args, env_extra):
    script = tmp / "tune_run.py"
    script.write_text(SCRIPT.format(root=ROOT))
    env = dict(os.environ, PYTHONPATH=os.path.join(ROOT, "tests"), NRV_TC_TUNE="1", **env_extra)
    env.pop("NRV_VIS_VARIANT", None)
    r = subprocess.run([sys.executable, str(script), *args], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("timings")][-1].split()
    return int(line[1]), int(line[3])


def test_cached_choices_are_reused_and_frames_identical(tmp_path):
    cache = tmp_path / "tune.txt"
    timed_a, count_a = _run(tmp_path, [str(tmp_path / "a.npy"), str(cache)], {"NRV_TUNE_CACHE": ""})
    assert timed_a > 0 and count_a > 0
    text = cache.read_text()
    assert "render multi=1" in text and "render multi=0" in text and "conv " in text
    timed_b, count_b = _run(tmp_path, [str(tmp_path / "b.npy")], {"NRV_TUNE_CACHE": str(cache)})
    assert timed_b == 0 and count_b == count_a
    assert np.array_equal(np.load(tmp_path / "a.npy"), np.load(tmp_path / "b.npy"))

