"""The C ABI library loads on the CPU host and exports every symbol include/nrv.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nrv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nrv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_19097_gb300 import build_lib, nrv
    build_lib.build()
    return nrv.lib()


def test_every_declared_symbol_is_exported(lib):
    from paper_2407_19097_gb300 import nrv
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(nrv.SIGNATURES), set(names) ^ set(nrv.SIGNATURES)


def test_host_side_queries(lib):
    from paper_2407_19097_gb300 import nrv
    from oracle import unet
    assert lib.nrv_version() == 1
    assert lib.nrv_pad8(540) == 544 and lib.nrv_pad8(1080) == 1080
    assert lib.nrv_netin_channels(nrv.PREC_FP8_E4M3) == 16 and lib.nrv_netin_channels(nrv.PREC_BF16) == 8
    # render-pass variants: brute force and culling ones, for one view and for batches
    assert lib.nrv_render_variants(0) >= 4 and lib.nrv_render_variants(1) >= 4
    for c0 in (3, 5, 6, 7):
        assert nrv.param_count(c0) == unet.param_count(c0)
        table = nrv.layer_table(c0)
        off = 0
        for (name, kind, ci, co, wo, bo), (n2, k2, ci2, co2) in zip(table, unet.layers(c0)):
            assert (name, ci, co) == (n2, ci2, co2)
            assert wo == off
            off = bo + co
        assert off == unet.param_count(c0)


def test_argument_errors(lib):
    from paper_2407_19097_gb300 import nrv
    d = nrv.nrv_scene_desc(1 << 32, 16, 16, 4, 3)
    h = ctypes.c_void_p()
    assert lib.nrv_create_scene(ctypes.byref(d), ctypes.byref(h)) == nrv.NRV_ERR_ARG
    assert b"2^32" in lib.nrv_last_error()
    d = nrv.nrv_scene_desc(10, 8, 16, 4, 3)          # misaligned xyz
    assert lib.nrv_create_scene(ctypes.byref(d), ctypes.byref(h)) == nrv.NRV_ERR_ARG
    d = nrv.nrv_scene_desc(10, 16, 16, 3, 3)         # bad stride
    assert lib.nrv_create_scene(ctypes.byref(d), ctypes.byref(h)) == nrv.NRV_ERR_ARG
    d = nrv.nrv_scene_desc(10, 16, 16, 4, 5)         # K > stride
    assert lib.nrv_create_scene(ctypes.byref(d), ctypes.byref(h)) == nrv.NRV_ERR_ARG
    d = nrv.nrv_scene_desc(10, 16, 16, 4, 3, 1, (1 << 32) - 10)   # shard indices past 2^32 - 1
    assert lib.nrv_create_scene(ctypes.byref(d), ctypes.byref(h)) == nrv.NRV_ERR_ARG
    d = nrv.nrv_scene_desc(1 << 30, 16, 16, 4, 3, 8, 0)       # strided indices past 2^32 - 1
    assert lib.nrv_create_scene(ctypes.byref(d), ctypes.byref(h)) == nrv.NRV_ERR_ARG
    assert lib.nrv_keys_flip_sign(None, 4, None) == nrv.NRV_ERR_ARG
    w = nrv.nrv_loss_weights(1.0, -0.5, 0.0)
    assert lib.nrv_recon_loss(16, 16, 1, 4, 4, ctypes.byref(w), 16, None, None) == nrv.NRV_ERR_ARG
    d = nrv.nrv_scene_desc(0, None, None, 4, 3)      # empty scene is valid
    assert lib.nrv_create_scene(ctypes.byref(d), ctypes.byref(h)) == nrv.NRV_OK
    assert lib.nrv_rasterize(h, None, 1, None, None) == nrv.NRV_ERR_ARG
    assert lib.nrv_scene_refresh(h) == nrv.NRV_OK
    assert lib.nrv_scene_refresh(None) == nrv.NRV_ERR_ARG
    assert lib.nrv_destroy_scene(h) == nrv.NRV_OK
    assert lib.nrv_create_net(9, ctypes.byref(h)) == nrv.NRV_ERR_ARG
    assert lib.nrv_create_net(5, ctypes.byref(h)) == nrv.NRV_OK
    assert lib.nrv_shade(h, 32, 1, 8, 8, 0, 32, None) == nrv.NRV_ERR_STATE   # no params yet
    assert lib.nrv_net_backward(h, 32, 32, None) == nrv.NRV_ERR_STATE
    assert lib.nrv_net_save(h, b"/nonexistent/net.bin", None) == nrv.NRV_ERR_STATE
    assert lib.nrv_net_get_params(h, 32, None) == nrv.NRV_ERR_STATE
    assert lib.nrv_net_load(h, b"/nonexistent/net.bin", None) == nrv.NRV_ERR_ARG
    assert lib.nrv_destroy_net(h) == nrv.NRV_OK


def test_tune_cache_file_host_side(lib, tmp_path):
    """The tuned-choice cache is host-side: a malformed or missing file is refused, a valid one
    loads and saves again with its entries."""
    from paper_2407_19097_gb300 import nrv
    bad = tmp_path / "bad.txt"
    bad.write_text("render multi=0 log2n=20 = seven\n")
    with pytest.raises(nrv.NrvError, match="expected"):
        nrv.tune_load(bad)
    with pytest.raises(nrv.NrvError):
        nrv.tune_load(tmp_path / "missing.txt")
    good = tmp_path / "good.txt"
    good.write_text("# comment\nrender multi=1 log2n=27 = 4\nconv test key = 2230020\n")
    nrv.tune_load(good)
    out = tmp_path / "out.txt"
    nrv.tune_save(out)
    assert "render multi=1 log2n=27 = 4" in out.read_text()
    assert "conv test key = 2230020" in out.read_text()
    assert lib.nrv_tune_count() >= 1
