"""Pins for the oracle's G-buffer packing and number-format conversions: hand-computed values
and the format definitions as implemented by torch's own casts (library routines)."""
import numpy as np
import torch

import nrv_inputs as I
import oracle


def _f2u(x):
    return np.array([x], np.float32).view(np.uint32)[0]


def test_pack_hand_values():
    H, W, Hn, Wn = 2, 3, 4, 8
    depth = np.zeros((H, W), np.uint32)
    mask = np.zeros((H, W), np.uint8)
    g = np.zeros((3, H, W), np.uint32)
    depth[0, 1] = _f2u(2.5)
    mask[0, 1] = 1
    g[0, 0, 1] = _f2u(3.0)
    g[1, 0, 1] = 1000
    g[2, 0, 1] = 0x00FF8040
    # a covered pixel whose words are zero, and an uncovered one holding garbage words
    mask[1, 2] = 1
    depth[1, 2] = _f2u(1.0)
    g[0, 1, 0] = _f2u(99.0)
    chans = [I.Channel(0, I.FMT_F32, 0, 2.0, 1.0), I.Channel(1, I.FMT_U32, 0, 0.5, -2.0),
             I.Channel(2, I.FMT_U8X4, 2, 0.5, 0.0), I.Channel(2, I.FMT_U8X4, 1, 1.0, 0.25)]
    out = oracle.pack(depth, mask, g, chans, 0.25, -0.125, Hn, Wn, 8, 0)
    assert out.shape == (Hn, Wn, 8) and out.dtype == np.float32
    np.testing.assert_array_equal(out[0, 1], [7.0, 498.0, 127.5, 128.25, 0.5, 1.0, 0.0, 0.0])
    np.testing.assert_array_equal(out[1, 2], [1.0, -2.0, 0.0, 0.25, 0.125, 1.0, 0.0, 0.0])
    rest = np.ones((Hn, Wn), bool)
    rest[0, 1] = rest[1, 2] = False
    assert np.all(out[rest] == 0.0)
    ob = oracle.pack(depth, mask, g, chans, 0.25, -0.125, Hn, Wn, 8, 1)
    ref = torch.from_numpy(out).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ob, ref)
    assert oracle.bf16_value(ob)[0, 1, 3] == 128.0                # 128.25 rounds to even
    o8 = oracle.pack(depth, mask, g, chans, 0.25, -0.125, Hn, Wn, 16, 2, 0.5)
    # 249 lies between the e4m3 neighbours 240 and 256 (spacing 16 in [128, 256)): 256
    np.testing.assert_array_equal(oracle.e4m3_value(o8[0, 1, :6]), [3.5, 256.0, 64.0, 64.0, 0.25, 0.5])


def test_bf16_matches_torch_round_to_nearest_even():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(100_000).astype(np.float32) * np.float32(1e3)
    ties = (rng.integers(0, 2**31, 2000, dtype=np.uint32) & np.uint32(0xFFFF0000)) | np.uint32(0x8000)
    x = np.concatenate([x, ties.view(np.float32), np.array([0.0, -0.0, 1e-40, -3e38, 3.4e38,
                                                             np.inf, -np.inf], np.float32)])
    x = x[np.isfinite(x) | np.isinf(x)]
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.bf16_bits(x), ref)


def test_e4m3_decode_matches_torch_for_all_codes():
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    mine = oracle.e4m3_value(codes)
    nan = np.isnan(ref)
    assert np.array_equal(nan, np.isnan(mine)) and nan.sum() == 2
    assert np.array_equal(ref[~nan], mine[~nan])


def test_e4m3_encode_matches_torch_in_range_and_saturates():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-448, 448, 50_000), rng.standard_normal(50_000),
                        rng.standard_normal(20_000) * 1e-2]).astype(np.float32)
    codes = np.arange(256, dtype=np.uint8)
    vals = oracle.e4m3_value(codes)
    fin = np.isfinite(vals)
    # exact midpoints between neighbouring codes exercise ties-to-even
    v = np.sort(np.unique(vals[fin]))
    mids = ((v[1:] + v[:-1]) / 2).astype(np.float32)
    x = np.concatenate([x, mids, vals[fin].astype(np.float32)])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(oracle.e4m3_bits(x), ref)
    # round trip of every finite code
    assert np.array_equal(oracle.e4m3_bits(vals[fin].astype(np.float32)), codes[fin])
    sat = oracle.e4m3_bits(np.array([449.0, 1e6, np.inf, -500.0, -np.inf], np.float32))
    assert sat.tolist() == [0x7E, 0x7E, 0x7E, 0xFE, 0xFE]
    assert oracle.e4m3_bits(np.array([np.nan], np.float32))[0] == 0x7F
