"""Parity of the tensor-core (tcgen05, FP16 or split BF16 operands, FP32
accumulation) cache integral with the CPU oracle.

Sampling, hits and Russian roulette are shared with the FP32 path and stay
bit-exact (signatures, counts); every cache output n is within 2e-2
relative of the oracle's; the two levels within 2e-2 of their own
magnitude; the pixel within 2e-2 of the largest of |pixel|, |L_c|, |L_r|;
and the frame MRSE against an oracle-rendered reference within 1% of the
oracle image's MRSE.
"""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import N, _compare_frames, _hash_cfg, _run_frame  # noqa: F401

pytestmark = pytest.mark.gpu

TC_TOL = 2e-2
PRECISIONS = {"fp16": 1, "bf16": 2}
# BF16 operands are split into hi + lo halves (each product taken as
# hi*hi + lo*hi + hi*lo, ~16 significant bits), so BF16 meets the same 2e-2
# bound per cache output as FP16, at the maximum.


def _check_rows(err, prec):
    assert err.max() <= TC_TOL, (prec, float(err.max()), float(np.percentile(err, 99)))


def _row_errors(g, o):
    valid = o["row_n"] > 0
    assert np.array_equal(valid, g["row_n"] > 0), "valid rows differ"
    return np.abs(g["row_n"][valid] - o["row_n"][valid]) / o["row_n"][valid]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_small_workload(N, oracle, prec):
    """64x64 Cornell box, frequency encoding, N = 8, M = 1 (S = 9)."""
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 1)
    sc = scenes.cornell_scene(64, 64, seed=1)
    g = _run_frame(N, cfg, params, sc, 64, 64, 8, 1, 4, 2, 1, precision=PRECISIONS[prec], rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(64, 64, 8, 1, 4, 2, 1), rows=True)
    err = _row_errors(g, o)
    _check_rows(err, prec)
    _compare_frames(g, o, tol=TC_TOL)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_hashgrid_glossy(N, oracle, prec):
    """256 glossy primitives, hash-grid cache (16 levels), N = 16, M = 1 (S = 17), 96x54."""
    cfg = _hash_cfg()
    params = scenes.init_params(cfg, 2)
    params[cfg.n_mlp_params:] = np.random.default_rng(0).uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    sc = scenes.cornell_scene(96, 54, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=7)
    g = _run_frame(N, cfg, params, sc, 96, 54, 16, 1, 5, 7, 1, precision=PRECISIONS[prec], rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(96, 54, 16, 1, 5, 7, 1), rows=True)
    err = _row_errors(g, o)
    _check_rows(err, prec)
    _compare_frames(g, o, tol=TC_TOL)


@pytest.mark.parametrize("W,H,Nc,M", [(1, 1, 3, 1), (17, 9, 4, 1), (31, 5, 64, 4), (13, 11, 0, 4), (40, 40, 32, 1)])
def test_tc_edge_shapes(N, oracle, W, H, Nc, M):
    """S = 4 (the smallest the tensor-core path takes), ragged pixel blocks,
    N = 64 with M = 4 (S = 68: one pixel spans tiles), N = 0."""
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 6)
    sc = scenes.cornell_scene(W, H, seed=4)
    g = _run_frame(N, cfg, params, sc, W, H, Nc, M, 4, 1, 3, precision=1, rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, Nc, M, 4, 1, 3), rows=True)
    err = _row_errors(g, o)
    if err.size:
        assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(g, o, tol=TC_TOL)


def test_tc_full_size_sampled_pixels(N, oracle):
    """The launch the benchmark times (1920x1080, 2^19-entry hash grid, FP16),
    checked on sampled pixels and all of their rows."""
    cfg = scenes.config_1080p()
    params = scenes.init_params(cfg, 1)
    rng = np.random.default_rng(1)
    params[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    W, H = 1920, 1080
    sc = scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=11)
    g = _run_frame(N, cfg, params, sc, W, H, 16, 1, 5, 11, 1, precision=1, rows=True)
    # with 152 SMs x 5 warpgroups, whole 128-pixel blocks cover pixels < 21 x 760 x 128 and the
    # remaining 30,720 are split into 760 blocks of 40-41 pixels: probe both sides of those seams
    tail0 = 21 * 760 * 128
    seams = [tail0 - 1, tail0, tail0 + 40, tail0 + 41, tail0 + 30720 * 379 // 760, W * H - 2]
    pix = np.unique(np.concatenate([rng.integers(0, W * H, 300), [0, 127, 128, W * H - 1], seams])).astype(np.uint32)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, 16, 1, 5, 11, 1), pixels=pix, rows=True)
    sub = {k: v[pix] for k, v in g.items()}
    err = _row_errors(sub, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(sub, o, tol=TC_TOL)


def test_tc_mrse_matches_oracle(N, oracle):
    """Frame MRSE of the FP16 tensor-core image against a path-traced
    reference (rendered by the oracle) is within 1% of the oracle image's."""
    import torch
    cfg = _hash_cfg()
    params = scenes.init_params(cfg, 3)
    params[cfg.n_mlp_params:] = np.random.default_rng(5).uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    W, H = 80, 45
    sc = scenes.cornell_scene(W, H, seed=2, n_prims=256, glossy=True, moving_emitter=True, frame=3)
    ref = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(W, H, 0, 64, 16, 1000, 7, cache_mode=1))["pixel"]
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, 16, 1, 5, 3, 1))
    g = _run_frame(N, cfg, params, sc, W, H, 16, 1, 5, 3, 1, precision=1)
    img = torch.zeros((W * H, 4), device="cuda")
    img[:, :3] = torch.from_numpy(g["pixel"]).cuda()
    refd = torch.zeros((W * H, 4), device="cuda")
    refd[:, :3] = torch.from_numpy(ref.astype(np.float32)).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    N.nirc_frame_mrse(img, refd, out)
    m_gpu = out.item()
    m_or = oracle.mrse(o["pixel"], ref.astype(np.float32).astype(np.float64))
    assert abs(m_gpu - m_or) <= 0.01 * m_or, (m_gpu, m_or)


# FP8 E4M3 hidden layers (3 mantissa bits, per-layer scales): the decisions
# stay bit-exact; the cache values carry E4M3 rounding through the hidden
# layers, so their error is bounded loosely here and reported in the
# precision sweep.
FP8_P50, FP8_P99 = 0.05, 0.3


@pytest.mark.parametrize("which", ["small", "hash"])
def test_tc_fp8(N, oracle, which):
    import torch
    if which == "small":
        cfg = scenes.config_small()
        params = scenes.init_params(cfg, 1)
        sc = scenes.cornell_scene(64, 64, seed=1)
        W, H, Nc, D, fr = 64, 64, 8, 4, 2
    else:
        cfg = _hash_cfg()
        params = scenes.init_params(cfg, 2)
        params[cfg.n_mlp_params:] = np.random.default_rng(0).uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
        sc = scenes.cornell_scene(96, 54, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=7)
        W, H, Nc, D, fr = 96, 54, 16, 5, 7
    g = _run_frame(N, cfg, params, sc, W, H, Nc, 1, D, fr, 1, precision=N.NIRC_FP8_E4M3_TC, rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, Nc, 1, D, fr, 1), rows=True)
    assert np.array_equal(g["sig"], o["sig"])
    assert np.array_equal(g["count"], o["count"])
    err = _row_errors(g, o)
    print(which, "fp8 row error p50 %.4f p99 %.4f max %.4f" % (np.percentile(err, 50), np.percentile(err, 99),
                                                                err.max()))
    assert np.percentile(err, 50) <= FP8_P50 and np.percentile(err, 99) <= FP8_P99


def test_tc_fp8_delayed_scaling_is_deterministic(N):
    """The first FP8 frame calibrates the activation scales with one FP16
    pass; each later frame scales with the amax the previous frame recorded.
    Two caches taken through the same frames give identical images, and
    frames after the first stay within FP8 rounding of each other."""
    import torch
    cfg = _hash_cfg()
    params = scenes.init_params(cfg, 5)
    params[cfg.n_mlp_params:] = np.random.default_rng(1).uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    sc = scenes.cornell_scene(64, 48, seed=3, n_prims=64, glossy=True)
    scd = N.scene_to_tensor(sc)
    runs = []
    for _ in range(2):
        cache = N.Cache(cfg)
        cache.set_params(params)
        N.nirc_set_precision(cache.h, N.NIRC_FP8_E4M3_TC)
        imgs, lcs = [], []
        for f in range(3):
            out = torch.empty((64 * 48, 4), device="cuda")
            lc = torch.empty((64 * 48, 3), device="cuda")
            N.nirc_estimate_frame(cache.h, scd, N.frame_desc(64, 48, 8, 1, 4, 1, 1, sc.n_prims), out, lc=lc)
            imgs.append(out.cpu().numpy())
            lcs.append(lc.cpu().numpy())
        N.nirc_sync(cache.h)
        runs.append((imgs, lcs))
        cache.close()
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    lc1, lc2 = runs[0][1][1], runs[0][1][2]
    scale = max(np.abs(lc1).max(), 1e-30)
    assert np.abs(lc1 - lc2).max() <= 0.1 * scale


@pytest.mark.parametrize("hidden", [1, 2, 6, 8])
def test_tc_hidden_layer_counts(N, oracle, hidden):
    """Other depths: one hidden layer (only the output bias through the MMA),
    two, and six / eight (two tiles of bias slots; the larger weight image
    leaves room for four warpgroups per CTA)."""
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=16, log2_table=12, hidden_layers=hidden)
    params = scenes.init_params(cfg, 9)
    rng = np.random.default_rng(9)
    params[:cfg.n_mlp_params] += rng.normal(0, 0.02, cfg.n_mlp_params).astype(np.float32)
    params[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    sc = scenes.cornell_scene(48, 40, seed=5, n_prims=64, glossy=True)
    g = _run_frame(N, cfg, params, sc, 48, 40, 8, 1, 4, 1, 2, precision=1, rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(48, 40, 8, 1, 4, 1, 2), rows=True)
    err = _row_errors(g, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(g, o, tol=TC_TOL)
