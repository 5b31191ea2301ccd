"""Parity of the paper's network input (NIRC_INPUT_SH: 12-level hash grid,
25 spherical harmonics of the direction, albedo + one-blob normal and
roughness) on every CUDA path with the CPU oracle: bare queries and the
frame estimate on the FP32 SIMT kernels (1e-4), the tensor-core kernels in
FP16 / BF16 (2e-2 per cache output, decisions bit-exact) at every S = N + M
including S < 4, the full-size 1080p launch on sampled pixels, FP8 hidden
layers, and the training gradient."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import FP32_TOL, N, _compare_frames, _near_kink, _run_frame  # noqa: F401
from test_gpu_tc import FP8_P50, FP8_P99, TC_TOL, _check_rows, _row_errors

pytestmark = pytest.mark.gpu


def _cfg():
    return scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=12, log2_table=14, hidden_layers=4,
                            input_encoding=scenes.INPUT_SH, lr=1e-2)


def _params(cfg, seed):
    p = scenes.init_params(cfg, seed)
    rng = np.random.default_rng(seed)
    p[:cfg.n_mlp_params] += rng.normal(0, 0.02, cfg.n_mlp_params).astype(np.float32)
    p[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    return p


@pytest.mark.parametrize("n", [1, 129, 5000])
def test_query_paper_input(N, oracle, n):
    import torch
    cfg = _cfg()
    params = _params(cfg, n)
    recs, dirs = scenes.random_query_rows(n, seed=n + 1)
    cache = N.Cache(cfg)
    cache.set_params(params)
    out = torch.empty((n, 3), device="cuda")
    N.nirc_query(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), out)
    got = out.cpu().numpy()
    cache.close()
    ref = oracle.query(cfg, params, recs, dirs)
    err = np.abs(got - ref) / np.abs(ref)
    assert err.max() <= FP32_TOL, err.max()


def _glossy(W=96, H=54, frame=7):
    return scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=frame)


def test_frame_paper_input_fp32(N, oracle):
    """256 glossy primitives, 96x54, N = 16, M = 1, depth 5, FP32 SIMT."""
    cfg = _cfg()
    params = _params(cfg, 2)
    sc = _glossy()
    g = _run_frame(N, cfg, params, sc, 96, 54, 16, 1, 5, 7, 1, rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(96, 54, 16, 1, 5, 7, 1), rows=True)
    _compare_frames(g, o)
    err = _row_errors(g, o)
    assert err.max() <= FP32_TOL, err.max()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_paper_input(N, oracle, prec):
    cfg = _cfg()
    params = _params(cfg, 2)
    sc = _glossy()
    code = N.NIRC_FP16_TC if prec == "fp16" else N.NIRC_BF16_TC
    g = _run_frame(N, cfg, params, sc, 96, 54, 16, 1, 5, 7, 1, precision=code, rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(96, 54, 16, 1, 5, 7, 1), rows=True)
    _check_rows(_row_errors(g, o), prec)
    _compare_frames(g, o, tol=TC_TOL)


@pytest.mark.parametrize("W,H,Nc,M", [(1, 1, 0, 1), (5, 3, 1, 1), (17, 9, 2, 1), (31, 5, 4, 1), (13, 11, 6, 1),
                                      (40, 40, 64, 4), (33, 7, 0, 4), (129, 3, 3, 0)])
def test_tc_paper_input_any_rows_per_pixel(N, oracle, W, H, Nc, M):
    """S = 1, 2, 3, 5, 7, 68, 4 and 3 (N = 0 and M = 0 included), ragged
    pixel blocks: the paper's input needs no one-hot window, so the
    tensor-core kernel takes every S."""
    cfg = _cfg()
    params = _params(cfg, 6)
    sc = scenes.cornell_scene(W, H, seed=4, n_prims=64, glossy=True)
    g = _run_frame(N, cfg, params, sc, W, H, Nc, M, 4, 1, 3, precision=N.NIRC_FP16_TC, rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, Nc, M, 4, 1, 3), rows=True)
    err = _row_errors(g, o)
    if err.size:
        assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(g, o, tol=TC_TOL)


def test_tc_paper_input_full_size_sampled_pixels(N, oracle):
    """The 1080p launch with the paper's input (2^19-entry 12-level grid,
    FP16), checked on sampled pixels and all of their rows."""
    cfg = scenes.config_paper_1080p()
    params = _params(cfg, 1)
    W, H = 1920, 1080
    sc = scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=11)
    g = _run_frame(N, cfg, params, sc, W, H, 16, 1, 5, 11, 1, precision=N.NIRC_FP16_TC, rows=True)
    rng = np.random.default_rng(2)
    pix = np.unique(np.concatenate([rng.integers(0, W * H, 300), [0, 127, 128, W * H - 1]])).astype(np.uint32)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, 16, 1, 5, 11, 1), pixels=pix, rows=True)
    sub = {k: v[pix] for k, v in g.items()}
    err = _row_errors(sub, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(sub, o, tol=TC_TOL)


def test_tc_paper_input_fp8(N, oracle):
    cfg = _cfg()
    params = _params(cfg, 2)
    sc = _glossy()
    g = _run_frame(N, cfg, params, sc, 96, 54, 16, 1, 5, 7, 1, precision=N.NIRC_FP8_E4M3_TC, rows=True)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(96, 54, 16, 1, 5, 7, 1), rows=True)
    assert np.array_equal(g["sig"], o["sig"])
    assert np.array_equal(g["count"], o["count"])
    err = _row_errors(g, o)
    print("paper input fp8 row error p50 %.4f p99 %.4f max %.4f" % (np.percentile(err, 50),
                                                                   np.percentile(err, 99), err.max()))
    assert np.percentile(err, 50) <= FP8_P50 and np.percentile(err, 99) <= FP8_P99


def test_train_step_paper_input(N, oracle):
    """Loss, every gradient and one Adam step of the FP32 training kernels
    against the oracle's FP64 gradient."""
    import torch
    cfg = _cfg()
    params = _params(cfg, 4)
    n = 3000
    recs, dirs, tg = scenes.training_batch(n, seed=22)
    recs["flags"][::13] = 0
    recs["flags"][_near_kink(oracle, cfg, params, recs, dirs)] = 0
    cache = N.Cache(cfg)
    cache.set_params(params)
    loss = torch.zeros(1, device="cuda")
    N.nirc_train_step(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(),
                      torch.from_numpy(tg).cuda(), loss)
    torch.cuda.synchronize()
    g_gpu = cache.get_grads().numpy().astype(np.float64)
    cache.close()
    loss_or, g_or = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    assert abs(loss.item() - loss_or) <= 1e-5 * abs(loss_or)
    for lo, hi in ((0, cfg.n_mlp_params), (cfg.n_mlp_params, cfg.n_params)):
        scale = np.abs(g_or[lo:hi]).max()
        assert np.abs(g_gpu[lo:hi] - g_or[lo:hi]).max() <= FP32_TOL * scale
    # the input-layer columns of the direction (SH) and of phi get gradient
    W0 = g_gpu[:64 * 64].reshape(64, 64)
    assert np.abs(W0[:, 24:49]).max() > 0 and np.abs(W0[:, 49:64]).max() > 0
