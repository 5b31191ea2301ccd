"""Environment light and the Neural Visibility Cache (light mode 2,
NIRC_OUT_VISIBILITY) against the oracle: sigmoid queries and training
gradients within 1e-4 (FP32), training records and visibility targets
bit-exact, and the direct-environment frame with a visibility cache (FP32
SIMT 1e-4, FP16 tensor cores 2e-2) and with a radiance cache (the generic
NIRC on the same task), decisions bit-exact."""
import dataclasses

import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import FP32_TOL, N, _compare_frames, _near_kink, _run_frame, rel_err  # noqa: F401
from test_gpu_tc import TC_TOL, _row_errors

pytestmark = pytest.mark.gpu


def _cfg(output=scenes.OUT_VISIBILITY, sh=False):
    return scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=12 if sh else 16, log2_table=14,
                            hidden_layers=4, input_encoding=scenes.INPUT_SH if sh else scenes.INPUT_FREQ,
                            output=output, lr=1e-2)


def _params(cfg, seed):
    p = scenes.init_params(cfg, seed)
    rng = np.random.default_rng(seed)
    p[:cfg.n_mlp_params] += rng.normal(0, 0.05, cfg.n_mlp_params).astype(np.float32)
    p[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    return p


@pytest.mark.parametrize("n", [1, 129, 4000])
def test_visibility_query_matches_oracle(N, oracle, n):
    import torch
    cfg = _cfg()
    params = _params(cfg, n)
    recs, dirs = scenes.random_query_rows(n, seed=n + 3)
    cache = N.Cache(cfg)
    cache.set_params(params)
    out = torch.empty((n, 3), device="cuda")
    N.nirc_query(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), out)
    got = out.cpu().numpy()
    cache.close()
    ref = oracle.query(cfg, params, recs, dirs)
    assert np.all((ref > 0) & (ref < 1))
    assert (np.abs(got - ref) / ref).max() <= FP32_TOL


@pytest.mark.parametrize("visibility", [1, 0])
def test_env_training_records_match_oracle(N, oracle, visibility):
    import torch
    W, H, T = 96, 64, 4099
    sc = scenes.env_scene(W, H, seed=2, n_prims=64, env_size=16)
    cache = N.Cache(_cfg(output=scenes.OUT_VISIBILITY if visibility else scenes.OUT_RADIANCE))
    recs = torch.empty((T, 16), device="cuda")
    dirs = torch.empty((T, 3), device="cuda")
    tg = torch.empty((T, 3), device="cuda")
    N.nirc_gen_train(cache.h, N.scene_to_tensor(sc), sc.n_prims, W, H, T, 3, 1, 4, recs, dirs, tg, light_mode=2)
    cache.close()
    orec, odir, otg, _ = oracle.gen_train(sc.blob(), W, H, T, 3, 1, 4, scenes.RECORD_DTYPE, light_mode=2,
                                          visibility=visibility)
    assert np.array_equal(N.records_from_tensor(recs).view(np.uint8), orec.view(np.uint8))
    assert np.array_equal(dirs.cpu().numpy().view(np.uint32), odir.view(np.uint32))
    assert np.array_equal(tg.cpu().numpy().astype(np.float64), otg)  # texel values or 0 / 1: exact


def test_visibility_train_step_matches_oracle(N, oracle):
    import torch
    cfg = _cfg()
    params = _params(cfg, 7)
    n = 3000
    recs, dirs, _ = scenes.training_batch(n, seed=23)
    tg = (np.random.default_rng(24).uniform(size=(n, 1)) < 0.6).astype(np.float32).repeat(3, axis=1)
    recs["flags"][::11] = 0
    recs["flags"][_near_kink(oracle, cfg, params, recs, dirs)] = 0
    cache = N.Cache(cfg)
    cache.set_params(params)
    loss = torch.zeros(1, device="cuda")
    N.nirc_train_step(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), torch.from_numpy(tg).cuda(),
                      loss)
    torch.cuda.synchronize()
    g_gpu = cache.get_grads().numpy().astype(np.float64)
    cache.close()
    loss_or, g_or = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    assert abs(loss.item() - loss_or) <= 1e-5 * abs(loss_or)
    for lo, hi in ((0, cfg.n_mlp_params), (cfg.n_mlp_params, cfg.n_params)):
        scale = np.abs(g_or[lo:hi]).max()
        assert np.abs(g_gpu[lo:hi] - g_or[lo:hi]).max() <= FP32_TOL * scale


@pytest.mark.parametrize("output", [scenes.OUT_VISIBILITY, scenes.OUT_RADIANCE])
def test_env_frame_fp32_matches_oracle(N, oracle, output):
    """Direct environment light at the shading point, N = 8 cache rows and
    M = 2 visibility rays, 64 primitives under the procedural sky."""
    cfg = _cfg(output)
    params = _params(cfg, 3)
    sc = scenes.env_scene(80, 60, seed=1, n_prims=64, env_size=32)
    g = _run_frame(N, cfg, params, sc, 80, 60, 8, 2, 1, 2, 1, rows=True, light_mode=2)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(80, 60, 8, 2, 1, 2, 1, light_mode=2), rows=True)
    _compare_frames(g, o)
    err = _row_errors(g, o)
    assert err.max() <= FP32_TOL, err.max()


@pytest.mark.parametrize("sh", [False, True])
def test_env_frame_tc_fp16_matches_oracle(N, oracle, sh):
    cfg = _cfg(sh=sh)
    params = _params(cfg, 4)
    sc = scenes.env_scene(80, 60, seed=1, n_prims=64, env_size=32)
    g = _run_frame(N, cfg, params, sc, 80, 60, 16, 1, 1, 2, 1, rows=True, light_mode=2, precision=N.NIRC_FP16_TC)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(80, 60, 16, 1, 1, 2, 1, light_mode=2), rows=True)
    err = _row_errors(g, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(g, o, tol=TC_TOL)


def test_env_frame_full_size_sampled_pixels(N, oracle):
    """1080p under the sky (256 primitives, 64^2 cube faces), N = 16, M = 1,
    FP16 visibility cache, sampled pixels."""
    cfg = dataclasses.replace(scenes.config_1080p(), output=scenes.OUT_VISIBILITY)
    params = _params(cfg, 1)
    W, H = 1920, 1080
    sc = scenes.env_scene(W, H, seed=1, n_prims=256, env_size=64)
    g = _run_frame(N, cfg, params, sc, W, H, 16, 1, 1, 5, 1, rows=True, light_mode=2, precision=N.NIRC_FP16_TC)
    rng = np.random.default_rng(6)
    pix = np.unique(np.concatenate([rng.integers(0, W * H, 300), [0, W * H - 1]])).astype(np.uint32)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, 16, 1, 1, 5, 1, light_mode=2), pixels=pix,
                        rows=True)
    sub = {k: v[pix] for k, v in g.items()}
    err = _row_errors(sub, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(sub, o, tol=TC_TOL)
