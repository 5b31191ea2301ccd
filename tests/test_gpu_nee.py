"""Light mode 1 (eq. Lsplit: the cache carries L_ind, direct light by
next-event estimation with MIS) on the GPU against the oracle: decisions
(camera hits, light choices, shadow rays, residual and continuation
directions, Russian roulette) bit-exact through the signatures and counts,
the FP32 path within 1e-4 and the FP16 tensor-core path within 2e-2, and
the training pass's records and directions bit for bit."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import FP32_TOL, N, _compare_frames, _hash_cfg, _run_frame, rel_err  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["small", "glossy256"])
@pytest.mark.parametrize("precision", [0, 1])
def test_nee_frame_matches_oracle(N, oracle, which, precision):
    if which == "small":
        cfg = scenes.config_small()
        params = scenes.init_params(cfg, 1)
        sc = scenes.cornell_scene(48, 40, seed=2)
        W, H, Nc, M, D = 48, 40, 8, 2, 4
    else:
        cfg = _hash_cfg()
        params = scenes.init_params(cfg, 2)
        params[cfg.n_mlp_params:] = np.random.default_rng(0).uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
        sc = scenes.cornell_scene(96, 54, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=9)
        W, H, Nc, M, D = 96, 54, 16, 1, 5
    g = _run_frame(N, cfg, params, sc, W, H, Nc, M, D, 9, 3, precision=precision, light_mode=1)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, Nc, M, D, 9, 3, light_mode=1))
    _compare_frames(g, o, tol=FP32_TOL if precision == 0 else 2e-2)


def test_nee_zero_cache_and_floor_scene(N, oracle):
    """Zero cache (plain NEE path tracing) on the floor-and-light scene and
    the Cornell box, M = 0 (light sampling only) and M = 3."""
    cfg = scenes.config_small()
    for sc, M in ((scenes.floor_light_scene(32, 32), 0), (scenes.floor_light_scene(32, 32, glossy=True), 3),
                  (scenes.cornell_scene(32, 32, seed=5, n_prims=40, glossy=True), 3)):
        g = _run_frame(N, cfg, None, sc, 32, 32, 4, M, 4, 1, 7, cache_mode=1, light_mode=1)
        o = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(32, 32, 4, M, 4, 1, 7, cache_mode=1, light_mode=1))
        _compare_frames(g, o)


@pytest.mark.parametrize("n_prims", [8, 256])
def test_nee_training_records_match_oracle(N, oracle, n_prims):
    import torch
    W, H, D, T = 120, 68, 5, 4099
    sc = scenes.cornell_scene(W, H, seed=1, n_prims=n_prims, glossy=n_prims > 8, moving_emitter=True, frame=4)
    cache = N.Cache(scenes.config_small())
    recs = torch.empty((T, 16), device="cuda")
    dirs = torch.empty((T, 3), device="cuda")
    tg = torch.empty((T, 3), device="cuda")
    N.nirc_gen_train(cache.h, N.scene_to_tensor(sc), sc.n_prims, W, H, T, 4, 1, D, recs, dirs, tg, light_mode=1)
    orec, odir, otg, _ = oracle.gen_train(sc.blob(), W, H, T, 4, 1, D, scenes.RECORD_DTYPE, light_mode=1)
    assert np.array_equal(N.records_from_tensor(recs).view(np.uint8), orec.view(np.uint8))
    assert np.array_equal(dirs.cpu().numpy().view(np.uint32), odir.view(np.uint32))
    err = rel_err(tg.cpu().numpy(), otg)
    assert err.max() <= FP32_TOL, err.max()
    assert (otg.max(1) > 0).mean() > 0.1  # far more non-zero targets than pure BSDF paths (~0.04 %)
    cache.close()
