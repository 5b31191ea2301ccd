"""The biased estimator with the Balanced Termination Heuristic
(NIRC_EST_BIASED_BTH) against the oracle: every decision (camera hits,
sampled directions, termination tests, light samples, shadow rays) and
every cache-sample decision bit-exact through the signatures and counts;
the pixel, the cache level and the cache values within 1e-4 (FP32 SIMT) or
2e-2 (FP16 tensor cores), in both light modes, with the frequency and the
paper's network input."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import FP32_TOL, N, _compare_frames, _hash_cfg, _run_frame  # noqa: F401
from test_gpu_tc import TC_TOL, _row_errors

pytestmark = pytest.mark.gpu

EST = 1


def _params(cfg, seed):
    p = scenes.init_params(cfg, seed)
    rng = np.random.default_rng(seed)
    p[:cfg.n_mlp_params] += rng.normal(0, 0.02, cfg.n_mlp_params).astype(np.float32)
    if cfg.n_hash_params:
        p[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    return p


def _sh_cfg():
    return scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=12, log2_table=14, hidden_layers=4,
                            input_encoding=scenes.INPUT_SH)


def _run_bth(N, cfg, params, sc, W, H, Nc, D, frame, seed, light_mode, precision=0, cache_mode=0,
             cache_const=(0, 0, 0)):
    import torch
    cache = N.Cache(cfg)
    if params is not None:
        cache.set_params(params)
    if precision:
        N.nirc_set_precision(cache.h, precision)
    scd = N.scene_to_tensor(sc)
    P = W * H
    out = torch.empty((P, 4), device="cuda")
    lc = torch.empty((P, 3), device="cuda")
    lr = torch.empty((P, 3), device="cuda")
    sig = torch.empty((P, 2), device="cuda", dtype=torch.int64)
    cnt = torch.empty(P, device="cuda", dtype=torch.int32)
    row_n = torch.full((P, max(Nc, 1), 3), -1.0, device="cuda")
    desc = N.frame_desc(W, H, Nc, 0, D, frame, seed, sc.n_prims, cache_mode, cache_const, light_mode=light_mode,
                        estimator=EST)
    N.nirc_estimate_frame(cache.h, scd, desc, out, lc, lr, sig, cnt, row_n if Nc else None)
    N.nirc_sync(cache.h)
    torch.cuda.synchronize()
    cache.close()
    res = dict(pixel=out[:, :3].cpu().numpy(), alpha=out[:, 3].cpu().numpy(), lc=lc.cpu().numpy(),
               lr=lr.cpu().numpy(), sig=sig.cpu().numpy().view(np.uint64), count=cnt.cpu().numpy().view(np.uint32))
    if Nc:
        res["row_n"] = row_n[:, :Nc].cpu().numpy()
    return res


def _oracle(oracle, cfg, params, sc, W, H, Nc, D, frame, seed, light_mode, pixels=None, cache_mode=0,
            cache_const=(0, 0, 0)):
    fd = oracle.oframe(W, H, Nc, 0, D, frame, seed, cache_mode=cache_mode, cache_const=cache_const,
                       light_mode=light_mode, estimator=EST)
    return oracle.estimate(cfg, params, sc.blob(), fd, pixels=pixels, rows=Nc > 0)


@pytest.mark.parametrize("light_mode", [0, 1])
@pytest.mark.parametrize("Nc", [1, 4, 16])
def test_bth_fp32_matches_oracle(N, oracle, light_mode, Nc):
    """256 glossy primitives, 96x54, depth 5, FP32 SIMT cache."""
    cfg = _hash_cfg()
    params = _params(cfg, 3)
    sc = scenes.cornell_scene(96, 54, seed=2, n_prims=256, glossy=True, moving_emitter=True, frame=4)
    g = _run_bth(N, cfg, params, sc, 96, 54, Nc, 5, 4, 1, light_mode)
    o = _oracle(oracle, cfg, params, sc, 96, 54, Nc, 5, 4, 1, light_mode)
    _compare_frames(g, o)
    err = _row_errors(g, o)
    assert err.max() <= FP32_TOL, err.max()
    assert np.all(g["lr"] == 0)


@pytest.mark.parametrize("light_mode", [0, 1])
@pytest.mark.parametrize("which", ["freq", "sh"])
def test_bth_tc_fp16_matches_oracle(N, oracle, light_mode, which):
    cfg = _hash_cfg() if which == "freq" else _sh_cfg()
    params = _params(cfg, 4)
    sc = scenes.cornell_scene(96, 54, seed=2, n_prims=256, glossy=True, moving_emitter=True, frame=4)
    g = _run_bth(N, cfg, params, sc, 96, 54, 16, 5, 4, 1, light_mode, precision=N.NIRC_FP16_TC)
    o = _oracle(oracle, cfg, params, sc, 96, 54, 16, 5, 4, 1, light_mode)
    err = _row_errors(g, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(g, o, tol=TC_TOL)


@pytest.mark.parametrize("W,H,Nc,D", [(1, 1, 1, 1), (17, 9, 0, 3), (33, 7, 5, 2), (129, 3, 64, 8)])
def test_bth_edge_shapes(N, oracle, W, H, Nc, D):
    """Ragged sizes, N = 0 (no cache level: the truncated path alone),
    depth 1 (every path stops at its first vertex), N = 64."""
    cfg = scenes.config_small()
    params = _params(cfg, 6)
    sc = scenes.cornell_scene(W, H, seed=4)
    g = _run_bth(N, cfg, params, sc, W, H, Nc, D, 1, 3, 1)
    o = _oracle(oracle, cfg, params, sc, W, H, Nc, D, 1, 3, 1)
    _compare_frames(g, o)


def test_bth_furnace_exact_on_gpu(N, oracle):
    """Inside the emitting Lambertian sphere with the exact constant cache the
    GPU's biased estimate is L_e / (1 - rho) in every pixel (FP32)."""
    rho = float(np.float32(0.6))
    sc = scenes.furnace_scene(64, 64, rho=rho, emission=1.0)
    L = 1.0 / (1 - rho)
    g = _run_bth(N, scenes.config_small(), None, sc, 64, 64, 8, 6, 0, 1, 0, cache_mode=2, cache_const=(L, L, L))
    assert np.allclose(g["pixel"], L, rtol=5e-6), np.abs(g["pixel"] - L).max()


def test_bth_full_size_sampled_pixels(N, oracle):
    """The 1080p workload in the biased mode (light mode 1, N = 16, FP16),
    checked on sampled pixels."""
    cfg = scenes.config_1080p()
    params = _params(cfg, 1)
    W, H = 1920, 1080
    sc = scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=11)
    g = _run_bth(N, cfg, params, sc, W, H, 16, 5, 11, 1, 1, precision=N.NIRC_FP16_TC)
    rng = np.random.default_rng(3)
    pix = np.unique(np.concatenate([rng.integers(0, W * H, 300), [0, W * H - 1]])).astype(np.uint32)
    o = _oracle(oracle, cfg, params, sc, W, H, 16, 5, 11, 1, 1, pixels=pix)
    sub = {k: v[pix] for k, v in g.items()}
    err = _row_errors(sub, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(sub, o, tol=TC_TOL)


def test_bth_requires_no_residual_samples(N):
    import torch
    cfg = scenes.config_small()
    cache = N.Cache(cfg)
    sc = scenes.cornell_scene(8, 8, seed=1)
    out = torch.empty((64, 4), device="cuda")
    with pytest.raises(N.NircError) as ei:
        N.nirc_estimate_frame(cache.h, N.scene_to_tensor(sc), N.frame_desc(8, 8, 4, 1, 3, 0, 1, sc.n_prims,
                                                                           estimator=EST), out)
    assert ei.value.status == N.NIRC_ERR_INVALID
    cache.close()
