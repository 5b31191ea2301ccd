"""The multi-vertex unbiased estimator (NIRC_EST_MULTI_VERTEX: the two
levels at the shading point and at the second and third vertex of every
residual path, N_c^1 / N_c^2 / N_c^3 cache samples) against the oracle:
decisions bit-exact, FP32 within 1e-4, FP16 tensor cores within 2e-2, in
both light modes and with both network inputs; the exact furnace on the
GPU."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import FP32_TOL, N, _compare_frames, _hash_cfg  # noqa: F401
from test_gpu_tc import TC_TOL, _row_errors

pytestmark = pytest.mark.gpu

EST = 2


def _params(cfg, seed):
    p = scenes.init_params(cfg, seed)
    rng = np.random.default_rng(seed)
    p[:cfg.n_mlp_params] += rng.normal(0, 0.02, cfg.n_mlp_params).astype(np.float32)
    if cfg.n_hash_params:
        p[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    return p


def _run(N, cfg, params, sc, W, H, N1, M, D, N2, N3, frame, seed, light_mode=0, precision=0, cache_mode=0,
         cache_const=(0, 0, 0)):
    import torch
    cache = N.Cache(cfg)
    if params is not None:
        cache.set_params(params)
    if precision:
        N.nirc_set_precision(cache.h, precision)
    P = W * H
    out = torch.empty((P, 4), device="cuda")
    lc = torch.empty((P, 3), device="cuda")
    lr = torch.empty((P, 3), device="cuda")
    sig = torch.empty((P, 2), device="cuda", dtype=torch.int64)
    cnt = torch.empty(P, device="cuda", dtype=torch.int32)
    row_n = torch.full((P, N1 + M, 3), -1.0, device="cuda")
    desc = N.frame_desc(W, H, N1, M, D, frame, seed, sc.n_prims, cache_mode, cache_const, light_mode=light_mode,
                        estimator=EST, n_cache2=N2, n_cache3=N3)
    N.nirc_estimate_frame(cache.h, N.scene_to_tensor(sc), desc, out, lc, lr, sig, cnt, row_n)
    N.nirc_sync(cache.h)
    torch.cuda.synchronize()
    cache.close()
    return dict(pixel=out[:, :3].cpu().numpy(), alpha=out[:, 3].cpu().numpy(), lc=lc.cpu().numpy(),
                lr=lr.cpu().numpy(), sig=sig.cpu().numpy().view(np.uint64), count=cnt.cpu().numpy().view(np.uint32),
                row_n=row_n.cpu().numpy())


def _oracle(oracle, cfg, params, sc, W, H, N1, M, D, N2, N3, frame, seed, light_mode=0, pixels=None, cache_mode=0,
            cache_const=(0, 0, 0)):
    fd = oracle.oframe(W, H, N1, M, D, frame, seed, cache_mode=cache_mode, cache_const=cache_const,
                       light_mode=light_mode, estimator=EST, n_cache2=N2, n_cache3=N3)
    return oracle.estimate(cfg, params, sc.blob(), fd, pixels=pixels, rows=True)


@pytest.mark.parametrize("light_mode", [0, 1])
@pytest.mark.parametrize("N1,M,N2,N3", [(16, 1, 5, 4), (4, 2, 3, 0), (0, 1, 6, 6), (8, 3, 0, 2)])
def test_multivertex_fp32_matches_oracle(N, oracle, light_mode, N1, M, N2, N3):
    cfg = _hash_cfg()
    params = _params(cfg, 5)
    sc = scenes.cornell_scene(64, 48, seed=3, n_prims=256, glossy=True, moving_emitter=True, frame=2)
    g = _run(N, cfg, params, sc, 64, 48, N1, M, 5, N2, N3, 2, 1, light_mode)
    o = _oracle(oracle, cfg, params, sc, 64, 48, N1, M, 5, N2, N3, 2, 1, light_mode)
    _compare_frames(g, o)
    err = _row_errors(g, o)
    if err.size:
        assert err.max() <= FP32_TOL, err.max()


@pytest.mark.parametrize("light_mode", [0, 1])
@pytest.mark.parametrize("which", ["freq", "sh"])
def test_multivertex_tc_fp16_matches_oracle(N, oracle, light_mode, which):
    """Vertex passes of S = 6 and 3 rows (the frequency input takes the FP32
    kernel below S = 4, the paper's input stays on the tensor cores)."""
    cfg = _hash_cfg() if which == "freq" else scenes.NetConfig(
        pos_encoding=scenes.POS_HASHGRID, hash_levels=12, log2_table=14, hidden_layers=4,
        input_encoding=scenes.INPUT_SH)
    params = _params(cfg, 6)
    sc = scenes.cornell_scene(64, 48, seed=3, n_prims=256, glossy=True, moving_emitter=True, frame=2)
    g = _run(N, cfg, params, sc, 64, 48, 16, 1, 5, 5, 2, 2, 1, light_mode, precision=N.NIRC_FP16_TC)
    o = _oracle(oracle, cfg, params, sc, 64, 48, 16, 1, 5, 5, 2, 2, 1, light_mode)
    err = _row_errors(g, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(g, o, tol=TC_TOL)


def test_multivertex_furnace_exact_on_gpu(N):
    """Emitting Lambertian sphere, exact constant cache, two segments after
    the shading point: every pixel is L_e / (1 - rho) (FP32)."""
    rho = float(np.float32(0.6))
    L = 1.0 / (1 - rho)
    sc = scenes.furnace_scene(48, 48, rho=rho, emission=1.0)
    g = _run(N, scenes.config_small(), None, sc, 48, 48, 4, 2, 2, 3, 5, 1, 3, cache_mode=2, cache_const=(L, L, L))
    assert np.allclose(g["pixel"], L, rtol=5e-6), np.abs(g["pixel"] - L).max()


def test_multivertex_full_size_sampled_pixels(N, oracle):
    """1080p, N_c = 16 / 5 / 4, M = 1, light mode 1, FP16, sampled pixels."""
    cfg = scenes.config_1080p()
    params = _params(cfg, 1)
    W, H = 1920, 1080
    sc = scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=11)
    g = _run(N, cfg, params, sc, W, H, 16, 1, 5, 5, 4, 11, 1, 1, precision=N.NIRC_FP16_TC)
    rng = np.random.default_rng(4)
    pix = np.unique(np.concatenate([rng.integers(0, W * H, 300), [0, W * H - 1]])).astype(np.uint32)
    o = _oracle(oracle, cfg, params, sc, W, H, 16, 1, 5, 5, 4, 11, 1, 1, pixels=pix)
    sub = {k: v[pix] for k, v in g.items()}
    err = _row_errors(sub, o)
    assert err.max() <= TC_TOL, float(err.max())
    _compare_frames(sub, o, tol=TC_TOL)
