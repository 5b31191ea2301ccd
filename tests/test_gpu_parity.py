"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Element by element on the same seeded inputs: integer work (hit primitives,
sample counts, decision signatures, record bits) bit-exact; floating point
within 1e-4 relative per output for the FP32 path, the relative error of a
pixel being |a - b| / max(|b|, 1e-3 mean|b|) so that values that cancel to
near zero are measured against the image scale.
"""
import math

import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def N():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04634_gb300 import build
    build.build()
    from paper_2412_04634_gb300 import nirc
    return nirc


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    floor = 1e-3 * max(np.abs(b).mean(), 1e-30)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def _hash_cfg():
    return scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=16, log2_table=14, hidden_layers=4,
                            lr=1e-2)


def _run_frame(N, cfg, params, scene, W, H, Nc, M, D, frame, seed, cache_mode=0, cache_const=(0, 0, 0),
               precision=0, rows=False, light_mode=0):
    import torch
    cache = N.Cache(cfg)
    if params is not None:
        cache.set_params(params)
    if precision:
        N.nirc_set_precision(cache.h, precision)
    sc = N.scene_to_tensor(scene)
    P = W * H
    out = torch.empty((P, 4), device="cuda")
    lc = torch.empty((P, 3), device="cuda")
    lr = torch.empty((P, 3), device="cuda")
    sig = torch.empty((P, 2), device="cuda", dtype=torch.int64)
    cnt = torch.empty(P, device="cuda", dtype=torch.int32)
    row_n = torch.full((P, Nc + M, 3), -1.0, device="cuda") if rows else None
    desc = N.frame_desc(W, H, Nc, M, D, frame, seed, scene.n_prims, cache_mode, cache_const, light_mode=light_mode)
    N.nirc_estimate_frame(cache.h, sc, desc, out, lc, lr, sig, cnt, row_n)
    N.nirc_sync(cache.h)
    torch.cuda.synchronize()
    cache.close()
    res = dict(pixel=out[:, :3].cpu().numpy(), alpha=out[:, 3].cpu().numpy(), lc=lc.cpu().numpy(),
               lr=lr.cpu().numpy(), sig=sig.cpu().numpy().view(np.uint64), count=cnt.cpu().numpy().view(np.uint32))
    if rows:
        res["row_n"] = row_n.cpu().numpy()
    return res


def frame_errors(g, o):
    """Relative errors of the two levels (each against its own magnitude,
    floored at 1e-3 of its mean) and of the pixel.  The pixel is L_e + L_c +
    L_r and the levels cancel by design (L_r subtracts the cache's
    prediction), so its error is measured against the largest of |pixel|,
    |L_c|, |L_r| and the oracle's sum of the absolute values of L_r's terms
    (the scale of the rounding error of a sum whose terms cancel)."""
    errs = {"lc": rel_err(g["lc"], o["lc"])}
    # L_r = 1/M sum w (L_i - n) cancels internally when the cache is close to
    # L_i: measure it against the cache term's size, which |L_c| estimates
    scale_r = np.maximum(np.abs(o["lr"]), np.abs(o["lc"]))
    if "lr_abs" in o:  # the terms of L_r (later-vertex cache terms included) before they cancel
        scale_r = np.maximum(scale_r, o["lr_abs"])
    scale_r = np.maximum(scale_r, 1e-3 * max(np.abs(o["lr"]).mean(), 1e-30))
    errs["lr"] = np.abs(np.asarray(g["lr"], np.float64) - o["lr"]) / scale_r
    scale = np.maximum.reduce([np.abs(o["pixel"]), np.abs(o["lc"]), np.abs(o["lr"])] +
                              ([o["lr_abs"]] if "lr_abs" in o else []))
    scale = np.maximum(scale, 1e-3 * max(np.abs(o["pixel"]).mean(), 1e-30))
    errs["pixel"] = np.abs(np.asarray(g["pixel"], np.float64) - o["pixel"]) / scale
    return errs


def plain_pixel_error(g, o):
    """The plain per-pixel relative error |a - b| / max(|b|, 1e-3 mean |b|),
    reported beside the asserted, cancellation-aware one of frame_errors:
    where the two levels cancel to a pixel near 0, this one measures the
    rounding of the level terms against the small difference they leave."""
    b = o["pixel"]
    return np.abs(np.asarray(g["pixel"], np.float64) - b) / np.maximum(np.abs(b), 1e-3 * max(np.abs(b).mean(), 1e-30))


def _compare_frames(g, o, tol=FP32_TOL, plain_p99=None):
    assert np.array_equal(g["sig"][:, 0], o["sig"][:, 0]), "path decision signatures differ"
    assert np.array_equal(g["sig"][:, 1], o["sig"][:, 1]), "cache sample signatures differ"
    assert np.array_equal(g["count"], o["count"])
    errs = frame_errors(g, o)
    stats = {k: (float(e.max()), float(np.percentile(e, 99))) for k, e in errs.items()}
    plain = plain_pixel_error(g, o)
    stats["pixel_plain"] = (float(plain.max()), float(np.percentile(plain, 99)))
    print("frame errors (max, p99):", {k: tuple(f"{x:.2e}" for x in v) for k, v in stats.items()})
    for key, err in errs.items():
        assert err.max() <= tol, (key, stats, np.unravel_index(err.argmax(), err.shape))
    if plain_p99 is not None:  # the plain per-pixel error, at the 99th percentile
        assert stats["pixel_plain"][1] <= plain_p99, stats
    assert np.all(g["alpha"] == 1.0)
    return stats


# ---------------------------------------------------------------------------
# cache queries
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["freq", "hash"])
@pytest.mark.parametrize("n", [1, 127, 129, 300, 5000])
def test_query_matches_oracle(N, oracle, which, n):
    import torch
    cfg = scenes.config_small() if which == "freq" else _hash_cfg()
    params = scenes.init_params(cfg, 3)
    rng = np.random.default_rng(n)
    params[:cfg.n_mlp_params] += rng.normal(0, 0.05, cfg.n_mlp_params).astype(np.float32)
    if cfg.n_hash_params:
        params[cfg.n_mlp_params:] = rng.uniform(-1, 1, cfg.n_hash_params).astype(np.float32)
    recs, dirs = scenes.random_query_rows(n, seed=n)
    cache = N.Cache(cfg)
    cache.set_params(params)
    out = torch.empty((n, 3), device="cuda")
    N.nirc_query(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), out)
    got = out.cpu().numpy()
    ref = oracle.query(cfg, params, recs, dirs)
    err = np.abs(got - ref) / np.abs(ref)
    assert err.max() <= FP32_TOL, err.max()


# ---------------------------------------------------------------------------
# two-level frame estimate
# ---------------------------------------------------------------------------

def test_frame_small_workload(N, oracle):
    """64x64 Cornell box, frequency encoding, N = 8, M = 1, depth 4."""
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 1)
    sc = scenes.cornell_scene(64, 64, seed=1)
    for frame in (0, 3):
        g = _run_frame(N, cfg, params, sc, 64, 64, 8, 1, 4, frame, 1, rows=True)
        o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(64, 64, 8, 1, 4, frame, 1), rows=True)
        _compare_frames(g, o, plain_p99=FP32_TOL)
        # every cache output (row) against the oracle's
        valid = o["row_n"] > 0
        assert np.array_equal(valid, g["row_n"] > 0)
        err = np.abs(g["row_n"][valid] - o["row_n"][valid]) / o["row_n"][valid]
        assert err.max() <= FP32_TOL, err.max()


def test_frame_glossy_hashgrid(N, oracle):
    """256-primitive glossy scene with the hash-grid cache at 96x54, N = 16, M = 1, depth 5."""
    cfg = _hash_cfg()
    params = scenes.init_params(cfg, 2)
    params[cfg.n_mlp_params:] = np.random.default_rng(0).uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    sc = scenes.cornell_scene(96, 54, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=7)
    g = _run_frame(N, cfg, params, sc, 96, 54, 16, 1, 5, 7, 1)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(96, 54, 16, 1, 5, 7, 1))
    _compare_frames(g, o, plain_p99=FP32_TOL)


@pytest.mark.parametrize("W,H,Nc,M", [(1, 1, 8, 1), (3, 5, 4, 2), (17, 9, 0, 3), (16, 16, 5, 0), (33, 7, 64, 4)])
def test_frame_edge_shapes(N, oracle, W, H, Nc, M):
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 5)
    sc = scenes.cornell_scene(W, H, seed=2)
    g = _run_frame(N, cfg, params, sc, W, H, Nc, M, 4, 1, 9)
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, Nc, M, 4, 1, 9))
    _compare_frames(g, o, plain_p99=FP32_TOL)


@pytest.mark.parametrize("n_prims", [17, 64, 1000])
def test_frame_bvh_scene_sizes(N, oracle, n_prims):
    """Scenes large enough to use the per-CTA hierarchy (>= 17 primitives, up
    to near the 1024 limit): every hit, hence every decision signature, must
    equal the oracle's brute-force nearest hit."""
    cfg = scenes.config_small()
    W, H = 48, 32
    sc = scenes.cornell_scene(W, H, seed=5, n_prims=n_prims, glossy=True, moving_emitter=True, frame=2)
    g = _run_frame(N, cfg, None, sc, W, H, 4, 2, 8, 1, 3, cache_mode=2, cache_const=(0.3, 0.5, 0.7))
    o = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(W, H, 4, 2, 8, 1, 3, cache_mode=2,
                                                            cache_const=(0.3, 0.5, 0.7)))
    _compare_frames(g, o, plain_p99=FP32_TOL)


def test_zero_and_constant_cache_modes(N, oracle):
    cfg = scenes.config_small()
    sc = scenes.cornell_scene(32, 32, seed=1)
    g = _run_frame(N, cfg, None, sc, 32, 32, 8, 2, 6, 0, 4, cache_mode=1)
    o = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(32, 32, 8, 2, 6, 0, 4, cache_mode=1))
    _compare_frames(g, o, plain_p99=FP32_TOL)
    assert np.all(g["lc"] == 0)
    L = (1.5, 2.0, 3.0)
    g = _run_frame(N, cfg, None, sc, 32, 32, 8, 1, 4, 0, 4, cache_mode=2, cache_const=L)
    o = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(32, 32, 8, 1, 4, 0, 4, cache_mode=2, cache_const=L))
    _compare_frames(g, o, plain_p99=FP32_TOL)


def test_furnace_scene(N, oracle):
    cfg = scenes.config_small()
    sc = scenes.furnace_scene(48, 48, rho=0.5, emission=1.0)
    g = _run_frame(N, cfg, None, sc, 48, 48, 4, 1, 64, 0, 3, cache_mode=2, cache_const=(2.0, 2.0, 2.0))
    o = oracle.estimate(cfg, None, sc.blob(), oracle.oframe(48, 48, 4, 1, 64, 0, 3, cache_mode=2,
                                                            cache_const=(2.0, 2.0, 2.0)))
    _compare_frames(g, o, plain_p99=FP32_TOL)
    assert np.allclose(g["lc"], 1.0, rtol=1e-6)


def test_full_size_sampled_pixels(N, oracle):
    """1920x1080, 256 primitives, hash grid (2^19 entries), N = 16, M = 1,
    depth 5: the launch the benchmark times, checked on sampled pixels."""
    import torch
    cfg = scenes.config_1080p()
    params = scenes.init_params(cfg, 1)
    rng = np.random.default_rng(1)
    params[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    W, H = 1920, 1080
    sc = scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True, frame=11)
    g = _run_frame(N, cfg, params, sc, W, H, 16, 1, 5, 11, 1)
    pix = np.unique(np.concatenate([rng.integers(0, W * H, 400), [0, W - 1, W * H - 1, (H // 2) * W + W // 2]]))
    o = oracle.estimate(cfg, params, sc.blob(), oracle.oframe(W, H, 16, 1, 5, 11, 1), pixels=pix.astype(np.uint32))
    sub = {k: v[pix] for k, v in g.items()}
    _compare_frames(sub, o, plain_p99=FP32_TOL)


# ---------------------------------------------------------------------------
# training records, training step, metrics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["small", "glossy"])
def test_gen_train_matches_oracle(N, oracle, which):
    import torch
    if which == "small":
        cfg, sc, W, H, D = scenes.config_small(), scenes.cornell_scene(64, 64, seed=1), 64, 64, 4
    else:
        W, H, D = 160, 90, 5
        cfg, sc = _hash_cfg(), scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True)
    T = 4099
    cache = N.Cache(cfg)
    recs = torch.empty((T, 16), device="cuda")
    dirs = torch.empty((T, 3), device="cuda")
    tg = torch.empty((T, 3), device="cuda")
    N.nirc_gen_train(cache.h, N.scene_to_tensor(sc), sc.n_prims, W, H, T, 2, 1, D, recs, dirs, tg)
    orec, odir, otg, _ = oracle.gen_train(sc.blob(), W, H, T, 2, 1, D, scenes.RECORD_DTYPE)
    grec = N.records_from_tensor(recs)
    assert np.array_equal(grec.view(np.uint8), orec.view(np.uint8)), "training records differ"
    assert np.array_equal(dirs.cpu().numpy().view(np.uint32), odir.view(np.uint32)), "training directions differ"
    err = rel_err(tg.cpu().numpy(), otg)
    assert err.max() <= FP32_TOL, err.max()
    cache.close()


def _near_kink(oracle, cfg, params, recs, dirs, margin=1e-4):
    """Samples with a hidden pre-activation within `margin` of zero (FP64
    forward of the oracle's encodings; used only to choose test inputs)."""
    p = params.astype(np.float64)
    E = np.stack([oracle.encode(cfg, p, recs[i:i + 1], dirs[i]) for i in range(len(recs))])
    off = 0
    x = E
    mask = np.zeros(len(recs), bool)
    for li, (o, i) in enumerate(cfg.layer_shapes()[:-1]):
        W = p[off:off + o * i].reshape(o, i)
        b = p[off + o * i:off + o * i + o]
        off += o * i + o
        pre = x @ W.T + b
        mask |= (np.abs(pre) < margin).any(1)
        x = np.maximum(pre, 0.0)
    return mask


@pytest.mark.parametrize("which", ["freq", "hash"])
def test_train_step_matches_oracle(N, oracle, which):
    import torch
    cfg = scenes.config_small() if which == "freq" else _hash_cfg()
    params = scenes.init_params(cfg, 4)
    n = 3000
    recs, dirs, tg = scenes.training_batch(n, seed=21)
    recs["flags"][::17] = 0  # some invalid records
    # a sample whose pre-activation sits within rounding of a ReLU kink can
    # switch sides between FP32 and FP64 and move the gradient by a whole
    # sample's contribution: leave such samples out (marked invalid)
    recs["flags"][_near_kink(oracle, cfg, params, recs, dirs)] = 0
    cache = N.Cache(cfg)
    cache.set_params(params)
    loss = torch.zeros(1, device="cuda")
    N.nirc_train_step(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(),
                      torch.from_numpy(tg).cuda(), loss)
    torch.cuda.synchronize()
    g_gpu = cache.get_grads().numpy().astype(np.float64)
    p_gpu = cache.get_params().numpy().astype(np.float64)
    loss_or, g_or = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    assert abs(loss.item() - loss_or) <= 1e-5 * abs(loss_or)
    for lo, hi in ((0, cfg.n_mlp_params), (cfg.n_mlp_params, cfg.n_params)):
        if hi <= lo:
            continue
        scale = np.abs(g_or[lo:hi]).max()
        assert np.abs(g_gpu[lo:hi] - g_or[lo:hi]).max() <= FP32_TOL * scale
    # one Adam step (lr, beta1 0.9, beta2 0.99, eps 1e-15)
    p_or = params.astype(np.float64)
    m = np.zeros_like(p_or)
    v = np.zeros_like(p_or)
    oracle.adam_step(p_or, m, v, g_or, 1, cfg.lr, cfg.beta1, cfg.beta2, cfg.adam_eps)
    strong = np.abs(g_or) > 1e-3 * np.abs(g_or).max()
    assert np.abs(p_gpu[strong] - p_or[strong]).max() <= 1e-6 + 1e-5 * cfg.lr
    # weak gradients: the step can be +-lr (sign at rounding level) but never more
    assert np.all(np.abs(p_gpu - params) <= cfg.lr * (1 + 1e-5) + 1e-7)
    untouched = g_or == 0
    assert np.array_equal(p_gpu[untouched], params[untouched].astype(np.float64))
    cache.close()


def test_mrse_matches_oracle(N, oracle):
    import torch
    rng = np.random.default_rng(3)
    n = 100003
    img = rng.uniform(0, 2, (n, 4)).astype(np.float32)
    ref = rng.uniform(0, 2, (n, 4)).astype(np.float32)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    N.nirc_frame_mrse(torch.from_numpy(img).cuda(), torch.from_numpy(ref).cuda(), out, eps=1e-2)
    # the call takes eps as a binary32 value; each term is formed in binary32
    # (subtract, two squares, add, divide: at most ~5 roundings of 2^-24) and
    # summed in FP64, so the mean of positive terms is within ~3e-7 relative
    want = oracle.mrse(img[:, :3].astype(np.float64), ref[:, :3].astype(np.float64), float(np.float32(1e-2)))
    assert abs(out.item() - want) <= 5e-7 * want


def test_small_workload_four_frames(N, oracle):
    """The 64x64 workload end to end: four frames, each followed by a
    training pass of 4096 paths and one Adam step.  Every frame is compared
    with the oracle run on the GPU's current weights (so the comparison does
    not depend on how the two training trajectories drift apart), every
    training pass bit for bit, every loss within 1e-5."""
    import torch
    cfg = scenes.config_small()
    params = scenes.init_params(cfg, 1)
    sc = scenes.cornell_scene(64, 64, seed=1)
    scd = N.scene_to_tensor(sc)
    cache = N.Cache(cfg)
    cache.set_params(params)
    T = 4096
    recs = torch.empty((T, 16), device="cuda")
    dirs = torch.empty((T, 3), device="cuda")
    tg = torch.empty((T, 3), device="cuda")
    loss = torch.zeros(1, device="cuda")
    P = 64 * 64
    for f in range(4):
        cur = cache.get_params().numpy()
        out = torch.empty((P, 4), device="cuda")
        lc = torch.empty((P, 3), device="cuda")
        lr = torch.empty((P, 3), device="cuda")
        sig = torch.empty((P, 2), device="cuda", dtype=torch.int64)
        cnt = torch.empty(P, device="cuda", dtype=torch.int32)
        N.nirc_estimate_frame(cache.h, scd, N.frame_desc(64, 64, 8, 1, 4, f, 1, sc.n_prims), out, lc, lr, sig, cnt)
        torch.cuda.synchronize()
        g = dict(pixel=out[:, :3].cpu().numpy(), alpha=out[:, 3].cpu().numpy(), lc=lc.cpu().numpy(),
                 lr=lr.cpu().numpy(), sig=sig.cpu().numpy().view(np.uint64), count=cnt.cpu().numpy().view(np.uint32))
        o = oracle.estimate(cfg, cur, sc.blob(), oracle.oframe(64, 64, 8, 1, 4, f, 1))
        _compare_frames(g, o, plain_p99=FP32_TOL)
        N.nirc_gen_train(cache.h, scd, sc.n_prims, 64, 64, T, f, 1, 4, recs, dirs, tg)
        orec, odir, otg, _ = oracle.gen_train(sc.blob(), 64, 64, T, f, 1, 4, scenes.RECORD_DTYPE)
        assert np.array_equal(N.records_from_tensor(recs).view(np.uint8), orec.view(np.uint8))
        assert np.array_equal(dirs.cpu().numpy().view(np.uint32), odir.view(np.uint32))
        N.nirc_train_step(cache.h, recs, dirs, tg, loss)
        torch.cuda.synchronize()
        loss_or, _ = oracle.loss_grad(cfg, cur, orec, odir, tg.cpu().numpy().astype(np.float64))
        assert abs(loss.item() - loss_or) <= 1e-5 * abs(loss_or), (f, loss.item(), loss_or)
    cache.close()
