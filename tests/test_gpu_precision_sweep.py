"""Precision sweep on the 1080p workload against the FP64 oracle.

The cache is trained on-line for 30 frames of the dynamic 1080p scene (256
primitives, hash grid 16 x 2 x 2^19, MLP 64 x 4), then frozen; frame 30 is
rendered with the layer arithmetic FP32 SIMT, FP16, split BF16 and FP8
(E4M3 hidden layers) tensor cores at
N = 4, 8, 16, 32, 64 (M = 1).  For each point, on about 65,536 sampled rows
(whole pixels, all of their rows): the per-row relative error of the cache
value n against the oracle (max and 99th percentile, relative to
max(|n|, 1e-3 mean n)); and the MRSE of the
sampled pixels against a 256-spp path-traced reference, for the GPU image
and for the oracle's image.  Set NIRC_SWEEP_OUT to a file name to get the
table as JSON.
"""
import json
import os

import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import N  # noqa: F401

pytestmark = pytest.mark.gpu

W, H = 1920, 1080
FRAMES = 30
T_TRAIN = 65536
NS = (4, 8, 16, 32, 64)
ROWS = 65536


def _mrse(img, ref, eps=1e-2):
    img = np.asarray(img, np.float64)[:, :3]
    ref = np.asarray(ref, np.float64)[:, :3]
    return float(np.mean((img - ref) ** 2 / (ref ** 2 + eps)))


@pytest.fixture(scope="module", params=["trained30", "init", "trained30_nee"])
def trained(N, request):
    """Cache weights after 30 training frames (or the initial weights) and
    the frame-30 scene.  With BSDF-sampled training paths and the small
    emitter, almost every training target is 0 and the trained cache sinks
    towards 0 in most of the scene (the oracle does the same), so the
    initial weights are swept as well to show the arithmetic on a network
    whose outputs are O(1), and light mode 1 (the cache learns L_ind, direct
    light by NEE + MIS), whose training targets are mostly non-zero."""
    import torch
    cfg = scenes.config_1080p()
    base = scenes.cornell_scene(W, H, seed=1, n_prims=256, glossy=True, moving_emitter=True)
    cache = N.Cache(cfg)
    p0 = scenes.init_params(cfg, 1)
    if request.param == "init":
        p0[cfg.n_mlp_params:] = np.random.default_rng(2).uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    cache.set_params(p0)
    recs = torch.empty((T_TRAIN, 16), device="cuda")
    dirs = torch.empty((T_TRAIN, 3), device="cuda")
    tgts = torch.empty((T_TRAIN, 3), device="cuda")
    lm = 1 if request.param.endswith("_nee") else 0
    for f in range(FRAMES if request.param.startswith("trained30") else 0):
        sc = N.scene_to_tensor(scenes.scene_at_frame(base, f))
        N.nirc_gen_train(cache.h, sc, base.n_prims, W, H, T_TRAIN, f, 1, 5, recs, dirs, tgts, light_mode=lm)
        N.nirc_train_step(cache.h, recs, dirs, tgts)
    torch.cuda.synchronize()
    params = cache.get_params().numpy()
    scene = scenes.scene_at_frame(base, FRAMES)
    sc = N.scene_to_tensor(scene)
    # reference: 256 spp of plain path tracing (zero cache), depth 16
    ref = torch.zeros((W * H, 4), device="cuda")
    tmp = torch.empty((W * H, 4), device="cuda")
    for k in range(16):
        N.nirc_estimate_frame(cache.h, sc, N.frame_desc(W, H, 0, 16, 16, 5000 + k, 1, scene.n_prims, cache_mode=1),
                              tmp)
        ref += tmp
    ref /= 16
    torch.cuda.synchronize()
    yield cfg, params, scene, sc, ref.cpu().numpy(), cache, request.param, lm
    cache.close()


def _gpu_frame(N, cache, sc, scene, Nc, precision, pix, lm):
    import torch
    N.nirc_set_precision(cache.h, precision)
    S = Nc + 1
    out = torch.empty((W * H, 4), device="cuda")
    row_n = torch.empty((W * H, S, 3), device="cuda")
    N.nirc_estimate_frame(cache.h, sc, N.frame_desc(W, H, Nc, 1, 5, FRAMES, 1, scene.n_prims, light_mode=lm), out,
                          row_n=row_n)
    idx = torch.from_numpy(pix.astype(np.int64)).cuda()
    sub_rows = row_n[idx].cpu().numpy().astype(np.float64)
    img = out.cpu().numpy()
    del row_n
    return img, sub_rows


def test_precision_sweep(N, oracle, trained):
    cfg, params, scene, sc, ref, cache, state, lm = trained
    precisions = {"fp32_simt": N.NIRC_FP32_SIMT, "fp16_tc": N.NIRC_FP16_TC, "bf16_tc": N.NIRC_BF16_TC,
                  "fp8_tc": N.NIRC_FP8_E4M3_TC}
    rng = np.random.default_rng(30)
    table = []
    for Nc in NS:
        S = Nc + 1
        pix = np.sort(rng.choice(W * H, (ROWS + S - 1) // S, replace=False)).astype(np.uint32)
        o = oracle.estimate(cfg, params, scene.blob(), oracle.oframe(W, H, Nc, 1, 5, FRAMES, 1, light_mode=lm),
                            pixels=pix, rows=True)
        m_or = _mrse(o["pixel"], ref[pix])
        for name, code in precisions.items():
            img, rows = _gpu_frame(N, cache, sc, scene, Nc, code, pix, lm)
            # rows of invalid samples are 0 on both sides; a valid row's n is
            # exp(z) > 0 in FP64 but can underflow to 0 in FP32 for z < -87,
            # so errors are taken against a floor of 1e-3 x the mean value
            valid = o["row_n"] > 0
            assert not np.any(rows[~valid]), (name, Nc)
            floor = 1e-3 * o["row_n"][valid].mean()
            err = np.abs(rows[valid] - o["row_n"][valid]) / np.maximum(o["row_n"][valid], floor)
            m_gpu = _mrse(img[pix], ref[pix])
            rec = {"weights": state, "light_mode": lm, "precision": name, "N": Nc, "rows": int(valid.sum() // 3), "row_err_max": float(err.max()),
                   "row_err_p99": float(np.percentile(err, 99)), "mrse_gpu": m_gpu, "mrse_oracle": m_or,
                   "mrse_rel_diff": abs(m_gpu - m_or) / m_or, "mrse_gpu_full_frame": _mrse(img, ref),
                   "rows_below_floor": int(np.sum(o["row_n"][valid] < floor)),
                   "rows_zero_on_gpu": int(np.sum(rows[valid] == 0)),
                   "max_oracle_where_gpu_zero": float(np.max(o["row_n"][valid & (rows == 0)], initial=0.0))}
            table.append(rec)
            print(json.dumps(rec))
    out = os.environ.get("NIRC_SWEEP_OUT")
    if out:
        with open(out + "." + state + ".json", "w") as f:
            json.dump(table, f, indent=1)
    for r in table:
        if r["precision"] == "fp32_simt":
            assert r["row_err_max"] <= 1e-4, r
        elif r["precision"] == "fp8_tc":
            # E4M3 keeps 3 mantissa bits and exp() turns z's absolute error into
            # n's relative error: ~36 % at the 99th percentile on trained
            # weights (reported); the frame MRSE moves by < 1 %
            assert r["row_err_p99"] <= 0.5, r
            assert r["mrse_rel_diff"] <= 0.05, r
        else:
            # FP16, and BF16 with split (hi + lo) operands: 2e-2 per cache output at the
            # maximum, although n = exp(z) turns z's absolute error into n's relative
            # error and trained logits of small radiance are -6 .. -10
            assert r["row_err_max"] <= 2e-2, r
            assert r["mrse_rel_diff"] <= 0.01, r
