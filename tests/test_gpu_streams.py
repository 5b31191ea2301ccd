"""Training records generated on a second stream while the frame estimate
runs on the first (the bench's frame step does this): both read only the
scene and use their own work counters, so the image, the decision
signatures and the training records are bit-identical to the serial
order."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import N  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_records_on_second_stream_match_serial(N, precision):
    import torch
    W, H, T = 320, 240, 1 << 14
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=16, log2_table=16, hidden_layers=4)
    sc = scenes.cornell_scene(W, H, seed=3, n_prims=256, glossy=True)
    cache = N.Cache(cfg)
    cache.set_params(scenes.init_params(cfg, 5))
    N.nirc_set_precision(cache.h, N.NIRC_FP16_TC if precision == "fp16" else N.NIRC_FP32_SIMT)
    scene = N.scene_to_tensor(sc)
    desc = N.frame_desc(W, H, 16, 1, 5, 7, 1, sc.n_prims)
    res = []
    for concurrent in (False, True):
        out = torch.empty((W * H, 4), device="cuda")
        sig = torch.empty((W * H, 2), dtype=torch.int64, device="cuda")
        recs = torch.empty((T, 16), device="cuda")
        dirs = torch.empty((T, 3), device="cuda")
        tgts = torch.empty((T, 3), device="cuda")
        main = torch.cuda.current_stream()
        if concurrent:
            side = torch.cuda.Stream()
            side.wait_stream(main)
            N.nirc_gen_train(cache.h, scene, sc.n_prims, W, H, T, 7, 1, 5, recs, dirs, tgts, stream=side)
            N.nirc_estimate_frame(cache.h, scene, desc, out, sig=sig)
            main.wait_stream(side)
        else:
            N.nirc_estimate_frame(cache.h, scene, desc, out, sig=sig)
            N.nirc_gen_train(cache.h, scene, sc.n_prims, W, H, T, 7, 1, 5, recs, dirs, tgts)
        N.nirc_sync(cache.h)
        res.append([x.cpu().numpy() for x in (out, sig, recs, dirs, tgts)])
    cache.close()
    for a, b in zip(*res):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_ray_counter(N):
    """nirc_frame_aux.rays: with no residual paths (M = 0) the path tracer
    traces exactly one camera ray per pixel; the count is reproducible and
    grows with M and with the path depth; it does not change the image."""
    import torch
    W, H = 160, 120
    cfg = scenes.config_small()
    sc = scenes.cornell_scene(W, H, seed=3, n_prims=64, glossy=True)
    cache = N.Cache(cfg)
    cache.set_params(scenes.init_params(cfg, 5))
    scene = N.scene_to_tensor(sc)

    def rays(M, D):
        r = torch.zeros(1, dtype=torch.int64, device="cuda")
        out = torch.empty((W * H, 4), device="cuda")
        N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, 8, M, D, 2, 1, sc.n_prims), out, rays=r)
        plain = torch.empty_like(out)
        N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, 8, M, D, 2, 1, sc.n_prims), plain)
        torch.cuda.synchronize()
        assert torch.equal(out, plain)
        return int(r.item())

    assert rays(0, 5) == W * H
    r1 = rays(1, 5)
    assert r1 == rays(1, 5)
    assert W * H < rays(1, 1) < r1 < rays(2, 5)
    cache.close()
