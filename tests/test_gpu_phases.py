"""Split frames (nirc_frame_desc.phase): NIRC_PHASE_TRACE then
NIRC_PHASE_CACHE give the image and every auxiliary output of one
NIRC_PHASE_ALL call bit for bit, also with another frame traced on
another stream after the cache pass; a cache pass without a matching
trace is refused."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import N  # noqa: F401

pytestmark = pytest.mark.gpu


def _aux(torch, P, M, N_c):
    return dict(lc=torch.zeros((P, 3), device="cuda"), lr=torch.zeros((P, 3), device="cuda"),
                sig=torch.zeros((P, 2), dtype=torch.int64, device="cuda"),
                count=torch.zeros(P, dtype=torch.int32, device="cuda"),
                row_n=torch.zeros((P * (N_c + M), 3), device="cuda"))


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("estimator", [0, 1, 2])
def test_split_frame_equals_whole(N, precision, estimator):
    import torch
    W, H, Nc = 160, 120, 8
    M = 0 if estimator == 1 else 1
    cfg = scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=16, log2_table=14, hidden_layers=4)
    sc = scenes.cornell_scene(W, H, seed=4, n_prims=64, glossy=True)
    cache = N.Cache(cfg)
    cache.set_params(scenes.init_params(cfg, 6))
    N.nirc_set_precision(cache.h, N.NIRC_FP16_TC if precision == "fp16" else N.NIRC_FP32_SIMT)
    scene = N.scene_to_tensor(sc)
    kw = dict(estimator=estimator, n_cache2=3 if estimator == 2 else 0, n_cache3=2 if estimator == 2 else 0)
    P = W * H
    out0 = torch.zeros((P, 4), device="cuda")
    aux0 = _aux(torch, P, M, Nc)
    N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 3, 1, sc.n_prims, **kw), out0, **aux0)
    out1 = torch.zeros((P, 4), device="cuda")
    aux1 = _aux(torch, P, M, Nc)
    N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 3, 1, sc.n_prims, phase=1, **kw), None,
                          **aux1)
    N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 3, 1, sc.n_prims, phase=2, **kw), out1,
                          **aux1)
    # the next frame traced on another stream after this frame's cache pass
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 4, 1, sc.n_prims, phase=1, **kw), None,
                          stream=side)
    torch.cuda.synchronize()
    assert torch.equal(out0, out1)
    for k in aux0:
        assert torch.equal(aux0[k], aux1[k]), k
    # frame 4 is traced now: a cache pass of frame 3 is refused, frame 4's runs
    with pytest.raises(N.NircError) as ei:
        N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 3, 1, sc.n_prims, phase=2, **kw), out1)
    assert ei.value.status == N.NIRC_ERR_INVALID
    N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 4, 1, sc.n_prims, phase=2, **kw), out1)
    N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 4, 1, sc.n_prims, **kw), out0)
    torch.cuda.synchronize()
    assert torch.equal(out0, out1)
    # a whole-frame call ends the traced state
    with pytest.raises(N.NircError):
        N.nirc_estimate_frame(cache.h, scene, N.frame_desc(W, H, Nc, M, 5, 4, 1, sc.n_prims, phase=2, **kw), out1)
    cache.close()
