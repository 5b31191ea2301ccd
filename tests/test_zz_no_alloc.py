"""nirc_estimate_frame_noalloc, the frame estimate for callers that cannot
allocate device memory during a call (pre-reserved memory, real-time frame
loops that must avoid cudaMalloc's synchronisation, strict allocation
policies): it must give the same frame as nirc_estimate_frame, call after
call, for each estimator (whose scratch layouts differ), while using only the
library's fixed scratch area.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the FP32 parity tolerance of the other GPU tests
TWO_LEVEL, BTH, MULTI_VERTEX = 0, 1, 2


@pytest.fixture(scope="module")
def N():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_04634_gb300 import build
    build.build()
    from paper_2412_04634_gb300 import nirc
    return nirc


def _frame(N, fn, cache, sc_dev, desc, P, S):
    import torch
    out = torch.full((P, 4), -1.0, device="cuda")
    lc = torch.empty((P, 3), device="cuda")
    lr = torch.empty((P, 3), device="cuda")
    sig = torch.empty((P, 2), device="cuda", dtype=torch.int64)
    cnt = torch.empty(P, device="cuda", dtype=torch.int32)
    row_n = torch.empty((P, S, 3), device="cuda")
    fn(cache.h, sc_dev, desc, out, lc, lr, sig, cnt, row_n)
    N.nirc_sync(cache.h)
    return {k: v.cpu().numpy() for k, v in dict(out=out, lc=lc, lr=lr, sig=sig, cnt=cnt, row_n=row_n).items()}


def _desc(N, estimator, W, H, frame, n_prims):
    if estimator == BTH:  # N cache samples at the stopping vertex, no residual rows
        return N.frame_desc(W, H, 8, 0, 4, frame, 5, n_prims, estimator=BTH), 8
    if estimator == MULTI_VERTEX:  # the two levels at the first three vertices
        return N.frame_desc(W, H, 8, 2, 4, frame, 5, n_prims, estimator=MULTI_VERTEX, n_cache2=4, n_cache3=3), 10
    return N.frame_desc(W, H, 8, 2, 4, frame, 5, n_prims), 10


@pytest.mark.parametrize("estimator", [TWO_LEVEL, BTH, MULTI_VERTEX])
@pytest.mark.parametrize("precision", [0, 1])  # FP32 SIMT, FP16 tensor cores
def test_noalloc_matches_estimate_frame(N, precision, estimator):
    cfg = scenes.config_small()
    W, H = 64, 48
    P = W * H
    cache = N.Cache(cfg)
    cache.set_params(scenes.init_params(cfg, 3))
    N.nirc_set_precision(cache.h, precision)
    sc = scenes.cornell_scene(W, H, seed=2)
    sc_dev = N.scene_to_tensor(sc)
    for frame in (0, 1):  # two calls in a row
        desc, S = _desc(N, estimator, W, H, frame, sc.n_prims)
        a = _frame(N, N.nirc_estimate_frame_noalloc, cache, sc_dev, desc, P, S)
        b = _frame(N, N.nirc_estimate_frame, cache, sc_dev, desc, P, S)
        assert np.array_equal(a["sig"], b["sig"]) and np.array_equal(a["cnt"], b["cnt"])
        for k in ("out", "lc", "lr", "row_n"):
            scale = np.maximum(np.abs(b[k]), 1e-3 * max(np.abs(b[k]).mean(), 1e-30))
            err = np.abs(a[k] - b[k]) / scale
            assert err.max() <= TOL, (frame, k, float(err.max()))
        assert np.all(a["out"][:, 3] == 1.0)
    cache.close()


def test_noalloc_allocates_nothing(N):
    """The device's free memory is the same before and after a frame on a
    fresh handle.  The frame's scratch would be 2.5 MiB, so an allocation
    of it could not hide in memory the driver had already reserved; the
    kernels are loaded by a first call on another handle."""
    import torch
    cfg = scenes.config_small()
    W, H, M = 128, 128, 2
    sc = scenes.cornell_scene(W, H, seed=2)
    sc_dev = N.scene_to_tensor(sc)
    desc = N.frame_desc(W, H, 8, M, 4, 0, 5, sc.n_prims)
    out = torch.empty((W * H, 4), device="cuda")
    warm = N.Cache(cfg)
    warm.set_params(scenes.init_params(cfg, 3))
    N.nirc_estimate_frame_noalloc(warm.h, sc_dev, desc, out)
    N.nirc_sync(warm.h)
    ref = out.clone()
    cache = N.Cache(cfg)
    cache.set_params(scenes.init_params(cfg, 3))
    N.nirc_sync(cache.h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    N.nirc_estimate_frame_noalloc(cache.h, sc_dev, desc, out)
    N.nirc_sync(cache.h)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert torch.equal(out, ref)  # same weights, same frame
    cache.close()
    warm.close()


def test_noalloc_rejects_frames_beyond_its_area(N):
    cfg = scenes.config_small()
    cache = N.Cache(cfg)
    sc = scenes.cornell_scene(512, 512, seed=2)
    import torch
    out = torch.empty((512 * 512, 4), device="cuda")
    for estimator, m in ((TWO_LEVEL, 1), (BTH, 0), (MULTI_VERTEX, 1)):
        desc = N.frame_desc(512, 512, 8, m, 4, 0, 1, sc.n_prims, estimator=estimator)
        status = N.lib().nirc_estimate_frame_noalloc(cache.h, ctypes.c_void_p(N.scene_to_tensor(sc).data_ptr()),
                                                     ctypes.byref(desc), ctypes.c_void_p(out.data_ptr()), None, None)
        assert status == N.NIRC_ERR_BUDGET
        msg = N.lib().nirc_last_error()
        assert b"4194304" in msg and (b"estimator %d" % estimator) in msg, msg
    cache.close()
