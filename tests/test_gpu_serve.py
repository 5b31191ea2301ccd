"""The frame-request server (include/nirc_serve.h) on the GPU: a served
frame is the frame the single-renderer calls produce, each request's result
is the same alone and in a mixed batch, admission respects the memory
budget, and graph launches match plain stream launches."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_parity import N, _hash_cfg  # noqa: F401

pytestmark = pytest.mark.gpu

T_TRAIN = 4096


def _scene_frames(seed, W=64, H=48, n_prims=64, n_frames=4):
    base = scenes.cornell_scene(W, H, seed=seed, n_prims=n_prims, glossy=True, moving_emitter=True)
    return [scenes.scene_at_frame(base, f) for f in range(n_frames)]


def _cache(N, cfg, seed, precision=1):
    """A scene cache in deterministic training mode, so that a scene's
    weights after k served frames do not depend on what else ran."""
    c = N.Cache(cfg)
    p = scenes.init_params(cfg, seed)
    p[cfg.n_mlp_params:] = np.random.default_rng(seed).uniform(-0.3, 0.3, cfg.n_hash_params).astype(np.float32)
    c.set_params(p)
    N.nirc_set_precision(c.h, precision)
    N.nirc_set_deterministic(c.h, True)
    return c


def _serve(N, requests, n_scenes, slots, max_batches, budget=256 << 20, use_graphs=True, cfg=None):
    """Run `requests` = [(id, scene, W, H, Nc, M, depth, frame)] through a
    fresh server over fresh caches; returns ({id: image}, stats, completions)."""
    import torch
    cfg = cfg or _hash_cfg()
    srv = N.Server(budget, slots=slots, max_batches=max_batches, train_samples=T_TRAIN, use_graphs=use_graphs)
    caches = [_cache(N, cfg, 10 + s) for s in range(n_scenes)]
    for s in range(n_scenes):
        assert srv.add_scene(caches[s], _scene_frames(1 + s), seed=1 + s) == s
    for r in requests:
        srv.submit(*r)
    shapes = {r[0]: (r[2], r[3]) for r in requests}
    imgs, comps = {}, []
    while len(imgs) < len(requests):
        for c in srv.poll(wait=True):
            assert c.status == 0
            W, H = shapes[c.id]
            imgs[c.id] = srv.image(c, W, H)
            comps.append((c.id, c.batch_size, c.t_submit, c.t_launch, c.t_done))
            srv.release(c.id)
    torch.cuda.synchronize()
    st = srv.stats()
    srv.close()
    for c in caches:
        c.close()
    return {k: v.cpu().numpy() for k, v in imgs.items()}, st, comps


def test_served_frame_equals_direct_calls(N):
    """One request = nirc_estimate_frame + nirc_gen_train + nirc_train_step."""
    import torch
    cfg = _hash_cfg()
    frames = _scene_frames(1)
    imgs, st, _ = _serve(N, [(7, 0, 64, 48, 8, 1, 4, 2)], 1, slots=4, max_batches=2, cfg=cfg)
    c = _cache(N, cfg, 10)
    sc = N.scene_to_tensor(frames[2])
    out = torch.empty((64 * 48, 4), device="cuda")
    N.nirc_estimate_frame(c.h, sc, N.frame_desc(64, 48, 8, 1, 4, 2, 1, frames[2].n_prims), out)
    torch.cuda.synchronize()
    assert np.array_equal(imgs[7], out.cpu().numpy())
    assert st["completed"] == 1 and st["failed"] == 0 and st["batches"] == 1
    c.close()


def test_each_result_same_alone_and_in_mix(N):
    """Per-scene request sequences served one request at a time (alone) and
    all interleaved in batches of up to 8 with 2 batches in flight (mix):
    the scene's frames and (deterministic) training steps keep their order,
    so every image is bit-identical."""
    reqs = []
    rid = 0
    sizes = [(64, 48, 8), (32, 32, 4), (80, 40, 16), (48, 48, 32)]
    for k in range(3):
        for s in range(4):
            W, H, Nc = sizes[(s + k) % 4]
            reqs.append((rid, s, W, H, Nc, 1, 4, k))
            rid += 1
    alone, st_a, _ = _serve(N, reqs, 4, slots=1, max_batches=1)
    mixed, st_m, comps = _serve(N, reqs, 4, slots=8, max_batches=2)
    assert st_a["max_batch_seen"] == 1
    assert st_m["max_batch_seen"] >= 2  # the mix really batched requests together
    for r in reqs:
        assert np.array_equal(mixed[r[0]], alone[r[0]]), r


def test_admission_respects_budget(N):
    """A 6 MiB arena holds three 128x96 requests at a time (image + frame
    scratch = 144 B per pixel = 1.77 MB each): everything completes, the
    arena never exceeds the budget, and a request larger than the arena is
    refused at submission."""
    import torch
    cfg = _hash_cfg()
    budget = 6 << 20
    srv = N.Server(budget, slots=8, max_batches=2, train_samples=T_TRAIN)
    caches = [_cache(N, cfg, 20 + s) for s in range(4)]
    for s in range(4):
        srv.add_scene(caches[s], _scene_frames(1 + s, 128, 96), seed=1 + s)
    n = 12
    for i in range(n):
        srv.submit(i, i % 4, 128, 96, 4, 1, 4, i // 4)
    with pytest.raises(N.NircError) as ei:
        srv.submit(99, 0, 1024, 1024, 4, 1, 4, 0)
    assert ei.value.status == N.NIRC_ERR_BUDGET
    done = 0
    while done < n:
        for c in srv.poll(wait=True):
            assert c.status == 0
            srv.release(c.id)
            done += 1
    st = srv.stats()
    assert st["arena_peak_bytes"] <= budget
    assert st["completed"] == n
    assert st["arena_peak_bytes"] >= 2 * 144 * 128 * 96  # requests did share the arena
    srv.close()
    torch.cuda.synchronize()
    for c in caches:
        c.close()


def test_unreleased_images_stall_then_resume(N):
    """Completed images hold arena memory until released: with the arena
    full of unreleased images the queue stalls (poll reports
    NIRC_ERR_BUDGET instead of blocking forever), and releasing resumes it."""
    cfg = _hash_cfg()
    per = 144 * 64 * 48  # image 16 + records 64 + bases 32 + one residual row 32 bytes per pixel
    budget = max(1 << 20, 3 * per)
    srv = N.Server(budget, slots=4, max_batches=1, train_samples=0)
    caches = [_cache(N, cfg, 30 + s) for s in range(2)]
    for s in range(2):
        srv.add_scene(caches[s], _scene_frames(1 + s), seed=1 + s)
    n = 60
    for i in range(n):
        srv.submit(i, i % 2, 64, 48, 4, 1, 4, i)
    held = []
    stalled = False
    while not stalled:
        try:
            got = srv.poll(wait=True)
        except N.NircError as e:
            assert e.status == N.NIRC_ERR_BUDGET
            stalled = True
            break
        held += [c.id for c in got]
    assert 0 < len(held) < n
    for i in held:
        srv.release(i)
    done = len(held)
    while done < n:
        for c in srv.poll(wait=True):
            srv.release(c.id)
            done += 1
    assert srv.stats()["completed"] == n
    srv.close()
    for c in caches:
        c.close()


def test_graph_launch_matches_stream_launch(N):
    reqs = [(i, i % 3, 48, 32, 8, 1, 4, i // 3) for i in range(9)]
    g, st_g, _ = _serve(N, reqs, 3, slots=3, max_batches=1, use_graphs=True)
    s, st_s, _ = _serve(N, reqs, 3, slots=3, max_batches=1, use_graphs=False)
    assert st_g["graph_instantiations"] + st_g["graph_updates"] == st_g["batches"]
    assert st_s["graph_instantiations"] + st_s["graph_updates"] == 0
    for r in reqs:
        assert np.array_equal(g[r[0]], s[r[0]]), r


def _direct_frame(N, cache, frames, W, H, Nc, M, D, frame, seed, light_mode=0):
    import torch
    sc = N.scene_to_tensor(frames[frame % len(frames)])
    out = torch.empty((W * H, 4), device="cuda")
    N.nirc_estimate_frame(cache.h, sc, N.frame_desc(W, H, Nc, M, D, frame, seed, frames[0].n_prims,
                                                    light_mode=light_mode), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _serve_lm(N, requests, precisions, slots=8):
    """Serve [(id, scene, W, H, Nc, M, depth, frame, light_mode)] over fresh
    caches (one per entry of `precisions`); all requests are queued before
    the first poll.  Returns ({id: image}, stats)."""
    import torch
    cfg = _hash_cfg()
    srv = N.Server(64 << 20, slots=slots, max_batches=1, train_samples=T_TRAIN)
    caches = [_cache(N, cfg, 10 + s, precision=p) for s, p in enumerate(precisions)]
    for s in range(len(precisions)):
        srv.add_scene(caches[s], _scene_frames(1 + s), seed=1 + s)
    for r in requests:
        srv.submit(*r)
    shapes = {r[0]: (r[2], r[3]) for r in requests}
    imgs = {}
    while len(imgs) < len(requests):
        for c in srv.poll(wait=True):
            assert c.status == 0
            imgs[c.id] = srv.image(c, *shapes[c.id]).cpu().numpy()
            srv.release(c.id)
    torch.cuda.synchronize()
    st = srv.stats()
    srv.close()
    for c in caches:
        c.close()
    return imgs, st


@pytest.mark.parametrize("light_modes", [(0, 0, 0, 0), (0, 1, 1, 0)])
def test_batch_frames_share_one_launch_per_kernel(N, light_modes):
    """A batch of requests of different resolutions and N over four caches
    is one launch of each path-tracing pass (camera, residual) per light mode
    and one cache-integral launch over the union of their pixels; each request's image is still exactly
    the frame a single renderer computes with its cache (first request of
    every scene: the weights before any served training step)."""
    sizes = [(64, 48, 8), (32, 32, 4), (80, 40, 16), (48, 48, 32)]
    reqs = []
    for k in range(3):
        for s in range(4):
            W, H, Nc = sizes[(s + k) % 4]
            reqs.append((4 * k + s, s, W, H, Nc, 1, 4, k, light_modes[s]))
    imgs, st = _serve_lm(N, reqs, [1, 1, 1, 1])
    modes_per_batch = len(set(light_modes))
    assert st["max_batch_seen"] >= 2
    assert 3 * st["batches"] <= st["frame_launches"] <= (1 + 2 * modes_per_batch) * st["batches"], st
    if modes_per_batch == 1:
        assert st["frame_launches"] == 3 * st["batches"], st
    cfg = _hash_cfg()
    for s in range(4):
        W, H, Nc = sizes[s % 4]
        c = _cache(N, cfg, 10 + s)
        ref = _direct_frame(N, c, _scene_frames(1 + s), W, H, Nc, 1, 4, 0, 1 + s, light_modes[s])
        c.close()
        assert np.array_equal(imgs[s], ref), s


def test_batch_of_mixed_precisions_runs_per_request(N):
    """Caches of different precisions cannot share the cache-integral launch:
    each request then runs its own frame kernels (three launches each), with
    the same images as single-renderer calls."""
    reqs = [(s, s, 48, 32, 8, 1, 4, 0, 0) for s in range(4)]
    precisions = [1, 2, 1, 2]  # FP16 and split BF16 tensor cores
    imgs, st = _serve_lm(N, reqs, precisions)
    assert st["frame_launches"] == 3 * len(reqs), st
    cfg = _hash_cfg()
    for s in range(4):
        c = _cache(N, cfg, 10 + s, precision=precisions[s])
        ref = _direct_frame(N, c, _scene_frames(1 + s), 48, 32, 8, 1, 4, 0, 1 + s)
        c.close()
        assert np.array_equal(imgs[s], ref), s
