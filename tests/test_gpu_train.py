"""Training-side parity of the CUDA path with the oracle: the backward of
the bare query (nirc_query_bwd) and its torch.autograd.Function wrapper,
activation recomputation against stored activations, and the
warp-aggregated hash-gradient scatter under heavy entry collisions."""
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


def _hash_cfg(levels=16, log2_table=14, hidden=4):
    return scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=levels, log2_table=log2_table,
                            hidden_layers=hidden, lr=1e-2)


def _near_kink(oracle, cfg, params, recs, dirs, margin=1e-4):
    """Rows with a hidden pre-activation within `margin` of zero (FP64
    forward of the oracle's encodings; used only to choose test inputs)."""
    p = params.astype(np.float64)
    E = np.stack([oracle.encode(cfg, p, recs[i:i + 1], dirs[i]) for i in range(len(recs))])
    off = 0
    x = E
    mask = np.zeros(len(recs), bool)
    for o, i in cfg.layer_shapes()[:-1]:
        W = p[off:off + o * i].reshape(o, i)
        b = p[off + o * i:off + o * i + o]
        off += o * i + o
        pre = x @ W.T + b
        mask |= (np.abs(pre) < margin).any(1)
        x = np.maximum(pre, 0.0)
    return mask


def _assert_grad_close(cfg, g_gpu, g_or, tol=FP32_TOL):
    for lo, hi in ((0, cfg.n_mlp_params), (cfg.n_mlp_params, cfg.n_params)):
        if hi <= lo:
            continue
        scale = np.abs(g_or[lo:hi]).max()
        err = np.abs(g_gpu[lo:hi] - g_or[lo:hi]).max()
        assert err <= tol * scale, (lo, hi, err, scale)


@pytest.mark.parametrize("which", ["freq", "hash"])
def test_query_bwd_matches_oracle(N, oracle, which):
    import torch
    cfg = scenes.config_small() if which == "freq" else _hash_cfg()
    params = scenes.init_params(cfg, 41)
    n = 3001
    recs, dirs = scenes.random_query_rows(n, seed=42)
    recs["flags"][::5] = 0  # the valid flag does not matter to a bare query
    rng = np.random.default_rng(43)
    gout = rng.normal(0, 1, (n, 3)).astype(np.float32)
    gout[_near_kink(oracle, cfg, params, recs, dirs)] = 0.0
    cache = N.Cache(cfg)
    cache.set_params(params)
    g = torch.empty(cfg.n_params, device="cuda")
    val = torch.zeros(1, device="cuda")
    N.nirc_query_bwd(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(),
                     torch.from_numpy(gout).cuda(), g, val)
    torch.cuda.synchronize()
    val_or, g_or = oracle.query_grad(cfg, params, recs, dirs, gout.astype(np.float64))
    assert abs(val.item() - val_or) <= 1e-5 * np.abs(gout).sum() * np.abs(oracle.query(cfg, params, recs, dirs)).max()
    g_gpu = g.cpu().numpy().astype(np.float64)
    _assert_grad_close(cfg, g_gpu, g_or)
    # the handle's gradient buffer holds the same vector
    assert np.array_equal(cache.get_grads().numpy(), g.cpu().numpy())
    # entries no row touches stay exactly zero
    assert np.all(g_gpu[g_or == 0] == 0)
    cache.close()


def test_query_bwd_empty_batch_zeroes_gradient(N):
    import torch
    cfg = scenes.config_small()
    cache = N.Cache(cfg)
    cache.set_params(scenes.init_params(cfg, 1))
    g = torch.full((cfg.n_params,), 7.0, device="cuda")
    empty_r = torch.empty((0, 16), device="cuda")
    empty_d = torch.empty((0, 3), device="cuda")
    N.nirc_query_bwd(cache.h, empty_r, empty_d, empty_d, g)
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
    cache.close()


def test_autograd_function(N, oracle):
    """NircQuery.apply: the forward equals nirc_query, the gradient equals
    nirc_query_bwd bit for bit and the oracle within FP32 tolerance, and a
    central difference along the gradient agrees with |g|^2."""
    import torch
    cfg = _hash_cfg(levels=8, log2_table=12, hidden=3)
    params = scenes.init_params(cfg, 51)
    rng = np.random.default_rng(52)
    params[cfg.n_mlp_params:] = rng.uniform(-0.2, 0.2, cfg.n_hash_params).astype(np.float32)
    n = 2000
    recs, dirs = scenes.random_query_rows(n, seed=53)
    target = rng.uniform(0.5, 2.0, (n, 3)).astype(np.float32)
    cache = N.Cache(cfg)
    cache.set_params(params)
    rt = N.records_to_tensor(recs)
    dt = torch.from_numpy(dirs).cuda()
    tt = torch.from_numpy(target).cuda()
    p = torch.from_numpy(params).cuda().requires_grad_(True)

    def f(pp):
        out = N.NircQuery.apply(pp, rt, dt, cache)
        return ((out - tt) ** 2).sum(), out

    loss, out = f(p)
    loss.backward()
    ref = torch.empty(n, 3, device="cuda")
    N.nirc_query(cache.h, rt, dt, ref)
    torch.cuda.synchronize()
    assert torch.equal(out.detach(), ref)
    gout = (2.0 * (out.detach() - tt)).contiguous()
    g2 = torch.empty(cfg.n_params, device="cuda")
    N.nirc_query_bwd(cache.h, rt, dt, gout, g2)
    torch.cuda.synchronize()
    # float atomics make the gradient order-dependent at rounding level
    gg = p.grad.detach()
    assert torch.allclose(gg, g2, rtol=0, atol=1e-6 * g2.abs().max().item())
    _, g_or = oracle.query_grad(cfg, params, recs, dirs, gout.cpu().numpy().astype(np.float64))
    _assert_grad_close(cfg, gg.cpu().numpy().astype(np.float64), g_or, tol=2e-4)
    # directional finite difference along the (normalised) gradient, in FP32
    v = gg / gg.norm()
    h = 1e-3
    with torch.no_grad():
        lp, _ = f(p.detach() + h * v)
        lm, _ = f(p.detach() - h * v)
    fd = (lp.item() - lm.item()) / (2 * h)
    assert abs(fd - gg.norm().item()) <= 2e-2 * gg.norm().item(), (fd, gg.norm().item())
    cache.close()


def test_recompute_matches_stored(N):
    """Activation recomputation in chunks (ragged last chunk) gives the loss,
    gradient and Adam step of the stored-activation pass."""
    import torch
    cfg = _hash_cfg()
    params = scenes.init_params(cfg, 61)
    n = 5000
    recs, dirs, tg = scenes.training_batch(n, seed=62)
    recs["flags"][::13] = 0
    rt = N.records_to_tensor(recs)
    dt = torch.from_numpy(dirs).cuda()
    tt = torch.from_numpy(tg).cuda()
    res = []
    for store in (True, False):
        cache = N.Cache(cfg)
        cache.set_params(params)
        N.nirc_set_train_mode(cache.h, store, 1024)
        loss = torch.zeros(1, device="cuda")
        N.nirc_train_step(cache.h, rt, dt, tt, loss)
        torch.cuda.synchronize()
        res.append((loss.item(), cache.get_grads().numpy().astype(np.float64),
                    cache.get_params().numpy().astype(np.float64)))
        cache.close()
    (l0, g0, p0), (l1, g1, p1) = res
    assert abs(l0 - l1) <= 1e-6 * abs(l0)
    _assert_grad_close(cfg, g1, g0, tol=1e-5)
    strong = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert np.abs(p1[strong] - p0[strong]).max() <= 1e-6


def test_sliced_weight_gradients_match_chunked(N):
    """Passes of >= 2^18 samples take their weight and bias gradients from
    k_grad_w_big (a block per layer and slice of the samples, a ragged last
    slice and stage here); 2^17-sample chunks of the same batch take them
    from k_grad_w: the two agree up to the order of the sums."""
    import torch
    cfg = _hash_cfg(hidden=4)
    params = scenes.init_params(cfg, 65)
    n = (1 << 18) + 123
    recs, dirs, tg = scenes.training_batch(n, seed=66)
    recs["flags"][::17] = 0
    rt, dt, tt = N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), torch.from_numpy(tg).cuda()
    res = []
    for store in (True, False):
        cache = N.Cache(cfg)
        cache.set_params(params)
        N.nirc_set_train_mode(cache.h, store, 1 << 17)
        N.nirc_train_step(cache.h, rt, dt, tt)
        torch.cuda.synchronize()
        res.append(cache.get_grads().numpy().astype(np.float64))
        cache.close()
    g_sliced, g_chunked = res
    _assert_grad_close(cfg, g_sliced, g_chunked, tol=1e-5)


def test_scatter_with_colliding_entries(N, oracle):
    """Many rows share a few positions, so whole warps hit the same table
    entries: the aggregated scatter must still add every contribution."""
    import torch
    # 2^14 entries: levels 0-1 (16^3, 24^3 cells) are dense and take the
    # warp-aggregated path, levels 2-5 are hashed
    cfg = _hash_cfg(levels=6, log2_table=14, hidden=2)
    params = scenes.init_params(cfg, 71)
    n = 4096
    recs, dirs, tg = scenes.training_batch(n, seed=72)
    rng = np.random.default_rng(73)
    pts = rng.uniform(0, 1, (5, 3))
    recs["p"] = pts[rng.integers(0, 5, n)]
    recs["p"][:64] = pts[0]  # two full warps on one point
    recs["flags"][100::9] = 0
    recs["flags"][_near_kink(oracle, cfg, params, recs, dirs)] = 0
    cache = N.Cache(cfg)
    cache.set_params(params)
    loss = torch.zeros(1, device="cuda")
    N.nirc_train_step(cache.h, N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(),
                      torch.from_numpy(tg).cuda(), loss)
    torch.cuda.synchronize()
    g_gpu = cache.get_grads().numpy().astype(np.float64)
    _, g_or = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    touched = np.nonzero(g_or[cfg.n_mlp_params:])[0]
    assert 0 < touched.size <= 5 * 8 * 6 * 2
    _assert_grad_close(cfg, g_gpu, g_or)
    cache.close()


@pytest.mark.parametrize("store", [True, False])
def test_deterministic_training_is_bit_reproducible(N, oracle, store):
    """Deterministic mode: two handles given the same state and batch take
    bit-identical training steps (loss, gradient, weights), and the
    gradient still matches the oracle within the FP32 tolerance."""
    import torch
    cfg = _hash_cfg()
    params = scenes.init_params(cfg, 81)
    n = 5000
    recs, dirs, tg = scenes.training_batch(n, seed=82)
    recs["flags"][::11] = 0
    recs["flags"][_near_kink(oracle, cfg, params, recs, dirs)] = 0
    rt = N.records_to_tensor(recs)
    dt = torch.from_numpy(dirs).cuda()
    tt = torch.from_numpy(tg).cuda()
    runs = []
    for _ in range(2):
        cache = N.Cache(cfg)
        cache.set_params(params)
        N.nirc_set_deterministic(cache.h, True)
        N.nirc_set_train_mode(cache.h, store, 1024)
        losses = []
        for _ in range(2):
            loss = torch.zeros(1, device="cuda")
            N.nirc_train_step(cache.h, rt, dt, tt, loss)
            losses.append(loss.item())
            if not runs and len(losses) == 1:
                g_first = cache.get_grads().numpy().astype(np.float64)
        torch.cuda.synchronize()
        runs.append((losses, cache.get_grads().numpy(), cache.get_params().numpy()))
        cache.close()
    (l0, g0, p0), (l1, g1, p1) = runs
    assert l0 == l1
    assert np.array_equal(g0, g1) and np.array_equal(p0, p1)
    _, g_or = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    _assert_grad_close(cfg, g_first, g_or)


def test_deterministic_query_bwd(N, oracle):
    import torch
    cfg = _hash_cfg()
    params = scenes.init_params(cfg, 91)
    n = 3000
    recs, dirs = scenes.random_query_rows(n, seed=92)
    gout = np.random.default_rng(93).normal(0, 1, (n, 3)).astype(np.float32)
    gout[_near_kink(oracle, cfg, params, recs, dirs)] = 0.0
    cache = N.Cache(cfg)
    cache.set_params(params)
    N.nirc_set_deterministic(cache.h, True)
    rt, dt, gt = N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), torch.from_numpy(gout).cuda()
    g1 = torch.empty(cfg.n_params, device="cuda")
    g2 = torch.empty(cfg.n_params, device="cuda")
    N.nirc_query_bwd(cache.h, rt, dt, gt, g1)
    N.nirc_query_bwd(cache.h, rt, dt, gt, g2)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    _, g_or = oracle.query_grad(cfg, params, recs, dirs, gout.astype(np.float64))
    _assert_grad_close(cfg, g1.cpu().numpy().astype(np.float64), g_or)
    cache.close()


def test_save_load_state_resumes_training_exactly(N):
    """Checkpoint after two deterministic steps, take two more; a fresh cache
    loaded from the checkpoint takes the same two steps to the same bits.
    A state of another configuration is refused."""
    import torch
    cfg = _hash_cfg(levels=8, log2_table=12, hidden=3)
    params = scenes.init_params(cfg, 91)
    batches = []
    for k in range(4):
        r, d, t = scenes.training_batch(2000, seed=100 + k)
        batches.append((N.records_to_tensor(r), torch.from_numpy(d).cuda(), torch.from_numpy(t).cuda()))
    a = N.Cache(cfg)
    a.set_params(params)
    N.nirc_set_deterministic(a.h, True)
    for rt, dt, tt in batches[:2]:
        N.nirc_train_step(a.h, rt, dt, tt)
    state = N.nirc_save_state(a.h)
    for rt, dt, tt in batches[2:]:
        N.nirc_train_step(a.h, rt, dt, tt)
    torch.cuda.synchronize()
    b = N.Cache(cfg)
    N.nirc_set_deterministic(b.h, True)
    N.nirc_load_state(b.h, state)
    for rt, dt, tt in batches[2:]:
        N.nirc_train_step(b.h, rt, dt, tt)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params().numpy(), b.get_params().numpy())
    other = N.Cache(_hash_cfg(levels=8, log2_table=12, hidden=2))
    with pytest.raises(N.NircError) as ei:
        N.nirc_load_state(other.h, state)
    assert ei.value.status == N.NIRC_ERR_INVALID
    for c in (a, b, other):
        c.close()
