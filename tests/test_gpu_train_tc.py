"""Tensor-core training (nirc_set_train_precision(NIRC_FP16_TC)): one
kernel per chunk runs the forward with FP16 operands, the loss of eq. 12 and
the backward with FP16 operands (deltas scaled per record by a power
of two) on tcgen05; the hash-table scatter stays FP32; the weight and bias
gradients of all layers are a second tcgen05 kernel (BF16 operands).

Checked against the oracle's FP64 loss and gradient on ragged batches with
invalid rows, for the frequency input, the 16-level hash grid, the paper's
input (12 levels + spherical harmonics + phi), the visibility output, and 1,
2 and 8 hidden layers; chunked recomputation against stored activations;
the loss curve of 30 Adam steps against FP32 training; deterministic mode
keeping the FP32 kernels; argument errors."""
import numpy as np
import pytest

from paper_2412_04634_gb300 import scenes
from test_gpu_train import N, _near_kink  # noqa: F401

pytestmark = pytest.mark.gpu

# FP16 operands keep 11 significant bits: the forward moves the logits by
# ~1e-3, the backward each delta by ~1e-3 relative, and the weight
# gradients, which sum thousands of records, by less (max error <=
# GRAD_TOL x max |g|).  A hash-table entry sums only the few records around
# it, so there a record counts alone: a hidden unit whose pre-activation
# lies within the FP16 rounding of 0 can switch its ReLU and move that
# record's whole delta.  The parity cases therefore mark invalid the
# records with a pre-activation within KINK_MARGIN of 0 in the oracle's
# FP64 forward (100x the FP16 rounding of these pre-activations), so that
# both sides take the same ReLU decisions, and bound the hash-table
# gradient's relative L2 error by HASH_L2_TOL; with every record kept the
# switches move it by a few percent (ALL_ROWS_L2_TOL).  A wrong index,
# sign or transposition anywhere gives O(1) errors.
LOSS_TOL = 1e-2
GRAD_TOL = 3e-2
HASH_L2_TOL = 1e-2
KINK_MARGIN = 1e-3
ALL_ROWS_L2_TOL = 8e-2
# Per hash-table entry (records near a ReLU kink excluded): the error of
# every entry against its running-error scale (the oracle's loss_grad_abs:
# the backward with every signed sum replaced by the sum of its terms'
# absolute values), which bounds rounding errors however much the terms
# cancel, inside a record's dL/de or across the records of an entry.  FP16
# operands move each term by ~1e-3; a wrong index or a lost contribution
# moves an entry by a whole contribution, which an entry touched by fewer
# than ~100 records shows above ENTRY_TOL though the table's relative L2
# stays small.
ENTRY_TOL = 5e-3  # measured <= 4.7e-4


def _hash_cfg(levels=16, hidden=4, **kw):
    return scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=levels, log2_table=14,
                            hidden_layers=hidden, lr=1e-2, **kw)


CONFIGS = {
    "freq": lambda: scenes.config_small(),
    "hash16": lambda: _hash_cfg(),
    "hash16_h1": lambda: _hash_cfg(hidden=1),
    "hash16_h2": lambda: _hash_cfg(hidden=2),
    "hash16_h8": lambda: _hash_cfg(hidden=8),
    "paper_sh": lambda: _hash_cfg(levels=12, input_encoding=scenes.INPUT_SH),
    "paper_sh_vis": lambda: _hash_cfg(levels=12, input_encoding=scenes.INPUT_SH, output=scenes.OUT_VISIBILITY),
    "hash12_freq": lambda: _hash_cfg(levels=12),
}


def _params(cfg, seed):
    p = scenes.init_params(cfg, seed)
    rng = np.random.default_rng(seed)
    p[:cfg.n_mlp_params] += rng.normal(0, 0.02, cfg.n_mlp_params).astype(np.float32)
    if cfg.n_hash_params:
        p[cfg.n_mlp_params:] = rng.uniform(-0.5, 0.5, cfg.n_hash_params).astype(np.float32)
    return p


def _batch(cfg, n, seed):
    recs, dirs, tg = scenes.training_batch(n, seed=seed)
    if cfg.output == scenes.OUT_VISIBILITY:
        tg = (np.random.default_rng(seed + 1).uniform(size=(n, 1)) < 0.6).astype(np.float32).repeat(3, axis=1)
    recs["flags"][::13] = 0
    return recs, dirs, tg


def _step(N, cfg, params, recs, dirs, tg, tc, store=True, chunk=1024, steps=1):
    import torch
    cache = N.Cache(cfg)
    cache.set_params(params)
    if tc:
        N.nirc_set_train_precision(cache.h, N.NIRC_FP16_TC)
    N.nirc_set_train_mode(cache.h, store, chunk)
    rt, dt, tt = N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), torch.from_numpy(tg).cuda()
    losses = []
    for _ in range(steps):
        loss = torch.zeros(1, device="cuda")
        N.nirc_train_step(cache.h, rt, dt, tt, loss)
        losses.append(loss)
    N.nirc_sync(cache.h)
    out = ([x.item() for x in losses], cache.get_grads().numpy().astype(np.float64),
           cache.get_params().numpy().astype(np.float64))
    cache.close()
    return out


def _grad_errors(cfg, g, g_ref):
    """Per block (MLP, hash table): max error / max |g_ref| and the relative
    L2 error; and the cosine of the whole gradient."""
    errs, l2 = [], []
    for lo, hi in ((0, cfg.n_mlp_params), (cfg.n_mlp_params, cfg.n_params)):
        if hi <= lo:
            continue
        d = g[lo:hi] - g_ref[lo:hi]
        errs.append(np.abs(d).max() / np.abs(g_ref[lo:hi]).max())
        l2.append(np.linalg.norm(d) / np.linalg.norm(g_ref[lo:hi]))
    cos = float(g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref)))
    return errs, l2, cos


def _hash_entry_errors(cfg, g, g_ref, g_abs):
    """Max over the table entries some record touches of |g - g_ref| / the
    entry's running-error scale, and the number of touched entries."""
    nm = cfg.n_mlp_params
    touched = g_abs[nm:] > 0
    err = np.abs(g[nm:] - g_ref[nm:])[touched] / g_abs[nm:][touched]
    assert np.all(g[nm:][~touched] == 0)
    return float(err.max()), int(touched.sum())


@pytest.mark.parametrize("name,n", [(k, 5000) for k in CONFIGS] + [("hash16", (1 << 16) + 301), ("hash16", 100)])
def test_tc_train_step_matches_oracle(N, oracle, name, n):
    """n = 5000: 39 tiles of 128 and a ragged tail of 8 (16-byte loads in
    the weight-gradient kernel); n = 2^16 + 301: 115 sample slices of the
    weight-gradient kernel with a ragged last one, rows of odd length
    (scalar loads); n = 100: one partly filled tile."""
    cfg = CONFIGS[name]()
    params = _params(cfg, 11)
    recs, dirs, tg = _batch(cfg, n, 12)
    kink = _near_kink(oracle, cfg, params, recs, dirs, margin=KINK_MARGIN)
    recs["flags"][kink] = 0
    (loss,), g_gpu, _ = _step(N, cfg, params, recs, dirs, tg, tc=True)
    loss_or, g_or = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    errs, l2, cos = _grad_errors(cfg, g_gpu, g_or)
    print(name, "rows kept", 1 - kink.mean(), "loss rel", abs(loss - loss_or) / abs(loss_or),
          "grad max rel (mlp, hash)", errs, "l2 rel", l2, "cos", cos)
    assert abs(loss - loss_or) <= LOSS_TOL * abs(loss_or)
    assert errs[0] <= GRAD_TOL, errs
    assert l2[0] <= GRAD_TOL, l2
    if len(l2) > 1:
        assert l2[1] <= HASH_L2_TOL, l2
        _, g_abs = oracle.loss_grad_abs(cfg, params, recs, dirs, tg.astype(np.float64))
        e_entry, n_touched = _hash_entry_errors(cfg, g_gpu, g_or, g_abs)
        print(name, "hash entries touched", n_touched, "max error / running-error scale", e_entry)
        assert e_entry <= ENTRY_TOL, e_entry
    assert cos >= 0.999
    # entries no valid record touches stay exactly zero
    assert np.all(g_gpu[cfg.n_mlp_params:][g_or[cfg.n_mlp_params:] == 0] == 0)


@pytest.mark.parametrize("name", ["hash16", "paper_sh"])
def test_tc_train_step_all_rows(N, oracle, name):
    """Every record kept, ReLU switches included: the hash-table gradient
    moves by a few percent (relative L2), the weight gradients as above."""
    cfg = CONFIGS[name]()
    params = _params(cfg, 11)
    recs, dirs, tg = _batch(cfg, 5000, 12)
    (loss,), g_gpu, _ = _step(N, cfg, params, recs, dirs, tg, tc=True)
    loss_or, g_or = oracle.loss_grad(cfg, params, recs, dirs, tg.astype(np.float64))
    errs, l2, cos = _grad_errors(cfg, g_gpu, g_or)
    print(name, "all rows: grad max rel", errs, "l2 rel", l2)
    assert abs(loss - loss_or) <= LOSS_TOL * abs(loss_or)
    assert errs[0] <= GRAD_TOL and l2[0] <= GRAD_TOL, errs
    assert l2[1] <= ALL_ROWS_L2_TOL, l2


def test_tc_train_recompute_matches_stored(N):
    """Chunks of 1024 records with the ragged last chunk, each its own launch,
    against the whole batch in one launch: the same per-record arithmetic,
    so only the order of the gradient sums differs."""
    cfg = _hash_cfg()
    params = _params(cfg, 21)
    recs, dirs, tg = _batch(cfg, 5000, 22)
    (l0,), g0, p0 = _step(N, cfg, params, recs, dirs, tg, tc=True, store=True)
    (l1,), g1, p1 = _step(N, cfg, params, recs, dirs, tg, tc=True, store=False, chunk=1024)
    assert abs(l0 - l1) <= 1e-6 * abs(l0)
    errs, _, _ = _grad_errors(cfg, g1, g0)
    assert max(errs) <= 1e-5, errs
    strong = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert np.abs(p1[strong] - p0[strong]).max() <= 1e-6


def test_tc_training_follows_fp32_training(N):
    """30 Adam steps on one batch: the tensor-core loss curve stays within a
    few percent of the FP32 one and falls as far."""
    cfg = _hash_cfg()
    params = _params(cfg, 31)
    recs, dirs, tg = _batch(cfg, 1 << 14, 32)
    l32, _, _ = _step(N, cfg, params, recs, dirs, tg, tc=False, steps=30)
    l16, _, _ = _step(N, cfg, params, recs, dirs, tg, tc=True, steps=30)
    l32, l16 = np.array(l32), np.array(l16)
    print("fp32", l32[[0, 9, 19, 29]], "tc", l16[[0, 9, 19, 29]])
    assert l32[-1] < 0.5 * l32[0]
    assert np.all(np.abs(l16 - l32) <= 0.05 * l32)


def test_deterministic_mode_keeps_fp32_kernels(N):
    """Deterministic training ignores the tensor-core setting: the step is
    bit-identical to deterministic FP32 training."""
    import torch
    cfg = _hash_cfg()
    params = _params(cfg, 41)
    recs, dirs, tg = _batch(cfg, 3000, 42)
    rt, dt, tt = N.records_to_tensor(recs), torch.from_numpy(dirs).cuda(), torch.from_numpy(tg).cuda()
    res = []
    for tc in (False, True):
        cache = N.Cache(cfg)
        cache.set_params(params)
        N.nirc_set_deterministic(cache.h, True)
        if tc:
            N.nirc_set_train_precision(cache.h, N.NIRC_FP16_TC)
        N.nirc_train_step(cache.h, rt, dt, tt)
        torch.cuda.synchronize()
        res.append((cache.get_grads().numpy(), cache.get_params().numpy()))
        cache.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_train_precision_arguments(N):
    cache = N.Cache(_hash_cfg())
    for bad in (N.NIRC_BF16_TC, N.NIRC_FP8_E4M3_TC, 7):
        with pytest.raises(N.NircError) as ei:
            N.nirc_set_train_precision(cache.h, bad)
        assert ei.value.status == N.NIRC_ERR_INVALID
    # back to FP32 and on again
    N.nirc_set_train_precision(cache.h, N.NIRC_FP16_TC)
    N.nirc_set_train_precision(cache.h, N.NIRC_FP32_SIMT)
    N.nirc_set_train_precision(cache.h, N.NIRC_FP16_TC)
    cache.close()
    # 8 levels x 2 features: 16 position features, not covered
    cache = N.Cache(_hash_cfg(levels=8))
    with pytest.raises(N.NircError) as ei:
        N.nirc_set_train_precision(cache.h, N.NIRC_FP16_TC)
    assert ei.value.status == N.NIRC_ERR_UNSUPPORTED
    cache.close()
