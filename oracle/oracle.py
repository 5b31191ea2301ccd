"""ctypes wrapper of the CPU oracle (oracle/nirc_oracle.c).

Test infrastructure only: used by tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg.  Inputs come from the seeded generator
(``paper_2412_04634_gb300.scenes``) as plain numpy arrays; this module takes
any object with the ``NetConfig`` fields and never imports the CUDA path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class OCfg(ctypes.Structure):
    _fields_ = [
        ("pos_encoding", ctypes.c_int32), ("hash_levels", ctypes.c_int32),
        ("feats_per_level", ctypes.c_int32), ("log2_table", ctypes.c_int32),
        ("base_res", ctypes.c_int32), ("freq_octaves", ctypes.c_int32),
        ("width", ctypes.c_int32), ("hidden_layers", ctypes.c_int32),
        ("input_encoding", ctypes.c_int32), ("output", ctypes.c_int32),
        ("growth", ctypes.c_double), ("z_clamp", ctypes.c_double),
        ("loss_eps", ctypes.c_double),
    ]


class OFrame(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
        ("n_cache", ctypes.c_uint32), ("n_resid", ctypes.c_uint32),
        ("max_depth", ctypes.c_uint32), ("frame", ctypes.c_uint32),
        ("seed", ctypes.c_uint64), ("cache_mode", ctypes.c_uint32),
        ("light_mode", ctypes.c_uint32), ("estimator", ctypes.c_uint32), ("n_cache2", ctypes.c_uint32),
        ("n_cache3", ctypes.c_uint32), ("cache_const", ctypes.c_double * 3),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        u32, u64, i32, f64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_u01.argtypes = [u32]
        L.orc_u01.restype = ctypes.c_float
        L.orc_param_count.argtypes = [P]
        L.orc_param_count.restype = u64
        L.orc_hash_level.argtypes = [P, i32, P, P, P]
        L.orc_encode.argtypes = [P, P, P, P, P]
        L.orc_mlp.argtypes = [P, P, P, P]
        L.orc_sh_basis.argtypes = [P, P]
        L.orc_one_blob.argtypes = [f64, i32, P]
        L.orc_query.argtypes = [P, P, P, P, u64, P]
        L.orc_estimate_pixels.argtypes = [P, P, P, P, P, u64, P, P, P, P, P, P, P]
        L.orc_gen_train.argtypes = [P, u32, u32, u64, u32, u64, u32, u32, u32, P, P, P, P]
        L.orc_env_texel.argtypes = [u32, P]
        L.orc_env_texel.restype = u32
        L.orc_nee_sample.argtypes = [P, P, u32, u32, u32, u32, u32, u32, P]
        L.orc_nee_sample.restype = u32
        L.orc_bsdf_eval.argtypes = [P, P, P, P]
        L.orc_bth_path.argtypes = [P, P, u32, P, P, P, P]
        L.orc_bth_path.restype = u32
        L.orc_sampler_pdf32.argtypes = [P, P]
        L.orc_sampler_pdf32.restype = ctypes.c_float
        L.orc_train_loss_grad.argtypes = [P, P, P, P, P, u64, P, P]
        L.orc_train_loss_grad.restype = f64
        L.orc_train_loss_grad_abs.argtypes = [P, P, P, P, P, u64, P]
        L.orc_train_loss_grad_abs.restype = f64
        L.orc_query_grad.argtypes = [P, P, P, P, P, u64, P]
        L.orc_query_grad.restype = f64
        L.orc_adam_step.argtypes = [u64, P, P, P, P, u32, f64, f64, f64, f64]
        L.orc_mrse.argtypes = [P, P, u64, f64]
        L.orc_mrse.restype = f64
        L.orc_trace.argtypes = [P, P, P, P]
        L.orc_trace.restype = ctypes.c_int
        L.orc_sample_bsdf.argtypes = [P, u32, u32, u32, u32, u32, P, P, P, P, P]
        L.orc_onb.argtypes = [P, P, P]
        L.orc_trace_path.argtypes = [P, P, P, u32, u32, u32, u32, u32, P]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def ocfg(cfg) -> OCfg:
    return OCfg(cfg.pos_encoding, cfg.hash_levels, cfg.feats_per_level, cfg.log2_table,
                cfg.base_res, cfg.freq_octaves, cfg.width, cfg.hidden_layers,
                int(getattr(cfg, "input_encoding", 0)), int(getattr(cfg, "output", 0)), float(cfg.growth), float(cfg.z_clamp), float(cfg.loss_eps))


def oframe(width, height, n_cache, n_resid, max_depth, frame, seed, cache_mode=0,
           cache_const=(0.0, 0.0, 0.0), light_mode=0, estimator=0, n_cache2=0, n_cache3=0) -> OFrame:
    f = OFrame(width, height, n_cache, n_resid, max_depth, frame, seed, cache_mode, light_mode, estimator, n_cache2,
               n_cache3)
    for k in range(3):
        f.cache_const[k] = float(cache_const[k])
    return f


def num_threads() -> int:
    return lib().orc_num_threads()


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def u01(x: int) -> float:
    return float(lib().orc_u01(int(x)))


def param_count(cfg) -> int:
    c = ocfg(cfg)
    return int(lib().orc_param_count(ctypes.byref(c)))


def _params64(params) -> np.ndarray:
    return np.ascontiguousarray(params, np.float64)


def hash_level(cfg, level: int, x):
    c = ocfg(cfg)
    xf = np.ascontiguousarray(x, np.float32)
    idx = np.zeros(8, np.uint32)
    w = np.zeros(8, np.float64)
    lib().orc_hash_level(ctypes.byref(c), level, _ptr(xf), _ptr(idx), _ptr(w))
    return idx, w


def encode(cfg, params, rec, w) -> np.ndarray:
    c = ocfg(cfg)
    p = _params64(params)
    r = np.ascontiguousarray(rec)
    wf = np.ascontiguousarray(w, np.float32)
    e = np.zeros(cfg.n_inputs, np.float64)
    lib().orc_encode(ctypes.byref(c), _ptr(p), _ptr(r), _ptr(wf), _ptr(e))
    return e


def sh_basis(w) -> np.ndarray:
    """The 25 real spherical harmonics (l <= 4, index l*l + l + m) of w."""
    wf = np.ascontiguousarray(w, np.float32)
    e = np.zeros(25, np.float64)
    lib().orc_sh_basis(_ptr(wf), _ptr(e))
    return e


def one_blob(s: float, k: int = 4) -> np.ndarray:
    e = np.zeros(k, np.float64)
    lib().orc_one_blob(float(s), int(k), _ptr(e))
    return e


def mlp(cfg, params, e) -> np.ndarray:
    c = ocfg(cfg)
    p = _params64(params)
    ev = np.ascontiguousarray(e, np.float64)
    z = np.zeros(3, np.float64)
    lib().orc_mlp(ctypes.byref(c), _ptr(p), _ptr(ev), _ptr(z))
    return z


def query(cfg, params, recs, dirs) -> np.ndarray:
    c = ocfg(cfg)
    p = _params64(params)
    r = np.ascontiguousarray(recs)
    d = np.ascontiguousarray(dirs, np.float32)
    n = r.shape[0]
    out = np.zeros((n, 3), np.float64)
    lib().orc_query(ctypes.byref(c), _ptr(p), _ptr(r), _ptr(d), n, _ptr(out))
    return out


def estimate(cfg, params, scene_blob, frame: OFrame, pixels=None, rows=False):
    """Two-level estimate of the listed pixels (all when None).
    Returns dict(pixel, lc, lr (n,3) f64; sig (n,2) u64; count (n,) u32;
    lr_abs (n,3) f64, the sum of the absolute values of L_r's terms; with
    rows=True also row_n (n, N+M, 3) f64, the cache value of each row)."""
    c = ocfg(cfg)
    p = _params64(params) if params is not None else np.zeros(1, np.float64)
    blob = np.ascontiguousarray(scene_blob, np.uint8)
    if pixels is None:
        n = frame.width * frame.height
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(pixels, np.uint32)
        n = pix.shape[0]
        pix_ptr = _ptr(pix)
    out = np.zeros((n, 3), np.float64)
    lc = np.zeros((n, 3), np.float64)
    lr = np.zeros((n, 3), np.float64)
    sig = np.zeros((n, 2), np.uint64)
    cnt = np.zeros(n, np.uint32)
    row_n = np.zeros((n, frame.n_cache + frame.n_resid, 3), np.float64) if rows else None
    lr_abs = np.zeros((n, 3), np.float64)
    lib().orc_estimate_pixels(ctypes.byref(c), _ptr(p), _ptr(blob), ctypes.byref(frame), pix_ptr, n,
                              _ptr(out), _ptr(lc), _ptr(lr), _ptr(sig), _ptr(cnt),
                              None if row_n is None else _ptr(row_n), _ptr(lr_abs))
    res = dict(pixel=out, lc=lc, lr=lr, sig=sig, count=cnt, lr_abs=lr_abs)
    if rows:
        res["row_n"] = row_n
    return res


def bth_path(scene_blob, frame: OFrame, pix: int, record_dtype):
    """The biased estimator's camera path of one pixel: (stopping vertex or
    0, its record, throughput, collected radiance, path signature)."""
    blob = np.ascontiguousarray(scene_blob, np.uint8)
    rec = np.zeros(1, record_dtype)
    beta = np.zeros(3, np.float64)
    le = np.zeros(3, np.float64)
    sig = np.zeros(1, np.uint64)
    at = lib().orc_bth_path(_ptr(blob), ctypes.byref(frame), int(pix), _ptr(rec), _ptr(beta), _ptr(le), _ptr(sig))
    return int(at), rec, beta, le, int(sig[0])


def sampler_pdf32(rec, wi) -> float:
    r = np.ascontiguousarray(rec)
    w = np.ascontiguousarray(wi, np.float32)
    return float(lib().orc_sampler_pdf32(_ptr(r), _ptr(w)))


def gen_train(scene_blob, width, height, T, frame, seed, max_depth, record_dtype, light_mode=0, visibility=0):
    blob = np.ascontiguousarray(scene_blob, np.uint8)
    recs = np.zeros(T, record_dtype)
    dirs = np.zeros((T, 3), np.float32)
    tg = np.zeros((T, 3), np.float64)
    sig = np.zeros(T, np.uint64)
    lib().orc_gen_train(_ptr(blob), width, height, T, frame, seed, max_depth, light_mode, int(visibility),
                        _ptr(recs), _ptr(dirs), _ptr(tg), _ptr(sig))
    return recs, dirs, tg, sig


def env_texel(size: int, d) -> int:
    dd = np.ascontiguousarray(d, np.float32)
    return int(lib().orc_env_texel(int(size), _ptr(dd)))


def nee_sample(scene_blob, rec, n_b, key, ctr013):
    """One light sample at a record (light mode 1): (contribution f64 (3,), decision word)."""
    blob = np.ascontiguousarray(scene_blob, np.uint8)
    r = np.ascontiguousarray(rec)
    out = np.zeros(3, np.float64)
    word = lib().orc_nee_sample(_ptr(blob), _ptr(r), n_b, key[0], key[1], ctr013[0], ctr013[1], ctr013[2],
                                _ptr(out))
    return out, int(word)


def bsdf_eval(rec, wi):
    """(f_r cos, sampling density) of the record's material for direction wi."""
    r = np.ascontiguousarray(rec)
    w = np.ascontiguousarray(wi, np.float32)
    fc = np.zeros(3, np.float64)
    pdf = np.zeros(1, np.float64)
    lib().orc_bsdf_eval(_ptr(r), _ptr(w), _ptr(fc), _ptr(pdf))
    return fc, float(pdf[0])


def loss_grad(cfg, params, recs, dirs, targets, den_fixed=None):
    """Relative-L2 loss and its stop-gradient training gradient.  With
    ``den_fixed`` (n, 3) the denominators are frozen at those values."""
    c = ocfg(cfg)
    p = _params64(params)
    r = np.ascontiguousarray(recs)
    d = np.ascontiguousarray(dirs, np.float32)
    t = np.ascontiguousarray(targets, np.float64)
    g = np.zeros(p.shape[0], np.float64)
    den = None if den_fixed is None else np.ascontiguousarray(den_fixed, np.float64)
    loss = lib().orc_train_loss_grad(ctypes.byref(c), _ptr(p), _ptr(r), _ptr(d), _ptr(t), r.shape[0],
                                     None if den is None else _ptr(den), _ptr(g))
    return float(loss), g


def loss_grad_abs(cfg, params, recs, dirs, targets):
    """loss_grad with the hash-table part replaced, per entry, by the sum of
    the absolute values of the records' contributions to it."""
    c = ocfg(cfg)
    p = _params64(params)
    r = np.ascontiguousarray(recs)
    d = np.ascontiguousarray(dirs, np.float32)
    t = np.ascontiguousarray(targets, np.float64)
    g = np.zeros(p.shape[0], np.float64)
    loss = lib().orc_train_loss_grad_abs(ctypes.byref(c), _ptr(p), _ptr(r), _ptr(d), _ptr(t), r.shape[0], _ptr(g))
    return float(loss), g


def query_grad(cfg, params, recs, dirs, gout):
    """Vector-Jacobian product of the bare cache query: returns
    (sum gout * n, d(sum gout * n)/dparams) over every record."""
    c = ocfg(cfg)
    p = _params64(params)
    r = np.ascontiguousarray(recs)
    d = np.ascontiguousarray(dirs, np.float32)
    go = np.ascontiguousarray(gout, np.float64)
    g = np.zeros(p.shape[0], np.float64)
    val = lib().orc_query_grad(ctypes.byref(c), _ptr(p), _ptr(r), _ptr(d), _ptr(go), r.shape[0], _ptr(g))
    return float(val), g


def adam_step(params, m, v, g, step, lr, beta1, beta2, eps):
    """In place on float64 arrays params, m, v."""
    for a in (params, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    gg = np.ascontiguousarray(g, np.float64)
    lib().orc_adam_step(params.shape[0], _ptr(params), _ptr(m), _ptr(v), _ptr(gg), step, lr, beta1, beta2, eps)


def mrse(img, ref, eps=1e-2) -> float:
    a = np.ascontiguousarray(img, np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(ref, np.float64).reshape(-1, 3)
    return float(lib().orc_mrse(_ptr(a), _ptr(b), a.shape[0], eps))


def trace(scene_blob, o, d):
    blob = np.ascontiguousarray(scene_blob, np.uint8)
    of = np.ascontiguousarray(o, np.float32)
    df = np.ascontiguousarray(d, np.float32)
    t = np.zeros(1, np.float32)
    prim = lib().orc_trace(_ptr(blob), _ptr(of), _ptr(df), _ptr(t))
    return prim, float(t[0])


def sample_bsdf(rec, key, ctr013):
    r = np.ascontiguousarray(rec)
    wi = np.zeros(3, np.float32)
    w = np.zeros(3, np.float64)
    valid = np.zeros(1, np.int32)
    rej = np.zeros(1, np.uint32)
    lobe = np.zeros(1, np.uint32)
    lib().orc_sample_bsdf(_ptr(r), key[0], key[1], ctr013[0], ctr013[1], ctr013[2],
                          _ptr(wi), _ptr(w), _ptr(valid), _ptr(rej), _ptr(lobe))
    return wi, w, bool(valid[0]), int(rej[0]), int(lobe[0])


def onb(n):
    nf = np.ascontiguousarray(n, np.float32)
    t = np.zeros(3, np.float32)
    b = np.zeros(3, np.float32)
    lib().orc_onb(_ptr(nf), _ptr(t), _ptr(b))
    return t, b


def trace_path(scene_blob, o, d, key, c0, c1, max_depth):
    blob = np.ascontiguousarray(scene_blob, np.uint8)
    of = np.ascontiguousarray(o, np.float32)
    df = np.ascontiguousarray(d, np.float32)
    L = np.zeros(3, np.float64)
    lib().orc_trace_path(_ptr(blob), _ptr(of), _ptr(df), key[0], key[1], c0, c1, max_depth, _ptr(L))
    return L
