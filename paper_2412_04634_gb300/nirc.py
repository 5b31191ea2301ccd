"""Thin ctypes binding of libnirc.so (include/nirc.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch CUDA tensors for device buffers (passed as raw pointers) and a torch
stream (defaults to the current stream).  All arithmetic runs in the
library's CUDA kernels; importing this module loads the library and raises
if it has not been built (``python -m paper_2412_04634_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnirc.so")

NIRC_OK, NIRC_ERR_INVALID, NIRC_ERR_OOM, NIRC_ERR_BUDGET, NIRC_ERR_CUDA, NIRC_ERR_TIMEOUT, NIRC_ERR_UNSUPPORTED = range(7)
NIRC_FP32_SIMT, NIRC_FP16_TC, NIRC_BF16_TC, NIRC_FP8_E4M3_TC = range(4)
NIRC_INPUT_FREQ, NIRC_INPUT_SH = range(2)
NIRC_EST_TWO_LEVEL, NIRC_EST_BIASED_BTH, NIRC_EST_MULTI_VERTEX = range(3)
NIRC_OUT_RADIANCE, NIRC_OUT_VISIBILITY = range(2)
NIRC_PHASE_ALL, NIRC_PHASE_TRACE, NIRC_PHASE_CACHE = range(3)
NIRC_MAX_PRIMS = 1024


class NircError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[nirc status {status}] {msg}")
        self.status = status


class nirc_config(ctypes.Structure):
    _fields_ = [
        ("pos_encoding", ctypes.c_uint32), ("hash_levels", ctypes.c_uint32),
        ("feats_per_level", ctypes.c_uint32), ("log2_table", ctypes.c_uint32),
        ("base_res", ctypes.c_uint32), ("growth", ctypes.c_float),
        ("freq_octaves", ctypes.c_uint32), ("width", ctypes.c_uint32),
        ("hidden_layers", ctypes.c_uint32), ("precision", ctypes.c_uint32),
        ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
        ("adam_eps", ctypes.c_float), ("loss_eps", ctypes.c_float), ("z_clamp", ctypes.c_float),
        ("input_encoding", ctypes.c_uint32), ("output", ctypes.c_uint32),
    ]


class nirc_frame_desc(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
        ("n_cache", ctypes.c_uint32), ("n_resid", ctypes.c_uint32),
        ("max_depth", ctypes.c_uint32), ("frame", ctypes.c_uint32),
        ("seed", ctypes.c_uint64), ("n_prims", ctypes.c_uint32),
        ("cache_mode", ctypes.c_uint32), ("cache_const", ctypes.c_float * 3),
        ("light_mode", ctypes.c_uint32), ("estimator", ctypes.c_uint32), ("n_cache2", ctypes.c_uint32),
        ("n_cache3", ctypes.c_uint32), ("phase", ctypes.c_uint32),
    ]


class nirc_frame_aux(ctypes.Structure):
    _fields_ = [("lc", ctypes.c_void_p), ("lr", ctypes.c_void_p),
                ("sig", ctypes.c_void_p), ("count", ctypes.c_void_p), ("row_n", ctypes.c_void_p),
                ("rays", ctypes.c_void_p)]


K_CLASSES = ["path_trace", "cache", "train_records", "train_fwd", "train_bwd", "train_gradw", "adam", "query"]


class nirc_timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_uint64 * 8)]


class nirc_server_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32), ("max_batches", ctypes.c_uint32),
                ("train_samples", ctypes.c_uint32), ("use_graphs", ctypes.c_uint32)]


class nirc_request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("scene", ctypes.c_uint32), ("width", ctypes.c_uint32),
                ("height", ctypes.c_uint32), ("n_cache", ctypes.c_uint32), ("n_resid", ctypes.c_uint32),
                ("max_depth", ctypes.c_uint32), ("frame", ctypes.c_uint32), ("light_mode", ctypes.c_uint32)]


class nirc_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_uint32),
                ("d_image", ctypes.c_void_p), ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class nirc_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "batches",
                                                 "graph_instantiations", "graph_updates", "arena_bytes",
                                                 "arena_peak_bytes", "resident_bytes")] + \
               [(n, ctypes.c_uint32) for n in ("queued", "in_flight", "max_batch_seen", "pad")] + \
               [("frame_launches", ctypes.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2412_04634_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    st = ctypes.c_int
    sig = {
        "nirc_param_count": ([P], u64),
        "nirc_create": ([P, P], st),
        "nirc_destroy": ([P], st),
        "nirc_set_params": ([P, P, i32, P], st),
        "nirc_load_params": ([P, P, i32, P], st),
        "nirc_set_train_mode": ([P, i32, u64], st),
        "nirc_set_deterministic": ([P, i32], st),
        "nirc_set_train_precision": ([P, u32], st),
        "nirc_query_bwd": ([P, P, P, P, u64, P, P, P], st),
        "nirc_get_params": ([P, P, i32, P], st),
        "nirc_get_grads": ([P, P, i32, P], st),
        "nirc_set_precision": ([P, u32], st),
        "nirc_state_bytes": ([P], u64),
        "nirc_save_state": ([P, P, u64, P], st),
        "nirc_load_state": ([P, P, u64, P], st),
        "nirc_sync": ([P, P], st),
        "nirc_query": ([P, P, P, u64, P, P], st),
        "nirc_estimate_frame": ([P, P, P, P, P, P], st),
        "nirc_estimate_frame_noalloc": ([P, P, P, P, P, P], st),
        "nirc_gen_train": ([P, P, u32, u32, u32, u64, u32, u64, u32, u32, P, P, P, P], st),
        "nirc_train_step": ([P, P, P, P, u64, P, P], st),
        "nirc_frame_mrse": ([P, P, u64, ctypes.c_float, P, P], st),
        "nirc_timing_enable": ([P, i32], st),
        "nirc_timing_read": ([P, P], st),
        "nirc_last_error": ([], ctypes.c_char_p),
        "nirc_server_create": ([P, P], st),
        "nirc_server_add_scene": ([P, P, P, u32, u64, u32, u64, P], st),
        "nirc_server_submit": ([P, P], st),
        "nirc_server_poll": ([P, P, u32, P, i32], st),
        "nirc_server_release": ([P, u64], st),
        "nirc_server_copy_image": ([P, u64, P, P], st),
        "nirc_server_drain": ([P], st),
        "nirc_server_stats_read": ([P, P], st),
        "nirc_server_clock": ([P], ctypes.c_double),
        "nirc_server_destroy": ([P], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


_lib = _load()


def lib():
    return _lib


def exported_symbols():
    return [n for n in dir(_lib) if n.startswith("nirc_")]


def _check(status: int):
    if status != NIRC_OK:
        raise NircError(status, _lib.nirc_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous(), "tensor must be contiguous"
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_config(cfg: scenes.NetConfig, precision: int = NIRC_FP32_SIMT) -> nirc_config:
    return nirc_config(cfg.pos_encoding, cfg.hash_levels, cfg.feats_per_level, cfg.log2_table, cfg.base_res,
                       cfg.growth, cfg.freq_octaves, cfg.width, cfg.hidden_layers, precision,
                       cfg.lr, cfg.beta1, cfg.beta2, cfg.adam_eps, cfg.loss_eps, cfg.z_clamp,
                       getattr(cfg, "input_encoding", 0), getattr(cfg, "output", 0))


def frame_desc(width, height, n_cache, n_resid, max_depth, frame, seed, n_prims, cache_mode=0,
               cache_const=(0.0, 0.0, 0.0), light_mode=0, estimator=0, n_cache2=0, n_cache3=0,
               phase=0) -> nirc_frame_desc:
    d = nirc_frame_desc(width, height, n_cache, n_resid, max_depth, frame, seed, n_prims, cache_mode)
    for k in range(3):
        d.cache_const[k] = float(cache_const[k])
    d.light_mode = light_mode
    d.estimator = estimator
    d.n_cache2 = n_cache2
    d.n_cache3 = n_cache3
    d.phase = phase
    return d


# --- entry points (same names as the C ABI) ----------------------------------

def nirc_param_count(cfg: nirc_config) -> int:
    return int(_lib.nirc_param_count(ctypes.byref(cfg)))


def nirc_create(cfg: nirc_config):
    h = ctypes.c_void_p()
    _check(_lib.nirc_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def nirc_destroy(h):
    _check(_lib.nirc_destroy(h))


def nirc_set_params(h, params: torch.Tensor, stream=None):
    on_dev = 1 if params.is_cuda else 0
    p = params.contiguous()
    _check(_lib.nirc_set_params(h, _ptr(p), on_dev, _stream(stream)))


def nirc_load_params(h, params: torch.Tensor, stream=None):
    on_dev = 1 if params.is_cuda else 0
    p = params.contiguous()
    _check(_lib.nirc_load_params(h, _ptr(p), on_dev, _stream(stream)))


def nirc_set_train_mode(h, store_activations: bool = True, recompute_chunk: int = 1 << 15):
    _check(_lib.nirc_set_train_mode(h, 1 if store_activations else 0, recompute_chunk))


def nirc_set_train_precision(h, precision: int):
    _check(_lib.nirc_set_train_precision(h, precision))


def nirc_set_deterministic(h, on: bool = True):
    _check(_lib.nirc_set_deterministic(h, 1 if on else 0))


def nirc_query_bwd(h, records: torch.Tensor, dirs: torch.Tensor, grad_out: torch.Tensor,
                   grad_params: torch.Tensor | None = None, value: torch.Tensor | None = None, stream=None):
    n = dirs.shape[0]
    _check(_lib.nirc_query_bwd(h, _ptr(records), _ptr(dirs), _ptr(grad_out), n, _ptr(grad_params), _ptr(value),
                               _stream(stream)))


def nirc_get_params(h, out: torch.Tensor, stream=None):
    _check(_lib.nirc_get_params(h, _ptr(out), 1 if out.is_cuda else 0, _stream(stream)))


def nirc_get_grads(h, out: torch.Tensor, stream=None):
    _check(_lib.nirc_get_grads(h, _ptr(out), 1 if out.is_cuda else 0, _stream(stream)))


def nirc_state_bytes(h) -> int:
    return int(_lib.nirc_state_bytes(h))


def nirc_save_state(h, stream=None) -> bytearray:
    """The cache's weights, Adam moments, step and configuration as bytes."""
    n = nirc_state_bytes(h)
    buf = (ctypes.c_char * n)()
    _check(_lib.nirc_save_state(h, buf, n, _stream(stream)))
    return bytearray(buf)


def nirc_load_state(h, state: bytes, stream=None):
    buf = (ctypes.c_char * len(state)).from_buffer_copy(bytes(state))
    _check(_lib.nirc_load_state(h, buf, len(state), _stream(stream)))


def nirc_set_precision(h, precision: int):
    _check(_lib.nirc_set_precision(h, precision))


def nirc_sync(h, stream=None):
    _check(_lib.nirc_sync(h, _stream(stream)))


def nirc_query(h, records: torch.Tensor, dirs: torch.Tensor, out: torch.Tensor, stream=None):
    n = dirs.shape[0]
    _check(_lib.nirc_query(h, _ptr(records), _ptr(dirs), n, _ptr(out), _stream(stream)))


def nirc_estimate_frame(h, scene: torch.Tensor, desc: nirc_frame_desc, out_rgba: torch.Tensor,
                        lc=None, lr=None, sig=None, count=None, row_n=None, rays=None, stream=None):
    aux = nirc_frame_aux(_ptr(lc), _ptr(lr), _ptr(sig), _ptr(count), _ptr(row_n), _ptr(rays))
    use_aux = any(x is not None for x in (lc, lr, sig, count, row_n, rays))
    _check(_lib.nirc_estimate_frame(h, _ptr(scene), ctypes.byref(desc), _ptr(out_rgba),
                                    ctypes.byref(aux) if use_aux else None, _stream(stream)))


def nirc_estimate_frame_noalloc(h, scene: torch.Tensor, desc: nirc_frame_desc, out_rgba: torch.Tensor,
                                lc=None, lr=None, sig=None, count=None, row_n=None, rays=None, stream=None):
    """nirc_estimate_frame on the library's fixed scratch area (no device
    allocation during the call).  Frames must fit its 4 MiB: W*H*(96+32*M)
    bytes for the two-level estimator, W*H*112 for the biased (BTH) one,
    W*H*(96+288*M) for the multi-vertex one."""
    aux = nirc_frame_aux(_ptr(lc), _ptr(lr), _ptr(sig), _ptr(count), _ptr(row_n), _ptr(rays))
    use_aux = any(x is not None for x in (lc, lr, sig, count, row_n, rays))
    _check(_lib.nirc_estimate_frame_noalloc(h, _ptr(scene), ctypes.byref(desc), _ptr(out_rgba),
                                            ctypes.byref(aux) if use_aux else None, _stream(stream)))


def nirc_gen_train(h, scene: torch.Tensor, n_prims, width, height, T, frame, seed, max_depth,
                   records: torch.Tensor, dirs: torch.Tensor, targets: torch.Tensor, stream=None, light_mode=0):
    _check(_lib.nirc_gen_train(h, _ptr(scene), n_prims, width, height, T, frame, seed, max_depth, light_mode,
                               _ptr(records), _ptr(dirs), _ptr(targets), _stream(stream)))


def nirc_train_step(h, records: torch.Tensor, dirs: torch.Tensor, targets: torch.Tensor, loss=None, stream=None):
    n = dirs.shape[0]
    _check(_lib.nirc_train_step(h, _ptr(records), _ptr(dirs), _ptr(targets), n, _ptr(loss), _stream(stream)))


def nirc_frame_mrse(img: torch.Tensor, ref: torch.Tensor, out: torch.Tensor, eps: float = 1e-2, stream=None):
    n = img.numel() // 4
    _check(_lib.nirc_frame_mrse(_ptr(img), _ptr(ref), n, eps, _ptr(out), _stream(stream)))


def nirc_timing_enable(h, enable: bool = True):
    _check(_lib.nirc_timing_enable(h, 1 if enable else 0))


def nirc_timing_read(h) -> dict:
    """{class: (total ms, kernels launched)} since the last enable."""
    t = nirc_timing()
    _check(_lib.nirc_timing_read(h, ctypes.byref(t)))
    return {name: (t.ms[i], int(t.launches[i])) for i, name in enumerate(K_CLASSES)}


# --- convenience ----------------------------------------------------------------

def records_to_tensor(recs, device="cuda") -> torch.Tensor:
    """Structured numpy records (scenes.RECORD_DTYPE) -> (n, 16) float32 device tensor (64 B rows)."""
    import numpy as np
    raw = np.ascontiguousarray(recs).view(np.float32).reshape(-1, 16)
    return torch.from_numpy(raw.copy()).to(device)


def records_from_tensor(t: torch.Tensor):
    import numpy as np
    raw = t.detach().cpu().contiguous().numpy().astype(np.float32, copy=False)
    return raw.view(scenes.RECORD_DTYPE).reshape(-1)


def scene_to_tensor(scene: scenes.Scene, device="cuda") -> torch.Tensor:
    """Scene blob as a 16-byte aligned uint8 device tensor."""
    blob = scene.blob()
    return torch.from_numpy(blob.copy()).to(device)


class Cache:
    """Owning wrapper of a nirc_handle."""

    def __init__(self, cfg: scenes.NetConfig, precision: int = NIRC_FP32_SIMT):
        self.cfg = cfg
        self.ccfg = make_config(cfg, precision)
        self.h = nirc_create(self.ccfg)
        self.n_params = nirc_param_count(self.ccfg)

    def close(self):
        if self.h is not None:
            nirc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params, stream=None):
        t = params if isinstance(params, torch.Tensor) else torch.from_numpy(params)
        assert t.numel() == self.n_params
        nirc_set_params(self.h, t.float().contiguous(), stream)

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32)
        nirc_get_params(self.h, out)
        return out

    def get_grads(self) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32)
        nirc_get_grads(self.h, out)
        return out


class NircQuery(torch.autograd.Function):
    """Differentiable cache query: ``NircQuery.apply(params, records, dirs, cache)``
    returns n = exp(min(MLP(enc(x, w, n)), z_clamp)) per row, (n, 3) float32.

    ``params`` is the flat FP32 parameter vector (nirc_param_count layout, a
    CUDA tensor); the forward loads it into the handle (nirc_load_params,
    the handle's Adam state is kept) and calls nirc_query; the backward
    reloads the same parameters and calls nirc_query_bwd.  Records and directions are not differentiated (they are
    samples of the estimator, not parameters)."""

    @staticmethod
    def forward(ctx, params, records, dirs, cache):
        assert params.is_cuda and params.dtype == torch.float32 and params.numel() == cache.n_params
        records = records.contiguous()
        dirs = dirs.contiguous().float()
        nirc_load_params(cache.h, params.detach().contiguous())
        out = torch.empty(dirs.shape[0], 3, device=dirs.device, dtype=torch.float32)
        nirc_query(cache.h, records, dirs, out)
        ctx.cache = cache
        ctx.save_for_backward(params.detach(), records, dirs)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        params, records, dirs = ctx.saved_tensors
        cache = ctx.cache
        # the handle may have been loaded with other weights since the forward
        nirc_load_params(cache.h, params.contiguous())
        g = torch.empty(cache.n_params, device=dirs.device, dtype=torch.float32)
        nirc_query_bwd(cache.h, records, dirs, grad_out.contiguous().float(), g)
        return g, None, None, None


# --- frame-request server (include/nirc_serve.h) -------------------------------

def nirc_server_create(cfg: nirc_server_config):
    h = ctypes.c_void_p()
    _check(_lib.nirc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def nirc_server_add_scene(srv, cache_h, frames: torch.Tensor, n_frames: int, frame_stride: int, n_prims: int,
                          seed: int) -> int:
    idx = ctypes.c_uint32()
    _check(_lib.nirc_server_add_scene(srv, cache_h, _ptr(frames), n_frames, frame_stride, n_prims, seed,
                                      ctypes.byref(idx)))
    return idx.value


def nirc_server_submit(srv, req: nirc_request):
    _check(_lib.nirc_server_submit(srv, ctypes.byref(req)))


def nirc_server_poll(srv, max_n: int = 64, wait: bool = False):
    buf = (nirc_completion * max(1, max_n))()
    n = ctypes.c_uint32()
    _check(_lib.nirc_server_poll(srv, buf, max_n, ctypes.byref(n), 1 if wait else 0))
    return [buf[i] for i in range(n.value)]


def nirc_server_copy_image(srv, rid: int, out: torch.Tensor, stream=None):
    _check(_lib.nirc_server_copy_image(srv, rid, _ptr(out), _stream(stream)))


def nirc_server_release(srv, rid: int):
    _check(_lib.nirc_server_release(srv, rid))


def nirc_server_drain(srv):
    _check(_lib.nirc_server_drain(srv))


def nirc_server_stats_read(srv) -> dict:
    st = nirc_server_stats()
    _check(_lib.nirc_server_stats_read(srv, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in nirc_server_stats._fields_ if n != "pad"}


def nirc_server_clock(srv) -> float:
    return float(_lib.nirc_server_clock(srv))


def nirc_server_destroy(srv):
    _check(_lib.nirc_server_destroy(srv))


class Server:
    """Owning wrapper of a nirc_server.  Scenes are (Cache, list of
    scenes.Scene key frames, seed); their blobs are uploaded into one device
    tensor per scene that the server reads for the scene's lifetime."""

    def __init__(self, budget_bytes: int, slots: int = 8, max_batches: int = 2, train_samples: int = 65536,
                 use_graphs: bool = True):
        self.h = nirc_server_create(nirc_server_config(budget_bytes, slots, max_batches, train_samples,
                                                       1 if use_graphs else 0))
        self._keep = []

    def add_scene(self, cache: "Cache", frames, seed: int) -> int:
        import numpy as np
        blobs = [f.blob() for f in frames]
        stride = (max(b.nbytes for b in blobs) + 15) // 16 * 16
        buf = np.zeros(stride * len(blobs), np.uint8)
        for k, b in enumerate(blobs):
            buf[k * stride:k * stride + b.nbytes] = b
        dev = torch.from_numpy(buf).cuda()
        self._keep.append((cache, dev))
        return nirc_server_add_scene(self.h, cache.h, dev, len(blobs), stride, frames[0].n_prims, seed)

    def submit(self, rid, scene, width, height, n_cache, n_resid, max_depth, frame, light_mode=0):
        nirc_server_submit(self.h, nirc_request(rid, scene, width, height, n_cache, n_resid, max_depth, frame,
                                                light_mode))

    def poll(self, wait=False, max_n=64):
        return nirc_server_poll(self.h, max_n, wait)

    def image(self, c: nirc_completion, width: int, height: int) -> torch.Tensor:
        """Copy a completed request's image (W*H x 4) into a new CUDA tensor."""
        out = torch.empty((width * height, 4), device="cuda")
        nirc_server_copy_image(self.h, c.id, out)
        return out

    def release(self, rid):
        nirc_server_release(self.h, rid)

    def drain(self):
        nirc_server_drain(self.h)

    def stats(self):
        return nirc_server_stats_read(self.h)

    def clock(self):
        return nirc_server_clock(self.h)

    def close(self):
        if self.h is not None:
            nirc_server_destroy(self.h)
            self.h = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
