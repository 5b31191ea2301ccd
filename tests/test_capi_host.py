"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function nirc.h declares, sizes parameters like the
input generator, and rejects bad arguments with a status instead of
aborting (all of these return before any CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_2412_04634_gb300 import build as nbuild
from paper_2412_04634_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def N():
    nbuild.build()
    from paper_2412_04634_gb300 import nirc
    return nirc


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nirc_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(N):
    declared = _declared()
    assert {"nirc_create", "nirc_query", "nirc_estimate_frame", "nirc_train_step", "nirc_destroy"} <= declared
    lib = ctypes.CDLL(N.LIB_PATH)
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("cfg", [scenes.config_small(), scenes.config_1080p(), scenes.config_paper_1080p(),
                                 scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=8, log2_table=12,
                                                  hidden_layers=2),
                                 scenes.NetConfig(input_encoding=scenes.INPUT_SH, hidden_layers=2)])
def test_param_count_matches_layout(N, cfg):
    assert N.nirc_param_count(N.make_config(cfg)) == cfg.n_params


def test_bad_arguments_return_status(N):
    bad = N.make_config(scenes.NetConfig(width=32))
    h = ctypes.c_void_p()
    assert N.lib().nirc_create(ctypes.byref(bad), ctypes.byref(h)) == N.NIRC_ERR_UNSUPPORTED
    assert b"width" in N.lib().nirc_last_error()
    bad = N.make_config(scenes.NetConfig(hidden_layers=0))
    assert N.lib().nirc_create(ctypes.byref(bad), ctypes.byref(h)) == N.NIRC_ERR_UNSUPPORTED
    bad = N.make_config(scenes.NetConfig(pos_encoding=7))
    assert N.lib().nirc_create(ctypes.byref(bad), ctypes.byref(h)) == N.NIRC_ERR_INVALID
    bad = N.make_config(scenes.NetConfig(input_encoding=2))
    assert N.lib().nirc_create(ctypes.byref(bad), ctypes.byref(h)) == N.NIRC_ERR_INVALID
    assert b"input_encoding" in N.lib().nirc_last_error()
    # more than 16 hash levels
    bad = N.make_config(scenes.NetConfig(pos_encoding=scenes.POS_HASHGRID, hash_levels=24, input_encoding=1))
    assert N.lib().nirc_create(ctypes.byref(bad), ctypes.byref(h)) == N.NIRC_ERR_UNSUPPORTED
    assert N.lib().nirc_create(None, ctypes.byref(h)) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_query(None, None, None, 5, None, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_train_step(None, None, None, None, 5, None, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_frame_mrse(None, None, 5, ctypes.c_float(0.01), None, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_query_bwd(None, None, None, None, 5, None, None, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_load_params(None, None, 0, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_set_train_mode(None, 1, 0) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_set_train_precision(None, 1) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_state_bytes(None) == 0
    assert N.lib().nirc_save_state(None, None, 0, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_load_state(None, None, 0, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_server_create(None, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_server_submit(None, None) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_server_poll(None, None, 0, None, 0) == N.NIRC_ERR_INVALID
    assert N.lib().nirc_server_destroy(None) == N.NIRC_OK
    assert N.lib().nirc_destroy(None) == N.NIRC_OK
    assert N.nirc_param_count(N.make_config(scenes.NetConfig(width=48))) == 0


def test_server_config_rejected_without_device(N):
    """Bad server configurations are refused before any device call."""
    h = ctypes.c_void_p()
    for cfg in (N.nirc_server_config(1 << 10, 4, 1, 0, 1), N.nirc_server_config(1 << 30, 0, 1, 0, 1),
                N.nirc_server_config(1 << 30, 17, 1, 0, 1), N.nirc_server_config(1 << 30, 4, 5, 0, 1)):
        assert N.lib().nirc_server_create(ctypes.byref(cfg), ctypes.byref(h)) == N.NIRC_ERR_INVALID
        assert b"slots" in N.lib().nirc_last_error()


def test_struct_layouts(N):
    assert ctypes.sizeof(N.nirc_request) == 40
    assert ctypes.sizeof(N.nirc_completion) == 48
    assert ctypes.sizeof(N.nirc_server_config) == 24
    assert ctypes.sizeof(N.nirc_frame_desc) == 72
    assert ctypes.sizeof(N.nirc_config) == 72
    assert scenes.RECORD_DTYPE.itemsize == 64
    assert scenes.PRIM_DTYPE.itemsize == 96 and scenes.HEADER_DTYPE.itemsize == 96
