"""CPU checks of the C ABI: the library loads, exports every entry point that
include/gp.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest
import torch

from paper_2603_20611_b300 import binding as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"GP_API\s+[\w\s\*]+?\b(gp_\w+)\s*\(", txt))
    return names


def test_header_declares_the_binding_exports():
    decl = declared_functions()
    assert decl, "no GP_API declarations found"
    assert decl == set(b.EXPORTS), decl ^ set(b.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(b.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_bounds_checked_variant_exports_the_same_symbols():
    """The -DGP_CHECK build of the same sources: same ABI, and it says which
    build it is (the default one says 0)."""
    path = os.path.join(os.path.dirname(b.LIB_PATH), "libgaussianpile_check.so")
    assert os.path.exists(path), "build() makes the bounds-checked variant too"
    chk = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(chk, name), name
    assert chk.gp_check_enabled() == 1
    assert ctypes.CDLL(os.path.join(os.path.dirname(b.LIB_PATH), "libgaussianpile.so")).gp_check_enabled() == 0


def test_config_defaults():
    cfg = b.gp_config()
    assert b.lib.gp_config_default(ctypes.byref(cfg)) == b.GP_OK
    assert cfg.eps == pytest.approx(1e-6)
    assert cfg.tile == 16 and cfg.deterministic == 0 and cfg.exp_mode == b.GP_EXP_POLY
    assert b.lib.gp_config_default(None) == b.GP_ERR_ARG


def test_create_rejects_bad_config_and_null():
    h = ctypes.c_void_p()
    assert b.lib.gp_create(None, 0, None) == b.GP_ERR_ARG
    cfg = b.gp_config()
    b.lib.gp_config_default(ctypes.byref(cfg))
    cfg.tile = 12
    assert b.lib.gp_create(ctypes.byref(h), 0, ctypes.byref(cfg)) == b.GP_ERR_ARG
    b.lib.gp_config_default(ctypes.byref(cfg))
    cfg.eps = 0.0
    assert b.lib.gp_create(ctypes.byref(h), 0, ctypes.byref(cfg)) == b.GP_ERR_ARG
    b.lib.gp_config_default(ctypes.byref(cfg))
    cfg.bwd_px = 3
    assert b.lib.gp_create(ctypes.byref(h), 0, ctypes.byref(cfg)) == b.GP_ERR_ARG


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error():
    h = ctypes.c_void_p()
    assert b.lib.gp_create(ctypes.byref(h), 0, None) == b.GP_ERR_CUDA
    assert h.value is None


def test_null_context_calls_fail_cleanly():
    assert b.lib.gp_render_slices(None, None, None, 0, 1, 1, 1.0, 2, None, None) == b.GP_ERR_ARG
    assert b.lib.gp_destroy(None) == b.GP_ERR_ARG
    assert b.lib.gp_last_error(None) == b"no context"
