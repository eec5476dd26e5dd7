"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/pnuc.h declares; record layouts agree with the header (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np

from paper_1309_7963_gb300 import pnuc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pnuc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pnuc_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = pnuc.load()
    names = declared_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), f"{name} declared in pnuc.h but not exported"


def test_record_layouts():
    assert pnuc.SECONDARY_DTYPE.itemsize == 32
    assert pnuc.RESIDUAL_DTYPE.itemsize == 64
    assert pnuc.SECONDARY_DTYPE.fields["T"][1] == 8
    assert pnuc.RESIDUAL_DTYPE.fields["Estar_cascade"][1] == 24
    assert C.sizeof(pnuc.pnuc_batch) == 56 and C.sizeof(pnuc.pnuc_output) == 40
    assert C.sizeof(pnuc.pnuc_tuning) == 20 and C.sizeof(pnuc.pnuc_config) == 20


def test_host_side_status_strings_without_gpu():
    lib = pnuc.load()
    assert lib.pnuc_status_string(0) == b"ok"
    assert lib.pnuc_status_string(3) == b"capacity exceeded"
    cfg = pnuc.pnuc_config()
    lib.pnuc_default_config(C.byref(cfg))
    assert cfg.max_steps == 100000 and cfg.max_attempts == 1000
    # argument checks happen before any CUDA call
    assert lib.pnuc_simulate(None, 0, 0, None, None, None) == 1
    assert lib.pnuc_create(None, None) == 1
    assert lib.pnuc_kernel_timing(None, 1) == 1
    assert lib.pnuc_kernel_times(None, None, None, None) == 1
    assert lib.pnuc_server_view(None, 1, None, None, None) == 1
    assert lib.pnuc_server_release(None, 1) == 1
    assert lib.pnuc_tally(None, None, None, 0, None, None, 0, None, None, None) == 1


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        return
    try:
        pnuc.Context(0)
    except RuntimeError as e:
        assert "no CPU fallback" in str(e)
    else:
        raise AssertionError("Context must fail loudly without a GPU")
