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
    assert C.sizeof(pnuc.pnuc_tuning) == 20 and C.sizeof(pnuc.pnuc_config) == 24


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
    assert lib.pnuc_tally_windows(None, 125, 0.0, 250.0, None, None, 4, None, 0, None, None) == 1


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


def test_python_mirrors_match_the_header(tmp_path):
    """Every struct of pnuc.h, compiled by the host C compiler: its size and each field's
    offset equal those of the binding's ctypes / numpy mirror."""
    import subprocess
    mirrors = {name: getattr(pnuc, name) for name in (
        "pnuc_config", "pnuc_batch", "pnuc_output", "pnuc_tuning", "pnuc_target_info", "pnuc_peaks",
        "pnuc_tally_spec", "pnuc_server_config", "pnuc_server_stats")}
    dtypes = {"pnuc_secondary": pnuc.SECONDARY_DTYPE, "pnuc_residual": pnuc.RESIDUAL_DTYPE,
              "pnuc_server_trace_entry": pnuc.TRACE_DTYPE}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pnuc.h"', "int main(void) {"]
    for name, cls in mirrors.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    for name, dt in dtypes.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f in dt.names:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    for name, cls in mirrors.items():
        assert got[(name, "sizeof")] == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
    for name, dt in dtypes.items():
        assert got[(name, "sizeof")] == dt.itemsize, name
        for f in dt.names:
            assert got[(name, f)] == dt.fields[f][1], (name, f)
