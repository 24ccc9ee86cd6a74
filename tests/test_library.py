"""The C ABI library builds for sm_103a, loads, and exports every entry
point include/dt.h declares.  No compute calls (no GPU needed)."""
import ctypes
import subprocess

import pytest

import paper_1902_07554_gb300 as gdt


def test_header_declares_the_boundary():
    names = gdt.declared_symbols()
    for required in ["dt_create", "dt_triangulate", "dt_get_simplices", "dt_destroy", "dt_get_stats",
                     "dt_last_error", "dt_eval_predicates", "dt_label_points", "dt_partition_graph"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = gdt._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in gdt.declared_symbols() if s not in exported]
    assert not missing, missing
    L = gdt.load_library()
    for s in gdt.declared_symbols():
        assert hasattr(L, s)


def test_config_default_and_bad_device():
    L = gdt.load_library()
    cfg = gdt.Config()
    assert L.dt_config_default(ctypes.byref(cfg)) == 0
    assert cfg.lp_rounds == 16 and abs(cfg.epsilon - 0.05) < 1e-15 and cfg.base_threshold == 2048
    ctx = ctypes.c_void_p()
    # device 4096 never exists: a clean error, no abort
    assert L.dt_create(ctypes.byref(ctx), 4096, None, None) == -1
    assert L.dt_last_error(None) == b"null context"
    assert L.dt_triangulate(None, None, 0, 2, 1, 0.0) == -1
