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


@pytest.mark.parametrize("cname,pyname", [("dt_config", "Config"), ("dt_stats", "Stats"),
                                          ("dt_validation", "Validation"), ("dt_kernel_profile", "KernelProfile"),
                                          ("dt_stream_info", "StreamInfo")])
def test_binding_structs_match_the_header(tmp_path, cname, pyname):
    """The ctypes mirrors have the header's field names, offsets and size
    (compiled from include/dt.h with the host C compiler)."""
    import os
    cls = getattr(gdt, pyname)
    fields = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dt.h"', 'int main(void) {',
             f'  printf("%zu\\n", sizeof({cname}));']
    lines += [f'  printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in fields]
