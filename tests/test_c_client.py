"""The C ABI from a plain C program (compiled with the host C compiler and
linked against the library): the header is valid C, and without a GPU every
call returns an error code instead of aborting."""
import os
import shutil
import subprocess

import pytest

import paper_1902_07554_gb300 as gdt

HERE = os.path.dirname(os.path.abspath(__file__))
INC = os.path.join(os.path.dirname(HERE), "include")


def test_c_client_links_and_fails_cleanly(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lib = gdt._build.build()
    libdir = os.path.dirname(lib)
    name = os.path.basename(lib)[3:-3]                 # libgb300dt.so -> gb300dt
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    exe = tmp_path / "c_client"
    subprocess.run([cc, "-std=c99", "-I", INC, os.path.join(HERE, "native", "c_client.c"), "-o", str(exe),
                    "-L", libdir, f"-l{name}", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cuda_lib}"], check=True)
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join([libdir, cuda_lib, env.get("LD_LIBRARY_PATH", "")])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0 and r.stdout.strip() in ("ok", "ok gpu"), r.stdout + r.stderr
