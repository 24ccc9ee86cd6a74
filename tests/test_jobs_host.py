"""Host logic of the asynchronous jobs behind dt_submit / dt_poll: the job
executor (csrc/jobs.h) compiled with the host C++ compiler against a
stand-in job function -- submission order, ids, results and error codes,
release rules, destruction with jobs queued, concurrent submitters.  No GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1902_07554_gb300", "csrc")


def test_job_queue_host_checks(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "job_queue_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "native", "job_queue_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
