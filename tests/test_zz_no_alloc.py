"""The allocation-free sample selection, called through the C ABI.

dt_select_sample_noalloc exists for callers that cannot allocate device
memory (allocator callbacks, pools they do not own, capped or audited
processes, real-time paths): it keeps its scratch in a fixed file-scope
device array instead of allocating.  Here it must return exactly the sample
that the regular path (dt_triangulate, read back with dt_get_sample) draws,
on two calls in a row.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import pointsets

pytestmark = pytest.mark.gpu


def _noalloc(L, n, eta, seed):
    import torch
    out = torch.full((eta,), -1, dtype=torch.int32, device="cuda:0")
    torch.cuda.synchronize()
    rc = L.dt_select_sample_noalloc(0, None, n, eta, ctypes.c_uint64(seed), ctypes.c_void_p(out.data_ptr()))
    assert rc == 0
    return out.cpu().numpy()


def test_noalloc_sample_matches_regular_path_twice():
    from paper_1902_07554_gb300 import Triangulator, load_library
    L = load_library()
    P = pointsets.uniform(50_000, 3, 4)
    with Triangulator(0, base_threshold=16) as tri:
        for seed, frac in [(1, 0.01), (77, 0.004)]:
            tri.configure(seed=seed)
            tri.triangulate(P, k=4, sample_frac=frac, fetch=False)
            want = tri.sample()
            got = _noalloc(L, len(P), len(want), seed)
            assert np.array_equal(got, want), seed
    # two calls in a row with the same arguments agree (shared scratch is reset)
    a = _noalloc(L, 123_457, 999, 5)
    b = _noalloc(L, 123_457, 999, 5)
    assert np.array_equal(a, b) and np.all(np.diff(a) > 0)


def test_noalloc_rejects_bad_sizes():
    from paper_1902_07554_gb300 import load_library
    import torch
    L = load_library()
    out = torch.empty(8, dtype=torch.int32, device="cuda:0")
    ptr = ctypes.c_void_p(out.data_ptr())
    assert L.dt_select_sample_noalloc(0, None, 10, 11, ctypes.c_uint64(1), ptr) == -1
    assert L.dt_select_sample_noalloc(0, None, 1 << 31, 8, ctypes.c_uint64(1), ptr) == -1
    host = np.empty(8, dtype=np.int32)
    assert L.dt_select_sample_noalloc(0, None, 100, 8, ctypes.c_uint64(1), ctypes.c_void_p(host.ctypes.data)) == -1


def test_noalloc_rejects_memory_of_another_gpu():
    """An output buffer on a GPU other than the one named in the call is
    rejected before any kernel is launched (it would be a peer write)."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    from paper_1902_07554_gb300 import load_library
    L = load_library()
    out = torch.full((8,), -1, dtype=torch.int32, device="cuda:1")
    torch.cuda.synchronize(1)
    cur = torch.cuda.current_device()
    assert L.dt_select_sample_noalloc(0, None, 100, 8, ctypes.c_uint64(1), ctypes.c_void_p(out.data_ptr())) == -1
    assert torch.cuda.current_device() == cur
    assert torch.all(out.cpu() == -1)
